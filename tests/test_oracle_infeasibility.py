"""Pins of the oracle's infeasibility detection (certificates from PDHG iterate
differences, the method of Applegate et al. behind the PDLP solver the paper
cites in Sec. II.E): hand-worked rays on tiny LPs, and agreement with the
dense simplex's phase 1 on branch-and-bound node LPs of a tiny UC instance."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.lp import LP, ray_check
from oracle.pdhg import PDLPOptions, pdhg_solve
from oracle.simplex import simplex_solve
from paper_2512_06715_gb300.instances import build_instance
from tests.conftest import instance_lp


def _box_lp():
    """x1 + x2 = 5 with 0 <= x <= 1: infeasible, since x1 + x2 <= 2."""
    return LP(K=sp.csr_matrix(np.array([[1.0, 1.0]])), q=np.array([5.0]), c=np.array([1.0, 2.0]),
              l=np.zeros(2), u=np.ones(2), m_eq=1)


def _free_lp():
    """x1 = 1 and x1 = 2 with x1 free (and x2 in [0, 1] unused by the rows)."""
    return LP(K=sp.csr_matrix(np.array([[1.0, 0.0], [1.0, 0.0]])), q=np.array([1.0, 2.0]),
              c=np.array([0.0, 1.0]), l=np.array([-np.inf, 0.0]), u=np.array([np.inf, 1.0]), m_eq=2)


def _unbounded_lp():
    """min -x1  s.t.  x1 - x2 >= 0,  x >= 0 (no upper bounds): unbounded below."""
    return LP(K=sp.csr_matrix(np.array([[1.0, -1.0]])), q=np.array([0.0]), c=np.array([-1.0, 0.0]),
              l=np.zeros(2), u=np.full(2, np.inf), m_eq=0)


def test_dual_ray_by_hand():
    """Box LP, y = 1: lambda = -K^T y = (-1, -1), both upper bounds finite, so no
    violation; objective q y - u^T lambda^- = 5 - 2 = 3 > 0: a Farkas certificate.
    y = -1: lambda = (1, 1) absorbed by the finite lower bounds 0, objective -5."""
    lp = _box_lp()
    r = ray_check(lp, np.zeros(2), np.array([1.0]))
    assert r.dual_ray_obj == 3.0 and r.dual_ray_viol == 0.0
    assert r.primal_infeasible(1e-8)
    r = ray_check(lp, np.zeros(2), np.array([-1.0]))
    assert r.dual_ray_obj == -5.0 and not r.primal_infeasible(1e-8)


def test_dual_ray_with_free_variable_by_hand():
    """x1 free forces lambda_1 = -(y1 + y2) = 0: y = (-1, 1) gives objective
    -1 + 2 = 1 with no violation; y = (1, 0) violates lambda_1 = -1 < 0 (no
    upper bound to absorb it) by 1 against an objective of 1."""
    lp = _free_lp()
    r = ray_check(lp, np.zeros(2), np.array([-1.0, 1.0]))
    assert r.dual_ray_obj == 1.0 and r.dual_ray_viol == 0.0 and r.primal_infeasible(1e-8)
    r = ray_check(lp, np.zeros(2), np.array([1.0, 0.0]))
    assert r.dual_ray_obj == 1.0 and r.dual_ray_viol == 1.0 and not r.primal_infeasible(1e-8)


def test_primal_ray_by_hand():
    """Unbounded LP: x = (1, 1) keeps K x = 0 >= 0 and x >= 0, cost -1 < 0;
    x = (0, 1) violates the row by 1 (K x = -1) and costs 0."""
    lp = _unbounded_lp()
    r = ray_check(lp, np.array([1.0, 1.0]), np.zeros(1))
    assert r.primal_ray_obj == -1.0 and r.primal_ray_viol == 0.0 and r.dual_infeasible(1e-8)
    r = ray_check(lp, np.array([0.0, 1.0]), np.zeros(1))
    assert r.primal_ray_obj == 0.0 and r.primal_ray_viol == 1.0 and not r.dual_infeasible(1e-8)
    # a bound that forbids the direction: x1 <= 1 turns (1, 1) into a violation of 1 per component
    lp.u = np.ones(2)
    r = ray_check(lp, np.array([1.0, 1.0]), np.zeros(1))
    assert r.primal_ray_viol == pytest.approx(np.sqrt(2.0)) and not r.dual_infeasible(1e-8)


@pytest.mark.parametrize("make,status", [(_box_lp, "primal_infeasible"), (_free_lp, "primal_infeasible"),
                                         (_unbounded_lp, "dual_infeasible")])
def test_pdhg_detects_by_hand_lps(make, status):
    lp = make()
    assert simplex_solve(lp).status == ("infeasible" if status == "primal_infeasible" else "unbounded")
    res = pdhg_solve(lp, tol=1e-8, max_attempts=200_000, opts=PDLPOptions(**dict(ruiz_iters=0)))
    assert res.status == status, (res.status, res.attempts)


def _uc_node(fix_period0_off: bool, seed=0):
    inst = build_instance(3, 3, 3, 2, seed=seed)
    lp = instance_lp(inst)
    l, u = lp.l.copy(), lp.u.copy()
    if fix_period0_off:
        j = inst.idx_u[0]           # every unit off in period 1: no supply against a positive load
    else:
        j = inst.idx_u[1, :1]       # one unit on in period 2
        l[j] = 1.0
    u[j] = np.where(fix_period0_off, 0.0, u[j])
    lp.l, lp.u = l, u
    return lp


@pytest.mark.parametrize("seed", [0, 1])
def test_uc_node_classification_matches_simplex(seed):
    """Node LPs without shed/spill slack: switching every unit off in a period
    with load is infeasible (phase 1 of the simplex), and PDHG returns a
    primal-infeasibility certificate; a node fixing one unit on stays feasible
    and PDHG reaches the simplex optimum without a false certificate."""
    bad = _uc_node(True, seed)
    assert simplex_solve(bad).status == "infeasible"
    res = pdhg_solve(bad, tol=1e-8, max_attempts=500_000)
    assert res.status == "primal_infeasible", (res.status, res.attempts)
    good = _uc_node(False, seed)
    sx = simplex_solve(good)
    assert sx.status == "optimal"
    res = pdhg_solve(good, tol=1e-9, max_attempts=500_000)
    assert res.status == "optimal"
    assert abs(res.primal_obj - sx.obj) <= 1e-7 * abs(sx.obj)
