"""Pins of the CPU oracle against facts that do not come from the oracle itself:
closed forms, strong duality, brute-force enumeration, an independent LP solver
(SciPy's HiGHS, when importable) and invariants of the method."""
import json
import os

import numpy as np
import pytest

from oracle.brute import milp_by_enumeration
from oracle.lp import LP, kkt, max_violation
from oracle.merit import merit_order
from oracle.pdhg import PDLPOptions, pdhg_solve
from oracle.scaling import rescale
from oracle.simplex import simplex_solve
from paper_2512_06715_gb300.instances import build_instance
from tests.conftest import instance_lp

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _highs(lp: LP):
    opt = pytest.importorskip("scipy.optimize")
    K = lp.K
    bounds = [(None if not np.isfinite(a) else a, None if not np.isfinite(b) else b)
              for a, b in zip(lp.l, lp.u)]
    r = opt.linprog(lp.c, A_ub=-K[lp.m_eq:], b_ub=-lp.q[lp.m_eq:], A_eq=K[: lp.m_eq],
                    b_eq=lp.q[: lp.m_eq], bounds=bounds, method="highs")
    assert r.status == 0
    return r


# --------------------------------------------------------------------------- closed form
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_merit_order_single_bus(seed):
    """One bus, one period: the relaxation is a continuous knapsack solved by
    merit order on c_g + NL_g / Pmax_g; the balance dual is the marginal price."""
    inst = build_instance(1, 0, 6, 1, seed=seed)
    lp = instance_lp(inst)
    d = float(inst.load.sum())
    obj, p, u, price = merit_order(d, inst.gen_pmax, inst.gen_cost, inst.gen_noload, inst.dt_hours)
    sx = simplex_solve(lp)
    assert sx.status == "optimal"
    assert abs(sx.obj - obj) <= 1e-9 * abs(obj)
    bal = int(inst.row_balance[0, 0])
    assert abs(sx.y[bal] - price) <= 1e-9 * price
    res = pdhg_solve(lp, tol=1e-9, max_attempts=200_000)
    assert res.status == "optimal"
    assert abs(res.primal_obj - obj) <= 1e-7 * abs(obj)
    assert abs(res.y[bal] - price) <= 1e-5 * price
    assert np.allclose(res.x[inst.idx_p[0]], p, atol=1e-5 * inst.gen_pmax.max())


# --------------------------------------------------------------------------- duality, KKT
def test_simplex_strong_duality_and_kkt():
    inst = build_instance(3, 3, 3, 2, seed=0)
    lp = instance_lp(inst)
    sx = simplex_solve(lp)
    assert sx.status == "optimal"
    r = kkt(lp, sx.x, sx.y)
    # exact vertex + exact duals: every optimality measure at round-off level
    assert r.rel_p < 1e-12 and r.rel_d < 1e-12 and r.rel_gap < 1e-12
    assert abs(r.primal_obj - r.dual_obj) <= 1e-9 * abs(r.primal_obj)
    assert np.all(sx.y[lp.m_eq:] >= -1e-9)
    # complementary slackness: inactive >= rows carry no dual
    slack = lp.K @ sx.x - lp.q
    inactive = np.where(slack[lp.m_eq:] > 1e-7)[0] + lp.m_eq
    assert np.all(np.abs(sx.y[inactive]) <= 1e-9)


def test_kkt_residual_directions():
    """Moving x by t e_j changes the equality residual by -t K e_j and the primal
    objective by t c_j; moving y changes lambda by -t K^T e_i."""
    inst = build_instance(3, 3, 3, 2, seed=0)
    lp = instance_lp(inst)
    sx = simplex_solve(lp)
    j = int(inst.idx_p[1, 0])
    t = 1e-3
    x2 = sx.x.copy()
    x2[j] += t
    r0, r1 = kkt(lp, sx.x, sx.y), kkt(lp, x2, sx.y)
    col = lp.K[:, j].toarray().ravel()
    eq = slice(0, lp.m_eq)
    assert np.allclose(r1.rp[eq] - r0.rp[eq], -t * col[eq], atol=1e-12)
    assert abs((r1.primal_obj - r0.primal_obj) - t * lp.c[j]) <= 1e-9 * abs(lp.c[j])
    # a dual move on a balance row (equality, free dual) shifts the dual objective by t q_i
    i = int(inst.row_balance[0, 0])
    y2 = sx.y.copy()
    y2[i] += t
    r2 = kkt(lp, sx.x, y2)
    assert r2.rel_d > r0.rel_d or r2.rel_gap > r0.rel_gap


def test_enumeration_bounds_3bus_2periods():
    """LP relaxation <= MILP optimum by enumerating all 2^(3x2) commitments;
    equality when the relaxed commitment is integral."""
    inst = build_instance(3, 3, 3, 2, seed=0)
    lp = instance_lp(inst)
    sx = simplex_solve(lp)
    best, sched = milp_by_enumeration(lp, inst.idx_u)
    assert np.isfinite(best)
    assert sx.obj <= best + 1e-7 * abs(best)
    u = sx.x[inst.idx_u.reshape(-1)]
    if np.all(np.minimum(np.abs(u), np.abs(u - 1)) < 1e-9):
        assert abs(sx.obj - best) <= 1e-7 * abs(best)
    with open(os.path.join(GOLDEN, "uc3bus_2periods.json")) as f:
        g = json.load(f)
    assert abs(sx.obj - g["lp_optimum"]) <= 1e-9 * abs(g["lp_optimum"])
    assert abs(best - g["milp_optimum"]) <= 1e-9 * abs(g["milp_optimum"])


def test_simplex_matches_highs():
    inst = build_instance(5, 6, 6, 4, seed=2)
    lp = instance_lp(inst)
    sx = simplex_solve(lp)
    r = _highs(lp)
    assert abs(sx.obj - r.fun) <= 1e-8 * abs(r.fun)


# --------------------------------------------------------------------------- scaling
def test_scaling_preserves_the_lp():
    """The rescaled LP has the same optimum, mapped by x = Dc x~, y = Dr y~."""
    inst = build_instance(3, 3, 3, 2, seed=1)
    lp = instance_lp(inst)
    slp, Dr, Dc = rescale(lp)
    a, b = simplex_solve(lp), simplex_solve(slp)
    assert abs(a.obj - b.obj) <= 1e-9 * abs(a.obj)
    assert max_violation(lp, Dc * b.x) <= 1e-7
    r = kkt(lp, Dc * b.x, Dr * b.y)
    assert r.rel_kkt < 1e-10


def test_ruiz_equilibrates():
    """After 10 Ruiz passes every row and column max of |K~| is close to 1."""
    inst = build_instance(24, 38, 33, 24, seed=0)
    lp = instance_lp(inst)
    slp, Dr, Dc = rescale(lp, ruiz_iters=10, pock_chambolle=False)
    A = abs(slp.K)
    rmax = A.max(axis=1).toarray().ravel()
    cmax = A.max(axis=0).toarray().ravel()
    nzr, nzc = rmax > 0, cmax > 0
    assert np.all(np.abs(rmax[nzr] - 1) < 1e-2)
    assert np.all(np.abs(cmax[nzc] - 1) < 1e-2)
    assert np.allclose(slp.K.toarray(), (Dr[:, None] * lp.K.toarray()) * Dc[None, :], rtol=1e-12)


# --------------------------------------------------------------------------- PDHG
def test_pdhg_fixed_point_is_the_optimum():
    """Saddle points are fixed points of the PDHG map for every step size and
    primal weight; a non-optimal start moves."""
    inst = build_instance(3, 3, 3, 2, seed=0)
    lp = instance_lp(inst)
    sx = simplex_solve(lp)
    for eta, omega in [(0.3, 1.0), (0.05, 40.0), (1.0, 0.01)]:
        res = pdhg_solve(lp, fixed=dict(eta=eta, omega=omega), stop_after=5, start=(sx.x, sx.y))
        assert np.allclose(res.x, sx.x, rtol=1e-9, atol=1e-9 * np.abs(sx.x).max())
        assert np.allclose(res.y, sx.y, rtol=1e-9, atol=1e-9 * np.abs(sx.y).max())
    y_off = sx.y.copy()
    y_off[inst.row_balance[0, 0]] += 1.0
    res = pdhg_solve(lp, fixed=dict(eta=0.3, omega=1.0), stop_after=1, start=(sx.x, y_off))
    assert np.abs(res.x - sx.x).max() > 1e-6 * np.abs(sx.x).max()


def test_pdhg_matches_simplex_small():
    inst = build_instance(3, 3, 3, 2, seed=0)
    lp = instance_lp(inst)
    sx = simplex_solve(lp)
    res = pdhg_solve(lp, tol=1e-10, max_attempts=500_000, record=True)
    assert res.status == "optimal"
    assert abs(res.primal_obj - sx.obj) <= 1e-8 * abs(sx.obj)
    # every accepted attempt satisfied the step-size condition eta <= eta_max
    for eta, omega, acc, eta_max, eta_next, own in res.attempt_log:
        if acc:
            assert eta <= eta_max


def test_pdhg_matches_highs_medium():
    inst = build_instance(8, 10, 6, 6, seed=5)
    lp = instance_lp(inst)
    r = _highs(lp)
    res = pdhg_solve(lp, tol=1e-8, max_attempts=1_000_000)
    assert res.status == "optimal"
    assert abs(res.primal_obj - r.fun) <= 1e-6 * abs(r.fun)
    assert max_violation(lp, res.x) <= 1e-6 * max(1.0, np.abs(lp.q).max())


def test_pdhg_replay_reproduces_run():
    """Replaying a run's own schedule reproduces it exactly (the replay path is
    what the GPU parity test uses)."""
    inst = build_instance(3, 3, 3, 2, seed=0)
    lp = instance_lp(inst)
    a = pdhg_solve(lp, tol=1e-30, stop_after=192, record=True)
    sched = dict(attempts=[(e[0], e[2]) for e in a.attempt_log],
                 checks=[(c["restart"], c["to_avg"]) for c in a.check_log])
    b = pdhg_solve(lp, tol=1e-30, stop_after=192, schedule=sched)
    assert np.array_equal(a.x_scaled, b.x_scaled) and np.array_equal(a.y_scaled, b.y_scaled)
