"""Infeasibility detection on the GPU (single and batched solves) against the
oracle: the same certificates from iterate differences (Applegate et al.'s
detection behind the PDLP method cited in Sec. II.E), and the classification
of branch-and-bound node LPs without slacks that the dense simplex's phase 1
gives."""
import numpy as np
import pytest

from oracle.pdhg import pdhg_solve
from oracle.simplex import simplex_solve
from paper_2512_06715_gb300.instances import build_instance, workload
from tests.conftest import instance_lp
from tests.test_oracle_infeasibility import _box_lp, _free_lp, _unbounded_lp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_06715_gb300 import build
    build.build()


def _ws_lp(lp, **kw):
    from paper_2512_06715_gb300.pdhg import Workspace, default_opts
    K = lp.K.tocsr()
    kw.setdefault("time_limit_s", 120.0)
    return Workspace(K.indptr.astype(np.int64), K.indices.astype(np.int32), K.data, lp.c, lp.l, lp.u, lp.q,
                     lp.m_eq, default_opts(**kw))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("make,status", [(_box_lp, "primal_infeasible"), (_free_lp, "primal_infeasible"),
                                         (_unbounded_lp, "dual_infeasible")])
def test_hand_lps(make, status, precision):
    lp = make()
    ref = pdhg_solve(lp, tol=1e-8, max_attempts=200_000)
    assert ref.status == status
    ws = _ws_lp(lp, precision=precision, tol=1e-8)
    _, _, r = ws.solve()
    assert r["status_name"] == status, r
    ws.close()


def _node_bounds(inst, period_off):
    """Bounds of a node LP without slacks that switches every unit off in the
    given period (None: one unit forced on in the last period, feasible)."""
    l, u = inst.l.copy(), inst.u.copy()
    if period_off is None:
        l[inst.idx_u[-1, 0]] = 1.0
    else:
        u[inst.idx_u[period_off]] = 0.0
    return l, u


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_uc_nodes_single(precision):
    """A 3-bus, 2-period node with every unit off in period 1 is infeasible
    (simplex phase 1) and the GPU returns a primal-infeasibility certificate,
    as the oracle does; the 24-bus relaxation with every unit off in period 6
    likewise; a feasible node is solved to optimality, not misclassified."""
    from paper_2512_06715_gb300.pdhg import Workspace, default_opts
    for inst, period in ((build_instance(3, 3, 3, 2, seed=0), 0), (workload("uc24_g33_T24"), 5)):
        lp = instance_lp(inst)
        l, u = _node_bounds(inst, period)
        lp.l, lp.u = l, u
        if inst.n < 100:
            assert simplex_solve(lp).status == "infeasible"
        assert pdhg_solve(lp, tol=1e-8, max_attempts=2_000_000).status == "primal_infeasible"
        ws = Workspace(inst.row_ptr, inst.col, inst.val, inst.c, l, u, inst.q, inst.m_eq,
                       default_opts(precision=precision, tol=1e-8, time_limit_s=120.0))
        _, _, r = ws.solve()
        assert r["status_name"] == "primal_infeasible", r
        ws.close()
    inst = build_instance(3, 3, 3, 2, seed=0)
    l, u = _node_bounds(inst, None)
    lp = instance_lp(inst)
    lp.l, lp.u = l, u
    sx = simplex_solve(lp)
    assert sx.status == "optimal"
    ws = Workspace(inst.row_ptr, inst.col, inst.val, inst.c, l, u, inst.q, inst.m_eq,
                   default_opts(precision=precision, tol=1e-8, time_limit_s=120.0))
    _, _, r = ws.solve()
    assert r["status_name"] == "optimal"
    assert abs(r["primal_obj"] - sx.obj) <= 1e-6 * abs(sx.obj)
    ws.close()


def test_batched_nodes_classified_like_the_simplex():
    """Eight node LPs of one 3-bus, 2-period instance without slacks, batched:
    the nodes switching every unit off in a period are infeasible, the others
    feasible; the batched statuses equal the simplex's classification, and the
    feasible nodes' objectives equal the simplex optima."""
    from paper_2512_06715_gb300.pdhg import Workspace, default_opts
    inst = build_instance(3, 3, 3, 2, seed=1)
    bounds = [_node_bounds(inst, [None, 0, None, 1][k % 4]) for k in range(8)]
    l_b = np.stack([b[0] for b in bounds])
    u_b = np.stack([b[1] for b in bounds])
    expect = []
    for l, u in bounds:
        lp = instance_lp(inst)
        lp.l, lp.u = l, u
        sx = simplex_solve(lp)
        expect.append(sx)
    ws = Workspace.from_instance(inst, default_opts(precision="mixed", tol=1e-8, time_limit_s=120.0))
    _, _, rb = ws.solve_batched(l_b, u_b)
    for k, (sx, r) in enumerate(zip(expect, rb)):
        if sx.status == "infeasible":
            assert r["status_name"] == "primal_infeasible", (k, r)
        else:
            assert sx.status == "optimal"
            assert r["status_name"] == "optimal", (k, r)
            assert abs(r["primal_obj"] - sx.obj) <= 1e-6 * abs(sx.obj)
    assert {s.status for s in expect} == {"infeasible", "optimal"}
    ws.close()
