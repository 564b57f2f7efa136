"""Batched node LPs (pdhg_solve_batched) against single-instance solves and the oracle."""
import numpy as np
import pytest

from oracle.lp import kkt, lp_from_arrays, max_violation
from paper_2512_06715_gb300.instances import build_instance, node_fixings

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_06715_gb300 import build
    build.build()


def _node_lp(inst, l, u):
    return lp_from_arrays(inst.row_ptr, inst.col, inst.val, inst.q, inst.c, l, u, inst.m_eq)


@pytest.mark.parametrize("B,tol", [(1, 1e-8), (8, 1e-8), (33, 1e-8), (64, 1e-8)])
def test_batched_matches_single_solves(B, tol):
    """Every node of the batch reaches rel-KKT <= 1.5 tol as the oracle
    recomputes it from the returned point, with violation <= 100 tol; up to 8
    nodes spread over the batch agree with the same node solved alone (objective
    within 100 tol relative).  B = 33 runs the 64-slot layout with 31 idle slots,
    B = 64 a full batch."""
    from paper_2512_06715_gb300.pdhg import Workspace, default_opts
    inst = build_instance(12, 18, 10, 12, seed=3, with_slack=True)
    l_b, u_b = node_fixings(inst, B)
    ws = Workspace.from_instance(inst, default_opts(precision="mixed", tol=tol, time_limit_s=300.0))
    xb, yb, rb = ws.solve_batched(l_b, u_b)
    xb, yb = xb.cpu().numpy(), yb.cpu().numpy()
    tb = ws.tuning()["batched"]  # the batched autotuner ran and chose a shape
    assert tb["rows_per_warp_dual"] in (1, 2, 4) and tb["rows_per_warp_adj"] in (1, 2, 4)
    assert tb["grid_dual"] > 0 and tb["grid_adj"] > 0
    alone = set(np.linspace(0, B - 1, min(B, 8)).round().astype(int).tolist())
    for k in range(B):
        assert rb[k]["status_name"] == "optimal", (k, rb[k])
        lp = _node_lp(inst, l_b[k], u_b[k])
        c = kkt(lp, xb[k], yb[k])
        assert c.rel_kkt <= 1.5 * tol, (k, c.rel_kkt, rb[k]["rel_kkt"])
        assert max_violation(lp, xb[k]) <= 100 * tol * max(1.0, np.abs(lp.q).max())
        if k not in alone:
            continue
        # the same node solved alone
        single = Workspace(inst.row_ptr, inst.col, inst.val, inst.c, l_b[k], u_b[k], inst.q, inst.m_eq,
                           default_opts(precision="mixed", tol=tol, time_limit_s=120.0))
        xs, ys, rs = single.solve()
        assert rs["status_name"] == "optimal"
        ps = kkt(lp, xs.cpu().numpy(), ys.cpu().numpy()).primal_obj
        assert abs(c.primal_obj - ps) <= 100 * tol * abs(ps), (k, c.primal_obj, ps)
        single.close()
    ws.close()


def test_batched_nodes_bound_the_root():
    """Fixing commitments only tightens the relaxation: every node's optimum is
    at least the root LP optimum (all solved to rel-KKT 1e-8, whose gap term
    bounds each objective's relative error by ~1e-8, hence the 1e-7 slack)."""
    from paper_2512_06715_gb300.pdhg import Workspace, default_opts
    inst = build_instance(12, 18, 10, 12, seed=4, with_slack=True)
    l_b, u_b = node_fixings(inst, 16, seed0=2000)
    ws = Workspace.from_instance(inst, default_opts(precision="mixed", tol=1e-8, time_limit_s=300.0))
    _, _, root = ws.solve()
    xb, yb, rb = ws.solve_batched(l_b, u_b)
    assert all(r["status_name"] == "optimal" for r in rb), [r["status_name"] for r in rb]
    for r in rb:
        assert r["primal_obj"] >= root["primal_obj"] * (1 - 1e-7)
    ws.close()


@pytest.mark.parametrize("rw,grid", [(1, 3), (2, 7), (4, 1)])
def test_batched_fixed_shape(rw, grid):
    """With the autotuner off, kernel_variant 1/2/4 and kernel_grid fix the
    batched sweeps' rows (columns) per warp and blocks; tiny grids make each
    warp sweep many row groups and the ragged tail.  Every node still reaches
    rel-KKT 1e-8 as the oracle recomputes it."""
    from paper_2512_06715_gb300.pdhg import Workspace, default_opts
    inst = build_instance(12, 18, 10, 12, seed=3, with_slack=True)
    B = 8
    l_b, u_b = node_fixings(inst, B)
    ws = Workspace.from_instance(inst, default_opts(precision="mixed", tol=1e-8, time_limit_s=300.0, autotune=0,
                                                    kernel_variant=rw, kernel_grid=grid))
    xb, yb, rb = ws.solve_batched(l_b, u_b)
    tb = ws.tuning()["batched"]
    assert (tb["rows_per_warp_dual"], tb["grid_dual"], tb["rows_per_warp_adj"], tb["grid_adj"]) == (rw, grid, rw, grid)
    xb, yb = xb.cpu().numpy(), yb.cpu().numpy()
    for k in range(B):
        assert rb[k]["status_name"] == "optimal", (k, rb[k])
        assert kkt(_node_lp(inst, l_b[k], u_b[k]), xb[k], yb[k]).rel_kkt <= 1.5e-8
    ws.close()
