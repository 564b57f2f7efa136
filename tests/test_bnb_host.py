"""Host logic of the branch-and-bound driver on the CPU: the node LPs of a
stand-in workspace are solved by the oracle's dense simplex (phase 1 reports
infeasible nodes as the GPU's certificates would), and the driver must reach
the MILP optimum found by enumerating every commitment schedule."""
import numpy as np
import pytest

from oracle.brute import milp_by_enumeration
from oracle.lp import LP
from oracle.simplex import simplex_solve
from paper_2512_06715_gb300.bnb import branch_and_bound
from paper_2512_06715_gb300.instances import build_instance
from tests.conftest import instance_lp

torch = pytest.importorskip("torch")


class SimplexNodes:
    """solve_batched with the shape of pdhg.Workspace's, on the CPU."""

    def __init__(self, lp):
        self.lp = lp
        self.device = torch.device("cpu")
        self.calls = 0

    def solve_batched(self, l_b, u_b, want_y=True):
        self.calls += 1
        xs, res = [], []
        for l, u in zip(l_b.numpy(), u_b.numpy()):
            sx = simplex_solve(LP(K=self.lp.K, q=self.lp.q, c=self.lp.c, l=l, u=u, m_eq=self.lp.m_eq))
            if sx.status == "optimal":
                xs.append(sx.x)
                res.append({"status_name": "optimal", "primal_obj": sx.obj, "dual_obj": sx.obj, "rel_kkt": 0.0})
            else:
                xs.append(np.zeros(self.lp.n))
                res.append({"status_name": "primal_infeasible", "primal_obj": np.nan, "dual_obj": np.nan,
                            "rel_kkt": np.nan})
        return torch.as_tensor(np.stack(xs)), None, res


@pytest.mark.parametrize("shape,seed", [((3, 3, 3, 2), 0), ((3, 3, 3, 2), 1), ((4, 4, 3, 3), 2)])
def test_bnb_logic_reaches_the_enumerated_optimum(shape, seed):
    inst = build_instance(*shape, seed=seed)
    lp = instance_lp(inst)
    best, _ = milp_by_enumeration(lp, inst.idx_u)
    ws = SimplexNodes(lp)
    res = branch_and_bound(ws, inst.idx_u, inst.l, inst.u, gap=1e-9)
    assert res.status == "optimal"
    assert abs(res.incumbent - best) <= 1e-9 * abs(best)
    assert res.bound <= res.incumbent
    assert res.nodes < 2 ** inst.idx_u.size  # the tree prunes


def test_bnb_small_batches_and_node_limit():
    """Batches of 2 nodes give the same optimum; a node limit of 1 stops at the
    root with a valid bound below the optimum."""
    inst = build_instance(4, 4, 3, 3, seed=2)
    lp = instance_lp(inst)
    best, _ = milp_by_enumeration(lp, inst.idx_u)
    res = branch_and_bound(SimplexNodes(lp), inst.idx_u, inst.l, inst.u, batch=2, gap=1e-9)
    assert res.status == "optimal" and abs(res.incumbent - best) <= 1e-9 * abs(best)
    res = branch_and_bound(SimplexNodes(lp), inst.idx_u, inst.l, inst.u, max_nodes=1, gap=1e-9)
    assert res.nodes == 1 and res.bound <= best + 1e-9 * abs(best)


class FlakyNodes(SimplexNodes):
    """Batched solves that leave every third node at the attempt limit (as FP32
    rays of some infeasible nodes do); the single FP64 solve on the workspace's
    own bounds resolves it, or not when `fp64_ok` is false."""

    def __init__(self, lp, fp64_ok=True):
        super().__init__(lp)
        self.fp64_ok = fp64_ok
        self.t = {"l": torch.as_tensor(lp.l.copy()), "u": torch.as_tensor(lp.u.copy())}
        self.opts = type("Opts", (), {"precision": 1, "max_iters": 100})()
        self.single = 0

    def set_opts(self, **kw):
        for k, v in kw.items():
            setattr(self.opts, k, v)

    def solve_batched(self, l_b, u_b, want_y=True):
        x, y, res = super().solve_batched(l_b, u_b, want_y)
        for k in range(0, len(res), 3):
            res[k] = {"status_name": "iteration_limit", "primal_obj": np.nan, "dual_obj": np.nan, "rel_kkt": 1e-3}
        return x, y, res

    def solve(self):
        self.single += 1
        assert self.opts.precision == "fp64"
        l, u = self.t["l"].numpy(), self.t["u"].numpy()
        if not self.fp64_ok:
            return torch.zeros(self.lp.n), None, {"status_name": "time_limit", "rel_kkt": 1e-3}
        sx = simplex_solve(LP(K=self.lp.K, q=self.lp.q, c=self.lp.c, l=l, u=u, m_eq=self.lp.m_eq))
        if sx.status != "optimal":
            return torch.zeros(self.lp.n), None, {"status_name": "primal_infeasible", "rel_kkt": np.nan}
        return torch.as_tensor(sx.x), None, {"status_name": "optimal", "primal_obj": sx.obj, "dual_obj": sx.obj,
                                             "rel_kkt": 0.0}


def test_bnb_retries_unresolved_nodes_in_fp64():
    """Nodes a batched call leaves unresolved are solved again alone in FP64 on
    the workspace's bounds, which are restored afterwards; the optimum is the
    enumerated one.  A node the FP64 solve leaves unresolved too raises."""
    inst = build_instance(4, 4, 3, 3, seed=2)
    lp = instance_lp(inst)
    best, _ = milp_by_enumeration(lp, inst.idx_u)
    ws = FlakyNodes(lp)
    res = branch_and_bound(ws, inst.idx_u, inst.l, inst.u, gap=1e-9)
    assert res.status == "optimal" and abs(res.incumbent - best) <= 1e-9 * abs(best)
    assert ws.single > 0 and res.log[-1]["fp64_retries"] == ws.single
    assert np.array_equal(ws.t["l"].numpy(), lp.l) and np.array_equal(ws.t["u"].numpy(), lp.u)
    assert ws.opts.precision == 1 and ws.opts.max_iters == 100
    with pytest.raises(RuntimeError, match="time_limit"):
        branch_and_bound(FlakyNodes(lp, fp64_ok=False), inst.idx_u, inst.l, inst.u, gap=1e-9)
