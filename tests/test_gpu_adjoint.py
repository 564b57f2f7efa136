"""Adjoint (pdhg_backward) and the autograd wrapper against the oracle.

Instances are made nondegenerate by relaxing every >= row by a seeded
U(0.5, 1) * 1e-5 * (1 + |q_i|), every finite bound of a non-fixed variable
outward by U(0.5, 1) * 1e-6 * (1 + |bound|) (commitment logic rows are
equalities, so relaxing rows alone leaves units that stay on or off
degenerate), and jittering each cost by (1 + 1e-6 U(-1, 1)); the optimal
vertex then has exactly n active constraints and both the simplex vertex and
its derivatives are unique.  Finite
differences use the oracle's dense simplex (exact vertices), central, along
seeded random directions of the load."""
import numpy as np
import pytest

from oracle.lp import LP, kkt
from oracle.simplex import simplex_solve
from paper_2512_06715_gb300.instances import build_instance

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_06715_gb300 import build
    build.build()


def _perturbed(inst, seed):
    rng = np.random.default_rng(seed)
    q = inst.q.copy()
    ineq = np.arange(inst.m) >= inst.m_eq
    q[ineq] -= rng.uniform(0.5, 1.0, ineq.sum()) * 1e-5 * (1.0 + np.abs(q[ineq]))
    c = inst.c * (1.0 + 1e-6 * rng.uniform(-1.0, 1.0, inst.n))
    l, u = inst.l.copy(), inst.u.copy()
    free_to_move = l < u
    lf = free_to_move & np.isfinite(l)
    uf = free_to_move & np.isfinite(u)
    l[lf] -= rng.uniform(0.5, 1.0, lf.sum()) * 1e-6 * (1.0 + np.abs(l[lf]))
    u[uf] += rng.uniform(0.5, 1.0, uf.sum()) * 1e-6 * (1.0 + np.abs(u[uf]))
    inst.l_pert, inst.u_pert = l, u
    return q, c


def _lp(inst, q, c):
    return LP(K=inst.scipy_csr(), q=q, c=c, l=inst.l_pert, u=inst.u_pert, m_eq=inst.m_eq)


def _active_count(lp, x, y):
    s = lp.K @ x - lp.q
    act_rows = lp.m_eq + int(np.sum((s[lp.m_eq:] < 1e-9 * (1 + np.abs(lp.q[lp.m_eq:])))))
    at_bound = np.sum((np.abs(x - lp.l) < 1e-9) | (np.abs(x - lp.u) < 1e-9))
    return act_rows + int(at_bound)


def _nondegenerate_instance():
    inst = build_instance(4, 4, 4, 3, seed=1)
    for seed in range(20):
        q, c = _perturbed(inst, seed)
        sx = simplex_solve(_lp(inst, q, c))
        if sx.status == "optimal" and _active_count(_lp(inst, q, c), sx.x, sx.y) == inst.n:
            return inst, q, c, sx
    pytest.skip("no nondegenerate perturbation found")


def _ws(inst, q, c):
    from paper_2512_06715_gb300.pdhg import Workspace, default_opts
    return Workspace(inst.row_ptr, inst.col, inst.val, c, inst.l_pert, inst.u_pert, q, inst.m_eq,
                     default_opts(precision="fp64", tol=1e-11, time_limit_s=120.0))


def test_cost_gradient_is_the_dual_and_the_primal():
    inst, q, c, sx = _nondegenerate_instance()
    ws = _ws(inst, q, c)
    x, y, r = ws.solve()
    assert r["status_name"] == "optimal"
    gq = torch.empty(inst.m, dtype=torch.float64, device="cuda")
    gc = torch.empty(inst.n, dtype=torch.float64, device="cuda")
    from paper_2512_06715_gb300 import pdhg
    rc = pdhg.lib().pdhg_backward(ws.ws, 1.0, None, gq.data_ptr(), gc.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream)
    assert rc == 0, pdhg.lib().pdhg_last_error()
    gq, gc = gq.cpu().numpy(), gc.cpu().numpy()
    bal = inst.row_balance.reshape(-1)
    scale = np.abs(sx.y[bal]).max()
    assert np.allclose(gq[bal], sx.y[bal], atol=1e-6 * scale, rtol=0)
    assert np.allclose(gc, sx.x, atol=1e-6 * np.abs(sx.x).max(), rtol=0)
    ws.close()


def test_dispatch_gradient_matches_finite_differences():
    """d(g_p^T p*)/d d along 8 seeded load directions: adjoint vs central finite
    differences of exact simplex vertices (h = 1e-6 relative)."""
    inst, q, c, sx = _nondegenerate_instance()
    ws = _ws(inst, q, c)
    x, y, r = ws.solve()
    assert r["status_name"] == "optimal"
    rng = np.random.default_rng(7)
    gx = np.zeros(inst.n)
    gx[inst.idx_p.reshape(-1)] = rng.standard_normal(inst.idx_p.size)
    gq = torch.empty(inst.m, dtype=torch.float64, device="cuda")
    gc = torch.empty(inst.n, dtype=torch.float64, device="cuda")
    gxt = torch.as_tensor(gx, device="cuda")
    from paper_2512_06715_gb300 import pdhg
    rc = pdhg.lib().pdhg_backward(ws.ws, 0.0, gxt.data_ptr(), gq.data_ptr(), gc.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream)
    assert rc == 0, pdhg.lib().pdhg_last_error()
    gq = gq.cpu().numpy()
    bal = inst.row_balance.reshape(-1)
    dmax = np.abs(q[bal]).max()
    h = 1e-6 * dmax
    for k in range(8):
        delta = rng.standard_normal(bal.size)
        delta /= np.abs(delta).max()
        qp, qm = q.copy(), q.copy()
        qp[bal] += h * delta
        qm[bal] -= h * delta
        fp = simplex_solve(_lp(inst, qp, c))
        fm = simplex_solve(_lp(inst, qm, c))
        fd = (gx @ fp.x - gx @ fm.x) / (2 * h)
        ad = gq[bal] @ delta
        assert abs(fd - ad) <= 1e-5 * max(abs(fd), 1e-12) + 1e-9, (k, fd, ad)
    ws.close()


def test_autograd_function():
    """UCRelax: torch.autograd through pdhg_solve / pdhg_backward."""
    from paper_2512_06715_gb300.autograd import UCRelax
    inst, q, c, sx = _nondegenerate_instance()
    relax = UCRelax(inst, q=q, c=c, l=inst.l_pert, u=inst.u_pert, tol=1e-11)
    bal = inst.row_balance
    d = torch.tensor(q[bal], dtype=torch.float64, device="cuda", requires_grad=True)
    ct = torch.tensor(c, dtype=torch.float64, device="cuda", requires_grad=True)
    cost, p = relax(d, ct)
    assert abs(cost.item() - sx.obj) <= 1e-8 * abs(sx.obj)
    (cost + 0.0 * p.sum()).backward()
    assert np.allclose(d.grad.cpu().numpy(), sx.y[bal], atol=1e-6 * np.abs(sx.y[bal]).max())
    assert np.allclose(ct.grad.cpu().numpy(), sx.x, atol=1e-6 * np.abs(sx.x).max())
    # backward differentiates the workspace's last solve, so a graph whose
    # workspace was solved again after its forward is refused
    cost1, _ = relax(d, ct)
    cost2, _ = relax(d, ct)
    with pytest.raises(RuntimeError, match="solved again"):
        cost1.backward()
    cost2.backward()
    relax.close()
