"""Active-set polish (pdhg_polish, crossover-lite) and the adjoint
(pdhg_backward) at an intermediate size: the perturbed, nondegenerate 24-bus,
24-period relaxation, checked against SciPy's HiGHS vertices and against the
oracle's polish of the same GPU point."""
import numpy as np
import pytest

from oracle.lp import kkt
from oracle.polish import polish
from paper_2512_06715_gb300.instances import workload
from tests.nondegenerate import highs_vertex, perturbed_lp

torch = pytest.importorskip("torch")
pytest.importorskip("scipy.optimize")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_06715_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def case():
    """Perturbed 24-bus LP, its HiGHS vertex, and a GPU FP64 solve to 1e-11
    (the rows whose dual and slack are both small need that accuracy for the
    active set to be read correctly)."""
    from paper_2512_06715_gb300.pdhg import Workspace, default_opts
    inst = workload("uc24_g33_T24")
    lp = perturbed_lp(inst, 0)
    xh, yh, obj = highs_vertex(lp)
    K = lp.K.tocsr()
    ws = Workspace(K.indptr.astype(np.int64), K.indices.astype(np.int32), K.data, lp.c, lp.l, lp.u, lp.q,
                   lp.m_eq, default_opts(precision="fp64", tol=1e-11, time_limit_s=300.0))
    x, y, r = ws.solve()
    assert r["status_name"] == "optimal", r
    yield inst, lp, ws, x.cpu().numpy(), y.cpu().numpy(), xh, yh, obj
    ws.close()


def test_polish_gives_the_vertex(case):
    inst, lp, ws, x, y, xh, yh, obj = case
    xp, yp, res = ws.polish()
    assert res["status_name"] == "ok", res
    assert res["active_rows"] == res["free_vars"]
    assert max(res["cg_residual_primal"], res["cg_residual_dual"]) <= 1e-9
    xp, yp = xp.cpu().numpy(), yp.cpu().numpy()
    # the HiGHS vertex (the iterative solves stop at relative residual <= 1e-9)
    assert np.abs(xp - xh).max() <= 1e-7 * np.abs(xh).max()
    assert np.abs(yp - yh).max() <= 1e-6 * np.abs(yh).max()
    assert abs(res["primal_obj"] - obj) <= 1e-9 * abs(obj)
    # the library's measures of the polished point equal the oracle's
    chk = kkt(lp, xp, yp)
    assert chk.rel_kkt <= 1e-9 and res["rel_kkt"] <= 1e-9
    assert abs(chk.rel_kkt - res["rel_kkt"]) <= 1e-3 * chk.rel_kkt + 1e-15
    assert res["bound_violation"] <= 1e-7 * np.abs(xh).max()
    assert res["dual_sign_violation"] <= 1e-6 * np.abs(yh).max()
    # the oracle's polish of the same GPU point (same active set, direct solver)
    ref = polish(lp, x, y)
    assert ref is not None
    assert np.abs(xp - ref[0]).max() <= 1e-7 * np.abs(ref[0]).max()
    assert np.abs(yp - ref[1]).max() <= 1e-6 * np.abs(ref[1]).max()


def test_polish_reports_a_degenerate_set():
    """The unperturbed 24-bus relaxation is degenerate: not square, nothing written."""
    from paper_2512_06715_gb300.pdhg import Workspace, default_opts
    inst = workload("uc24_g33_T24")
    ws = Workspace.from_instance(inst, default_opts(precision="fp64", tol=1e-9, time_limit_s=120.0))
    ws.solve()
    x, y, res = ws.polish()
    assert res["status_name"] == "not_square" and x is None
    assert res["active_rows"] != res["free_vars"]
    ws.close()


def test_adjoint_against_highs_duals_and_finite_differences(case):
    """d cost / d load = the balance duals of the HiGHS vertex (1e-6 of the
    largest); d (g_p^T p*) / d load along 16 seeded directions = central finite
    differences of HiGHS vertices, each re-solved on its own active set by the
    oracle's polish, at h = 1e-6 of the largest load (1e-5 relative)."""
    from paper_2512_06715_gb300 import pdhg
    inst, lp, ws, x, y, xh, yh, obj = case
    bal = inst.row_balance.reshape(-1)
    stream = torch.cuda.current_stream().cuda_stream
    gq = torch.empty(inst.m, dtype=torch.float64, device="cuda")
    gc = torch.empty(inst.n, dtype=torch.float64, device="cuda")
    rc = pdhg.lib().pdhg_backward(ws.ws, 1.0, None, gq.data_ptr(), gc.data_ptr(), stream)
    assert rc == 0, pdhg.lib().pdhg_last_error()
    g = gq.cpu().numpy()
    assert np.abs(g[bal] - yh[bal]).max() <= 1e-6 * np.abs(yh[bal]).max()
    assert np.abs(gc.cpu().numpy() - xh).max() <= 1e-6 * np.abs(xh).max()
    rng = np.random.default_rng(11)
    gx = np.zeros(inst.n)
    gx[inst.idx_p.reshape(-1)] = rng.standard_normal(inst.idx_p.size)
    gxt = torch.as_tensor(gx, device="cuda")
    rc = pdhg.lib().pdhg_backward(ws.ws, 0.0, gxt.data_ptr(), gq.data_ptr(), gc.data_ptr(), stream)
    assert rc == 0, pdhg.lib().pdhg_last_error()
    g = gq.cpu().numpy()
    h = 1e-6 * np.abs(lp.q[bal]).max()
    q0 = lp.q.copy()
    errs = []
    for k in range(16):
        delta = rng.standard_normal(bal.size)
        delta /= np.abs(delta).max()
        sides = []
        for sgn in (1.0, -1.0):
            lp.q = q0.copy()
            lp.q[bal] += sgn * h * delta
            xv, yv, _ = highs_vertex(lp)
            # the vertex re-solved on its own active set (active-set polish)
            pv = polish(lp, xv, yv)
            sides.append(pv[0] if pv is not None else xv)
        fd = (gx @ sides[0] - gx @ sides[1]) / (2 * h)
        ad = g[bal] @ delta
        errs.append(abs(fd - ad) / max(abs(fd), 1e-12))
    lp.q = q0
    assert max(errs) <= 1e-5, errs
