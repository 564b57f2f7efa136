"""GPU parity of the PDHG path (through the C ABI) against the CPU oracle."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.lp import kkt, lp_from_arrays, max_violation
from oracle.pdhg import pdhg_solve
from oracle.scaling import rescale
from paper_2512_06715_gb300.instances import build_instance, workload
from tests.conftest import instance_lp
from tests.parity_helpers import rel_err, replay_and_compare, returned_candidate

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_06715_gb300 import build
    build.build()


def _ws(inst, **kw):
    from paper_2512_06715_gb300.pdhg import Workspace, default_opts
    kw.setdefault("time_limit_s", 120.0)
    return Workspace.from_instance(inst, default_opts(**kw))


def _random_lp(m, n, seed, long_rows=()):
    """Random sparse LP with empty rows, one-entry rows, long rows and a ragged
    tail (m, n not multiples of 32)."""
    rng = np.random.default_rng(seed)
    rows = []
    for i in range(m):
        if i % 17 == 3:
            k = 0
        elif i % 5 == 1:
            k = 1
        elif i in long_rows:
            k = min(n, 150)
        else:
            k = int(rng.integers(2, 9))
        cols = np.sort(rng.choice(n, size=k, replace=False))
        rows.append(cols)
    row_ptr = np.zeros(m + 1, np.int64)
    row_ptr[1:] = np.cumsum([len(r) for r in rows])
    col = np.concatenate(rows).astype(np.int32) if row_ptr[-1] else np.zeros(0, np.int32)
    val = rng.uniform(-3, 3, size=len(col)) * np.exp(rng.uniform(-4, 4, size=len(col)))
    c = rng.uniform(-1, 1, n)
    l = np.where(rng.random(n) < 0.3, -np.inf, -rng.uniform(0, 5, n))
    u = np.where(rng.random(n) < 0.3, np.inf, rng.uniform(0, 5, n))
    q = rng.uniform(-1, 1, m)
    return row_ptr, col, val, c, l, u, q


@pytest.mark.parametrize("shape", [(1000, 777), (45, 1000), (3001, 2999)])
def test_spmv_and_scaling_parity(shape):
    from paper_2512_06715_gb300.pdhg import PREC_FP64, PREC_MIXED, Workspace, default_opts
    m, n = shape
    rp, col, val, c, l, u, q = _random_lp(m, n, seed=m + n, long_rows=(7, m - 1))
    m_eq = m // 3
    ws = Workspace(rp, col, val, c, l, u, q, m_eq, default_opts())
    ws.prepare()
    Dr, Dc = (t.cpu().numpy() for t in ws.scaling())
    lp = lp_from_arrays(rp, col, val, q, c, l, u, m_eq, n=n)
    slp, Dr_o, Dc_o = rescale(lp)
    assert np.allclose(Dr, Dr_o, rtol=1e-12, atol=0)
    assert np.allclose(Dc, Dc_o, rtol=1e-12, atol=0)
    K = slp.K
    rng = np.random.default_rng(1)
    xv, yv = rng.standard_normal(n), rng.standard_normal(m)
    kx = ws.apply_K(torch.from_numpy(xv)).cpu().numpy()
    kty = ws.apply_K(torch.from_numpy(yv), transpose=True).cpu().numpy()
    scale_r = (abs(K) @ np.abs(xv)) + 1e-300
    scale_c = (abs(K.T) @ np.abs(yv)) + 1e-300
    assert np.all(np.abs(kx - K @ xv) <= 1e-14 * scale_r)
    assert np.all(np.abs(kty - K.T @ yv) <= 1e-14 * scale_c)
    kx32 = ws.apply_K(torch.from_numpy(xv), precision=PREC_MIXED).cpu().numpy()
    kty32 = ws.apply_K(torch.from_numpy(yv), transpose=True, precision=PREC_MIXED).cpu().numpy()
    assert np.all(np.abs(kx32 - K @ xv) <= 2e-6 * scale_r)
    assert np.all(np.abs(kty32 - K.T @ yv) <= 2e-6 * scale_c)
    # empty rows give exact zeros
    empty = np.where(np.diff(rp) == 0)[0]
    assert np.all(kx[empty] == 0.0)
    ws.close()


@pytest.mark.parametrize("variant,grid", [(-1, 0), (1, 3), (2, 3), (4, 2), (0, 0), (0, 3), (8, 3), (9, 2),
                                          (16, 0), (16, 3), (17, 2), (18, 0), (18, 3), (19, 2),
                                          (20, 0), (20, 3), (21, 2)])
def test_fixed_step_iterates_match_oracle(tiny24, variant, grid):
    """Constant steps, no restarts: iterates after 128 attempts agree with the
    oracle to 1e-10 relative, for every variant of the per-attempt kernels
    (1, 2, 4 slices per warp; 0 software pipelined) with the default grid and
    with 2-3 blocks, where each warp sweeps many slices and the ragged last one."""
    inst, lp = tiny24
    slp, _, _ = rescale(lp)
    eta = 0.9 / np.abs(slp.K.data).max()
    omega = np.linalg.norm(slp.c) / np.linalg.norm(slp.q)
    ws = _ws(inst, fixed_eta=eta, fixed_omega=omega, max_iters=128, tol=1e-30,
             kernel_variant=variant, kernel_grid=grid)
    x, y, r = ws.solve()
    x, y = x.cpu().numpy(), y.cpu().numpy()
    ref = pdhg_solve(lp, fixed=dict(eta=eta, omega=omega), stop_after=128)
    err = rel_err(x, y, returned_candidate(lp, ref, r))
    assert err <= 1e-10, err
    assert r["iterations"] == 128 and r["restarts"] == 0


def test_adaptive_schedule_replay(tiny24):
    """Adaptive steps and restarts on the 24-bus relaxation: 192 attempts (three
    checks, restarts at the first two) replayed in the oracle."""
    inst, lp = tiny24
    ws = _ws(inst, max_iters=192, tol=1e-30, trace=1)
    replay_and_compare(ws, lp, 192)
    ws.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_tiny_matches_oracle(tiny24, tiny24_oracle, precision):
    inst, lp = tiny24
    ws = _ws(inst, precision=precision, tol=1e-8)
    x, y, r = ws.solve()
    x, y = x.cpu().numpy(), y.cpu().numpy()
    assert r["status_name"] == "optimal", r
    chk = kkt(lp, x, y)
    assert chk.rel_kkt <= 1.5e-8, chk.rel_kkt
    assert abs(chk.rel_kkt - r["rel_kkt"]) <= 1e-2 * r["rel_kkt"] + 1e-12
    ref = tiny24_oracle
    assert abs(chk.primal_obj - ref.primal_obj) <= 1e-6 * abs(ref.primal_obj)
    assert max_violation(lp, x) <= 1e-7 * max(1.0, np.abs(lp.q).max())
    assert r["time_to_tol"][0] > 0 and r["time_to_tol"][2] >= r["time_to_tol"][0]


@pytest.mark.parametrize("variant", [0, 2, 4, 8, 9, 16, 17, 18, 19, 20, 21])
def test_fp32_kernel_variants_solve(tiny24, tiny24_oracle, variant):
    """Each non-default FP32 variant on a 3-block grid (every warp sweeps many
    slices and the ragged last one) solves the 24-bus relaxation to rel-KKT 1e-8
    in mixed precision: objective within 1e-6 of the oracle's, violation <= 1e-7."""
    inst, lp = tiny24
    ws = _ws(inst, precision="mixed", tol=1e-8, kernel_variant=variant, kernel_grid=3, time_limit_s=300.0)
    x, y, r = ws.solve()
    x, y = x.cpu().numpy(), y.cpu().numpy()
    assert r["status_name"] == "optimal", r
    chk = kkt(lp, x, y)
    assert chk.rel_kkt <= 1.5e-8, chk.rel_kkt
    ref = tiny24_oracle
    assert abs(chk.primal_obj - ref.primal_obj) <= 1e-6 * abs(ref.primal_obj)
    assert max_violation(lp, x) <= 1e-7 * max(1.0, np.abs(lp.q).max())
    assert ws.tuning()["fp32"]["unroll_dual"] == variant and ws.tuning()["fp32"]["grid_dual"] == 3
    ws.close()


@pytest.mark.parametrize("variant", [0, 2, 4, 8, 9, 16, 17, 18, 19, 20, 21])
def test_fp32_kernel_variants_fixed_step(tiny24, variant):
    """FP32 iterates of every kernel variant on 3 blocks (each warp sweeps many
    slices and the ragged last one) equal those of the one-slice variant on the
    default grid after 128 fixed-step attempts (rows are summed in the same order
    by every variant; only the step-size partials, unused with fixed steps, are
    reduced differently; 1e-5 allows for FMA contraction differing between the
    variants), and agree with the FP64 oracle to FP32 accuracy."""
    inst, lp = tiny24
    slp, _, _ = rescale(lp)
    eta = 0.9 / np.abs(slp.K.data).max()
    omega = np.linalg.norm(slp.c) / np.linalg.norm(slp.q)
    out = []
    for v, g in ((1, 0), (variant, 3)):
        ws = _ws(inst, precision="mixed", fixed_eta=eta, fixed_omega=omega, max_iters=128, tol=1e-30,
                 kernel_variant=v, kernel_grid=g)
        x, y, r = ws.solve()
        assert r["iterations"] == 128 and r["restarts"] == 0
        out.append((x.cpu().numpy(), y.cpu().numpy()))
    (x1, y1), (xv, yv) = out
    assert np.abs(xv - x1).max() <= 1e-5 * np.abs(x1).max()
    assert np.abs(yv - y1).max() <= 1e-5 * np.abs(y1).max()
    ref = pdhg_solve(lp, fixed=dict(eta=eta, omega=omega), stop_after=128)
    err = rel_err(xv, yv, returned_candidate(lp, ref, r))
    assert err <= 1e-4, err


@pytest.mark.parametrize("seed", [0, 1])
def test_solve_small_vs_oracle(seed):
    inst = build_instance(8, 10, 6, 6, seed=seed)
    lp = instance_lp(inst)
    ref = pdhg_solve(lp, tol=1e-9, max_attempts=1_000_000)
    for prec in ("fp64", "mixed"):
        ws = _ws(inst, precision=prec, tol=1e-9)
        x, y, r = ws.solve()
        x, y = x.cpu().numpy(), y.cpu().numpy()
        assert r["status_name"] == "optimal"
        assert abs(kkt(lp, x, y).primal_obj - ref.primal_obj) <= 1e-7 * abs(ref.primal_obj)


def test_limits_and_cancel(tiny24):
    inst, lp = tiny24
    ws = _ws(inst, max_iters=256, tol=1e-12)
    _, _, r = ws.solve()
    assert r["status_name"] == "iteration_limit" and r["iterations"] == 256
    ws.set_opts(max_iters=10_000_000, time_limit_s=0.002)
    _, _, r = ws.solve()
    assert r["status_name"] in ("time_limit", "optimal")
    flag = torch.ones(1, dtype=torch.int32).pin_memory()
    ws.set_opts(time_limit_s=60.0, cancel_flag=flag.data_ptr())
    _, _, r = ws.solve()
    assert r["status_name"] == "cancelled" and r["iterations"] == 64


def test_nan_data_reports_numeric():
    from paper_2512_06715_gb300.pdhg import PDHGError
    inst = build_instance(6, 8, 6, 6, seed=0)
    inst.c = inst.c.copy()
    inst.c[3] = np.nan
    ws = _ws(inst)
    with pytest.raises(PDHGError, match="NUMERIC"):
        ws.solve()


def test_staged_variant_refuses_oversized_slices():
    """The staged kernels (variants 16, 17) hold whole slices in shared-memory
    chunks; a matrix with a 150-entry row (a slice wider than a chunk) is
    refused before any launch, and the autotuner skips them there."""
    from paper_2512_06715_gb300.pdhg import PDHGError, Workspace, default_opts
    m, n = 300, 400
    rp, col, val, c, l, u, q = _random_lp(m, n, seed=5, long_rows=(7,))
    ws = Workspace(rp, col, val, c, l, u, q, m // 3, default_opts(kernel_variant=16, max_iters=64))
    with pytest.raises(PDHGError, match="UNSUPPORTED"):
        ws.solve()
    ws.close()
    ws = Workspace(rp, col, val, c, l, u, q, m // 3, default_opts(max_iters=64))
    ws.solve()
    assert ws.tuning()["fp64"]["unroll_dual"] not in (16, 17, 18, 19)
    ws.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("variant,grid", [(1, 0), (0, 0), (2, 3), (0, 3)])
def test_launch_overlap_is_bit_identical(tiny24, precision, variant, grid):
    """Programmatic dependent launch changes only when each per-attempt kernel
    starts reading the matrix: 1024 adaptive attempts (restarts, primal-weight
    updates, refinement folds in mixed precision) give bitwise the same
    iterates, decisions and counts with and without it, in the CUDA graph and
    launched from the host."""
    inst, _ = tiny24
    runs = {}
    for overlap in (1, 0):
        for host_loop in (0, 1):
            ws = _ws(inst, precision=precision, max_iters=1024, tol=1e-30, kernel_variant=variant,
                     kernel_grid=grid, launch_overlap=overlap, host_loop=host_loop)
            x, y, r = ws.solve()
            assert r["launch_overlap"] == overlap, r
            runs[(overlap, host_loop)] = (x.cpu().numpy(), y.cpu().numpy(), r)
            ws.close()
    x0, y0, r0 = runs[(0, 0)]
    for key, (x, y, r) in runs.items():
        assert np.array_equal(x, x0) and np.array_equal(y, y0), key
        for k in ("iterations", "accepted", "restarts", "rel_kkt", "omega", "eta", "ir_rounds"):
            assert r[k] == r0[k], (key, k, r[k], r0[k])
