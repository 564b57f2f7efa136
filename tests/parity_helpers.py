"""Comparison helpers shared by the GPU parity tests (GPU result vs oracle)."""
import numpy as np

from oracle.lp import kkt
from oracle.pdhg import pdhg_solve


def returned_candidate(lp, ref, r):
    """The oracle candidate (current iterate or average since the last restart)
    that the GPU reports it returned, after checking that the choice is the
    oracle's own (the smaller rel-KKT) whenever the two do not tie."""
    rc = kkt(lp, ref.x_cur, ref.y_cur).rel_kkt
    ra = kkt(lp, ref.x_avg, ref.y_avg).rel_kkt
    if abs(ra - rc) > 1e-6 * max(ra, rc):
        assert bool(r["returned_average"]) == (ra < rc), (ra, rc, r["returned_average"])
    return (ref.x_avg, ref.y_avg) if r["returned_average"] else (ref.x_cur, ref.y_cur)


def rel_err(x, y, cand):
    a, b = cand
    return max(np.abs(x - a).max() / np.abs(a).max(), np.abs(y - b).max() / np.abs(b).max())


def replay_and_compare(ws, lp, attempts):
    """Runs `attempts` adaptive attempts on the GPU with the trace on, replays the
    GPU's step sizes and accept/restart decisions in the oracle, and checks:
    the oracle's own accept and restart decisions equal the GPU's; eta_max
    agrees to 1e-8 and the next step to 1e-5 (the GPU takes the factors
    (k+1)^-0.3, (k+1)^-0.6 in FP32); the primal weight, which the oracle never
    replays but updates itself at each restart from its own iterates, agrees
    at every attempt and after every check to 1e-10; the returned iterate is the
    oracle's choice of candidate and agrees to 1e-10 relative."""
    x, y, r = ws.solve()
    x, y = x.cpu().numpy(), y.cpu().numpy()
    ta, tc = ws.trace()
    assert len(ta) == attempts and len(tc) == attempts // 64
    sched = dict(attempts=[(e[0], int(e[2])) for e in ta], checks=[(int(c[1]), int(c[2])) for c in tc])
    ref = pdhg_solve(lp, tol=1e-30, stop_after=attempts, schedule=sched, record=True)
    own = np.array([a[5] for a in ref.attempt_log])
    assert np.array_equal(own, ta[:, 2].astype(int))
    eta_max_o = np.array([a[3] for a in ref.attempt_log])
    eta_next_o = np.array([a[4] for a in ref.attempt_log])
    fin = np.isfinite(eta_max_o)
    assert np.allclose(ta[fin, 3], eta_max_o[fin], rtol=1e-8)
    assert np.allclose(ta[fin, 4], eta_next_o[fin], rtol=1e-5)
    omega_o = np.array([a[1] for a in ref.attempt_log])
    assert np.allclose(ta[:, 1], omega_o, rtol=1e-10, atol=0)
    omega_after_o = np.array([c["omega_after"] for c in ref.check_log])
    assert np.allclose(tc[:, 3], omega_after_o, rtol=1e-10, atol=0), (tc[:, 3], omega_after_o)
    assert tc[:, 1].sum() >= 1  # at least one restart moved the primal weight
    for c_gpu, c_or in zip(tc[:-1], ref.check_log[:-1]):
        assert int(c_gpu[1]) == int(c_or["restart_own"])
        if int(c_gpu[1]):
            assert int(c_gpu[2]) == int(c_or["to_avg_own"])
    err = rel_err(x, y, returned_candidate(lp, ref, r))
    assert err <= 1e-10, err
    return r
