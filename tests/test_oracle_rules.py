"""Hand-worked pins of the oracle's PDLP rules (step size, restart, primal
weight) and of the Pock-Chambolle pass of the rescaling.

The paper cites Applegate et al. for the adaptive step sizes and restarts of
its PDHG (Sec. II.E) without stating them; these tests fix the oracle's
reading of those rules with values worked out by hand on tiny problems, so
that a swapped operand, a wrong exponent index or a flipped inequality fails
here on the CPU instead of being carried into the GPU parity tests."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.lp import LP
from oracle.pdhg import (PDLPOptions, pdhg_solve, primal_weight_update, restart_decision,
                         step_size_update)
from oracle.scaling import rescale
from tests.conftest import instance_lp

NO_SCALING = dict(ruiz_iters=0, pock_chambolle=False)


def _two_var_lp():
    """min 6 x1 + 8 x2  s.t.  x1 + 2 x2 = 5,  -10 <= x <= 10.

    With no rescaling: eta_0 = 1 / max|K| = 1/2, omega_0 = ||c|| / ||q|| = 10/5 = 2,
    so tau = eta/omega = 1/4 and sigma = eta*omega = 1."""
    K = sp.csr_matrix(np.array([[1.0, 2.0]]))
    return LP(K=K, q=np.array([5.0]), c=np.array([6.0, 8.0]), l=np.array([-10.0, -10.0]),
              u=np.array([10.0, 10.0]), m_eq=1)


def test_first_two_attempts_by_hand():
    """Attempt 1 from x = 0, y = 0:
         x1 = x0 - tau c = (-1.5, -2),  K x1 = -5.5,
         y1 = y0 + sigma (q - 2 K x1 + K x0) = 5 + 11 = 16,
         ||dx||^2 = 6.25, ||dy||^2 = 256, dy^T K dx = 16 * (-5.5) = -88,
         eta_max = (omega ||dx||^2 + ||dy||^2 / omega) / (2 |dy^T K dx|)
                 = (12.5 + 128) / 176,
         accepted (1/2 <= eta_max), k = 1 so the factors use 2^-0.3 and 2^-0.6.
       Attempt 2 with eta = eta_1, tau = eta/2, sigma = 2 eta, K^T y1 = (16, 32):
         dx = -tau (c - K^T y1) = (10 tau, 24 tau), K dx = 58 tau,
         dy = sigma (q - 2 K x2 + K x1) = sigma (10.5 - 116 tau),
         and k = 2 uses 3^-0.3, 3^-0.6."""
    opts = PDLPOptions(**NO_SCALING)
    r = pdhg_solve(_two_var_lp(), tol=1e-30, stop_after=2, opts=opts, record=True)
    eta0, om0, acc0, emax0, enext0, _ = r.attempt_log[0]
    assert (eta0, om0, acc0) == (0.5, 2.0, 1)
    assert emax0 == pytest.approx(140.5 / 176.0, rel=1e-15)
    eta1 = min((1.0 - 2.0 ** -0.3) * 140.5 / 176.0, (1.0 + 2.0 ** -0.6) * 0.5)
    assert enext0 == pytest.approx(eta1, rel=1e-15)
    assert eta1 == pytest.approx(0.149878058590619, rel=1e-12)  # the reduction branch wins

    eta, om, acc, emax, enext, _ = r.attempt_log[1]
    assert (eta, om, acc) == (pytest.approx(eta1, rel=1e-15), 2.0, 1)
    tau, sigma = eta1 / 2.0, 2.0 * eta1
    dx = np.array([10.0 * tau, 24.0 * tau])
    dy = sigma * (10.5 - 116.0 * tau)
    emax_hand = (2.0 * (dx @ dx) + dy * dy / 2.0) / (2.0 * abs(dy * 58.0 * tau))
    assert emax == pytest.approx(emax_hand, rel=1e-13)
    assert enext == pytest.approx(min((1.0 - 3.0 ** -0.3) * emax_hand, (1.0 + 3.0 ** -0.6) * eta1),
                                  rel=1e-13)
    assert np.allclose(r.x_cur, [-1.5 + 10.0 * tau, -2.0 + 24.0 * tau], rtol=1e-14)
    assert np.allclose(r.y_cur, [16.0 + dy], rtol=1e-14)


def test_step_rule_rejects_and_shrinks():
    """A step larger than eta_max is rejected and the next step is the reduction
    branch: eta = 3 with movement 2 * 1 + 4 / 2 = 4 and interaction 2 * |2| = 4 gives
    eta_max = 1 < 3; at k = 7, eta' = (1 - 8^-0.3) * 1 = 1 - 2^-0.9."""
    opts = PDLPOptions()
    acc, emax, enext = step_size_update(3.0, 2.0, np.array([1.0, 0.0]), np.array([2.0]), np.array([1.0]),
                                        7, opts)
    assert not acc
    assert emax == 1.0
    assert enext == pytest.approx(1.0 - 2.0 ** -0.9, rel=1e-15)
    # interaction zero: eta_max infinite, accepted, growth branch (1 + 8^-0.6) eta
    acc, emax, enext = step_size_update(3.0, 2.0, np.array([1.0]), np.array([0.0]), np.array([1.0]), 7, opts)
    assert acc and emax == np.inf
    assert enext == pytest.approx(3.0 * (1.0 + 2.0 ** -1.8), rel=1e-15)


def test_kkt_omega_and_primal_weight_at_first_restart_by_hand():
    """Checking after every attempt (check_every = 1): after attempt 1 the
    artificial restart fires (1 attempt since restart >= 0.36 * 1).
         r_p = q - K x1 = 10.5, lambda = c - K^T y1 = (-10, -24) (both bounds
         finite, so r_d = 0), P = c^T x1 = -25, D = q y1 - u^T lambda^- = 80 - 340,
         KKT_omega = sqrt(2 * 10.5^2 + 235^2),  rel_kkt = 10.5 / (1 + 5) = 1.75.
       Primal weight: Dx = ||x1 - x0|| = 2.5, Dy = |y1 - y0| = 16, theta = 1/2:
         omega' = exp(0.5 log(16 / 2.5) + 0.5 log 2) = sqrt(12.8)
       (swapping Dx and Dy would give sqrt(0.3125))."""
    opts = PDLPOptions(check_every=1, **NO_SCALING)
    r = pdhg_solve(_two_var_lp(), tol=1e-30, stop_after=1, opts=opts, record=True)
    c0 = r.check_log[0]
    assert c0["kkt_cur"] == pytest.approx(np.sqrt(2.0 * 10.5 ** 2 + 235.0 ** 2), rel=1e-14)
    assert c0["rel_cur"] == pytest.approx(1.75, rel=1e-15)
    assert c0["restart"] and not c0["to_avg"]
    assert c0["omega_after"] == pytest.approx(np.sqrt(12.8), rel=1e-14)
    assert r.omega == pytest.approx(np.sqrt(12.8), rel=1e-14)


def test_primal_weight_update_by_hand():
    # log-space midpoint of omega and Dy/Dx
    assert primal_weight_update(1.0, 1.0, 4.0, 0.5) == pytest.approx(2.0, rel=1e-15)
    assert primal_weight_update(4.0, 3.0, 3.0, 0.5) == pytest.approx(2.0, rel=1e-15)
    assert primal_weight_update(1.0, 4.0, 1.0, 0.5) == pytest.approx(0.5, rel=1e-15)
    # theta weights the new ratio: theta = 1 takes Dy/Dx, theta = 0 keeps omega
    assert primal_weight_update(5.0, 2.0, 6.0, 1.0) == pytest.approx(3.0, rel=1e-15)
    assert primal_weight_update(5.0, 2.0, 6.0, 0.0) == pytest.approx(5.0, rel=1e-15)
    # a distance at or below 1e-10 leaves omega unchanged
    assert primal_weight_update(7.0, 1e-11, 1.0, 0.5) == 7.0
    assert primal_weight_update(7.0, 1.0, 1e-10, 0.5) == 7.0


@pytest.mark.parametrize(
    "kcur,kavg,has_avg,kkt0,prev,since,total,expect",
    [
        # sufficient decay: candidate <= 0.2 KKT_0
        (0.19, 0.5, True, 1.0, 0.1, 1, 1000, (True, False)),
        (0.5, 0.2, True, 1.0, 0.1, 1, 1000, (True, True)),
        (0.21, 0.5, True, 1.0, 0.3, 1, 1000, (False, False)),
        # necessary decay: <= 0.8 KKT_0 and larger than at the previous check
        (0.5, 0.9, True, 1.0, 0.4, 1, 1000, (True, False)),
        (0.5, 0.9, True, 1.0, 0.6, 1, 1000, (False, False)),
        (0.81, 0.9, True, 1.0, 0.5, 1, 1000, (False, False)),
        # artificial: attempts since the restart >= 0.36 of all attempts
        (0.9, 0.95, True, 1.0, 0.5, 36, 100, (True, False)),
        (0.9, 0.95, True, 1.0, 0.5, 35, 100, (False, False)),
        # no average yet: the current iterate is the candidate even if kavg is smaller
        (0.5, 0.1, False, 1.0, 0.6, 1, 1000, (False, False)),
    ])
def test_restart_decision_scripted(kcur, kavg, has_avg, kkt0, prev, since, total, expect):
    restart, to_avg, kc = restart_decision(kcur, kavg, has_avg, kkt0, prev, since, total, PDLPOptions())
    assert (restart, to_avg) == expect
    assert kc == (kavg if to_avg else kcur)


def test_restart_sequence_scripted():
    """A scripted KKT_omega sequence through the oracle's decision function with
    its own bookkeeping of KKT_0 and the previous value, late in a run (10^5
    attempts before, so the artificial rule stays silent): 1 -> 0.7 (decreasing:
    no restart) -> 0.75 (an increase below 0.8: restart, KKT_0 = 0.75) -> 0.5,
    0.4 (above 0.2 * 0.75 = 0.15 and decreasing: no restart) -> 0.14 (sufficient:
    restart)."""
    opts = PDLPOptions()
    kkt0, prev, since, total = 1.0, 1.0, 0, 100_000
    seq = [0.7, 0.75, 0.5, 0.4, 0.14]
    got = []
    for v in seq:
        since += 64
        total += 64
        restart, _, kc = restart_decision(v, np.inf, False, kkt0, prev, since, total, opts)
        prev = kc
        if restart:
            kkt0, prev, since = kc, kc, 0
        got.append(restart)
    assert got == [False, True, False, False, True]


def test_pock_chambolle_pass_by_hand():
    """K = [[1, 1], [0, 1]], no Ruiz passes: row sums (2, 1), column sums (1, 2),
    Dr = (1/sqrt 2, 1), Dc = (1, 1/sqrt 2), K~ = [[1/sqrt 2, 1/2], [0, 1/sqrt 2]],
    whose largest singular value is exactly 1 (sigma^2 = (1.25 + 0.75) / 2)."""
    K = sp.csr_matrix(np.array([[1.0, 1.0], [0.0, 1.0]]))
    lp = LP(K=K, q=np.zeros(2), c=np.zeros(2), l=np.zeros(2), u=np.ones(2), m_eq=0)
    slp, Dr, Dc = rescale(lp, ruiz_iters=0, pock_chambolle=True)
    s = 1.0 / np.sqrt(2.0)
    assert np.allclose(Dr, [s, 1.0], rtol=1e-15)
    assert np.allclose(Dc, [1.0, s], rtol=1e-15)
    assert np.allclose(slp.K.toarray(), [[s, 0.5], [0.0, s]], rtol=1e-15)
    assert np.linalg.norm(slp.K.toarray(), 2) == pytest.approx(1.0, rel=1e-14)
    # a row's l1 sum may exceed 1 (here 1/sqrt 2 + 1/2); the bound is on the 2-norm
    assert np.abs(slp.K.toarray()).sum(axis=1).max() > 1.0


def test_ruiz_passes_by_hand():
    """K = [[4, 1], [1, 0]]: pass 1 divides by sqrt of the row and column maxima
    (4, 1) -> Dr = Dc = (1/2, 1), K1 = [[1, 1/2], [1/2, 0]]; pass 2 (maxima (1, 1/2))
    -> Dr = Dc = (1/2, sqrt 2)."""
    K = sp.csr_matrix(np.array([[4.0, 1.0], [1.0, 0.0]]))
    lp = LP(K=K, q=np.zeros(2), c=np.zeros(2), l=np.zeros(2), u=np.ones(2), m_eq=0)
    slp, Dr, Dc = rescale(lp, ruiz_iters=1, pock_chambolle=False)
    assert np.allclose(Dr, [0.5, 1.0], rtol=1e-15) and np.allclose(Dc, [0.5, 1.0], rtol=1e-15)
    assert np.allclose(slp.K.toarray(), [[1.0, 0.5], [0.5, 0.0]], rtol=1e-15)
    _, Dr, Dc = rescale(lp, ruiz_iters=2, pock_chambolle=False)
    assert np.allclose(Dr, [0.5, np.sqrt(2.0)], rtol=1e-15)
    assert np.allclose(Dc, [0.5, np.sqrt(2.0)], rtol=1e-15)


def _power_norm(A, iters=300, seed=0):
    """Largest singular value of a sparse matrix by power iteration on A^T A."""
    v = np.random.default_rng(seed).standard_normal(A.shape[1])
    AT = A.T.tocsr()
    for _ in range(iters):
        v = AT @ (A @ v)
        v /= np.linalg.norm(v)
    return float(np.sqrt(np.linalg.norm(AT @ (A @ v))))


def test_pock_chambolle_bounds_the_norm(tiny24):
    """After Ruiz and the alpha = 1 Pock-Chambolle pass, ||K~||_2 <= 1 (Schur test
    with weights sqrt of the pass's row and column sums); without the pass the
    Ruiz-only matrix has a norm well above 1 on the UC relaxation.  The bound is
    what makes constant steps eta < 1 stable in the full-size parity test."""
    _, lp = tiny24
    slp, _, _ = rescale(lp, ruiz_iters=10, pock_chambolle=True)
    rlp, _, _ = rescale(lp, ruiz_iters=10, pock_chambolle=False)
    nrm = _power_norm(slp.K)
    assert 0.5 < nrm <= 1.0 + 1e-12, nrm
    assert _power_norm(rlp.K) > 1.5
    # the Pock-Chambolle factors are 1/sqrt of the Ruiz-scaled matrix's l1 sums
    A = abs(rlp.K)
    r, c = np.asarray(A.sum(axis=1)).ravel(), np.asarray(A.sum(axis=0)).ravel()
    back = sp.diags(np.sqrt(r)) @ slp.K @ sp.diags(np.sqrt(c)) - rlp.K
    assert abs(back).max() <= 1e-12 * abs(rlp.K).max()
