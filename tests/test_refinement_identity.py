"""The refinement reading (correction LP of Gleixner, Steffy and Wolter with one
scale factor Delta for both sides): PDHG on the correction LP from x^ = y^ = 0 is,
mapped back by x* + x^/Delta and y* + y^/Delta, PDHG on the LP itself restarted at
(x*, y*) with the same step size and primal weight.  This is what lets a mixed-
precision refinement round end at a restart without changing the method's
dynamics.  Checked with the oracle's PDHG iteration (Sec. II.E form, constant
steps), CPU only."""
import numpy as np
import pytest

from oracle.lp import LP, kkt
from oracle.pdhg import pdhg_solve
from oracle.scaling import rescale


def _correction(lp: LP, xs, ys, delta):
    return LP(K=lp.K, q=delta * (lp.q - lp.K @ xs), c=delta * (lp.c - lp.K.T @ ys),
              l=delta * (lp.l - xs), u=delta * (lp.u - xs), m_eq=lp.m_eq,
              y_lo=delta * (lp.dual_lower() - ys))


@pytest.mark.parametrize("delta", [1.0, 1e3, 1e6])
def test_correction_round_is_a_restart_in_new_coordinates(tiny24, delta):
    inst, lp = tiny24
    slp, _, _ = rescale(lp)
    eta = 0.9 / np.abs(slp.K.data).max()
    omega = np.linalg.norm(slp.c) / np.linalg.norm(slp.q)
    fixed = dict(eta=eta, omega=omega)
    first = pdhg_solve(lp, fixed=fixed, stop_after=300)       # a point far from optimal
    xs, ys = first.x_cur, first.y_cur
    plain = pdhg_solve(lp, fixed=fixed, stop_after=200, start=(xs, ys))
    corr = pdhg_solve(_correction(lp, xs, ys, delta), fixed=fixed, stop_after=200,
                      start=(np.zeros(lp.n), np.zeros(lp.m)))
    x_back = xs + corr.x_cur / delta
    y_back = ys + corr.y_cur / delta
    assert np.abs(x_back - plain.x_cur).max() <= 1e-9 * np.abs(plain.x_cur).max()
    assert np.abs(y_back - plain.y_cur).max() <= 1e-9 * np.abs(plain.y_cur).max()


def test_correction_residuals_and_saddle_scale_with_delta(tiny24):
    """At mapped points the correction LP's primal and dual residuals are Delta times
    the LP's, and its saddle function is Delta^2 times the LP's up to a constant:
    L^(x^, y^) = Delta^2 (L(x, y) - L(x*, y*)).  Objective-like terms (the gap)
    therefore grow like Delta^2 and residuals like Delta, which is why the restart
    test weights the gap back to round-0 units."""
    inst, lp = tiny24
    slp, _, _ = rescale(lp)
    eta = 0.9 / np.abs(slp.K.data).max()
    omega = np.linalg.norm(slp.c) / np.linalg.norm(slp.q)
    r = pdhg_solve(lp, fixed=dict(eta=eta, omega=omega), stop_after=400)
    xs, ys = r.x_cur, r.y_cur
    r2 = pdhg_solve(lp, fixed=dict(eta=eta, omega=omega), stop_after=50, start=(xs, ys))
    x, y = r2.x_cur, r2.y_cur
    delta = 1e4
    xh, yh = delta * (x - xs), delta * (y - ys)
    lph = _correction(lp, xs, ys, delta)
    a, b = kkt(lp, x, y), kkt(lph, xh, yh)
    assert np.linalg.norm(b.rp - delta * a.rp) <= 1e-9 * delta * np.linalg.norm(a.rp)
    assert np.linalg.norm(b.rd - delta * a.rd) <= 1e-9 * delta * np.linalg.norm(a.rd)

    def saddle(p, u, v):
        return p.c @ u - v @ (p.K @ u - p.q)

    lhs = saddle(lph, xh, yh)
    rhs = delta ** 2 * (saddle(lp, x, y) - saddle(lp, xs, ys))
    assert lhs == pytest.approx(rhs, rel=1e-8)
