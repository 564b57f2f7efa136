"""Active-set polish of a near-optimal point to a basic solution (oracle; test
infrastructure).

Reading of the crossover step the paper's pipeline applies to the PDHG point
(Sec. III.B), restricted to what a nondegenerate optimum allows: read the
active set off the point in the rescaled space of ``oracle.scaling`` -- every
equality row, a >= row when its dual exceeds its slack (y~_i > (K~x~ - q~)_i),
a variable held at a bound when its reduced cost lambda~ = c~ - K~^T y~ exceeds
its distance to that bound (or l = u) -- and, if the set is square (active rows
= free variables F), solve the two square systems of that basis
    K~_{A,F} x~_F = q~_A - K~_{A,B} x~_B     (x~_B at its bounds)
    K~_{A,F}^T y~_A = c~_F                   (y~ = 0 off A)
with a sparse direct solver (the library primitive), and return the point in
the original scaling.  Returns None when the set is not square.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import spsolve

from .lp import LP
from .scaling import rescale


def active_set(slp: LP, x_s: np.ndarray, y_s: np.ndarray):
    """(active rows, free variables, value of each variable at its bound)."""
    s = slp.K @ x_s - slp.q
    rows = np.ones(slp.m, bool)
    rows[slp.m_eq:] = y_s[slp.m_eq:] > s[slp.m_eq:]
    lam = slp.c - slp.K.T @ y_s
    lf, uf = np.isfinite(slp.l), np.isfinite(slp.u)
    xfix = x_s.copy()
    at_lo = (lf & uf & (slp.l == slp.u)) | (lf & (lam > 0) & (lam > x_s - np.where(lf, slp.l, 0.0)))
    at_up = ~at_lo & uf & (lam < 0) & (-lam > np.where(uf, slp.u, 0.0) - x_s)
    xfix[at_lo] = slp.l[at_lo]
    xfix[at_up] = slp.u[at_up]
    free = ~(at_lo | at_up)
    return rows, free, xfix


def polish(lp: LP, x: np.ndarray, y: np.ndarray, ruiz_iters: int = 10, pock_chambolle: bool = True):
    slp, Dr, Dc = rescale(lp, ruiz_iters, pock_chambolle)
    rows, free, xfix = active_set(slp, x / Dc, y / Dr)
    if rows.sum() != free.sum():
        return None
    K = sp.csr_matrix(slp.K)
    S = K[rows][:, free].tocsc()
    xB = np.where(free, 0.0, xfix)
    b = slp.q[rows] - K[rows] @ xB
    xs = xfix.copy()
    xs[free] = spsolve(S, b)
    ys = np.zeros(slp.m)
    ys[rows] = spsolve(S.T.tocsc(), slp.c[free])
    return Dc * xs, Dr * ys
