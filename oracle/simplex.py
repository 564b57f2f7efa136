"""Dense two-phase tableau simplex with Bland's rule, FP64 (oracle; test infrastructure).

For tiny LPs in the general form of ``oracle.lp`` only.  The LP is brought to
standard form  min c'^T z, A z = b, z >= 0  by
  x_j = l_j + z_j            (finite l_j; plus row z_j + s_j = u_j - l_j if u_j finite)
  x_j = u_j - z_j            (l_j = -inf, finite u_j)
  x_j = z+_j - z-_j          (free)
  K_i x - s_i = q_i          (>= rows, s_i >= 0)
Phase 1 minimises the sum of artificial variables; phase 2 the cost.  Bland's
rule (lowest index enters; ties in the ratio test leave by lowest basic index)
guarantees termination.  Duals come out of the final tableau: with the
artificial columns kept, y = c_B B^-1 equals minus their phase-2 reduced costs.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .lp import LP


@dataclass
class SimplexResult:
    status: str          # "optimal" | "infeasible" | "unbounded"
    x: np.ndarray | None
    y: np.ndarray | None  # duals of the rows of K (L = c^T x - y^T (Kx - q))
    obj: float


def _pivot(T: np.ndarray, r: int, s: int) -> None:
    T[r] /= T[r, s]
    col = T[:, s].copy()
    col[r] = 0.0
    T -= np.outer(col, T[r])


def _run(T: np.ndarray, basis: list[int], allowed: np.ndarray, eps: float = 1e-11) -> str:
    m = T.shape[0] - 1
    for _ in range(50_000):
        rc = T[-1, :-1]
        cand = np.where((rc < -eps) & allowed)[0]
        if cand.size == 0:
            return "optimal"
        s = int(cand[0])
        colv = T[:m, s]
        pos = colv > eps
        if not pos.any():
            return "unbounded"
        ratios = np.full(m, np.inf)
        ratios[pos] = T[:m, -1][pos] / colv[pos]
        best = ratios.min()
        ties = np.where(ratios <= best + 1e-12 * max(1.0, abs(best)))[0]
        r = int(min(ties, key=lambda i: basis[i]))
        _pivot(T, r, s)
        basis[r] = s
    raise RuntimeError("simplex did not terminate")


def simplex_solve(lp: LP) -> SimplexResult:
    K = lp.K.toarray()
    m, n = K.shape
    l, u, c, q = lp.l, lp.u, lp.c, lp.q
    # column map: x = off + M z
    cols = []      # list of (j, sign)
    off = np.zeros(n)
    ub_rows = []   # (z column, bound)
    for j in range(n):
        if np.isfinite(l[j]):
            off[j] = l[j]
            cols.append((j, 1.0))
            if np.isfinite(u[j]):
                ub_rows.append((len(cols) - 1, u[j] - l[j]))
        elif np.isfinite(u[j]):
            off[j] = u[j]
            cols.append((j, -1.0))
        else:
            cols.append((j, 1.0))
            cols.append((j, -1.0))
    nz = len(cols)
    n_in = m - lp.m_eq
    n_ub = len(ub_rows)
    n_s = n_in + n_ub
    rows = m + n_ub
    A = np.zeros((rows, nz + n_s))
    b = np.zeros(rows)
    cz = np.zeros(nz + n_s)
    for k, (j, sgn) in enumerate(cols):
        A[:m, k] = sgn * K[:, j]
        cz[k] = sgn * c[j]
    b[:m] = q - K @ off
    for i in range(lp.m_eq, m):
        A[i, nz + (i - lp.m_eq)] = -1.0
    for t, (k, bound) in enumerate(ub_rows):
        A[m + t, k] = 1.0
        A[m + t, nz + n_in + t] = 1.0
        b[m + t] = bound
    sign = np.where(b < 0, -1.0, 1.0)
    A *= sign[:, None]
    b *= sign
    N = nz + n_s
    # tableau: [A | I_art | b]; last row = objective
    T = np.zeros((rows + 1, N + rows + 1))
    T[:rows, :N] = A
    T[:rows, N:N + rows] = np.eye(rows)
    T[:rows, -1] = b
    basis = list(range(N, N + rows))
    # phase 1
    T[-1, N:N + rows] = 1.0
    for i in range(rows):
        T[-1] -= T[i]
    allowed = np.ones(N + rows, dtype=bool)
    st = _run(T, basis, allowed)
    if -T[-1, -1] > 1e-8 * max(1.0, np.abs(b).max()):
        return SimplexResult("infeasible", None, None, np.nan)
    # drive artificials out of the basis
    redundant = []
    for i in range(rows):
        if basis[i] >= N:
            nzc = np.where(np.abs(T[i, :N]) > 1e-9)[0]
            if nzc.size:
                _pivot(T, i, int(nzc[0]))
                basis[i] = int(nzc[0])
            else:
                redundant.append(i)
    # phase 2 objective row
    T[-1, :] = 0.0
    T[-1, :N] = cz
    for i in range(rows):
        if basis[i] < N and cz[basis[i]] != 0.0:
            T[-1] -= cz[basis[i]] * T[i]
    allowed = np.zeros(N + rows, dtype=bool)
    allowed[:N] = True
    st = _run(T, basis, allowed)
    if st != "optimal":
        return SimplexResult(st, None, None, np.nan)
    z = np.zeros(N + rows)
    for i in range(rows):
        z[basis[i]] = T[i, -1]
    x = off.copy()
    for k, (j, sgn) in enumerate(cols):
        x[j] += sgn * z[k]
    # duals of the standard-form rows: y = c_B B^-1 = -(phase-2 reduced cost of artificials)
    ystd = -T[-1, N:N + rows] * sign
    for i in redundant:
        ystd[i] = 0.0
    y = ystd[:m].copy()
    return SimplexResult("optimal", x, y, float(c @ x))
