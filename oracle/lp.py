"""LP in PDLP general form and its optimality measures (oracle; test infrastructure).

The paper writes the LP as min c^T x s.t. Ax <= b, x >= 0 with the saddle
function L(x, y) = c^T x - y^T A x + b^T y and a y-ascent step (Sec. II.E).
That statement is inconsistent in its signs (the y-step and L imply Ax >= b)
and its dual update carries no projection onto y >= 0.  The reading used
throughout is the PDLP general form the cited Applegate et al. work uses:

    min c^T x  s.t.  K_i x = q_i (i < m_eq),  K_i x >= q_i (i >= m_eq),  l <= x <= u
    L(x, y) = c^T x - y^T (K x - q),   x in [l, u],   y_i free (i < m_eq), y_i >= y_lo_i

which reduces to the paper's L with A = K, b = q and the y-update of Sec. II.E
plus the projection onto the dual cone.  y_lo defaults to 0 on the >= rows.

Optimality measures (l2, on the unscaled LP, FP64):
  r_p      = q - Kx on equality rows, (q - Kx)^+ on >= rows
  lambda   = c - K^T y;  lambda_proj keeps the sign each finite bound allows
  r_d      = lambda - lambda_proj
  P(x)     = c^T x + sum_{>= rows} y_lo_i * min(q - Kx, 0)_i
  D(y)     = q^T y + sum_j (l_j lambda_proj_j^+ - u_j lambda_proj_j^-)
  rel_p    = ||r_p|| / (1 + ||q||),  rel_d = ||r_d|| / (1 + ||c||)
  rel_gap  = |P - D| / (1 + |P| + |D|)
  rel_kkt  = max(rel_p, rel_d, rel_gap)

``ray_check`` tests candidate rays for the infeasibility certificates of the
same LP (see ``RayCheck``).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


@dataclass
class LP:
    K: sp.csr_matrix
    q: np.ndarray
    c: np.ndarray
    l: np.ndarray
    u: np.ndarray
    m_eq: int
    y_lo: np.ndarray | None = None  # [m]; -inf on equality rows; default 0 on >= rows

    @property
    def m(self) -> int:
        return self.K.shape[0]

    @property
    def n(self) -> int:
        return self.K.shape[1]

    def dual_lower(self) -> np.ndarray:
        if self.y_lo is not None:
            return np.asarray(self.y_lo, dtype=np.float64)
        lo = np.zeros(self.m)
        lo[: self.m_eq] = -np.inf
        return lo


def lp_from_arrays(row_ptr, col, val, q, c, l, u, m_eq, n=None, y_lo=None) -> LP:
    m = len(row_ptr) - 1
    n = len(c) if n is None else n
    K = sp.csr_matrix((np.asarray(val, np.float64), np.asarray(col), np.asarray(row_ptr)), shape=(m, n))
    return LP(K=K, q=np.asarray(q, np.float64), c=np.asarray(c, np.float64), l=np.asarray(l, np.float64),
              u=np.asarray(u, np.float64), m_eq=int(m_eq), y_lo=None if y_lo is None else np.asarray(y_lo))


def project_reduced_cost(lam: np.ndarray, l: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Part of lambda = c - K^T y that the bounds can absorb: lambda_j >= 0 needs a
    finite lower bound, lambda_j <= 0 a finite upper bound."""
    lf = np.isfinite(l)
    uf = np.isfinite(u)
    pos = np.where(lf, np.maximum(lam, 0.0), 0.0)
    neg = np.where(uf, np.minimum(lam, 0.0), 0.0)
    return pos + neg


@dataclass
class KKT:
    primal_obj: float
    dual_obj: float
    rp: np.ndarray
    rd: np.ndarray
    rel_p: float
    rel_d: float
    rel_gap: float

    @property
    def rel_kkt(self) -> float:
        return max(self.rel_p, self.rel_d, self.rel_gap)


def kkt(lp: LP, x: np.ndarray, y: np.ndarray) -> KKT:
    Kx = lp.K @ x
    KTy = lp.K.T @ y
    slack = lp.q - Kx
    rp = slack.copy()
    rp[lp.m_eq:] = np.maximum(rp[lp.m_eq:], 0.0)
    lam = lp.c - KTy
    lam_proj = project_reduced_cost(lam, lp.l, lp.u)
    rd = lam - lam_proj
    y_lo = lp.dual_lower()
    ineq = np.arange(lp.m) >= lp.m_eq
    # infinite bounds are masked before they multiply (no inf * 0 is formed)
    ylo_fin = ineq & np.isfinite(y_lo)
    ylo_term = np.where(ylo_fin, y_lo, 0.0) * np.where(ylo_fin, np.minimum(slack, 0.0), 0.0)
    P = float(lp.c @ x + ylo_term.sum())
    lf = np.isfinite(lp.l)
    uf = np.isfinite(lp.u)
    bound = (np.where(lf, lp.l, 0.0) * np.where(lf, np.maximum(lam_proj, 0.0), 0.0)).sum() - \
        (np.where(uf, lp.u, 0.0) * np.where(uf, np.maximum(-lam_proj, 0.0), 0.0)).sum()
    D = float(lp.q @ y + bound)
    rel_p = float(np.linalg.norm(rp) / (1.0 + np.linalg.norm(lp.q)))
    rel_d = float(np.linalg.norm(rd) / (1.0 + np.linalg.norm(lp.c)))
    rel_gap = abs(P - D) / (1.0 + abs(P) + abs(D))
    return KKT(P, D, rp, rd, rel_p, rel_d, rel_gap)


@dataclass
class RayCheck:
    """Certificate test of two candidate rays of the LP (Applegate et al.'s
    infeasibility detection for PDHG, which the paper's cited PDLP method uses).

    dual ray y (proves primal infeasibility; Farkas):
      lambda = -K^T y (the dual constraints with c = 0),
      violations: y_i < 0 on >= rows; lambda_j > 0 where l_j = -inf;
                  lambda_j < 0 where u_j = +inf,
      objective  q^T y + sum_j (l_j lambda_j^+ - u_j lambda_j^-) over finite bounds.
    primal ray x (proves dual infeasibility, i.e. an unbounded LP):
      violations: (K x)_i != 0 on equality rows, (K x)_i < 0 on >= rows,
                  x_j < 0 where l_j is finite, x_j > 0 where u_j is finite,
      objective  c^T x.
    Violations are measured in the l2 norm of all violated components."""
    dual_ray_obj: float
    dual_ray_viol: float
    primal_ray_obj: float
    primal_ray_viol: float

    def primal_infeasible(self, eps: float) -> bool:
        return self.dual_ray_obj > 0.0 and self.dual_ray_viol <= eps * self.dual_ray_obj

    def dual_infeasible(self, eps: float) -> bool:
        return self.primal_ray_obj < 0.0 and self.primal_ray_viol <= eps * (-self.primal_ray_obj)


def ray_check(lp: LP, dx: np.ndarray, dy: np.ndarray) -> RayCheck:
    lf = np.isfinite(lp.l)
    uf = np.isfinite(lp.u)
    ineq = np.arange(lp.m) >= lp.m_eq
    # dual ray
    lam = -(lp.K.T @ dy)
    v_sign = np.where(ineq, np.minimum(dy, 0.0), 0.0)
    v_lam = np.where(lf, 0.0, np.maximum(lam, 0.0)) + np.where(uf, 0.0, np.minimum(lam, 0.0))
    d_obj = float(lp.q @ dy + (np.where(lf, lp.l, 0.0) * np.where(lf, np.maximum(lam, 0.0), 0.0)).sum()
                  - (np.where(uf, lp.u, 0.0) * np.where(uf, np.maximum(-lam, 0.0), 0.0)).sum())
    d_viol = float(np.sqrt(v_sign @ v_sign + v_lam @ v_lam))
    # primal ray
    Kx = lp.K @ dx
    v_row = np.where(ineq, np.minimum(Kx, 0.0), Kx)
    v_bnd = np.where(lf, np.minimum(dx, 0.0), 0.0) + np.where(uf, np.maximum(dx, 0.0), 0.0)
    p_obj = float(lp.c @ dx)
    p_viol = float(np.sqrt(v_row @ v_row + v_bnd @ v_bnd))
    return RayCheck(d_obj, d_viol, p_obj, p_viol)


def max_violation(lp: LP, x: np.ndarray) -> float:
    """Largest absolute violation of rows and bounds at x (unscaled)."""
    Kx = lp.K @ x
    v_eq = np.abs(Kx[: lp.m_eq] - lp.q[: lp.m_eq])
    v_in = np.maximum(lp.q[lp.m_eq:] - Kx[lp.m_eq:], 0.0)
    v_l = np.maximum(lp.l - x, 0.0)
    v_u = np.maximum(x - lp.u, 0.0)
    return float(max(v_eq.max(initial=0.0), v_in.max(initial=0.0), v_l.max(initial=0.0),
                     v_u.max(initial=0.0)))
