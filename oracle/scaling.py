"""Diagonal rescaling before PDHG (oracle; test infrastructure).

The paper defers PDHG's practical enhancements to Applegate et al. (Sec. II.E);
their PDLP applies Ruiz equilibration followed by a Pock-Chambolle step.  The
reading used here: 10 Ruiz passes in the l_inf norm, then one Pock-Chambolle
pass with alpha = 1, each pass computing row and column factors from the
current matrix simultaneously:

  Ruiz:  r_i = 1/sqrt(max_j |K_ij|),  s_j = 1/sqrt(max_i |K_ij|)
  PC:    r_i = 1/sqrt(sum_j |K_ij|),  s_j = 1/sqrt(sum_i |K_ij|)
  (a factor is 1 where the row or column is all zero)

and the scaled problem is K~ = diag(Dr) K diag(Dc), c~ = Dc c, q~ = Dr q,
l~ = l / Dc, u~ = u / Dc, y_lo~ = y_lo / Dr, with x = Dc x~ and y = Dr y~.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .lp import LP


def _inv_sqrt(v: np.ndarray) -> np.ndarray:
    out = np.ones_like(v)
    nz = v > 0
    out[nz] = 1.0 / np.sqrt(v[nz])
    return out


def rescale(lp: LP, ruiz_iters: int = 10, pock_chambolle: bool = True):
    """Return (scaled LP, Dr, Dc)."""
    K = lp.K.tocsr().astype(np.float64)
    Dr = np.ones(lp.m)
    Dc = np.ones(lp.n)
    for _ in range(ruiz_iters):
        A = abs(K)
        r = _inv_sqrt(A.max(axis=1).toarray().ravel())
        s = _inv_sqrt(A.max(axis=0).toarray().ravel())
        K = sp.diags(r) @ K @ sp.diags(s)
        Dr *= r
        Dc *= s
    if pock_chambolle:
        A = abs(K)
        r = _inv_sqrt(np.asarray(A.sum(axis=1)).ravel())
        s = _inv_sqrt(np.asarray(A.sum(axis=0)).ravel())
        K = sp.diags(r) @ K @ sp.diags(s)
        Dr *= r
        Dc *= s
    K = sp.csr_matrix(K)
    y_lo = lp.dual_lower() / Dr
    scaled = LP(K=K, q=Dr * lp.q, c=Dc * lp.c, l=lp.l / Dc, u=lp.u / Dc, m_eq=lp.m_eq, y_lo=y_lo)
    return scaled, Dr, Dc
