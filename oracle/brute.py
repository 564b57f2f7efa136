"""Enumeration of commitment schedules on tiny instances (oracle; test infrastructure).

The LP relaxation bound must not exceed the optimum of the UC MILP, and it
equals it when the relaxed commitment comes out integral.  On instances with a
handful of generators and periods the MILP optimum is found by enumerating all
u in {0,1}^(G x T): each schedule fixes u through its bounds and the remaining
LP (start-up/shut-down, dispatch, angles) is solved by the dense simplex.
"""
from __future__ import annotations

import itertools

import numpy as np

from .lp import LP
from .simplex import simplex_solve


def milp_by_enumeration(lp: LP, idx_u: np.ndarray):
    """idx_u: [T, G] variable indices of u.  Returns (best objective, best schedule)."""
    T, G = idx_u.shape
    flat = idx_u.reshape(-1)
    best, best_sched = np.inf, None
    for bits in itertools.product((0.0, 1.0), repeat=flat.size):
        l = lp.l.copy()
        u = lp.u.copy()
        l[flat] = bits
        u[flat] = bits
        sub = LP(K=lp.K, q=lp.q, c=lp.c, l=l, u=u, m_eq=lp.m_eq, y_lo=lp.y_lo)
        res = simplex_solve(sub)
        if res.status == "optimal" and res.obj < best:
            best, best_sched = res.obj, np.array(bits).reshape(T, G)
    return best, best_sched
