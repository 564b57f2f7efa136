"""Nondegenerate perturbations of UC relaxations for the active-set tests
(test infrastructure; no solver arithmetic).

The UC relaxation is degenerate at its optimum (a unit that is off makes
several constraints tight at once, shutdown variables cost nothing).  A
seeded perturbation relaxes every >= row by U(0.5, 1) * rel_row * (1 + |q_i|),
moves every finite bound of a non-fixed variable outward by
U(0.5, 1) * rel_bound * (1 + |bound|), multiplies each cost by
(1 + rel_cost * U(-1, 1)) and gives every zero-cost bounded variable (not the
angles) a cost U(0.5, 1) * add_cost.  At the 24-bus size the defaults make the
optimal vertex nondegenerate (as many active rows as free variables, checked
by the tests), which smaller perturbations do not."""
from __future__ import annotations

import numpy as np

from oracle.lp import LP
from paper_2512_06715_gb300.instances import VAR_THETA


def perturbed_lp(inst, seed: int, rel_row=1e-2, rel_bound=1e-3, rel_cost=1e-2, add_cost=1.0) -> LP:
    rng = np.random.default_rng(seed)
    q = inst.q.copy()
    ineq = np.arange(inst.m) >= inst.m_eq
    q[ineq] -= rng.uniform(0.5, 1.0, ineq.sum()) * rel_row * (1.0 + np.abs(q[ineq]))
    c = inst.c * (1.0 + rel_cost * rng.uniform(-1.0, 1.0, inst.n))
    zero = (c == 0.0) & (inst.var_kind != VAR_THETA)
    c[zero] += add_cost * rng.uniform(0.5, 1.0, zero.sum())
    l, u = inst.l.copy(), inst.u.copy()
    movable = l < u
    lf = movable & np.isfinite(l)
    uf = movable & np.isfinite(u)
    l[lf] -= rng.uniform(0.5, 1.0, lf.sum()) * rel_bound * (1.0 + np.abs(l[lf]))
    u[uf] += rng.uniform(0.5, 1.0, uf.sum()) * rel_bound * (1.0 + np.abs(u[uf]))
    return LP(K=inst.scipy_csr(), q=q, c=c, l=l, u=u, m_eq=inst.m_eq)


def highs_vertex(lp: LP):
    """Optimal vertex and duals (L = c^T x - y^T (Kx - q)) from SciPy's HiGHS."""
    import scipy.optimize as opt
    K = lp.K
    bounds = [(None if not np.isfinite(a) else a, None if not np.isfinite(b) else b)
              for a, b in zip(lp.l, lp.u)]
    r = opt.linprog(lp.c, A_ub=-K[lp.m_eq:], b_ub=-lp.q[lp.m_eq:], A_eq=K[: lp.m_eq], b_eq=lp.q[: lp.m_eq],
                    bounds=bounds, method="highs")
    assert r.status == 0, r.message
    y = np.concatenate([r.eqlin.marginals, -r.ineqlin.marginals])
    return r.x, y, float(r.fun)
