"""Single-bus, single-period economic dispatch by merit order (oracle; test infrastructure).

With one bus (no network) and one period (no ramp, logic or minimum up/down
rows; start-up fixed to 0) the DC-UC relaxation is

    min sum_g dt (c_g p_g + NL_g u_g)  s.t.  sum_g p_g = d,
        Pmin_g u_g <= p_g <= Pmax_g u_g,  0 <= u_g <= 1,  p_g >= 0.

For any p the cheapest feasible u is u_g = p_g / Pmax_g (Pmin_g u_g <= p_g
holds since Pmin <= Pmax), so the relaxation is a continuous knapsack over
p_g in [0, Pmax_g] with unit price dt (c_g + NL_g / Pmax_g): fill generators in
ascending price until d is met.  The balance-row dual equals the price of the
marginal (partly loaded) generator; when d falls exactly on a breakpoint any
value between the two adjacent prices is dual optimal.
"""
from __future__ import annotations

import numpy as np


def merit_order(d: float, pmax: np.ndarray, cost: np.ndarray, noload: np.ndarray, dt: float):
    """Return (objective, p, u, marginal_price)."""
    price = dt * (cost + noload / pmax)
    order = np.argsort(price, kind="stable")
    p = np.zeros_like(pmax)
    rem = float(d)
    marginal = float(price[order[0]])
    for g in order:
        if rem <= 0.0:
            break
        take = min(rem, float(pmax[g]))
        p[g] = take
        rem -= take
        marginal = float(price[g])
    if rem > 1e-9 * max(1.0, d):
        raise ValueError("load exceeds total capacity")
    u = p / pmax
    obj = float(price @ p)
    return obj, p, u, marginal
