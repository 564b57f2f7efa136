"""Instance generator invariants (host only)."""
import numpy as np
import pytest

from paper_2512_06715_gb300.instances import (ROW_BALANCE, ROW_FLOW_NEG, ROW_FLOW_POS, ROW_LOGIC,
                                              VAR_THETA, build_instance, workload)
from tests.conftest import instance_lp


def test_counts_tiny():
    inst = workload("uc24_g33_T24")
    G, N, L, T = 33, 24, 38, 24
    assert inst.n == T * (4 * G + N)
    m_expect = N * T + G * (T - 1) + 2 * L * T + 2 * G * T + 2 * G * (T - 1) + 2 * G * (T - 1)
    assert inst.m == m_expect
    assert inst.m_eq == N * T + G * (T - 1)
    assert np.all(inst.row_kind[: inst.m_eq] <= ROW_LOGIC)
    assert np.all(inst.row_kind[inst.m_eq:] >= ROW_FLOW_POS)
    assert np.all(np.diff(inst.row_ptr) >= 1)


def test_csr_sorted_unique():
    inst = workload("uc24_g33_T24")
    for i in range(inst.m):
        cols = inst.col[inst.row_ptr[i]:inst.row_ptr[i + 1]]
        assert np.all(np.diff(cols) > 0)


def test_network_rows():
    inst = workload("uc24_g33_T24")
    A = inst.scipy_csr().tocsr()
    theta = inst.var_kind == VAR_THETA
    bal = np.where(inst.row_kind == ROW_BALANCE)[0]
    # Laplacian part of every balance row sums to zero (flows conserve power)
    s = np.asarray(A[bal][:, theta].sum(axis=1)).ravel()
    assert np.allclose(s, 0.0, atol=1e-9 * np.abs(A.data).max())
    # the two flow-limit rows of each line are negatives of each other
    fp = np.where(inst.row_kind == ROW_FLOW_POS)[0]
    fn = np.where(inst.row_kind == ROW_FLOW_NEG)[0]
    assert len(fp) == len(fn)
    assert abs(A[fp] + A[fn]).max() == 0.0


def test_all_on_dispatch_feasible():
    """The proportional all-on dispatch that the line-limit floor is built for is
    feasible, so the relaxation is feasible by construction."""
    from oracle.lp import max_violation
    inst = workload("uc24_g33_T24")
    lp = instance_lp(inst)
    T, G = inst.idx_p.shape
    x = np.zeros(inst.n)
    D = inst.load.sum(axis=1)
    share = inst.gen_pmax / inst.gen_pmax.sum()
    for t in range(T):
        x[inst.idx_p[t]] = D[t] * share
        x[inst.idx_u[t]] = 1.0
    # angles: solve the balance rows for theta (grounded at bus 0)
    A = inst.scipy_csr().tocsr()
    bal = inst.row_balance
    import scipy.sparse.linalg as spla
    for t in range(T):
        rows = bal[t]
        th = inst.idx_theta[t]
        rhs = inst.q[rows] - A[rows] @ x
        B = A[rows][:, th[1:]]
        sol = spla.lsqr(B, rhs, atol=1e-14, btol=1e-14, iter_lim=10000)[0]
        x[th[1:]] = sol
    assert max_violation(lp, x) <= 1e-6 * np.abs(inst.q).max()


def test_invalid_params():
    with pytest.raises(ValueError):
        build_instance(0, 0, 1, 1)
    with pytest.raises(ValueError):
        build_instance(5, 3, 1, 1)  # fewer lines than the ring needs


def test_node_fixings_rules():
    """Node bounds fix 1-5% of the commitments to 0/1, only commitments, and keep
    opposite fixings of a unit at least max(min up, min down) + 1 periods apart."""
    from paper_2512_06715_gb300.instances import VAR_U, node_fixings
    inst = build_instance(12, 18, 10, 24, seed=2, with_slack=True)
    l_b, u_b = node_fixings(inst, 16, seed0=1000)
    T, G = inst.idx_u.shape
    sep = np.maximum(inst.gen_min_up, inst.gen_min_dn) + 1
    for k in range(16):
        changed = np.where((l_b[k] != inst.l) | (u_b[k] != inst.u))[0]
        assert np.all(inst.var_kind[changed] == VAR_U)
        assert 0 < changed.size <= int(round(0.05 * T * G)) + 1
        assert np.all(l_b[k][changed] == u_b[k][changed])
        for g in range(G):
            fixed = [(t, l_b[k][inst.idx_u[t, g]]) for t in range(T)
                     if l_b[k][inst.idx_u[t, g]] == u_b[k][inst.idx_u[t, g]]]
            for t1, v1 in fixed:
                for t2, v2 in fixed:
                    if v1 != v2:
                        assert abs(t1 - t2) >= sep[g]
    l2, u2 = node_fixings(inst, 16, seed0=1000)
    assert np.array_equal(l_b, l2) and np.array_equal(u_b, u2)


def test_deterministic():
    a = workload("uc24_g33_T24", seed=3)
    b = workload("uc24_g33_T24", seed=3)
    c = workload("uc24_g33_T24", seed=4)
    assert np.array_equal(a.val, b.val) and np.array_equal(a.q, b.q)
    assert not np.array_equal(a.q, c.q)


@pytest.mark.parametrize("net", ["uc4224_g600", "uc6049_g850", "uc6717_g1000"])
def test_go3_division_horizons(net):
    """The GO3 division workloads (D1: 18 steps over a day, D2: 48 over two
    days, D3: 42 over a week) build with those horizons and the network's size;
    the step length sets the minimum up/down windows and the hourly costs."""
    from paper_2512_06715_gb300.instances import GO3_DIVISIONS, workload
    sizes = {}
    for div, d in GO3_DIVISIONS.items():
        inst = workload(f"{net}_{div}")
        T = d["n_periods"]
        assert inst.n_periods == T and inst.idx_p.shape[0] == T
        assert inst.dt_hours == pytest.approx(d["horizon_hours"] / T)
        G, N = inst.n_gen, inst.n_bus
        assert inst.n == T * (4 * G + N)
        # windows in periods: ceil(h / dt) with h in 2..6 hours
        assert inst.gen_min_up.max() <= int(np.ceil(6.0 / inst.dt_hours - 1e-9))
        # p costs are hourly rates times the step length
        p0 = inst.idx_p[0]
        assert np.allclose(inst.c[p0], inst.gen_cost * inst.dt_hours)
        sizes[div] = inst.n
    assert sizes["D2"] > sizes["D3"] > sizes["D1"]
