"""The generated rows and costs follow the DC unit-commitment formulation the
instances stand in for (host only): costs, generation limits, commitment logic,
ramping with start-up/shut-down ramp max(Pmin, R), minimum up/down windows
truncated at the second period, balance right-hand sides and the load profile."""
import numpy as np
import pytest

from paper_2512_06715_gb300.instances import (ROW_BALANCE, ROW_LOGIC, ROW_MIN_DN, ROW_MIN_UP, ROW_PMAX,
                                              ROW_PMIN, ROW_RAMP_DN, ROW_RAMP_UP, build_instance)


@pytest.fixture(scope="module")
def inst():
    return build_instance(12, 18, 10, 24, seed=5)


def _rows(inst, kind):
    A = inst.scipy_csr().tocsr()
    return A, np.where(inst.row_kind == kind)[0]


def _row_dict(A, i):
    s, e = A.indptr[i], A.indptr[i + 1]
    return dict(zip(A.indices[s:e].tolist(), A.data[s:e].tolist()))


def _find(A, rows, must):
    """The rows of `rows` whose support contains every variable of `must`."""
    return [i for i in rows if all(v in _row_dict(A, i) for v in must)]


def test_costs_scale_with_period_length(inst):
    T, G = inst.idx_p.shape
    dt = inst.dt_hours
    assert dt == pytest.approx(24.0 / T)
    for t in range(T):
        assert np.allclose(inst.c[inst.idx_p[t]], inst.gen_cost * dt)
        assert np.allclose(inst.c[inst.idx_u[t]], inst.gen_noload * dt)


def test_generation_limits(inst):
    A, rows_min = _rows(inst, ROW_PMIN)
    _, rows_max = _rows(inst, ROW_PMAX)
    T, G = inst.idx_p.shape
    for t in (0, T // 2, T - 1):
        for g in range(G):
            p, u = inst.idx_p[t, g], inst.idx_u[t, g]
            (i,) = _find(A, rows_min, (p, u))
            d = _row_dict(A, i)
            assert d[p] == 1.0 and d[u] == pytest.approx(-0.3 * inst.gen_pmax[g]) and inst.q[i] == 0.0
            (i,) = _find(A, rows_max, (p, u))
            d = _row_dict(A, i)
            assert d[p] == -1.0 and d[u] == pytest.approx(inst.gen_pmax[g]) and inst.q[i] == 0.0
            assert inst.u[p] == pytest.approx(inst.gen_pmax[g]) and inst.l[p] == 0.0


def test_commitment_logic_and_first_period(inst):
    A, rows = _rows(inst, ROW_LOGIC)
    T, G = inst.idx_p.shape
    assert len(rows) == G * (T - 1)
    for g in range(G):
        # no initial state: start-up and shut-down are fixed to 0 in the first period
        assert inst.u[inst.idx_v[0, g]] == 0.0 and inst.u[inst.idx_w[0, g]] == 0.0
        for t in (1, T - 1):
            u, u0, v, w = inst.idx_u[t, g], inst.idx_u[t - 1, g], inst.idx_v[t, g], inst.idx_w[t, g]
            (i,) = _find(A, rows, (u, u0, v, w))
            assert _row_dict(A, i) == {u: 1.0, u0: -1.0, v: -1.0, w: 1.0} and inst.q[i] == 0.0


def test_ramping_rows(inst):
    A, up = _rows(inst, ROW_RAMP_UP)
    _, dn = _rows(inst, ROW_RAMP_DN)
    T, G = inst.idx_p.shape
    R = 0.5 * inst.gen_pmax * inst.dt_hours
    SR = np.maximum(0.3 * inst.gen_pmax, R)
    for g in range(G):
        for t in (1, T - 1):
            p, p0 = inst.idx_p[t, g], inst.idx_p[t - 1, g]
            (i,) = _find(A, up, (p, p0, inst.idx_v[t, g]))
            d = _row_dict(A, i)
            assert d[p0] == 1.0 and d[p] == -1.0
            assert d[inst.idx_u[t - 1, g]] == pytest.approx(R[g]) and d[inst.idx_v[t, g]] == pytest.approx(SR[g])
            (i,) = _find(A, dn, (p, p0, inst.idx_w[t, g]))
            d = _row_dict(A, i)
            assert d[p] == 1.0 and d[p0] == -1.0
            assert d[inst.idx_u[t, g]] == pytest.approx(R[g]) and d[inst.idx_w[t, g]] == pytest.approx(SR[g])


@pytest.mark.parametrize("kind", [ROW_MIN_UP, ROW_MIN_DN])
def test_minimum_up_down_windows(inst, kind):
    A, rows = _rows(inst, kind)
    T, G = inst.idx_p.shape
    sw = inst.idx_v if kind == ROW_MIN_UP else inst.idx_w
    win = inst.gen_min_up if kind == ROW_MIN_UP else inst.gen_min_dn
    for g in range(G):
        for t in range(1, T):
            u = inst.idx_u[t, g]
            cand = [i for i in _find(A, rows, (u, sw[t, g])) if len(_row_dict(A, i)) > 1]
            assert len(cand) == 1
            d = _row_dict(A, cand[0])
            # window tau = max(2, t - W + 1) .. t in 1-based periods
            lo = max(1, t - int(win[g]) + 1)
            expect = {int(sw[tau, g]): -1.0 for tau in range(lo, t + 1)}
            expect[int(u)] = 1.0 if kind == ROW_MIN_UP else -1.0
            assert d == pytest.approx(expect)
            assert inst.q[cand[0]] == (0.0 if kind == ROW_MIN_UP else -1.0)


def test_balance_rhs_and_load_profile(inst):
    T, N = inst.row_balance.shape
    assert np.allclose(inst.q[inst.row_balance], inst.load)
    D = inst.load.sum(axis=1)
    h = (np.arange(T) + 0.5) * inst.dt_hours
    s = 0.6 + 0.25 * np.exp(-(h - 9.0) ** 2 / 4.5) + 0.4 * np.exp(-(h - 19.0) ** 2 / 8.0)
    assert np.allclose(D, 0.7 * inst.gen_pmax.sum() * s / s.max(), rtol=1e-12)
    # the bus shares are fixed over the day
    w = inst.load / D[:, None]
    assert np.allclose(w, w[0][None, :], rtol=1e-12)
