"""Seeded synthetic DC unit-commitment instances (input generator).

Thin ctypes binding of ``uc_lp_build`` (``include/uc_lp.h``).  This module holds
no solver arithmetic: it only produces the LP data that the GPU solver and the
CPU checker both consume.  Workload presets carry the bus counts and horizons
of the paper's networks (Sec. II.B: 4224-, 6049- and 6717-bus systems).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field
from pathlib import Path

import numpy as np

_LIB = None

VAR_P, VAR_U, VAR_V, VAR_W, VAR_THETA, VAR_SHED, VAR_SPILL = range(7)
(ROW_BALANCE, ROW_LOGIC, ROW_FLOW_POS, ROW_FLOW_NEG, ROW_PMIN, ROW_PMAX, ROW_RAMP_UP,
 ROW_RAMP_DN, ROW_MIN_UP, ROW_MIN_DN) = range(10)


class _Params(C.Structure):
    _fields_ = [
        ("n_bus", C.c_int32), ("n_line", C.c_int32), ("n_gen", C.c_int32), ("n_periods", C.c_int32),
        ("seed", C.c_uint64), ("with_slack", C.c_int32), ("reserved", C.c_int32),
        ("horizon_hours", C.c_double), ("s_base", C.c_double), ("peak_frac", C.c_double),
    ]


class _LP(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("m", C.c_int64), ("m_eq", C.c_int64), ("nnz", C.c_int64),
        ("row_ptr", C.POINTER(C.c_int64)), ("col", C.POINTER(C.c_int32)), ("val", C.POINTER(C.c_double)),
        ("c", C.POINTER(C.c_double)), ("l", C.POINTER(C.c_double)), ("u", C.POINTER(C.c_double)),
        ("q", C.POINTER(C.c_double)),
        ("var_kind", C.POINTER(C.c_int32)), ("row_kind", C.POINTER(C.c_int32)),
        ("n_gen", C.c_int32), ("n_bus", C.c_int32), ("n_line", C.c_int32), ("n_periods", C.c_int32),
        ("idx_p", C.POINTER(C.c_int64)), ("idx_u", C.POINTER(C.c_int64)),
        ("idx_v", C.POINTER(C.c_int64)), ("idx_w", C.POINTER(C.c_int64)),
        ("idx_theta", C.POINTER(C.c_int64)), ("row_balance", C.POINTER(C.c_int64)),
        ("load", C.POINTER(C.c_double)), ("gen_bus", C.POINTER(C.c_int32)),
        ("line_from", C.POINTER(C.c_int32)), ("line_to", C.POINTER(C.c_int32)),
        ("gen_pmax", C.POINTER(C.c_double)), ("gen_cost", C.POINTER(C.c_double)),
        ("gen_noload", C.POINTER(C.c_double)),
        ("gen_min_up", C.POINTER(C.c_int32)), ("gen_min_dn", C.POINTER(C.c_int32)),
        ("dt_hours", C.c_double),
    ]


def _lib():
    global _LIB
    if _LIB is None:
        path = Path(__file__).resolve().parent / "lib" / "libucgen.so"
        if not path.exists():
            raise RuntimeError(f"{path} is missing: run __graft_entry__.build() first")
        lib = C.CDLL(str(path))
        lib.uc_lp_build.argtypes = [C.POINTER(_Params), C.POINTER(C.POINTER(_LP))]
        lib.uc_lp_build.restype = C.c_int
        lib.uc_lp_free.argtypes = [C.POINTER(_LP)]
        lib.uc_lp_free.restype = None
        lib.uc_lp_last_error.argtypes = []
        lib.uc_lp_last_error.restype = C.c_char_p
        _LIB = lib
    return _LIB


@dataclass
class UCInstance:
    """One DC-UC LP relaxation in PDLP form (equalities first, then >= rows)."""
    n: int
    m: int
    m_eq: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    c: np.ndarray
    l: np.ndarray
    u: np.ndarray
    q: np.ndarray
    var_kind: np.ndarray
    row_kind: np.ndarray
    n_gen: int
    n_bus: int
    n_line: int
    n_periods: int
    idx_p: np.ndarray
    idx_u: np.ndarray
    idx_v: np.ndarray
    idx_w: np.ndarray
    idx_theta: np.ndarray
    row_balance: np.ndarray
    load: np.ndarray
    gen_bus: np.ndarray
    line_from: np.ndarray
    line_to: np.ndarray
    gen_pmax: np.ndarray
    gen_cost: np.ndarray
    gen_noload: np.ndarray
    gen_min_up: np.ndarray
    gen_min_dn: np.ndarray
    dt_hours: float
    params: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def scipy_csr(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.row_ptr), shape=(self.m, self.n))


def build_instance(n_bus: int, n_line: int, n_gen: int, n_periods: int, seed: int = 0,
                   with_slack: bool = False, horizon_hours: float = 24.0, s_base: float = 100.0,
                   peak_frac: float = 0.7) -> UCInstance:
    lib = _lib()
    p = _Params(n_bus, n_line, n_gen, n_periods, seed, int(with_slack), 0, horizon_hours, s_base, peak_frac)
    out = C.POINTER(_LP)()
    rc = lib.uc_lp_build(C.byref(p), C.byref(out))
    if rc != 0:
        raise ValueError(f"uc_lp_build failed ({rc}): {lib.uc_lp_last_error().decode()}")
    try:
        lp = out.contents
        n, m, T, G, N, L = lp.n, lp.m, lp.n_periods, lp.n_gen, lp.n_bus, lp.n_line

        def arr(ptr, k, dt):
            if k == 0:
                return np.zeros(0, dtype=dt)
            return np.ctypeslib.as_array(ptr, shape=(k,)).astype(dt, copy=True)

        nnz = lp.nnz
        inst = UCInstance(
            n=n, m=m, m_eq=lp.m_eq,
            row_ptr=arr(lp.row_ptr, m + 1, np.int64), col=arr(lp.col, nnz, np.int32),
            val=arr(lp.val, nnz, np.float64), c=arr(lp.c, n, np.float64), l=arr(lp.l, n, np.float64),
            u=arr(lp.u, n, np.float64), q=arr(lp.q, m, np.float64),
            var_kind=arr(lp.var_kind, n, np.int32), row_kind=arr(lp.row_kind, m, np.int32),
            n_gen=G, n_bus=N, n_line=L, n_periods=T,
            idx_p=arr(lp.idx_p, T * G, np.int64).reshape(T, G), idx_u=arr(lp.idx_u, T * G, np.int64).reshape(T, G),
            idx_v=arr(lp.idx_v, T * G, np.int64).reshape(T, G), idx_w=arr(lp.idx_w, T * G, np.int64).reshape(T, G),
            idx_theta=arr(lp.idx_theta, T * N, np.int64).reshape(T, N),
            row_balance=arr(lp.row_balance, T * N, np.int64).reshape(T, N),
            load=arr(lp.load, T * N, np.float64).reshape(T, N),
            gen_bus=arr(lp.gen_bus, G, np.int32), line_from=arr(lp.line_from, L, np.int32),
            line_to=arr(lp.line_to, L, np.int32), gen_pmax=arr(lp.gen_pmax, G, np.float64),
            gen_cost=arr(lp.gen_cost, G, np.float64), gen_noload=arr(lp.gen_noload, G, np.float64),
            gen_min_up=arr(lp.gen_min_up, G, np.int32), gen_min_dn=arr(lp.gen_min_dn, G, np.int32),
            dt_hours=lp.dt_hours,
            params=dict(n_bus=n_bus, n_line=n_line, n_gen=n_gen, n_periods=n_periods, seed=seed,
                        with_slack=with_slack),
        )
    finally:
        lib.uc_lp_free(out)
    return inst


def node_fixings(inst: UCInstance, n_nodes: int, seed0: int = 1000, lo_frac: float = 0.01,
                 hi_frac: float = 0.05):
    """Bounds of branch-and-bound node LPs: node k fixes a random U(lo_frac, hi_frac)
    share of the commitment variables u_gt to 0 or 1 (p = 1/2) through l = u, with
    numpy's PCG64 seeded by seed0 + k.  Fixings of one generator to opposite values
    stay at least max(min up, min down) + 1 periods apart, so that with shed/spill
    slacks every node stays feasible.  Returns (l_b, u_b), each [n_nodes, n]."""
    T, G = inst.idx_u.shape
    l_b = np.repeat(inst.l[None, :], n_nodes, axis=0)
    u_b = np.repeat(inst.u[None, :], n_nodes, axis=0)
    sep = np.maximum(inst.gen_min_up, inst.gen_min_dn) + 1
    for k in range(n_nodes):
        rng = np.random.default_rng(seed0 + k)
        frac = rng.uniform(lo_frac, hi_frac)
        count = max(1, int(round(frac * T * G)))
        cells = rng.permutation(T * G)[:count]
        vals = rng.integers(0, 2, size=count)
        fixed = {}  # g -> list of (t, v)
        for cell, v in zip(cells, vals):
            t, g = divmod(int(cell), G)
            if any(v2 != v and abs(t - t2) < sep[g] for t2, v2 in fixed.get(g, [])):
                continue
            fixed.setdefault(g, []).append((t, int(v)))
            j = inst.idx_u[t, g]
            l_b[k, j] = u_b[k, j] = float(v)
    return l_b, u_b


# Workloads named by what they are (bus count, generators, horizon).
WORKLOADS = {
    # 24 buses in a ring + 14 chords, 33 generators, 24 hourly periods
    "uc24_g33_T24": dict(n_bus=24, n_line=38, n_gen=33, n_periods=24),
    # 4224-bus network, 600 generators, 48 half-hourly periods
    "uc4224_g600_T48": dict(n_bus=4224, n_line=5900, n_gen=600, n_periods=48),
    # 6717-bus network, 1000 generators, 96 quarter-hourly periods
    "uc6717_g1000_T96": dict(n_bus=6717, n_line=9200, n_gen=1000, n_periods=96),
    # 6049-bus network, 850 generators, 48 periods, with shed/spill slacks
    "uc6049_g850_T48_slack": dict(n_bus=6049, n_line=8470, n_gen=850, n_periods=48, with_slack=True),
    # 4224-bus network, 600 generators, 24 hourly periods
    "uc4224_g600_T24": dict(n_bus=4224, n_line=5900, n_gen=600, n_periods=24),
    # 200-bus network, 60 generators, 24 hourly periods, with shed/spill slacks
    "uc200_g60_T24_slack": dict(n_bus=200, n_line=300, n_gen=60, n_periods=24, with_slack=True),
}

# The horizons of the GO Challenge 3 divisions the paper solves (Sec. II.B,
# Table I): D1 a day in 18 steps, D2 two days in 48 steps, D3 a week in 42
# steps, on each of the three networks (uniform steps here: 24/18 h, 1 h, 4 h).
GO3_DIVISIONS = {"D1": dict(n_periods=18, horizon_hours=24.0),
                 "D2": dict(n_periods=48, horizon_hours=48.0),
                 "D3": dict(n_periods=42, horizon_hours=168.0)}
GO3_NETWORKS = {"uc4224_g600": dict(n_bus=4224, n_line=5900, n_gen=600),
                "uc6049_g850": dict(n_bus=6049, n_line=8470, n_gen=850),
                "uc6717_g1000": dict(n_bus=6717, n_line=9200, n_gen=1000)}
for _net, _np in GO3_NETWORKS.items():
    for _div, _dp in GO3_DIVISIONS.items():
        WORKLOADS[f"{_net}_{_div}"] = dict(**_np, **_dp)


def workload(name: str, seed: int = 0) -> UCInstance:
    return build_instance(seed=seed, **WORKLOADS[name])
