"""Python binding of the GB300 PDHG solver (``include/pdhg.h``).

Argument marshalling only: every step of the solve runs in the CUDA kernels of
``lib/libucpdhg.so``.  PyTorch supplies device memory and the CUDA stream.
There is no fallback: if the library is missing the calls raise.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from pathlib import Path

import numpy as np

PDHG_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "CUDA", -3: "NUMERIC", -4: "TIMEOUT", -5: "UNSUPPORTED", -6: "NOMEM"}
STATUS = {0: "round", 1: "optimal", 2: "iteration_limit", 3: "time_limit", 4: "cancelled", 5: "numeric",
          6: "primal_infeasible", 7: "dual_infeasible"}
PREC_FP64, PREC_MIXED = 0, 1


class pdhg_problem(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int64), ("m_eq", C.c_int64), ("nnz", C.c_int64),
                ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p),
                ("c", C.c_void_p), ("l", C.c_void_p), ("u", C.c_void_p), ("q", C.c_void_p)]


class pdhg_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("precision", C.c_int32), ("check_every", C.c_int32),
                ("max_iters", C.c_int64), ("time_limit_s", C.c_double),
                ("beta_sufficient", C.c_double), ("beta_necessary", C.c_double),
                ("beta_artificial", C.c_double), ("omega_smoothing", C.c_double),
                ("step_reduction_exp", C.c_double), ("step_growth_exp", C.c_double),
                ("ruiz_iters", C.c_int32), ("pock_chambolle", C.c_int32),
                ("ir_reduction", C.c_double),
                ("ir_max_rounds", C.c_int32), ("trace", C.c_int32),
                ("fixed_eta", C.c_double), ("fixed_omega", C.c_double),
                ("bound_obj_rescale", C.c_int32), ("artificial_total", C.c_int32),
                ("host_loop", C.c_int32), ("autotune", C.c_int32), ("cancel_flag", C.c_void_p),
                ("kernel_variant", C.c_int32), ("kernel_grid", C.c_int32), ("infeas_tol", C.c_double),
                ("ir_fold_checks", C.c_int32), ("launch_overlap", C.c_int32)]


class pdhg_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("ir_rounds", C.c_int32), ("iterations", C.c_int64),
                ("accepted", C.c_int64), ("restarts", C.c_int64), ("checks", C.c_int64),
                ("rel_p", C.c_double), ("rel_d", C.c_double), ("rel_gap", C.c_double),
                ("rel_kkt", C.c_double), ("primal_obj", C.c_double), ("dual_obj", C.c_double),
                ("solve_seconds", C.c_double), ("time_to_tol", C.c_double * 3),
                ("iters_to_tol", C.c_int64 * 3), ("eta", C.c_double), ("omega", C.c_double),
                ("kernel_launches", C.c_int64), ("returned_average", C.c_int32), ("launch_overlap", C.c_int32)]

    def to_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["time_to_tol"] = list(self.time_to_tol)
        d["iters_to_tol"] = list(self.iters_to_tol)
        d["status_name"] = STATUS.get(self.status, str(self.status))
        return d


class pdhg_polish_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("cg_iterations_primal", C.c_int32),
                ("cg_iterations_dual", C.c_int32), ("reserved", C.c_int32),
                ("active_rows", C.c_int64), ("free_vars", C.c_int64),
                ("rel_p", C.c_double), ("rel_d", C.c_double), ("rel_gap", C.c_double),
                ("rel_kkt", C.c_double), ("primal_obj", C.c_double), ("dual_obj", C.c_double),
                ("bound_violation", C.c_double), ("dual_sign_violation", C.c_double),
                ("cg_residual_primal", C.c_double), ("cg_residual_dual", C.c_double)]

    def to_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["status_name"] = POLISH_STATUS.get(self.status, str(self.status))
        return d


POLISH_STATUS = {1: "ok", 2: "not_square", 3: "no_convergence"}

# exported symbols of include/pdhg.h and their signatures
_SIGS = {
    "pdhg_opts_default": ([C.POINTER(pdhg_opts)], C.c_int),
    "pdhg_workspace_create": ([C.POINTER(pdhg_problem), C.POINTER(pdhg_opts), C.POINTER(C.c_void_p),
                               C.c_void_p], C.c_int),
    "pdhg_workspace_destroy": ([C.c_void_p], None),
    "pdhg_set_opts": ([C.c_void_p, C.POINTER(pdhg_opts)], C.c_int),
    "pdhg_solve": ([C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(pdhg_result), C.c_void_p], C.c_int),
    "pdhg_solve_batched": ([C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                            C.POINTER(pdhg_result), C.c_void_p], C.c_int),
    "pdhg_backward": ([C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "pdhg_last_error": ([], C.c_char_p),
    "pdhg_polish": ([C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(pdhg_polish_result), C.c_void_p], C.c_int),
    "pdhg_prepare": ([C.c_void_p, C.c_void_p], C.c_int),
    "pdhg_get_scaling": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "pdhg_apply_K": ([C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "pdhg_get_trace": ([C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.POINTER(C.c_int64),
                        C.POINTER(C.c_int64)], C.c_int),
    "pdhg_get_tuning": ([C.c_void_p, C.POINTER(C.c_int32)], C.c_int),
    "pdhg_rescale_noalloc": ([C.POINTER(pdhg_problem), C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                              C.c_void_p], C.c_int),
    "pdhg_time_kernels": ([C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double),
                           C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p], C.c_int),
}

_LIB = None


def lib_path() -> Path:
    return Path(__file__).resolve().parent / "lib" / "libucpdhg.so"


def lib():
    """Load libucpdhg.so (raises if it was not built: there is no fallback)."""
    global _LIB
    if _LIB is None:
        path = lib_path()
        if not path.exists():
            raise RuntimeError(f"{path} is missing: the CUDA solver must be built "
                               "(__graft_entry__.build()); there is no CPU fallback")
        L = C.CDLL(str(path))
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _LIB = L
    return _LIB


class PDHGError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != PDHG_OK:
        msg = lib().pdhg_last_error().decode()
        raise PDHGError(f"{what} failed: {ERRORS.get(rc, rc)}: {msg}")


def default_opts(**kw) -> pdhg_opts:
    o = pdhg_opts()
    _check(lib().pdhg_opts_default(C.byref(o)), "pdhg_opts_default")
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PREC_MIXED if v.lower() in ("mixed", "fp32", "f32") else PREC_FP64
        setattr(o, k, v)
    return o


def _stream_ptr(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Workspace:
    """Owns the device copy of one LP (torch tensors) and a solver workspace."""

    def __init__(self, row_ptr, col, val, c, l, u, q, m_eq: int, opts: pdhg_opts | None = None,
                 device="cuda", stream=None):
        import torch
        dev = torch.device(device)
        self.t = dict(
            row_ptr=torch.as_tensor(np.asarray(row_ptr, np.int64), device=dev),
            col=torch.as_tensor(np.asarray(col, np.int32), device=dev),
            val=torch.as_tensor(np.asarray(val, np.float64), device=dev),
            c=torch.as_tensor(np.asarray(c, np.float64), device=dev),
            l=torch.as_tensor(np.asarray(l, np.float64), device=dev),
            u=torch.as_tensor(np.asarray(u, np.float64), device=dev),
            q=torch.as_tensor(np.asarray(q, np.float64), device=dev),
        )
        self.n = int(self.t["c"].numel())
        self.m = int(self.t["q"].numel())
        self.m_eq = int(m_eq)
        self.device = dev
        self.prob = pdhg_problem(self.n, self.m, self.m_eq, int(self.t["col"].numel()),
                                 *(self.t[k].data_ptr() for k in ("row_ptr", "col", "val", "c", "l", "u", "q")))
        self.opts = opts if opts is not None else default_opts()
        self.generation = 0  # solves run on this workspace (pdhg_backward differentiates the last)
        self.ws = C.c_void_p()
        with torch.cuda.device(dev):
            _check(lib().pdhg_workspace_create(C.byref(self.prob), C.byref(self.opts), C.byref(self.ws),
                                               _stream_ptr(stream)), "pdhg_workspace_create")

    @classmethod
    def from_instance(cls, inst, opts=None, device="cuda", stream=None):
        return cls(inst.row_ptr, inst.col, inst.val, inst.c, inst.l, inst.u, inst.q, inst.m_eq, opts,
                   device, stream)

    def close(self):
        if self.ws:
            lib().pdhg_workspace_destroy(self.ws)
            self.ws = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_opts(self, **kw):
        for k, v in kw.items():
            if k == "precision" and isinstance(v, str):
                v = PREC_MIXED if v.lower() in ("mixed", "fp32", "f32") else PREC_FP64
            setattr(self.opts, k, v)
        _check(lib().pdhg_set_opts(self.ws, C.byref(self.opts)), "pdhg_set_opts")

    def solve(self, stream=None, x_out=None, y_out=None):
        """Returns (x, y, result dict); x, y are FP64 torch tensors on the device."""
        import torch
        x = x_out if x_out is not None else torch.empty(self.n, dtype=torch.float64, device=self.device)
        y = y_out if y_out is not None else torch.empty(self.m, dtype=torch.float64, device=self.device)
        r = pdhg_result()
        self.generation += 1
        _check(lib().pdhg_solve(self.ws, x.data_ptr(), y.data_ptr(), C.byref(r), _stream_ptr(stream)),
               "pdhg_solve")
        return x, y, r.to_dict()

    def solve_batched(self, l_b, u_b, stream=None, want_y=True):
        """B node LPs sharing K, c, q with bounds l_b, u_b [B, n] (original order).
        Returns (x [B, n], y [B, m] or None, list of result dicts)."""
        import torch
        l_b = torch.as_tensor(l_b, dtype=torch.float64, device=self.device).contiguous()
        u_b = torch.as_tensor(u_b, dtype=torch.float64, device=self.device).contiguous()
        B = int(l_b.shape[0])
        x = torch.empty((B, self.n), dtype=torch.float64, device=self.device)
        y = torch.empty((B, self.m), dtype=torch.float64, device=self.device) if want_y else None
        res = (pdhg_result * B)()
        self.generation += 1
        _check(lib().pdhg_solve_batched(self.ws, B, l_b.data_ptr(), u_b.data_ptr(), x.data_ptr(),
                                        y.data_ptr() if y is not None else None, res, _stream_ptr(stream)),
               "pdhg_solve_batched")
        return x, y, [r.to_dict() for r in res]

    def polish(self, stream=None):
        """Active-set polish of the last solve (pdhg_polish).  Returns (x, y,
        result dict); x, y are None unless the active set was square."""
        import torch
        x = torch.empty(self.n, dtype=torch.float64, device=self.device)
        y = torch.empty(self.m, dtype=torch.float64, device=self.device)
        r = pdhg_polish_result()
        _check(lib().pdhg_polish(self.ws, x.data_ptr(), y.data_ptr(), C.byref(r), _stream_ptr(stream)),
               "pdhg_polish")
        d = r.to_dict()
        if d["status_name"] == "not_square":
            return None, None, d
        return x, y, d

    def prepare(self, stream=None):
        _check(lib().pdhg_prepare(self.ws, _stream_ptr(stream)), "pdhg_prepare")

    def scaling(self, stream=None):
        import torch
        Dr = torch.empty(self.m, dtype=torch.float64, device=self.device)
        Dc = torch.empty(self.n, dtype=torch.float64, device=self.device)
        _check(lib().pdhg_get_scaling(self.ws, Dr.data_ptr(), Dc.data_ptr(), _stream_ptr(stream)),
               "pdhg_get_scaling")
        return Dr, Dc

    def apply_K(self, v, transpose=False, precision=PREC_FP64, stream=None):
        import torch
        v = v.to(device=self.device, dtype=torch.float64).contiguous()
        out = torch.empty(self.n if transpose else self.m, dtype=torch.float64, device=self.device)
        _check(lib().pdhg_apply_K(self.ws, int(bool(transpose)), precision, v.data_ptr(), out.data_ptr(),
                                  _stream_ptr(stream)), "pdhg_apply_K")
        return out

    def trace(self, cap_a=1 << 16, cap_c=1 << 17):
        a = np.zeros((cap_a, 5))
        c = np.zeros((cap_c, 12))
        na, nc = C.c_int64(), C.c_int64()
        _check(lib().pdhg_get_trace(self.ws, a.ctypes.data, cap_a, c.ctypes.data, cap_c, C.byref(na),
                                    C.byref(nc)), "pdhg_get_trace")
        return a[: min(na.value, cap_a)], c[: min(nc.value, cap_c)]

    def tuning(self):
        cfg = (C.c_int32 * 12)()
        _check(lib().pdhg_get_tuning(self.ws, cfg), "pdhg_get_tuning")
        names = ("unroll_dual", "grid_dual", "unroll_adj", "grid_adj")
        bnames = ("rows_per_warp_dual", "grid_dual", "rows_per_warp_adj", "grid_adj")
        return {"fp64": dict(zip(names, cfg[0:4])), "fp32": dict(zip(names, cfg[4:8])),
                "batched": dict(zip(bnames, cfg[8:12]))}

    def time_kernels(self, precision=PREC_FP64, reps=20, stream=None):
        md, ma, bd, ba = C.c_double(), C.c_double(), C.c_double(), C.c_double()
        _check(lib().pdhg_time_kernels(self.ws, precision, reps, C.byref(md), C.byref(ma), C.byref(bd),
                                       C.byref(ba), _stream_ptr(stream)), "pdhg_time_kernels")
        return dict(ms_dual=md.value, ms_adj=ma.value, bytes_dual=bd.value, bytes_adj=ba.value)


def header_symbols() -> list[str]:
    """Function names declared in include/pdhg.h."""
    import re
    text = (Path(__file__).resolve().parent.parent / "include" / "pdhg.h").read_text()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(pdhg_\w+)\s*\(", text, re.M)))
