"""torch.autograd interface: optimal cost and dispatch of the DC-UC relaxation
as differentiable functions of the load d [T, N] and the cost vector c [n].

Forward runs pdhg_solve with the load written into the balance rows of the
right-hand side; backward runs pdhg_backward (implicit differentiation of the
KKT system on the detected active set), so the gradient with respect to d is
the balance-row part of the gradient with respect to the right-hand side.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import pdhg


def _make_fn():
    import torch

    class Fn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, d, c, relax):
            ws = relax.ws
            ws.t["q"].index_copy_(0, relax.bal, d.detach().reshape(-1).to(torch.float64))
            ws.t["c"].copy_(c.detach().to(torch.float64))
            x, y, r = ws.solve()
            if r["status_name"] != "optimal":
                raise pdhg.PDHGError(f"UCRelax forward: solver status {r['status_name']}")
            ctx.relax = relax
            ctx.d_shape = d.shape
            # pdhg_backward differentiates the workspace's last solve: remember which
            ctx.generation = ws.generation
            # the optimal cost c^T x* as the library evaluated it in FP64
            cost = torch.tensor(r["primal_obj"], dtype=torch.float64, device=ws.device)
            p = x.index_select(0, relax.idx_p).reshape(relax.T, relax.G)
            return cost, p

        @staticmethod
        def backward(ctx, g_cost, g_p):
            relax = ctx.relax
            ws = relax.ws
            if ws.generation != ctx.generation:
                raise pdhg.PDHGError(
                    "UCRelax backward: the workspace was solved again after this forward; "
                    "run backward before the next forward on the same UCRelax")
            gq = torch.empty(ws.m, dtype=torch.float64, device=ws.device)
            gc = torch.empty(ws.n, dtype=torch.float64, device=ws.device)
            gx_ptr = None
            if g_p is not None and bool(torch.count_nonzero(g_p)):
                gx = torch.zeros(ws.n, dtype=torch.float64, device=ws.device)
                gx.index_copy_(0, relax.idx_p, g_p.reshape(-1).to(torch.float64))
                gx_ptr = gx.data_ptr()
            gcost = float(g_cost) if g_cost is not None else 0.0
            rc = pdhg.lib().pdhg_backward(ws.ws, gcost, gx_ptr, gq.data_ptr(), gc.data_ptr(),
                                          torch.cuda.current_stream(ws.device).cuda_stream)
            pdhg._check(rc, "pdhg_backward")
            grad_d = gq.index_select(0, relax.bal).reshape(ctx.d_shape)
            return grad_d, gc, None

    return Fn


class UCRelax:
    """Callable (d, c) -> (cost, p) with gradients through the GPU solver."""

    def __init__(self, inst, q=None, c=None, l=None, u=None, tol: float = 1e-8,
                 precision: str = "fp64", device="cuda", time_limit_s: float = 600.0):
        import torch
        self.inst = inst
        q0 = inst.q if q is None else np.asarray(q, np.float64)
        c0 = inst.c if c is None else np.asarray(c, np.float64)
        l0 = inst.l if l is None else np.asarray(l, np.float64)
        u0 = inst.u if u is None else np.asarray(u, np.float64)
        self.ws = pdhg.Workspace(inst.row_ptr, inst.col, inst.val, c0, l0, u0, q0, inst.m_eq,
                                 pdhg.default_opts(precision=precision, tol=tol, time_limit_s=time_limit_s),
                                 device=device)
        self.bal = torch.as_tensor(inst.row_balance.reshape(-1), device=self.ws.device)
        self.idx_p = torch.as_tensor(inst.idx_p.reshape(-1), device=self.ws.device)
        self.T, self.G = inst.idx_p.shape
        self._fn = _make_fn()

    def __call__(self, d, c):
        return self._fn.apply(d, c, self)

    def close(self):
        self.ws.close()
