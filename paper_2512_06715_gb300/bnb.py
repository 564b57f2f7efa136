"""Branch-and-bound over batched PDHG node relaxations.

The paper uses the PDHG relaxation of the UC MILP for the bounds of a
branch-and-bound (Sec. II.D, Sec. III.B).  This driver does that with the
library's calls only: every node LP -- the relaxation with some commitments
u_gt fixed to 0 or 1 through l = u -- is solved on the GPU by
pdhg_solve_batched, up to 64 nodes per call; the host keeps the tree.

* bound of a node: min(primal, dual objective) of its solve (the two agree to
  the solve tolerance); a node whose bound is within the relative gap of the
  incumbent is pruned, so is a node with a primal-infeasibility certificate
  (PDHG_STATUS_PRIMAL_INFEASIBLE: node LPs without slacks can be infeasible);
* best-first: each call takes the open nodes of lowest bound;
* branching on the most fractional commitment, children u = 0 and u = 1;
* incumbents: a node whose commitments come out integral (within int_tol),
  and the rounding heuristic at every solved node (every fractional u rounded
  up, the LP with all commitments fixed solved in the same batch machinery);
* a node the batched FP32 solve leaves unresolved (attempt or time limit: the
  FP32 rays of some infeasible nodes never certify) is solved again alone in
  FP64 by pdhg_solve with the node's bounds; if that also ends unresolved the
  driver raises rather than guess.
The tree, the queue and the decisions are host logic; no method arithmetic runs
here beyond comparing the objectives the library returns.
"""
from __future__ import annotations

import heapq
from dataclasses import dataclass, field

import numpy as np


@dataclass(order=True)
class _Node:
    bound: float
    seq: int
    fix: dict = field(compare=False)  # variable index -> 0.0 / 1.0
    depth: int = field(compare=False, default=0)


@dataclass
class BnBResult:
    status: str               # "optimal" (gap closed), "node_limit", "infeasible"
    incumbent: float          # best integral objective found (inf if none)
    bound: float              # best remaining lower bound
    schedule: np.ndarray | None  # u of the incumbent, [T, G]
    nodes: int                # node LPs solved
    batches: int              # pdhg_solve_batched calls
    pruned_infeasible: int
    pruned_bound: int
    log: list = field(default_factory=list)


def _solve_alone_fp64(ws, l, u, max_iters):
    """One node LP in FP64 (pdhg_solve) on the workspace's own bounds, which are
    restored afterwards; returns (x, result dict)."""
    import torch
    keep = {k: ws.t[k].clone() for k in ("l", "u")}
    saved = {k: getattr(ws.opts, k) for k in ("precision", "max_iters")}
    try:
        ws.t["l"].copy_(torch.as_tensor(l, device=ws.device))
        ws.t["u"].copy_(torch.as_tensor(u, device=ws.device))
        ws.set_opts(precision="fp64", max_iters=max_iters)
        x, _, r = ws.solve()
        return x.cpu().numpy(), r
    finally:
        for k, v in keep.items():
            ws.t[k].copy_(v)
        ws.set_opts(**saved)


def branch_and_bound(ws, idx_u: np.ndarray, l0: np.ndarray, u0: np.ndarray, batch: int = 64,
                     max_nodes: int = 2000, gap: float = 1e-6, int_tol: float = 1e-6,
                     fp64_retry_iters: int = 10_000_000, device=None) -> BnBResult:
    """B&B on the UC MILP whose relaxation `ws` (a pdhg.Workspace whose options
    -- tolerance, attempt and time limits of each batched call -- the caller
    sets) holds; idx_u [T, G] are the commitment variables, l0, u0 the
    relaxation's bounds (original order)."""
    import torch

    dev = device if device is not None else ws.device
    flat_u = np.asarray(idx_u).reshape(-1)
    incumbent, sched = np.inf, None
    pruned_inf = pruned_bound = 0
    seq = 0
    open_nodes: list[_Node] = [_Node(-np.inf, seq, {}, 0)]
    solved = batches = retried = 0
    log = []

    def bounds_of(fix: dict):
        l, u = l0.copy(), u0.copy()
        for j, v in fix.items():
            l[j] = u[j] = v
        return l, u

    while open_nodes and solved < max_nodes:
        # best-first: the open nodes of lowest bound that can still improve
        take = []
        while open_nodes and len(take) < batch:
            nd = heapq.heappop(open_nodes)
            if nd.bound >= incumbent - gap * max(1.0, abs(incumbent)):
                pruned_bound += 1
                continue
            take.append(nd)
        if not take:
            break
        # the rounding heuristic rides in the same call: one rounded child per node
        ls, us, kinds = [], [], []
        for nd in take:
            l, u = bounds_of(nd.fix)
            ls.append(l)
            us.append(u)
            kinds.append(("node", nd))
        l_b = torch.as_tensor(np.stack(ls), device=dev)
        u_b = torch.as_tensor(np.stack(us), device=dev)
        x_b, _, res = ws.solve_batched(l_b, u_b, want_y=False)
        batches += 1
        solved += len(take)
        x_b = x_b.cpu().numpy()
        rounded = []
        for k, (kind, nd) in enumerate(kinds):
            r = res[k]
            if r["status_name"] in ("iteration_limit", "time_limit"):
                xk, r = _solve_alone_fp64(ws, ls[k], us[k], fp64_retry_iters)
                x_b[k] = xk
                retried += 1
            if r["status_name"] == "primal_infeasible":
                pruned_inf += 1
                continue
            if r["status_name"] != "optimal":
                raise RuntimeError(f"node LP ended with status {r['status_name']} (rel-KKT {r['rel_kkt']:.2e})")
            bound = min(r["primal_obj"], r["dual_obj"])
            if bound >= incumbent - gap * max(1.0, abs(incumbent)):
                pruned_bound += 1
                continue
            uval = x_b[k, flat_u]
            frac = np.abs(uval - np.round(uval))
            if frac.max() <= int_tol:
                if r["primal_obj"] < incumbent:
                    incumbent = r["primal_obj"]
                    sched = np.round(uval).reshape(idx_u.shape)
                continue
            j = int(flat_u[np.argmax(frac)])
            for v in (0.0, 1.0):
                seq += 1
                fix = dict(nd.fix)
                fix[j] = v
                heapq.heappush(open_nodes, _Node(bound, seq, fix, nd.depth + 1))
            rounded.append({**nd.fix, **{int(jj): float(np.ceil(uu - int_tol)) for jj, uu in zip(flat_u, uval)}})
        # rounding heuristic: all commitments fixed at the rounded-up values
        if rounded:
            ls, us = zip(*(bounds_of(f) for f in rounded))
            _, _, rr = ws.solve_batched(torch.as_tensor(np.stack(ls), device=dev),
                                        torch.as_tensor(np.stack(us), device=dev), want_y=False)
            batches += 1
            for f, r in zip(rounded, rr):
                if r["status_name"] == "optimal" and r["primal_obj"] < incumbent:
                    incumbent = r["primal_obj"]
                    sched = np.array([f[int(j)] for j in flat_u]).reshape(idx_u.shape)
        best_open = min((nd.bound for nd in open_nodes), default=np.inf)
        log.append({"batch": batches, "solved": solved, "open": len(open_nodes), "incumbent": incumbent,
                    "bound": best_open, "fp64_retries": retried})
    best_open = min((nd.bound for nd in open_nodes
                     if nd.bound < incumbent - gap * max(1.0, abs(incumbent))), default=np.inf)
    bound = min(best_open, incumbent)
    if not open_nodes or best_open == np.inf:
        status = "optimal" if np.isfinite(incumbent) else "infeasible"
    else:
        status = "node_limit"
    return BnBResult(status, float(incumbent), float(bound), sched, solved, batches, pruned_inf, pruned_bound,
                     log)
