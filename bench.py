#!/usr/bin/env python
"""Benchmark of the GB300 PDHG hot path on a synthetic DC unit-commitment relaxation.

One JSON line on stdout (rank 0).  Headline: effective SpMV HBM GB/s of the
mixed-precision (FP32 iterates, FP64 KKT/refinement) PDHG on the 6717-bus,
96-period relaxation -- the algorithmic bytes of the two fused SpMV kernels
(K x' + dual step, K^T y' + primal step) of every step attempt, divided by the
device time of whole solver calls.  A step is one pdhg_solve call from a cold
start capped at --attempts step attempts: Ruiz + Pock-Chambolle rescaling, the
FP32 copies, PDHG attempts, an FP64 KKT check with restart/primal-weight logic
every 64 attempts and the output.  The same step in plain FP64, the
time-to-tolerance of both precisions (capped), the dominant kernel's roofline,
an end-to-end run through host buffers and the CPU oracle are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) each rank solves its own replica (the LP does not shard:
replicas only) and rank 0 reports the whole-job aggregate.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import threading
import time
from pathlib import Path

# The CPU oracle leg reports "cores": 1; keep NumPy's BLAS (vector norms) on one
# thread so that the figure is what ran.  Set before NumPy loads its BLAS.
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "SpMV HBM GB/s (mixed-precision PDHG; time to rel-KKT 1e-8 and node LPs/s reported beside)"
DEFAULT_WORKLOAD = "uc6717_g1000_T96"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=DEFAULT_WORKLOAD)
    p.add_argument("--attempts", type=int, default=4096, help="step attempts per solver call")
    p.add_argument("--ttt-limit", type=float, default=300.0,
                   help="seconds cap of the mixed-precision time-to-tolerance solve (0 = skip)")
    p.add_argument("--ttt-limit-fp64", type=float, default=360.0,
                   help="seconds cap of the FP64 time-to-tolerance solve")
    p.add_argument("--ttt-small", default="uc24_g33_T24",
                   help="workload solved to rel-KKT 1e-8 in both precisions beside the capped large solves")
    p.add_argument("--ttt-trace", default="",
                   help="directory: record the per-check trace of the capped time-to-tolerance solves "
                        "there (numpy arrays and a markdown summary)")
    p.add_argument("--ttt-opt", action="append", default=[],
                   help="extra solver option name=value for the time-to-tolerance solves (repeatable)")
    p.add_argument("--cpu-ttt-limit", type=float, default=60.0,
                   help="seconds cap of each CPU oracle time-to-tolerance solve (0 = skip)")
    p.add_argument("--cpu-attempts", type=int, default=64, help="oracle attempts of the CPU sample")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--kernel-variant", type=int, default=-1,
                   help="force a per-attempt kernel variant (0 pipelined, 1, 2, 4) for profiling")
    p.add_argument("--kernel-grid", type=int, default=0, help="force the per-attempt kernels' grid")
    p.add_argument("--nodes-workload", default="uc6049_g850_T48_slack",
                   help="shared LP of the batched node relaxations")
    p.add_argument("--nodes", type=int, default=64, help="node LPs of the batched measurement")
    p.add_argument("--nodes-attempts", type=int, default=640,
                   help="attempts per node of the batched-vs-sequential node throughput (0: skip)")
    p.add_argument("--nodes-tol", type=float, default=0.0,
                   help="> 0: solve every node to this rel-KKT instead (converged node LPs/s)")
    p.add_argument("--nodes-cap", type=float, default=600.0, help="seconds cap of the converged node solves")
    p.add_argument("--nodes-seq", type=int, default=2,
                   help="nodes solved one at a time for the sequential comparison")
    p.add_argument("--nodes-conv-workload", default="uc200_g60_T24_slack",
                   help="node LPs solved to --nodes-conv-tol (converged node LPs/s)")
    p.add_argument("--nodes-conv-tol", type=float, default=1e-4, help="0: skip the converged node measurement")
    p.add_argument("--nodes-rows-per-warp", type=int, default=-1, choices=[-1, 1, 2, 4],
                   help="with --no-autotune: rows (columns) per warp of the batched sweeps")
    p.add_argument("--nodes-grid", type=int, default=0,
                   help="with --no-autotune: blocks of the batched sweeps (0: default)")
    p.add_argument("--host-loop", action="store_true",
                   help="launch the per-check bodies from the host instead of one CUDA graph "
                        "(same kernels; profilers cannot see kernels inside conditional graphs)")
    p.add_argument("--launch-overlap", action="store_true",
                   help="programmatic dependent launch of the per-attempt kernels (default: plain launches)")
    p.add_argument("--no-autotune", action="store_true",
                   help="default launch shapes instead of timing the variants (profiler replays "
                        "distort those timings)")
    return p.parse_args()


# --------------------------------------------------------------------------- helpers
def algorithmic_bytes(n, m, nnz, elt):
    """Per attempt, CSR-equivalent: matrix stream (value + int32 column + int32 row
    pointer) of K and K^T, each gathered vector once, each streamed vector once.
    FP32 gathers x and x' (K x recomputed) and streams y_lo; FP64 gathers x' and
    streams the stored K x in and K x' out."""
    if elt == 4:
        dual = nnz * (elt + 4) + 4 * m + 2 * elt * n + elt * m * 6
    else:
        dual = nnz * (elt + 4) + 4 * m + elt * n + elt * m * 7
    adj = nnz * (elt + 4) + 4 * n + elt * m + elt * n * 8
    return dual, adj


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [s.strip() for s in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dual_kernel_name(variant: int) -> str:
    """Template name of the FP32 K x' kernel a tuning variant launches (the
    second template argument of the sliced-ELL forms is the number of resident
    blocks per SM they are compiled for)."""
    return {0: "k_dual_pipe<float, 5>", 1: "k_dual<float, 1, 6>", 2: "k_dual<float, 2, 4>",
            4: "k_dual<float, 4, 4>", 8: "k_dual<float, 1, 8>", 9: "k_dual_pipe<float, 8>",
            16: "k_dual_staged<float, 1>", 17: "k_dual_staged<float, 2>",
            18: "k_dual_rs<float, 1>", 19: "k_dual_rs<float, 2>",
            20: "k_dual_ring<float, 3>", 21: "k_dual_ring<float, 4>"}.get(variant, f"variant {variant}")


def dual_kernel_source(variant: int) -> Path:
    """Source file that holds the K x' kernel of a tuning variant."""
    csrc = ROOT / "paper_2512_06715_gb300" / "csrc"
    if variant in (16, 17):
        return csrc / "pdhg_staged.cu"
    if variant in (18, 19):
        return csrc / "pdhg_rowstaged.cu"
    if variant in (20, 21):
        return csrc / "pdhg_ring.cu"
    return csrc / "pdhg_kernels.cu"


def measured_peaks() -> dict:
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def dram_traffic_record(kernel_src: Path, kernel: str):
    """Per-launch DRAM bytes of the dominant kernel from the committed ncu summary,
    valid only for the same kernel variant and while its source is unchanged
    since the capture."""
    rec = ROOT / "profiles" / "dram_traffic.json"
    if not rec.exists():
        return None
    h = hashlib.sha256(kernel_src.read_bytes()).hexdigest()[:16]
    recs = json.loads(rec.read_text())
    for d in recs if isinstance(recs, list) else [recs]:
        if isinstance(d, dict) and d.get("kernel_source_sha256_16") == h and d.get("kernel") == kernel:
            return d
    return None


# --------------------------------------------------------------------------- CPU oracle leg
def cpu_oracle_gbs(inst, attempts: int):
    """The FP64 CPU oracle timed on the host cores on a bounded sample: one
    oracle solve (rescaling included) capped at `attempts` step attempts."""
    from oracle.lp import lp_from_arrays
    from oracle.pdhg import pdhg_solve
    lp = lp_from_arrays(inst.row_ptr, inst.col, inst.val, inst.q, inst.c, inst.l, inst.u, inst.m_eq)
    t0 = time.perf_counter()
    pdhg_solve(lp, tol=1e-30, stop_after=attempts)
    dt = time.perf_counter() - t0
    d, a = algorithmic_bytes(inst.n, inst.m, inst.nnz, 8)
    gbs = attempts * (d + a) / dt / 1e9
    return gbs, dt


def write_trace(out_dir: Path, tag: str, checks, r: dict, extra: dict):
    """Per-check trace of a solve: the array (columns as pdhg_get_trace documents)
    and a markdown table of about 40 evenly spaced checks plus every restart."""
    out_dir.mkdir(parents=True, exist_ok=True)
    np.save(out_dir / f"trace_{tag}.npy", checks)
    lines = [f"# Per-check trace: {tag}", "", "Command (GB300, one GPU):", "```",
             "python " + " ".join(sys.argv), "```", "",
             f"Options beyond the defaults: {extra or 'none'}.  Final status {r['status_name']}, "
             f"rel-KKT {r['rel_kkt']:.3e}, {r['iterations']} attempts, {r['restarts']} restarts, "
             f"{r['ir_rounds']} refinement rounds, primal weight {r['omega']:.4g}; seconds to 1e-4/1e-6/1e-8: "
             f"{[round(t, 2) for t in r['time_to_tol']]}.", "",
             "rel_p, rel_d and rel_gap are those of the current iterate; the solver returns the better of the "
             "current and the average candidate.", "",
             "| attempts | restart (to avg) | omega after | rel-KKT current / average | rel_p | rel_d | rel_gap |",
             "|---|---|---|---|---|---|---|"]
    if len(checks):
        idx = sorted(set(np.linspace(0, len(checks) - 1, 40).round().astype(int).tolist()) |
                     set(np.where(checks[:, 1] > 0)[0].tolist()))
        for i in idx:
            c = checks[i]
            rs = ("yes (avg)" if c[2] else "yes") if c[1] else ""
            lines.append(f"| {int(c[0])} | {rs} | {c[3]:.4g} | {c[6]:.2e} / {c[7]:.2e} | {c[8]:.2e} | "
                         f"{c[9]:.2e} | {c[10]:.2e} |")
    (out_dir / f"trace_{tag}.md").write_text("\n".join(lines) + "\n")


def cpu_oracle_ttt(names, cap_s: float) -> dict:
    """The CPU oracle's own time to rel-KKT 1e-4 / 1e-6 / 1e-8 (one core, capped):
    seconds and attempts when each level was first reached at a check, -1 if not
    within the cap."""
    from oracle.lp import lp_from_arrays
    from oracle.pdhg import pdhg_solve
    from paper_2512_06715_gb300.instances import workload
    out = {}
    for name in names:
        inst = workload(name)
        lp = lp_from_arrays(inst.row_ptr, inst.col, inst.val, inst.q, inst.c, inst.l, inst.u, inst.m_eq)
        t0 = time.perf_counter()
        stamps = {}

        def on_check(k, rel):
            now = time.perf_counter() - t0
            for t in (1e-4, 1e-6, 1e-8):
                if rel <= t and t not in stamps:
                    stamps[t] = (now, k)
            return now >= cap_s

        res = pdhg_solve(lp, tol=1e-8, max_attempts=10**9, on_check=on_check)
        out[name] = {"cores": 1, "cap_s": cap_s, "status": res.status, "rel_kkt": res.rel_kkt,
                     "attempts": res.attempts, "seconds": time.perf_counter() - t0,
                     "seconds_to_1e-4_1e-6_1e-8": [stamps.get(t, (-1.0, -1))[0] for t in (1e-4, 1e-6, 1e-8)],
                     "attempts_to_1e-4_1e-6_1e-8": [stamps.get(t, (-1.0, -1))[1] for t in (1e-4, 1e-6, 1e-8)]}
    return out


def cpu_recheck(returned: dict, insts: dict) -> dict:
    """The oracle's rel-KKT and objective of each point the GPU returned in the
    time-to-tolerance solves (the library's reported values beside them)."""
    from oracle.lp import kkt, lp_from_arrays
    from paper_2512_06715_gb300.instances import workload
    out = {}
    for key, (x, y, r) in returned.items():
        name = key.split("@")[1] if "@" in key else next(iter(insts))
        inst = insts.get(name) or workload(name)
        lp = lp_from_arrays(inst.row_ptr, inst.col, inst.val, inst.q, inst.c, inst.l, inst.u, inst.m_eq)
        k = kkt(lp, x, y)
        out[key] = {"oracle_rel_kkt": k.rel_kkt, "oracle_primal_obj": k.primal_obj,
                    "reported_rel_kkt": r["rel_kkt"], "reported_primal_obj": r["primal_obj"]}
    return out


# --------------------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2512_06715_gb300.instances import workload
    inst = workload(args.workload)
    steps = []
    for i in range(args.warmup + args.steps):
        gbs, dt = cpu_oracle_gbs(inst, args.cpu_attempts)
        if i >= args.warmup:
            steps.append((gbs, dt))
    value = float(np.mean([g for g, _ in steps]))
    ms = float(np.mean([d for _, d in steps]) * 1e3)
    sample = f"{args.cpu_attempts} oracle attempts (rescaling included) per step on {args.workload}"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n": inst.n, "m": inst.m, "nnz": inst.nnz},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- our arm
def max_over_ranks(value: float, device) -> float:
    """The slowest rank's value (replicas: the job ends when the last one does)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def node_partition(B: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous block [start, stop) of the B node LPs that `rank` solves; the
    blocks of all ranks cover 0..B-1 once and differ in size by at most one.
    Node LPs are independent, so the partition needs no data exchange."""
    base, extra = divmod(B, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def gather_node_results(local: list, start: int, world: int) -> list:
    """Every rank's per-node results, in node order, on every rank (host objects
    over the process group, once at the end: not a data-path collective)."""
    if world == 1:
        return list(local)
    import torch.distributed as dist
    parts = [None] * world
    dist.all_gather_object(parts, (start, list(local)))
    out = []
    for _, part in sorted(parts, key=lambda p: p[0]):
        out.extend(part)
    return out


def node_throughput(args, dev, stream, pdhg, world=1, rank=0, workload_name=None, tol=None):
    """Node LPs of one shared K (64 seeded commitment fixings), partitioned
    over the ranks (node_partition) and solved by each rank in one
    pdhg_solve_batched call, against the same nodes solved one at a time.
    --nodes-tol > 0: every node to that rel-KKT (converged node LPs/s, per-node
    attempt histogram); else every node advanced --nodes-attempts attempts
    (node-attempts/s).  Device time with CUDA events, max over ranks."""
    import torch
    from paper_2512_06715_gb300.instances import node_fixings, workload

    workload_name = workload_name or args.nodes_workload
    tol = args.nodes_tol if tol is None else tol
    inst = workload(workload_name)
    B = args.nodes
    l_np, u_np = node_fixings(inst, B)
    start, stop = node_partition(B, world, rank)
    converged = tol > 0
    kw = dict(precision="mixed", host_loop=int(args.host_loop), autotune=int(not args.no_autotune))
    if converged:
        lim = dict(tol=tol, max_iters=10**9, time_limit_s=args.nodes_cap)
    else:
        lim = dict(tol=1e-12, max_iters=args.nodes_attempts, time_limit_s=600.0)
    o = pdhg.default_opts(**lim, **kw)
    # the batched sweeps' fixed shape (read only with --no-autotune)
    ob = pdhg.default_opts(**lim, **kw, kernel_variant=args.nodes_rows_per_warp, kernel_grid=args.nodes_grid)

    def event_time(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) * 1e-3, out

    local = []
    tb = 0.0
    tuning = None
    if stop > start:
        l_b = torch.as_tensor(l_np[start:stop], device=dev)
        u_b = torch.as_tensor(u_np[start:stop], device=dev)
        wb = pdhg.Workspace.from_instance(inst, ob, device=dev)
        if not converged:
            wb.solve_batched(l_b, u_b, want_y=False)  # allocations, graph
        tb, (_, _, rb) = event_time(lambda: wb.solve_batched(l_b, u_b, want_y=False))
        tuning = wb.tuning()["batched"]
        wb.close()
        local = [{"node": start + k, "status": r["status_name"], "attempts": r["iterations"],
                  "rel_kkt": r["rel_kkt"], "ir_rounds": r["ir_rounds"]} for k, r in enumerate(rb)]
    tb = max_over_ranks(tb, dev)
    nodes = gather_node_results(local, start, world)
    # one node at a time (rank 0): `seq` nodes spread over the batch
    seq = max(1, min(args.nodes_seq, B))
    t_seq, att_seq = [], []
    if rank == 0:
        for k in np.linspace(0, B - 1, seq).round().astype(int):
            w1 = pdhg.Workspace(inst.row_ptr, inst.col, inst.val, inst.c, l_np[k], u_np[k], inst.q,
                                inst.m_eq, o, device=dev)
            if not converged:
                w1.solve()
            t1, (_, _, r1) = event_time(lambda: w1.solve())
            w1.close()
            t_seq.append(t1)
            att_seq.append(r1["iterations"])
    total_att = sum(n["attempts"] for n in nodes)
    out = {"workload": workload_name, "n": inst.n, "m": inst.m, "nnz": inst.nnz, "nodes": B,
           "ranks": world, "partition": [list(node_partition(B, world, r)) for r in range(world)],
           "batched_tuning": tuning}
    if converged:
        att = np.array([n["attempts"] for n in nodes])
        statuses = sorted({n["status"] for n in nodes})
        t_seq_total = float(np.mean(t_seq)) * B if t_seq else None
        out.update({"tol": tol, "cap_s": args.nodes_cap, "statuses": statuses,
                    "optimal": sum(n["status"] == "optimal" for n in nodes),
                    "batched_s": tb, "batched_node_lps_per_s": B / tb,
                    "sequential_node_lps_per_s": (B / t_seq_total) if t_seq_total else None,
                    "ratio": (t_seq_total / tb) if t_seq_total else None,
                    "sequential_sample": {"nodes": seq, "mean_s": float(np.mean(t_seq)) if t_seq else None,
                                          "mean_attempts": float(np.mean(att_seq)) if att_seq else None},
                    "attempts_histogram": {"bins": np.histogram(att, bins=8)[1].round().astype(int).tolist(),
                                           "counts": np.histogram(att, bins=8)[0].tolist()},
                    "attempts_min_median_max": [int(att.min()), int(np.median(att)), int(att.max())],
                    "note": "node LPs/s = nodes / wall time to rel-KKT tol (batched: one call per rank, "
                            "max over ranks; sequential: mean single mixed solve x nodes)"})
    else:
        nb = total_att / tb
        ns = (sum(att_seq) / sum(t_seq)) if t_seq else None
        out.update({"attempts_per_node": args.nodes_attempts, "batched_node_attempts_per_s": nb,
                    "sequential_node_attempts_per_s": ns, "ratio": (nb / ns) if ns else None,
                    "batched_ms_per_attempt": tb / max(n["attempts"] for n in nodes) * 1e3,
                    "note": "node-attempts/s at equal attempt budgets per node"})
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2512_06715_gb300 import pdhg
    from paper_2512_06715_gb300.instances import workload

    inst = workload(args.workload)
    n, m, nnz = inst.n, inst.m, inst.nnz
    stream = torch.cuda.current_stream()

    def opts(prec, attempts, tol=1e-8, tl=600.0):
        return pdhg.default_opts(precision=prec, max_iters=attempts, tol=tol, time_limit_s=tl,
                                 host_loop=int(args.host_loop), autotune=int(not args.no_autotune),
                                 kernel_variant=args.kernel_variant, kernel_grid=args.kernel_grid,
                                 launch_overlap=int(args.launch_overlap))

    ws = pdhg.Workspace.from_instance(inst, opts("mixed", args.attempts), device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(prec, k, w):
        ws.set_opts(precision=pdhg.PREC_MIXED if prec == "mixed" else pdhg.PREC_FP64,
                    max_iters=args.attempts, tol=1e-8, time_limit_s=600.0)
        res = None
        for _ in range(w):
            _, _, res = ws.solve()
        barrier()
        total = 0.0
        launches = 0
        for _ in range(k):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, _, res = ws.solve()
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1) * 1e-3
            launches += res["kernel_launches"]
        barrier()
        return total, res, launches

    # headline: mixed precision
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    t_mixed, r_mixed, launches = timed("mixed", args.steps, args.warmup)
    clk = clocks.stop()
    t64, r64, _ = timed("fp64", max(1, args.steps // 2), 1)
    d32, a32 = algorithmic_bytes(n, m, nnz, 4)
    d64, a64 = algorithmic_bytes(n, m, nnz, 8)
    att32 = r_mixed["iterations"]
    att64 = r64["iterations"]
    sec_per_step = max_over_ranks(t_mixed / args.steps, dev)
    value = world * att32 * (d32 + a32) / sec_per_step / 1e9
    fp64_gbs = att64 * (d64 + a64) / (t64 / max(1, args.steps // 2)) / 1e9

    # dominant kernel, timed alone on this stream with CUDA events
    tk = ws.time_kernels(pdhg.PREC_MIXED, reps=20)
    achieved = tk["bytes_dual"] / (tk["ms_dual"] * 1e-3) / 1e9
    peaks = measured_peaks()
    dvar = ws.tuning()["fp32"]["unroll_dual"]
    kname = dual_kernel_name(dvar)
    traffic = dram_traffic_record(dual_kernel_source(dvar), kname)
    roofline = {"bound": "hbm", "kernel": kname + " (K x' + projected dual step)",
                "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "peak_source": peaks["source"] + " (burst)",
                "traffic": (traffic["bytes_per_launch"] if traffic else None),
                "algorithmic_bytes_per_launch": tk["bytes_dual"], "ms_per_launch": tk["ms_dual"],
                "adjoint_kernel_gbs": tk["bytes_adj"] / (tk["ms_adj"] * 1e-3) / 1e9}

    # end to end through host buffers: H2D of the LP values, solve, D2H of x, y
    host = {k: ws.t[k].cpu().pin_memory() for k in ("val", "c", "l", "u", "q")}
    xo = torch.empty(n, dtype=torch.float64).pin_memory()
    yo = torch.empty(m, dtype=torch.float64).pin_memory()
    ws.set_opts(precision=pdhg.PREC_MIXED, max_iters=args.attempts)
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = (n + m) * 8
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_att = 0
    e0.record(stream)
    for _ in range(args.steps):
        for k, v in host.items():
            ws.t[k].copy_(v, non_blocking=True)
        x, y, r = ws.solve()
        xo.copy_(x, non_blocking=True)
        yo.copy_(y, non_blocking=True)
        e_att += r["iterations"]
    e1.record(stream)
    e1.synchronize()
    e2e_s = e0.elapsed_time(e1) * 1e-3
    e2e = {"value": world * e_att * (d32 + a32) / e2e_s / 1e9, "unit": "GB/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "note": "each step copies the LP's values (val, c, l, u, q) from pinned host memory, solves, and "
                   "copies x, y back; the workspace (sliced-ELL layout of the sparsity pattern, device "
                   "buffers, CUDA graph) is built once before the timed region"}

    # time to tolerance: the large LP in both precisions (capped), the small one to 1e-8
    ttt = {}
    returned = {}  # points the CPU leg re-checks with the oracle
    if args.ttt_limit > 0:
        extra = {}
        for kv in args.ttt_opt:
            k, v = kv.split("=")
            extra[k] = float(v) if any(ch in v for ch in ".e") else int(v)
        arms = [("mixed", args.ttt_limit)] + ([("fp64", args.ttt_limit_fp64)] if args.ttt_limit_fp64 > 0 else [])
        for prec, cap in arms:
            ws.set_opts(precision=pdhg.PREC_MIXED if prec == "mixed" else pdhg.PREC_FP64,
                        max_iters=10**9, tol=1e-8, time_limit_s=cap, trace=int(bool(args.ttt_trace)), **extra)
            x, y, r = ws.solve()
            if args.ttt_trace:
                write_trace(Path(args.ttt_trace), f"{args.workload}_{prec}", ws.trace()[1], r, extra)
            returned[prec] = (x.cpu().numpy(), y.cpu().numpy(), r)
            ttt[prec] = {"status": r["status_name"], "rel_kkt": r["rel_kkt"],
                         "seconds_to_1e-4_1e-6_1e-8": r["time_to_tol"],
                         "attempts_to_1e-4_1e-6_1e-8": r["iters_to_tol"],
                         "cap_s": cap, "attempts": r["iterations"],
                         "attempts_per_s": r["iterations"] / r["solve_seconds"], "omega": r["omega"],
                         "ir_rounds": r["ir_rounds"], "primal_obj": r["primal_obj"]}
        ratios = {}
        for i, t in enumerate(("1e-4", "1e-6", "1e-8")):
            if "fp64" not in ttt:
                ratios[t] = None
                continue
            a_m, a_f = ttt["mixed"]["seconds_to_1e-4_1e-6_1e-8"][i], ttt["fp64"]["seconds_to_1e-4_1e-6_1e-8"][i]
            ratios[t] = (a_f / a_m) if (a_m > 0 and a_f > 0) else None
        ttt["fp64_over_mixed_seconds"] = ratios
        # the small relaxation, both precisions to 1e-8
        inst_s = workload(args.ttt_small)
        small = {}
        for prec in ("mixed", "fp64"):
            w2 = pdhg.Workspace.from_instance(inst_s, pdhg.default_opts(precision=prec, tol=1e-8, time_limit_s=300.0),
                                              device=dev)
            w2.solve()  # tuning, graph
            x2, y2, r2 = w2.solve()
            returned[f"{prec}@{args.ttt_small}"] = (x2.cpu().numpy(), y2.cpu().numpy(), r2)
            w2.close()
            small[prec] = {"status": r2["status_name"], "rel_kkt": r2["rel_kkt"], "seconds": r2["solve_seconds"],
                           "attempts": r2["iterations"], "seconds_to_1e-4_1e-6_1e-8": r2["time_to_tol"]}
        s_m, s_f = small["mixed"]["seconds"], small["fp64"]["seconds"]
        small["fp64_over_mixed_seconds_to_1e-8"] = s_f / s_m if (small["mixed"]["status"] == "optimal" and
                                                                 small["fp64"]["status"] == "optimal") else None
        ttt[args.ttt_small] = small

    nodes = (node_throughput(args, dev, stream, pdhg, world, rank)
             if (args.nodes_attempts > 0 or args.nodes_tol > 0) else None)
    nodes_conv = (node_throughput(args, dev, stream, pdhg, world, rank, args.nodes_conv_workload,
                                  args.nodes_conv_tol) if args.nodes_conv_tol > 0 else None)

    cpu = None
    if rank == 0 and not args.no_cpu:
        gbs, dt = cpu_oracle_gbs(inst, args.cpu_attempts)
        cpu = {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"{args.cpu_attempts} oracle attempts (rescaling included) on {args.workload}, {dt:.1f} s"}
        if args.cpu_ttt_limit > 0:
            cpu["time_to_tolerance"] = cpu_oracle_ttt([args.ttt_small, "uc4224_g600_T48"], args.cpu_ttt_limit)
        cpu["gpu_points_rechecked"] = cpu_recheck(returned, {args.workload: inst})

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec_per_step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "m": m, "nnz": nnz,
                       "attempts_per_step": args.attempts, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "256 MiB buffer written between timed steps; working set > L2"},
            "dtype_detail": "FP32 matrix and iterates, FP64 KKT/gap/restart reductions and refinement",
            "attempts_per_s": {"mixed": att32 / sec_per_step, "fp64": att64 / (t64 / max(1, args.steps // 2))},
            "fp64_gbs": fp64_gbs,
            "time_to_tolerance": ttt,
            "node_lps": nodes,
            "node_lps_converged": nodes_conv,
            "roofline": roofline,
            "gpu_launches": launches,
            "kernel_tuning": ws.tuning(),
            "launch_overlap": bool(r_mixed.get("launch_overlap", 0)),
            "e2e": e2e,
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    ws.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
