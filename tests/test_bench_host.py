"""Host logic of bench.py without a GPU: the reference arm (the CPU oracle) in one
process and under a two-rank launch, and the max-over-ranks timing on gloo."""
import json
import os
import socket
import subprocess
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
ARGS = ["--impl", "reference", "--workload", "uc24_g33_T24", "--steps", "1", "--warmup", "0",
        "--cpu-attempts", "4"]


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _json_lines(out: str) -> list[dict]:
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def test_reference_arm_prints_one_line():
    p = subprocess.run([sys.executable, "bench.py", *ARGS], cwd=ROOT, capture_output=True, text=True,
                       timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = _json_lines(p.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "GB/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_reference_arm_two_ranks_rank0_only():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--gpus", "2", *ARGS]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600,
                       env={**os.environ, "OMP_NUM_THREADS": "1"})
    assert p.returncode == 0, p.stderr[-2000:]
    lines = _json_lines(p.stdout)
    assert len(lines) == 1 and lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2


def _max_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, str(ROOT))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    q.put((rank, bench.max_over_ranks(1.5 + rank, torch.device("cpu"))))
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_max_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got == {0: 2.5, 1: 2.5}


def test_dram_traffic_record_matches_kernel_and_source(tmp_path, monkeypatch):
    """The committed traffic figure is used only for the same kernel variant and an
    unchanged kernel source; the record file may hold one record or a list."""
    import hashlib
    sys.path.insert(0, str(ROOT))
    import bench
    src = tmp_path / "k.cu"
    src.write_text("kernel source")
    h = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", tmp_path)
    rec = {"kernel": "k_dual<float, 1>", "bytes_per_launch": 1.0, "kernel_source_sha256_16": h}
    for content in (rec, [rec, {**rec, "kernel": "k_dual_pipe<float>", "bytes_per_launch": 2.0}]):
        (prof / "dram_traffic.json").write_text(json.dumps(content))
        assert bench.dram_traffic_record(src, "k_dual<float, 1>")["bytes_per_launch"] == 1.0
        assert bench.dram_traffic_record(src, "k_dual<float, 4>") is None
    src.write_text("changed")
    assert bench.dram_traffic_record(src, "k_dual<float, 1>") is None


def test_node_partition_covers_every_node_once():
    sys.path.insert(0, str(ROOT))
    import bench
    for B in (1, 7, 64, 65):
        for world in (1, 2, 3, 8):
            blocks = [bench.node_partition(B, world, r) for r in range(world)]
            covered = [k for a, b in blocks for k in range(a, b)]
            assert covered == list(range(B))
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1


def _gather_worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, str(ROOT))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    start, stop = bench.node_partition(9, world, rank)
    local = [{"node": k, "rank": rank} for k in range(start, stop)]
    q.put((rank, bench.gather_node_results(local, start, world)))
    dist.destroy_process_group()


def test_node_results_gather_gloo():
    """Two ranks solve their blocks of 9 nodes; every rank ends with all 9
    results in node order, each from the rank whose block holds it."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gather_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    for rank in (0, 1):
        assert [d["node"] for d in got[rank]] == list(range(9))
        assert [d["rank"] for d in got[rank]] == [0] * 5 + [1] * 4


def test_every_autotuner_variant_names_its_kernel_and_source():
    """The roofline line names the K x' kernel of whatever variant the autotuner
    picks and looks its DRAM record up under that kernel's source file: every
    variant the autotuner times maps to a template instance defined in the file
    named, and the committed record's kernels are among them."""
    import re
    sys.path.insert(0, str(ROOT))
    import bench
    api = (ROOT / "paper_2512_06715_gb300" / "csrc" / "pdhg_api.cu").read_text()
    m = re.search(r"const int unrolls\[\d+\] = \{([^}]*)\}", api)
    variants = [int(v) for v in m.group(1).split(",")]
    names = set()
    for v in variants:
        name = bench.dual_kernel_name(v)
        assert not name.startswith("variant"), v
        base = name.split("<")[0]
        src = bench.dual_kernel_source(v)
        assert src.exists() and re.search(r"\b%s\s*\(" % base, src.read_text()), (v, name, src)
        names.add(name)
    recs = json.loads((ROOT / "profiles" / "dram_traffic.json").read_text())
    for r in recs:
        assert r["kernel"] in names, r["kernel"]
        assert (ROOT / r["source"]).exists(), r["source"]


def test_write_trace_table(tmp_path):
    """The per-check trace summary: the array is saved, the table lists about 40
    evenly spaced checks plus every restart, with the command that made it."""
    import numpy as np
    sys.path.insert(0, str(ROOT))
    import bench
    n = 200
    checks = np.zeros((n, 12))
    checks[:, 0] = 64 * np.arange(1, n + 1)
    checks[[3, 77, 150], 1] = 1           # restarts
    checks[77, 2] = 1                     # one of them to the average
    checks[:, 3] = 2.0
    checks[:, 6] = np.logspace(0, -6, n)  # rel-KKT of the current iterate
    checks[:, 7] = np.logspace(0, -7, n)
    r = {"status_name": "time_limit", "rel_kkt": 1e-7, "iterations": 64 * n, "restarts": 3, "ir_rounds": 5,
         "omega": 2.0, "time_to_tol": [1.0, 2.0, -1.0]}
    bench.write_trace(tmp_path, "case_mixed", checks, r, {"bound_obj_rescale": 1})
    assert np.array_equal(np.load(tmp_path / "trace_case_mixed.npy"), checks)
    md = (tmp_path / "trace_case_mixed.md").read_text()
    rows = [l for l in md.splitlines() if l.startswith("| ") and l[2].isdigit()]
    assert 40 <= len(rows) <= 43
    assert any(l.startswith("| 4992 | yes (avg)") for l in rows)  # check 77 (0-based, 64 x 78 attempts): to the average
    assert any(l.startswith("| 256 | yes |") for l in rows)
    assert "python " in md and "bound_obj_rescale" in md
