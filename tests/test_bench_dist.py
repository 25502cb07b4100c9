"""Host logic of the multi-rank bench on CPU: two gloo ranks (one process
each, rendezvous on 127.0.0.1) reduce their timed regions to the slowest
rank's, compute the whole-job rate from it, and on the reference arm only
rank 0 does any work or prints.  No GPU is involved."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        local_ms = 100.0 + 25.0 * rank          # rank 1 is the slow one
        ms = bench.max_over_ranks(local_ms, ws)
        rate = bench.whole_job_rate(ws, 30, ms)
        env = bench.dist_env()
        # reference arm: ranks other than 0 return without output
        out = io.StringIO()
        if rank != 0:
            with redirect_stdout(out):
                bench.run_reference(type("A", (), {"workload": "small", "warmup": 3, "steps": 1, "gpus": ws,
                                                    "sample": 16, "sample_iters": 1, "seed": 1})())
        q.put((rank, ms, rate, env, out.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate, env, printed in res:
        assert ms == pytest.approx(125.0)
        assert rate == pytest.approx(2 * 30 / 0.125)
        assert env == (2, rank, rank)
        assert printed == ""


def test_single_rank_helpers_need_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.whole_job_rate(1, 10, 500.0) == pytest.approx(20.0)


def test_recorded_traffic_follows_its_kernel_source(tmp_path, monkeypatch):
    """A traffic record is scaled per voxel while the kernel text it was
    captured from is unchanged (whole file, or the kernel from its first
    line to its closing brace), and gives None once that text changes."""
    import hashlib
    import json
    sys.path.insert(0, ROOT)
    import bench
    src = tmp_path / "k.cu"
    src.write_text("int a;\n__global__ void k_one(int* p)\n{\n    p[0] = 1;\n}\n__global__ void k_two()\n{\n}\n")
    begin = "__global__ void k_one("
    text = bench.kernel_source_text(str(src), begin)
    assert text.startswith(begin.encode()) and text.endswith(b"p[0] = 1;\n}\n")
    (tmp_path / "profiles").mkdir()
    rec = dict(kernel_source="k.cu", kernel_begin=begin, kernel_source_sha256=hashlib.sha256(text).hexdigest(),
               captured_voxels=1000, dram_bytes_read=6000, dram_bytes_write=2000)
    (tmp_path / "profiles" / "t.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("t", 4000) == pytest.approx(32000.0)
    src.write_text(src.read_text().replace("k_two()\n{\n}", "k_two()\n{\n    return;\n}"))
    assert bench.recorded_traffic("t", 4000) == pytest.approx(32000.0)     # another kernel changed
    src.write_text(src.read_text().replace("p[0] = 1;", "p[0] = 2;"))
    assert bench.recorded_traffic("t", 4000) is None                        # this kernel changed
    assert bench.recorded_traffic("missing", 4000) is None


def test_batched_volumes_shard_across_ranks():
    """The batched workload's volumes go to ranks with no exchange: each
    volume to exactly one rank, deterministically, the largest first to the
    least-loaded rank (so no rank holds more than the lightest rank plus the
    largest volume)."""
    import numpy as np

    sys.path.insert(0, ROOT)
    import bench
    from paper_2608_14112_b300 import inputs
    sizes = [int(np.prod(s)) for s in inputs.BATCHED_SHAPES]
    assert bench.shard_volumes(sizes, 1, 0) == list(range(len(sizes)))
    for ws in (2, 3, 4, 8):
        shards = [bench.shard_volumes(sizes, ws, r) for r in range(ws)]
        assert sorted(i for s in shards for i in s) == list(range(len(sizes)))
        assert shards == [bench.shard_volumes(sizes, ws, r) for r in range(ws)]
        loads = [sum(sizes[i] for i in s) for s in shards]
        assert max(loads) - min(loads) <= max(sizes)
