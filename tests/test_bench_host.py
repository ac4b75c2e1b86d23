"""Host-side logic of bench.py (CPU only), including the multi-rank path
with two gloo ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def test_clock_rejection_rules():
    assert not bench.rejected(None)
    assert not bench.rejected({"sm_mhz": 1900, "sm_max_mhz": 2070, "reasons": ["sw_power_cap"]})
    assert bench.rejected({"sm_mhz": 1900, "sm_max_mhz": 2070, "reasons": ["hw_slowdown"]})
    assert bench.rejected({"sm_mhz": 600, "sm_max_mhz": 2070, "reasons": []})


def test_fp32_peak_formula():
    assert bench.fp32_peak_tflops(152, 2070) == pytest.approx(80.54, rel=1e-3)


def test_profiled_traffic_requires_current_sources(tmp_path, monkeypatch):
    p = tmp_path / "prof.md"
    p.write_text(f"kernel_source_hash: {bench.kernel_source_hash()}\ntraffic_bytes_per_launch: 1.5e9\n")
    monkeypatch.setattr(bench, "PROFILE", str(p))
    assert bench.profiled_traffic() == 1.5e9
    p.write_text("kernel_source_hash: 0000\ntraffic_bytes_per_launch: 1.5e9\n")
    assert bench.profiled_traffic() is None


def test_profiled_traffic_requires_the_same_tiling(tmp_path, monkeypatch):
    p = tmp_path / "prof.md"
    p.write_text(f"kernel_source_hash: {bench.kernel_source_hash()}\ntiling: 16, 2, 1536, 0, 5\n"
                 "traffic_bytes_per_launch: 2.5e7\n")
    monkeypatch.setattr(bench, "PROFILE", str(p))
    assert bench.profiled_traffic((16, 2, 1536, 0, 5)) == 2.5e7
    assert bench.profiled_traffic((16, 2, 1024, 0, 5)) is None


def test_cpu_baseline_reports_all_cores_and_one_core():
    """The oracle leg of the benchmark: a bounded sample timed on all host cores
    and a sixteenth of it on one core, with the keys the benchmark line needs;
    the sampled rows it returns are the oracle's own outputs."""
    import numpy as np
    import oracle
    from paper_1205_1222_gb300 import inputs
    w = inputs.cluster(3000, 9, 24, 64)
    base, o, rows = bench.cpu_baseline(w, 320)
    assert base["kind"] == "oracle" and base["unit"] == "interactions/s" and base["value"] > 0
    assert base["cores"] >= 1 and "sample" in base
    one = base["single_thread"]
    assert one["cores"] == 1 and one["value"] > 0
    assert len(rows) == 320 and np.all(np.diff(rows) > 0)
    x, v = oracle.predict(w.x0, w.v0, w.a0, w.adot0, w.t0, w.t)
    ref = oracle.regular(x, v, w.m, w.act[rows], w.h[rows], cap=w.cap)
    assert np.array_equal(o["F"], ref["F"]) and np.array_equal(o["list"], ref["list"])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [10.0 + rank * 5.0, 3.0 - rank]          # rank 1 is slower on the first timing
    mx = bench.max_over_ranks(ms, "cpu")
    val = bench.job_value(1000, world, mx[0])
    q.put((rank, mx, val))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_over_ranks_and_job_value():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, val in res:
        assert mx == [15.0, 3.0]
        assert val == pytest.approx(1000 * 2 / 0.015)
