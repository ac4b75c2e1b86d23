#!/usr/bin/env python
"""Benchmark of the regular-force hot path (one JSON line on stdout).

A step is one pass of the whole path on one GPU: predict all j-particles to
the block time (nb_predict) and compute the regular force, jerk and neighbour
lists of the active set (nb_regular_force), inputs resident in HBM.  The
workload is the paper-scale cluster: a Kroupa-IMF Plummer sphere, N = 131072,
every particle active, ~100 neighbours, list capacity 256, two-float (mixed)
form.  The FP64 and plain FP32 forms of the same step are timed beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torch.distributed.run) every rank runs its own
replica on its own GPU (independent problems: weak scaling, no collective on
the data path); value is the interactions of all ranks over the slowest rank's
time.  --impl reference times the FP64 CPU oracle on bounded samples of the
same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("regular-force interactions/s and % FP32 peak at N=131072, mixed vs FP64 form, "
          "rel err ≤1e-6")
FLOPS_PER_INTERACTION = 60       # convention for one force + jerk interaction
L2_FLUSH_BYTES = 256 << 20       # > 129 MB L2
PROFILE = os.path.join(ROOT, "profiles", "regf_mixed_n131072.md")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="mixed", choices=["mixed", "fp64", "fp32"])
    ap.add_argument("--n-act", type=int, default=0, help="active particles (0 = all)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the FP64/FP32 side measurements")
    ap.add_argument("--cpu-sample", type=int, default=8192, help="active particles in the oracle sample")
    ap.add_argument("--accuracy-rows", default="all", choices=["all", "sample"],
                    help="rows of the accuracy check against the oracle: every active particle (about 15 s "
                         "of host work at N = n_act = 131072), or the timed CPU-baseline sample")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer measurement")
    ap.add_argument("--no-side", action="store_true",
                    help="skip the compact side workloads of the default line (batched clusters, offset cluster "
                         "with hard pairs, block-step sweep)")
    ap.add_argument("--config", default="", help="kernel tiling warps,ipw,jtile,packed[,split] "
                                                 "(default: the autotuner's choice)")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (library default tiling)")
    ap.add_argument("--workload", default="headline", choices=["headline", "batched64", "offset-pairs", "velocity", "irregular", "blockstep",
                                                      "needed"],
                    help="headline: the benchmark line; batched64: 64 independent clusters, one persistent "
                         "launch in a CUDA graph vs one launch per cluster; offset-pairs: N=262144 offset "
                         "cluster with 10%% hard pairs, FP32 vs two-float vs FP64 with errors; velocity: the "
                         "headline workload with the velocity neighbour criterion; irregular: the irregular "
                         "force over the lists of the headline workload; blockstep: N=16384 with active "
                         "subsets of 16..16384, two-float (autotuned) and FP64 forms; needed: all-j vs "
                         "needed-only prediction for the irregular force on the same subsets")
    ap.add_argument("--n", type=int, default=131072,
                    help="j-particles (131072 = the benchmark workload; smaller N builds the same kind of "
                         "cluster, used for profiling captures)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(n_act, n=131072):
    from paper_1205_1222_gb300 import inputs
    if n == 131072:
        w = inputs.cached(inputs.config3)
    else:
        w = inputs.cached(inputs.cluster, n, 3, 100, 256, "hierarchy", 2.0**-10, "kroupa",
                          key=f"kroupa_plummer_n{n}")
    if n_act and n_act < w.n:
        w = inputs.subset(w, n_act, 3)
    return w


def describe(w, mode):
    return {
        "workload": f"Kroupa-IMF Plummer sphere N={w.n}, n_act={w.n_act}, ~100 neighbours, cap {w.cap}, "
                    f"seed 3, steps 2^-3..2^-12, {mode} form",
        "N": w.n, "n_act": w.n_act, "cap": w.cap, "mode": mode, "neighbour_criterion": "|R| < h",
        "interactions_per_step": w.n * w.n_act,
        "l2": "flushed between timed steps (256 MB device write outside the timed events)",
    }


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="nbclk", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.device)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not self.path:
            return None
        rows = []
        for line in open(self.path):
            p = [s.strip() for s in line.split(",")]
            if len(p) < 9:
                continue
            try:
                rows.append((float(p[1]), float(p[2]), p[5], p[6], p[7], p[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        mx = max(r[1] for r in rows)
        busy = [r for r in rows if r[0] > 0.5 * mx] or rows
        reasons = set()
        for r in rows:
            for name, flag in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                                  r[2:]):
                if flag.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r[0] for r in busy), "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(rows)}


def rejected(clk):
    if not clk:
        return False
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
    if bad & set(clk["reasons"]):
        return True
    return clk["sm_mhz"] < 0.5 * clk["sm_max_mhz"] and not clk["reasons"]


# -------------------------------------------------------------- helpers

# Sources that define the profiled regular-force kernel and its launch: the
# committed ncu summary's traffic is reported only while these are unchanged.
# The device code of the profiled kernel (its launch shape is the tiling the
# summary names, which profiled_traffic() also checks).
KERNEL_SOURCES = ("nb_device.cuh", "nb_regf.cuh", "nb_pair_ops.cuh", "nb_regf3.cuh", "nb_regf_ws.cuh",
                  "nb_kernels.cuh")


def kernel_source_hash():
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1205_1222_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(tiling=None):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources and, when it names one, the same tiling
    (else None)."""
    if not os.path.exists(PROFILE):
        return None
    text = open(PROFILE).read()
    mh = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", text)
    mt = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    mc = re.search(r"tiling:\s*([0-9, ]+)", text)
    if not mh or not mt or mh.group(1) != kernel_source_hash():
        return None
    if mc and tiling is not None and [int(x) for x in mc.group(1).split(",")] != list(tiling):
        return None
    return float(mt.group(1))


def fp32_peak_tflops(sm_count, mhz):
    # 128 FP32 lanes per SM, 2 flops per fused multiply-add
    return sm_count * 128 * 2 * mhz * 1e6 / 1e12


def max_sm_mhz():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return float(json.load(open(p))["sm_max_mhz"]), "MEASURED_PEAKS.json sm_max_mhz"
        except Exception:
            pass
    return 2070.0, "nominal maximum SM clock"


def max_over_ranks(vals, device):
    """Element-wise maximum of per-rank timings (the slowest rank sets the pace)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def job_value(interactions_per_rank, world, ms_max):
    """Whole-job throughput: all ranks' interactions over the slowest rank's step time."""
    return interactions_per_rank * world / (ms_max / 1e3)


# -------------------------------------------------------------- GPU arm

class Runner:
    """Device-resident inputs and outputs of one workload, and one step."""

    def __init__(self, w, mode, device, cfg=""):
        import numpy as np
        import torch

        from paper_1205_1222_gb300 import Context, binding as B, mode_id
        self.B, self.torch, self.np = B, torch, np
        self.w, self.mode, self.device = w, mode_id(mode), device
        self.ctx = Context(w.n, device=device)
        dv = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=f"cuda:{device}")
        self.d = {k: dv(getattr(w, k)) for k in ("x0", "v0", "a0", "adot0", "m", "t0", "h")}
        self.d["act"] = dv(w.act, torch.int32)
        self.out = self.ctx.alloc_outputs(w.n_act, w.cap, pot=True)
        self.use_pot = False
        self.stream = torch.cuda.current_stream(device)
        self.form = B.MODE_FORM[self.mode]
        self.launches = 0
        self.use_dtr = False
        if w.dtr is not None:
            self.d["dtr"] = dv(w.dtr)
        if cfg:
            f = [int(x) for x in cfg.split(",")]
            B.nb_set_kernel_config(self.ctx.h, self.mode, B.nb_kcfg(f[0], f[1], f[2], f[4] if len(f) > 4 else 0,
                                                                    f[3]))
        self.cfg = B.nb_get_active_config(self.ctx.h, self.mode).as_tuple()

    def predict(self):
        d = self.d
        self.B.nb_predict(self.ctx.h, 0, self.w.n, d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"],
                          self.w.t, self.form, self.stream)
        self.launches += 1

    def force(self):
        d, o = self.d, self.out
        self.B.nb_regular_force(self.ctx.h, 0, self.w.n, self.w.n_act, d["act"], d["h"],
                                d["dtr"] if self.use_dtr else None, self.w.cap,
                                self.mode, o["F"], o["J"], o["pot"] if self.use_pot else None, o["nnb"], o["list"],
                                o["ovf"], self.stream)
        self.launches += self.ctx.last_launches()

    def timed(self, steps, flush):
        torch = self.torch
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
        for s in range(steps):
            flush.zero_()
            ev[s][0].record(self.stream)
            self.predict()
            ev[s][1].record(self.stream)
            self.force()
            ev[s][2].record(self.stream)
        torch.cuda.synchronize(self.device)
        step_ms = [e[0].elapsed_time(e[2]) for e in ev]
        force_ms = [e[1].elapsed_time(e[2]) for e in ev]
        return step_ms, force_ms

    def graph_step_us(self, reps=20):
        """Device time per step of `reps` steps (prediction + force) captured in
        one CUDA graph and replayed back to back (L2 warm, no host launches):
        the floor a compiled caller's block step reaches.  Minimum of 3 replays."""
        torch = self.torch
        side = torch.cuda.Stream(self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        old, launches = self.stream, self.launches
        self.stream = side
        try:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.stream(side):
                self.predict(); self.force()   # split scratch reserved before the capture
                torch.cuda.synchronize(self.device)
                with torch.cuda.graph(g, stream=side):
                    for _ in range(reps):
                        self.predict(); self.force()
            g.replay()
            torch.cuda.synchronize(self.device)
            best = float("inf")
            for _ in range(3):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(); g.replay(); b.record()
                torch.cuda.synchronize(self.device)
                best = min(best, a.elapsed_time(b) * 1e3 / reps)
            return best
        finally:
            self.stream, self.launches = old, launches

    def autotune(self, reps=1):
        """Native autotuner on this workload (untimed); later calls use its choice."""
        from paper_1205_1222_gb300 import autotune
        self.predict()
        t0 = time.perf_counter()
        best, ms = self.ctx.autotune(self.d["act"], self.d["h"], self.w.n, cap=self.w.cap, mode=self.mode,
                                     dtr=self.d["dtr"] if self.use_dtr else None, pot=self.use_pot,
                                     out=self.out, reps=reps, stream=self.stream)
        self.cfg = best.as_tuple()
        return {"best": list(self.cfg), "best_ms": ms, "seconds": time.perf_counter() - t0,
                "table": autotune.table(self.ctx)}

    def load_tuned(self, rows):
        for r in rows:
            t = self.B.nb_tuned()
            t.mode, t.flags, t.act_class, t.j_class = r["mode"], r["flags"], r["act_class"], r["j_class"]
            t.cfg = self.B.nb_kcfg(*r["cfg"])
            self.B.nb_set_tuned(self.ctx.h, t)

    def outputs(self):
        return {k: v.cpu().numpy() for k, v in self.out.items() if v is not None}

    def close(self):
        self.ctx.close()


def e2e_measure(w, mode, device, steps, tuned=()):
    """The same step through nb_step_host: host (pinned) inputs in, host outputs out."""
    import numpy as np
    import torch

    from paper_1205_1222_gb300 import Context, binding as B, mode_id
    pin = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).pin_memory()
    hx = {k: pin(getattr(w, k)) for k in ("x0", "v0", "a0", "adot0", "m", "t0", "h")}
    act = pin(w.act, torch.int32)
    F = torch.empty((w.n_act, 3), dtype=torch.float64).pin_memory()
    J = torch.empty_like(F)
    nnb = torch.empty(w.n_act, dtype=torch.int32).pin_memory()
    lst = torch.empty((w.n_act, w.cap), dtype=torch.int32).pin_memory()
    ovf = torch.empty(w.n_act, dtype=torch.uint8).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in list(hx.values()) + [act])
    d2h = sum(t.numel() * t.element_size() for t in (F, J, nnb, lst, ovf))
    with Context(w.n, device=device) as ctx:
        st = torch.cuda.current_stream(device)
        for r in tuned:
            t = B.nb_tuned()
            t.mode, t.flags, t.act_class, t.j_class = r["mode"], r["flags"], r["act_class"], r["j_class"]
            t.cfg = B.nb_kcfg(*r["cfg"])
            B.nb_set_tuned(ctx.h, t)

        def step():
            B.nb_step_host(ctx.h, w.n, hx["x0"], hx["v0"], hx["a0"], hx["adot0"], hx["m"], hx["t0"], w.t, w.n_act,
                           act, hx["h"], None, w.cap, mode_id(mode), F, J, None, nnb, lst, ovf, st)
        step()
        step()
        t0 = time.perf_counter()
        for _ in range(steps):
            step()
        dt = (time.perf_counter() - t0) / steps
    return {"value": w.n * w.n_act / dt, "unit": "interactions/s", "ms_per_step": dt * 1e3,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "api": "nb_step_host (pinned host buffers, copies inside the timed call)"}


def accuracy(g, o, rows, cap):
    """Max / RMS relative error per output and list mismatches on the sampled rows."""
    import numpy as np

    def rel(a, b):
        nb = np.linalg.norm(b, axis=1)
        return np.linalg.norm(a - b, axis=1) / np.where(nb > 0, nb, 1.0)
    eF = rel(g["F"][rows], o["F"])
    eJ = rel(g["J"][rows], o["J"])
    k = np.minimum(o["nnb"], cap)
    filled = np.arange(cap)[None, :] < k[:, None]
    bad = (g["nnb"][rows] != o["nnb"]) | np.any(np.where(filled, g["list"][rows], -1) !=
                                               np.where(filled, o["list"], -1), axis=1)
    return {"F_max": float(eF.max()), "F_rms": float(np.sqrt((eF ** 2).mean())),
            "J_max": float(eJ.max()), "J_rms": float(np.sqrt((eJ ** 2).mean())),
            "list_mismatches": int(bad.sum()), "sampled": int(len(rows))}


def cpu_baseline(w, sample):
    """The FP64 oracle, as it stands, on a bounded sample of the active set."""
    import numpy as np

    import oracle
    rows = np.sort(np.random.default_rng(12345).choice(w.n_act, min(sample, w.n_act), replace=False))
    x, v = oracle.predict(w.x0, w.v0, w.a0, w.adot0, w.t0, w.t)
    threads = oracle.default_threads()
    t0 = time.perf_counter()
    o = oracle.regular(x, v, w.m, w.act[rows], w.h[rows], cap=w.cap, threads=threads)
    dt = time.perf_counter() - t0
    base = {"value": len(rows) * w.n / dt, "unit": "interactions/s", "cores": threads, "kind": "oracle",
            "sample": f"{len(rows)} sampled active particles x all {w.n} j-particles "
                      f"({len(rows) * w.n:.3g} interactions, FP64 C, OpenMP over i, {dt:.2f} s wall)"}
    one = rows[:max(1, len(rows) // 16)]   # the same oracle on one core, a sixteenth of the sample
    t1 = time.perf_counter()
    oracle.regular(x, v, w.m, w.act[one], w.h[one], cap=w.cap, threads=1)
    d1 = time.perf_counter() - t1
    base["single_thread"] = {"value": len(one) * w.n / d1, "cores": 1,
                             "sample": f"{len(one)} of the sampled active particles x all {w.n} j-particles "
                                       f"({d1:.2f} s wall)"}
    return base, o, rows


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    device = local if world > 1 else 0
    torch.cuda.set_device(device)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", device))
    from paper_1205_1222_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    w = workload(args.n_act, args.n)
    r = Runner(w, args.mode, device, args.config)
    tune = None
    if not args.config and not args.no_tune and args.mode != "fp64":
        tune = r.autotune()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=f"cuda:{device}")
    for _ in range(max(args.warmup, 3)):
        r.predict()
        r.force()
    torch.cuda.synchronize(device)
    st = r.ctx.sync_status()
    assert st == 0, f"device status {st}"

    def region():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(device)
        r.launches = 0
        with ClockSampler(device) as cs:
            t0 = time.perf_counter()
            step_ms, force_ms = r.timed(args.steps, flush)
            wall = time.perf_counter() - t0
        if world > 1:
            torch.distributed.barrier()
        return step_ms, force_ms, wall, cs.summary()

    step_ms, force_ms, wall, clk = region()
    remeasured = False
    if rejected(clk):
        step_ms, force_ms, wall, clk = region()
        remeasured = True
    ms = statistics.mean(step_ms)
    fms = statistics.mean(force_ms)
    launches = r.launches
    if world > 1:
        ms, fms = max_over_ranks([ms, fms], f"cuda:{device}")
    inter = w.n * w.n_act
    value = job_value(inter, world, ms)
    sm = r.ctx.sm_count()
    mhz, mhz_src = max_sm_mhz()
    peak = fp32_peak_tflops(sm, mhz)
    achieved = FLOPS_PER_INTERACTION * inter / (fms / 1e3) / 1e12
    g_main = r.outputs()
    r.close()

    # end to end through the host-buffer API: every rank runs its replica, the
    # slowest rank sets the whole job's time (as for the device-timed value)
    e2e = None
    if not args.no_e2e:
        if world > 1:
            torch.distributed.barrier()
        e2e = e2e_measure(w, args.mode, device, max(1, min(args.steps, 5)), tune["table"] if tune else ())
        if world > 1:
            e2e_ms = max_over_ranks([e2e["ms_per_step"]], f"cuda:{device}")[0]
            e2e.update(ms_per_step=e2e_ms, value=job_value(inter, world, e2e_ms),
                       h2d_bytes_per_step=e2e["h2d_bytes_per_step"] * world,
                       d2h_bytes_per_step=e2e["d2h_bytes_per_step"] * world)

    if rank != 0:
        if world > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return

    line = {
        "metric": METRIC, "value": value, "unit": "interactions/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.mode != "fp64" else "f64", "data": "synthetic",
        "config": dict(describe(w, args.mode), parallelism=f"replicas{world}" if world > 1 else "single"),
    }
    line["timing"] = {
        "events": "CUDA events on the launching stream around each step; L2 flushed before each",
        "step_ms_mean": ms, "step_ms_median": statistics.median(step_ms),
        "force_ms_mean": fms, "force_ms_median": statistics.median(force_ms),
        "predict_ms_mean": statistics.mean(a - b for a, b in zip(step_ms, force_ms)),
        "step_ms_min": min(step_ms), "step_ms_max": max(step_ms),
    }
    line["roofline"] = {
        "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
        "traffic": profiled_traffic(r.cfg),
        "kernel": "regular force + jerk + list kernel, one launch per step; tiling (warps, ipw, jtile, "
                  f"split, packed) = {r.cfg}",
        "kernel_ms": fms,
        "peak_basis": f"{sm} SMs x 128 FP32 lanes x 2 flops x {mhz:.0f} MHz ({mhz_src}); "
                      f"{FLOPS_PER_INTERACTION} flops per interaction",
    }
    if clk:
        line["roofline"]["peak_at_measured_clock"] = fp32_peak_tflops(sm, clk["sm_mhz"])
        line["roofline"]["frac_at_measured_clock"] = achieved / line["roofline"]["peak_at_measured_clock"]
    if tune:
        line["autotune"] = {"chosen": tune["best"], "best_ms": tune["best_ms"], "seconds": tune["seconds"],
                            "note": "native nb_autotune over every compiled tiling and j-split, before the "
                                    "timed region"}
    line["gpu_launches"] = launches
    line["clocks"] = clk
    if remeasured:
        line["clocks_remeasured"] = True
    line["wall_s_timed_region"] = wall

    forms = {}
    outs = {args.mode: g_main}
    if not args.no_forms and world == 1:   # the other forms and the oracle leg: one GPU only
        # the exact two-float pair form (two-float velocity differences too) beside the default
        for label, mode, cfg in (("fp64", "fp64", ""), ("fp32", "fp32", ""), ("mixed", "mixed", ""),
                                 ("mixed_exact_pair", "mixed", "16,2,1536,14")):
            if mode == args.mode and not cfg and not args.config:
                forms[label] = {"value": value / world, "ms_per_step": ms, "kernel_ms": fms, "tiling": r.cfg}
                continue
            rr = Runner(w, mode, device, cfg)
            if mode == "fp32" and not args.no_tune:
                rr.autotune()
            rr.predict(); rr.force()
            torch.cuda.synchronize(device)
            k = 2 if mode == "fp64" else args.steps
            sm_, fm_ = rr.timed(k, flush)
            forms[label] = {"value": inter / (statistics.mean(sm_) / 1e3), "ms_per_step": statistics.mean(sm_),
                            "kernel_ms": statistics.mean(fm_), "steps": k, "tiling": rr.cfg,
                            "frac_fp32_peak": FLOPS_PER_INTERACTION * inter / (statistics.mean(fm_) / 1e3) / 1e12 / peak}
            outs[label] = rr.outputs()
            rr.close()
        line["forms"] = forms
    if e2e is not None:
        line["e2e"] = e2e
    if not args.no_cpu_baseline and world == 1:
        base, o, rows = cpu_baseline(w, args.cpu_sample)
        line["cpu_baseline"] = base
        acc_note = f"the {len(rows)} rows of the CPU-baseline sample"
        if args.accuracy_rows == "all" and len(rows) < w.n_act:
            import numpy as np

            import oracle
            t0 = time.perf_counter()
            x, v = oracle.predict(w.x0, w.v0, w.a0, w.adot0, w.t0, w.t)
            o = oracle.regular(x, v, w.m, w.act, w.h, cap=w.cap, threads=oracle.default_threads())
            rows = np.arange(w.n_act)
            acc_note = f"every one of the {w.n_act} active rows (oracle {time.perf_counter() - t0:.1f} s)"
        line["accuracy_vs_oracle"] = {m: accuracy(g, o, rows, w.cap) for m, g in outs.items()}
        line["accuracy_vs_oracle"]["rows"] = acc_note
    if not args.no_side and world == 1:
        line.update(side_workloads(args, peak))
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    print(json.dumps(line), flush=True)


def side_workloads(args, peak):
    """Compact results of the other benchmark configurations, each bounded to
    a few seconds: the 64-cluster batched launch (cfg4), the offset cluster
    with hard pairs at 4096 active in every form (cfg5) and the block-step
    sweep of active-set sizes (cfg2).  Each is timed outside the headline's
    timed region; the full records come from --workload batched64 /
    offset-pairs / blockstep."""
    out = {}
    t0 = time.perf_counter()
    b = batched_result(args, steps=5)
    acc = b["accuracy_vs_oracle"]
    out["cfg4"] = {
        "workload": "64 Plummer clusters, N 1024..32768, n_act 8..N, seed 4 (N_total %d, n_act_total %d)"
                    % (b["config"]["N_total"], b["config"]["n_act_total"]),
        "graph_ms": b["ms_per_step"], "value": b["value"],
        "frac_fp32_peak": FLOPS_PER_INTERACTION * b["value"] / 1e12 / peak,
        "per_cluster_ms": b["per_cluster_launches"]["ms_per_step"], "speedup_vs_per_cluster": b["speedup_vs_per_cluster"],
        "plan_tiling": b["plan_tiling"], "F_max": acc["F_max"], "J_max": acc["J_max"],
        "list_mismatches": acc["list_mismatches"], "rows_beyond_relative_bar": acc["rows_beyond_relative_bar"],
        "rows_beyond_u_times_term_length_sum": acc["rows_beyond_u_times_term_length_sum"],
        "graph_vs_per_cluster_list_mismatches": b["graph_vs_per_cluster_list_mismatches"],
        "seconds": time.perf_counter() - t0}
    t0 = time.perf_counter()
    o = offset_result(args, n_acts=(4096,), steps=3)
    out["cfg5"] = {"workload": "Plummer N=262144 at |x_c|=1e3, 10% hard pairs, 4096 active, oracle on all 4096 rows",
                   "forms": {k.split("@")[0]: {"value": f["value"], "kernel_ms": f["kernel_ms"],
                                                "frac_fp32_peak": FLOPS_PER_INTERACTION * f["value"] / 1e12 / peak,
                                                "F_max": f["accuracy"]["F_max"], "J_max": f["accuracy"]["J_max"],
                                                "list_mismatches": f["accuracy"]["list_mismatches"]}
                             for k, f in o["forms"].items()},
                   "seconds": time.perf_counter() - t0}
    t0 = time.perf_counter()
    bs = blockstep_result(args, steps=3)
    out["cfg2"] = {"workload": "Plummer N=16384, random active subsets, prediction + force per step",
                   "sizes": [{"n_act": r["n_act"], "mixed_graph_step_us": r["mixed"]["graph_step_us"],
                              "mixed_step_us_l2_flushed": r["mixed"]["step_ms"] * 1e3,
                              "fp64_graph_step_us": r["fp64"]["graph_step_us"],
                              "mixed_F_max": r["mixed"]["accuracy"]["F_max"],
                              "mixed_J_max": r["mixed"]["accuracy"]["J_max"],
                              "list_mismatches": r["mixed"]["accuracy"]["list_mismatches"]} for r in bs["sizes"]],
                   "seconds": time.perf_counter() - t0}
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np

    import oracle
    w = workload(args.n_act, args.n)
    x, v = oracle.predict(w.x0, w.v0, w.a0, w.adot0, w.t0, w.t)
    threads = oracle.default_threads()
    sample = min(256, w.n_act)
    rng = np.random.default_rng(7)

    def step():
        rows = np.sort(rng.choice(w.n_act, sample, replace=False))
        oracle.predict(w.x0, w.v0, w.a0, w.adot0, w.t0, w.t)
        oracle.regular(x, v, w.m, w.act[rows], w.h[rows], cap=w.cap, threads=threads)
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    value = sample * w.n / dt
    desc = (f"each step: FP64 oracle prediction of all {w.n} j plus the regular force of {sample} sampled "
            f"active particles ({sample * w.n:.3g} interactions), OpenMP over i")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "interactions/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": describe(w, "fp64 oracle"),
            "cpu_baseline": {"value": value, "unit": "interactions/s", "cores": threads, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "interactions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------- side workloads

def _timed_events(fn, steps, flush, stream, torch):
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(steps)]
    for s in range(steps):
        flush.zero_()
        ev[s][0].record(stream)
        fn()
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    return [e[0].elapsed_time(e[1]) for e in ev]


def run_batched(args):
    print(json.dumps(batched_result(args)), flush=True)


def batched_result(args, steps=None):
    """64 independent clusters (N log-uniform in [1024, 32768], n_act log-uniform
    in [8, N]): prediction of all clusters in one launch plus the regular force
    of all of them as one persistent launch (and the split merge) replayed from
    a CUDA graph, against one nb_regular_force call per cluster."""
    import numpy as np
    import torch

    from paper_1205_1222_gb300 import Context, binding as B, build, inputs, mode_id
    build.build()
    torch.cuda.set_device(0)
    ws = inputs.cached(inputs.config4)
    offs = np.cumsum([0] + [w.n + (w.n % 2) for w in ws])
    total = int(offs[-1])
    # one j-set: clusters at even offsets, padded slots get zero mass far away
    x0 = np.zeros((total, 3)); v0 = np.zeros((total, 3)); a0 = np.zeros((total, 3)); ad = np.zeros((total, 3))
    m = np.zeros(total); t0 = np.full(total, ws[0].t)
    for w, o in zip(ws, offs):
        x0[o:o + w.n], v0[o:o + w.n], a0[o:o + w.n], ad[o:o + w.n] = w.x0, w.v0, w.a0, w.adot0
        m[o:o + w.n], t0[o:o + w.n] = w.m, w.t0
    for o, w in zip(offs, ws):
        if w.n % 2:
            x0[o + w.n] = 1e6
    dev = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    mode = mode_id(args.mode)
    inter = int(sum(w.n * w.n_act for w in ws))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    with Context(total) as ctx:
        d = {k: dev(v) for k, v in (("x0", x0), ("v0", v0), ("a0", a0), ("ad", ad), ("m", m), ("t0", t0))}
        keep, cl = [], []
        for w, o in zip(ws, offs):
            a, h = dev(w.act, torch.int32), dev(w.h)
            out = ctx.alloc_outputs(w.n_act, w.cap)
            keep.append((a, h, out))
            cl.append(B.nb_cluster(int(o), w.n, w.n_act, w.cap, a.data_ptr(), h.data_ptr(), None,
                                   out["F"].data_ptr(), out["J"].data_ptr(), None, out["nnb"].data_ptr(),
                                   out["list"].data_ptr(), out["ovf"].data_ptr()))
        stream = torch.cuda.Stream()
        form = B.MODE_FORM[mode]

        def predict():
            B.nb_predict(ctx.h, 0, total, d["x0"], d["v0"], d["a0"], d["ad"], d["m"], d["t0"], ws[0].t, form, stream)

        with torch.cuda.stream(stream):
            predict()
            pcfg = None
            if args.config:
                f = [int(x) for x in args.config.split(",")]
                pcfg = B.nb_kcfg(f[0], f[1], f[2], f[4] if len(f) > 4 else 0, f[3])
            plan = B.nb_plan_create(ctx.h, cl, mode, pcfg)
            tuned = None
            try:
                if pcfg is None and not args.no_tune:
                    t0 = time.perf_counter()
                    best, best_ms = B.nb_plan_autotune(plan, reps=2, stream=stream, ctx=ctx.h)
                    tuned = {"chosen": list(best.as_tuple()), "best_ms": best_ms,
                             "seconds": time.perf_counter() - t0,
                             "note": "native nb_plan_autotune over every compiled tiling x j-split length on the "
                                     "plan's own clusters, before the timed region"}
                plan_cfg = list(B.nb_plan_get_config(plan).as_tuple())
                B.nb_plan_capture(plan, stream=stream, ctx=ctx.h)
                for _ in range(max(args.warmup, 3)):
                    predict(); B.nb_plan_launch(plan, stream=stream, ctx=ctx.h)
                graph_ms = _timed_events(lambda: (predict(), B.nb_plan_launch(plan, stream=stream, ctx=ctx.h)),
                                         steps or args.steps, flush, stream, torch)
                plan_launches = 1 + B.nb_plan_launches(plan)
                stream.synchronize()
                graph_out = [{k: v.cpu().numpy() for k, v in out.items() if v is not None} for _, _, out in keep]
            finally:
                B.nb_plan_destroy(plan)

            def per_cluster():
                predict()
                for w, o, (a, h, out) in zip(ws, offs, keep):
                    B.nb_regular_force(ctx.h, int(o), w.n, w.n_act, a, h, None, w.cap, mode, out["F"], out["J"],
                                       None, out["nnb"], out["list"], out["ovf"], stream)
            for _ in range(max(args.warmup, 3)):
                per_cluster()
            loop_ms = _timed_events(per_cluster, steps or args.steps, flush, stream, torch)
            stream.synchronize()
            loop_out = [{k: v.cpu().numpy() for k, v in out.items() if v is not None} for _, _, out in keep]
        st = ctx.sync_status(stream)
    g, l = statistics.mean(graph_ms), statistics.mean(loop_ms)
    # correctness of the timed outputs: lists of the graph-replayed plan equal
    # to the per-cluster calls', and every row of every cluster against the
    # oracle (FP64, all host cores)
    import oracle
    mism = sum(int(np.any(a[k] != b[k])) for a, b in zip(graph_out, loop_out) for k in ("nnb", "list", "ovf"))
    eFs, eJs, bad, beyond, outside = [], [], 0, 0, 0
    u = 2.0 ** -24
    t0 = time.perf_counter()
    for w, go in zip(ws, graph_out):
        x, v = oracle.predict(w.x0, w.v0, w.a0, w.adot0, w.t0, w.t)
        o = oracle.regular(x, v, w.m, w.act, w.h, cap=w.cap)
        SF, SJ = oracle.regular_mag(x, v, w.m, w.act, w.h)
        acc = accuracy(go, o, np.arange(w.n_act), w.cap)
        eFs.append(acc["F_max"]); eJs.append(acc["J_max"]); bad += acc["list_mismatches"]
        dF = np.linalg.norm(go["F"] - o["F"], axis=1); nF = np.linalg.norm(o["F"], axis=1)
        dJ = np.linalg.norm(go["J"] - o["J"], axis=1); nJ = np.linalg.norm(o["J"], axis=1)
        rel_ok = (dF <= 1e-6 * nF) & (dJ <= 1e-5 * nJ)
        beyond += int((~rel_ok).sum())
        outside += int((~(rel_ok | ((dF <= u * SF) & (dJ <= u * SJ)))).sum())
    oracle_s = time.perf_counter() - t0
    return {
        "metric": "regular-force interactions/s, 64 independent clusters, one persistent launch in a CUDA graph",
        "value": inter / (g / 1e3), "unit": "interactions/s", "n_gpus": 1, "steps": steps or args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": g, "higher_is_better": True, "dtype": "f32",
        "data": "synthetic", "status": st,
        "config": {"workload": "64 equal-mass Plummer clusters, N log-uniform in [1024, 32768], n_act "
                               "log-uniform in [8, N], ~64 neighbours, cap 256, seed 4",
                   "mode": args.mode, "N_total": int(sum(w.n for w in ws)),
                   "n_act_total": int(sum(w.n_act for w in ws)), "interactions_per_step": inter,
                   "l2": "flushed between timed steps"},
        "per_cluster_launches": {"value": inter / (l / 1e3), "ms_per_step": l,
                                 "launches_per_step": 1 + len(ws)},
        "graph_launches_per_step": plan_launches, "speedup_vs_per_cluster": l / g,
        "plan_tiling": plan_cfg, "autotune": tuned,
        "accuracy_vs_oracle": {"rows": "every row of every cluster", "F_max": max(eFs), "J_max": max(eJs),
                               "list_mismatches": bad, "rows_beyond_relative_bar": beyond,
                               "rows_beyond_u_times_term_length_sum": outside, "oracle_seconds": oracle_s},
        "graph_vs_per_cluster_list_mismatches": mism,
    }


def run_offset_pairs(args):
    print(json.dumps(offset_result(args)), flush=True)


def offset_result(args, n_acts=None, steps=None):
    """N = 262144 cluster offset to |x_c| = 1e3 with 10% of the particles in hard
    pairs: FP32, two-float (default and exact pair form) and FP64 forms, their
    throughput and their errors against the oracle on sampled rows."""
    import numpy as np
    import torch

    import oracle
    from paper_1205_1222_gb300 import build, inputs
    build.build()
    torch.cuda.set_device(0)
    full = inputs.cached(inputs.config5)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    x, v = oracle.predict(full.x0, full.v0, full.a0, full.adot0, full.t0, full.t)
    res = {}
    for n_act in (n_acts or (4096, full.n)):
        w = full if n_act == full.n else inputs.subset(full, n_act, 5)
        rows = np.arange(w.n_act) if w.n_act <= 4096 else \
            np.sort(np.random.default_rng(5).choice(w.n_act, 4096, replace=False))
        o = oracle.regular(x, v, w.m, w.act[rows], w.h[rows], cap=w.cap)
        for label, mode, cfg in (("fp32", "fp32", ""), ("mixed", "mixed", ""), ("mixed_exact_pair", "mixed", "16,2,1536,14"),
                                 ("fp64", "fp64", "")):
            r = Runner(w, mode, 0, cfg)
            if not cfg and mode != "fp64" and not args.no_tune:
                r.autotune()
            r.predict(); r.force()
            k = 1 if mode == "fp64" and n_act == full.n else (steps or max(2, min(args.steps, 5)))
            ms = statistics.mean(r.timed(k, flush)[1])
            g = r.outputs()
            r.close()
            res[f"{label}@{n_act}"] = {"value": w.n * w.n_act / (ms / 1e3), "kernel_ms": ms, "tiling": r.cfg,
                                       "accuracy": accuracy(g, o, rows, w.cap)}
    return {
        "metric": "regular-force interactions/s and errors vs the FP64 oracle, offset cluster with hard pairs",
        "unit": "interactions/s", "n_gpus": 1, "dtype": "f32/f64", "data": "synthetic",
        "config": {"workload": "equal-mass Plummer, N=262144, centre at |x|=1e3, 10% in hard pairs "
                               "(separations 1e-5..1e-2), ~128 neighbours, cap 256, seed 5",
                   "n_act": list(n_acts or (4096, full.n)), "oracle_rows": "all 4096 / a seeded 4096-row sample"},
        "forms": res,
    }


def run_velocity(args):
    """The headline workload with the velocity criterion min(|R|, |R + dtr V|) < h
    (dtr per particle from the regular steps 2^-6 .. 2^-9) against the plain
    criterion, and the plain criterion with the potential output, two-float
    form, with errors on sampled rows."""
    import numpy as np
    import torch

    import oracle
    from paper_1205_1222_gb300 import build, inputs
    build.build()
    torch.cuda.set_device(0)
    w = inputs.cached(inputs.cluster, 131072, 3, 100, 256, "hierarchy", 2.0**-10, "kroupa", 0.0, 0.0, None, None,
                      (2.0**-6, 2.0**-7, 2.0**-8, 2.0**-9), key="kroupa_plummer_n131072_dtr")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    rows = np.sort(np.random.default_rng(7).choice(w.n_act, 2048, replace=False))
    x, v = oracle.predict(w.x0, w.v0, w.a0, w.adot0, w.t0, w.t)
    res = {}
    for crit in ("plain", "velocity", "plain+potential"):
        o = oracle.regular(x, v, w.m, w.act[rows], w.h[rows], dtr=w.dtr[rows] if crit == "velocity" else None,
                           cap=w.cap, with_pot=crit.endswith("potential"))
        r = Runner(w, args.mode, 0, "")
        r.use_dtr = crit == "velocity"
        r.use_pot = crit.endswith("potential")
        if not args.no_tune:
            r.autotune()
        r.predict(); r.force()
        ms = statistics.mean(r.timed(max(2, min(args.steps, 5)), flush)[1])
        g = r.outputs()
        r.close()
        res[crit] = {"value": w.n * w.n_act / (ms / 1e3), "kernel_ms": ms, "tiling": r.cfg,
                     "accuracy": accuracy(g, o, rows, w.cap)}
        if r.use_pot:
            rp = np.abs(g["pot"][rows] - o["pot"]) / np.abs(o["pot"])
            res[crit]["accuracy"]["pot_max"] = float(rp.max())
    print(json.dumps({
        "metric": "regular-force interactions/s with the velocity neighbour criterion vs the plain one",
        "unit": "interactions/s", "n_gpus": 1, "dtype": "f32", "data": "synthetic", "mode": args.mode,
        "config": {"workload": "Kroupa-IMF Plummer sphere N=131072, all active, ~100 neighbours, cap 256, seed 3, "
                               "dtr per particle in {2^-6..2^-9}", "oracle_rows": 2048},
        "criteria": res, "cost_of_velocity_criterion": res["velocity"]["kernel_ms"] / res["plain"]["kernel_ms"],
        "cost_of_potential": res["plain+potential"]["kernel_ms"] / res["plain"]["kernel_ms"],
    }), flush=True)


def run_irregular(args):
    """The irregular force (Sec. 3.3 step (iv)) over the neighbour lists of the
    headline workload, all three forms, against the oracle on sampled rows; the
    work is a gather of each neighbour's predicted record."""
    import numpy as np
    import torch

    import oracle
    from paper_1205_1222_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    w = workload(args.n_act, args.n)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    rows = np.sort(np.random.default_rng(11).choice(w.n_act, 2048, replace=False))
    x, v = oracle.predict(w.x0, w.v0, w.a0, w.adot0, w.t0, w.t)
    oF, oJ = oracle.irregular(x, v, w.m, w.act[rows], w.h[rows])
    res = {}
    bytes_per = {"fp64": 64, "mixed": 64, "fp32": 32}
    for mode in ("fp64", "mixed", "fp32"):
        r = Runner(w, mode, 0, "")
        r.predict(); r.force()
        torch.cuda.synchronize()
        nnb = r.out["nnb"]
        pairs = int(nnb.sum().item())
        stream = r.stream
        res_out = {}

        def irr():
            res_out["o"] = r.ctx.irregular_force(r.d["act"], nnb, r.out["list"], w.n, w.cap, mode=mode, stream=stream)
        for _ in range(3):
            irr()
        ms = statistics.mean(_timed_events(irr, max(3, min(args.steps, 10)), flush, stream, torch))
        st = r.ctx.sync_status()
        g = {k: v.cpu().numpy() for k, v in res_out["o"].items() if v is not None}
        r.close()

        def rel(a, b):
            nb = np.linalg.norm(b, axis=1)
            return np.linalg.norm(a - b, axis=1) / np.where(nb > 0, nb, 1.0)
        algo = pairs * (bytes_per[mode] + 4) + w.n_act * (2 * bytes_per[mode] + 8 + 48)
        res[mode] = {"value": pairs / (ms / 1e3), "kernel_ms": ms, "status": st, "neighbour_pairs": pairs,
                     "algorithmic_GBps": algo / (ms / 1e3) / 1e9,
                     "F_max": float(rel(g["F"][rows], oF).max()), "J_max": float(rel(g["J"][rows], oJ).max())}
    print(json.dumps({
        "metric": "irregular-force neighbour interactions/s over the regular-force lists",
        "unit": "interactions/s", "n_gpus": 1, "dtype": "f64/f32", "data": "synthetic",
        "config": {"workload": describe(w, "all")["workload"], "oracle_rows": 2048,
                   "bytes": "per neighbour: its predicted record (64 B FP64 / two-float, 32 B FP32) + 4 B index"},
        "forms": res,
    }), flush=True)


def run_blockstep(args):
    print(json.dumps(blockstep_result(args)), flush=True)


def blockstep_result(args, steps=None):
    """Block-step active subsets of the N = 16384 Plummer cluster (n_act = 16 ..
    16384, steps 2^-3 .. 2^-12): prediction plus regular force per step for the
    two-float form (autotuned per size class) and the FP64 form, with errors
    against the oracle on every row."""
    import numpy as np
    import torch

    import oracle
    from paper_1205_1222_gb300 import build, inputs
    build.build()
    torch.cuda.set_device(0)
    full = inputs.cached(inputs.config2)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    x, v = oracle.predict(full.x0, full.v0, full.a0, full.adot0, full.t0, full.t)
    res = []
    for n_act in (16, 64, 256, 1024, 4096, 16384):
        w = full if n_act == full.n else inputs.subset(full, n_act, 2)
        o = oracle.regular(x, v, w.m, w.act, w.h, cap=w.cap)
        row = {"n_act": n_act}
        for mode in ("mixed", "fp64"):
            r = Runner(w, mode, 0, "")
            if mode == "mixed" and not args.no_tune:
                r.autotune()
            for _ in range(3):
                r.predict(); r.force()
            step_ms, force_ms = r.timed(steps or max(3, min(args.steps, 10)), flush)
            g = r.outputs()
            graph_us = r.graph_step_us()
            r.close()
            row[mode] = {"step_ms": statistics.mean(step_ms), "kernel_ms": statistics.mean(force_ms),
                         "graph_step_us": graph_us,
                         "interactions_per_s": w.n * n_act / (statistics.mean(step_ms) / 1e3), "tiling": r.cfg,
                         "accuracy": accuracy(g, o, np.arange(n_act), w.cap)}
        res.append(row)
    return {
        "metric": "regular-force interactions/s per block step (prediction included) across active-set sizes",
        "unit": "interactions/s", "n_gpus": 1, "dtype": "f32/f64", "data": "synthetic",
        "config": {"workload": "equal-mass Plummer N=16384, seed 2, ~64 neighbours, cap 256, random active subsets",
                   "l2": "flushed between timed steps; graph_step_us: 20 steps replayed from one CUDA graph, "
                         "L2 warm"},
        "sizes": res,
    }


def _graph_us(fn, device, reps=20):
    """Device time per call of `reps` calls of fn(stream) captured in one CUDA
    graph and replayed (L2 warm, no host launches); best of 3 replays."""
    import torch
    side = torch.cuda.Stream(device)
    side.wait_stream(torch.cuda.current_stream(device))
    with torch.cuda.stream(side):
        fn(side)
        torch.cuda.synchronize(device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            for _ in range(reps):
                fn(side)
    g.replay()
    torch.cuda.synchronize(device)
    best = float("inf")
    for _ in range(3):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(); g.replay(); b.record()
        torch.cuda.synchronize(device)
        best = min(best, a.elapsed_time(b) * 1e3 / reps)
    return best


def run_needed(args):
    """Needed-only prediction (Sec. 3.5, the NPACT switch) on the N = 16384
    cluster and on the N = 131072 Kroupa cluster: for active subsets of 16 ..
    4096, the prediction that the irregular force needs (all j; only the
    active particles and their listed neighbours; the library's switch
    between the two) plus the irregular force, graph-replayed per step; the
    irregular results of the needed-only and full predictions are compared
    bit for bit."""
    import numpy as np
    import torch

    import oracle
    from paper_1205_1222_gb300 import Context, binding as B, build, inputs
    build.build()
    torch.cuda.set_device(0)
    dv = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    out_sets = []
    for label, full in (("N=16384 equal-mass Plummer, seed 2", inputs.cached(inputs.config2)),
                        ("N=131072 Kroupa Plummer, seed 3", inputs.cached(inputs.config3))):
        x, v = oracle.predict(full.x0, full.v0, full.a0, full.adot0, full.t0, full.t)
        d = {k: dv(getattr(full, k)) for k in ("x0", "v0", "a0", "adot0", "m", "t0")}
        res = []
        for n_act in (16, 64, 256, 1024, 4096):
            w = inputs.subset(full, n_act, 2)
            o = oracle.regular(x, v, w.m, w.act, w.h, cap=w.cap)
            act, nnb, lst = dv(w.act, torch.int32), dv(o["nnb"], torch.int32), dv(o["list"], torch.int32)
            named = np.zeros(full.n, dtype=bool)
            named[w.act] = True
            for k in range(n_act):
                named[o["list"][k, :min(o["nnb"][k], w.cap)]] = True
            row = {"n_act": n_act, "named_slots": int(named.sum()), "list_entries": int(o["nnb"].sum())}
            with Context(full.n) as ctx:
                ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], full.t, forms=B.NB_FORM_MIXED)

                def pred_all(st):
                    B.nb_predict(ctx.h, 0, full.n, d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], full.t,
                                 B.NB_FORM_MIXED | B.NB_KEEP_FRAME, st)

                def pred_needed(st, only=True):
                    B.nb_predict_needed(ctx.h, 0, full.n, n_act, act, nnb, lst, w.cap, d["x0"], d["v0"], d["a0"],
                                        d["adot0"], d["m"], d["t0"], full.t,
                                        B.NB_FORM_MIXED | (B.NB_NEEDED_ONLY if only else 0), st)
                outs = {}

                def irr(st, key):
                    outs[key] = ctx.irregular_force(act, nnb, lst, full.n, w.cap, mode="mixed", stream=st)
                row["predict_all_us"] = _graph_us(pred_all, 0)
                row["predict_needed_us"] = _graph_us(pred_needed, 0)
                row["predict_switch_us"] = _graph_us(lambda st: pred_needed(st, only=False), 0)
                row["all_plus_irregular_us"] = _graph_us(lambda st: (pred_all(st), irr(st, "all")), 0)
                row["needed_plus_irregular_us"] = _graph_us(lambda st: (pred_needed(st), irr(st, "needed")), 0)
                torch.cuda.synchronize()
                row["status"] = ctx.sync_status()
                row["bit_identical"] = bool(torch.equal(outs["all"]["F"], outs["needed"]["F"]) and
                                            torch.equal(outs["all"]["J"], outs["needed"]["J"]))
            res.append(row)
        cross = next((r["n_act"] for r in res if r["predict_needed_us"] >= r["predict_all_us"]), None)
        out_sets.append({"workload": label, "N": full.n, "sizes": res, "needed_slower_from_n_act": cross})
    print(json.dumps({
        "metric": "prediction time per block step for the irregular force: all j vs needed-only",
        "unit": "us", "n_gpus": 1, "dtype": "f64 polynomial, two-float stored form", "data": "synthetic",
        "config": {"workload": "random active subsets, ~64 / ~100 neighbours, cap 256",
                   "timing": "20 calls replayed from one CUDA graph, best of 3, L2 warm"},
        "sets": out_sets,
    }), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched64":
        run_batched(args)
    elif args.workload == "offset-pairs":
        run_offset_pairs(args)
    elif args.workload == "velocity":
        run_velocity(args)
    elif args.workload == "irregular":
        run_irregular(args)
    elif args.workload == "blockstep":
        run_blockstep(args)
    elif args.workload == "needed":
        run_needed(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
