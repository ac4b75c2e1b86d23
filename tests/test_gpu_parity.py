"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

Small cases span several j-tiles, ragged tails and every compiled kernel
configuration; the full-size cases use the launch configuration the benchmark
times and compare sampled active particles one by one, plus properties that
hold at any size (every particle's neighbour count equals the count the
radius was constructed for).
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1205_1222_gb300 import Context, binding as B, build, inputs, mode_id
from tests.gpu_util import (TOL, compare, compare_conditioned, dev, direct_sum_accel, gpu_run, list_mismatches,
                            oracle_predicted, oracle_run, rel_err, upload)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


@pytest.fixture(scope="module")
def cfg1():
    return inputs.config1(accel=direct_sum_accel)


@pytest.fixture(scope="module")
def cfg2():
    return inputs.cached(inputs.config2)


# ------------------------------------------------------------ small cases

@pytest.mark.parametrize("mode", ["fp64", "mixed", "fp32"])
def test_config1_plummer_1024(cfg1, mode):
    g = gpu_run(cfg1, mode)
    assert g["status"] == 0
    o = oracle_run(cfg1)
    compare(g, o, cfg1.cap, mode, lists=(mode != "fp32"))
    if mode == "fp32":
        assert list_mismatches(g, o, cfg1.cap) <= cfg1.n_act // 50


def test_predictor_matches_oracle(cfg1):
    import torch
    w = cfg1
    with Context(w.n) as ctx:
        d = upload(w)
        ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t)
        x = torch.empty((w.n, 3), dtype=torch.float64, device="cuda")
        v = torch.empty_like(x)
        m = torch.empty(w.n, dtype=torch.float64, device="cuda")
        B.nb_get_predicted(ctx.h, 0, w.n, x, v, m)
        torch.cuda.synchronize()
        xo, vo = oracle_predicted(w)
        assert np.max(np.abs(x.cpu().numpy() - xo)) <= 4e-16 * np.max(np.abs(xo)) * 4
        assert np.max(np.abs(v.cpu().numpy() - vo)) <= 4e-16 * np.max(np.abs(vo)) * 4
        assert np.array_equal(m.cpu().numpy(), w.m)


@pytest.mark.parametrize("n_act", [16, 64, 256, 1024, 4096, 16384])
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_config2_block_step_sweep(cfg2, n_act, mode):
    w = inputs.subset(cfg2, n_act, 2) if n_act < cfg2.n else cfg2
    g = gpu_run(w, mode)
    assert g["status"] == 0
    compare(g, oracle_run(w), w.cap, mode)


@pytest.mark.parametrize("n,n_act", [(33, 33), (1000, 31), (1537, 200), (2049, 2049), (4097, 65)])
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_ragged_sizes(n, n_act, mode):
    w = inputs.cluster(n, 100 + n, min(16, n - 2) if n > 3 else 1, 64,
                       act=np.sort(np.random.default_rng(n).choice(n, n_act, replace=False)))
    g = gpu_run(w, mode)
    assert g["status"] == 0
    compare(g, oracle_run(w), w.cap, mode)


def test_two_bodies():
    """Two particles: each sees the other (h > r) or feels it (h < r)."""
    import types
    for h, nnb in ((0.5, 0), (3.0, 1)):
        w = inputs.cluster(40, 21, 8, 4)
        w2 = types.SimpleNamespace(**{k: getattr(w, k) for k in ("x0", "v0", "a0", "adot0", "m", "t0", "t")})
        for k in ("x0", "v0", "a0", "adot0", "m", "t0"):
            setattr(w2, k, getattr(w, k)[:2].copy())
        w2.x0[1] = w2.x0[0] + np.array([1.0, 0.5, -0.25])
        w2.n, w2.n_act, w2.cap, w2.dtr = 2, 2, 4, None
        w2.act = np.array([0, 1], dtype=np.int32)
        w2.h = np.array([h, h])
        for mode in ("fp64", "mixed", "fp32"):
            g = gpu_run(w2, mode)
            o = oracle_run(w2)
            assert np.all(g["nnb"] == nnb)
            compare(g, o, 4, mode)


def test_zero_radius_gives_the_full_sum():
    w = inputs.cluster(3000, 7, 8, 16)
    w.h[:] = 0.0
    for mode in ("fp64", "mixed"):
        g = gpu_run(w, mode)
        assert np.all(g["nnb"] == 0) and np.all(g["ovf"] == 0)
        x, v = oracle_predicted(w)
        F, J = oracle.full(x, v, w.m, w.act)
        ftol, jtol = TOL[mode]
        assert rel_err(g["F"], F).max() <= ftol and rel_err(g["J"], J).max() <= jtol


@pytest.mark.parametrize("cap", [0, 1, 7, 300])
def test_everyone_a_neighbour_and_overflow(cap):
    n = 700
    w = inputs.cluster(n, 8, 8, cap)
    w.h[:] = 1e4
    g = gpu_run(w, "mixed", cap=cap)
    assert g["status"] == 0
    assert np.all(g["nnb"] == n - 1)
    assert np.all(g["ovf"] == (1 if n - 1 > cap else 0))
    assert np.all(g["F"] == 0) and np.all(g["J"] == 0)
    if cap > 0:
        o = oracle_run(w, cap=cap)
        k = min(cap, n - 1)
        assert np.array_equal(g["list"][:, :k], o["list"][:, :k])


@pytest.mark.parametrize("mode", ["fp64", "mixed", "fp32"])
def test_coincident_particles_inside_the_sphere(mode):
    """Pairs of distinct particles at exactly the same predicted position and
    velocity (their whole start-of-step state copied) are neighbours of each
    other: listed, kept out of the force and jerk, no NaN anywhere."""
    import dataclasses
    w = inputs.cluster(3000, 71, 32, 64)
    x0, v0, a0, ad, t0 = (np.array(a) for a in (w.x0, w.v0, w.a0, w.adot0, w.t0))
    src = np.arange(0, 3000, 97)
    dst = (src + 500) % 3000
    for arr in (x0, v0, a0, ad, t0):
        arr[dst] = arr[src]
    X, V = oracle.predict(x0, v0, a0, ad, t0, w.t)
    h, _ = inputs.choose_radii(X, V, np.arange(w.n), 24, 40, np.random.default_rng(72))
    w2 = dataclasses.replace(w, x0=x0, v0=v0, a0=a0, adot0=ad, t0=t0, h=h)
    g = gpu_run(w2, mode)
    o = oracle_run(w2)
    assert g["status"] == 0 and np.isfinite(g["F"]).all() and np.isfinite(g["J"]).all()
    for a, b in zip(src, dst):   # each copy is in the other's list
        assert b in o["list"][a][:o["nnb"][a]] and a in o["list"][b][:o["nnb"][b]]
    compare(g, o, w2.cap, mode, lists=(mode != "fp32"))


def test_empty_active_set_launches_nothing():
    w = inputs.cluster(500, 9, 8, 16, act=np.zeros(0, dtype=np.int32))
    g = gpu_run(w, "mixed")
    assert g["status"] == 0 and g["launches"] == 0 and g["F"].shape == (0, 3)


@pytest.mark.parametrize("mode", ["fp64", "mixed", "fp32"])
def test_velocity_criterion(mode):
    w = inputs.cluster(6000, 11, 48, 128, dtr_steps=(2.0**-5, 2.0**-6, 2.0**-7, 2.0**-8))
    g = gpu_run(w, mode)
    o = oracle_run(w)
    compare(g, o, w.cap, mode, lists=(mode != "fp32"))


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_potential(mode):
    w = inputs.cluster(5000, 12, 40, 96)
    g = gpu_run(w, mode, pot=True)
    compare(g, oracle_run(w, pot=True), w.cap, mode, pot=True)


def test_j_range_offset_in_a_larger_context():
    w = inputs.cluster(2500, 13, 30, 64)
    with Context(w.n + 5000) as ctx:
        g = gpu_run(w, "mixed", ctx=ctx, j_offset=777)
    compare(g, oracle_run(w), w.cap, "mixed")


@pytest.mark.parametrize("mode", ["mixed", "fp32"])
@pytest.mark.parametrize("vel,pot", [(True, False), (False, True), (True, True)])
def test_odd_first_slot_with_velocity_criterion_or_potential(mode, vel, pot):
    """A j-range at an odd slot cannot be read as j-pairs: the call runs on a
    per-particle-layout kernel compiled with the same flags."""
    w = inputs.cluster(3000, 31, 40, 64, act=np.arange(0, 3000, 7, dtype=np.int32),
                       dtr_steps=(2.0**-6, 2.0**-8) if vel else None)
    with Context(w.n + 3) as ctx:
        g = gpu_run(w, mode, pot=pot, ctx=ctx, j_offset=3)
    assert g["status"] == 0
    compare(g, oracle_run(w, pot=pot), w.cap, mode, pot=pot and mode != "fp32", lists=(mode != "fp32"))


def _sweep_cases(count=24, seed=2026):
    """Seeded random combinations of size, active count, neighbour count, list
    capacity (0 and overflowing ones included), form, velocity criterion,
    potential, j-range offset (odd ones take the per-particle layout) and
    j-split (default tiling, or 1 or 3 tiles per split)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(rng.integers(40, 9000))
        out.append(dict(k=k, n=n, n_act=int(rng.integers(1, n + 1)), k_nb=int(rng.integers(1, min(80, n - 4))),
                        cap=int(rng.choice([0, 1, 16, 64, 128, 256])), mode=str(rng.choice(["fp64", "mixed", "mixed"])),
                        vel=bool(rng.random() < 0.4), pot=bool(rng.random() < 0.4),
                        off=int(rng.choice([0, 0, 1, 2, 777])), split=int(rng.choice([0, 0, 1, 3]))))
    return out


@pytest.mark.parametrize("c", _sweep_cases(), ids=lambda c: f"case{c['k']}-{c['mode']}")
def test_random_sweep(c):
    act = np.sort(np.random.default_rng(1000 + c["k"]).choice(c["n"], c["n_act"], replace=False)).astype(np.int32)
    w = inputs.cluster(c["n"], 500 + c["k"], c["k_nb"], max(c["cap"], 1), act=act,
                       dtr_steps=(2.0**-6, 2.0**-8) if c["vel"] else None)
    cfg = None
    if c["split"]:
        d = B.nb_get_kernel_config(mode_id(c["mode"]), 0).as_tuple()   # the default tiling
        cfg = B.nb_kcfg(d[0], d[1], d[2], c["split"], d[4])
    with Context(c["n"] + c["off"]) as ctx:
        g = gpu_run(w, c["mode"], cap=c["cap"], pot=c["pot"], ctx=ctx, j_offset=c["off"], cfg=cfg)
    assert g["status"] == 0
    compare(g, oracle_run(w, cap=c["cap"], pot=c["pot"]), c["cap"], c["mode"], pot=c["pot"])


def _block_edge_cases():
    # (tiling, i-block size): list-warp kernels own 12 x 2 = 24 particles per
    # CTA block, the 16-warp j-pair kernels 32
    tilings = [((16, 2, 1024, 0, 9), 24), ((16, 2, 1536, 0, 14), 24), ((16, 2, 512, 0, 5), 32),
               ((16, 2, 512, 0, 2), 32)]
    out = []
    for t, ib in tilings:
        for n_act in (1, ib - 1, ib + 1, 37 * ib + 1, 152 * ib + 1):
            for split in (0, 2):
                out.append((t, n_act, split))
    return out


@pytest.mark.parametrize("tiling,n_act,split", _block_edge_cases(),
                         ids=lambda v: "-".join(map(str, v)) if isinstance(v, tuple) else str(v))
def test_last_i_block_part_filled(tiling, n_act, split):
    """The last CTA block of active particles holds one particle (n_act = 1
    mod the i-block), or is one short of full, with and without j-splits
    (split = 2: two 512/1024/1536-j tiles per work item): the end-of-item
    stores and the split merge must write exactly rows 0 .. n_act-1, and a
    full grid round plus one particle (152 blocks + 1) must wrap to the next
    round."""
    import torch
    n = 6000
    w = inputs.cluster(n, 4100 + n_act, 40, 64,
                       act=np.sort(np.random.default_rng(n_act).choice(n, n_act, replace=False)))
    cfg = B.nb_kcfg(tiling[0], tiling[1], tiling[2], split, tiling[4])
    with Context(n) as ctx:
        d = upload(w)
        ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t)
        ctx.set_config("mixed", cfg)
        # outputs with a guard row past the end that must stay untouched
        out = ctx.alloc_outputs(n_act + 1, w.cap)
        for k in ("F", "J"):
            out[k].fill_(7.0)
        out["nnb"].fill_(-9); out["ovf"].fill_(5)
        view = {k: (v[:n_act] if v is not None else None) for k, v in out.items()}
        ctx.regular_force(d["act"], d["h"], w.n, cap=w.cap, mode="mixed", out=view)
        assert ctx.sync_status() == 0
        if split:
            assert ctx.last_launches() == 2
        g = {k: v.cpu().numpy() for k, v in out.items() if v is not None}
    assert np.all(g["F"][n_act] == 7.0) and np.all(g["J"][n_act] == 7.0)
    assert g["nnb"][n_act] == -9 and g["ovf"][n_act] == 5 and np.all(g["list"][n_act] == -1)
    compare({k: v[:n_act] for k, v in g.items()}, oracle_run(w), w.cap, "mixed")


def test_split_and_unsplit_paths_agree():
    w = inputs.cluster(20000, 14, 64, 256, act=np.arange(0, 20000, 97, dtype=np.int32))
    o = oracle_run(w)
    for warps, ipw, jt, packed in ((16, 2, 512, 2), (8, 4, 512, 0)):
        one = gpu_run(w, "mixed", cfg=B.nb_kcfg(warps, ipw, jt, 1000, packed))   # one split per i-block
        many = gpu_run(w, "mixed", cfg=B.nb_kcfg(warps, ipw, jt, 1, packed))     # one tile per split
        assert one["launches"] == 1 and many["launches"] == 2
        for g in (one, many):
            compare(g, o, w.cap, "mixed")
        assert np.array_equal(one["list"], many["list"])


def _all_cfgs():
    try:
        build.build()
        out = []
        for mode in ("fp64", "mixed", "fp32"):
            for i in range(B.nb_num_kernel_configs(mode_id(mode))):
                out.append((mode, B.nb_get_kernel_config(mode_id(mode), i).as_tuple()))
        return out
    except Exception:   # no compiler: the list is empty and the module's fixture fails instead
        return []


@pytest.mark.parametrize("mode,cfg", _all_cfgs())
def test_every_compiled_configuration(mode, cfg):
    w = inputs.cluster(3100, 15, 40, 128, act=np.arange(0, 3100, 6, dtype=np.int32))
    for split in (0, 1):
        g = gpu_run(w, mode, cfg=B.nb_kcfg(cfg[0], cfg[1], cfg[2], split, cfg[4]))
        assert g["status"] == 0
        compare(g, oracle_run(w), w.cap, mode, lists=(mode != "fp32"))


def test_repeat_calls_are_bit_identical():
    w = inputs.cluster(9000, 16, 50, 128)
    a = gpu_run(w, "mixed")
    b = gpu_run(w, "mixed")
    for k in ("F", "J", "nnb", "list", "ovf"):
        assert np.array_equal(a[k], b[k])


@pytest.mark.parametrize("mode", ["fp64", "mixed", "fp32"])
def test_back_to_back_calls_and_graph_replay(mode):
    """Predictor, regular force (split over several work items, so the merge
    runs) and irregular force back to back on one stream, three times over, and
    the predictor + force captured once into a CUDA graph (the split scratch
    already reserved by the earlier calls) and replayed: every output is
    bit-identical to a single call's and matches the oracle."""
    import torch
    n = 12000
    act = np.sort(np.random.default_rng(5).choice(n, 40, replace=False)).astype(np.int32)
    w = inputs.cluster(n, 17, 50, 128, act=act)
    d = upload(w)
    o = oracle_run(w)
    keys = ("F", "J", "nnb", "list", "ovf")

    def steps(ctx, stream):
        out = ctx.alloc_outputs(w.n_act, w.cap)
        for _ in range(3):
            ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t, stream=stream)
            ctx.regular_force(d["act"], d["h"], w.n, cap=w.cap, mode=mode, out=out, stream=stream)
            launches = ctx.last_launches()
            irr = ctx.irregular_force(d["act"], out["nnb"], out["list"], w.n, w.cap, mode=mode, stream=stream)
        assert ctx.sync_status(stream) == 0
        res = {k: out[k].cpu().numpy() for k in keys}
        res["irrF"], res["irrJ"] = irr["F"].cpu().numpy(), irr["J"].cpu().numpy()
        return res, launches

    with Context(n) as ctx:
        on, launches = steps(ctx, None)
        assert launches == 2, "the call should be split, so that the merge kernel runs"
        single = gpu_run(w, mode, ctx=ctx)
        for k in keys:
            assert np.array_equal(on[k], single[k]), k
        compare(on, o, w.cap, mode, lists=(mode != "fp32"))

        stream = torch.cuda.Stream()
        stream.wait_stream(torch.cuda.current_stream())
        out = ctx.alloc_outputs(w.n_act, w.cap)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            with torch.cuda.graph(graph, stream=stream):
                ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t, stream=stream)
                ctx.regular_force(d["act"], d["h"], w.n, cap=w.cap, mode=mode, out=out, stream=stream)
        for _ in range(2):
            out["F"].zero_(); out["list"].fill_(-1); out["nnb"].fill_(-5)
            graph.replay()
            torch.cuda.synchronize()
            assert ctx.sync_status() == 0
            for k in keys:
                assert np.array_equal(out[k].cpu().numpy(), on[k]), k


# -------------------------------------------------------- batched / graph

def _batch(nc=7, seed=40):
    rng = np.random.default_rng(seed)
    ws = []
    for c in range(nc):
        n = int(rng.integers(700, 3500))
        na = int(rng.integers(1, n))
        act = np.sort(rng.choice(n, na, replace=False)).astype(np.int32)
        ws.append(inputs.cluster(n, seed * 100 + c, 40, 128, act=act))
    return ws


@pytest.mark.parametrize("mode,even", [("fp64", False), ("mixed", False), ("mixed", True), ("fp32", True)])
def test_batched_plan_and_graph(mode, even):
    """Batched plan (one persistent launch + merge) and its CUDA-graph replay.
    Even slot offsets let the j-pair kernels serve the batch; odd ones take
    the per-particle layout."""
    import torch
    ws = _batch()
    offs = np.cumsum([0] + [w.n + 13 for w in ws])   # gaps between the clusters' slots
    if even:
        offs = offs + (offs % 2)
    with Context(int(offs[-1])) as ctx:
        keep, cl = [], []
        for w, off in zip(ws, offs):
            d = upload(w)
            ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t, offset=int(off))
            out = ctx.alloc_outputs(w.n_act, w.cap)
            keep.append((d, out))
            cl.append(B.nb_cluster(int(off), w.n, w.n_act, w.cap, d["act"].data_ptr(), d["h"].data_ptr(),
                                   None, out["F"].data_ptr(), out["J"].data_ptr(), None,
                                   out["nnb"].data_ptr(), out["list"].data_ptr(), out["ovf"].data_ptr()))
        plan = B.nb_plan_create(ctx.h, cl, mode_id(mode))
        try:
            B.nb_plan_run(plan, ctx=ctx.h)
            assert ctx.sync_status() == 0
            first = [{k: v.cpu().numpy() for k, v in out.items() if v is not None} for _, out in keep]
            for (w, g) in zip(ws, first):
                compare(g, oracle_run(w), w.cap, mode, lists=(mode != "fp32"))
            for _, out in keep:
                out["F"].zero_(); out["list"].fill_(-1); out["nnb"].fill_(-5)
            stream = torch.cuda.Stream()
            B.nb_plan_capture(plan, stream=stream, ctx=ctx.h)
            B.nb_plan_launch(plan, stream=stream, ctx=ctx.h)
            stream.synchronize()
            assert ctx.sync_status() == 0
            for (d, out), g in zip(keep, first):
                for k in ("F", "J", "nnb", "list", "ovf"):
                    assert np.array_equal(out[k].cpu().numpy(), g[k])
        finally:
            B.nb_plan_destroy(plan)


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_one_shot_batched_call_matches_the_plan(mode):
    """nb_regular_force_batched (plan built, run, waited for, freed) gives the
    outputs of an explicit plan bit for bit, and the oracle's."""
    ws = _batch(nc=5, seed=52)
    offs = np.cumsum([0] + [w.n + (w.n % 2) + 2 for w in ws])
    with Context(int(offs[-1])) as ctx:
        outs = []
        for rep in range(2):
            keep, cl = [], []
            for w, off in zip(ws, offs):
                d = upload(w)
                if rep == 0:
                    ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t, offset=int(off))
                out = ctx.alloc_outputs(w.n_act, w.cap)
                keep.append((d, out))
                cl.append(B.nb_cluster(int(off), w.n, w.n_act, w.cap, d["act"].data_ptr(), d["h"].data_ptr(),
                                       None, out["F"].data_ptr(), out["J"].data_ptr(), None,
                                       out["nnb"].data_ptr(), out["list"].data_ptr(), out["ovf"].data_ptr()))
            if rep == 0:
                B.nb_regular_force_batched(ctx.h, cl, mode_id(mode))
                assert ctx.last_launches() >= 1
            else:
                plan = B.nb_plan_create(ctx.h, cl, mode_id(mode))
                try:
                    B.nb_plan_run(plan, ctx=ctx.h)
                    assert ctx.sync_status() == 0
                finally:
                    B.nb_plan_destroy(plan)
            outs.append([{k: v.cpu().numpy() for k, v in out.items() if v is not None} for _, out in keep])
    for w, a, b in zip(ws, outs[0], outs[1]):
        for k in ("F", "J", "nnb", "list", "ovf"):
            assert np.array_equal(a[k], b[k]), k
        compare(a, oracle_run(w), w.cap, mode)


@pytest.mark.parametrize("mode,odd", [("mixed", False), ("mixed", True), ("fp64", True)])
def test_batched_plan_with_mixed_flags(mode, odd):
    """A plan whose clusters differ in flags: some with the velocity criterion,
    some with the potential, some with neither.  The plan runs one kernel with
    the union of the flags; each cluster must still get exactly its own
    criterion and outputs.  With odd slot offsets the plan takes the
    per-particle layout."""
    rng = np.random.default_rng(61)
    ws, vel, pot = [], [], []
    for c in range(6):
        n = int(rng.integers(600, 3000))
        act = np.sort(rng.choice(n, int(rng.integers(1, n)), replace=False)).astype(np.int32)
        v, q = c % 3 == 0, c % 2 == 1
        ws.append(inputs.cluster(n, 900 + c, 40, 64, act=act, dtr_steps=(2.0**-6, 2.0**-8) if v else None))
        vel.append(v)
        pot.append(q)
    offs = np.cumsum([0] + [w.n + 5 for w in ws])
    offs = offs + 1 if odd else offs + (offs % 2)
    with Context(int(offs[-1])) as ctx:
        keep, cl = [], []
        for w, off, q in zip(ws, offs, pot):
            d = upload(w)
            ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t, offset=int(off))
            out = ctx.alloc_outputs(w.n_act, w.cap, pot=q)
            keep.append((d, out))
            cl.append(B.nb_cluster(int(off), w.n, w.n_act, w.cap, d["act"].data_ptr(), d["h"].data_ptr(),
                                   d["dtr"].data_ptr() if d["dtr"] is not None else None,
                                   out["F"].data_ptr(), out["J"].data_ptr(),
                                   out["pot"].data_ptr() if q else None,
                                   out["nnb"].data_ptr(), out["list"].data_ptr(), out["ovf"].data_ptr()))
        plan = B.nb_plan_create(ctx.h, cl, mode_id(mode))
        try:
            B.nb_plan_run(plan, ctx=ctx.h)
            assert ctx.sync_status() == 0
            for (d, out), w, q in zip(keep, ws, pot):
                g = {k: v.cpu().numpy() for k, v in out.items() if v is not None}
                compare(g, oracle_run(w, pot=q), w.cap, mode, pot=q)
        finally:
            B.nb_plan_destroy(plan)


# Degenerate clusters in one plan: no active particle, one particle active,
# j-ranges of 5, 63, 64 and 65 slots (a single part-filled step), of 1023, 1024
# and 1025 (a tile boundary, the last tile holding one j) and 2049, a list cap
# that overflows, at even and odd slot offsets.  Every tiling family serves
# it, including j-splits of one tile, whose work lists leave CTAs with
# different item counts.
_EDGE = [(5, 5, 8), (63, 63, 16), (64, 1, 16), (65, 7, 16), (700, 0, 16), (1023, 500, 16),
         (1024, 1, 16), (1025, 1025, 4), (2049, 33, 16)]


@pytest.mark.parametrize("cfg,odd", [(None, False), (None, True), ((16, 2, 1024, 1, 9), False),
                                     ((16, 2, 1024, 1, 5), False), ((16, 2, 512, 2, 5), False),
                                     ((8, 2, 512, 1, 0), True)],
                         ids=["default-even", "default-odd", "list-warps-1-tile", "j-pair-1-tile",
                              "j-pair-512-2-tiles", "scalar-odd-1-tile"])
def test_plan_of_degenerate_clusters(cfg, odd):
    ws = []
    for c, (n, na, cap) in enumerate(_EDGE):
        act = np.sort(np.random.default_rng(300 + c).choice(n, max(na, 1), replace=False)).astype(np.int32)
        ws.append(inputs.cluster(n, 310 + c, min(8, n - 2), cap, act=act))
    gaps = [w.n + 3 for w in ws]
    offs = np.cumsum([0] + gaps)
    offs = offs + 1 if odd else offs + (offs % 2)
    with Context(int(offs[-1]) + 1) as ctx:
        keep, cl = [], []
        for (n, na, cap), w, off in zip(_EDGE, ws, offs):
            d = upload(w)
            ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t, offset=int(off))
            out = ctx.alloc_outputs(max(na, 1), w.cap)
            keep.append((d, out))
            cl.append(B.nb_cluster(int(off), w.n, na, w.cap, d["act"].data_ptr(), d["h"].data_ptr(), None,
                                   out["F"].data_ptr(), out["J"].data_ptr(), None, out["nnb"].data_ptr(),
                                   out["list"].data_ptr(), out["ovf"].data_ptr()))
        plan = B.nb_plan_create(ctx.h, cl, B.NB_MIXED, None if cfg is None else B.nb_kcfg(*cfg))
        try:
            if cfg is not None:
                assert B.nb_plan_get_config(plan).as_tuple() == cfg
            for _, out in keep:
                out["F"].fill_(7.0); out["list"].fill_(-1); out["nnb"].fill_(-5)
            B.nb_plan_run(plan, ctx=ctx.h)
            assert ctx.sync_status() == 0
            got = [{k: v.cpu().numpy() for k, v in out.items() if v is not None} for _, out in keep]
        finally:
            B.nb_plan_destroy(plan)
    for (n, na, cap), w, g in zip(_EDGE, ws, got):
        if na == 0:
            assert g["nnb"][0] == -5 and np.all(g["F"][0] == 7.0)   # nothing written for an empty active set
            continue
        x, v = oracle_predicted(w)
        SF, SJ = oracle.regular_mag(x, v, w.m, w.act, w.h)
        o = oracle_run(w)
        compare_conditioned(g, o, SF, SJ, w.cap, "mixed")
        if n == 1025:
            assert np.any(o["ovf"] == 1)   # the cap of 4 overflows


def test_tail_split_call():
    """A call whose i-blocks fill four rounds of the persistent grid and part of
    a fifth (16384 of N = 16384 active in the list-warp tiling's 24-particle
    i-blocks) runs the whole rounds with unsplit j-ranges and the remaining
    i-blocks with split ones: three launches (two force kernels and the merge),
    every row against the oracle, and the scratch estimate covers the split
    part."""
    n = 16384
    w = inputs.cluster(n, 4242, 64, 256)
    with Context(n) as ctx:
        d = upload(w)
        ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t)
        ctx.set_config("mixed", B.nb_kcfg(16, 2, 1024, 0, 9))
        out = ctx.alloc_outputs(w.n_act + 1, w.cap)
        for k in ("F", "J"):
            out[k].fill_(7.0)
        out["nnb"].fill_(-9)
        view = {k: (v[:w.n_act] if v is not None else None) for k, v in out.items()}
        ctx.regular_force(d["act"], d["h"], w.n, cap=w.cap, mode="mixed", out=view)
        assert ctx.sync_status() == 0
        assert ctx.last_launches() == 3
        assert ctx.scratch_bytes(w.n, w.n_act, w.cap, "mixed") > 0
        g = {k: v.cpu().numpy() for k, v in out.items() if v is not None}
    assert np.all(g["F"][w.n_act] == 7.0) and g["nnb"][w.n_act] == -9   # the guard row is untouched
    compare({k: v[:w.n_act] for k, v in g.items()}, oracle_run(w), w.cap, "mixed")


def test_tail_split_call_captured_after_reserving_its_scratch():
    """The scratch estimate of a call that runs as two parts is enough to
    capture its first run in a CUDA graph: after nb_reserve(nb_scratch_bytes(..))
    the capture needs no allocation, and two replays give an eager call's
    outputs bit for bit (and the oracle's within the two-float tolerances)."""
    import torch
    n = 16384
    w = inputs.cluster(n, 4243, 64, 256)
    keys = ("F", "J", "nnb", "list", "ovf")
    with Context(n) as ctx:
        d = upload(w)
        ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t)
        # the kernel's launch attributes, set by a call of the same tiling that needs no split scratch
        ctx.set_config("mixed", B.nb_kcfg(16, 2, 1024, 16, 9))
        ctx.regular_force(d["act"][:24], d["h"][:24], w.n, cap=w.cap, mode="mixed")
        assert ctx.sync_status() == 0 and ctx.last_launches() == 1
        ctx.set_config("mixed", B.nb_kcfg(16, 2, 1024, 0, 9))
        need = ctx.scratch_bytes(w.n, w.n_act, w.cap, "mixed")
        assert need > 0
        ctx.reserve(need)
        stream = torch.cuda.Stream()
        stream.wait_stream(torch.cuda.current_stream())
        out = ctx.alloc_outputs(w.n_act, w.cap)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            with torch.cuda.graph(graph, stream=stream):
                ctx.regular_force(d["act"], d["h"], w.n, cap=w.cap, mode="mixed", out=out, stream=stream)
        assert ctx.last_launches() == 3
        for _ in range(2):
            out["F"].zero_(); out["list"].fill_(-1); out["nnb"].fill_(-5)
            graph.replay()
            torch.cuda.synchronize()
            assert ctx.sync_status() == 0
        got = {k: out[k].cpu().numpy() for k in keys}
        eager = gpu_run(w, "mixed", ctx=ctx)
    for k in keys:
        assert np.array_equal(got[k], eager[k]), k
    compare(got, oracle_run(w), w.cap, "mixed")


# ------------------------------------------------------------- host step

def test_host_step_matches_oracle():
    import torch
    w = inputs.cluster(8000, 17, 48, 128, act=np.arange(0, 8000, 3, dtype=np.int32))
    pin = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).pin_memory()
    hx = {k: pin(getattr(w, k)) for k in ("x0", "v0", "a0", "adot0", "m", "t0", "h")}
    act = pin(w.act, torch.int32)
    F = torch.empty((w.n_act, 3), dtype=torch.float64).pin_memory()
    J = torch.empty_like(F)
    nnb = torch.empty(w.n_act, dtype=torch.int32).pin_memory()
    lst = torch.full((w.n_act, w.cap), -1, dtype=torch.int32).pin_memory()
    ovf = torch.empty(w.n_act, dtype=torch.uint8).pin_memory()
    with Context(w.n) as ctx:
        B.nb_step_host(ctx.h, w.n, hx["x0"], hx["v0"], hx["a0"], hx["adot0"], hx["m"], hx["t0"], w.t, w.n_act,
                       act, hx["h"], None, w.cap, B.NB_MIXED, F, J, None, nnb, lst, ovf)
    g = {"F": F.numpy(), "J": J.numpy(), "nnb": nnb.numpy(), "list": lst.numpy(), "ovf": ovf.numpy()}
    compare(g, oracle_run(w), w.cap, "mixed")


@pytest.mark.parametrize("flags", [False, True])
def test_host_step_in_chunks_matches_the_device_call(flags):
    """A large active set goes through nb_step_host in chunks (98304 active on a
    152-SM GB300: chunks of 8, 9 and 9 rounds of the persistent grid, then the
    last, part-filled round alone), each chunk's results copied back while the
    next computes: outputs are bit-identical to one device call on the same
    inputs, and match the oracle on sampled rows; with `flags` the call also
    uses the velocity criterion and returns the potential."""
    import torch
    w = inputs.cluster(100000, 19, 48, 128, act=np.arange(0, 98304, dtype=np.int32),
                       dtr_steps=(2.0**-6, 2.0**-8) if flags else None)
    pin = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).pin_memory()
    hx = {k: pin(getattr(w, k)) for k in ("x0", "v0", "a0", "adot0", "m", "t0", "h")}
    act = pin(w.act, torch.int32)
    dtr = pin(w.dtr) if flags else None
    F = torch.empty((w.n_act, 3), dtype=torch.float64).pin_memory()
    J = torch.empty_like(F)
    pot = torch.empty(w.n_act, dtype=torch.float64).pin_memory() if flags else None
    nnb = torch.empty(w.n_act, dtype=torch.int32).pin_memory()
    lst = torch.zeros((w.n_act, w.cap), dtype=torch.int32).pin_memory()
    ovf = torch.empty(w.n_act, dtype=torch.uint8).pin_memory()
    with Context(w.n) as ctx:
        B.nb_step_host(ctx.h, w.n, hx["x0"], hx["v0"], hx["a0"], hx["adot0"], hx["m"], hx["t0"], w.t, w.n_act,
                       act, hx["h"], dtr, w.cap, B.NB_MIXED, F, J, pot, nnb, lst, ovf)
        assert ctx.last_launches() >= 3, "prediction and at least two force launches"
        one = gpu_run(w, "mixed", ctx=ctx, pot=flags)
    g = {"F": F.numpy(), "J": J.numpy(), "nnb": nnb.numpy(), "list": lst.numpy(), "ovf": ovf.numpy()}
    if flags:
        g["pot"] = pot.numpy()
    for k in g:
        assert np.array_equal(g[k], one[k]), k
    rows = np.sort(np.random.default_rng(3).choice(w.n_act, 256, replace=False))
    compare(g, oracle_run(w, rows=rows, pot=flags), w.cap, "mixed", rows=rows, pot=flags)


# ------------------------------------------------- device-side error paths

def test_invalid_device_inputs_are_reported_not_faulted():
    import torch
    w = inputs.cluster(2000, 18, 20, 64, act=np.arange(0, 2000, 10, dtype=np.int32))
    with Context(w.n) as ctx:
        d = upload(w)
        ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t)
        bad = d["act"].clone()
        bad[3] = w.n + 5          # out of range
        bad[7] = -1
        h = d["h"].clone()
        h[11] = -1.0              # negative radius
        h[12] = float("nan")
        out = ctx.regular_force(bad, h, w.n, cap=w.cap, mode="mixed")
        assert ctx.sync_status() == B.NB_ERR_DEVICE_INPUT
        # the context stays usable and the valid particles are still right
        good = ctx.regular_force(d["act"], d["h"], w.n, cap=w.cap, mode="mixed")
        assert ctx.sync_status() == 0
        g = {k: v.cpu().numpy() for k, v in good.items() if v is not None}
        compare(g, oracle_run(w), w.cap, "mixed")
        o = {k: v.cpu().numpy() for k, v in out.items() if v is not None}
        ok = np.setdiff1d(np.arange(w.n_act), [3, 7, 11, 12])
        assert np.array_equal(o["nnb"][ok], g["nnb"][ok])


def test_bounded_wait_times_out_cleanly():
    """A copy barrier that can never complete (the test hook asks for more
    bytes than are copied): every wait gives up after its bound, the kernel
    returns and the status says NB_ERR_TIMEOUT; afterwards the context works."""
    w = inputs.cluster(3000, 19, 20, 64, act=np.arange(0, 3000, 50, dtype=np.int32))
    with Context(w.n) as ctx:
        d = upload(w)
        ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t)
        B.nb_debug_set_wait(ctx.h, 20_000_000, 16)        # 20 ms bound, 16 bytes never arrive
        ctx.regular_force(d["act"], d["h"], w.n, cap=w.cap, mode="mixed")
        assert ctx.sync_status() == B.NB_ERR_TIMEOUT
        B.nb_debug_set_wait(ctx.h, 0, 0)
        out = ctx.regular_force(d["act"], d["h"], w.n, cap=w.cap, mode="mixed")
        assert ctx.sync_status() == 0
        g = {k: v.cpu().numpy() for k, v in out.items() if v is not None}
        compare(g, oracle_run(w), w.cap, "mixed")


def test_argument_errors_are_host_side():
    w = inputs.cluster(500, 20, 8, 16)
    with Context(w.n) as ctx:
        d = upload(w)
        with pytest.raises(B.NbError) as e:      # nothing predicted yet
            ctx.regular_force(d["act"], d["h"], w.n, cap=16, mode="mixed")
        assert e.value.status == B.NB_ERR_STATE
        ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t, forms=B.NB_FORM_MIXED)
        with pytest.raises(B.NbError) as e:      # FP64 form not written
            ctx.regular_force(d["act"], d["h"], w.n, cap=16, mode="fp64")
        assert e.value.status == B.NB_ERR_STATE
        with pytest.raises(B.NbError) as e:      # j-range past the context
            ctx.regular_force(d["act"], d["h"], w.n + 1, cap=16, mode="mixed")
        assert e.value.status == B.NB_ERR_ARG


# ------------------------------------------------------------ full sizes

@pytest.fixture(scope="module")
def cfg3():
    return inputs.cached(inputs.config3)


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_config3_kroupa_131072_active_2048(cfg3, mode):
    w = inputs.subset(cfg3, 2048, 3)
    g = gpu_run(w, mode)
    assert g["status"] == 0
    compare(g, oracle_run(w), w.cap, mode)


@pytest.fixture(scope="module")
def cfg3_oracle(cfg3):
    """The oracle on every row of the benchmark's workload (1.7e10 FP64
    interactions, OpenMP over all host cores)."""
    return oracle_run(cfg3)


@pytest.mark.parametrize("tiling", [None, (16, 2, 1536, 0, 14)], ids=["default", "exact_pair"])
def test_config3_all_active_every_row(cfg3, cfg3_oracle, tiling):
    """The benchmark's workload (N = n_act = 131072, two-float form) in the
    launch configuration the benchmark times (the default tiling, which the
    autotuner also picks at this size) and in the exact pair form: every one
    of the 131072 rows against the oracle, element by element (force, jerk,
    count, overflow flag and every list entry), and every particle's count
    equal to the count its radius was built for."""
    w = cfg3
    g = gpu_run(w, "mixed", cfg=None if tiling is None else B.nb_kcfg(*tiling))
    assert g["status"] == 0
    assert np.array_equal(g["nnb"], w.meta["K"])
    eF, eJ = compare(g, cfg3_oracle, w.cap, "mixed")
    print(f"all {w.n_act} rows: force max {eF.max():.2e} rms {np.sqrt((eF ** 2).mean()):.2e}, "
          f"jerk max {eJ.max():.2e} rms {np.sqrt((eJ ** 2).mean()):.2e}")


@pytest.fixture(scope="module")
def cfg5():
    return inputs.cached(inputs.config5)


def test_config5_offset_hard_pairs(cfg5):
    """|x_c| = 1e3 and 10% hard pairs: the two-float and FP64 forms keep exact
    lists; the plain FP32 form is only reported (it is expected to lose them)."""
    w = inputs.subset(cfg5, 4096, 5)
    o = oracle_run(w)
    for mode in ("fp64", "mixed"):
        g = gpu_run(w, mode)
        assert g["status"] == 0
        compare(g, o, w.cap, mode)
    g = gpu_run(w, "fp32")
    print("fp32 list mismatches at offset 1e3:", list_mismatches(g, o, w.cap),
          "max force err", rel_err(g["F"], o["F"]).max())


# ---------------------------------------------------------- framed kernel

@pytest.mark.parametrize("offset,pairs", [(0.0, 0.0), (1e3, 0.1)])
def test_framed_two_float_kernel(offset, pairs):
    """Morton-sorted active set with frame coordinates for compact blocks: exact
    lists and the two-float tolerances, also with a 1e3 centre offset and hard
    pairs; most blocks of an all-active set are compact."""
    w = inputs.cluster(20000, 31, 64, 256, offset=offset, pair_frac=pairs)
    framed = None
    for i in range(B.nb_num_kernel_configs(B.NB_MIXED)):
        c = B.nb_get_kernel_config(B.NB_MIXED, i)
        if c.packed == 4:
            framed = c
            break
    assert framed is not None
    with Context(w.n) as ctx:
        g = gpu_run(w, "mixed", ctx=ctx, cfg=framed)
        compact, blocks = B.nb_debug_frame_stats(ctx.h)
    assert g["status"] == 0
    assert blocks == (w.n_act + framed.warps * framed.ipw - 1) // (framed.warps * framed.ipw)
    print("compact blocks", compact, "of", blocks)
    assert compact > 0.5 * blocks, (compact, blocks)
    compare(g, oracle_run(w), w.cap, "mixed")


def test_default_mixed_kernel_is_two_float_positions(cfg2):
    """Unless configured otherwise, two-float calls run the j-pair kernel with
    two-float positions and FP32 velocity differences and four list warps
    (tiling packed = 5 + 4)."""
    with Context(cfg2.n) as ctx:
        g = gpu_run(cfg2, "mixed", ctx=ctx)
        c = ctx.active_config("mixed")
        assert c.packed == 9 and c.warps == 16
    # the force kernel (two when whole grid rounds run unsplit before a split
    # remainder) and the merge of j-splits; no sort (which adds ten launches)
    assert g["launches"] <= 3
    compare(g, oracle_run(cfg2), cfg2.cap, "mixed")


# velocity dispersion (1D) of the Henon-unit Plummer sphere: sqrt(1/6)
SIGMA = 6.0 ** -0.5


@pytest.mark.parametrize("bulk", [1.0, 4.0, 100.0])
def test_two_float_positions_with_bulk_velocity(bulk):
    """A cluster moving at `bulk` velocity dispersions through the caller's
    frame: the predictor stores the float forms' velocities relative to the
    cluster's own frame velocity, so the FP32 velocity differences of the
    default kernels (packed 5 and, with list warps, 9) meet the two-float
    tolerances with exact lists at 100 dispersions as at rest; so does the
    exact pair form (packed = 2)."""
    u = np.array([1.0, -0.5, 0.25])
    w = inputs.cluster(8192, 37, 64, 256, bulk_v=bulk * SIGMA * u / np.linalg.norm(u))
    o = oracle_run(w)
    for cfg in (B.nb_kcfg(16, 2, 512, 0, 5), B.nb_kcfg(16, 2, 512, 0, 2), None):   # None: the default (9)
        g = gpu_run(w, "mixed", cfg=cfg)
        assert g["status"] == 0
        compare(g, o, w.cap, "mixed")


def test_frame_velocity_is_the_sampled_mean_and_matters():
    """The frame velocity is the mean start velocity of 32 particles spread
    evenly over the predicted range; predicting the same moving cluster with
    a zero frame instead (nb_set_frame + NB_KEEP_FRAME: FP32 velocities in the
    caller's frame, as without the frame) loses the jerk tolerance of the
    default form at 100 dispersions, so the test above does depend on the
    frame."""
    u = np.array([1.0, -0.5, 0.25])
    bulk = 100.0 * SIGMA * u / np.linalg.norm(u)
    w = inputs.cluster(8192, 37, 64, 256, bulk_v=bulk)
    o = oracle_run(w)
    with Context(w.n) as ctx:
        d = upload(w)
        ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t)
        k = (np.arange(32) * w.n) // 32
        want = w.v0[k].astype(np.float32).astype(np.float64).mean(axis=0)
        got = np.array(B.nb_get_frame(ctx.h))
        assert np.allclose(got, want, rtol=0, atol=1e-4), (got, want)
        g_frame = gpu_run(w, "mixed", ctx=ctx)
        B.nb_set_frame(ctx.h, [0.0, 0.0, 0.0])
        g_zero = gpu_run(w, "mixed", ctx=ctx, forms=B.NB_FORM_MIXED | B.NB_KEEP_FRAME)
        assert B.nb_get_frame(ctx.h) == [0.0, 0.0, 0.0]
    eJ_frame = rel_err(g_frame["J"], o["J"]).max()
    eJ_zero = rel_err(g_zero["J"], o["J"]).max()
    print(f"jerk error at 100 dispersions: frame {eJ_frame:.2e}, zero frame {eJ_zero:.2e}")
    assert eJ_frame <= TOL["mixed"][1] < eJ_zero


def test_a_range_predicted_under_two_frames_is_refused():
    """Two halves of one cluster predicted in separate calls each get their
    own frame; a force call over both halves is refused (NB_ERR_STATE) rather
    than mixing them.  With NB_KEEP_FRAME on the second call the halves share
    the first call's frame and the call matches the oracle."""
    import torch
    w = inputs.cluster(4000, 38, 32, 64, bulk_v=[3.0, 0.0, 0.0])
    o = oracle_run(w)
    half = w.n // 2
    with Context(w.n) as ctx:
        d = upload(w)
        sl = lambda k, a, b: d[k][a:b]
        for keep in (0, B.NB_KEEP_FRAME):
            ctx.predict(*(sl(k, 0, half) for k in ("x0", "v0", "a0", "adot0", "m", "t0")), w.t, offset=0)
            ctx.predict(*(sl(k, half, w.n) for k in ("x0", "v0", "a0", "adot0", "m", "t0")), w.t, offset=half,
                        forms=keep)
            if not keep:
                with pytest.raises(B.NbError) as e:
                    ctx.regular_force(d["act"], d["h"], w.n, cap=w.cap, mode="mixed")
                assert e.value.status == B.NB_ERR_STATE and "frame" in str(e.value)
                # the FP64 form holds velocities in the caller's frame and is unaffected
                g64 = ctx.regular_force(d["act"], d["h"], w.n, cap=w.cap, mode="fp64")
                assert ctx.sync_status() == 0
                compare({k: v.cpu().numpy() for k, v in g64.items() if v is not None}, o, w.cap, "fp64")
                # a call inside one half is fine
                ctx.regular_force(d["act"][:10], d["h"][:10], half, cap=w.cap, mode="mixed")
                assert ctx.sync_status() == 0
            else:
                g = ctx.regular_force(d["act"], d["h"], w.n, cap=w.cap, mode="mixed")
                assert ctx.sync_status() == 0
                compare({k: v.cpu().numpy() for k, v in g.items() if v is not None}, o, w.cap, "mixed")