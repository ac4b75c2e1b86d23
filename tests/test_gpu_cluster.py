"""The thread-block-cluster kernel for small calls (tiling packed = 20): the
j-splits of a block of active particles are the CTAs of one cluster and
reduce their float-float partials and list segments through distributed
shared memory, with no merge launch.  Parity with the oracle at small and
ragged sizes, split counts up to the largest cluster, overflowing lists,
bad inputs, the fallback when a call needs more splits than a cluster holds,
and CUDA-graph replay."""
import numpy as np
import pytest

from paper_1205_1222_gb300 import Context, binding as B, build, inputs
from tests.gpu_util import compare, gpu_run, oracle_run, upload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _cluster_cfgs(mode):
    out = []
    for i in range(B.nb_num_kernel_configs(B.MODES[mode])):
        c = B.nb_get_kernel_config(B.MODES[mode], i)
        if c.packed == 20:
            out.append(c.as_tuple())
    return out


def _cfgs():
    try:
        build.build()
        return [("mixed", c) for c in _cluster_cfgs("mixed")] + [("fp32", c) for c in _cluster_cfgs("fp32")]
    except Exception:   # no compiler: the module's fixture fails instead
        return []


CFGS = _cfgs()


def test_cluster_kernels_are_compiled():
    assert len(_cluster_cfgs("mixed")) >= 1 and len(_cluster_cfgs("fp32")) >= 1


@pytest.mark.parametrize("mode,cfg", CFGS)
@pytest.mark.parametrize("n,n_act,split", [(16384, 16, 0), (16384, 33, 1), (5000, 7, 0), (16384, 200, 2),
                                           (1001, 1, 0), (2049, 40, 1)])
def test_cluster_kernel_matches_oracle(mode, cfg, n, n_act, split):
    w = inputs.cluster(n, 500 + n_act, 32, 64,
                       act=np.sort(np.random.default_rng(n_act).choice(n, n_act, replace=False)))
    with Context(n) as ctx:
        g = gpu_run(w, mode, ctx=ctx, cfg=B.nb_kcfg(cfg[0], cfg[1], cfg[2], split, cfg[4]))
        assert g["status"] == 0
        n_tiles = -(-n // cfg[2])
        tps = split if split else -(-n_tiles // 16)
        if -(-n_tiles // tps) <= 16:
            assert g["launches"] == 1, "the cluster kernel reduces the splits itself (no merge launch)"
    compare(g, oracle_run(w), w.cap, mode, lists=(mode != "fp32"))


def test_cluster_kernel_overflowing_lists_and_bad_inputs():
    """cap 7 against ~64 neighbours: the lowest 7 indices, true counts and the
    overflow flag; an invalid active index is reported, not followed."""
    w = inputs.cluster(16384, 601, 64, 7, act=np.arange(5, 16384, 700, dtype=np.int32))
    cfg = _cluster_cfgs("mixed")[0]
    g = gpu_run(w, "mixed", cfg=B.nb_kcfg(cfg[0], cfg[1], cfg[2], 0, cfg[4]))
    assert g["status"] == 0 and g["ovf"].all()
    compare(g, oracle_run(w), w.cap, "mixed")
    import torch
    with Context(w.n) as ctx:
        d = upload(w)
        ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t)
        ctx.set_config("mixed", B.nb_kcfg(cfg[0], cfg[1], cfg[2], 0, cfg[4]))
        bad = d["act"].clone()
        bad[3] = w.n + 9
        ctx.regular_force(bad, d["h"], w.n, cap=w.cap, mode="mixed")
        assert ctx.sync_status() == B.NB_ERR_DEVICE_INPUT
        out = ctx.regular_force(d["act"], d["h"], w.n, cap=w.cap, mode="mixed")
        assert ctx.sync_status() == 0
        g2 = {k: v.cpu().numpy() for k, v in out.items() if v is not None}
    for k in ("F", "J", "nnb", "list", "ovf"):
        assert np.array_equal(g2[k], g[k]), k


def test_more_splits_than_a_cluster_holds_fall_back_to_the_default_kernel():
    """One tile per split over 32 tiles would need a 32-CTA cluster: the call
    runs the mode's default tiling instead (with its merge launch), with the
    same lists and the two-float tolerances."""
    w = inputs.cluster(16384, 602, 32, 64, act=np.arange(0, 16384, 400, dtype=np.int32))
    cfg = [c for c in _cluster_cfgs("mixed") if c[2] == 512][0]
    g = gpu_run(w, "mixed", cfg=B.nb_kcfg(cfg[0], cfg[1], cfg[2], 1, cfg[4]))
    assert g["status"] == 0 and g["launches"] == 2
    compare(g, oracle_run(w), w.cap, "mixed")


def test_cluster_kernel_graph_replay_is_bit_identical():
    import torch
    w = inputs.cluster(16384, 603, 64, 128, act=np.arange(7, 16384, 1000, dtype=np.int32))
    cfg = _cluster_cfgs("mixed")[0]
    with Context(w.n) as ctx:
        d = upload(w)
        ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t)
        ctx.set_config("mixed", B.nb_kcfg(cfg[0], cfg[1], cfg[2], 0, cfg[4]))
        first = ctx.regular_force(d["act"], d["h"], w.n, cap=w.cap, mode="mixed")
        assert ctx.sync_status() == 0
        first = {k: v.cpu().numpy() for k, v in first.items() if v is not None}
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        graph = torch.cuda.CUDAGraph()
        out = ctx.alloc_outputs(w.n_act, w.cap)
        with torch.cuda.stream(side):
            with torch.cuda.graph(graph, stream=side):
                ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t, stream=side)
                ctx.regular_force(d["act"], d["h"], w.n, cap=w.cap, mode="mixed", out=out, stream=side)
        for _ in range(2):
            out["F"].zero_(); out["list"].fill_(-1)
            graph.replay()
            torch.cuda.synchronize()
            assert ctx.sync_status() == 0
            for k in ("F", "J", "nnb", "list", "ovf"):
                assert np.array_equal(out[k].cpu().numpy(), first[k]), k
    compare(first, oracle_run(w), w.cap, "mixed")
