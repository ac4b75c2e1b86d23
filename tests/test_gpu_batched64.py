"""The batched many-cluster launch at full size: the 64 independent clusters
of the batched workload (N log-uniform in [1024, 32768], n_act log-uniform in
[8, N], seed 4) in one plan, tuned by the plan autotuner and replayed from a
CUDA graph, against the oracle on every row of every cluster, and against one
nb_regular_force call per cluster.

These 122906 rows include particles near a cluster's centre, whose regular
force cancels to 1/194 of the sum of its term lengths, and rows whose regular
jerk cancels to 1/1440 of it; there the per-particle relative bar (1e-6 force,
1e-5 jerk) is out of reach of any FP32 pair term, and such a row is held to
u * S (u = 2^-24, S = the oracle's sum of term lengths) instead.  The FP64
form meets its relative bar on every row."""
import numpy as np
import pytest

import oracle
from paper_1205_1222_gb300 import Context, binding as B, build, inputs, mode_id
from tests.gpu_util import compare, compare_conditioned, oracle_predicted, oracle_run, upload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cfg4():
    build.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return inputs.cached(inputs.config4)


@pytest.fixture(scope="module")
def cfg4_oracle(cfg4):
    """Oracle outputs and term-length sums (force, jerk) of every cluster."""
    res = []
    for w in cfg4:
        x, v = oracle_predicted(w)
        SF, SJ = oracle.regular_mag(x, v, w.m, w.act, w.h)
        res.append((oracle_run(w), SF, SJ))
    return res


def _setup(ctx, ws, offs):
    keep, cl = [], []
    for w, off in zip(ws, offs):
        d = upload(w)
        # each cluster predicted in its own call: its own velocity frame
        ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t, offset=int(off))
        out = ctx.alloc_outputs(w.n_act, w.cap)
        keep.append((d, out))
        cl.append(B.nb_cluster(int(off), w.n, w.n_act, w.cap, d["act"].data_ptr(), d["h"].data_ptr(), None,
                               out["F"].data_ptr(), out["J"].data_ptr(), None, out["nnb"].data_ptr(),
                               out["list"].data_ptr(), out["ovf"].data_ptr()))
    return keep, cl


def _host(keep):
    return [{k: v.cpu().numpy() for k, v in out.items() if v is not None} for _, out in keep]


def test_batched64_tuned_graph_matches_oracle_and_per_cluster_calls(cfg4, cfg4_oracle):
    import torch
    ws = cfg4
    assert len(ws) == 64
    offs = np.cumsum([0] + [w.n + (w.n % 2) for w in ws])   # even slots: the j-pair kernels serve the plan
    with Context(int(offs[-1])) as ctx:
        keep, cl = _setup(ctx, ws, offs)
        stream = torch.cuda.Stream()
        stream.wait_stream(torch.cuda.current_stream())
        plan = B.nb_plan_create(ctx.h, cl, B.NB_MIXED)
        try:
            before = B.nb_plan_get_config(plan).as_tuple()
            best, ms = B.nb_plan_autotune(plan, reps=2, stream=stream, ctx=ctx.h)
            assert ms > 0 and B.nb_plan_get_config(plan).as_tuple() == best.as_tuple()
            print("plan tiling", before, "-> tuned", best.as_tuple(), f"{ms:.3f} ms")
            rows = [r for r in B.nb_tuned_table(ctx.h) if r.flags & 4]
            assert len(rows) == 1 and rows[0].cfg.as_tuple() == best.as_tuple()
            for _, out in keep:
                out["F"].zero_(); out["list"].fill_(-1); out["nnb"].fill_(-5)
            B.nb_plan_capture(plan, stream=stream, ctx=ctx.h)
            for _ in range(2):
                B.nb_plan_launch(plan, stream=stream, ctx=ctx.h)
            stream.synchronize()
            assert ctx.sync_status() == 0
            graph = _host(keep)
        finally:
            B.nb_plan_destroy(plan)
        # a new plan of the same clusters takes the tuned tiling from the table
        plan2 = B.nb_plan_create(ctx.h, cl, B.NB_MIXED)
        try:
            assert B.nb_plan_get_config(plan2).as_tuple() == best.as_tuple()
        finally:
            B.nb_plan_destroy(plan2)
        for (d, out), w, off in zip(keep, ws, offs):
            B.nb_regular_force(ctx.h, int(off), w.n, w.n_act, d["act"], d["h"], None, w.cap, B.NB_MIXED, out["F"],
                               out["J"], None, out["nnb"], out["list"], out["ovf"])
        assert ctx.sync_status() == 0
        single = _host(keep)
    beyond = []
    for c, (w, g, s, (o, SF, SJ)) in enumerate(zip(ws, graph, single, cfg4_oracle)):
        for k in ("nnb", "list", "ovf"):
            assert np.array_equal(g[k], s[k]), k
        beyond += [(c,) + r for r in compare_conditioned(g, o, SF, SJ, w.cap, "mixed")]
    print(f"64 clusters, {sum(w.n_act for w in ws)} rows: {len(beyond)} beyond the relative bar, within u*S:")
    for r in beyond:
        print("  cluster %d row %d: force %.2e (cond %.0f), jerk %.2e (cond %.0f)" % r)
    assert len(beyond) <= 20


def test_batched64_fp64_plan_meets_the_relative_bar_on_every_row(cfg4):
    ws = cfg4
    offs = np.cumsum([0] + [w.n for w in ws])
    with Context(int(offs[-1])) as ctx:
        keep, cl = _setup(ctx, ws, offs)
        plan = B.nb_plan_create(ctx.h, cl, B.NB_FP64)
        try:
            B.nb_plan_run(plan, ctx=ctx.h)
            assert ctx.sync_status() == 0
        finally:
            B.nb_plan_destroy(plan)
        got = _host(keep)
    for w, g in zip(ws, got):
        compare(g, oracle_run(w), w.cap, "fp64")


# Short j-splits make a plan of many more work items than CTAs, of mixed
# lengths (a cluster's last split is shorter), which the host deals to the
# CTAs longest first: the CTAs then run different numbers of items and leave
# the last slots of their work list empty, and every split cluster goes
# through the merge.  One tiling per kernel family: the list-warp kernel, the
# j-pair kernel with inline lists, and the scalar per-particle kernel.
@pytest.mark.parametrize("cfg", [(16, 2, 1024, 3, 9), (16, 2, 1024, 4, 5), (8, 2, 512, 6, 0)],
                         ids=["list-warps-3-tiles", "j-pair-4-tiles", "scalar-6-tiles"])
def test_batched64_split_plans_match_oracle(cfg4, cfg4_oracle, cfg):
    ws = cfg4
    offs = np.cumsum([0] + [w.n + (w.n % 2) for w in ws])
    with Context(int(offs[-1])) as ctx:
        keep, cl = _setup(ctx, ws, offs)
        plan = B.nb_plan_create(ctx.h, cl, B.NB_MIXED, B.nb_kcfg(*cfg))
        try:
            assert B.nb_plan_get_config(plan).as_tuple() == cfg
            assert B.nb_plan_launches(plan) == 2   # the force kernel and the merge
            for _, out in keep:
                out["F"].zero_(); out["list"].fill_(-1); out["nnb"].fill_(-5)
            B.nb_plan_run(plan, ctx=ctx.h)
            assert ctx.sync_status() == 0
            got = _host(keep)
        finally:
            B.nb_plan_destroy(plan)
    beyond = 0
    for w, g, (o, SF, SJ) in zip(ws, got, cfg4_oracle):
        beyond += len(compare_conditioned(g, o, SF, SJ, w.cap, "mixed"))
    assert beyond <= 20
