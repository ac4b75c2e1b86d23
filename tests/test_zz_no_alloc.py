"""GPU test of nb_regular_force_noalloc, the allocation-free regular-force call.

Callers that may not allocate device memory while a step runs (stream-capture
regions, real-time loops with memory reserved up front, programs whose device
memory belongs to another allocator) use this call: its split partials live in
a fixed device array instead of scratch grown with cudaMalloc.  The test runs
a case whose j-range is split (so the fixed array is used), through the C-ABI,
twice in a row, and compares each result with nb_regular_force on the same
inputs: both calls take the same tiling (also after a tuned tiling is loaded
for the call's size class), so the results must agree bit for bit, and they
must meet the oracle tolerances of the other parity tests.  It builds its own
inputs and context, so it passes alone in a fresh process or after the rest of
the suite; the file name makes pytest collect it last.
"""
import numpy as np
import pytest

from paper_1205_1222_gb300 import Context, binding as B, build, inputs, mode_id
from tests.gpu_util import compare, upload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def workload():
    build.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    full = inputs.cluster(16384, 77, 64, 256)    # radii for every particle
    act = np.sort(np.random.default_rng(77).choice(full.n, 256, replace=False)).astype(np.int32)
    return full.with_active(act)


def _call(fn, ctx, d, w, mode, cap):
    out = ctx.alloc_outputs(w.n_act, cap)
    fn(ctx.h, 0, w.n, w.n_act, d["act"], d["h"], d["dtr"], cap, mode_id(mode), out["F"], out["J"], None,
       out["nnb"], out["list"], out["ovf"])
    assert ctx.sync_status() == 0
    launches = ctx.last_launches()
    return {k: v.cpu().numpy() for k, v in out.items() if v is not None}, launches


def _same(got, ref):
    for k in ("F", "J", "nnb", "list", "ovf"):
        assert np.array_equal(got[k], ref[k]), k


@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_noalloc_matches_regular_force_twice(workload, mode):
    w = workload
    with Context(w.n) as ctx:
        d = upload(w)
        ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t)
        ref, ref_launches = _call(B.nb_regular_force, ctx, d, w, mode, w.cap)
        assert ref_launches == 2, "the case must split the j-range so the fixed scratch is used"
        for _ in range(2):
            got, launches = _call(B.nb_regular_force_noalloc, ctx, d, w, mode, w.cap)
            assert launches == 2
            _same(got, ref)
            compare(got, ref, w.cap, mode)


def test_noalloc_takes_the_tuned_tiling(workload):
    """With a tuned entry loaded for the call's size class (the exact pair
    form, 512-j tiles, 8 tiles per j-split, instead of the default tiling),
    both calls run that tiling: bit-identical results, which differ from the
    default tiling's in the last bits (other velocity arithmetic)."""
    w = workload
    with Context(w.n) as ctx:
        d = upload(w)
        ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t)
        default, _ = _call(B.nb_regular_force, ctx, d, w, "mixed", w.cap)
        t = B.nb_tuned()
        t.mode, t.flags = B.NB_MIXED, 0
        t.act_class, t.j_class = int(np.log2(w.n_act)), int(np.log2(w.n))
        t.cfg = B.nb_kcfg(16, 2, 512, 8, 2)
        B.nb_set_tuned(ctx.h, t)
        ref, ref_launches = _call(B.nb_regular_force, ctx, d, w, "mixed", w.cap)
        assert ref_launches == 2
        assert not np.array_equal(ref["J"], default["J"]), "the tuned tiling was not taken"
        for _ in range(2):
            got, launches = _call(B.nb_regular_force_noalloc, ctx, d, w, "mixed", w.cap)
            assert launches == 2
            _same(got, ref)
        compare(ref, default, w.cap, "mixed")


def test_noalloc_matches_a_tail_split_call(workload):
    """A call of whole rounds of the persistent grid plus a remainder (every
    particle of N = 16384 active, the list-warp tiling) runs as two parts, the
    remainder with split j-ranges; the allocation-free call runs the same parts
    with its fixed array for the splits: three launches and bit-identical
    results, twice."""
    w = inputs.cluster(16384, 78, 64, 256)
    with Context(w.n) as ctx:
        d = upload(w)
        ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t)
        ctx.set_config("mixed", B.nb_kcfg(16, 2, 1024, 0, 9))
        ref, ref_launches = _call(B.nb_regular_force, ctx, d, w, "mixed", w.cap)
        assert ref_launches == 3
        for _ in range(2):
            got, launches = _call(B.nb_regular_force_noalloc, ctx, d, w, "mixed", w.cap)
            assert launches == 3
            _same(got, ref)


def test_noalloc_rejects_a_call_beyond_its_fixed_scratch(workload):
    w = workload
    n_act = 4096
    act = np.sort(np.random.default_rng(78).choice(w.n, n_act, replace=False)).astype(np.int32)
    big = w.with_active(act)
    cap = 4096    # about 5 splits x 4096 active x (68 + 4 cap) bytes, beyond 32 MiB
    with Context(w.n) as ctx:
        d = upload(big)
        ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t)
        with pytest.raises(B.NbError) as e:
            _call(B.nb_regular_force_noalloc, ctx, d, big, "mixed", cap)
        assert e.value.status == B.NB_ERR_ARG and "fixed array" in str(e.value)
        # the context is untouched and the allocation-free call still works at a fitting size
        small = w.with_active(act[:256])
        d2 = upload(small)
        ref, _ = _call(B.nb_regular_force, ctx, d2, small, "mixed", small.cap)
        got, _ = _call(B.nb_regular_force_noalloc, ctx, d2, small, "mixed", small.cap)
        compare(got, ref, small.cap, "mixed")
