"""Needed-only prediction (Sec. 3.5, the NPACT switch of Appendix C): only the
active particles and their listed neighbours are predicted to the new block
time; the irregular force over those lists then matches the oracle's
irregular sum at that time, and equals bit for bit the irregular force after
a full prediction."""
import numpy as np
import pytest

import oracle
from paper_1205_1222_gb300 import Context, binding as B, build, inputs, mode_id
from tests.gpu_util import TOL, dev, rel_err, upload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _later(w, n_act, seed):
    """The workload's j-set at a later block time t2, an active subset, and the
    oracle's neighbour lists at t2."""
    sub = inputs.subset(w, n_act, seed)
    t2 = w.t + 2.0 ** -9
    x2, v2 = oracle.predict(w.x0, w.v0, w.a0, w.adot0, w.t0, t2)
    o = oracle.regular(x2, v2, w.m, sub.act, sub.h, cap=w.cap)
    return sub, t2, x2, v2, o


def _predicted64(ctx, n):
    import torch
    x = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    v = torch.empty_like(x)
    B.nb_get_predicted(ctx.h, 0, n, x, v)
    torch.cuda.synchronize()
    return x.cpu().numpy(), v.cpu().numpy()


@pytest.mark.parametrize("n_act", [16, 100])
def test_needed_only_prediction_predicts_exactly_the_named_slots(n_act):
    import torch
    w = inputs.cached(inputs.config2)
    sub, t2, x2, v2, o = _later(w, n_act, 5)
    with Context(w.n) as ctx:
        d = upload(w)
        ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t)
        x1, v1 = _predicted64(ctx, w.n)
        act, nnb, lst = dev(sub.act, torch.int32), dev(o["nnb"], torch.int32), dev(o["list"], torch.int32)
        B.nb_predict_needed(ctx.h, 0, w.n, sub.n_act, act, nnb, lst, w.cap, d["x0"], d["v0"], d["a0"],
                            d["adot0"], d["m"], d["t0"], t2, forms=B.NB_NEEDED_ONLY)
        assert ctx.sync_status() == 0 and ctx.last_launches() == 1
        xg, vg = _predicted64(ctx, w.n)
    named = np.zeros(w.n, dtype=bool)
    named[sub.act] = True
    for k in range(sub.n_act):
        named[o["list"][k, :min(o["nnb"][k], w.cap)]] = True
    assert named.sum() < w.n
    # named slots: the polynomial at t2 (as the full predictor's test bounds it)
    assert np.max(np.abs(xg[named] - x2[named])) <= 16e-16 * np.max(np.abs(x2))
    assert np.max(np.abs(vg[named] - v2[named])) <= 16e-16 * np.max(np.abs(v2))
    # every other slot keeps the values of the earlier prediction, bit for bit
    assert np.array_equal(xg[~named], x1[~named]) and np.array_equal(vg[~named], v1[~named])


@pytest.mark.parametrize("mode", ["fp64", "mixed", "fp32"])
def test_irregular_force_after_needed_only_prediction(mode):
    import torch
    w = inputs.cached(inputs.config2)
    sub, t2, x2, v2, o = _later(w, 64, 6)
    oF, oJ = oracle.irregular(x2, v2, w.m, sub.act, sub.h)
    with Context(w.n) as ctx:
        d = upload(w)
        act, nnb, lst = dev(sub.act, torch.int32), dev(o["nnb"], torch.int32), dev(o["list"], torch.int32)
        ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], t2)
        full = ctx.irregular_force(act, nnb, lst, w.n, w.cap, mode=mode)
        full = {k: v.cpu().numpy() for k, v in full.items() if v is not None}
        # the frame stays that of the full prediction; the block time moves on
        ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t, forms=B.NB_KEEP_FRAME)
        B.nb_predict_needed(ctx.h, 0, w.n, sub.n_act, act, nnb, lst, w.cap, d["x0"], d["v0"], d["a0"],
                            d["adot0"], d["m"], d["t0"], t2, forms=B.NB_NEEDED_ONLY)
        part = ctx.irregular_force(act, nnb, lst, w.n, w.cap, mode=mode)
        assert ctx.sync_status() == 0
        part = {k: v.cpu().numpy() for k, v in part.items() if v is not None}
    for k in ("F", "J"):
        assert np.array_equal(part[k], full[k]), k
    if mode != "fp32":
        ftol, jtol = TOL[mode]
        assert rel_err(part["F"], oF).max() <= ftol and rel_err(part["J"], oJ).max() <= jtol


def test_the_switch_predicts_the_whole_range_when_that_is_cheaper():
    """At n = 16384 the full prediction is the cheaper launch for any active
    set (the NPACT switch's other side): all slots then hold the polynomial
    at t2."""
    import torch
    w = inputs.cached(inputs.config2)
    sub, t2, x2, v2, o = _later(w, 16, 8)
    with Context(w.n) as ctx:
        d = upload(w)
        ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t)
        act, nnb, lst = dev(sub.act, torch.int32), dev(o["nnb"], torch.int32), dev(o["list"], torch.int32)
        B.nb_predict_needed(ctx.h, 0, w.n, sub.n_act, act, nnb, lst, w.cap, d["x0"], d["v0"], d["a0"],
                            d["adot0"], d["m"], d["t0"], t2)
        assert ctx.sync_status() == 0
        xg, vg = _predicted64(ctx, w.n)
    assert np.max(np.abs(xg - x2)) <= 16e-16 * np.max(np.abs(x2))
    assert np.max(np.abs(vg - v2)) <= 16e-16 * np.max(np.abs(v2))


def test_needed_only_prediction_refuses_what_it_cannot_do():
    import torch
    w = inputs.cluster(2000, 81, 16, 32)
    with Context(w.n) as ctx:
        d = upload(w)
        act = dev(np.arange(10, dtype=np.int32), torch.int32)
        nnb = dev(np.zeros(10, dtype=np.int32), torch.int32)
        lst = dev(np.zeros((10, w.cap), dtype=np.int32), torch.int32)
        args = (ctx.h, 0, w.n, 10, act, nnb, lst, w.cap, d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"],
                w.t)
        ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t, forms=B.NB_FORM_MIXED)
        with pytest.raises(B.NbError) as e:          # a form the last prediction did not write
            B.nb_predict_needed(*args, forms=B.NB_FORM_FP64)
        assert e.value.status == B.NB_ERR_STATE
        B.nb_set_frame(ctx.h, [1.0, 0.0, 0.0])       # another frame than the range's
        with pytest.raises(B.NbError) as e:
            B.nb_predict_needed(*args)
        assert e.value.status == B.NB_ERR_STATE and "frame" in str(e.value)
        ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t)
        with pytest.raises(B.NbError) as e:          # range past the context
            B.nb_predict_needed(ctx.h, 1, w.n, 10, act, nnb, lst, w.cap, d["x0"], d["v0"], d["a0"], d["adot0"],
                                d["m"], d["t0"], w.t)
        assert e.value.status == B.NB_ERR_ARG
        # an entry outside the range is skipped and reported, not followed
        bad = np.zeros((10, w.cap), dtype=np.int32)
        bad[3, 0] = w.n + 5
        nnb1 = dev(np.ones(10, dtype=np.int32), torch.int32)
        B.nb_predict_needed(ctx.h, 0, w.n, 10, act, nnb1, dev(bad, torch.int32), w.cap, d["x0"], d["v0"], d["a0"],
                            d["adot0"], d["m"], d["t0"], w.t, forms=B.NB_NEEDED_ONLY)
        assert ctx.sync_status() == B.NB_ERR_DEVICE_INPUT
        B.nb_predict_needed(*args)
        assert ctx.sync_status() == 0


def test_needed_only_prediction_replays_from_a_cuda_graph():
    """A captured needed-only prediction + irregular force, replayed after the
    inputs changed in place: every replay predicts the named slots afresh (the
    call holds no state between calls), so the replay equals a direct call on
    the new inputs."""
    import torch
    w = inputs.cached(inputs.config2)
    sub, t2, x2, v2, o = _later(w, 64, 7)
    with Context(w.n) as ctx:
        d = upload(w)
        act, nnb, lst = dev(sub.act, torch.int32), dev(o["nnb"], torch.int32), dev(o["list"], torch.int32)
        ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t)

        def step(stream=None):
            B.nb_predict_needed(ctx.h, 0, w.n, sub.n_act, act, nnb, lst, w.cap, d["x0"], d["v0"], d["a0"],
                                d["adot0"], d["m"], d["t0"], t2, forms=B.NB_NEEDED_ONLY, stream=stream)
            return ctx.irregular_force(act, nnb, lst, w.n, w.cap, mode="mixed", stream=stream)

        direct = []
        for scale in (1.0, 1.5):
            d["v0"].copy_(dev(w.v0 * scale))
            direct.append({k: v.cpu().numpy() for k, v in step().items() if v is not None})
        assert not np.array_equal(direct[0]["J"], direct[1]["J"])
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                out = step(stream=side)
        for scale, want in zip((1.0, 1.5, 1.0), (direct[0], direct[1], direct[0])):
            d["v0"].copy_(dev(w.v0 * scale))
            torch.cuda.synchronize()
            g.replay()
            torch.cuda.synchronize()
            assert ctx.sync_status() == 0
            for k in ("F", "J"):
                assert np.array_equal(out[k].cpu().numpy(), want[k]), (scale, k)
