"""The native autotuner: it picks a compiled tiling, later calls of the same
size class use it, and the table survives a JSON round trip."""
import numpy as np
import pytest

from paper_1205_1222_gb300 import Context, autotune, binding as B, inputs
from tests.gpu_util import compare, oracle_run, upload

pytestmark = pytest.mark.gpu


def _ctx_with(w):
    ctx = Context(w.n)
    d = upload(w)
    ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t)
    return ctx, d


def test_autotune_picks_a_compiled_tiling_and_keeps_parity():
    w = inputs.config2(n_act=1024)
    ctx, d = _ctx_with(w)
    with ctx:
        best, ms = ctx.autotune(d["act"], d["h"], w.n, cap=w.cap, mode="mixed", reps=1)
        assert ms > 0
        compiled = [B.nb_get_kernel_config(B.NB_MIXED, i).as_tuple()[:3] + (B.nb_get_kernel_config(B.NB_MIXED, i).packed,)
                    for i in range(B.nb_num_kernel_configs(B.NB_MIXED))]
        assert best.as_tuple()[:3] + (best.packed,) in compiled
        rows = autotune.table(ctx)
        assert len(rows) == 1
        assert rows[0]["mode"] == B.NB_MIXED and rows[0]["flags"] == 0
        assert rows[0]["act_class"] == 10 and rows[0]["j_class"] == 14
        out = ctx.regular_force(d["act"], d["h"], w.n, cap=w.cap, mode="mixed")
        assert ctx.sync_status() == 0
        g = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
        compare(g, oracle_run(w), w.cap, "mixed")


def test_tuned_entry_is_used_by_calls_of_its_class_only():
    """A tuned entry with another tiling changes the summation order of the
    calls of its class (results differ in the last bits, lists are equal);
    removing the entry restores the default results bit for bit, and calls of
    another class never see it."""
    w = inputs.cluster(65536, 41, 32, 64)
    ctx, d = _ctx_with(w)
    g = lambda o: {k: (v.cpu().numpy() if v is not None else None) for k, v in o.items()}
    with ctx:
        q = w.n // 4
        base = g(ctx.regular_force(d["act"], d["h"], w.n, cap=w.cap, mode="mixed"))
        base_q = g(ctx.regular_force(d["act"][:q], d["h"][:q], w.n, cap=w.cap, mode="mixed"))
        t = B.nb_tuned()
        t.mode, t.flags, t.act_class, t.j_class = B.NB_MIXED, 0, 16, 16
        t.cfg = B.nb_kcfg(16, 2, 512, 8, 2)            # exact pair form, 8 tiles per j-split
        B.nb_set_tuned(ctx.h, t)
        tuned = g(ctx.regular_force(d["act"], d["h"], w.n, cap=w.cap, mode="mixed"))
        assert np.array_equal(tuned["nnb"], base["nnb"]) and np.array_equal(tuned["list"], base["list"])
        assert not np.array_equal(tuned["F"], base["F"])
        assert np.abs(tuned["F"] - base["F"]).max() <= 1e-6 * np.abs(base["F"]).max()
        other = g(ctx.regular_force(d["act"][:q], d["h"][:q], w.n, cap=w.cap, mode="mixed"))
        assert np.array_equal(other["F"], base_q["F"])
        t.cfg = B.nb_kcfg(0, 0, 0, 0, 0)
        B.nb_set_tuned(ctx.h, t)
        assert B.nb_tuned_table(ctx.h) == []
        again = g(ctx.regular_force(d["act"], d["h"], w.n, cap=w.cap, mode="mixed"))
        assert np.array_equal(again["F"], base["F"]) and np.array_equal(again["J"], base["J"])
        assert ctx.sync_status() == 0


def test_tuned_table_round_trip(tmp_path):
    w = inputs.config2(n_act=256)
    ctx, d = _ctx_with(w)
    with ctx:
        ctx.autotune(d["act"], d["h"], w.n, cap=w.cap, mode="fp32", reps=1)
        rows = autotune.table(ctx)
        path = str(tmp_path / "tuned.json")
        autotune.save(ctx, path, "test")
    with Context(16) as other:
        assert autotune.load(other, path) == len(rows) == 1
        back = autotune.table(other)
        assert [(r["mode"], r["flags"], r["act_class"], r["j_class"], r["cfg"]) for r in back] == \
               [(r["mode"], r["flags"], r["act_class"], r["j_class"], r["cfg"]) for r in rows]


def test_set_tuned_rejects_a_tiling_that_is_not_compiled():
    with Context(16) as ctx:
        t = B.nb_tuned()
        t.mode, t.flags, t.act_class, t.j_class = B.NB_MIXED, 0, 4, 4
        t.cfg = B.nb_kcfg(7, 3, 100, 0, 2)
        with pytest.raises(B.NbError) as e:
            B.nb_set_tuned(ctx.h, t)
        assert e.value.status == B.NB_ERR_UNSUPPORTED
