"""Irregular force over the neighbour lists on the GPU (Sec. 3.3 step (iv)):
parity with the oracle's irregular sum, F_reg + F_irr = the full direct sum,
the potential split, and device-side rejection of bad list entries."""
import numpy as np
import pytest

import oracle
from paper_1205_1222_gb300 import Context, binding as B, inputs
from tests.gpu_util import TOL, oracle_predicted, rel_err, upload

pytestmark = pytest.mark.gpu


def _run(w, mode, pot=False, forms=0):
    with Context(w.n) as ctx:
        d = upload(w)
        ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t, forms=forms)
        reg = ctx.regular_force(d["act"], d["h"], w.n, cap=w.cap, mode=mode, pot=pot)
        irr = ctx.irregular_force(d["act"], reg["nnb"], reg["list"], w.n, w.cap, mode=mode, pot=pot)
        st = ctx.sync_status()
        g = lambda o: {k: (v.cpu().numpy() if v is not None else None) for k, v in o.items()}
        return g(reg), g(irr), st


@pytest.mark.parametrize("mode", ["fp64", "mixed", "fp32"])
def test_irregular_force_matches_oracle(mode):
    w = inputs.config2(n_act=1024)
    reg, irr, st = _run(w, mode)
    assert st == 0
    assert not reg["ovf"].any()
    x, v = oracle_predicted(w)
    oF, oJ = oracle.irregular(x, v, w.m, w.act, w.h)
    eF, eJ = rel_err(irr["F"], oF), rel_err(irr["J"], oJ)
    ftol, jtol = TOL[mode]
    print(mode, "irregular max rel err F", eF.max(), "J", eJ.max())
    assert eF.max() <= ftol and eJ.max() <= jtol


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_regular_plus_irregular_is_the_full_sum(mode):
    w = inputs.cluster(6000, 43, 48, 128, act=np.arange(0, 6000, 5, dtype=np.int32))
    reg, irr, st = _run(w, mode, pot=True)
    assert st == 0 and not reg["ovf"].any()
    x, v = oracle_predicted(w)
    fF, fJ, fP = oracle.full(x, v, w.m, w.act, with_pot=True)
    ftol, jtol = TOL[mode]
    assert rel_err(reg["F"] + irr["F"], fF).max() <= ftol
    assert rel_err(reg["J"] + irr["J"], fJ).max() <= jtol
    assert (np.abs(reg["pot"] + irr["pot"] - fP) / np.abs(fP)).max() <= ftol


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_irregular_force_with_velocity_criterion_at_an_odd_slot(mode):
    """Lists built with the velocity criterion, the j-range at an odd slot of a
    larger context, the potential on: the irregular sum matches the oracle's
    irregular sum over the same neighbour sets."""
    w = inputs.cluster(5000, 47, 48, 128, act=np.arange(1, 5000, 6, dtype=np.int32),
                       dtr_steps=(2.0**-5, 2.0**-7))
    off = 1001
    with Context(w.n + off + 2) as ctx:
        d = upload(w)
        ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t, offset=off)
        reg = ctx.regular_force(d["act"], d["h"], w.n, dtr=d["dtr"], cap=w.cap, mode=mode, j_begin=off)
        irr = ctx.irregular_force(d["act"], reg["nnb"], reg["list"], w.n, w.cap, mode=mode, j_begin=off, pot=True)
        assert ctx.sync_status() == 0
        assert not reg["ovf"].cpu().numpy().any()
        gF, gJ = irr["F"].cpu().numpy(), irr["J"].cpu().numpy()
    x, v = oracle_predicted(w)
    oF, oJ = oracle.irregular(x, v, w.m, w.act, w.h, dtr=w.dtr)
    ftol, jtol = TOL[mode]
    assert rel_err(gF, oF).max() <= ftol and rel_err(gJ, oJ).max() <= jtol


def test_two_float_irregular_force_on_hard_pairs_far_from_the_origin():
    """Hard pairs at separations down to 1e-5 at |x| = 1e3: the two-float
    differences keep the irregular force at the two-float tolerances, which
    FP32 differences cannot."""
    w = inputs.cluster(20000, 47, 64, 256, offset=1e3, pair_frac=0.1, act=np.arange(0, 20000, 7, dtype=np.int32))
    reg, irr, st = _run(w, "mixed")
    assert st == 0 and not reg["ovf"].any()
    x, v = oracle_predicted(w)
    oF, oJ = oracle.irregular(x, v, w.m, w.act, w.h)
    ftol, jtol = TOL["mixed"]
    assert rel_err(irr["F"], oF).max() <= ftol
    assert rel_err(irr["J"], oJ).max() <= jtol


@pytest.mark.parametrize("case", ["config2", "kroupa"])
def test_two_float_irregular_force_has_float_float_accuracy(case):
    """The two-float form sums float-float pair terms (about 46 significant
    bits from two FP32 values): every row within 1e-9 of the oracle's
    irregular sum, three orders below the two-float tolerances.  The bar: each
    float-float operation rounds at ~2^-46, a term is ~20 operations deep
    (~1e-12), and the irregular sums here cancel to no less than ~1e-3 of the
    sum of their terms' lengths.  (Far from the origin the stored two-float
    coordinates themselves limit close pairs: 2^-48 |x| at |x| = 1e3 is 4e-7
    of a 1e-5 separation; the hard-pair test above holds that case to the
    two-float tolerances.)"""
    if case == "config2":
        w = inputs.config2(n_act=1024)
    else:
        w = inputs.cluster(20000, 48, 100, 256, masses="kroupa", act=np.arange(0, 20000, 7, dtype=np.int32))
    reg, irr, st = _run(w, "mixed", pot=True)
    assert st == 0 and not reg["ovf"].any()
    x, v = oracle_predicted(w)
    oF, oJ = oracle.irregular(x, v, w.m, w.act, w.h)
    eF, eJ = rel_err(irr["F"], oF), rel_err(irr["J"], oJ)
    print(case, "float-float irregular max rel err F %.2e J %.2e" % (eF.max(), eJ.max()))
    assert eF.max() <= 1e-9 and eJ.max() <= 1e-9


def test_irregular_force_rejects_bad_entries_on_the_device():
    import torch
    w = inputs.config1()
    with Context(w.n) as ctx:
        d = upload(w)
        ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t)
        reg = ctx.regular_force(d["act"], d["h"], w.n, cap=w.cap, mode="mixed")
        assert ctx.sync_status() == 0
        lst = reg["list"].clone()
        lst[3, 0] = int(w.act[3])        # self
        lst[5, 0] = w.n + 7              # outside the j-range
        ctx.irregular_force(d["act"], reg["nnb"], lst, w.n, w.cap, mode="mixed")
        assert ctx.sync_status() == B.NB_ERR_DEVICE_INPUT
        # a clean call afterwards is unaffected
        irr = ctx.irregular_force(d["act"], reg["nnb"], reg["list"], w.n, w.cap, mode="mixed")
        assert ctx.sync_status() == 0
        assert torch.isfinite(irr["F"]).all()


def test_irregular_force_argument_errors():
    with Context(64) as ctx:
        with pytest.raises(B.NbError) as e:
            B.nb_irregular_force(ctx.h, 0, 100, 1, 0, 0, 0, 4, B.NB_MIXED, 0, 0)
        assert e.value.status == B.NB_ERR_ARG
