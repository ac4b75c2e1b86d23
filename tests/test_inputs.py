"""Properties of the seeded input generators (CPU only)."""
import math

import numpy as np
import pytest

import oracle
from paper_1205_1222_gb300 import inputs


def _pair_dist(X, act):
    d = np.linalg.norm(X[None, :, :] - X[act][:, None, :], axis=2)
    d[np.arange(len(act)), act] = np.nan
    return d


def test_plummer_is_in_virial_equilibrium_in_henon_units():
    rng = np.random.default_rng(np.random.PCG64(7))
    n = 2048
    X, V = inputs.plummer(n, rng)
    m = np.full(n, 1.0 / n)
    kin = 0.5 * (m * (V * V).sum(1)).sum()
    d = np.linalg.norm(X[:, None] - X[None], axis=2)
    iu = np.triu_indices(n, 1)
    pot = -(m[iu[0]] * m[iu[1]] / d[iu]).sum()
    assert abs(kin + pot - (-0.25)) < 0.02          # E = -1/4
    assert abs(2 * kin / -pot - 1.0) < 0.1          # Q = 0.5
    assert np.allclose(X.mean(0), 0, atol=1e-12) and np.allclose(V.mean(0), 0, atol=1e-12)


def test_kroupa_masses():
    m = inputs.kroupa_masses(200000, np.random.default_rng(3))
    assert abs(m.sum() - 1.0) < 1e-12
    msun = m / m.min() * 0.08   # back to solar masses up to sampling of the minimum
    assert msun.max() <= 100.0 * 1.01
    # fraction above the break ~ (analytic) 0.23 for this IMF
    frac = (msun > 0.5).mean()
    assert 0.15 < frac < 0.32


def test_config1_prediction_lands_on_block_state_and_keeps_margin():
    w = inputs.config1()
    assert w.n == 1024 and w.n_act == 1024 and w.cap == 128 and w.dtr is None
    assert np.all(w.t - w.t0 == 2.0**-10)
    x, v = oracle.predict(w.x0, w.v0, w.a0, w.adot0, w.t0, w.t)
    assert np.max(np.abs(x - w.X)) < 1e-14 and np.max(np.abs(v - w.V)) < 1e-13
    d = _pair_dist(x, w.act)
    rel = np.abs(d / w.h[:, None] - 1.0)
    assert np.nanmin(rel) >= 0.99e-6
    nnb = (d < w.h[:, None]).sum(1)
    assert 24 <= nnb.min() and nnb.max() <= 40 and abs(nnb.mean() - 32) < 1.5


def test_velocity_criterion_radii_keep_margin():
    w = inputs.cluster(1500, 17, 40, 128, dtr_steps=(2.0**-5, 2.0**-6, 2.0**-7))
    x, v = oracle.predict(w.x0, w.v0, w.a0, w.adot0, w.t0, w.t)
    R = x[None, :, :] - x[w.act][:, None, :]
    Vr = v[None, :, :] - v[w.act][:, None, :]
    q = np.minimum(np.linalg.norm(R, axis=2), np.linalg.norm(R + w.dtr[:, None, None] * Vr, axis=2))
    q[np.arange(w.n_act), w.act] = np.nan
    rel = np.abs(q / w.h[:, None] - 1)
    assert np.nanmin(rel) >= 0.99e-6
    nnb = (q < w.h[:, None]).sum(1)
    assert abs(nnb.mean() - 40) < 3


def test_hard_pairs_are_inside_each_others_sphere():
    w = inputs.cluster(4096, 5, 64, 256, offset=1e3, pair_frac=0.1)
    prim, sec, sep = w.meta["pair_primary"], w.meta["pair_secondary"], w.meta["pair_sep"]
    assert len(prim) == round(0.05 * 4096)
    d = np.linalg.norm(w.X[prim] - w.X[sec], axis=1)
    np.testing.assert_allclose(d, sep, rtol=0, atol=1e-12)   # FP64 ulp at |x| ~ 600
    h = w.meta["h_all"]
    assert np.all(h[prim] > sep) and np.all(h[sec] > sep)
    assert abs(np.linalg.norm(w.X.mean(0)) - 1e3) < 1.0


def test_subsets_and_batch_shapes():
    w = inputs.cluster(3000, 2, 16, 64)
    s = inputs.subset(w, 100, 2)
    assert s.n_act == 100 and np.all(np.diff(s.act) > 0)
    assert np.array_equal(s.h, w.meta["h_all"][s.act])
    rng = np.random.default_rng(0)
    ns = np.rint(np.exp(rng.uniform(math.log(1024), math.log(32768), 64)))
    assert ns.min() >= 1024 and ns.max() <= 32768
