"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

The paper (Nitadori & Aarseth 2012) prints no worked numeric example, so the
oracle is pinned by closed forms derived by hand (tests/golden/two_body.txt),
by calculus (the jerk is the time derivative of the force; the predictor is a
Taylor polynomial with the given derivatives), by conservation laws (Newton's
third law), by the split identity F_reg + F_irr = F_full, by exact symmetries
(power-of-two scaling, dyadic translation and boosts, relabelling) and by a
pure-Python brute force for the neighbour sets on tiny N.  Each test names the
plausible mistake it would catch.
"""
import math
import os

import numpy as np
import pytest

import oracle
from tests.brute_force import neighbour_sets

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "two_body.txt")


def _rand_system(n, seed, spread=1.0, dyadic=False):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-spread, spread, (n, 3))
    v = rng.uniform(-0.5, 0.5, (n, 3))
    m = rng.uniform(0.5, 1.5, n) / n
    if dyadic:  # multiples of 2^-20: translations by small powers of two stay exact
        x = np.round(x * 2**20) / 2**20
        v = np.round(v * 2**20) / 2**20
        m = np.round(m * 2**30) / 2**30
    return x, v, m


def _load_golden():
    cases = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        lhs, rhs = line.split("->")
        a = [float(t) for t in lhs.split()]
        b = [float(t) for t in rhs.split()]
        cases.append((a[0], np.array(a[1:4]), np.array(a[4:7]), np.array(b[0:3]), np.array(b[3:6])))
    return cases


@pytest.mark.parametrize("case", range(5))
def test_two_body_closed_form(case):
    """Catches a wrong power of r, a sign flip of R or V, or a wrong factor 3."""
    m_j, R, V, F_exp, J_exp = _load_golden()[case]
    x = np.array([[0.0, 0, 0], R]); v = np.array([[0.0, 0, 0], V])
    m = np.array([1.0, m_j])
    out = oracle.regular(x, v, m, act=[0], h=[0.0], cap=4)
    np.testing.assert_allclose(out["F"][0], F_exp, rtol=0, atol=1e-15)
    np.testing.assert_allclose(out["J"][0], J_exp, rtol=0, atol=1e-15)
    assert out["nnb"][0] == 0 and out["ovf"][0] == 0
    # Inside the neighbour sphere the pair leaves the regular sums and enters the list.
    r = float(np.linalg.norm(R))
    out = oracle.regular(x, v, m, act=[0], h=[r * 1.5], cap=4)
    assert np.all(out["F"] == 0) and np.all(out["J"] == 0)
    assert out["nnb"][0] == 1 and out["list"][0, 0] == 1
    # ... and the irregular sum picks it up unchanged.
    Fi, Ji = oracle.irregular(x, v, m, act=[0], h=[r * 1.5])
    np.testing.assert_allclose(Fi[0], F_exp, atol=1e-15)
    np.testing.assert_allclose(Ji[0], J_exp, atol=1e-15)


def _force_at(x, v, m, act, h, tau):
    return oracle.regular(x + tau * v, v, m, act, h, cap=len(x))


@pytest.mark.parametrize("use_h", [False, True])
def test_jerk_is_time_derivative_of_force(use_h):
    """J = dF/dt along straight-line motion.  Catches any error in the jerk
    formula independently of how it is written (sign, factor 3, power of r)."""
    n = 24
    x, v, m = _rand_system(n, seed=11)
    act = np.arange(n, dtype=np.int32)
    if use_h:
        # radii well between pair distances so the list does not change over +-tau
        d = np.linalg.norm(x[:, None, :] - x[None, :, :], axis=2)
        d[np.arange(n), np.arange(n)] = np.inf
        s = np.sort(d, axis=1)
        h = np.sqrt(s[:, 3] * s[:, 4])
    else:
        h = np.zeros(n)
    base = oracle.regular(x, v, m, act, h, cap=n)
    tau = 1e-4
    fp = _force_at(x, v, m, act, h, tau)
    fm = _force_at(x, v, m, act, h, -tau)
    fp2 = _force_at(x, v, m, act, h, 2 * tau)
    fm2 = _force_at(x, v, m, act, h, -2 * tau)
    for o in (fp, fm, fp2, fm2):
        assert np.array_equal(o["nnb"], base["nnb"])
    # fourth-order central difference
    dF = (8 * (fp["F"] - fm["F"]) - (fp2["F"] - fm2["F"])) / (12 * tau)
    scale = np.linalg.norm(base["J"], axis=1)[:, None]
    assert np.max(np.abs(dF - base["J"]) / scale) < 1e-7


def test_newton_third_law():
    """sum m_i F_i = 0 and sum m_i J_i = 0 with all particles active and no
    split, and with one uniform radius (a symmetric neighbour relation).
    Catches an asymmetric term, e.g. R = x_i - x_j in one place only."""
    n = 64
    x, v, m = _rand_system(n, seed=3)
    act = np.arange(n, dtype=np.int32)
    for h in (np.zeros(n), np.full(n, 0.4)):
        o = oracle.regular(x, v, m, act, h, cap=n)
        for key in ("F", "J"):
            tot = (m[:, None] * o[key]).sum(axis=0)
            scale = (m * np.linalg.norm(o[key], axis=1)).sum()
            assert np.max(np.abs(tot)) < 1e-12 * scale


@pytest.mark.parametrize("with_dtr", [False, True])
def test_regular_plus_irregular_is_full(with_dtr):
    """F_reg + F_irr = F_full (Sec. 1, Sec. 3.3): the split is a partition.
    Catches a pair counted twice or dropped at the boundary."""
    n = 200
    x, v, m = _rand_system(n, seed=5)
    rng = np.random.default_rng(6)
    act = rng.choice(n, 50, replace=False).astype(np.int32)
    h = rng.uniform(0.05, 0.6, 50)
    dtr = rng.uniform(0.0, 0.3, 50) if with_dtr else None
    reg = oracle.regular(x, v, m, act, h, dtr=dtr, cap=n)
    Fi, Ji = oracle.irregular(x, v, m, act, h, dtr=dtr)
    Ff, Jf = oracle.full(x, v, m, act)
    for a, b, c in ((reg["F"], Fi, Ff), (reg["J"], Ji, Jf)):
        err = np.linalg.norm(a + b - c, axis=1) / np.linalg.norm(c, axis=1)
        assert np.max(err) < 1e-12
    assert reg["nnb"].sum() > 0


@pytest.mark.parametrize("with_dtr", [False, True])
@pytest.mark.parametrize("n", [2, 7, 33, 64])
def test_neighbour_sets_brute_force(n, with_dtr):
    """Exact neighbour sets and ascending order vs the pure-Python brute force."""
    x, v, m = _rand_system(n, seed=100 + n)
    rng = np.random.default_rng(n)
    act = rng.permutation(n).astype(np.int32)[: max(1, n // 2)]
    h = rng.uniform(0.1, 1.2, len(act))
    dtr = rng.uniform(0, 0.5, len(act)) if with_dtr else None
    o = oracle.regular(x, v, m, act, h, dtr=dtr, cap=n)
    ref = neighbour_sets(x.tolist(), v.tolist(), act.tolist(), h.tolist(),
                         None if dtr is None else dtr.tolist())
    for a, lst in enumerate(ref):
        assert o["nnb"][a] == len(lst)
        assert o["list"][a, : len(lst)].tolist() == lst
        assert int(act[a]) not in lst


def test_overflow_keeps_lowest_indices():
    """List capacity: true count, lowest `cap` indices ascending, overflow flag."""
    n = 40
    x, v, m = _rand_system(n, seed=9, spread=0.3)
    act = np.array([0, 5, 39], dtype=np.int32)
    h = np.array([10.0, 0.2, 10.0])  # 0 and 39 see everyone
    ref = neighbour_sets(x.tolist(), v.tolist(), act.tolist(), h.tolist())
    for cap in (0, 1, 7, 39, 50):
        o = oracle.regular(x, v, m, act, h, cap=cap)
        for a, lst in enumerate(ref):
            assert o["nnb"][a] == len(lst)
            k = min(cap, len(lst))
            assert o["list"][a, :k].tolist() == lst[:k]
            assert o["ovf"][a] == (1 if len(lst) > cap else 0)
        # the force does not depend on the capacity
        o2 = oracle.regular(x, v, m, act, h, cap=n)
        assert np.array_equal(o["F"], o2["F"])


def test_power_of_two_scaling_is_exact():
    """x -> 2x, h -> 2h: F -> F/4 and J -> J/8 bit for bit (every operation
    scales by a power of two).  Catches a wrong power of r in either term."""
    n = 50
    x, v, m = _rand_system(n, seed=21)
    act = np.arange(0, n, 3, dtype=np.int32)
    h = np.full(len(act), 0.3)
    a = oracle.regular(x, v, m, act, h, cap=n)
    b = oracle.regular(2 * x, v, m, act, 2 * h, cap=n)
    assert np.array_equal(b["F"], a["F"] / 4)
    assert np.array_equal(b["J"], a["J"] / 8)
    assert np.array_equal(a["list"], b["list"])
    # velocities x2 as well: J -> J/4
    c = oracle.regular(2 * x, 2 * v, m, act, 2 * h, cap=n)
    assert np.array_equal(c["J"], a["J"] / 4)


def test_translation_and_boost_invariance_exact():
    """A dyadic translation of all positions and a dyadic boost of all
    velocities leave R and V, hence F, J and the lists, bit-identical."""
    n = 50
    x, v, m = _rand_system(n, seed=22, dyadic=True)
    act = np.arange(0, n, 2, dtype=np.int32)
    h = np.full(len(act), 0.35)
    dtr = np.full(len(act), 0.125)
    a = oracle.regular(x, v, m, act, h, dtr=dtr, cap=n)
    b = oracle.regular(x + np.array([4.0, -8.0, 2.0]), v + np.array([0.5, 0.25, -1.0]),
                       m, act, h, dtr=dtr, cap=n)
    for k in ("F", "J", "nnb", "list"):
        assert np.array_equal(a[k], b[k])


def test_relabelling_permutes_lists():
    """Renumbering the particles renumbers the lists and changes F, J only by
    summation order.  Catches an index mix-up between i and j."""
    n = 60
    x, v, m = _rand_system(n, seed=23)
    act = np.arange(n, dtype=np.int32)
    h = np.full(n, 0.4)
    a = oracle.regular(x, v, m, act, h, cap=n)
    p = np.random.default_rng(1).permutation(n)       # new index k holds old p[k]
    inv = np.argsort(p)
    b = oracle.regular(x[p], v[p], m[p], inv[act].astype(np.int32), h, cap=n)
    np.testing.assert_allclose(b["F"], a["F"], rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(b["J"], a["J"], rtol=1e-13, atol=1e-12)
    for i in range(n):
        la = a["list"][i, : a["nnb"][i]]
        lb = b["list"][i, : b["nnb"][i]]
        assert sorted(inv[la].tolist()) == lb.tolist()


def test_zero_radius_and_empty_inputs():
    n = 30
    x, v, m = _rand_system(n, seed=24)
    act = np.arange(n, dtype=np.int32)
    reg = oracle.regular(x, v, m, act, np.zeros(n), cap=8)
    Ff, Jf = oracle.full(x, v, m, act)
    assert np.all(reg["nnb"] == 0) and np.all(reg["ovf"] == 0)
    assert np.array_equal(reg["F"], Ff) and np.array_equal(reg["J"], Jf)
    empty = oracle.regular(x, v, m, np.zeros(0, dtype=np.int32), np.zeros(0), cap=8)
    assert empty["F"].shape == (0, 3)


def test_coincident_pair_outside_sphere_is_rejected():
    x = np.array([[0.0, 0, 0], [0.0, 0, 0], [1.0, 0, 0]])
    v = np.zeros((3, 3)); m = np.ones(3)
    with pytest.raises(oracle.OracleError):
        oracle.regular(x, v, m, [0], [0.0], cap=4)
    # inside the sphere the coincident pair is just a neighbour
    o = oracle.regular(x, v, m, [0], [0.5], cap=4)
    assert o["list"][0, 0] == 1 and o["nnb"][0] == 1


def test_potential_matches_two_body():
    x = np.array([[0.0, 0, 0], [3.0, 4.0, 0]]); v = np.zeros((2, 3)); m = np.array([1.0, 2.0])
    o = oracle.regular(x, v, m, [0], [0.0], cap=2, with_pot=True)
    assert o["pot"][0] == pytest.approx(2.0 / 5.0, rel=0, abs=1e-16)


# ---------------------------------------------------------------- predictor

def _pred_inputs(n, seed):
    rng = np.random.default_rng(seed)
    return (rng.normal(size=(n, 3)), rng.normal(size=(n, 3)), rng.normal(size=(n, 3)),
            rng.normal(size=(n, 3)))


def test_predictor_zero_step_is_identity():
    x0, v0, a0, j0 = _pred_inputs(20, 1)
    t0 = np.full(20, 0.75)
    x, v = oracle.predict(x0, v0, a0, j0, t0, 0.75)
    assert np.array_equal(x, x0) and np.array_equal(v, v0)


def test_predictor_derivatives_at_start():
    """Symmetric differences of the predicted trajectory at dt = 0 recover
    v0, a0 and adot0 (a cubic's differences are exact up to rounding).
    Catches a wrong Taylor coefficient (e.g. dt^2 instead of dt^2/2)."""
    n = 16
    x0, v0, a0, j0 = _pred_inputs(n, 2)
    t0 = np.zeros(n)
    tau = 2.0**-6

    def X(dt):
        return oracle.predict(x0, v0, a0, j0, t0, dt)[0]

    def Vp(dt):
        return oracle.predict(x0, v0, a0, j0, t0, dt)[1]

    d1 = (X(tau) - X(-tau)) / (2 * tau)                 # = v0 + j0 tau^2/6
    d2 = (X(tau) - 2 * X(0.0) + X(-tau)) / tau**2       # = a0 exactly for a cubic
    d3 = (X(2 * tau) - 2 * X(tau) + 2 * X(-tau) - X(-2 * tau)) / (2 * tau**3)  # = adot0
    np.testing.assert_allclose(d1, v0 + j0 * tau**2 / 6, rtol=0, atol=1e-12)
    np.testing.assert_allclose(d2, a0, rtol=0, atol=1e-9)
    np.testing.assert_allclose(d3, j0, rtol=0, atol=1e-6)
    # the predicted velocity is the time derivative of the predicted position
    for dt in (0.1, -0.3, 0.55):
        dx = (X(dt + tau) - X(dt - tau)) / (2 * tau)
        np.testing.assert_allclose(dx, Vp(dt) + j0 * tau**2 / 6, rtol=0, atol=1e-11)


def test_predictor_composes_like_a_cubic():
    """Predicting t0 -> t1 and then t1 -> t2 (with the acceleration carried to
    t1 along the cubic) equals predicting t0 -> t2."""
    n = 10
    x0, v0, a0, j0 = _pred_inputs(n, 3)
    t1, t2 = 0.25, 0.625
    x1, v1 = oracle.predict(x0, v0, a0, j0, np.zeros(n), t1)
    a1 = a0 + j0 * t1
    x2, v2 = oracle.predict(x1, v1, a1, j0, np.full(n, t1), t2)
    x2d, v2d = oracle.predict(x0, v0, a0, j0, np.zeros(n), t2)
    np.testing.assert_allclose(x2, x2d, rtol=0, atol=1e-14)
    np.testing.assert_allclose(v2, v2d, rtol=0, atol=1e-14)


def test_predictor_is_third_order_on_a_kepler_orbit():
    """On a circular orbit (r = 1, unit central mass) with the exact a and
    da/dt, the position error of the prediction falls as dt^4."""
    errs = []
    for dt in (0.04, 0.02, 0.01):
        x0 = np.array([[1.0, 0, 0]]); v0 = np.array([[0.0, 1.0, 0]])
        a0 = np.array([[-1.0, 0, 0]]); j0 = np.array([[0.0, -1.0, 0]])
        x, _ = oracle.predict(x0, v0, a0, j0, np.zeros(1), dt)
        exact = np.array([math.cos(dt), math.sin(dt), 0.0])
        errs.append(np.linalg.norm(x[0] - exact))
    assert 14 < errs[0] / errs[1] < 18 and 14 < errs[1] / errs[2] < 18


def test_exact_boundary_pair_is_regular():
    """A pair at exactly |R| = h_i is not a neighbour (the list uses "< h_i")
    and therefore belongs to the regular sum: the two sums partition j != i."""
    x = np.array([[0.0, 0, 0], [0.5, 0, 0], [0.0, 0.25, 0]])
    v = np.zeros((3, 3)); m = np.array([1.0, 1.0, 1.0])
    o = oracle.regular(x, v, m, [0], [0.5], cap=4)
    assert o["nnb"][0] == 1 and o["list"][0, 0] == 2
    np.testing.assert_allclose(o["F"][0], [4.0, 0, 0], rtol=0, atol=0)
    # with the velocity criterion the boundary is the same strict test
    v2 = np.array([[0.0, 0, 0], [1.0, 0, 0], [0.0, 0, 0]])
    o = oracle.regular(x, v2, m, [0], [0.5], dtr=[0.0], cap=4)
    assert o["nnb"][0] == 1


# ------------------------------------------------- conditioning of the sums

@pytest.mark.parametrize("case", range(5))
def test_term_length_sums_of_a_single_source_are_its_force_and_jerk(case):
    """With one regular source the length sums are the lengths of the force
    and jerk themselves (hand-derived closed forms of tests/golden); inside
    the sphere the source is not counted.  Catches a wrong power of r or a
    jerk term that differs from the regular sum's."""
    m_j, R, V, F_exp, J_exp = _load_golden()[case]
    x = np.array([[0.0, 0, 0], R]); v = np.array([[0.0, 0, 0], V])
    m = np.array([1.0, m_j])
    SF, SJ = oracle.regular_mag(x, v, m, act=[0], h=[0.0])
    assert abs(SF[0] - np.linalg.norm(F_exp)) <= 1e-15 * np.linalg.norm(F_exp)
    assert abs(SJ[0] - np.linalg.norm(J_exp)) <= 1e-14 * max(np.linalg.norm(J_exp), 1e-300)
    SF, SJ = oracle.regular_mag(x, v, m, act=[0], h=[1.5 * np.linalg.norm(R)])
    assert SF[0] == 0.0 and SJ[0] == 0.0


def test_term_length_sums_see_the_cancellation():
    """Two equal masses at +-r on the x axis, at rest: the forces cancel
    (F = 0) while SF = 2 m / r^2; moving with velocity u along y, each jerk
    term has length m u / r^3 and they add up (J = 2 m u / r^3 = SJ).  Random
    systems: SF >= |F|, SJ >= |J| with equality only without cancellation."""
    r, mj, u = 0.75, 0.125, 0.5
    x = np.array([[0.0, 0, 0], [r, 0, 0], [-r, 0, 0]])
    v = np.array([[0.0, 0, 0], [0, u, 0], [0, u, 0]])
    m = np.array([1.0, mj, mj])
    out = oracle.regular(x, v, m, act=[0], h=[0.0], cap=4)
    SF, SJ = oracle.regular_mag(x, v, m, act=[0], h=[0.0])
    assert np.all(out["F"][0] == 0.0)
    assert SF[0] == 2 * mj / r**2
    np.testing.assert_allclose(out["J"][0], [0, 2 * mj * u / r**3, 0], rtol=1e-15)
    assert abs(SJ[0] - 2 * mj * u / r**3) <= 1e-15 * SJ[0]
    x, v, m = _rand_system(40, seed=5)
    act = np.arange(40, dtype=np.int32)
    h = np.full(40, 0.3)
    out = oracle.regular(x, v, m, act, h, cap=40)
    SF, SJ = oracle.regular_mag(x, v, m, act, h)
    assert np.all(SF >= np.linalg.norm(out["F"], axis=1) * (1 - 1e-14))
    assert np.all(SJ >= np.linalg.norm(out["J"], axis=1) * (1 - 1e-14))
    assert np.median(SF / np.linalg.norm(out["F"], axis=1)) > 1.0
