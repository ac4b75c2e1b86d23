"""Seeded synthetic inputs shaped like the paper's benchmark clusters.

The paper times NBODY6 on equal-mass Plummer spheres in Henon units
(G = M = 1, E = -1/4; Sec. 4) with N = 8k..256k.  No data set ships with it,
so every workload here is generated from a seed.  This module serves the CUDA
path and the oracle alike and holds none of the method's arithmetic: it never
evaluates a pair force, a neighbour test or the predictor.  It only

* samples Plummer spheres (the Aarseth-Henon-Wielen 1974 recipe) and Kroupa
  (2001) masses,
* places hard pairs and offsets the cluster centre,
* picks neighbour radii from k-nearest-neighbour distances (scipy cKDTree),
  with a margin so that no pair distance lies within a relative 1e-6 of a
  radius (the neighbour decision is then the same in any precision that
  resolves a relative 1e-6),
* builds the start-of-step state.  The block-time state (X, V) is sampled
  first and the radii are chosen on it; the start-of-step state (x0, v0) is
  then back-filled from (X, V), the derivatives (a0, adot0) and the step dt so
  that the third-order Taylor prediction lands on (X, V) up to rounding.  The
  back-fill solves for the start values; the prediction itself is left to the
  code under test.

The derivatives (a0, adot0) default to the smooth field of the Plummer
potential (a background field, not a sum over particles).  Callers that want
them "from a prior direct sum" pass their own arrays through ``accel``.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field

import numpy as np

HENON_PLUMMER_B = 3.0 * math.pi / 16.0  # Plummer scale length for E = -1/4, M = 1, G = 1
MARGIN = 1e-6                            # relative gap kept between every |r_ij| and r_i
BLOCK_TIME = 2.0                         # the paper times runs from t = 2 (Sec. 4)


@dataclass
class Workload:
    """One regular-force call: a predicted-to-be j-set plus an active set."""
    name: str
    x0: np.ndarray          # [n,3] start-of-step positions (FP64)
    v0: np.ndarray          # [n,3] start-of-step velocities
    a0: np.ndarray          # [n,3] accelerations at t0
    adot0: np.ndarray       # [n,3] their time derivatives at t0
    m: np.ndarray           # [n]   masses
    t0: np.ndarray          # [n]   start-of-step times
    t: float                # block time
    act: np.ndarray         # [n_act] int32 indices of the active particles
    h: np.ndarray           # [n_act] neighbour radii
    dtr: np.ndarray | None  # [n_act] regular steps for the velocity criterion, or None
    cap: int                # neighbour-list capacity
    X: np.ndarray = field(repr=False, default=None)  # [n,3] block-time positions (construction target)
    V: np.ndarray = field(repr=False, default=None)
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.m.shape[0])

    @property
    def n_act(self) -> int:
        return int(self.act.shape[0])

    def with_active(self, act, h_all=None, dtr_all=None, name=None) -> "Workload":
        """Same j-set, another active subset (radii taken from the per-particle table)."""
        act = np.ascontiguousarray(act, dtype=np.int32)
        h_all = self.meta["h_all"] if h_all is None else h_all
        dtr = None
        if dtr_all is not None:
            dtr = np.ascontiguousarray(dtr_all[act], dtype=np.float64)
        return Workload(name or self.name, self.x0, self.v0, self.a0, self.adot0, self.m, self.t0,
                        self.t, act, np.ascontiguousarray(h_all[act]), dtr, self.cap, self.X, self.V,
                        dict(self.meta))


# ----------------------------------------------------------------- sampling

def plummer(n: int, rng: np.random.Generator):
    """Equal-mass Plummer sphere in Henon units (Aarseth, Henon & Wielen 1974).

    Radii from the inverted cumulative mass, isotropic directions, speeds by
    von Neumann rejection on q^2 (1-q^2)^(7/2), then the centre of mass is
    moved to rest at the origin.  Returns positions and velocities [n,3].
    """
    x = np.empty((n, 3))
    v = np.empty((n, 3))
    # radii (cut the extreme tail at 0.999 of the mass like the usual recipe)
    mass_frac = rng.uniform(0.0, 0.999, n)
    r = 1.0 / np.sqrt(mass_frac ** (-2.0 / 3.0) - 1.0)
    x[:] = _isotropic(rng, n) * r[:, None]
    # speeds: g(q) = q^2 (1 - q^2)^3.5 <= 0.1
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        q1 = rng.uniform(0.0, 1.0, todo.size)
        y = rng.uniform(0.0, 0.1, todo.size)
        ok = y < q1 * q1 * (1.0 - q1 * q1) ** 3.5
        q[todo[ok]] = q1[ok]
        todo = todo[~ok]
    vesc = math.sqrt(2.0) * (1.0 + r * r) ** (-0.25)
    v[:] = _isotropic(rng, n) * (q * vesc)[:, None]
    # Plummer units (a = 1) -> Henon units
    x *= HENON_PLUMMER_B
    v /= math.sqrt(HENON_PLUMMER_B)
    x -= x.mean(axis=0)
    v -= v.mean(axis=0)
    return x, v


def _isotropic(rng, n):
    z = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    s = np.sqrt(1.0 - z * z)
    return np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)


def kroupa_masses(n: int, rng: np.random.Generator, lo=0.08, brk=0.5, hi=100.0,
                  alpha1=1.3, alpha2=2.3):
    """Kroupa (2001) two-segment IMF on [lo, hi] Msun, normalised to sum 1.

    dN/dm ~ m^-alpha1 below the break and m^-alpha2 above, continuous at the
    break; each segment is sampled by inverting its power-law CDF.
    """
    def seg_int(a, m1, m2):
        return (m2 ** (1 - a) - m1 ** (1 - a)) / (1 - a)
    w1 = seg_int(alpha1, lo, brk)
    w2 = brk ** (alpha2 - alpha1) * seg_int(alpha2, brk, hi)   # continuity at the break
    pick_low = rng.uniform(0, 1, n) < w1 / (w1 + w2)
    u = rng.uniform(0, 1, n)

    def inv(a, m1, m2, u):
        e = 1 - a
        return (m1 ** e + u * (m2 ** e - m1 ** e)) ** (1 / e)
    m = np.where(pick_low, inv(alpha1, lo, brk, u), inv(alpha2, brk, hi, u))
    return m / m.sum()


def plummer_field(X, V, M=1.0, b=HENON_PLUMMER_B):
    """Smooth field of a Plummer potential of mass M and scale b at (X, V):
    acceleration -M X/(r^2+b^2)^(3/2) and its derivative along the motion.
    A background field only; used to give the predictor realistic a, da/dt."""
    s2 = (X * X).sum(axis=1) + b * b
    s3 = s2 ** 1.5
    xv = (X * V).sum(axis=1)
    a = -M * X / s3[:, None]
    adot = -M * (V / s3[:, None] - 3.0 * (xv / (s3 * s2))[:, None] * X)
    return a, adot


def power_of_two_steps(n, rng, kmin=3, kmax=12):
    """Per-particle steps 2^-k with k uniform in [kmin, kmax] (block hierarchy)."""
    return np.ldexp(1.0, -rng.integers(kmin, kmax + 1, n))


def backfill(X, V, a0, adot0, dt):
    """Start-of-step (x0, v0) whose third-order Taylor prediction over dt gives (X, V)."""
    dt = np.asarray(dt, dtype=np.float64)[:, None]
    v0 = V - a0 * dt - adot0 * (dt * dt / 2.0)
    x0 = X - v0 * dt - a0 * (dt * dt / 2.0) - adot0 * (dt * dt * dt / 6.0)
    return x0, v0


def place_hard_pairs(X, V, m, frac, rng, log_sep=(-5.0, -2.0)):
    """Turn a fraction `frac` of the particles into bound pairs.

    For frac*n/2 pairs a secondary is moved next to a primary at separation
    10^U(log_sep) in a random direction, on a circular relative orbit.
    Returns the (primary, secondary) index arrays and the separations.
    """
    n = X.shape[0]
    npairs = int(round(frac * n / 2))
    idx = rng.permutation(n)[: 2 * npairs]
    prim, sec = idx[:npairs], idx[npairs:]
    sep = 10.0 ** rng.uniform(log_sep[0], log_sep[1], npairs)
    u = _isotropic(rng, npairs)
    w = np.cross(u, _isotropic(rng, npairs))
    w /= np.linalg.norm(w, axis=1)[:, None]
    vorb = np.sqrt((m[prim] + m[sec]) / sep)
    X[sec] = X[prim] + sep[:, None] * u
    V[sec] = V[prim] + vorb[:, None] * w
    return prim, sec, sep


# ------------------------------------------------------------- radii choice

def choose_radii(X, V, who, k_lo, k_hi, rng, dtr=None, margin=MARGIN, chunk=8192):
    """Neighbour radii for the particles `who`, from k-nearest distances.

    Particle i gets K_i uniform in [k_lo, k_hi] and a radius strictly between
    its K_i-th and (K_i+1)-th nearest distances (geometric interpolation with
    a random weight), moved to the next gap if the chosen one is narrower than
    the margin.  With `dtr` (per-particle regular steps, one of a few values)
    the distance is min(|R|, |R + dtr_i V|) (the velocity criterion of the
    paper's Sec. 3.2); its K nearest are found from two trees.
    Every pair distance of i then differs from r_i by a relative `margin` or
    more.  Returns (h, K) for `who`.
    """
    from scipy.spatial import cKDTree

    who = np.asarray(who)
    n = X.shape[0]
    kq = min(n, k_hi + 3)
    K = rng.integers(k_lo, k_hi + 1, who.size)
    wgt = rng.uniform(0.3, 0.7, who.size)
    h = np.empty(who.size)
    tree = cKDTree(X)
    trees_v = {}
    if dtr is not None:
        for d in np.unique(dtr[who]):
            trees_v[float(d)] = cKDTree(X + d * V)
    for s in range(0, who.size, chunk):
        sl = slice(s, min(s + chunk, who.size))
        ii = who[sl]
        _, nb = tree.query(X[ii], k=kq, workers=-1)
        if dtr is None:
            cand = nb
        else:
            cand = np.empty((ii.size, 2 * kq), dtype=np.int64)
            cand[:, :kq] = nb
            for d, tv in trees_v.items():
                rows = np.nonzero(dtr[ii] == d)[0]
                if rows.size:
                    _, nb2 = tv.query(X[ii[rows]] + d * V[ii[rows]], k=kq, workers=-1)
                    cand[rows, kq:] = nb2
            cand = np.sort(cand, axis=1)
        R = X[cand] - X[ii][:, None, :]
        q = np.sqrt((R * R).sum(axis=2))
        if dtr is not None:
            P = R + dtr[ii][:, None, None] * (V[cand] - V[ii][:, None, :])
            q = np.minimum(q, np.sqrt((P * P).sum(axis=2)))
            dup = np.zeros_like(q, dtype=bool)
            dup[:, 1:] = cand[:, 1:] == cand[:, :-1]
            q[dup] = np.inf
        q[cand == ii[:, None]] = np.inf        # self
        q.sort(axis=1)
        for r in range(ii.size):
            k = int(K[sl][r])
            while True:
                lo_d, hi_d = q[r, k - 1], q[r, k]
                hh = lo_d ** (1 - wgt[sl][r]) * hi_d ** wgt[sl][r]
                if hh > lo_d * (1 + margin) and hh < hi_d * (1 - margin):
                    break
                k += 1
                if k >= q.shape[1] - 1:
                    raise RuntimeError("no radius gap wider than the margin")
            h[s + r] = hh
            K[s + r] = k
    return h, K


# ------------------------------------------------------------------ configs

def _cache_dir():
    d = os.environ.get("NBREG_INPUT_CACHE", os.path.join("/tmp", "nbreg_inputs"))
    os.makedirs(d, exist_ok=True)
    return d


def cluster(n, seed, k_nb, cap, dt_mode="hierarchy", dt_fixed=2.0**-10, masses="equal",
            offset=0.0, pair_frac=0.0, act=None, accel=None, dtr_steps=None, name=None, bulk_v=None):
    """One Plummer cluster at block time t = 2 with per-particle radii.

    n          particles; seed: PCG64 seed
    k_nb       mean neighbour count (each particle gets K in [0.75 k, 1.25 k])
    cap        list capacity stored in the workload
    dt_mode    "fixed" (all steps dt_fixed) or "hierarchy" (2^-3 .. 2^-12)
    masses     "equal" or "kroupa"
    offset     |centre| of the cluster (along (1,1,1))
    pair_frac  fraction of particles placed in hard pairs
    act        active indices (default: all particles)
    accel      None (Plummer field) or a callable (X, V, m) -> (a0, adot0)
    dtr_steps  None (plain criterion) or a tuple of regular steps drawn per particle
    bulk_v     None or a velocity (3-vector) added to every particle
    """
    rng = np.random.default_rng(np.random.PCG64(seed))
    X, V = plummer(n, rng)
    m = np.full(n, 1.0 / n) if masses == "equal" else kroupa_masses(n, rng)
    meta = {"seed": seed, "k_nb": k_nb}
    if pair_frac > 0:
        prim, sec, sep = place_hard_pairs(X, V, m, pair_frac, rng)
        meta.update(pair_primary=prim, pair_secondary=sec, pair_sep=sep)
    if offset:
        X += offset / math.sqrt(3.0)
    if bulk_v is not None:
        V = V + np.asarray(bulk_v, dtype=np.float64)
    if dt_mode == "fixed":
        dt = np.full(n, dt_fixed)
    else:
        dt = power_of_two_steps(n, rng)
    dtr_all = None
    if dtr_steps is not None:
        dtr_all = rng.choice(np.asarray(dtr_steps, dtype=np.float64), n)
    act = np.arange(n, dtype=np.int32) if act is None else np.asarray(act, dtype=np.int32)
    who = np.arange(n) if act.size == n else np.unique(act)
    k_lo, k_hi = max(1, int(round(0.75 * k_nb))), max(1, int(round(1.25 * k_nb)))
    k_hi = min(k_hi, n - 3)
    k_lo = min(k_lo, k_hi)
    h_who, K_who = choose_radii(X, V, who, k_lo, k_hi, rng, dtr=dtr_all)
    h_all = np.full(n, np.nan)
    h_all[who] = h_who
    meta.update(h_all=h_all, dtr_all=dtr_all, K=K_who)
    if accel is None:
        a0, adot0 = plummer_field(X - (offset / math.sqrt(3.0) if offset else 0.0), V)
    else:
        a0, adot0 = accel(X, V, m)
    x0, v0 = backfill(X, V, a0, adot0, dt)
    t = BLOCK_TIME
    t0 = t - dt
    h = np.ascontiguousarray(h_all[act])
    dtr = None if dtr_all is None else np.ascontiguousarray(dtr_all[act])
    return Workload(name or f"plummer-n{n}-s{seed}", x0, v0, a0, adot0, m, t0, t, act, h, dtr,
                    int(cap), X, V, meta)


# Workloads shaped like the five benchmark configurations.

def config1(accel=None):
    """Equal-mass Plummer, N = 1024, seed 1, all active, dt = 2^-10, ~32 nb, cap 128."""
    return cluster(1024, 1, 32, 128, dt_mode="fixed", accel=accel, name="plummer-n1024")


def config2(n_act=None):
    """Equal-mass Plummer, N = 16384, seed 2, steps 2^-3..2^-12, ~64 nb, cap 256.
    Returns the all-active workload; use ``subset(w, n_act, seed)`` for the sweep."""
    w = cluster(16384, 2, 64, 256, name="plummer-n16384")
    return w if n_act is None else subset(w, n_act, 2)


def config3(n_act=None):
    """Kroupa-IMF Plummer, N = 131072, seed 3, ~100 nb, cap 256."""
    w = cluster(131072, 3, 100, 256, masses="kroupa", name="plummer-kroupa-n131072")
    return w if n_act is None else subset(w, n_act, 3)


def config4(n_clusters=64, seed=4):
    """64 independent equal-mass Plummer clusters, N log-uniform in [1024, 32768],
    n_act log-uniform in [8, N], ~64 nb, cap 256."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    ns = np.rint(np.exp(rng.uniform(math.log(1024), math.log(32768), n_clusters))).astype(int)
    out = []
    for c, n in enumerate(ns):
        na = int(round(math.exp(rng.uniform(math.log(8), math.log(n)))))
        act = np.sort(rng.choice(n, na, replace=False)).astype(np.int32)
        out.append(cluster(int(n), seed * 1000 + c, 64, 256, act=act, name=f"cluster{c}-n{n}"))
    return out


def config5(n_act=None, n=262144):
    """Offset (|x_c| = 1e3) Plummer, N = 262144, seed 5, 10% hard pairs, ~128 nb, cap 256."""
    w = cluster(n, 5, 128, 256, offset=1e3, pair_frac=0.10, name=f"plummer-offset-pairs-n{n}")
    return w if n_act is None else subset(w, n_act, 5)


def subset(w: Workload, n_act: int, seed: int) -> Workload:
    """A seeded random active subset (without replacement, ascending)."""
    rng = np.random.default_rng(np.random.PCG64(seed * 7919 + n_act))
    act = np.sort(rng.choice(w.n, n_act, replace=False)).astype(np.int32)
    return w.with_active(act, dtr_all=w.meta.get("dtr_all"), name=f"{w.name}-act{n_act}")


def cached(fn, *args, key=None):
    """Memoise a generated workload on disk (npz under /tmp or $NBREG_INPUT_CACHE)."""
    import pickle
    key = key or (fn.__name__ + "_" + "_".join(str(a) for a in args))
    path = os.path.join(_cache_dir(), key + ".pkl")
    if os.path.exists(path):
        with open(path, "rb") as f:
            return pickle.load(f)
    w = fn(*args)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "wb") as f:
        pickle.dump(w, f, protocol=pickle.HIGHEST_PROTOCOL)
    os.replace(tmp, path)
    return w
