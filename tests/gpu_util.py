"""Helpers of the GPU parity tests: run a workload through the C-ABI and
through the oracle, and compare element by element."""
import numpy as np

import oracle
from paper_1205_1222_gb300 import Context, mode_id

# Tolerances (relative 2-norm error per active particle).
#  * mixed two-float form: the bar the method is held to (force 1e-6, jerk 1e-5);
#  * FP64 form: rounding of an FP64 sum of N terms in another order plus the
#    FP64 reciprocal square root, bounded by ~N eps (Sum|f|/|F|) < 1e-10 for
#    the sizes tested here;
#  * plain FP32 form: reported, only loosely bounded where it is asserted.
TOL = {
    "fp64": (1e-10, 1e-10),
    "mixed": (1e-6, 1e-5),
    "fp32": (1e-4, 1e-3),
}


def dev(a, dtype=None):
    import torch
    dtype = dtype or torch.float64
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def upload(w):
    import torch
    return {
        "x0": dev(w.x0), "v0": dev(w.v0), "a0": dev(w.a0), "adot0": dev(w.adot0), "m": dev(w.m),
        "t0": dev(w.t0), "act": dev(w.act, torch.int32), "h": dev(w.h),
        "dtr": None if w.dtr is None else dev(w.dtr),
    }


def gpu_run(w, mode, cap=None, pot=False, ctx=None, j_offset=0, cfg=None, forms=0):
    """Predict + regular force on the GPU; returns numpy outputs, status, launches."""
    cap = w.cap if cap is None else cap
    own = ctx is None
    if own:
        ctx = Context(w.n + j_offset)
    try:
        d = upload(w)
        ctx.predict(d["x0"], d["v0"], d["a0"], d["adot0"], d["m"], d["t0"], w.t, offset=j_offset, forms=forms)
        if cfg is not None:
            ctx.set_config(mode, cfg)
        out = ctx.regular_force(d["act"], d["h"], w.n, dtr=d["dtr"], cap=cap, mode=mode, j_begin=j_offset,
                                pot=pot)
        status = ctx.sync_status()
        res = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
        res["status"] = status
        res["launches"] = ctx.last_launches()
        if cfg is not None:
            ctx.set_config(mode, None)
        return res
    finally:
        if own:
            ctx.close()


def oracle_predicted(w):
    return oracle.predict(w.x0, w.v0, w.a0, w.adot0, w.t0, w.t)


def oracle_run(w, cap=None, pot=False, rows=None):
    """Oracle outputs for all active particles, or for the rows `rows` of the active set."""
    cap = w.cap if cap is None else cap
    x, v = oracle_predicted(w)
    act, h, dtr = w.act, w.h, w.dtr
    if rows is not None:
        act, h = act[rows], h[rows]
        dtr = None if dtr is None else dtr[rows]
    return oracle.regular(x, v, w.m, act, h, dtr=dtr, cap=cap, with_pot=pot)


def rel_err(a, b):
    nb = np.linalg.norm(b, axis=1)
    d = np.linalg.norm(a - b, axis=1)
    return np.where(nb > 0, d / np.where(nb > 0, nb, 1.0), d)


def compare(g, o, cap, mode, rows=None, pot=False, lists=True):
    """Assert parity of GPU outputs `g` (optionally restricted to `rows`) with oracle `o`."""
    sel = (lambda a: a) if rows is None else (lambda a: a[rows])
    if lists:
        assert np.array_equal(sel(g["nnb"]), o["nnb"]), "neighbour counts differ"
        assert np.array_equal(sel(g["ovf"]), o["ovf"]), "overflow flags differ"
        if cap > 0:
            k = np.minimum(o["nnb"], cap)
            filled = np.arange(cap)[None, :] < k[:, None]
            gl = sel(g["list"])
            assert np.array_equal(np.where(filled, gl, -1), np.where(filled, o["list"], -1)), "lists differ"
            assert np.all(gl[~filled] == -1), "entries written past min(nnb, cap)"
    ftol, jtol = TOL[mode]
    eF = rel_err(sel(g["F"]), o["F"])
    eJ = rel_err(sel(g["J"]), o["J"])
    assert eF.max() <= ftol, f"force rel err {eF.max():.3e} > {ftol}"
    assert eJ.max() <= jtol, f"jerk rel err {eJ.max():.3e} > {jtol}"
    if pot:
        eP = np.abs(sel(g["pot"]) - o["pot"]) / np.abs(o["pot"])
        assert eP.max() <= ftol, f"potential rel err {eP.max():.3e}"
    return eF, eJ


# Unit roundoff of FP32.  A float-form pair term carries a relative rounding
# error of up to ~10 u (the approximate reciprocal square root enters r^-3
# three times; the differences, r^2 and the products add a few u), so on a
# row whose regular sum cancels to a small fraction of the sum of its term
# lengths S (condition number S / |F|), no FP32 term arithmetic reaches the
# per-particle relative bar; such a row is held to an absolute error of
# u * S instead (the per-term errors, largely independent, sum to well under
# their worst case over the hundreds of dominant terms).
U32 = 2.0 ** -24


def compare_conditioned(g, o, SF, SJ, cap, mode):
    """compare() for rows that may be ill-conditioned: lists exact; each row
    within the relative bar of `mode`, or within u * S (S = SF, SJ from
    oracle.regular_mag).  Returns the rows that needed the second bound,
    with their errors and condition numbers."""
    assert np.array_equal(g["nnb"], o["nnb"]), "neighbour counts differ"
    assert np.array_equal(g["ovf"], o["ovf"]), "overflow flags differ"
    k = np.minimum(o["nnb"], cap)
    filled = np.arange(cap)[None, :] < k[:, None]
    assert np.array_equal(np.where(filled, g["list"], -1), np.where(filled, o["list"], -1)), "lists differ"
    ftol, jtol = TOL[mode]
    dF = np.linalg.norm(g["F"] - o["F"], axis=1)
    dJ = np.linalg.norm(g["J"] - o["J"], axis=1)
    nF = np.linalg.norm(o["F"], axis=1)
    nJ = np.linalg.norm(o["J"], axis=1)
    okF = (dF <= ftol * nF) | (dF <= U32 * SF)
    okJ = (dJ <= jtol * nJ) | (dJ <= U32 * SJ)
    bad = np.nonzero(~(okF & okJ))[0]
    assert bad.size == 0, [(int(r), dF[r] / nF[r], dF[r] / SF[r], dJ[r] / nJ[r], dJ[r] / SJ[r]) for r in bad[:5]]
    cond = np.nonzero((dF > ftol * nF) | (dJ > jtol * nJ))[0]
    return [(int(r), float(dF[r] / nF[r]), float(SF[r] / nF[r]), float(dJ[r] / nJ[r]), float(SJ[r] / nJ[r]))
            for r in cond]


def list_mismatches(g, o, cap, rows=None):
    """Number of active particles whose count or stored list differs."""
    sel = (lambda a: a) if rows is None else (lambda a: a[rows])
    bad = sel(g["nnb"]) != o["nnb"]
    k = np.minimum(o["nnb"], cap)
    filled = np.arange(cap)[None, :] < k[:, None]
    bad |= np.any(np.where(filled, sel(g["list"]), -1) != np.where(filled, o["list"], -1), axis=1)
    return int(bad.sum())


def direct_sum_accel(X, V, m):
    """a, da/dt from the oracle's unsplit FP64 direct sum (a 'prior direct sum')."""
    F, J = oracle.full(X, V, m, np.arange(len(m), dtype=np.int32))
    return F, J
