"""Persistence of the autotuner's table (the tuning itself is native).

``nb_autotune`` in libnbreg times every compiled tiling and j-split of a mode
on a caller's call and records the fastest for the call's size class (mode,
flags, floor(log2 n_act), floor(log2 n_j)) in the context; later calls of the
class use it.  This module saves that table as JSON and loads it into another
context, so a run can start from the tilings an earlier run measured on the
same GPU.
"""
from __future__ import annotations

import json

from . import binding as _b

FORMAT = "nbreg-tuned-v1"


def table(ctx) -> list:
    """The context's tuned entries as plain dicts."""
    h = ctx.h if hasattr(ctx, "h") else ctx
    rows = []
    for t in _b.nb_tuned_table(h):
        rows.append({"mode": t.mode, "flags": t.flags, "act_class": t.act_class, "j_class": t.j_class,
                     "cfg": list(t.cfg.as_tuple()), "ms": float(t.ms)})
    return rows


def save(ctx, path: str, device_name: str = "") -> None:
    """Write the tuned table of `ctx` to `path` (JSON)."""
    with open(path, "w") as f:
        json.dump({"format": FORMAT, "device": device_name, "entries": table(ctx)}, f, indent=1)


def load(ctx, path: str) -> int:
    """Insert the entries saved in `path` into `ctx`; returns how many were
    accepted (entries whose tiling the loaded library does not compile are skipped)."""
    h = ctx.h if hasattr(ctx, "h") else ctx
    with open(path) as f:
        doc = json.load(f)
    if doc.get("format") != FORMAT:
        raise ValueError(f"{path}: not a {FORMAT} file")
    n = 0
    for e in doc["entries"]:
        t = _b.nb_tuned()
        t.mode, t.flags, t.act_class, t.j_class = e["mode"], e["flags"], e["act_class"], e["j_class"]
        t.cfg = _b.nb_kcfg(*e["cfg"])
        t.ms = 0.0
        try:
            _b.nb_set_tuned(h, t)
            n += 1
        except _b.NbError as err:
            if err.status != _b.NB_ERR_UNSUPPORTED:
                raise
    return n
