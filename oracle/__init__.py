"""FP64 CPU oracle for the Ahmad-Cohen regular force (test infrastructure).

This package is the plain, slow reference that the CUDA path is checked
against.  It is test infrastructure: only the test suite, the smoke check and
the benchmark's CPU-baseline / reference leg may import it.  The CUDA library
never imports, links or calls it, and it shares no code with the CUDA path.

The arithmetic lives in ``nb_oracle.c`` (plain C, IEEE double, one loop per
definition of the paper); this module only compiles it with gcc and marshals
numpy arrays through ctypes.  Definitions followed (Nitadori & Aarseth 2012):

* ``predict``    - Sec. 3.3 step (iii): Taylor prediction of every j-particle
  to the block time (positions to dt^3, velocities to dt^2).
* ``regular``    - Sec. 3.3 step (vi) with the neighbour criterion of Sec. 3.2:
  regular force, regular jerk, neighbour list (ascending, lowest ``cap``
  entries kept, true count, overflow flag), optional potential.
* ``irregular``  - Sec. 3.3 step (iv): the same terms over the neighbour set.
* ``full``       - the unsplit direct sum over all j != i.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nb_oracle.c")
_LIB = os.path.join(_HERE, "_nb_oracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK = 0
ORC_ERR_ARG = -1
ORC_ERR_COINCIDENT = -2


class OracleError(RuntimeError):
    pass


def compile_source(src: str, out: str) -> str:
    """Compile an oracle C source into a shared library (gcc, -O2, OpenMP).

    No value-changing optimisation flags are used (no -ffast-math, FP
    contraction off), so every operation is one rounded IEEE double op.
    """
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", src, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile nb_oracle.c into _nb_oracle.so next to it (if out of date)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    return compile_source(_SRC, _LIB)


def open_library(path: str):
    """Load an oracle shared library and declare its C signatures."""
    lib = ctypes.CDLL(path)
    _declare(lib)
    return lib


_override = None


@contextlib.contextmanager
def using_library(path: str):
    """Route this module's functions through another compiled oracle (used by
    the tests that plant a mistake in a copy of the oracle source)."""
    global _override
    prev = _override
    _override = open_library(path)
    try:
        yield
    finally:
        _override = prev


def _load():
    global _lib
    if _override is not None:
        return _override
    with _lock:
        if _lib is not None:
            return _lib
        build()
        _lib = open_library(_LIB)
        return _lib


def _declare(lib):
    P = ctypes.c_void_p
    i64, i32, dbl, cint = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_int
    lib.orc_predict.argtypes = [i64, P, P, P, P, P, dbl, P, P]
    lib.orc_regular.argtypes = [i64, P, P, P, i32, P, P, P, i32, P, P, P, P, P, P, cint]
    lib.orc_irregular.argtypes = [i64, P, P, P, i32, P, P, P, P, P, cint]
    lib.orc_full.argtypes = [i64, P, P, P, i32, P, P, P, P, cint]
    lib.orc_regular_mag.argtypes = [i64, P, P, P, i32, P, P, P, P, P, cint]
    for f in (lib.orc_predict, lib.orc_regular, lib.orc_irregular, lib.orc_full, lib.orc_regular_mag):
        f.restype = cint
    lib.orc_default_threads.argtypes = []
    lib.orc_default_threads.restype = cint


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != shape:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, what):
    if rc == ORC_ERR_COINCIDENT:
        raise OracleError(f"{what}: coincident pair j != i outside the neighbour set (undefined input)")
    if rc != ORC_OK:
        raise OracleError(f"{what}: bad arguments (rc={rc})")


def default_threads() -> int:
    return int(_load().orc_default_threads())


def predict(x0, v0, a0, adot0, t0, t):
    """Predicted positions and velocities at block time ``t`` (Sec. 3.3 iii)."""
    lib = _load()
    x0 = _f64(x0); n = x0.shape[0]
    v0, a0, adot0 = _f64(v0, (n, 3)), _f64(a0, (n, 3)), _f64(adot0, (n, 3))
    t0 = _f64(t0, (n,))
    x = np.empty((n, 3)); v = np.empty((n, 3))
    _check(lib.orc_predict(n, _ptr(x0), _ptr(v0), _ptr(a0), _ptr(adot0), _ptr(t0),
                           float(t), _ptr(x), _ptr(v)), "predict")
    return x, v


def regular(x, v, m, act, h, dtr=None, cap=256, with_pot=False, threads=0):
    """Regular force/jerk/neighbour list for active particles (Sec. 3.3 vi).

    Returns a dict with F, J ([n_act,3]), nnb ([n_act] int32), list
    ([n_act,cap] int32, entries past min(nnb,cap) are -1), ovf ([n_act] uint8)
    and, if ``with_pot``, pot ([n_act]).
    """
    lib = _load()
    x = _f64(x); n = x.shape[0]
    v, m = _f64(v, (n, 3)), _f64(m, (n,))
    act = np.ascontiguousarray(act, dtype=np.int32); na = act.shape[0]
    h = _f64(h, (na,))
    dtr = None if dtr is None else _f64(dtr, (na,))
    F = np.zeros((na, 3)); J = np.zeros((na, 3))
    pot = np.zeros(na) if with_pot else None
    nnb = np.zeros(na, dtype=np.int32)
    lst = np.full((na, max(cap, 0)), -1, dtype=np.int32)
    ovf = np.zeros(na, dtype=np.uint8)
    _check(lib.orc_regular(n, _ptr(x), _ptr(v), _ptr(m), na, _ptr(act), _ptr(h), _ptr(dtr),
                           int(cap), _ptr(F), _ptr(J), _ptr(pot), _ptr(nnb),
                           _ptr(lst) if cap > 0 else None, _ptr(ovf), int(threads)), "regular")
    out = {"F": F, "J": J, "nnb": nnb, "list": lst, "ovf": ovf}
    if with_pot:
        out["pot"] = pot
    return out


def irregular(x, v, m, act, h, dtr=None, threads=0):
    """Irregular force/jerk over the neighbour set (Sec. 3.3 iv)."""
    lib = _load()
    x = _f64(x); n = x.shape[0]
    v, m = _f64(v, (n, 3)), _f64(m, (n,))
    act = np.ascontiguousarray(act, dtype=np.int32); na = act.shape[0]
    h = _f64(h, (na,))
    dtr = None if dtr is None else _f64(dtr, (na,))
    F = np.zeros((na, 3)); J = np.zeros((na, 3))
    _check(lib.orc_irregular(n, _ptr(x), _ptr(v), _ptr(m), na, _ptr(act), _ptr(h), _ptr(dtr),
                             _ptr(F), _ptr(J), int(threads)), "irregular")
    return F, J


def regular_mag(x, v, m, act, h, dtr=None, threads=0):
    """Sums of the lengths of the regular force and jerk terms of each active
    particle (SF, SJ): the condition numbers of the regular sums are SF/|F|
    and SJ/|J|."""
    lib = _load()
    x = _f64(x); n = x.shape[0]
    v, m = _f64(v, (n, 3)), _f64(m, (n,))
    act = np.ascontiguousarray(act, dtype=np.int32); na = act.shape[0]
    h = _f64(h, (na,))
    dtr = None if dtr is None else _f64(dtr, (na,))
    SF = np.zeros(na); SJ = np.zeros(na)
    _check(lib.orc_regular_mag(n, _ptr(x), _ptr(v), _ptr(m), na, _ptr(act), _ptr(h), _ptr(dtr),
                               _ptr(SF), _ptr(SJ), int(threads)), "regular_mag")
    return SF, SJ


def full(x, v, m, act, with_pot=False, threads=0):
    """Unsplit direct sum over all j != i: returns (F, J) or (F, J, pot)."""
    lib = _load()
    x = _f64(x); n = x.shape[0]
    v, m = _f64(v, (n, 3)), _f64(m, (n,))
    act = np.ascontiguousarray(act, dtype=np.int32); na = act.shape[0]
    F = np.zeros((na, 3)); J = np.zeros((na, 3))
    pot = np.zeros(na) if with_pot else None
    _check(lib.orc_full(n, _ptr(x), _ptr(v), _ptr(m), na, _ptr(act), _ptr(F), _ptr(J),
                        _ptr(pot), int(threads)), "full")
    return (F, J, pot) if with_pot else (F, J)
