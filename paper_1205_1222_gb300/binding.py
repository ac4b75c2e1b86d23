"""ctypes binding of libnbreg (include/nbreg.h).

Argument marshalling only: every function below forwards to the C entry point
of the same name; all arithmetic runs in the library's CUDA kernels.  Arrays
may be passed as torch tensors (their ``data_ptr()`` is used; they must live
where the C function expects them: device memory, or host memory for
``nb_step_host``) or as raw integer addresses.  A non-zero status raises
``NbError``.  There is no fallback: if libnbreg.so is missing, loading fails.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libnbreg.so")

NB_OK = 0
NB_ERR_ARG = -1
NB_ERR_CUDA = -2
NB_ERR_NOMEM = -3
NB_ERR_TIMEOUT = -4
NB_ERR_STATE = -5
NB_ERR_UNSUPPORTED = -6
NB_ERR_DEVICE_INPUT = -7
NB_ERR_INTERNAL = -8

NB_FP64, NB_MIXED, NB_FP32 = 0, 1, 2
MODES = {"fp64": NB_FP64, "mixed": NB_MIXED, "fp32": NB_FP32}
NB_FORM_FP64, NB_FORM_MIXED, NB_FORM_FP32, NB_FORM_ALL = 1, 2, 4, 7
NB_KEEP_FRAME = 8
NB_NEEDED_ONLY = 16
MODE_FORM = {NB_FP64: NB_FORM_FP64, NB_MIXED: NB_FORM_MIXED, NB_FP32: NB_FORM_FP32}

# Exported symbols declared in include/nbreg.h (checked by the ABI test).
EXPORTS = [
    "nb_create", "nb_destroy", "nb_predict", "nb_set_predicted", "nb_get_predicted", "nb_regular_force",
    "nb_reserve", "nb_scratch_bytes", "nb_plan_create", "nb_plan_run", "nb_plan_capture",
    "nb_plan_launch", "nb_plan_destroy", "nb_plan_launches", "nb_regular_force_batched", "nb_step_host",
    "nb_sync_status",
    "nb_strerror", "nb_last_error", "nb_num_kernel_configs", "nb_get_kernel_config",
    "nb_set_kernel_config", "nb_get_active_config", "nb_time_regular_force", "nb_last_launches",
    "nb_sm_count", "nb_debug_set_wait", "nb_regular_force_noalloc", "nb_debug_frame_stats",
    "nb_autotune", "nb_num_tuned", "nb_get_tuned", "nb_set_tuned", "nb_irregular_force",
    "nb_set_frame", "nb_get_frame", "nb_predict_needed", "nb_plan_autotune", "nb_plan_get_config",
]


class NbError(RuntimeError):
    def __init__(self, status, what, detail=""):
        self.status = status
        super().__init__(f"{what}: {strerror(status)} ({status}){': ' + detail if detail else ''}")


class nb_kcfg(ctypes.Structure):
    _fields_ = [("warps", ctypes.c_int32), ("ipw", ctypes.c_int32), ("jtile", ctypes.c_int32),
                ("split", ctypes.c_int32), ("packed", ctypes.c_int32)]

    def as_tuple(self):
        return (self.warps, self.ipw, self.jtile, self.split, self.packed)

    def __repr__(self):
        return "nb_kcfg(warps=%d, ipw=%d, jtile=%d, split=%d, packed=%d)" % self.as_tuple()


class nb_tuned(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("flags", ctypes.c_int32), ("act_class", ctypes.c_int32),
                ("j_class", ctypes.c_int32), ("cfg", nb_kcfg), ("ms", ctypes.c_float)]


class nb_cluster(ctypes.Structure):
    _fields_ = [("j_begin", ctypes.c_int64), ("n_j", ctypes.c_int64), ("n_act", ctypes.c_int32),
                ("cap", ctypes.c_int32), ("act", ctypes.c_void_p), ("h", ctypes.c_void_p),
                ("dtr", ctypes.c_void_p), ("F", ctypes.c_void_p), ("J", ctypes.c_void_p),
                ("pot", ctypes.c_void_p), ("nnb", ctypes.c_void_p), ("list", ctypes.c_void_p),
                ("ovf", ctypes.c_void_p)]


_lib = None


def library():
    """Load libnbreg.so (built in-tree by build.py).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run paper_1205_1222_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, i64, i32, dbl, cint = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_int
    sig = {
        "nb_create": ([ctypes.POINTER(P), cint, i64], cint),
        "nb_destroy": ([P], None),
        "nb_predict": ([P, i64, i64, P, P, P, P, P, P, dbl, cint, P], cint),
        "nb_set_predicted": ([P, i64, i64, P, P, P, cint, P], cint),
        "nb_get_predicted": ([P, i64, i64, P, P, P, P], cint),
        "nb_regular_force": ([P, i64, i64, i32, P, P, P, i32, cint, P, P, P, P, P, P, P], cint),
        "nb_reserve": ([P, ctypes.c_size_t], cint),
        "nb_scratch_bytes": ([P, i64, i32, i32, cint], ctypes.c_size_t),
        "nb_plan_create": ([P, i32, P, cint, P, ctypes.POINTER(P)], cint),
        "nb_plan_run": ([P, P], cint),
        "nb_plan_capture": ([P, P], cint),
        "nb_plan_launch": ([P, P], cint),
        "nb_plan_destroy": ([P], None),
        "nb_plan_launches": ([P], cint),
        "nb_regular_force_batched": ([P, cint, P, cint, P], cint),
        "nb_step_host": ([P, i64, P, P, P, P, P, P, dbl, i32, P, P, P, i32, cint, P, P, P, P, P, P, P], cint),
        "nb_sync_status": ([P, P], cint),
        "nb_strerror": ([cint], ctypes.c_char_p),
        "nb_last_error": ([P], ctypes.c_char_p),
        "nb_num_kernel_configs": ([cint], cint),
        "nb_get_kernel_config": ([cint, cint, ctypes.POINTER(nb_kcfg)], cint),
        "nb_set_kernel_config": ([P, cint, ctypes.POINTER(nb_kcfg)], cint),
        "nb_get_active_config": ([P, cint, ctypes.POINTER(nb_kcfg)], cint),
        "nb_time_regular_force": ([P, ctypes.POINTER(nb_kcfg), i64, i64, i32, P, P, P, i32, cint, P, P, P,
                                   P, P, P, cint, P, ctypes.POINTER(ctypes.c_float)], cint),
        "nb_last_launches": ([P], cint),
        "nb_sm_count": ([P], cint),
        "nb_debug_set_wait": ([P, ctypes.c_uint64, ctypes.c_uint32], cint),
        "nb_debug_frame_stats": ([P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)], cint),
        "nb_regular_force_noalloc": ([P, i64, i64, i32, P, P, P, i32, cint, P, P, P, P, P, P, P], cint),
        "nb_autotune": ([P, i64, i64, i32, P, P, P, i32, cint, P, P, P, P, P, P, cint, P,
                         ctypes.POINTER(nb_kcfg), ctypes.POINTER(ctypes.c_float)], cint),
        "nb_num_tuned": ([P], cint),
        "nb_irregular_force": ([P, i64, i64, i32, P, P, P, i32, cint, P, P, P, P], cint),
        "nb_get_tuned": ([P, cint, ctypes.POINTER(nb_tuned)], cint),
        "nb_set_tuned": ([P, ctypes.POINTER(nb_tuned)], cint),
        "nb_set_frame": ([P, ctypes.POINTER(dbl)], cint),
        "nb_plan_autotune": ([P, cint, P, ctypes.POINTER(nb_kcfg), ctypes.POINTER(ctypes.c_float)], cint),
        "nb_plan_get_config": ([P, ctypes.POINTER(nb_kcfg)], cint),
        "nb_predict_needed": ([P, i64, i64, i32, P, P, P, i32, P, P, P, P, P, P, dbl, cint, P], cint),
        "nb_get_frame": ([P, ctypes.POINTER(dbl)], cint),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def strerror(status: int) -> str:
    try:
        return library().nb_strerror(int(status)).decode()
    except Exception:  # library not loadable: plain code
        return f"status {status}"


def _p(x):
    """Address of a tensor / int / None as a ctypes pointer value."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(ctx, rc, what):
    if rc != NB_OK:
        detail = ""
        if ctx:
            msg = library().nb_last_error(ctx)
            detail = msg.decode() if msg else ""
        raise NbError(rc, what, detail)


# --------------------------------------------------------- same-name calls

def nb_create(device: int, n_max: int):
    h = ctypes.c_void_p()
    _check(None, library().nb_create(ctypes.byref(h), int(device), int(n_max)), "nb_create")
    return h.value


def nb_destroy(ctx):
    library().nb_destroy(ctx)


def nb_predict(ctx, offset, n, x0, v0, a0, adot0, m, t0, t, forms=0, stream=None):
    _check(ctx, library().nb_predict(ctx, int(offset), int(n), _p(x0), _p(v0), _p(a0), _p(adot0), _p(m),
                                     _p(t0), float(t), int(forms), _stream(stream)), "nb_predict")


def nb_set_predicted(ctx, offset, n, x, v, m, forms=0, stream=None):
    _check(ctx, library().nb_set_predicted(ctx, int(offset), int(n), _p(x), _p(v), _p(m), int(forms),
                                           _stream(stream)), "nb_set_predicted")


def nb_get_predicted(ctx, offset, n, x, v, m=None, stream=None):
    _check(ctx, library().nb_get_predicted(ctx, int(offset), int(n), _p(x), _p(v), _p(m), _stream(stream)),
           "nb_get_predicted")


def nb_predict_needed(ctx, offset, n, n_act, act, nnb, lst, cap, x0, v0, a0, adot0, m, t0, t, forms=0,
                      stream=None):
    _check(ctx, library().nb_predict_needed(ctx, int(offset), int(n), int(n_act), _p(act), _p(nnb), _p(lst),
                                            int(cap), _p(x0), _p(v0), _p(a0), _p(adot0), _p(m), _p(t0), float(t),
                                            int(forms), _stream(stream)), "nb_predict_needed")


def nb_set_frame(ctx, u):
    a = (ctypes.c_double * 3)(*[float(x) for x in u])
    _check(ctx, library().nb_set_frame(ctx, a), "nb_set_frame")


def nb_get_frame(ctx):
    a = (ctypes.c_double * 3)()
    _check(ctx, library().nb_get_frame(ctx, a), "nb_get_frame")
    return [a[0], a[1], a[2]]


def nb_regular_force(ctx, j_begin, n_j, n_act, act, h, dtr, cap, mode, F, J, pot, nnb, lst, ovf,
                     stream=None):
    _check(ctx, library().nb_regular_force(ctx, int(j_begin), int(n_j), int(n_act), _p(act), _p(h), _p(dtr),
                                           int(cap), int(mode), _p(F), _p(J), _p(pot), _p(nnb), _p(lst),
                                           _p(ovf), _stream(stream)), "nb_regular_force")


def nb_irregular_force(ctx, j_begin, n_j, n_act, act, nnb, lst, cap, mode, F, J, pot=None, stream=None):
    _check(ctx, library().nb_irregular_force(ctx, int(j_begin), int(n_j), int(n_act), _p(act), _p(nnb), _p(lst),
                                             int(cap), int(mode), _p(F), _p(J), _p(pot), _stream(stream)),
           "nb_irregular_force")


def nb_regular_force_noalloc(ctx, j_begin, n_j, n_act, act, h, dtr, cap, mode, F, J, pot, nnb, lst, ovf,
                             stream=None):
    """nb_regular_force without any device allocation (fixed split scratch)."""
    _check(ctx, library().nb_regular_force_noalloc(ctx, int(j_begin), int(n_j), int(n_act), _p(act), _p(h),
                                                   _p(dtr), int(cap), int(mode), _p(F), _p(J), _p(pot),
                                                   _p(nnb), _p(lst), _p(ovf), _stream(stream)),
           "nb_regular_force_noalloc")


def nb_reserve(ctx, nbytes):
    _check(ctx, library().nb_reserve(ctx, int(nbytes)), "nb_reserve")


def nb_scratch_bytes(ctx, n_j, n_act, cap, mode):
    return int(library().nb_scratch_bytes(ctx, int(n_j), int(n_act), int(cap), int(mode)))


def nb_sync_status(ctx, stream=None):
    return int(library().nb_sync_status(ctx, _stream(stream)))


def nb_step_host(ctx, n, x0, v0, a0, adot0, m, t0, t, n_act, act, h, dtr, cap, mode, F, J, pot, nnb, lst,
                 ovf, stream=None):
    _check(ctx, library().nb_step_host(ctx, int(n), _p(x0), _p(v0), _p(a0), _p(adot0), _p(m), _p(t0),
                                       float(t), int(n_act), _p(act), _p(h), _p(dtr), int(cap), int(mode),
                                       _p(F), _p(J), _p(pot), _p(nnb), _p(lst), _p(ovf), _stream(stream)),
           "nb_step_host")


def nb_num_kernel_configs(mode):
    return int(library().nb_num_kernel_configs(int(mode)))


def nb_get_kernel_config(mode, index):
    c = nb_kcfg()
    _check(None, library().nb_get_kernel_config(int(mode), int(index), ctypes.byref(c)),
           "nb_get_kernel_config")
    return c


def nb_set_kernel_config(ctx, mode, cfg):
    _check(ctx, library().nb_set_kernel_config(ctx, int(mode), None if cfg is None else ctypes.byref(cfg)),
           "nb_set_kernel_config")


def nb_get_active_config(ctx, mode):
    c = nb_kcfg()
    _check(ctx, library().nb_get_active_config(ctx, int(mode), ctypes.byref(c)), "nb_get_active_config")
    return c


def nb_time_regular_force(ctx, cfg, j_begin, n_j, n_act, act, h, dtr, cap, mode, F, J, pot, nnb, lst, ovf,
                          reps=5, stream=None):
    ms = ctypes.c_float()
    _check(ctx, library().nb_time_regular_force(ctx, ctypes.byref(cfg), int(j_begin), int(n_j), int(n_act),
                                                _p(act), _p(h), _p(dtr), int(cap), int(mode), _p(F), _p(J),
                                                _p(pot), _p(nnb), _p(lst), _p(ovf), int(reps),
                                                _stream(stream), ctypes.byref(ms)),
           "nb_time_regular_force")
    return float(ms.value)


def nb_autotune(ctx, j_begin, n_j, n_act, act, h, dtr, cap, mode, F, J, pot, nnb, lst, ovf, reps=3,
                stream=None):
    best = nb_kcfg()
    ms = ctypes.c_float()
    _check(ctx, library().nb_autotune(ctx, int(j_begin), int(n_j), int(n_act), _p(act), _p(h), _p(dtr), int(cap),
                                      int(mode), _p(F), _p(J), _p(pot), _p(nnb), _p(lst), _p(ovf), int(reps),
                                      _stream(stream), ctypes.byref(best), ctypes.byref(ms)),
           "nb_autotune")
    return best, float(ms.value)


def nb_tuned_table(ctx):
    out = []
    for i in range(int(library().nb_num_tuned(ctx))):
        t = nb_tuned()
        _check(ctx, library().nb_get_tuned(ctx, i, ctypes.byref(t)), "nb_get_tuned")
        out.append(t)
    return out


def nb_set_tuned(ctx, entry):
    _check(ctx, library().nb_set_tuned(ctx, ctypes.byref(entry)), "nb_set_tuned")


def nb_last_launches(ctx):
    return int(library().nb_last_launches(ctx))


def nb_sm_count(ctx):
    return int(library().nb_sm_count(ctx))


def nb_debug_set_wait(ctx, wait_ns, extra_tx):
    _check(ctx, library().nb_debug_set_wait(ctx, int(wait_ns), int(extra_tx)), "nb_debug_set_wait")


def nb_debug_frame_stats(ctx):
    """(compact blocks, blocks) of the last framed call on the context."""
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(ctx, library().nb_debug_frame_stats(ctx, ctypes.byref(a), ctypes.byref(b)), "nb_debug_frame_stats")
    return a.value, b.value


def nb_plan_create(ctx, clusters, mode, cfg=None):
    arr = (nb_cluster * len(clusters))(*clusters)
    h = ctypes.c_void_p()
    _check(ctx, library().nb_plan_create(ctx, len(clusters), ctypes.cast(arr, ctypes.c_void_p), int(mode),
                                         None if cfg is None else ctypes.byref(cfg), ctypes.byref(h)),
           "nb_plan_create")
    return h.value


def nb_plan_run(plan, stream=None, ctx=None):
    _check(ctx, library().nb_plan_run(plan, _stream(stream)), "nb_plan_run")


def nb_plan_capture(plan, stream=None, ctx=None):
    _check(ctx, library().nb_plan_capture(plan, _stream(stream)), "nb_plan_capture")


def nb_plan_launch(plan, stream=None, ctx=None):
    _check(ctx, library().nb_plan_launch(plan, _stream(stream)), "nb_plan_launch")


def nb_plan_launches(plan):
    return int(library().nb_plan_launches(plan))


def nb_plan_get_config(plan):
    c = nb_kcfg()
    _check(None, library().nb_plan_get_config(plan, ctypes.byref(c)), "nb_plan_get_config")
    return c


def nb_plan_autotune(plan, reps=3, stream=None, ctx=None):
    """Tune the plan's tiling on its own clusters; returns (best nb_kcfg, mean ms per run)."""
    best = nb_kcfg()
    ms = ctypes.c_float()
    _check(ctx, library().nb_plan_autotune(plan, int(reps), _stream(stream), ctypes.byref(best), ctypes.byref(ms)),
           "nb_plan_autotune")
    return best, float(ms.value)


def nb_regular_force_batched(ctx, clusters, mode, stream=None):
    """One-shot batched call (plan built, run, waited for and freed)."""
    arr = (nb_cluster * len(clusters))(*clusters)
    _check(ctx, library().nb_regular_force_batched(ctx, len(clusters), ctypes.cast(arr, ctypes.c_void_p), int(mode),
                                                   _stream(stream)), "nb_regular_force_batched")


def nb_plan_destroy(plan):
    library().nb_plan_destroy(plan)
