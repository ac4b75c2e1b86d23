"""GB300-native Ahmad-Cohen regular force for direct N-body integration.

For every active particle of a block step the CUDA library libnbreg computes
the regular force, its time derivative and the neighbour list after predicting
all j-particles to the block time (Nitadori & Aarseth 2012, Sec. 3.2-3.4).
The C-ABI is include/nbreg.h; ``binding`` holds the same-name ctypes calls and
``Context`` below is a thin torch-tensor convenience over them (it allocates
output tensors and forwards pointers; it computes nothing itself).
"""
from __future__ import annotations

from . import binding as _b
from .binding import (MODES, NB_FORM_ALL, NB_FORM_FP32, NB_FORM_FP64, NB_FORM_MIXED, NB_FP32,
                      NB_FP64, NB_KEEP_FRAME, NB_MIXED, NbError, nb_kcfg)

__all__ = ["Context", "NbError", "MODES", "NB_FP64", "NB_MIXED", "NB_FP32", "NB_FORM_ALL",
           "NB_FORM_FP64", "NB_FORM_MIXED", "NB_FORM_FP32", "NB_KEEP_FRAME", "nb_kcfg", "mode_id"]


def mode_id(mode) -> int:
    return MODES[mode] if isinstance(mode, str) else int(mode)


class Context:
    """One libnbreg context (the paper's GPUNB_OPEN ... GPUNB_CLOSE)."""

    def __init__(self, n_max: int, device: int = 0):
        self.device = int(device)
        self.n_max = int(n_max)
        self.h = _b.nb_create(self.device, self.n_max)

    def close(self):
        if self.h:
            _b.nb_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # j-set -----------------------------------------------------------------
    def predict(self, x0, v0, a0, adot0, m, t0, t, offset=0, forms=0, stream=None):
        _b.nb_predict(self.h, offset, m.shape[0], x0, v0, a0, adot0, m, t0, t, forms, stream)

    def set_predicted(self, x, v, m, offset=0, forms=0, stream=None):
        _b.nb_set_predicted(self.h, offset, m.shape[0], x, v, m, forms, stream)

    # regular force ---------------------------------------------------------
    def alloc_outputs(self, n_act, cap, pot=False):
        import torch
        dev = torch.device("cuda", self.device)
        return {
            "F": torch.empty((n_act, 3), dtype=torch.float64, device=dev),
            "J": torch.empty((n_act, 3), dtype=torch.float64, device=dev),
            "pot": torch.empty((n_act,), dtype=torch.float64, device=dev) if pot else None,
            "nnb": torch.empty((n_act,), dtype=torch.int32, device=dev),
            "list": torch.full((n_act, cap), -1, dtype=torch.int32, device=dev) if cap > 0 else None,
            "ovf": torch.empty((n_act,), dtype=torch.uint8, device=dev),
        }

    def regular_force(self, act, h, n_j, dtr=None, cap=256, mode="mixed", j_begin=0, pot=False,
                      out=None, stream=None):
        n_act = int(act.shape[0])
        out = out or self.alloc_outputs(n_act, cap, pot)
        _b.nb_regular_force(self.h, j_begin, n_j, n_act, act, h, dtr, cap, mode_id(mode), out["F"],
                            out["J"], out["pot"] if pot else None, out["nnb"], out["list"], out["ovf"], stream)
        return out

    def irregular_force(self, act, nnb, lst, n_j, cap, mode="mixed", j_begin=0, pot=False, stream=None):
        """Irregular force and jerk over the neighbour lists (FP64 outputs)."""
        import torch
        n_act = int(act.shape[0])
        dev = torch.device("cuda", self.device)
        out = {"F": torch.empty((n_act, 3), dtype=torch.float64, device=dev),
               "J": torch.empty((n_act, 3), dtype=torch.float64, device=dev),
               "pot": torch.empty((n_act,), dtype=torch.float64, device=dev) if pot else None}
        _b.nb_irregular_force(self.h, j_begin, n_j, n_act, act, nnb, lst, cap, mode_id(mode), out["F"], out["J"],
                              out["pot"], stream)
        return out

    def sync_status(self, stream=None) -> int:
        return _b.nb_sync_status(self.h, stream)

    def last_launches(self) -> int:
        return _b.nb_last_launches(self.h)

    def sm_count(self) -> int:
        return _b.nb_sm_count(self.h)

    def reserve(self, nbytes):
        _b.nb_reserve(self.h, nbytes)

    def scratch_bytes(self, n_j, n_act, cap, mode):
        return _b.nb_scratch_bytes(self.h, n_j, n_act, cap, mode_id(mode))

    def set_config(self, mode, cfg):
        _b.nb_set_kernel_config(self.h, mode_id(mode), cfg)

    def active_config(self, mode):
        return _b.nb_get_active_config(self.h, mode_id(mode))

    def autotune(self, act, h, n_j, dtr=None, cap=256, mode="mixed", j_begin=0, pot=False, out=None,
                 reps=3, stream=None):
        """Tune the tiling for this call's size class (native nb_autotune);
        returns (best nb_kcfg, mean ms per call).  Overwrites `out`."""
        n_act = int(act.shape[0])
        out = out or self.alloc_outputs(n_act, cap, pot)
        return _b.nb_autotune(self.h, j_begin, n_j, n_act, act, h, dtr, cap, mode_id(mode), out["F"], out["J"],
                              out["pot"] if pot else None, out["nnb"], out["list"], out["ovf"], reps, stream)
