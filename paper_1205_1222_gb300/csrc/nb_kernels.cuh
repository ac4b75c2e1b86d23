// Registry entry for one instantiation of the regular-force kernel.
#pragma once

#include "nb_aux.cuh"
#include "nb_regf.cuh"
#include "nb_regf3.cuh"
#include "nb_regf_ws.cuh"
#include "nb_regf_cl.cuh"

#define NB_KERNEL_ENTRY(FORM, MODE, W, I, JT, FL)                                       \
    {                                                                                   \
        MODE, W, I, JT, FL, 0, reinterpret_cast<const void *>(&nb::regf_kernel<FORM, W, I, JT, FL>), \
            128 + 2 * FORM::NS * FORM::EB * JT                                          \
    }

// NST: depth of the j-tile ring; U: j-pairs per lane per step.
#define NB_KERNEL_ENTRY3(FORM, MODE, W, I, JT, NST, U, FL, MINB)                        \
    {                                                                                   \
        MODE, W, I, JT, FL, (U) == 1 ? 2 : 3,                                           \
            reinterpret_cast<const void *>(&nb::regf3_kernel<FORM, nb::NoFrame, W, I, JT, NST, U, FL, MINB>), \
            nb::pair_smem_bytes<FORM, W, I, JT, NST>(((FL) & 2) != 0)                  \
    }

// Two-float positions with FP32 velocities (packed = 5), j-pair kernel.
#define NB_KERNEL_ENTRY5(W, I, JT, NST, FL, MINB)                                       \
    {                                                                                   \
        1, W, I, JT, FL, 5,                                                             \
            reinterpret_cast<const void *>(&nb::regf3_kernel<nb::PairMixedX, nb::NoFrame, W, I, JT, NST, 1, FL, MINB>), \
            nb::pair_smem_bytes<nb::PairMixedX, W, I, JT, NST>(((FL) & 2) != 0)        \
    }

// j-pair kernel with WC compute warps and NL list warps (packed = 5 + NL) and
// a four-slot flag ring; the entry's warps field is the CTA's total (WC + NL).
#define NB_KERNEL_ENTRY6(FORM, MODE, WC, NL, I, JT, NST, FL)                            \
    {                                                                                   \
        MODE, (WC) + (NL), I, JT, FL, 5 + (NL),                                         \
            reinterpret_cast<const void *>(&nb::regf3ws_kernel<FORM, WC, NL, I, JT, NST, FL, 4>), \
            nb::ws_smem_bytes<FORM, WC, NL, I, JT, NST, 4>(((FL) & 2) != 0), NL        \
    }

// The exact pair form (two-float position and velocity differences) with NL
// list warps: packed = 10 + NL.
#define NB_KERNEL_ENTRY7(WC, NL, I, JT, NST, FL)                                        \
    {                                                                                   \
        1, (WC) + (NL), I, JT, FL, 10 + (NL),                                           \
            reinterpret_cast<const void *>(&nb::regf3ws_kernel<nb::PairMixed, WC, NL, I, JT, NST, FL>), \
            nb::ws_smem_bytes<nb::PairMixed, WC, NL, I, JT, NST>(((FL) & 2) != 0), NL  \
    }

// Thread-block-cluster kernel for small calls (packed = 20): the j-splits of
// a block of active particles are the CTAs of one cluster and reduce through
// distributed shared memory.  smem is the size without the list segments
// (those add W * I * cap * 4 bytes at launch).
#define NB_KERNEL_ENTRY_CL(FORM, MODE, W, I, JT, FL)                                    \
    {                                                                                   \
        MODE, W, I, JT, FL, 20, reinterpret_cast<const void *>(&nb::regf_cl_kernel<FORM, W, I, JT, FL>), \
            nb::ClLayout<FORM, W, I, JT>::bytes(((FL) & 2) != 0, 0)                     \
    }

// Framed two-float kernel (packed = 4): compact blocks of the spatially sorted
// active set use frame coordinates, the others the per-pair two-float form.
#define NB_KERNEL_ENTRY4(W, I, JT, NST, U, FL, MINB)                                    \
    {                                                                                   \
        1, W, I, JT, FL, 4,                                                             \
            reinterpret_cast<const void *>(                                             \
                &nb::regf3_kernel<nb::PairMixed, nb::FramedMixed, W, I, JT, NST, U, FL, MINB>), \
            nb::pair_smem_bytes<nb::PairMixed, W, I, JT, NST>(((FL) & 2) != 0)         \
    }
