// Registry entry for one instantiation of the regular-force kernel.
#pragma once

#include "nb_aux.cuh"
#include "nb_regf.cuh"
#include "nb_regf2.cuh"
#include "nb_regf3.cuh"

#define NB_KERNEL_ENTRY(FORM, MODE, W, I, JT, FL)                                       \
    {                                                                                   \
        MODE, W, I, JT, FL, 0, reinterpret_cast<const void *>(&nb::regf_kernel<FORM, W, I, JT, FL>), \
            128 + 2 * FORM::NS * FORM::EB * JT                                          \
    }

// MINB: resident CTAs per SM the register allocation must allow.
#define NB_KERNEL_ENTRY2(FORM, MODE, W, I, JT, FL, MINB)                                \
    {                                                                                   \
        MODE, W, I, JT, FL, 1,                                                          \
            reinterpret_cast<const void *>(&nb::regf2_kernel<FORM, W, I, JT, FL, MINB>), \
            nb::packed_smem_bytes<FORM, W, I, JT>(((FL) & 2) != 0)                     \
    }

#define NB_KERNEL_ENTRY3(FORM, MODE, W, I, JT, FL, MINB)                                \
    {                                                                                   \
        MODE, W, I, JT, FL, 2,                                                          \
            reinterpret_cast<const void *>(&nb::regf3_kernel<FORM, W, I, JT, FL, MINB>), \
            nb::pair_smem_bytes<FORM, W, I, JT>(((FL) & 2) != 0)                       \
    }
