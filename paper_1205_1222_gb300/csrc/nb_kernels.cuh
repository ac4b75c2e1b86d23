// Registry entry for one instantiation of the regular-force kernel.
#pragma once

#include "nb_aux.cuh"
#include "nb_regf.cuh"

#define NB_KERNEL_ENTRY(FORM, MODE, W, I, JT, FL)                                       \
    {                                                                                   \
        MODE, W, I, JT, FL, reinterpret_cast<const void *>(&nb::regf_kernel<FORM, W, I, JT, FL>), \
            128 + 2 * FORM::NS * FORM::EB * JT                                          \
    }
