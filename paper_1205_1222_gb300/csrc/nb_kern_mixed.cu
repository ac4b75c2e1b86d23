// Compiled configurations of the two-float (NB_MIXED) regular-force kernel:
// packed f32x2 j-pair kernels (two-float positions with FP32 velocity
// differences, with separate list warps (the default) or without; the exact
// two-float pair form; the framed form) and the scalar kernel.  The first entry of each
// flag value is the default; all flag-0 entries form the autotuner's search
// space.
#include "nb_kernels.cuh"

namespace nb {

static const KernelEntry g_mixed[] = {
    NB_KERNEL_ENTRY6(PairMixedX, 1, 12, 4, 2, 1024, 4, 0),
    NB_KERNEL_ENTRY6(PairMixedX, 1, 12, 4, 2, 1024, 4, 1),
    NB_KERNEL_ENTRY6(PairMixedX, 1, 12, 4, 2, 1024, 4, 2),
    NB_KERNEL_ENTRY6(PairMixedX, 1, 12, 4, 2, 1024, 4, 3),
    NB_KERNEL_ENTRY7(12, 4, 2, 1536, 2, 0),                 // exact pair form with list warps
    NB_KERNEL_ENTRY5(16, 2, 1024, 4, 0, 1),
    NB_KERNEL_ENTRY5(16, 2, 1024, 4, 1, 1),
    NB_KERNEL_ENTRY5(16, 2, 1024, 4, 2, 1),
    NB_KERNEL_ENTRY5(16, 2, 1024, 4, 3, 1),
    NB_KERNEL_ENTRY5(12, 2, 1024, 4, 0, 1),
    NB_KERNEL_ENTRY5(16, 2, 512, 4, 0, 1),
    NB_KERNEL_ENTRY5(16, 2, 1536, 2, 0, 1),
    NB_KERNEL_ENTRY3(PairMixed, 1, 16, 2, 512, 4, 1, 0, 1),
    NB_KERNEL_ENTRY3(PairMixed, 1, 16, 2, 512, 4, 1, 1, 1),
    NB_KERNEL_ENTRY3(PairMixed, 1, 16, 2, 512, 4, 1, 2, 1),
    NB_KERNEL_ENTRY3(PairMixed, 1, 16, 2, 512, 4, 1, 3, 1),
    NB_KERNEL_ENTRY3(PairMixed, 1, 16, 2, 512, 4, 2, 0, 1),
    NB_KERNEL_ENTRY3(PairMixed, 1, 12, 2, 512, 4, 1, 0, 1),
    NB_KERNEL_ENTRY_CL(PairMixedX, 1, 8, 2, 1024, 0),   // cluster kernels for small calls
    NB_KERNEL_ENTRY_CL(PairMixedX, 1, 16, 2, 1024, 0),
    NB_KERNEL_ENTRY_CL(PairMixedX, 1, 8, 2, 512, 0),
    NB_KERNEL_ENTRY_CL(PairMixedX, 1, 8, 1, 1024, 0),   // 8 particles per block: half the work per CTA
    NB_KERNEL_ENTRY_CL(PairMixedX, 1, 16, 1, 1024, 0),
    NB_KERNEL_ENTRY_CL(PairMixedX, 1, 4, 2, 1024, 0),
    NB_KERNEL_ENTRY4(16, 2, 512, 4, 1, 0, 1),
    NB_KERNEL_ENTRY4(16, 2, 512, 4, 1, 2, 1),
    NB_KERNEL_ENTRY4(12, 2, 512, 4, 1, 0, 1),
    NB_KERNEL_ENTRY(FormMixed, 1, 8, 4, 512, 0),
    NB_KERNEL_ENTRY(FormMixed, 1, 4, 4, 512, 0),
    NB_KERNEL_ENTRY(FormMixed, 1, 8, 2, 512, 0),
    NB_KERNEL_ENTRY(FormMixed, 1, 16, 2, 512, 0),
    // per-particle layout with the velocity criterion and/or the potential: the
    // fallback for a j-range that starts at an odd slot
    NB_KERNEL_ENTRY(FormMixed, 1, 8, 2, 512, 1),
    NB_KERNEL_ENTRY(FormMixed, 1, 8, 2, 512, 2),
    NB_KERNEL_ENTRY(FormMixed, 1, 8, 2, 512, 3),
};

const KernelEntry *kernels_mixed(int *count)
{
    *count = static_cast<int>(sizeof(g_mixed) / sizeof(g_mixed[0]));
    return g_mixed;
}

}  // namespace nb
