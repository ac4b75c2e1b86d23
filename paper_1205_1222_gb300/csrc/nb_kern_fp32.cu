// Compiled configurations of the plain FP32 (NB_FP32) regular-force kernel.
#include "nb_kernels.cuh"

namespace nb {

static const KernelEntry g_fp32[] = {
    NB_KERNEL_ENTRY6(PairFP32, 2, 12, 4, 2, 1024, 4, 0),
    NB_KERNEL_ENTRY3(PairFP32, 2, 16, 2, 1024, 4, 1, 0, 1),
    NB_KERNEL_ENTRY3(PairFP32, 2, 16, 2, 1024, 4, 1, 1, 1),
    NB_KERNEL_ENTRY3(PairFP32, 2, 16, 2, 1024, 4, 1, 2, 1),
    NB_KERNEL_ENTRY3(PairFP32, 2, 16, 2, 1024, 4, 1, 3, 1),
    NB_KERNEL_ENTRY3(PairFP32, 2, 16, 2, 2048, 2, 1, 0, 1),
    NB_KERNEL_ENTRY3(PairFP32, 2, 16, 2, 512, 4, 1, 0, 1),
    NB_KERNEL_ENTRY3(PairFP32, 2, 16, 2, 512, 4, 2, 0, 1),
    NB_KERNEL_ENTRY3(PairFP32, 2, 8, 4, 512, 4, 1, 0, 1),
    NB_KERNEL_ENTRY_CL(PairFP32, 2, 8, 2, 1024, 0),   // cluster kernel for small calls
    NB_KERNEL_ENTRY(FormFP32, 2, 8, 4, 512, 0),
    NB_KERNEL_ENTRY(FormFP32, 2, 8, 8, 512, 0),
    NB_KERNEL_ENTRY(FormFP32, 2, 8, 2, 512, 0),
    // per-particle layout with the velocity criterion and/or the potential: the
    // fallback for a j-range that starts at an odd slot
    NB_KERNEL_ENTRY(FormFP32, 2, 8, 2, 512, 1),
    NB_KERNEL_ENTRY(FormFP32, 2, 8, 2, 512, 2),
    NB_KERNEL_ENTRY(FormFP32, 2, 8, 2, 512, 3),
};

const KernelEntry *kernels_fp32(int *count)
{
    *count = static_cast<int>(sizeof(g_fp32) / sizeof(g_fp32[0]));
    return g_fp32;
}

}  // namespace nb
