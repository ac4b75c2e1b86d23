// Compiled configurations of the FP64 (NB_FP64) regular-force kernel.
#include "nb_kernels.cuh"

namespace nb {

static const KernelEntry g_fp64[] = {
    NB_KERNEL_ENTRY(FormFP64, 0, 8, 2, 256, 0),
    NB_KERNEL_ENTRY(FormFP64, 0, 8, 2, 256, 1),
    NB_KERNEL_ENTRY(FormFP64, 0, 8, 2, 256, 2),
    NB_KERNEL_ENTRY(FormFP64, 0, 8, 2, 256, 3),
    NB_KERNEL_ENTRY(FormFP64, 0, 8, 4, 256, 0),
};

const KernelEntry *kernels_fp64(int *count)
{
    *count = static_cast<int>(sizeof(g_fp64) / sizeof(g_fp64[0]));
    return g_fp64;
}

}  // namespace nb
