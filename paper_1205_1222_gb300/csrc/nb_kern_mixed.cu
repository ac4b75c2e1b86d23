// Compiled configurations of the two-float (NB_MIXED) regular-force kernel:
// packed f32x2 i-pair kernels and the scalar kernel.  The first entry of each
// flag value is the default; all flag-0 entries form the autotuner's search
// space.
#include "nb_kernels.cuh"

namespace nb {

static const KernelEntry g_mixed[] = {
    NB_KERNEL_ENTRY3(PairMixed, 1, 16, 2, 512, 0, 1),
    NB_KERNEL_ENTRY3(PairMixed, 1, 12, 2, 512, 1, 1),
    NB_KERNEL_ENTRY3(PairMixed, 1, 12, 2, 512, 2, 1),
    NB_KERNEL_ENTRY3(PairMixed, 1, 12, 2, 512, 3, 1),
    NB_KERNEL_ENTRY3(PairMixed, 1, 12, 2, 512, 0, 1),
    NB_KERNEL_ENTRY3(PairMixed, 1, 8, 2, 512, 0, 1),
    NB_KERNEL_ENTRY3(PairMixed, 1, 16, 2, 256, 0, 1),
    NB_KERNEL_ENTRY2(PackedMixed, 1, 12, 4, 256, 0, 1),
    NB_KERNEL_ENTRY2(PackedMixed, 1, 12, 4, 256, 1, 1),
    NB_KERNEL_ENTRY2(PackedMixed, 1, 12, 4, 256, 2, 1),
    NB_KERNEL_ENTRY2(PackedMixed, 1, 12, 4, 256, 3, 1),
    NB_KERNEL_ENTRY2(PackedMixed, 1, 8, 4, 256, 0, 1),
    NB_KERNEL_ENTRY2(PackedMixed, 1, 16, 2, 256, 0, 1),
    NB_KERNEL_ENTRY2(PackedMixed, 1, 8, 2, 256, 0, 2),
    NB_KERNEL_ENTRY2(PackedMixed, 1, 12, 4, 512, 0, 1),
    NB_KERNEL_ENTRY2(PackedMixed, 1, 4, 4, 256, 0, 1),
    NB_KERNEL_ENTRY(FormMixed, 1, 8, 4, 512, 0),
    NB_KERNEL_ENTRY(FormMixed, 1, 4, 4, 512, 0),
    NB_KERNEL_ENTRY(FormMixed, 1, 8, 2, 512, 0),
    NB_KERNEL_ENTRY(FormMixed, 1, 16, 2, 512, 0),
    NB_KERNEL_ENTRY(FormMixed, 1, 8, 4, 256, 0),
    NB_KERNEL_ENTRY(FormMixed, 1, 8, 4, 1024, 0),
    NB_KERNEL_ENTRY(FormMixed, 1, 4, 8, 256, 0),
};

const KernelEntry *kernels_mixed(int *count)
{
    *count = static_cast<int>(sizeof(g_mixed) / sizeof(g_mixed[0]));
    return g_mixed;
}

}  // namespace nb
