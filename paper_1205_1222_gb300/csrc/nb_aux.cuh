// Host-visible declarations of the predictor / merge kernels and of the
// regular-force kernel registry.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "nb_device.cuh"

namespace nb {

struct PredParams {
    int64_t offset, n;
    const double *x0, *v0, *a0, *adot0, *m, *t0;   // a0 == nullptr: copy x0, v0 unchanged
    double t;
    int forms;
    // Frame velocity u of the float forms (their velocities are stored as
    // v - u): keep_frame != 0 reads it from frame; otherwise every block
    // computes the same u from a sample of this call's start velocities and
    // block 0 stores it to frame.
    int keep_frame;
    double *frame;     // [3], context-owned device memory
    double4_32a *pos64, *vel64;
    float4 *mx_hi, *mx_lo, *mv_hi, *mv_lo;
    float4 *pos32, *vel32;
    float4 *pim[7];    // pair-interleaved two-float streams (j-pair P = slot / 2)
    float4 *pif[4];    // pair-interleaved FP32 streams
};

// Needed-only prediction: the slots an irregular-force call reads (the
// active particles and the first min(nnb, cap) entries of their lists), in
// the context's current frame (pp.keep_frame = 1).  A slot named several
// times is predicted by each thread that names it, with the same result.
struct NeededParams {
    PredParams pp;                 // the range [pp.offset, pp.offset + pp.n) and its arrays
    int32_t n_act, cap;
    const int32_t *act, *nnb, *list;
    int *status;                   // DEV_BAD_INPUT on an index outside the range or a negative count
};

struct MergeParams {
    ClusterDesc d0;                // single cluster (table == nullptr)
    const ClusterDesc *table;      // cluster table of a batched plan
    const int64_t *act_begin;      // [n_clusters] prefix of n_act over the merged clusters
    const int32_t *cluster_of;     // [n_clusters] index into table of each merged cluster
    int32_t n_clusters;            // merged clusters
    int64_t n_total;               // total merged active particles (one warp each)
    int ff;                        // 1: split slots hold float-float pairs (float forms), 0: doubles (FP64 form)
    int *status;                   // device status word (DEV_BOUNDS if a list read would leave its row)
};

void launch_predict(const PredParams &p, cudaStream_t st);
void launch_predict_needed(const NeededParams &p, cudaStream_t st);
void launch_merge(const MergeParams &p, cudaStream_t st);

// One compiled instantiation of the regular-force kernel.
struct KernelEntry {
    int mode;        // 0 FP64, 1 MIXED, 2 FP32
    int warps, ipw, jtile;
    int flags;       // bit 0: velocity criterion, bit 1: potential
    int packed;      // 20: thread-block-cluster kernel for small calls (nb_regf_cl.cuh);
                     // 0: scalar kernel (nb_regf.cuh),
                     // 2: f32x2 over j-pairs on the pair-interleaved streams (nb_regf3.cuh),
                     // 3: as 2 with two j-pairs per lane per step; 4: framed; 5: two-float
                     // positions with FP32 velocity differences; 5 + NL / 10 + NL: the
                     // arithmetic of 5 / 2 with NL list warps (nb_regf_ws.cuh)
    const void *fn;
    int smem;        // dynamic shared memory bytes
    int lists = 0;   // list warps of the CTA (they own no active particles)
};

const KernelEntry *kernels_fp64(int *count);
const KernelEntry *kernels_mixed(int *count);
const KernelEntry *kernels_fp32(int *count);

}  // namespace nb
