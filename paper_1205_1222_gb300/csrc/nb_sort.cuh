// Spatial ordering of the active set and per-block frames (nb_sort.cu).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace nb {

constexpr int SORT_DIGIT_BITS = 10;            // radix of the key sort (three passes over 30-bit keys)
constexpr int SORT_BINS = 1 << SORT_DIGIT_BITS;
constexpr int SORT_CHUNK = 1024;               // keys per warp in the histogram and scatter passes
// Largest |c - x_i| / h_i a block may have for its frame to be used.  With
// u = 2^-24, A = x_j - c and B = c - x_i each formed in two-float and rounded
// once err by at most 2u|A| and 2u|B|, and their FP32 sum adds u|dx|; since
// |A| <= |dx| + |B|, dx errs by at most 3u|dx| + 4u|B|.  At |dx| ~ h_i,
// r^2 (three fused multiply-adds) then errs by at most 9u + 8u beta relative,
// plus u for h^2 in FP32: for beta = 2.5 that is 1.8e-6, inside the 2e-6
// margin on r^2 that the inputs keep (1e-6 on the radius), so neighbour
// decisions agree with the exact two-float ones.
constexpr double FRAME_BETA = 2.5;

struct SortParams {
    int n_act, n_j;
    int64_t j_begin;
    const int32_t *act;
    const double *h;
    const float4 *pos_hi, *pos_lo, *vel_hi, *vel_lo;   // two-float per-particle streams
};

// Frame of one block of sorted active particles.
struct FrameRec {
    double cx[3], cv[3];   // centroid of positions and velocities
    int compact;           // 1 when max |c - x_i| / h_i <= FRAME_BETA
    int pad;
};

struct SortBuffers {
    unsigned *bbox;        // 6 ordered-float words
    int *n_compact;        // count of compact blocks of the last sort
    unsigned *k0, *k1;
    int *v0, *v1;
    int *ghist;
    FrameRec *frames;
};

size_t sort_scratch_bytes(int n_act, int n_blocks);
SortBuffers carve_sort(void *base, int n_act, int n_blocks);
const int *launch_sort_and_frames(const SortParams &p, const SortBuffers &s, int per_block, int n_blocks,
                                  cudaStream_t st);

}  // namespace nb
