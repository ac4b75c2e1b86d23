// Irregular force over neighbour lists (Sec. 3.3 step (iv)): launch interface.
#pragma once

#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

#include "nb_device.cuh"

namespace nb {

struct IrrParams {
    int64_t j_begin;      // first slot of the j-range in the predicted set
    int32_t n_j;          // j-particles of the range (list entries index it)
    int32_t n_act;        // active particles
    int32_t cap;          // list row length
    const int32_t *act;   // [n_act] index of each active particle in the j-range
    const int32_t *nnb;   // [n_act] neighbour counts; min(nnb, cap) entries are summed
    const int32_t *list;  // [n_act][cap] neighbour indices in the j-range
    JSet js;              // FP64: pos, vel; two-float: x hi, x lo, v hi, v lo; FP32: pos, vel
    double *F, *J, *pot;  // [n_act][3], [n_act][3], [n_act] or nullptr
    int *status;          // device status word (DEV_BAD_INPUT on an invalid index or count)
};

cudaError_t launch_irregular(const IrrParams &p, int mode, int sm_count, cudaStream_t st);

}  // namespace nb
