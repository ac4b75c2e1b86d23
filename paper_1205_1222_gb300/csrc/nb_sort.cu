// Spatial ordering of the active set and the per-block frames of the framed
// two-float kernel.
//
// The framed kernel evaluates the two-float difference x_j - x_i as
// (x_j - c) + (c - x_i) with both parts rounded to FP32, c being a frame
// centre shared by the CTA's block of active particles.  That is as exact as
// the per-pair two-float difference only when every x_i of the block lies
// close to c on the scale of its neighbour radius, so the active particles are
// first ordered along a Morton curve (30-bit keys of their positions in the
// bounding box of the active set, LSD radix sort with 10-bit digits, stable),
// and each block of consecutive sorted particles gets a frame record: the
// centroid of its positions and velocities (FP64) and a flag telling whether
// max |c - x_i| / h_i stays within FRAME_BETA.  Blocks that fail the test are
// computed by the exact two-float path.
#include <cfloat>
#include <cstdint>
#include <utility>

#include "nb_sort.cuh"

namespace nb {

namespace {

__device__ __forceinline__ unsigned ordered_bits(float f)   // monotone float -> uint
{
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float from_ordered(unsigned u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}
__device__ __forceinline__ unsigned spread10(unsigned v)   // 10 bits -> every third bit
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__global__ void bbox_init_kernel(unsigned *bb)
{
    if (threadIdx.x < 3) { bb[threadIdx.x] = 0xffffffffu; bb[3 + threadIdx.x] = 0u; }
}

// Bounding box of the active positions (hi parts of the two-float form).
__global__ void bbox_kernel(const SortParams p, unsigned *bb)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned mn[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, mx[3] = {0u, 0u, 0u};
    if (k < p.n_act) {
        const int a = p.act[k];
        if (a >= 0 && a < p.n_j) {
            const float4 x = p.pos_hi[p.j_begin + a];
            const unsigned v[3] = {ordered_bits(x.x), ordered_bits(x.y), ordered_bits(x.z)};
            for (int c = 0; c < 3; c++) { mn[c] = v[c]; mx[c] = v[c]; }
        }
    }
    for (int c = 0; c < 3; c++) {
        for (int o = 16; o > 0; o >>= 1) {
            mn[c] = min(mn[c], __shfl_xor_sync(0xffffffffu, mn[c], o));
            mx[c] = max(mx[c], __shfl_xor_sync(0xffffffffu, mx[c], o));
        }
    }
    if ((threadIdx.x & 31) == 0)
        for (int c = 0; c < 3; c++) { atomicMin(&bb[c], mn[c]); atomicMax(&bb[3 + c], mx[c]); }
}

__global__ void keys_kernel(const SortParams p, const unsigned *bb, unsigned *keys, int *vals)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= p.n_act) return;
    unsigned key = 0x3fffffffu;   // invalid entries sort last
    const int a = p.act[k];
    if (a >= 0 && a < p.n_j) {
        const float4 x = p.pos_hi[p.j_begin + a];
        const float xs[3] = {x.x, x.y, x.z};
        unsigned q[3];
        for (int c = 0; c < 3; c++) {
            const float lo = from_ordered(bb[c]), hi = from_ordered(bb[3 + c]);
            const float span = hi - lo;
            const float t = span > 0.f ? (xs[c] - lo) / span : 0.f;
            q[c] = static_cast<unsigned>(fminf(fmaxf(t * 1024.f, 0.f), 1023.f));
        }
        key = spread10(q[0]) | (spread10(q[1]) << 1) | (spread10(q[2]) << 2);
    }
    keys[k] = key;
    vals[k] = k;
}

// One warp per chunk of SORT_CHUNK keys: digit histogram of the chunk.
__global__ void hist_kernel(const unsigned *keys, int n, int shift, int nchunk, int *ghist)
{
    __shared__ int h[SORT_BINS];
    const int lane = threadIdx.x, chunk = blockIdx.x;
    for (int b = lane; b < SORT_BINS; b += 32) h[b] = 0;
    __syncwarp();
    for (int r = 0; r < SORT_CHUNK; r += 32) {
        const int k = chunk * SORT_CHUNK + r + lane;
        if (k < n) atomicAdd(&h[(keys[k] >> shift) & (SORT_BINS - 1)], 1);
    }
    __syncwarp();
    for (int b = lane; b < SORT_BINS; b += 32) ghist[b * nchunk + chunk] = h[b];
}

// Exclusive scan of the digit-major histogram (one block).
__global__ void scan_kernel(int *ghist, int total)
{
    __shared__ int part[1024];
    const int t = threadIdx.x;
    const int per = (total + blockDim.x - 1) / blockDim.x;
    const int b0 = min(total, t * per), b1 = min(total, b0 + per);
    int s = 0;
    for (int i = b0; i < b1; i++) s += ghist[i];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < blockDim.x; o <<= 1) {
        const int v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = part[t] - s;
    for (int i = b0; i < b1; i++) {
        const int c = ghist[i];
        ghist[i] = run;
        run += c;
    }
}

// Stable scatter of one chunk: keys are ranked round by round (32 at a time,
// in order) with a match over equal digits.
__global__ void scatter_kernel(const unsigned *kin, const int *vin, unsigned *kout, int *vout, int n, int shift,
                               int nchunk, const int *goff)
{
    __shared__ int cnt[SORT_BINS];
    const int lane = threadIdx.x, chunk = blockIdx.x;
    for (int b = lane; b < SORT_BINS; b += 32) cnt[b] = 0;
    __syncwarp();
    for (int r = 0; r < SORT_CHUNK; r += 32) {
        const int k = chunk * SORT_CHUNK + r + lane;
        const bool ok = k < n;
        const unsigned key = ok ? kin[k] : 0u;
        const int d = ok ? static_cast<int>((key >> shift) & (SORT_BINS - 1)) : SORT_BINS;
        const unsigned same = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(same & ((1u << lane) - 1u));
        if (ok) {
            const int pos = goff[d * nchunk + chunk] + cnt[d] + rank;
            kout[pos] = key;
            vout[pos] = vin[k];
        }
        __syncwarp();
        if (ok && rank == 0) cnt[d] += __popc(same);
        __syncwarp();
    }
}

// One warp per block of `per_block` consecutive sorted active particles:
// centroid of positions and velocities, and the compactness flag.
__global__ void frame_kernel(const SortParams p, const int *perm, int per_block, int n_blocks, FrameRec *frames,
                             int *n_compact)
{
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n_blocks) return;
    double x[3] = {0, 0, 0}, v[3] = {0, 0, 0};
    int count = 0;
    bool bad = false;
    for (int s = lane; s < per_block; s += 32) {
        const int slot = w * per_block + s;
        if (slot >= p.n_act) continue;
        const int k = perm[slot];
        const int a = p.act[k];
        const double h = p.h[k];
        if (a < 0 || a >= p.n_j || !(h >= 0.0) || h > DBL_MAX) { bad = true; continue; }
        const float4 xh = p.pos_hi[p.j_begin + a], xl = p.pos_lo[p.j_begin + a];
        const float4 vh = p.vel_hi[p.j_begin + a], vl = p.vel_lo[p.j_begin + a];
        x[0] += static_cast<double>(xh.x) + xl.x; x[1] += static_cast<double>(xh.y) + xl.y;
        x[2] += static_cast<double>(xh.z) + xl.z;
        v[0] += static_cast<double>(vh.x) + vl.x; v[1] += static_cast<double>(vh.y) + vl.y;
        v[2] += static_cast<double>(vh.z) + vl.z;
        count++;
    }
    for (int o = 16; o > 0; o >>= 1) {
        for (int c = 0; c < 3; c++) {
            x[c] += __shfl_xor_sync(0xffffffffu, x[c], o);
            v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
        }
        count += __shfl_xor_sync(0xffffffffu, count, o);
    }
    bad = __any_sync(0xffffffffu, bad);
    FrameRec f{};
    for (int c = 0; c < 3; c++) {
        f.cx[c] = count ? x[c] / count : 0.0;
        f.cv[c] = count ? v[c] / count : 0.0;
    }
    double worst = 0.0;   // max |c - x_i| / h_i over the block
    for (int s = lane; s < per_block; s += 32) {
        const int slot = w * per_block + s;
        if (slot >= p.n_act) continue;
        const int k = perm[slot];
        const int a = p.act[k];
        const double h = p.h[k];
        if (a < 0 || a >= p.n_j || !(h >= 0.0) || h > DBL_MAX) continue;
        const float4 xh = p.pos_hi[p.j_begin + a], xl = p.pos_lo[p.j_begin + a];
        const double d0 = static_cast<double>(xh.x) + xl.x - f.cx[0];
        const double d1 = static_cast<double>(xh.y) + xl.y - f.cx[1];
        const double d2 = static_cast<double>(xh.z) + xl.z - f.cx[2];
        const double dist = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        worst = fmax(worst, h > 0.0 ? dist / h : (dist > 0.0 ? DBL_MAX : 0.0));
    }
    for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
    f.compact = (!bad && count > 0 && worst <= FRAME_BETA) ? 1 : 0;
    if (lane == 0) {
        frames[w] = f;
        if (f.compact) atomicAdd(n_compact, 1);
    }
}

}  // namespace

size_t sort_scratch_bytes(int n_act, int n_blocks)
{
    const size_t n = static_cast<size_t>(n_act);
    const size_t nchunk = (n + SORT_CHUNK - 1) / SORT_CHUNK;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    return al(64) + 4 * al(n * 4) + al(nchunk * SORT_BINS * 4) + al(static_cast<size_t>(n_blocks) * sizeof(FrameRec));
}

SortBuffers carve_sort(void *base, int n_act, int n_blocks)
{
    const size_t n = static_cast<size_t>(n_act);
    const size_t nchunk = (n + SORT_CHUNK - 1) / SORT_CHUNK;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    char *p = static_cast<char *>(base);
    SortBuffers s;
    s.bbox = reinterpret_cast<unsigned *>(p); p += al(64);
    s.n_compact = reinterpret_cast<int *>(s.bbox + 8);
    s.k0 = reinterpret_cast<unsigned *>(p); p += al(n * 4);
    s.k1 = reinterpret_cast<unsigned *>(p); p += al(n * 4);
    s.v0 = reinterpret_cast<int *>(p); p += al(n * 4);
    s.v1 = reinterpret_cast<int *>(p); p += al(n * 4);
    s.ghist = reinterpret_cast<int *>(p); p += al(nchunk * SORT_BINS * 4);
    s.frames = reinterpret_cast<FrameRec *>(p);
    return s;
}

// Sort the active set and build the frames.  Leaves the permutation (sorted
// slot -> position in act) in the returned pointer.  9 launches.
const int *launch_sort_and_frames(const SortParams &p, const SortBuffers &s, int per_block, int n_blocks,
                                  cudaStream_t st)
{
    const int n = p.n_act;
    const int threads = 256;
    const int blocks = (n + threads - 1) / threads;
    const int nchunk = (n + SORT_CHUNK - 1) / SORT_CHUNK;
    bbox_init_kernel<<<1, 32, 0, st>>>(s.bbox);
    bbox_kernel<<<blocks, threads, 0, st>>>(p, s.bbox);
    keys_kernel<<<blocks, threads, 0, st>>>(p, s.bbox, s.k0, s.v0);
    unsigned *kin = s.k0, *kout = s.k1;
    int *vin = s.v0, *vout = s.v1;
    for (int shift = 0; shift < 30; shift += SORT_DIGIT_BITS) {
        hist_kernel<<<nchunk, 32, 0, st>>>(kin, n, shift, nchunk, s.ghist);
        scan_kernel<<<1, 1024, 0, st>>>(s.ghist, nchunk * SORT_BINS);
        scatter_kernel<<<nchunk, 32, 0, st>>>(kin, vin, kout, vout, n, shift, nchunk, s.ghist);
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    cudaMemsetAsync(s.n_compact, 0, sizeof(int), st);
    const int fthreads = 256;
    const int fblocks = (n_blocks * 32 + fthreads - 1) / fthreads;
    frame_kernel<<<fblocks, fthreads, 0, st>>>(p, vin, per_block, n_blocks, s.frames, s.n_compact);
    return vin;
}

}  // namespace nb
