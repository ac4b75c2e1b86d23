// Irregular force and jerk over the neighbour lists (Sec. 3.3 step (iv),
// Sec. 3.5): for each active particle i, the Newtonian force
//   F_i = sum_{j in L_i} m_j R / |R|^3,  J_i = sum_{j in L_i} m_j (V / |R|^3 - 3 (R.V) R / |R|^5)
// (and optionally the potential sum m_j / |R|) over the entries of its list,
// R = x_j - x_i, V = v_j - v_i, from the context's predicted j-set.  The paper
// evaluates this sum on the host with SSE/AVX; here it is one warp per active
// particle, lanes over the list entries, FP64 accumulation and a warp
// reduction.  The work is a gather of ~100 scattered j per i: bound by L2 / HBM
// access, not by arithmetic.
//
// Forms: FP64 throughout; two-float coordinates and mass (Sec. 3.5 keeps
// two-float coordinates for this sum, since close pairs live here) with the
// pair terms in float-float arithmetic (unevaluated sums of two FP32 values,
// about 46 significant bits) on the FP32 pipe: the irregular sum of a few
// neighbours cancels (an FP32 mass alone cost ~6e-7 with Kroupa masses, FP32
// terms ~1e-6 at 1e-5 separations 1e3 from the origin), and on GB300 a
// float-float term of ~350 FP32 operations costs a fraction of the ~40 FP64
// operations of an FP64 term (the FP64 pipe runs at 1/64 of the FP32 rate);
// plain FP32 differences and terms.
#include <cfloat>

#include "nb_irr.cuh"

namespace nb {

namespace {

struct IrrTerm {
    double f[3], j[3], p;
};

__device__ __forceinline__ void add_term(IrrTerm &a, double m, double rinv, const double dx[3], const double dv[3])
{
    const double rinv2 = rinv * rinv;
    const double mr = m * rinv;
    const double mr3 = mr * rinv2;
    const double al = 3.0 * (dx[0] * dv[0] + dx[1] * dv[1] + dx[2] * dv[2]) * rinv2;
    for (int c = 0; c < 3; c++) {
        a.f[c] += mr3 * dx[c];
        a.j[c] += mr3 * (dv[c] - al * dx[c]);
    }
    a.p += mr;
}

__device__ __forceinline__ void add_term_f(IrrTerm &a, float m, const float dx[3], const float dv[3])
{
    const float r2 = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
    const float rinv = rsqrtf(r2);
    const float rinv2 = rinv * rinv;
    const float mr = m * rinv;
    const float mr3 = mr * rinv2;
    const float al = 3.f * (dx[0] * dv[0] + dx[1] * dv[1] + dx[2] * dv[2]) * rinv2;
    for (int c = 0; c < 3; c++) {
        a.f[c] += static_cast<double>(mr3 * dx[c]);
        a.j[c] += static_cast<double>(mr3 * (dv[c] - al * dx[c]));
    }
    a.p += static_cast<double>(mr);
}

// ------------------------------------------------------------- float-float
// A value h + l held as two FP32 numbers with |l| <= ulp(h)/2 after
// normalisation.  The error-free transformations are the published ones:
// Knuth's TwoSum, Dekker's FastTwoSum and the FMA form of the exact product
// (the product's rounding error is fma(a, b, -p)).
struct FF {
    float h, l;
};

__device__ __forceinline__ FF two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp))};
}
__device__ __forceinline__ FF fast_two_sum(float a, float b)   // |a| >= |b| (or a = 0)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ FF two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ FF ffadd(FF a, FF b)
{
    FF s = two_sum(a.h, b.h);
    return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ FF ffmul(FF a, FF b)
{
    FF p = two_prod(a.h, b.h);
    return fast_two_sum(p.h, __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l)));
}
__device__ __forceinline__ FF ffmul_f(FF a, float b)
{
    FF p = two_prod(a.h, b);
    return fast_two_sum(p.h, __fmaf_rn(a.l, b, p.l));
}
// (ah + al) - (bh + bl) of two two-float numbers, normalised.
__device__ __forceinline__ FF ffdiff2(float ah, float al, float bh, float bl)
{
    FF s = two_sum(ah, -bh);
    return fast_two_sum(s.h, __fadd_rn(s.l, __fsub_rn(al, bl)));
}
// 1/sqrt(x): the FP32 reciprocal square root y refined by one Newton step
// evaluated in float-float, y + y (1 - x y^2) / 2 (1 - q.h is exact for
// q = x y^2 near 1, so the correction carries the residual's full precision).
__device__ __forceinline__ FF ffrsqrt(FF x)
{
    const float y = rsqrtf(x.h);
    const FF q = ffmul(x, two_prod(y, y));
    const float d = __fsub_rn(__fsub_rn(1.0f, q.h), q.l);
    return fast_two_sum(y, __fmul_rn(__fmul_rn(y, d), 0.5f));
}

// Irregular sum of the two-float form, float-float pair terms and sums.
template <bool POT>
__global__ void __launch_bounds__(256) irr_ff_kernel(const IrrParams p)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    const float4 *xh = reinterpret_cast<const float4 *>(p.js.s[0]);
    const float4 *xl = reinterpret_cast<const float4 *>(p.js.s[1]);
    const float4 *vh = reinterpret_cast<const float4 *>(p.js.s[2]);
    const float4 *vl = reinterpret_cast<const float4 *>(p.js.s[3]);
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); i < p.n_act;
         i += warps) {
        const int a = p.act[i];
        const int nn = p.nnb[i];
        if (a < 0 || a >= p.n_j || nn < 0) {
            if (lane == 0) atomicOr(p.status, DEV_BAD_INPUT);
            continue;
        }
        const int k = min(nn, p.cap);
        const int64_t si = p.j_begin + a;
        const int32_t *row = p.list + i * static_cast<int64_t>(p.cap);
        const float4 ih = xh[si], il = xl[si], jh = vh[si], jl = vl[si];
        FF acc[8];
        for (int c = 0; c < 8; c++) acc[c] = FF{0.f, 0.f};
        for (int e = lane; e < k; e += 32) {
            const int j = row[e];
            if (j < 0 || j >= p.n_j || j == a) { atomicOr(p.status, DEV_BAD_INPUT); continue; }
            const int64_t sj = p.j_begin + j;
            const float4 ah = xh[sj], al = xl[sj], bh = vh[sj], bl = vl[sj];
            const FF dx[3] = {ffdiff2(ah.x, al.x, ih.x, il.x), ffdiff2(ah.y, al.y, ih.y, il.y),
                              ffdiff2(ah.z, al.z, ih.z, il.z)};
            const FF dv[3] = {ffdiff2(bh.x, bl.x, jh.x, jl.x), ffdiff2(bh.y, bl.y, jh.y, jl.y),
                              ffdiff2(bh.z, bl.z, jh.z, jl.z)};
            const FF r2 = ffadd(ffadd(ffmul(dx[0], dx[0]), ffmul(dx[1], dx[1])), ffmul(dx[2], dx[2]));
            const FF rinv = ffrsqrt(r2);
            const FF rinv2 = ffmul(rinv, rinv);
            const FF mr = ffmul(FF{ah.w, al.w}, rinv);   // two-float mass
            const FF mr3 = ffmul(mr, rinv2);
            const FF rv = ffadd(ffadd(ffmul(dx[0], dv[0]), ffmul(dx[1], dv[1])), ffmul(dx[2], dv[2]));
            const FF alpha = ffmul_f(ffmul(rv, rinv2), -3.0f);
#pragma unroll
            for (int c = 0; c < 3; c++) {
                acc[c] = ffadd(acc[c], ffmul(mr3, dx[c]));
                acc[3 + c] = ffadd(acc[3 + c], ffmul(mr3, ffadd(dv[c], ffmul(alpha, dx[c]))));
            }
            if (POT) acc[6] = ffadd(acc[6], mr);
        }
        // Reduce-scatter of the eight float-float slots over the lanes (as in
        // the FP64 form): lane L ends with slot 4 b4 + 2 b3 + b2 of its lane
        // bits summed over all lanes, in 9 float-float additions per lane.
        FF k4[4], k2[2];
        {
            const bool lo = (lane & 16) == 0;
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const FF send = lo ? acc[c + 4] : acc[c];
                const FF got{__shfl_xor_sync(0xffffffffu, send.h, 16), __shfl_xor_sync(0xffffffffu, send.l, 16)};
                k4[c] = ffadd(lo ? acc[c] : acc[c + 4], got);
            }
        }
        {
            const bool lo = (lane & 8) == 0;
#pragma unroll
            for (int c = 0; c < 2; c++) {
                const FF send = lo ? k4[c + 2] : k4[c];
                const FF got{__shfl_xor_sync(0xffffffffu, send.h, 8), __shfl_xor_sync(0xffffffffu, send.l, 8)};
                k2[c] = ffadd(lo ? k4[c] : k4[c + 2], got);
            }
        }
        FF k1;
        {
            const bool lo = (lane & 4) == 0;
            const FF send = lo ? k2[1] : k2[0];
            const FF got{__shfl_xor_sync(0xffffffffu, send.h, 4), __shfl_xor_sync(0xffffffffu, send.l, 4)};
            k1 = ffadd(lo ? k2[0] : k2[1], got);
        }
        for (int o = 2; o > 0; o >>= 1)
            k1 = ffadd(k1, FF{__shfl_xor_sync(0xffffffffu, k1.h, o), __shfl_xor_sync(0xffffffffu, k1.l, o)});
        const int comp = 4 * ((lane >> 4) & 1) + 2 * ((lane >> 3) & 1) + ((lane >> 2) & 1);
        if ((lane & 3) == 0) {
            const double val = static_cast<double>(k1.h) + static_cast<double>(k1.l);
            if (comp < 3) p.F[3 * i + comp] = val;
            else if (comp < 6) p.J[3 * i + comp - 3] = val;
            else if (POT && comp == 6) p.pot[i] = val;
        }
    }
}

template <int MODE, bool POT>
__global__ void __launch_bounds__(256) irr_kernel(const IrrParams p)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); i < p.n_act;
         i += warps) {
        const int a = p.act[i];
        const int nn = p.nnb[i];
        if (a < 0 || a >= p.n_j || nn < 0) {
            if (lane == 0) atomicOr(p.status, DEV_BAD_INPUT);
            continue;
        }
        const int k = min(nn, p.cap);
        const int64_t si = p.j_begin + a;
        const int32_t *row = p.list + i * static_cast<int64_t>(p.cap);
        IrrTerm t{};
        if (MODE == 0) {   // FP64
            const double4_32a xi = reinterpret_cast<const double4_32a *>(p.js.s[0])[si];
            const double4_32a vi = reinterpret_cast<const double4_32a *>(p.js.s[1])[si];
            for (int e = lane; e < k; e += 32) {
                const int j = row[e];
                if (j < 0 || j >= p.n_j || j == a) { atomicOr(p.status, DEV_BAD_INPUT); continue; }
                const double4_32a xj = reinterpret_cast<const double4_32a *>(p.js.s[0])[p.j_begin + j];
                const double4_32a vj = reinterpret_cast<const double4_32a *>(p.js.s[1])[p.j_begin + j];
                const double dx[3] = {xj.x - xi.x, xj.y - xi.y, xj.z - xi.z};
                const double dv[3] = {vj.x - vi.x, vj.y - vi.y, vj.z - vi.z};
                const double r2 = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
                add_term(t, xj.w, rsqrt(r2), dx, dv);
            }
        } else {   // FP32
            const float4 *x = reinterpret_cast<const float4 *>(p.js.s[0]);
            const float4 *v = reinterpret_cast<const float4 *>(p.js.s[1]);
            const float4 xi = x[si], vi = v[si];
            for (int e = lane; e < k; e += 32) {
                const int j = row[e];
                if (j < 0 || j >= p.n_j || j == a) { atomicOr(p.status, DEV_BAD_INPUT); continue; }
                const int64_t sj = p.j_begin + j;
                const float4 xj = x[sj], vj = v[sj];
                const float dx[3] = {xj.x - xi.x, xj.y - xi.y, xj.z - xi.z};
                const float dv[3] = {vj.x - vi.x, vj.y - vi.y, vj.z - vi.z};
                add_term_f(t, xj.w, dx, dv);
            }
        }
        // Reduce-scatter over the lanes: at each of the first three levels a lane
        // keeps half of the components it still holds and adds its partner's copy
        // of them, so lane L ends with component 4 b4 + 2 b3 + b2 of its lane bits;
        // two more levels sum that component over the remaining lanes.  That is 9
        // FP64 additions per lane instead of 35 (GB300's FP64 pipe is narrow).
        const double c8[8] = {t.f[0], t.f[1], t.f[2], t.j[0], t.j[1], t.j[2], POT ? t.p : 0.0, 0.0};
        double k4[4], k2[2];
        {
            const bool lo = (lane & 16) == 0;
#pragma unroll
            for (int c = 0; c < 4; c++)
                k4[c] = (lo ? c8[c] : c8[c + 4]) + __shfl_xor_sync(0xffffffffu, lo ? c8[c + 4] : c8[c], 16);
        }
        {
            const bool lo = (lane & 8) == 0;
#pragma unroll
            for (int c = 0; c < 2; c++)
                k2[c] = (lo ? k4[c] : k4[c + 2]) + __shfl_xor_sync(0xffffffffu, lo ? k4[c + 2] : k4[c], 8);
        }
        const bool lo4 = (lane & 4) == 0;
        double k1 = (lo4 ? k2[0] : k2[1]) + __shfl_xor_sync(0xffffffffu, lo4 ? k2[1] : k2[0], 4);
        k1 += __shfl_xor_sync(0xffffffffu, k1, 2);
        k1 += __shfl_xor_sync(0xffffffffu, k1, 1);
        const int comp = 4 * ((lane >> 4) & 1) + 2 * ((lane >> 3) & 1) + ((lane >> 2) & 1);
        if ((lane & 3) == 0) {
            if (comp < 3) p.F[3 * i + comp] = k1;
            else if (comp < 6) p.J[3 * i + comp - 3] = k1;
            else if (POT && comp == 6) p.pot[i] = k1;
        }
    }
}

template <int MODE>
cudaError_t launch_mode(const IrrParams &p, int grid, cudaStream_t st)
{
    if (p.pot) irr_kernel<MODE, true><<<grid, 256, 0, st>>>(p);
    else irr_kernel<MODE, false><<<grid, 256, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_irregular(const IrrParams &p, int mode, int sm_count, cudaStream_t st)
{
    if (p.n_act <= 0) return cudaSuccess;
    const int64_t want = (static_cast<int64_t>(p.n_act) + 7) / 8;   // 8 warps (active particles) per block
    const int grid = static_cast<int>(std::min<int64_t>(want, static_cast<int64_t>(sm_count) * 8));
    if (mode == 0) return launch_mode<0>(p, grid, st);
    if (mode == 1) {
        if (p.pot) irr_ff_kernel<true><<<grid, 256, 0, st>>>(p);
        else irr_ff_kernel<false><<<grid, 256, 0, st>>>(p);
        return cudaGetLastError();
    }
    return launch_mode<2>(p, grid, st);
}

}  // namespace nb
