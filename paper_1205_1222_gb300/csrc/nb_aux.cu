// Predictor and split-merge kernels of libnbreg.
//
//  * predict_kernel: advances every j-particle to the block time with the
//    third-order Taylor polynomial in a, da/dt (Sec. 3.3 step (iii); the
//    paper does this on the host before GPUNB_SEND) and writes the stored
//    copies the force kernels read: FP64 double4 (x,y,z,m) + (vx,vy,vz,0),
//    two-float float4 hi/lo pairs of position and velocity (mass in the
//    hi-position w), and plain FP32 float4 copies; the two float forms are
//    also written pair-interleaved (float4 k of j-pair P holds components of
//    slots 2P and 2P+1) for the j-pair packed kernels.  The float forms hold
//    velocities relative to a frame velocity u (v - u formed in FP64, then
//    rounded), so that an FP32 velocity difference v_j - v_i, which rounds
//    |v_i - u| + |v_j - u| rather than |v_i| + |v_j|, is as accurate for a
//    cluster moving through the caller's frame as for one at rest in it.  u is
//    the mean start velocity of kFrameSamples particles spread evenly over the
//    call's range (every block computes the same value, in the same order, so
//    no launch or grid-wide step is added), or the context's stored frame.
//  * predict_needed_kernel: the same prediction for only the slots that an
//    irregular-force call reads (Sec. 3.5: the host library predicts only the
//    particles it needs when they are few, the NPACT switch of Appendix C):
//    one thread per (active particle, list slot).  A slot named by several
//    threads is predicted by each of them with identical results: removing
//    the duplicates costs more dependent global-memory round trips than the
//    repeated FP64 work of the small calls this kernel is for.
//  * merge_kernel: one warp per active particle of a cluster whose j-range
//    was split over several work items; sums the per-split partial force,
//    jerk and potential in a fixed order (float-float pairs for the float
//    forms, on the FP32 pipe; FP64 for the FP64 form) and concatenates the
//    per-split partial lists in split order (ascending j), keeping the first
//    `cap` entries (Sec. 3.4: force reduction and list gathering kernels).
#include <cstdint>

#include "nb_aux.cuh"

namespace nb {

namespace {

// Write this slot's values into float4 k of its j-pair for the NQ streams:
// stream q holds (v[2q] of both slots, v[2q+1] of both slots).  The even slot
// writes whole float4s with its partner's values (a shuffle from the next
// lane); an even slot without a partner in this call, and an odd slot whose
// partner is not in this call, write their own halves only.
template <int NQ>
__device__ __forceinline__ void write_pairs(float4 *const *streams, const float (&v)[2 * NQ], int64_t s, bool live,
                                            bool even, bool partner_in)
{
    const int64_t P = s >> 1;
    const int lane = threadIdx.x & 31;
    // the odd slot of a pair whose even slot is outside the call, or in another warp
    const bool odd_alone = !even && (lane == 0);
#pragma unroll
    for (int q = 0; q < NQ; q++) {
        const float o0 = __shfl_down_sync(0xffffffffu, v[2 * q], 1);
        const float o1 = __shfl_down_sync(0xffffffffu, v[2 * q + 1], 1);
        if (!live) continue;
        if (even && partner_in) {
            streams[q][P] = make_float4(v[2 * q], o0, v[2 * q + 1], o1);
        } else if (even || odd_alone) {
            float *f = reinterpret_cast<float *>(streams[q] + P);
            const int h = even ? 0 : 1;
            f[h] = v[2 * q];
            f[2 + h] = v[2 * q + 1];
        }
    }
}

}  // namespace

// Frame velocity of this call: the plain mean of the start velocities of
// particles floor(k n / S), k = 0 .. S-1 (S = min(n, 32): lane k loads one),
// summed in FP32 over an xor butterfly of the lanes, so every lane of every
// warp gets the same bits (each addition is commutative).  Any velocity near
// the cluster's bulk motion serves; the mean of the sample is one within
// about a dispersion / 5.  The sample's loads are issued first and summed
// after the polynomial, so their latency overlaps the slot's own loads.
// All lanes of the warp must call both halves.
struct FrameSample {
    float s[3];
};

__device__ __forceinline__ FrameSample frame_sample(const PredParams &p)
{
    FrameSample f{{0.f, 0.f, 0.f}};
    if (p.keep_frame) return f;
    const int64_t S = p.n < 32 ? p.n : 32;
    const int64_t k = threadIdx.x & 31;
    if (k < S) {   // every warp reads the same 32 records: through the read-only (L1) path
        const int64_t j = k * p.n / S;
        for (int c = 0; c < 3; c++) f.s[c] = __double2float_rn(__ldg(p.v0 + 3 * j + c));
    }
    return f;
}

__device__ __forceinline__ void frame_velocity(const PredParams &p, FrameSample f, double (&u)[3])
{
    if (p.keep_frame) {
        for (int c = 0; c < 3; c++) u[c] = p.frame[c];
        return;
    }
    const int64_t S = p.n < 32 ? p.n : 32;
    for (int o = 16; o > 0; o >>= 1)
        for (int c = 0; c < 3; c++) f.s[c] += __shfl_xor_sync(0xffffffffu, f.s[c], o);
    for (int c = 0; c < 3; c++) u[c] = S > 0 ? static_cast<double>(f.s[c] / static_cast<float>(S)) : 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (int c = 0; c < 3; c++) p.frame[c] = u[c];
}

// Third-order Taylor polynomial of element j of the call's arrays (Horner
// form of x0 + v0 dt + a dt^2/2 + ad dt^3/6 and v0 + a dt + ad dt^2/2), or
// the given state itself for nb_set_predicted (a0 == nullptr).
__device__ __forceinline__ void taylor(const PredParams &p, int64_t j, double (&x)[3], double (&v)[3])
{
    if (p.a0) {
        const double dt = p.t - p.t0[j];
        for (int k = 0; k < 3; k++) {
            const double x0 = p.x0[3 * j + k], v0 = p.v0[3 * j + k];
            const double a = p.a0[3 * j + k], ad = p.adot0[3 * j + k];
            x[k] = fma(dt, fma(dt, fma(dt, ad * (1.0 / 6.0), a * 0.5), v0), x0);
            v[k] = fma(dt, fma(dt, ad * 0.5, a), v0);
        }
    } else {
        for (int k = 0; k < 3; k++) { x[k] = p.x0[3 * j + k]; v[k] = p.v0[3 * j + k]; }
    }
}

__global__ void predict_kernel(const PredParams p)
{
    const FrameSample fs = frame_sample(p);
    const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    // every lane takes part in the shuffles; lanes past the end only pass values along
    const bool live = j < p.n;
    if (!__any_sync(0xffffffffu, live)) return;
    double x[3] = {0, 0, 0}, v[3] = {0, 0, 0};
    const double m = live ? p.m[j] : 0.0;
    if (live) taylor(p, j, x, v);
    double u[3];
    frame_velocity(p, fs, u);
    const int64_t s = p.offset + j;
    if ((p.forms & 1) && live) {
        p.pos64[s] = make_double4_32a(x[0], x[1], x[2], m);
        p.vel64[s] = make_double4_32a(v[0], v[1], v[2], 0.0);
    }
    // Pair-interleaved copies: the thread of the even slot of j-pair s / 2
    // gathers its partner's values with a shuffle and writes whole float4s.
    // Slots are consecutive across the warp's lanes, and the partner of a
    // range's last slot (odd offset + n) is outside the range: that half is
    // left as it is (a later prediction of that slot fills it).
    const bool even = (s & 1) == 0;
    const bool partner_in = ((threadIdx.x & 31) + 1 < 32) && (j + 1 < p.n);
    double vr[3];   // velocity in the frame of the float forms
    for (int k = 0; k < 3; k++) vr[k] = v[k] - u[k];
    if (p.forms & 2) {
        float xh[3], xl[3], vh[3], vl[3];
        for (int k = 0; k < 3; k++) {
            xh[k] = __double2float_rn(x[k]);
            xl[k] = __double2float_rn(x[k] - static_cast<double>(xh[k]));
            vh[k] = __double2float_rn(vr[k]);
            vl[k] = __double2float_rn(vr[k] - static_cast<double>(vh[k]));
        }
        const float mh = __double2float_rn(m);
        const float ml = __double2float_rn(m - static_cast<double>(mh));
        if (live) {
            p.mx_hi[s] = make_float4(xh[0], xh[1], xh[2], mh);
            p.mx_lo[s] = make_float4(xl[0], xl[1], xl[2], ml);
            p.mv_hi[s] = make_float4(vh[0], vh[1], vh[2], 0.f);
            p.mv_lo[s] = make_float4(vl[0], vl[1], vl[2], 0.f);
        }
        const float vals[14] = {xh[0], xh[1], xh[2], mh, xl[0], xl[1], xl[2],
                                vh[0], vh[1], vh[2], vl[0], vl[1], vl[2], 0.f};
        write_pairs<7>(p.pim, vals, s, live, even, partner_in);
    }
    if (p.forms & 4) {
        const float vals[8] = {__double2float_rn(x[0]), __double2float_rn(x[1]), __double2float_rn(x[2]),
                               __double2float_rn(m), __double2float_rn(vr[0]), __double2float_rn(vr[1]),
                               __double2float_rn(vr[2]), 0.f};
        if (live) {
            p.pos32[s] = make_float4(vals[0], vals[1], vals[2], vals[3]);
            p.vel32[s] = make_float4(vals[4], vals[5], vals[6], 0.f);
        }
        write_pairs<4>(p.pif, vals, s, live, even, partner_in);
    }
}

// Store slot s's values as its halves of float4 k of j-pair s / 2 in each of
// the NQ pair-interleaved streams (stream q holds (v[2q], v[2q+1]) of both
// slots of the pair), without touching the partner slot's halves.
template <int NQ>
__device__ __forceinline__ void write_pair_halves(float4 *const *streams, const float (&v)[2 * NQ], int64_t s)
{
    const int h = static_cast<int>(s & 1);
#pragma unroll
    for (int q = 0; q < NQ; q++) {
        float *f = reinterpret_cast<float *>(streams[q] + (s >> 1));
        f[h] = v[2 * q];
        f[2 + h] = v[2 * q + 1];
    }
}

__global__ void predict_needed_kernel(const NeededParams np)
{
    const PredParams &p = np.pp;
    const int64_t per = static_cast<int64_t>(np.cap) + 1;   // the particle itself, then its list row
    const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= static_cast<int64_t>(np.n_act) * per) return;
    const int64_t k = t / per;
    const int e = static_cast<int>(t - k * per);
    int64_t j;   // index in the range
    if (e == 0) {
        j = np.act[k];
    } else {
        const int nn = np.nnb[k];
        if (nn < 0) {
            if (e == 1) atomicOr(np.status, DEV_BAD_INPUT);
            return;
        }
        if (e - 1 >= min(nn, np.cap)) return;
        j = np.list[k * np.cap + (e - 1)];
    }
    if (j < 0 || j >= p.n) { atomicOr(np.status, DEV_BAD_INPUT); return; }
    const int64_t s = p.offset + j;
    double x[3], v[3], u[3];
    taylor(p, j, x, v);
    const double m = p.m[j];
    for (int c = 0; c < 3; c++) u[c] = p.frame[c];
    double vr[3];
    for (int c = 0; c < 3; c++) vr[c] = v[c] - u[c];
    if (p.forms & 1) {
        p.pos64[s] = make_double4_32a(x[0], x[1], x[2], m);
        p.vel64[s] = make_double4_32a(v[0], v[1], v[2], 0.0);
    }
    if (p.forms & 2) {
        float xh[3], xl[3], vh[3], vl[3];
        for (int c = 0; c < 3; c++) {
            xh[c] = __double2float_rn(x[c]);
            xl[c] = __double2float_rn(x[c] - static_cast<double>(xh[c]));
            vh[c] = __double2float_rn(vr[c]);
            vl[c] = __double2float_rn(vr[c] - static_cast<double>(vh[c]));
        }
        const float mh = __double2float_rn(m);
        const float ml = __double2float_rn(m - static_cast<double>(mh));
        p.mx_hi[s] = make_float4(xh[0], xh[1], xh[2], mh);
        p.mx_lo[s] = make_float4(xl[0], xl[1], xl[2], ml);
        p.mv_hi[s] = make_float4(vh[0], vh[1], vh[2], 0.f);
        p.mv_lo[s] = make_float4(vl[0], vl[1], vl[2], 0.f);
        const float vals[14] = {xh[0], xh[1], xh[2], mh, xl[0], xl[1], xl[2],
                                vh[0], vh[1], vh[2], vl[0], vl[1], vl[2], 0.f};
        write_pair_halves<7>(p.pim, vals, s);
    }
    if (p.forms & 4) {
        const float vals[8] = {__double2float_rn(x[0]), __double2float_rn(x[1]), __double2float_rn(x[2]),
                               __double2float_rn(m), __double2float_rn(vr[0]), __double2float_rn(vr[1]),
                               __double2float_rn(vr[2]), 0.f};
        p.pos32[s] = make_float4(vals[0], vals[1], vals[2], vals[3]);
        p.vel32[s] = make_float4(vals[4], vals[5], vals[6], 0.f);
        write_pair_halves<4>(p.pif, vals, s);
    }
}


__global__ void merge_kernel(const MergeParams p)
{
    const int64_t w = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= p.n_total) return;
    ClusterDesc d;
    int64_t i;
    if (p.table) {
        int lo = 0, hi = p.n_clusters - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (p.act_begin[mid] <= w) lo = mid; else hi = mid - 1;
        }
        d = p.table[p.cluster_of[lo]];
        i = w - p.act_begin[lo];
    } else {
        d = p.d0;
        i = w;
    }
    const int S = d.n_split;
    const int64_t na = d.n_act;
    double sum[7] = {0, 0, 0, 0, 0, 0, 0};
    float sh[7] = {0, 0, 0, 0, 0, 0, 0}, sl[7] = {0, 0, 0, 0, 0, 0, 0};
    int running = 0;
    for (int s0 = 0; s0 < S; s0 += 32) {
        const int s = s0 + lane;
        int c = 0;
        if (s < S) {
            c = d.pcnt[s * na + i];
            if (p.ff) {
                const float2 *q = reinterpret_cast<const float2 *>(d.pF + (s * na + i) * 8);
                for (int k = 0; k < 7; k++) {
                    const float2 v = q[k];
                    ff_add_ff(sh[k], sl[k], v.x, v.y);
                }
            } else {
                const double *q = d.pF + (s * na + i) * 8;
                for (int k = 0; k < 7; k++) sum[k] += q[k];
            }
        }
        int incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        // Copy the chunk's entries that still fit, one entry per lane per
        // round: entry e of the chunk belongs to the last split whose
        // exclusive prefix is <= e (found by a binary search over the lanes).
        const int excl = incl - c;
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        const int ncopy = max(0, min(total, d.cap - running));
        int32_t *to = d.list + i * d.cap + running;
        for (int r = 0; r < ncopy; r += 32) {
            const int e = r + lane;
            int src = 0;
            for (int step = 16; step > 0; step >>= 1) {
                const int ex = __shfl_sync(0xffffffffu, excl, src + step);
                if (ex <= e) src += step;
            }
            const int off = e - __shfl_sync(0xffffffffu, excl, src);
            // off < min(count of split src, cap) and s0 + src < S by construction
            if (e < ncopy) {
                if (off >= 0 && off < d.cap && s0 + src < S)
                    to[e] = d.plist[(static_cast<int64_t>(s0 + src) * na + i) * d.cap + off];
                else
                    atomicOr(p.status, DEV_BOUNDS);
            }
        }
        running += total;
    }
    if (p.ff) {
        // float-float butterfly, then lane k < 7 converts component k: one FP64
        // add per lane instead of 35 on every lane (GB300's FP64 pipe is narrow)
        for (int o = 16; o > 0; o >>= 1)
            for (int k = 0; k < 7; k++) {
                const float h2 = __shfl_xor_sync(0xffffffffu, sh[k], o);
                const float l2 = __shfl_xor_sync(0xffffffffu, sl[k], o);
                ff_add_ff(sh[k], sl[k], h2, l2);
            }
        float h = 0.f, l = 0.f;
#pragma unroll
        for (int k = 0; k < 7; k++)
            if (k == lane) { h = sh[k]; l = sl[k]; }
        const double v = static_cast<double>(h) + static_cast<double>(l);
        if (lane < 3) d.F[3 * i + lane] = v;
        else if (lane < 6) d.J[3 * i + lane - 3] = v;
        else if (lane == 6 && d.pot) d.pot[i] = v;
    } else {
        for (int o = 16; o > 0; o >>= 1)
            for (int k = 0; k < 7; k++) sum[k] += __shfl_xor_sync(0xffffffffu, sum[k], o);
        if (lane == 0) {
            for (int k = 0; k < 3; k++) { d.F[3 * i + k] = sum[k]; d.J[3 * i + k] = sum[3 + k]; }
            if (d.pot) d.pot[i] = sum[6];
        }
    }
    if (lane == 0) {
        d.nnb[i] = running;
        d.ovf[i] = running > d.cap ? 1 : 0;
    }
}

void launch_predict(const PredParams &p, cudaStream_t st)
{
    if (p.n <= 0) return;
    // The polynomial and the two-float splits run on the FP64 pipe (two lanes
    // per SM per clock on this part), so a call is bound by the SMs it reaches:
    // small blocks spread a 16384-slot call over every SM instead of 64 of them.
    const int threads = 64;
    const int64_t blocks = (p.n + threads - 1) / threads;
    predict_kernel<<<static_cast<unsigned>(blocks), threads, 0, st>>>(p);
}

void launch_predict_needed(const NeededParams &p, cudaStream_t st)
{
    const int64_t threads_total = static_cast<int64_t>(p.n_act) * (static_cast<int64_t>(p.cap) + 1);
    if (threads_total <= 0) return;
    // 64-thread blocks, as for the full prediction: the FP64 polynomial is
    // bound by the SMs it reaches
    const int threads = 64;
    const int64_t blocks = (threads_total + threads - 1) / threads;
    predict_needed_kernel<<<static_cast<unsigned>(blocks), threads, 0, st>>>(p);
}

void launch_merge(const MergeParams &p, cudaStream_t st)
{
    if (p.n_total <= 0) return;
    // one warp per block: a small merge spreads over as many SMs as it has particles
    const int threads = 32;
    const int64_t blocks = (p.n_total * 32 + threads - 1) / threads;
    merge_kernel<<<static_cast<unsigned>(blocks), threads, 0, st>>>(p);
}

}  // namespace nb
