// Regular force + jerk + neighbour list kernel (Nitadori & Aarseth 2012,
// Sec. 3.3 step (vi), neighbour criterion of Sec. 3.2), persistent over work
// items (cluster, i-block, j-split).
//
// GB300 layout of the work (not the paper's one-thread-per-i layout):
//   * a warp owns an i-tile of I active particles; its 32 lanes take 32
//     consecutive j-particles at a time, so every lane evaluates I pairs per
//     step and the neighbour flags of one i over 32 consecutive j form one
//     ballot mask; the ascending list is compacted warp-wide with the ballot
//     and a population-count prefix (Sec. 3.4 stores indices with a running
//     counter per thread instead);
//   * a CTA of W warps shares a j-tile of JT particles staged in shared memory
//     by bulk asynchronous copies (TMA, cp.async.bulk) into a two-stage ring
//     guarded by mbarriers; the streams are SoA float4/double4 so a warp's
//     shared-memory loads are conflict-free;
//   * the pair test is a select on the reciprocal distance (the paper's
//     predicated "rinv1 = 0", Listing B2 semantics); the list append is a
//     warp-uniform branch taken only when some lane found a neighbour;
//   * float forms keep FP32 partial sums per lane for at most 64 j-steps and
//     fold them into float-float (TwoSum) totals; the totals are reduced
//     across lanes in float-float and written in FP64.  With more than one
//     j-split per i-block, per-split FP64 partials and partial lists go to a
//     scratch area and a merge kernel concatenates them (Sec. 3.4: "force
//     reduction and list gathering").
#pragma once

#include <cfloat>

#include "nb_device.cuh"

namespace nb {

constexpr float FAR_F = 1.0e18f;   // position of padding lanes: r^2 ~ 1e36 stays finite
constexpr double FAR_D = 1.0e100;

struct AccF {
    float f[3], j[3], p;
};
struct TotF {
    float fh[3], fl[3], jh[3], jl[3], ph, pl;
};
struct AccD {
    double f[3], j[3], p;
};

// ----------------------------------------------------------------- forms

// Two-float positions and velocities: hi = fl(x), lo = fl(x - hi).
struct FormMixed {
    static constexpr int NS = 4;        // posm_hi, pos_lo, vel_hi, vel_lo
    static constexpr int EB = 16;       // bytes per stream element
    static constexpr bool F64 = false;
    using Acc = AccF;
    struct IS {
        float xh[3], xl[3], vh[3], vl[3], h2, dtr;
    };
    struct JS {
        float xh[3], m, xl[3], vh[3], vl[3];
    };
    static __device__ __forceinline__ void load_i(IS &s, const JSet &js, int64_t slot)
    {
        const float4 a = reinterpret_cast<const float4 *>(js.s[0])[slot];
        const float4 b = reinterpret_cast<const float4 *>(js.s[1])[slot];
        const float4 c = reinterpret_cast<const float4 *>(js.s[2])[slot];
        const float4 d = reinterpret_cast<const float4 *>(js.s[3])[slot];
        s.xh[0] = a.x; s.xh[1] = a.y; s.xh[2] = a.z;
        s.xl[0] = b.x; s.xl[1] = b.y; s.xl[2] = b.z;
        s.vh[0] = c.x; s.vh[1] = c.y; s.vh[2] = c.z;
        s.vl[0] = d.x; s.vl[1] = d.y; s.vl[2] = d.z;
    }
    static __device__ __forceinline__ void clear_i(IS &s)
    {
        for (int k = 0; k < 3; k++) s.xh[k] = s.xl[k] = s.vh[k] = s.vl[k] = 0.f;
        s.h2 = -1.f;
        s.dtr = 0.f;
    }
    static __device__ __forceinline__ void set_radius(IS &s, double h, double dtr)
    {
        s.h2 = fmaxf(__double2float_rn(h * h), FLT_MIN);   // FLT_MIN: self (r2 = 0) is inside
        s.dtr = __double2float_rn(dtr);
    }
    template <int JT>
    static __device__ __forceinline__ void load_j(JS &s, const unsigned char *st, int jl)
    {
        const float4 *p = reinterpret_cast<const float4 *>(st);
        const float4 a = p[jl], b = p[JT + jl], c = p[2 * JT + jl], d = p[3 * JT + jl];
        s.xh[0] = a.x; s.xh[1] = a.y; s.xh[2] = a.z; s.m = a.w;
        s.xl[0] = b.x; s.xl[1] = b.y; s.xl[2] = b.z;
        s.vh[0] = c.x; s.vh[1] = c.y; s.vh[2] = c.z;
        s.vl[0] = d.x; s.vl[1] = d.y; s.vl[2] = d.z;
    }
    static __device__ __forceinline__ void far_j(JS &s)
    {
        for (int k = 0; k < 3; k++) { s.xh[k] = FAR_F; s.xl[k] = 0.f; s.vh[k] = 0.f; s.vl[k] = 0.f; }
        s.m = 0.f;
    }
    template <bool VC, bool POT>
    static __device__ __forceinline__ bool pair(const IS &i, const JS &j, Acc &a)
    {
        // two-float differences: (xj_hi - xi_hi) + (xj_lo - xi_lo)
        const float dx = (j.xh[0] - i.xh[0]) + (j.xl[0] - i.xl[0]);
        const float dy = (j.xh[1] - i.xh[1]) + (j.xl[1] - i.xl[1]);
        const float dz = (j.xh[2] - i.xh[2]) + (j.xl[2] - i.xl[2]);
        const float ux = (j.vh[0] - i.vh[0]) + (j.vl[0] - i.vl[0]);
        const float uy = (j.vh[1] - i.vh[1]) + (j.vl[1] - i.vl[1]);
        const float uz = (j.vh[2] - i.vh[2]) + (j.vl[2] - i.vl[2]);
        return tail<VC, POT>(i.h2, i.dtr, j.m, dx, dy, dz, ux, uy, uz, a);
    }
    template <bool VC, bool POT>
    static __device__ __forceinline__ bool tail(float h2, float dtr, float m, float dx, float dy,
                                                float dz, float ux, float uy, float uz, Acc &a)
    {
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        const float rv = fmaf(dz, uz, fmaf(dy, uy, dx * ux));
        float q = r2;
        if (VC) {
            const float px = fmaf(dtr, ux, dx), py = fmaf(dtr, uy, dy), pz = fmaf(dtr, uz, dz);
            q = fminf(r2, fmaf(pz, pz, fmaf(py, py, px * px)));
        }
        const bool nb = q < h2;
        float rinv = rsqrtf(r2);
        rinv = nb ? 0.f : rinv;
        const float rinv2 = rinv * rinv;
        const float mr = m * rinv;
        const float mr3 = mr * rinv2;
        const float al = -3.f * (rv * rinv2);
        a.f[0] = fmaf(mr3, dx, a.f[0]);
        a.f[1] = fmaf(mr3, dy, a.f[1]);
        a.f[2] = fmaf(mr3, dz, a.f[2]);
        a.j[0] = fmaf(mr3, fmaf(al, dx, ux), a.j[0]);
        a.j[1] = fmaf(mr3, fmaf(al, dy, uy), a.j[1]);
        a.j[2] = fmaf(mr3, fmaf(al, dz, uz), a.j[2]);
        if (POT) a.p += mr;
        return nb;
    }
};

// Plain FP32 positions and velocities.
struct FormFP32 {
    static constexpr int NS = 2;        // posm, vel
    static constexpr int EB = 16;
    static constexpr bool F64 = false;
    using Acc = AccF;
    struct IS {
        float x[3], v[3], h2, dtr;
    };
    struct JS {
        float x[3], m, v[3];
    };
    static __device__ __forceinline__ void load_i(IS &s, const JSet &js, int64_t slot)
    {
        const float4 a = reinterpret_cast<const float4 *>(js.s[0])[slot];
        const float4 b = reinterpret_cast<const float4 *>(js.s[1])[slot];
        s.x[0] = a.x; s.x[1] = a.y; s.x[2] = a.z;
        s.v[0] = b.x; s.v[1] = b.y; s.v[2] = b.z;
    }
    static __device__ __forceinline__ void clear_i(IS &s)
    {
        for (int k = 0; k < 3; k++) s.x[k] = s.v[k] = 0.f;
        s.h2 = -1.f;
        s.dtr = 0.f;
    }
    static __device__ __forceinline__ void set_radius(IS &s, double h, double dtr)
    {
        s.h2 = fmaxf(__double2float_rn(h * h), FLT_MIN);
        s.dtr = __double2float_rn(dtr);
    }
    template <int JT>
    static __device__ __forceinline__ void load_j(JS &s, const unsigned char *st, int jl)
    {
        const float4 *p = reinterpret_cast<const float4 *>(st);
        const float4 a = p[jl], b = p[JT + jl];
        s.x[0] = a.x; s.x[1] = a.y; s.x[2] = a.z; s.m = a.w;
        s.v[0] = b.x; s.v[1] = b.y; s.v[2] = b.z;
    }
    static __device__ __forceinline__ void far_j(JS &s)
    {
        for (int k = 0; k < 3; k++) { s.x[k] = FAR_F; s.v[k] = 0.f; }
        s.m = 0.f;
    }
    template <bool VC, bool POT>
    static __device__ __forceinline__ bool pair(const IS &i, const JS &j, Acc &a)
    {
        return FormMixed::tail<VC, POT>(i.h2, i.dtr, j.m, j.x[0] - i.x[0], j.x[1] - i.x[1],
                                        j.x[2] - i.x[2], j.v[0] - i.v[0], j.v[1] - i.v[1],
                                        j.v[2] - i.v[2], a);
    }
};

// FP64 throughout.
struct FormFP64 {
    static constexpr int NS = 2;        // posm, vel as 32-byte double4
    static constexpr int EB = 32;
    static constexpr bool F64 = true;
    using Acc = AccD;
    struct IS {
        double x[3], v[3], h2, dtr;
    };
    struct JS {
        double x[3], m, v[3];
    };
    static __device__ __forceinline__ void load_i(IS &s, const JSet &js, int64_t slot)
    {
        const double4_32a a = reinterpret_cast<const double4_32a *>(js.s[0])[slot];
        const double4_32a b = reinterpret_cast<const double4_32a *>(js.s[1])[slot];
        s.x[0] = a.x; s.x[1] = a.y; s.x[2] = a.z;
        s.v[0] = b.x; s.v[1] = b.y; s.v[2] = b.z;
    }
    static __device__ __forceinline__ void clear_i(IS &s)
    {
        for (int k = 0; k < 3; k++) s.x[k] = s.v[k] = 0.0;
        s.h2 = -1.0;
        s.dtr = 0.0;
    }
    static __device__ __forceinline__ void set_radius(IS &s, double h, double dtr)
    {
        s.h2 = fmax(h * h, DBL_MIN);
        s.dtr = dtr;
    }
    template <int JT>
    static __device__ __forceinline__ void load_j(JS &s, const unsigned char *st, int jl)
    {
        const double4_32a *p = reinterpret_cast<const double4_32a *>(st);
        const double4_32a a = p[jl], b = p[JT + jl];
        s.x[0] = a.x; s.x[1] = a.y; s.x[2] = a.z; s.m = a.w;
        s.v[0] = b.x; s.v[1] = b.y; s.v[2] = b.z;
    }
    static __device__ __forceinline__ void far_j(JS &s)
    {
        for (int k = 0; k < 3; k++) { s.x[k] = FAR_D; s.v[k] = 0.0; }
        s.m = 0.0;
    }
    template <bool VC, bool POT>
    static __device__ __forceinline__ bool pair(const IS &i, const JS &j, Acc &a)
    {
        const double dx = j.x[0] - i.x[0], dy = j.x[1] - i.x[1], dz = j.x[2] - i.x[2];
        const double ux = j.v[0] - i.v[0], uy = j.v[1] - i.v[1], uz = j.v[2] - i.v[2];
        const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
        const double rv = fma(dz, uz, fma(dy, uy, dx * ux));
        double q = r2;
        if (VC) {
            const double px = fma(i.dtr, ux, dx), py = fma(i.dtr, uy, dy), pz = fma(i.dtr, uz, dz);
            q = fmin(r2, fma(pz, pz, fma(py, py, px * px)));
        }
        const bool nb = q < i.h2;
        double rinv = rsqrt(r2);
        rinv = nb ? 0.0 : rinv;
        const double rinv2 = rinv * rinv;
        const double mr = j.m * rinv;
        const double mr3 = mr * rinv2;
        const double al = -3.0 * (rv * rinv2);
        a.f[0] = fma(mr3, dx, a.f[0]);
        a.f[1] = fma(mr3, dy, a.f[1]);
        a.f[2] = fma(mr3, dz, a.f[2]);
        a.j[0] = fma(mr3, fma(al, dx, ux), a.j[0]);
        a.j[1] = fma(mr3, fma(al, dy, uy), a.j[1]);
        a.j[2] = fma(mr3, fma(al, dz, uz), a.j[2]);
        if (POT) a.p += mr;
        return nb;
    }
};

// ------------------------------------------------------------ the kernel

template <class Fm, int JT>
__device__ __forceinline__ void issue_tile(const RegfParams &p, const ClusterDesc &d, int tile,
                                           uint32_t seq, uint64_t *bar, unsigned char *stages)
{
    constexpr int STAGE = Fm::NS * Fm::EB * JT;
    uint64_t *b = &bar[seq & 1];
    unsigned char *st = stages + (seq & 1) * STAGE;
    const int count = min(JT, d.n_j - tile * JT);
    const uint32_t bytes = static_cast<uint32_t>(count) * Fm::EB;
    mbar_arrive_expect_tx(b, bytes * Fm::NS + p.extra_tx);
    const int64_t first = d.j_begin + static_cast<int64_t>(tile) * JT;
#pragma unroll
    for (int k = 0; k < Fm::NS; k++)
        tma_bulk_g2s(st + k * JT * Fm::EB,
                     static_cast<const unsigned char *>(p.js.s[k]) + first * Fm::EB, bytes, b);
}

template <class Fm, int W, int I, int JT, int FLAGS>
__global__ void __launch_bounds__(W * 32) regf_kernel(const RegfParams p)
{
    constexpr bool VC = (FLAGS & 1) != 0;
    constexpr bool POT = (FLAGS & 2) != 0;
    constexpr int STEPS = JT / 32;
    constexpr int STAGE = Fm::NS * Fm::EB * JT;
    constexpr int FOLD_TILES = JT >= 2048 ? 1 : 2048 / JT;   // <= 64 j-steps per lane per FP32 partial
    using Acc = typename Fm::Acc;
    using IS = typename Fm::IS;
    using JS = typename Fm::JS;

    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    unsigned char *stages = smem + 128;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    uint32_t g = 0;        // tile sequence number of this CTA: stage g & 1, phase (g >> 1) & 1
    uint32_t issued = 0;   // tiles issued so far (thread 0)
    bool aborted = false;

    for (int64_t pos = blockIdx.x; pos < p.n_items; pos += gridDim.x) {
        int cl, ib, sp;
        if (!item_at(p, pos, cl, ib, sp)) continue;
        ClusterDesc d;
        if (p.work) d = p.table[cl]; else d = p.d0;
        const int tb = sp * d.tiles_per_split;
        const int te = min(tb + d.tiles_per_split, d.n_tiles);

        if (tid == 0) {
            if (tb < te) { issue_tile<Fm, JT>(p, d, tb, g, bar, stages); issued = g + 1; }
            if (tb + 1 < te) { issue_tile<Fm, JT>(p, d, tb + 1, g + 1, bar, stages); issued = g + 2; }
        }

        // i-tile of this warp
        IS is[I];
        int gi[I], idx[I];
        int32_t *lrow[I];
        int cnt[I];
        Acc acc[I];
        TotF tot[I];
#pragma unroll
        for (int k = 0; k < I; k++) {
            idx[k] = (ib * W + warp) * I + k;
            gi[k] = -1;
            cnt[k] = 0;
            lrow[k] = nullptr;
            Fm::clear_i(is[k]);
            bool ok = idx[k] < d.n_act;
            if (ok) {
                const int a = d.act[idx[k]];
                const double hv = d.h[idx[k]];
                const double dt = (VC && d.dtr) ? d.dtr[idx[k]] : 0.0;
                ok = a >= 0 && a < d.n_j && hv >= 0.0 && hv <= DBL_MAX;
                if (!ok) {
                    if (lane == 0) atomicOr(p.status, DEV_BAD_INPUT);
                } else {
                    gi[k] = a;
                    Fm::load_i(is[k], p.js, d.j_begin + a);
                    Fm::set_radius(is[k], hv, dt);
                    lrow[k] = d.n_split == 1
                                  ? d.list + static_cast<int64_t>(idx[k]) * d.cap
                                  : d.plist + (static_cast<int64_t>(sp) * d.n_act + idx[k]) * d.cap;
                }
            }
            if (!ok) idx[k] = -1;
            acc[k].f[0] = acc[k].f[1] = acc[k].f[2] = 0;
            acc[k].j[0] = acc[k].j[1] = acc[k].j[2] = 0;
            acc[k].p = 0;
            for (int c = 0; c < 3; c++) tot[k].fh[c] = tot[k].fl[c] = tot[k].jh[c] = tot[k].jl[c] = 0.f;
            tot[k].ph = tot[k].pl = 0.f;
        }

        for (int t = tb; t < te; ++t, ++g) {
            const bool ok = mbar_wait_bounded(&bar[g & 1], (g >> 1) & 1, p.wait_ns);
            const unsigned char *st = stages + (g & 1) * STAGE;
            const int jt0 = t * JT;
            const int count = min(JT, d.n_j - jt0);
            if (ok) {
                const bool tailtile = count < JT;
                const int nsteps = tailtile ? (count + 31) >> 5 : STEPS;   // steps that hold a j
#pragma unroll 2
                for (int s = 0; s < nsteps; ++s) {
                    const int jl = s * 32 + lane;
                    JS js;
                    Fm::template load_j<JT>(js, st, jl);
                    if (tailtile && jl >= count) Fm::far_j(js);
                    bool f[I];
                    bool any = false;
#pragma unroll
                    for (int k = 0; k < I; k++) {
                        f[k] = Fm::template pair<VC, POT>(is[k], js, acc[k]);
                        any |= f[k];
                    }
                    if (__any_sync(0xffffffffu, any)) {
                        const int jg = jt0 + jl;
#pragma unroll
                        for (int k = 0; k < I; k++) {
                            const bool fk = f[k] && jg != gi[k];
                            const unsigned mask = __ballot_sync(0xffffffffu, fk);
                            if (mask) {
                                const int pos = cnt[k] + __popc(mask & lanemask_lt());
                                if (fk && pos < d.cap) lrow[k][pos] = jg;
                                cnt[k] += __popc(mask);
                            }
                        }
                    }
                }
            }
            if (!Fm::F64 && ((t - tb + 1) % FOLD_TILES == 0 || t + 1 == te)) {
#pragma unroll
                for (int k = 0; k < I; k++) {
                    for (int c = 0; c < 3; c++) {
                        ff_add(tot[k].fh[c], tot[k].fl[c], static_cast<float>(acc[k].f[c]));
                        ff_add(tot[k].jh[c], tot[k].jl[c], static_cast<float>(acc[k].j[c]));
                        acc[k].f[c] = 0;
                        acc[k].j[c] = 0;
                    }
                    if (POT) { ff_add(tot[k].ph, tot[k].pl, static_cast<float>(acc[k].p)); acc[k].p = 0; }
                }
            }
            if (__syncthreads_or(!ok)) { aborted = true; break; }   // g = the tile that failed
            if (tid == 0 && t + 2 < te) { issue_tile<Fm, JT>(p, d, t + 2, g + 2, bar, stages); issued = g + 3; }
        }
        if (aborted) break;

        // reduce over the 32 lanes and write
        if constexpr (Fm::F64) {
#pragma unroll
            for (int k = 0; k < I; k++) {
                double out[7];
                for (int c = 0; c < 3; c++) { out[c] = acc[k].f[c]; out[3 + c] = acc[k].j[c]; }
                out[6] = acc[k].p;
                for (int o = 16; o > 0; o >>= 1)
                    for (int c = 0; c < 7; c++) out[c] += __shfl_xor_sync(0xffffffffu, out[c], o);
                if (lane == 0 && row_ok(d, sp, idx[k], p.status)) {
                    const int64_t i = idx[k];
                    if (d.n_split == 1) {
                        for (int c = 0; c < 3; c++) { d.F[3 * i + c] = out[c]; d.J[3 * i + c] = out[3 + c]; }
                        if (POT && d.pot) d.pot[i] = out[6];
                    } else {
                        double *q = d.pF + (static_cast<int64_t>(sp) * d.n_act + i) * 8;
                        for (int c = 0; c < 7; c++) q[c] = POT || c < 6 ? out[c] : 0.0;
                    }
                }
            }
        } else {
            constexpr int NC = POT ? 7 : 6;
            FFKeep<I> kept{};
#pragma unroll
            for (int k = 0; k < I; k++) {
                float hi[7], lo[7];
                for (int c = 0; c < 3; c++) {
                    hi[c] = tot[k].fh[c]; lo[c] = tot[k].fl[c];
                    hi[3 + c] = tot[k].jh[c]; lo[3 + c] = tot[k].jl[c];
                }
                hi[6] = tot[k].ph; lo[6] = tot[k].pl;
                for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                    for (int c = 0; c < NC; c++) {
                        const float h2 = __shfl_xor_sync(0xffffffffu, hi[c], o);
                        const float l2 = __shfl_xor_sync(0xffffffffu, lo[c], o);
                        ff_add_ff(hi[c], lo[c], h2, l2);
                    }
                }
#pragma unroll
                for (int c = 0; c < NC; c++) ff_keep(kept, k, c, hi[c], lo[c]);
            }
            write_item_ff<I, NC>(d, sp, kept, idx, p.status);
        }
#pragma unroll
        for (int k = 0; k < I; k++) {
            if (lane == 0 && row_ok(d, sp, idx[k], p.status)) {
                const int64_t i = idx[k];
                if (d.n_split == 1) {
                    d.nnb[i] = cnt[k];
                    d.ovf[i] = cnt[k] > d.cap ? 1 : 0;
                } else {
                    d.pcnt[static_cast<int64_t>(sp) * d.n_act + i] = cnt[k];
                }
            }
        }
    }

    if (aborted) {
        if (tid == 0) {
            atomicOr(p.status, DEV_TIMEOUT);
            // let the copies still in flight land before the CTA's shared memory goes away
            for (uint32_t q = g; q < issued; ++q) mbar_wait_bounded(&bar[q & 1], (q >> 1) & 1, p.wait_ns);
        }
    }
}

}  // namespace nb
