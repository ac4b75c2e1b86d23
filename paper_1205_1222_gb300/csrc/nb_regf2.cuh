// Packed-FP32 variant of the regular-force kernel (Sec. 3.3 step (vi),
// criterion of Sec. 3.2) for the float forms.
//
// Same work decomposition as nb_regf.cuh (a warp owns an i-tile, lanes take
// consecutive j from a TMA-filled shared-memory tile, ballot + popc list
// compaction), with three changes:
//   * the pair arithmetic of two i-particles runs in one instruction:
//     Blackwell's f32x2 add/sub/mul/fma operate on a pair of FP32 values held
//     in a 64-bit register pair, so the i-tile is processed as I/2 i-pairs
//     and every FP32 add, multiply and fused multiply-add of an interaction
//     issues once per two pairs (i, j); the j-values are broadcast to both
//     halves once per j-step; the neighbour test, the reciprocal square root
//     and the select stay scalar;
//   * the j-tiles flow through an NST-stage ring without CTA-wide barriers:
//     each warp waits on the stage's full mbarrier, computes, and counts
//     itself out of the stage on a shared counter; the last warp out refills
//     the stage with the tile NST steps ahead (every warp tracks that
//     look-ahead position), so warps drift freely within the ring;
//   * per-lane float-float totals live in shared memory (folded every
//     FOLD_STEPS j-steps), which leaves the register file to the i-pairs and
//     the FP32 partial sums.
#pragma once

#include <cfloat>

#include "nb_device.cuh"
#include "nb_regf.cuh"

namespace nb {

typedef unsigned long long f2;   // two FP32 values in a 64-bit register pair (.x = first of the pair)

__device__ __forceinline__ f2 pk(float a, float b)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ f2 bc(float a) { return pk(a, a); }
__device__ __forceinline__ void up(f2 v, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b)
{
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// Hardware reciprocal square root approximation (PTX rsqrt.approx; a zero
// argument gives +inf, which the neighbour select replaces by 0 for self).
__device__ __forceinline__ float rsqrt_hw(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct Acc2 {
    f2 f[3], j[3], p;
};

// Shared tail of the packed pair terms: r^2, R.V, neighbour test, 1/r, force,
// jerk (and potential) for an i-pair against one j.
template <bool VC, bool POT>
__device__ __forceinline__ void tail2(f2 h2, f2 dtr, f2 m, f2 dx, f2 dy, f2 dz, f2 ux, f2 uy, f2 uz,
                                      Acc2 &a, bool &fa, bool &fb)
{
    const f2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
    const f2 rv = fma2(dz, uz, fma2(dy, uy, mul2(dx, ux)));
    float r2a, r2b, qa, qb, ha, hb;
    up(r2, r2a, r2b);
    qa = r2a;
    qb = r2b;
    if (VC) {
        const f2 px = fma2(dtr, ux, dx), py = fma2(dtr, uy, dy), pz = fma2(dtr, uz, dz);
        float pa, pb;
        up(fma2(pz, pz, fma2(py, py, mul2(px, px))), pa, pb);
        qa = fminf(qa, pa);
        qb = fminf(qb, pb);
    }
    up(h2, ha, hb);
    fa = qa < ha;
    fb = qb < hb;
    float ra = rsqrt_hw(r2a), rb = rsqrt_hw(r2b);
    ra = fa ? 0.f : ra;
    rb = fb ? 0.f : rb;
    const f2 rinv = pk(ra, rb);
    const f2 rinv2 = mul2(rinv, rinv);
    const f2 mr = mul2(m, rinv);
    const f2 mr3 = mul2(mr, rinv2);
    const f2 al = mul2(bc(-3.f), mul2(rv, rinv2));
    a.f[0] = fma2(mr3, dx, a.f[0]);
    a.f[1] = fma2(mr3, dy, a.f[1]);
    a.f[2] = fma2(mr3, dz, a.f[2]);
    a.j[0] = fma2(mr3, fma2(al, dx, ux), a.j[0]);
    a.j[1] = fma2(mr3, fma2(al, dy, uy), a.j[1]);
    a.j[2] = fma2(mr3, fma2(al, dz, uz), a.j[2]);
    if (POT) a.p = add2(a.p, mr);
}

// Two-float (mixed) form, packed over i-pairs.  i-values are stored negated so
// every difference is an add.
struct PackedMixed {
    static constexpr int NS = 4, EB = 16;
    using JS = FormMixed::JS;
    struct JB {   // j-values broadcast to both halves of a pair, built once per j-step
        f2 xh[3], xl[3], vh[3], vl[3], m;
    };
    static __device__ __forceinline__ void bcast(const JS &j, JB &b)
    {
        for (int c = 0; c < 3; c++) {
            b.xh[c] = bc(j.xh[c]);
            b.xl[c] = bc(j.xl[c]);
            b.vh[c] = bc(j.vh[c]);
            b.vl[c] = bc(j.vl[c]);
        }
        b.m = bc(j.m);
    }
    struct IP {
        f2 nxh[3], nxl[3], nvh[3], nvl[3], h2, dtr;
    };
    template <int JT>
    static __device__ __forceinline__ void load_j(JS &s, const unsigned char *st, int jl)
    {
        FormMixed::load_j<JT>(s, st, jl);
    }
    static __device__ __forceinline__ void far_j(JS &s) { FormMixed::far_j(s); }
    static __device__ __forceinline__ void set_i(IP &ip, const JSet &js, int64_t sa, int64_t sb, float h2a,
                                                 float h2b, float dta, float dtb)
    {
        FormMixed::IS a, b;
        FormMixed::clear_i(a);
        FormMixed::clear_i(b);
        if (sa >= 0) FormMixed::load_i(a, js, sa);
        if (sb >= 0) FormMixed::load_i(b, js, sb);
        for (int c = 0; c < 3; c++) {
            ip.nxh[c] = pk(-a.xh[c], -b.xh[c]);
            ip.nxl[c] = pk(-a.xl[c], -b.xl[c]);
            ip.nvh[c] = pk(-a.vh[c], -b.vh[c]);
            ip.nvl[c] = pk(-a.vl[c], -b.vl[c]);
        }
        ip.h2 = pk(h2a, h2b);
        ip.dtr = pk(dta, dtb);
    }
    template <bool VC, bool POT>
    static __device__ __forceinline__ void pair(const IP &i, const JB &j, Acc2 &a, bool &fa, bool &fb)
    {
        const f2 dx = add2(add2(j.xh[0], i.nxh[0]), add2(j.xl[0], i.nxl[0]));
        const f2 dy = add2(add2(j.xh[1], i.nxh[1]), add2(j.xl[1], i.nxl[1]));
        const f2 dz = add2(add2(j.xh[2], i.nxh[2]), add2(j.xl[2], i.nxl[2]));
        const f2 ux = add2(add2(j.vh[0], i.nvh[0]), add2(j.vl[0], i.nvl[0]));
        const f2 uy = add2(add2(j.vh[1], i.nvh[1]), add2(j.vl[1], i.nvl[1]));
        const f2 uz = add2(add2(j.vh[2], i.nvh[2]), add2(j.vl[2], i.nvl[2]));
        tail2<VC, POT>(i.h2, i.dtr, j.m, dx, dy, dz, ux, uy, uz, a, fa, fb);
    }
};

// Plain FP32 form, packed over i-pairs.
struct PackedFP32 {
    static constexpr int NS = 2, EB = 16;
    using JS = FormFP32::JS;
    struct JB {
        f2 x[3], v[3], m;
    };
    static __device__ __forceinline__ void bcast(const JS &j, JB &b)
    {
        for (int c = 0; c < 3; c++) {
            b.x[c] = bc(j.x[c]);
            b.v[c] = bc(j.v[c]);
        }
        b.m = bc(j.m);
    }
    struct IP {
        f2 nx[3], nv[3], h2, dtr;
    };
    template <int JT>
    static __device__ __forceinline__ void load_j(JS &s, const unsigned char *st, int jl)
    {
        FormFP32::load_j<JT>(s, st, jl);
    }
    static __device__ __forceinline__ void far_j(JS &s) { FormFP32::far_j(s); }
    static __device__ __forceinline__ void set_i(IP &ip, const JSet &js, int64_t sa, int64_t sb, float h2a,
                                                 float h2b, float dta, float dtb)
    {
        FormFP32::IS a, b;
        FormFP32::clear_i(a);
        FormFP32::clear_i(b);
        if (sa >= 0) FormFP32::load_i(a, js, sa);
        if (sb >= 0) FormFP32::load_i(b, js, sb);
        for (int c = 0; c < 3; c++) {
            ip.nx[c] = pk(-a.x[c], -b.x[c]);
            ip.nv[c] = pk(-a.v[c], -b.v[c]);
        }
        ip.h2 = pk(h2a, h2b);
        ip.dtr = pk(dta, dtb);
    }
    template <bool VC, bool POT>
    static __device__ __forceinline__ void pair(const IP &i, const JB &j, Acc2 &a, bool &fa, bool &fb)
    {
        tail2<VC, POT>(i.h2, i.dtr, j.m, add2(j.x[0], i.nx[0]), add2(j.x[1], i.nx[1]), add2(j.x[2], i.nx[2]),
                       add2(j.v[0], i.nv[0]), add2(j.v[1], i.nv[1]), add2(j.v[2], i.nv[2]), a, fa, fb);
    }
};

// (hi, lo) pairs += p with the rounding error kept (TwoSum on both halves).
__device__ __forceinline__ void ff_add2(f2 &hi, f2 &lo, f2 p)
{
    const f2 s = add2(hi, p);
    const f2 bp = sub2(s, hi);
    const f2 e = add2(sub2(hi, sub2(s, bp)), sub2(p, bp));
    hi = s;
    lo = add2(lo, e);
}


template <class Fm, int W, int I, int JT>
struct PackedLayout {
    static constexpr int NST = 4;                                  // stages of the j-tile ring
    static constexpr int STAGE = Fm::NS * Fm::EB * JT;
    static constexpr int STAGES = 128;                             // barriers + release counters first
    static constexpr int TOT = STAGES + NST * STAGE;
    __host__ __device__ static constexpr int tot_bytes(bool pot) { return W * (I / 2) * (pot ? 7 : 6) * 32 * 16; }
    __host__ __device__ static constexpr int cnt(bool pot) { return TOT + tot_bytes(pot); }
    __host__ __device__ static constexpr int gi(bool pot) { return cnt(pot) + W * I * 4; }
    __host__ __device__ static constexpr int desc(bool pot) { return gi(pot) + W * I * 4; }
    __host__ __device__ static constexpr int bytes(bool pot) { return desc(pot) + W * static_cast<int>(sizeof(ClusterDesc)); }
};

template <class Fm, int W, int I, int JT>
constexpr int packed_smem_bytes(bool pot)
{
    return PackedLayout<Fm, W, I, JT>::bytes(pot);
}

// Position in the CTA's sequence of j-tiles: the work item, the tile in it,
// the item's tile end, and the j-range the copies read.
struct TileCursor {
    int64_t item;
    int64_t jb;
    int nj, tile, te;
};

__device__ __forceinline__ void cursor_set(const RegfParams &p, TileCursor &c)
{
    if (c.item >= p.n_items) return;
    int64_t item_begin, jb;
    int n_split, tps, n_tiles, nj;
    if (p.table) {
        const ClusterDesc &d = p.table[find_cluster(p, c.item)];
        item_begin = d.item_begin; jb = d.j_begin; nj = d.n_j;
        n_split = d.n_split; tps = d.tiles_per_split; n_tiles = d.n_tiles;
    } else {
        item_begin = p.d0.item_begin; jb = p.d0.j_begin; nj = p.d0.n_j;
        n_split = p.d0.n_split; tps = p.d0.tiles_per_split; n_tiles = p.d0.n_tiles;
    }
    const int64_t local = c.item - item_begin;
    const int sp = static_cast<int>(local % n_split);
    c.jb = jb;
    c.nj = nj;
    c.tile = sp * tps;
    c.te = min(c.tile + tps, n_tiles);
}

__device__ __forceinline__ void cursor_next(const RegfParams &p, TileCursor &c)
{
    if (++c.tile < c.te) return;
    c.item += gridDim.x;
    cursor_set(p, c);
}

template <class Fm, int JT, int NST>
__device__ __forceinline__ void issue_at(const RegfParams &p, const TileCursor &c, uint32_t seq, uint64_t *full,
                                         unsigned char *stages)
{
    constexpr int STAGE = Fm::NS * Fm::EB * JT;
    const int s = seq % NST;
    uint64_t *b = &full[s];
    unsigned char *st = stages + s * STAGE;
    const int count = min(JT, c.nj - c.tile * JT);
    const uint32_t bytes = static_cast<uint32_t>(count) * Fm::EB;
    mbar_arrive_expect_tx(b, bytes * Fm::NS + p.extra_tx);
    const int64_t first = c.jb + static_cast<int64_t>(c.tile) * JT;
#pragma unroll
    for (int k = 0; k < Fm::NS; k++)
        tma_bulk_g2s(st + k * JT * Fm::EB, static_cast<const unsigned char *>(p.js.s[k]) + first * Fm::EB, bytes,
                     b);
}

template <class Fm, int W, int I, int JT, int FLAGS, int MINB>
__global__ void __launch_bounds__(W * 32, MINB) regf2_kernel(const RegfParams p)
{
    static_assert(I % 2 == 0, "the i-tile is processed in pairs");
    using L = PackedLayout<Fm, W, I, JT>;
    constexpr bool VC = (FLAGS & 1) != 0;
    constexpr bool POT = (FLAGS & 2) != 0;
    constexpr int IP = I / 2;
    constexpr int NC = POT ? 7 : 6;
    constexpr int NST = L::NST;
    constexpr int STEPS = JT / 32;
    constexpr int FOLD_STEPS = 128;                               // j-steps per lane per FP32 partial
    constexpr int FOLD_TILES = STEPS >= FOLD_STEPS ? 1 : FOLD_STEPS / STEPS;
    using JS = typename Fm::JS;
    using JB = typename Fm::JB;
    using IPt = typename Fm::IP;

    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    int *rel = reinterpret_cast<int *>(smem + 8 * NST);
    unsigned char *stages = smem + L::STAGES;
    float4 *s_tot = reinterpret_cast<float4 *>(smem + L::TOT);
    int *s_cnt = reinterpret_cast<int *>(smem + L::cnt(POT));
    int *s_gi = reinterpret_cast<int *>(smem + L::gi(POT));
    ClusterDesc *s_d = reinterpret_cast<ClusterDesc *>(smem + L::desc(POT));

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    TileCursor la;
    la.item = blockIdx.x;
    cursor_set(p, la);
    if (tid == 0) {
        for (int s = 0; s < NST; s++) {
            mbar_init(&full[s], 1);
            rel[s] = 0;
        }
        fence_mbar_init();
        TileCursor c0 = la;
        for (int q = 0; q < NST && c0.item < p.n_items; ++q) {
            issue_at<Fm, JT, NST>(p, c0, q, full, stages);
            cursor_next(p, c0);
        }
    }
    for (int q = 0; q < NST && la.item < p.n_items; ++q) cursor_next(p, la);   // look-ahead = sequence NST
    __syncthreads();

    uint32_t g = 0;
    bool aborted = false;
    float4 *mytot = s_tot + warp * IP * NC * 32 + lane;    // + (pair * NC + comp) * 32
    int *mycnt = s_cnt + warp * I;
    int *mygi = s_gi + warp * I;
    ClusterDesc &d = s_d[warp];

    for (int64_t item = blockIdx.x; item < p.n_items && !aborted; item += gridDim.x) {
        if (lane == 0) d = p.table ? p.table[find_cluster(p, item)] : p.d0;
        __syncwarp();
        const int64_t local = item - d.item_begin;
        const int ib = static_cast<int>(local / d.n_split);
        const int sp = static_cast<int>(local - static_cast<int64_t>(ib) * d.n_split);
        const int tb = sp * d.tiles_per_split;
        const int te = min(tb + d.tiles_per_split, d.n_tiles);

        // the warp's i-pairs
        IPt ip[IP];
        Acc2 acc[IP];
        const int i0 = (ib * W + warp) * I;
#pragma unroll
        for (int q = 0; q < IP; q++) {
            int64_t slot[2];
            float h2v[2], dtv[2];
            for (int h = 0; h < 2; h++) {
                const int idx = i0 + 2 * q + h;
                slot[h] = -1;
                h2v[h] = -1.f;
                dtv[h] = 0.f;
                int gi = -1;
                if (idx < d.n_act) {
                    const int a = d.act[idx];
                    const double hv = d.h[idx];
                    if (a >= 0 && a < d.n_j && hv >= 0.0 && hv <= DBL_MAX) {
                        gi = a;
                        slot[h] = d.j_begin + a;
                        h2v[h] = fmaxf(__double2float_rn(hv * hv), FLT_MIN);   // self (r2 = 0) is inside
                        dtv[h] = (VC && d.dtr) ? __double2float_rn(d.dtr[idx]) : 0.f;
                    } else if (lane == 0) {
                        atomicOr(p.status, DEV_BAD_INPUT);
                    }
                }
                if (lane == 0) { mygi[2 * q + h] = gi; mycnt[2 * q + h] = 0; }
            }
            Fm::set_i(ip[q], p.js, slot[0], slot[1], h2v[0], h2v[1], dtv[0], dtv[1]);
            for (int c = 0; c < 3; c++) acc[q].f[c] = acc[q].j[c] = 0ull;
            acc[q].p = 0ull;
            for (int c = 0; c < NC; c++) mytot[(q * NC + c) * 32] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncwarp();

        for (int t = tb; t < te; ++t, ++g) {
            const int s = g % NST;
            if (!mbar_wait_bounded(&full[s], (g / NST) & 1, p.wait_ns)) { aborted = true; break; }
            const unsigned char *st = stages + s * L::STAGE;
            const int jt0 = t * JT;
            const int count = min(JT, d.n_j - jt0);
            const bool tailtile = count < JT;
#pragma unroll 2
            for (int k = 0; k < STEPS; ++k) {
                const int jl = k * 32 + lane;
                JS js;
                Fm::template load_j<JT>(js, st, jl);
                if (tailtile && jl >= count) Fm::far_j(js);
                JB jb;
                Fm::bcast(js, jb);
                bool f[I];
                bool any = false;
#pragma unroll
                for (int q = 0; q < IP; q++) {
                    Fm::template pair<VC, POT>(ip[q], jb, acc[q], f[2 * q], f[2 * q + 1]);
                    any |= f[2 * q] | f[2 * q + 1];
                }
                if (__any_sync(0xffffffffu, any)) {
                    const int jg = jt0 + jl;
#pragma unroll
                    for (int k2 = 0; k2 < I; k2++) {
                        const bool fk = f[k2] && jg != mygi[k2];
                        const unsigned mask = __ballot_sync(0xffffffffu, fk);
                        if (mask) {
                            const int c0 = mycnt[k2];
                            const int pos = c0 + __popc(mask & lanemask_lt());
                            if (fk && pos < d.cap) {
                                const int64_t idx = i0 + k2;
                                int32_t *row = d.n_split == 1
                                                   ? d.list + idx * d.cap
                                                   : d.plist + (static_cast<int64_t>(sp) * d.n_act + idx) * d.cap;
                                row[pos] = jg;
                            }
                            __syncwarp();
                            if (lane == 0) mycnt[k2] = c0 + __popc(mask);
                            __syncwarp();
                        }
                    }
                }
            }
            // count this warp out of the stage; the last one refills it NST tiles ahead
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                if (atomicAdd(&rel[s], 1) == W - 1) {
                    rel[s] = 0;
                    if (la.item < p.n_items) issue_at<Fm, JT, NST>(p, la, g + NST, full, stages);
                }
            }
            cursor_next(p, la);
            if ((t - tb + 1) % FOLD_TILES == 0 || t + 1 == te) {
#pragma unroll
                for (int q = 0; q < IP; q++) {
#pragma unroll
                    for (int c = 0; c < NC; c++) {
                        f2 &part = c < 3 ? acc[q].f[c] : (c < 6 ? acc[q].j[c - 3] : acc[q].p);
                        float4 *slot = mytot + (q * NC + c) * 32;
                        float4 v = *slot;
                        f2 hi = pk(v.x, v.y), lo = pk(v.z, v.w);
                        ff_add2(hi, lo, part);
                        up(hi, v.x, v.y);
                        up(lo, v.z, v.w);
                        *slot = v;
                        part = 0ull;
                    }
                }
            }
        }
        if (aborted) break;

        // reduce the float-float totals over the 32 lanes and write
#pragma unroll
        for (int q = 0; q < IP; q++) {
            for (int h = 0; h < 2; h++) {
                double out[7] = {0, 0, 0, 0, 0, 0, 0};
                for (int c = 0; c < NC; c++) {
                    const float4 v = mytot[(q * NC + c) * 32];
                    float hi = h ? v.y : v.x, lo = h ? v.w : v.z;
                    for (int o = 16; o > 0; o >>= 1) {
                        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
                        const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
                        ff_add_ff(hi, lo, h2, l2);
                    }
                    out[c] = static_cast<double>(hi) + static_cast<double>(lo);
                }
                const int k = 2 * q + h;
                const int64_t i = i0 + k;
                if (lane == 0 && mygi[k] >= 0) {
                    const int cnt = mycnt[k];
                    if (d.n_split == 1) {
                        for (int c = 0; c < 3; c++) { d.F[3 * i + c] = out[c]; d.J[3 * i + c] = out[3 + c]; }
                        if (POT && d.pot) d.pot[i] = out[6];
                        d.nnb[i] = cnt;
                        d.ovf[i] = cnt > d.cap ? 1 : 0;
                    } else {
                        double *o8 = d.pF + (static_cast<int64_t>(sp) * d.n_act + i) * 8;
                        for (int c = 0; c < 7; c++) o8[c] = c < NC ? out[c] : 0.0;
                        d.pcnt[static_cast<int64_t>(sp) * d.n_act + i] = cnt;
                    }
                }
            }
        }
        __syncwarp();
    }

    if (aborted && lane == 0) {
        atomicOr(p.status, DEV_TIMEOUT);
        // let copies that may still be in flight land before the CTA's shared memory goes away
        for (uint32_t q = g; q < g + NST; ++q) mbar_wait_bounded(&full[q % NST], (q / NST) & 1, p.wait_ns);
    }
}

}  // namespace nb
