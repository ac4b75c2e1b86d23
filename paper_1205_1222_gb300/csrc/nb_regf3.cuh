// j-pair packed variant of the regular-force kernel (Sec. 3.3 step (vi),
// criterion of Sec. 3.2) for the float forms.
//
// The f32x2 instructions of Blackwell (add/sub/mul/fma on two FP32 values in
// a 64-bit register pair) are fed with pairs of j-particles: every lane takes
// the two consecutive j of one j-pair per step, so a warp covers 64 j per
// step, and the i-particle values are broadcast to both halves once per work
// item.  The predicted j-set is stored pair-interleaved for this kernel: for
// j-pair P (slots 2P, 2P+1) stream k holds one float4 with two components of
// both particles, e.g. (x_a, x_b, y_a, y_b), so one 128-bit shared-memory
// load yields two ready register pairs and no lane ever moves a value into a
// pair.  The j-tiles flow through an NSTAGE-deep TMA ring without CTA-wide
// barriers: each warp waits on the stage's full mbarrier, computes its pair
// terms, and counts itself out of the stage on a shared counter before its
// list pass (which reads only flags kept in registers); the last warp out refills the
// stage with the tile NSTAGE steps ahead (every warp tracks that look-ahead
// position), so warps drift freely within the ring.  Per-lane float-float
// totals live in shared memory (folded every FOLD_STEPS_J / _F steps), leaving the
// register file to the i-values and the FP32 partial sums.  The pair terms of
// a tile run as straight-line code that only records, per i-particle, the
// neighbour flags of the lane's two j in each 64-j unit (two bits per unit);
// after the tile the lists are compacted from the flagged units with ballot +
// popc over the interleaved (lane, half) order, which is ascending j, so the
// list holds exactly the pairs that the force sums left out.
#pragma once

#include <cfloat>
#include <type_traits>

#include "nb_pair_ops.cuh"
#include "nb_sort.cuh"

namespace nb {

// Frame centre of a block of active particles, position and velocity in
// two-float (hi + lo) form (used by the framed form only).
struct Frame2 {
    float xh[3], xl[3], vh[3], vl[3];
};

// Two-float (mixed) form, pair-interleaved: 7 float4 streams per j-pair
//   q0 (xh_a, xh_b, yh_a, yh_b)  q1 (zh_a, zh_b, m_a, m_b)  q2 (xl_a, xl_b, yl_a, yl_b)
//   q3 (zl_a, zl_b, vxh_a, vxh_b)  q4 (vyh_a, vyh_b, vzh_a, vzh_b)
//   q5 (vxl_a, vxl_b, vyl_a, vyl_b)  q6 (vzl_a, vzl_b, 0, 0)
struct PairMixed {
    static constexpr int NS = 7;
    struct IB {   // one i-particle, negated, broadcast to both halves
        f2 nxh[3], nxl[3], nvh[3], nvl[3], h2, dtr;
    };
    struct JP {   // one j-pair
        f2 xh[3], m, xl[3], vh[3], vl[3];
    };
    template <int NP>
    static __device__ __forceinline__ void load_j(JP &s, const unsigned char *st, int pl)
    {
        const ulonglong2 *q = reinterpret_cast<const ulonglong2 *>(st);
        const ulonglong2 a = q[pl], b = q[NP + pl], c = q[2 * NP + pl], d = q[3 * NP + pl];
        const ulonglong2 e = q[4 * NP + pl], f = q[5 * NP + pl], g = q[6 * NP + pl];
        s.xh[0] = a.x; s.xh[1] = a.y; s.xh[2] = b.x; s.m = b.y;
        s.xl[0] = c.x; s.xl[1] = c.y; s.xl[2] = d.x;
        s.vh[0] = d.y; s.vh[1] = e.x; s.vh[2] = e.y;
        s.vl[0] = f.x; s.vl[1] = f.y; s.vl[2] = g.x;
    }
    // Replace the invalid half(s) of a pair by a zero-mass particle far away.
    static __device__ __forceinline__ void mask(JP &s, bool va, bool vb)
    {
        auto fix = [&](f2 &v, float far) {
            float a, b;
            up(v, a, b);
            v = pk(va ? a : far, vb ? b : far);
        };
        for (int c = 0; c < 3; c++) {
            fix(s.xh[c], FAR_F);
            fix(s.xl[c], 0.f);
            fix(s.vh[c], 0.f);
            fix(s.vl[c], 0.f);
        }
        fix(s.m, 0.f);
    }
    static __device__ __forceinline__ void set_i(IB &ib, const JSet &soa, int64_t slot, float h2, float dtr,
                                                 const Frame2 &)
    {
        FormMixed::IS a;
        FormMixed::clear_i(a);
        if (slot >= 0) FormMixed::load_i(a, soa, slot);
        for (int c = 0; c < 3; c++) {
            ib.nxh[c] = bc(-a.xh[c]);
            ib.nxl[c] = bc(-a.xl[c]);
            ib.nvh[c] = bc(-a.vh[c]);
            ib.nvl[c] = bc(-a.vl[c]);
        }
        ib.h2 = bc(h2);
        ib.dtr = bc(dtr);
    }
    static __device__ __forceinline__ void diffs(const IB &i, const JP &j, f2 &dx, f2 &dy, f2 &dz, f2 &ux, f2 &uy,
                                                 f2 &uz)
    {
        dx = add2(add2(j.xh[0], i.nxh[0]), add2(j.xl[0], i.nxl[0]));
        dy = add2(add2(j.xh[1], i.nxh[1]), add2(j.xl[1], i.nxl[1]));
        dz = add2(add2(j.xh[2], i.nxh[2]), add2(j.xl[2], i.nxl[2]));
        ux = add2(add2(j.vh[0], i.nvh[0]), add2(j.vl[0], i.nvl[0]));
        uy = add2(add2(j.vh[1], i.nvh[1]), add2(j.vl[1], i.nvl[1]));
        uz = add2(add2(j.vh[2], i.nvh[2]), add2(j.vl[2], i.nvl[2]));
    }
    template <bool VC, bool POT>
    static __device__ __forceinline__ void pair(const IB &i, const JP &j, Acc2 &a, bool &fa, bool &fb)
    {
        f2 dx, dy, dz, ux, uy, uz;
        diffs(i, j, dx, dy, dz, ux, uy, uz);
        tail2<VC, POT>(i.h2, i.dtr, j.m, dx, dy, dz, ux, uy, uz, a, fa, fb);
    }
};

// Two-float positions, FP32 velocities: the first five streams of the
// two-float layout (q0..q4: xh, m, xl, vh).  x_j - x_i keeps the two-float
// difference of PairMixed; v_j - v_i is the FP32 difference of the rounded
// velocities, whose absolute error u (|v_i| + |v_j|) stays at the level of
// the other FP32 roundings of a pair term when the velocities are given in
// a frame where they are of the order of the velocity dispersion (the
// centre-of-mass frame of an N-body integration).  Positions get no such
// help: a cluster far from the origin, or a close pair, needs the low parts.
struct PairMixedX {
    static constexpr int NS = 5;
    struct IB {
        f2 nxh[3], nxl[3], nv[3], h2, dtr;
    };
    struct JP {
        f2 xh[3], m, xl[3], v[3];
    };
    template <int NP>
    static __device__ __forceinline__ void load_j(JP &s, const unsigned char *st, int pl)
    {
        const ulonglong2 *q = reinterpret_cast<const ulonglong2 *>(st);
        const ulonglong2 a = q[pl], b = q[NP + pl], c = q[2 * NP + pl], d = q[3 * NP + pl];
        const ulonglong2 e = q[4 * NP + pl];
        s.xh[0] = a.x; s.xh[1] = a.y; s.xh[2] = b.x; s.m = b.y;
        s.xl[0] = c.x; s.xl[1] = c.y; s.xl[2] = d.x;
        s.v[0] = d.y; s.v[1] = e.x; s.v[2] = e.y;
    }
    static __device__ __forceinline__ void mask(JP &s, bool va, bool vb)
    {
        auto fix = [&](f2 &v, float far) {
            float a, b;
            up(v, a, b);
            v = pk(va ? a : far, vb ? b : far);
        };
        for (int c = 0; c < 3; c++) {
            fix(s.xh[c], FAR_F);
            fix(s.xl[c], 0.f);
            fix(s.v[c], 0.f);
        }
        fix(s.m, 0.f);
    }
    static __device__ __forceinline__ void set_i(IB &ib, const JSet &soa, int64_t slot, float h2, float dtr,
                                                 const Frame2 &)
    {
        FormMixed::IS a;
        FormMixed::clear_i(a);
        if (slot >= 0) FormMixed::load_i(a, soa, slot);
        for (int c = 0; c < 3; c++) {
            ib.nxh[c] = bc(-a.xh[c]);
            ib.nxl[c] = bc(-a.xl[c]);
            ib.nv[c] = bc(-a.vh[c]);
        }
        ib.h2 = bc(h2);
        ib.dtr = bc(dtr);
    }
    static __device__ __forceinline__ void diffs(const IB &i, const JP &j, f2 &dx, f2 &dy, f2 &dz, f2 &ux, f2 &uy,
                                                 f2 &uz)
    {
        dx = add2(add2(j.xh[0], i.nxh[0]), add2(j.xl[0], i.nxl[0]));
        dy = add2(add2(j.xh[1], i.nxh[1]), add2(j.xl[1], i.nxl[1]));
        dz = add2(add2(j.xh[2], i.nxh[2]), add2(j.xl[2], i.nxl[2]));
        ux = add2(j.v[0], i.nv[0]);
        uy = add2(j.v[1], i.nv[1]);
        uz = add2(j.v[2], i.nv[2]);
    }
    template <bool VC, bool POT>
    static __device__ __forceinline__ void pair(const IB &i, const JP &j, Acc2 &a, bool &fa, bool &fb)
    {
        f2 dx, dy, dz, ux, uy, uz;
        diffs(i, j, dx, dy, dz, ux, uy, uz);
        tail2<VC, POT>(i.h2, i.dtr, j.m, dx, dy, dz, ux, uy, uz, a, fa, fb);
    }
};

// Plain FP32 form, pair-interleaved: 4 float4 streams per j-pair
//   q0 (x_a, x_b, y_a, y_b)  q1 (z_a, z_b, m_a, m_b)  q2 (vx_a, vx_b, vy_a, vy_b)  q3 (vz_a, vz_b, 0, 0)
struct PairFP32 {
    static constexpr int NS = 4;
    struct IB {
        f2 nx[3], nv[3], h2, dtr;
    };
    struct JP {
        f2 x[3], m, v[3];
    };
    template <int NP>
    static __device__ __forceinline__ void load_j(JP &s, const unsigned char *st, int pl)
    {
        const ulonglong2 *q = reinterpret_cast<const ulonglong2 *>(st);
        const ulonglong2 a = q[pl], b = q[NP + pl], c = q[2 * NP + pl], d = q[3 * NP + pl];
        s.x[0] = a.x; s.x[1] = a.y; s.x[2] = b.x; s.m = b.y;
        s.v[0] = c.x; s.v[1] = c.y; s.v[2] = d.x;
    }
    static __device__ __forceinline__ void mask(JP &s, bool va, bool vb)
    {
        auto fix = [&](f2 &v, float far) {
            float a, b;
            up(v, a, b);
            v = pk(va ? a : far, vb ? b : far);
        };
        for (int c = 0; c < 3; c++) {
            fix(s.x[c], FAR_F);
            fix(s.v[c], 0.f);
        }
        fix(s.m, 0.f);
    }
    static __device__ __forceinline__ void set_i(IB &ib, const JSet &soa, int64_t slot, float h2, float dtr,
                                                 const Frame2 &)
    {
        FormFP32::IS a;
        FormFP32::clear_i(a);
        if (slot >= 0) FormFP32::load_i(a, soa, slot);
        for (int c = 0; c < 3; c++) {
            ib.nx[c] = bc(-a.x[c]);
            ib.nv[c] = bc(-a.v[c]);
        }
        ib.h2 = bc(h2);
        ib.dtr = bc(dtr);
    }
    template <bool VC, bool POT>
    static __device__ __forceinline__ void pair(const IB &i, const JP &j, Acc2 &a, bool &fa, bool &fb)
    {
        tail2<VC, POT>(i.h2, i.dtr, j.m, add2(j.x[0], i.nx[0]), add2(j.x[1], i.nx[1]), add2(j.x[2], i.nx[2]),
                       add2(j.v[0], i.nv[0]), add2(j.v[1], i.nv[1]), add2(j.v[2], i.nv[2]), a, fa, fb);
    }
};

// Framed two-float form.  A tile of the pair-interleaved two-float stream is
// rewritten in place (frame_tile) as FP32 offsets from the block's frame
// centre c, in the FP32 stream layout; the i-values are c - x_i, formed in
// two-float and rounded once.  A pair term is then the FP32 form's
// arithmetic: dx = (x_j - c) + (c - x_i), one add per component.
struct FramedMixed : PairFP32 {
    static __device__ __forceinline__ void set_i(IB &ib, const JSet &soa, int64_t slot, float h2, float dtr,
                                                 const Frame2 &fr)
    {
        FormMixed::IS a;
        FormMixed::clear_i(a);
        if (slot >= 0) FormMixed::load_i(a, soa, slot);
        for (int c = 0; c < 3; c++) {
            ib.nx[c] = bc((fr.xh[c] - a.xh[c]) + (fr.xl[c] - a.xl[c]));
            ib.nv[c] = bc((fr.vh[c] - a.vh[c]) + (fr.vl[c] - a.vl[c]));
        }
        ib.h2 = bc(h2);
        ib.dtr = bc(dtr);
    }
};

// Rewrite the j-pairs of a two-float tile (7 streams of NP float4) in place as
// FP32 offsets from the frame centre, in the FP32 layout (streams 0..3).  Each
// lane reads all seven float4 of its pairs before writing any of them.
template <int NP>
__device__ __forceinline__ void frame_tile(unsigned char *st, const Frame2 &fr, int lane)
{
    ulonglong2 *q = reinterpret_cast<ulonglong2 *>(st);
    f2 nxh[3], nxl[3], nvh[3], nvl[3];
    for (int c = 0; c < 3; c++) {
        nxh[c] = bc(-fr.xh[c]);
        nxl[c] = bc(-fr.xl[c]);
        nvh[c] = bc(-fr.vh[c]);
        nvl[c] = bc(-fr.vl[c]);
    }
    for (int pl = lane; pl < NP; pl += 32) {
        const ulonglong2 a = q[pl], b = q[NP + pl], c = q[2 * NP + pl], d = q[3 * NP + pl];
        const ulonglong2 e = q[4 * NP + pl], f = q[5 * NP + pl], g = q[6 * NP + pl];
        ulonglong2 o0, o1, o2, o3;
        o0.x = add2(add2(a.x, nxh[0]), add2(c.x, nxl[0]));
        o0.y = add2(add2(a.y, nxh[1]), add2(c.y, nxl[1]));
        o1.x = add2(add2(b.x, nxh[2]), add2(d.x, nxl[2]));
        o1.y = b.y;   // masses
        o2.x = add2(add2(d.y, nvh[0]), add2(f.x, nvl[0]));
        o2.y = add2(add2(e.x, nvh[1]), add2(f.y, nvl[1]));
        o3.x = add2(add2(e.y, nvh[2]), add2(g.x, nvl[2]));
        o3.y = 0ull;
        q[pl] = o0;
        q[NP + pl] = o1;
        q[2 * NP + pl] = o2;
        q[3 * NP + pl] = o3;
    }
}

// List target of one i-particle of a warp (shared memory; the running count
// stays in a register).
struct __align__(16) ListRec {
    int32_t *row;   // its list row (final, or its j-split's partial row)
    int32_t gi;     // its own index in the j-range (-1: no particle), skipped as self
    int32_t pad;
};

// Marker for the kernels without frames.
struct NoFrame {};

template <class T>
struct FormTag {
    using type = T;
};

template <class Fm, int W, int I, int JT, int NST_>
struct PairLayout {
    static constexpr int NST = NST_;                               // stages of the j-tile ring
    static constexpr int NP = JT / 2;                              // j-pairs per tile
    static constexpr int STAGE = Fm::NS * 16 * NP;
    static constexpr int STAGES = 256;                             // barriers and counters first
    // float-float totals: one (hi, lo) float2 per (warp, i, component, lane)
    static constexpr int TOT = STAGES + NST * STAGE;
    __host__ __device__ static constexpr int tot_bytes(bool pot) { return W * I * (pot ? 7 : 6) * 32 * 8; }
    // per (warp, i): the list row and the i's own j-index
    __host__ __device__ static constexpr int rec(bool pot) { return TOT + tot_bytes(pot); }
    __host__ __device__ static constexpr int desc(bool pot) { return rec(pot) + W * I * 16; }
    __host__ __device__ static constexpr int bytes(bool pot)
    {
        return desc(pot) + W * static_cast<int>(sizeof(ClusterDesc));
    }
};

template <class Fm, int W, int I, int JT, int NST>
constexpr int pair_smem_bytes(bool pot)
{
    return PairLayout<Fm, W, I, JT, NST>::bytes(pot);
}

// Copy the pair-interleaved tile at cursor c into ring slot seq % NST.  The
// j-range starts at an even slot (checked on the host), so tile t covers
// j-pairs (jb + t*JT)/2 ... and a ragged tail copies ceil(count/2) pairs.
template <class Fm, int JT, int NST>
__device__ __forceinline__ void issue_pairs(const RegfParams &p, const TileCursor &c, uint32_t seq, uint64_t *full,
                                            unsigned char *stages)
{
    constexpr int NP = JT / 2;
    constexpr int STAGE = Fm::NS * 16 * NP;
    const int s = seq % NST;
    uint64_t *b = &full[s];
    unsigned char *st = stages + s * STAGE;
    const int count = min(JT, c.nj - c.tile * JT);
    const uint32_t bytes = static_cast<uint32_t>((count + 1) / 2) * 16;
    mbar_arrive_expect_tx(b, bytes * Fm::NS + p.extra_tx);
    const int64_t first = (c.jb + static_cast<int64_t>(c.tile) * JT) / 2;
#pragma unroll
    for (int k = 0; k < Fm::NS; k++)
        tma_bulk_g2s(st + k * NP * 16, static_cast<const unsigned char *>(p.js.s[k]) + first * 16, bytes, b);
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Fm: the exact (per-pair two-float or FP32) form; Ff: NoFrame, or the framed
// form used for the work items whose block of active particles is compact.
template <class Fm, class Ff, int W, int I, int JT, int NSTAGE, int U, int FLAGS, int MINB>
__global__ void __launch_bounds__(W * 32, MINB) regf3_kernel(const RegfParams p)
{
    static_assert(NSTAGE <= 9, "ring barriers, counters and the look-ahead cursor share the first 256 bytes");
    static_assert((JT / 64) % U == 0, "a tile holds a whole number of steps");
    using L = PairLayout<Fm, W, I, JT, NSTAGE>;
    constexpr bool FRAMED = !std::is_same<Ff, NoFrame>::value;
    constexpr bool VC = (FLAGS & 1) != 0;
    constexpr bool POT = (FLAGS & 2) != 0;
    constexpr int NC = POT ? 7 : 6;
    constexpr int NST = L::NST;
    constexpr int NP = L::NP;
    constexpr int STEPS = NP / 32;                                // a step covers 64 j
    // Steps (128 j per lane) per FP32 partial of the jerk, and of the force and
    // potential: the jerk sum cancels far more (|J| can be ~1e-3 of the sum of
    // its terms' magnitudes), so its partials are folded into the float-float
    // totals more often.
    constexpr int FOLD_STEPS_J = 64, FOLD_STEPS_F = 256;
    constexpr int FOLD_TILES_J = STEPS >= FOLD_STEPS_J ? 1 : FOLD_STEPS_J / STEPS;
    constexpr int FOLD_TILES_F = STEPS >= FOLD_STEPS_F ? 1 : FOLD_STEPS_F / STEPS;
    using Bits = typename std::conditional<2 * STEPS <= 32, uint32_t, uint64_t>::type;
    static_assert(2 * STEPS <= 64, "two neighbour flags per unit of a tile fit 64 bits");

    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);          // tile landed (TMA)
    uint64_t *xf = full + NST;                                    // tile rewritten in frame coordinates
    int *rel = reinterpret_cast<int *>(xf + NST);                 // warps done with the stage
    int *claim = rel + NST;                                       // warps that reached the stage
    // the ring's look-ahead: the tile that the next refill copies (only the
    // thread that refills a stage reads and advances it)
    TileCursor *s_la = reinterpret_cast<TileCursor *>(claim + NST);
    unsigned char *stages = smem + L::STAGES;
    float2 *s_tot = reinterpret_cast<float2 *>(smem + L::TOT);
    ListRec *s_rec = reinterpret_cast<ListRec *>(smem + L::rec(POT));
    ClusterDesc *s_d = reinterpret_cast<ClusterDesc *>(smem + L::desc(POT));

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < NST; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&xf[s], 1);
            rel[s] = 0;
            claim[s] = 0;
        }
        fence_mbar_init();
        TileCursor c0;
        c0.item = blockIdx.x;
        cursor_set(p, c0);
        for (int q = 0; q < NST && c0.item < p.n_items; ++q) {
            issue_pairs<Fm, JT, NST>(p, c0, q, full, stages);
            cursor_next(p, c0);
        }
        *s_la = c0;   // look-ahead = sequence NST
    }
    __syncthreads();

    uint32_t g = 0;
    bool aborted = false;
    float2 *mytot = s_tot + warp * I * NC * 32 + lane;   // + (i * NC + comp) * 32: (hi, lo)
    ListRec *myrec = s_rec + warp * I;
    ClusterDesc &d = s_d[warp];

    // One work item (i-block ib, j-split sp) with the pair arithmetic of form P.
    auto run_item = [&](auto form_tag, int ib, int sp, bool framed_item, const Frame2 &fr) {
        using P = typename decltype(form_tag)::type;
        using JP = typename P::JP;
        using IB = typename P::IB;
        const int tb = sp * d.tiles_per_split;
        const int te = min(tb + d.tiles_per_split, d.n_tiles);
        IB ipart[I];
        Acc2 acc[I];
        int oidx[I];                 // output row of each i (its position in act)
        int cnt[I];                  // neighbours found so far (the same in every lane)
        const int i0 = (ib * W + warp) * I;
#pragma unroll
        for (int k = 0; k < I; k++) {
            const int slot_i = i0 + k;
            int idx = -1;
            int64_t slot = -1;
            float h2v = -1.f, dtv = 0.f;
            int gi = -1;
            if (slot_i < d.n_act) {
                idx = d.perm ? d.perm[slot_i] : slot_i;
                const int a = d.act[idx];
                const double hv = d.h[idx];
                if (a >= 0 && a < d.n_j && hv >= 0.0 && hv <= DBL_MAX) {
                    gi = a;
                    slot = d.j_begin + a;
                    h2v = fmaxf(__double2float_rn(hv * hv), FLT_MIN);   // self (r2 = 0) is inside
                    dtv = (VC && d.dtr) ? __double2float_rn(d.dtr[idx]) : 0.f;
                } else if (lane == 0) {
                    atomicOr(p.status, DEV_BAD_INPUT);
                }
            }
            oidx[k] = gi >= 0 ? idx : -1;
            if (lane == 0) {
                ListRec r;
                r.row = gi < 0 ? nullptr
                               : d.n_split == 1 ? d.list + static_cast<int64_t>(idx) * d.cap
                                                : d.plist + (static_cast<int64_t>(sp) * d.n_act + idx) * d.cap;
                r.gi = gi;
                r.pad = 0;
                myrec[k] = r;
            }
            cnt[k] = 0;
            P::set_i(ipart[k], p.soa, slot, h2v, dtv, fr);
            for (int c = 0; c < 3; c++) acc[k].f[c] = acc[k].j[c] = 0ull;
            acc[k].p = 0ull;
            for (int c = 0; c < NC; c++) mytot[(k * NC + c) * 32] = make_float2(0.f, 0.f);
        }
        __syncwarp();

        for (int t = tb; t < te; ++t, ++g) {
            const int s = g % NST;
            if (!mbar_wait_bounded(&full[s], (g / NST) & 1, p.wait_ns)) { aborted = true; break; }
            unsigned char *st = stages + s * L::STAGE;
            if constexpr (FRAMED) {
                // the first warp to reach the tile rewrites it in frame coordinates
                int first = 0;
                if (lane == 0) first = atomicAdd(&claim[s], 1) == 0;
                first = __shfl_sync(0xffffffffu, first, 0);
                if (first) {
                    if (framed_item) frame_tile<NP>(st, fr, lane);
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&xf[s]);
                } else if (!mbar_wait_bounded(&xf[s], (g / NST) & 1, p.wait_ns)) {
                    aborted = true;
                    break;
                }
            }
            const int jt0 = t * JT;
            const int count = min(JT, d.n_j - jt0);

            // Pair terms of the whole tile: U j-pairs per lane per step (U * 64
            // consecutive j for the warp), no branch; the neighbour flags of
            // unit (pair-step) k*U+u and i-particle q go to bits 2(k*U+u) (first
            // particle of the lane's pair) and 2(k*U+u)+1 (second) of bits[q].
            Bits bits[I];
#pragma unroll
            for (int q = 0; q < I; q++) bits[q] = 0u;
            auto step = [&](int k, auto tail_c) {
                constexpr bool tail = decltype(tail_c)::value;
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int pl = (k * U + u) * 32 + lane;
                    JP jp;
                    P::template load_j<NP>(jp, st, pl);
                    if (tail) P::mask(jp, 2 * pl < count, 2 * pl + 1 < count);
#pragma unroll
                    for (int q = 0; q < I; q++) {
                        bool fa, fb;
                        P::template pair<VC, POT>(ipart[q], jp, acc[q], fa, fb);
                        const int b = 2 * (k * U + u);
                        bits[q] |= (fa ? Bits(1) << b : Bits(0)) | (fb ? Bits(2) << b : Bits(0));
                    }
                }
            };
            if (count == JT) {
#pragma unroll
                for (int k = 0; k < STEPS / U; ++k) step(k, std::false_type{});
            } else {
                // the last tile of a j-range: only the steps that hold a j
                const int whole = count / (U * 64);   // steps with no padding
#pragma unroll 1
                for (int k = 0; k < whole; ++k) step(k, std::false_type{});
                if (count - whole * U * 64 > 0) step(whole, std::true_type{});
            }
            // count this warp out of the stage (the list pass below reads only the
            // flags); the last one refills it NST tiles ahead
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                if (atomicAdd(&rel[s], 1) == W - 1) {
                    // every warp has left the stage, the refiller of the previous
                    // one among them: its cursor update is visible after the fence
                    __threadfence_block();
                    rel[s] = 0;
                    if constexpr (FRAMED) {
                        claim[s] = 0;
                        fence_proxy_async_smem();   // the stage was written through the generic proxy
                    }
                    TileCursor la = *s_la;
                    if (la.item < p.n_items) {
                        issue_pairs<Fm, JT, NST>(p, la, g + NST, full, stages);
                        cursor_next(p, la);
                        *s_la = la;
                    }
                }
            }

            // Neighbour lists of the tile, in ascending j: for each i-particle,
            // the flagged units in order; within a unit the order is (lane, half).
            {
                const int cap = d.cap;
                const unsigned lt = lanemask_lt();
#pragma unroll
                for (int q = 0; q < I; q++) {
                    const Bits b = bits[q] & ~self_bit<Bits>(myrec[q].gi - jt0, JT, lane);   // the particle itself
                    Bits todo = reduce_or_bits(b);
                    if (!todo) continue;
                    int32_t *const row = myrec[q].row;
                    int n = cnt[q];
                    while (todo) {
                        const int unit = lowest_bit(todo) >> 1;
                        todo &= ~(Bits(3) << (2 * unit));
                        const int ja = jt0 + 2 * (unit * 32 + lane);
                        const bool xa = (b >> (2 * unit)) & 1u, xb = (b >> (2 * unit + 1)) & 1u;
                        const unsigned ma = __ballot_sync(0xffffffffu, xa);
                        const unsigned mb = __ballot_sync(0xffffffffu, xb);
                        const int pa = n + __popc(ma & lt) + __popc(mb & lt);
                        const int pb = pa + (xa ? 1 : 0);
                        if (xa && pa < cap) row[pa] = ja;
                        if (xb && pb < cap) row[pb] = ja + 1;
                        n += __popc(ma) + __popc(mb);
                    }
                    cnt[q] = n;
                }
            }

            auto fold = [&](int c) {
#pragma unroll
                for (int q = 0; q < I; q++) {
                    f2 &part = c < 3 ? acc[q].f[c] : (c < 6 ? acc[q].j[c - 3] : acc[q].p);
                    float2 *slot = mytot + (q * NC + c) * 32;
                    float2 v = *slot;
                    float pa, pb;
                    up(part, pa, pb);
                    ff_add(v.x, v.y, pa + pb);   // the two halves' partials first, then TwoSum
                    *slot = v;
                    part = 0ull;
                }
            };
            const bool last = t + 1 == te;
            if ((t - tb + 1) % FOLD_TILES_J == 0 || last) {
#pragma unroll
                for (int c = 3; c < 6; c++) fold(c);
            }
            if ((t - tb + 1) % FOLD_TILES_F == 0 || last) {
#pragma unroll
                for (int c = 0; c < 3; c++) fold(c);
                if (POT) fold(6);
            }
        }
        if (aborted) return;

        // reduce the float-float totals over the 32 lanes, then write
        float th[8 * I], tl[8 * I];
#pragma unroll
        for (int q = 0; q < I; q++) {
#pragma unroll
            for (int c = 0; c < 8; c++) {
                const float2 v = c < NC ? mytot[(q * NC + c) * 32] : make_float2(0.f, 0.f);
                th[8 * q + c] = v.x;
                tl[8 * q + c] = v.y;
            }
        }
        ff_reduce_scatter<8 * I>(th, tl);
        write_item_rs<I, NC>(d, sp, th[0], tl[0], oidx, p.status);
#pragma unroll
        for (int q = 0; q < I; q++) {
            const int64_t i = oidx[q];
            if (lane == 0 && row_ok(d, sp, i, p.status)) {
                const int nq = cnt[q];
                if (d.n_split == 1) {
                    d.nnb[i] = nq;
                    d.ovf[i] = nq > d.cap ? 1 : 0;
                } else {
                    d.pcnt[static_cast<int64_t>(sp) * d.n_act + i] = nq;
                }
            }
        }
        __syncwarp();
    };

    for (int64_t pos = blockIdx.x; pos < p.n_items && !aborted; pos += gridDim.x) {
        int cl, ib, sp;
        if (!item_at(p, pos, cl, ib, sp)) continue;
        if (lane == 0) d = p.work ? p.table[cl] : p.d0;
        __syncwarp();
        Frame2 fr{};
        bool framed_item = false;
        if constexpr (FRAMED) {
            if (d.frames) {
                const FrameRec f = d.frames[ib];
                framed_item = f.compact != 0;
                for (int c = 0; c < 3; c++) {
                    fr.xh[c] = __double2float_rn(f.cx[c]);
                    fr.xl[c] = __double2float_rn(f.cx[c] - static_cast<double>(fr.xh[c]));
                    fr.vh[c] = __double2float_rn(f.cv[c]);
                    fr.vl[c] = __double2float_rn(f.cv[c] - static_cast<double>(fr.vh[c]));
                }
            }
            if (framed_item) run_item(FormTag<Ff>{}, ib, sp, true, fr);
            else run_item(FormTag<Fm>{}, ib, sp, false, fr);
        } else {
            run_item(FormTag<Fm>{}, ib, sp, false, fr);
        }
    }

    if (aborted && lane == 0) {
        atomicOr(p.status, DEV_TIMEOUT);
        for (uint32_t q = g; q < g + NST; ++q) mbar_wait_bounded(&full[q % NST], (q / NST) & 1, p.wait_ns);
    }
}

}  // namespace nb
