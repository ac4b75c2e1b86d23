// Device-side definitions shared by the kernels of libnbreg: work-item
// descriptors, the asynchronous-copy (TMA bulk) and mbarrier primitives, the
// float-float helpers and the device status bits.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace nb {

struct FrameRec;   // nb_sort.cuh

// Device status bits (OR-ed into the context's status word).
enum : int {
    DEV_TIMEOUT = 1,    // a bounded wait on a copy ran out
    DEV_BAD_INPUT = 2,  // an active index or a radius was invalid
    DEV_BOUNDS = 4,     // a bounds check of the library's own output indexing failed
};

// Predicted j-set of one precision form: base pointers of its streams.
struct JSet {
    const void *s[8];
};

// One cluster of a regular-force launch, as the kernels see it.
struct ClusterDesc {
    int64_t j_begin;       // first slot of the cluster in the predicted set
    int32_t n_j;           // j-particles
    int32_t n_act;         // active particles
    int32_t cap;           // list capacity
    int32_t n_split;       // j-splits (work items per i-block)
    int32_t tiles_per_split;
    int32_t n_tiles;       // ceil(n_j / jtile)
    int32_t n_iblk;        // ceil(n_act / (warps * ipw))
    int32_t pad0;
    int64_t item_begin;    // first work item of this cluster
    const int32_t *act;
    const double *h;
    const double *dtr;
    double *F, *J, *pot;
    int32_t *nnb;
    int32_t *list;
    uint8_t *ovf;
    // split scratch (n_split > 1): 8 doubles (F3, J3, pot, -) per (split, i),
    // a count per (split, i) and `cap` list slots per (split, i)
    double *pF;
    int32_t *pcnt;
    int32_t *plist;
    // framed kernels: processing order of the active set (slot -> position in
    // act) and one frame per block of W*I consecutive slots; both nullptr otherwise
    const int32_t *perm;
    const FrameRec *frames;
};

struct RegfParams {
    JSet js;                      // streams the j-tiles are copied from
    JSet soa;                     // per-particle (SoA) streams of the same form, for the i-values
    ClusterDesc d0;               // used when work == nullptr (a single call)
    const ClusterDesc *table;     // device table of clusters (batched launch)
    // batched launch: the work list, one (cluster, i-block, j-split, 0) per
    // slot (cluster < 0: an empty slot); CTA b takes slots b, b + grid, ...
    const int4 *work;
    int32_t n_clusters;
    int64_t n_items;              // work items (single call) or slots of the work list
    int *status;
    uint64_t wait_ns;             // bound of every mbarrier wait
    uint32_t extra_tx;            // test hook: bytes expected beyond the copies (0 normally);
                                  // > 0 makes every copy wait run out, exercising the time-out path
};

// Work item at slot `pos` of the launch: its cluster's table index, i-block
// and j-split.  A batched launch reads them from the plan's work list (one
// 16-byte load; false for an empty slot), a single call derives them from
// the slot number (i-block major, j-split minor).
__device__ __forceinline__ bool item_at(const RegfParams &p, int64_t pos, int &cl, int &ib, int &sp)
{
    if (p.work) {
        const int4 r = p.work[pos];
        cl = r.x;
        ib = r.y;
        sp = r.z;
        return cl >= 0;
    }
    cl = 0;
    ib = static_cast<int>(pos / p.d0.n_split);
    sp = static_cast<int>(pos - static_cast<int64_t>(ib) * p.d0.n_split);
    return true;
}

// ------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Bulk asynchronous copy global -> shared (the untiled TMA path), completing
// `bytes` transactions on `bar`.  dst, src 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void tma_bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                             uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// As mbar_try_wait, but the waiting threads may be suspended (issuing
// nothing) for up to `hint_ns` nanoseconds until the phase completes.
__device__ __forceinline__ bool mbar_try_wait_suspend(uint64_t *bar, uint32_t parity, uint32_t hint_ns)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of `bar`, giving up after `limit_ns` nanoseconds.
// Returns false on time-out (the caller reports it and stops).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (true) {
        if (mbar_try_wait_suspend(bar, parity, 20000u)) return true;   // sleep up to 20 us per try
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// ---------------------------------------------------------- float-float

// hi + lo += p with the rounding error of the high part kept (Knuth's TwoSum).
__device__ __forceinline__ void ff_add(float &hi, float &lo, float p)
{
    const float s = __fadd_rn(hi, p);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    hi = s;
    lo = __fadd_rn(lo, e);
}

// (hi, lo) += (h2, l2), result renormalised so that |lo| <= ulp(hi)/2.
__device__ __forceinline__ void ff_add_ff(float &hi, float &lo, float h2, float l2)
{
    const float s = __fadd_rn(hi, h2);
    const float bp = __fsub_rn(s, hi);
    float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(h2, bp));
    e = __fadd_rn(e, __fadd_rn(lo, l2));
    hi = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}

// End of a work item in the float forms.  After the float-float totals of the
// warp's I particles are reduced over the lanes (every lane then holds all of
// them), lane 8q + c (mod 32; round (8q + c) / 32) keeps component c (F 0..2,
// J 3..5, potential 6) of particle q with ff_keep, and write_item_ff stores it:
// in FP64 to the outputs when the call is not split, else as the float-float
// pair itself into the (split, particle) slot of the split scratch
// (components NC..6 as zeros), which the merge sums in float-float.  So one
// FP64 conversion per lane replaces one per component on every lane: the FP64
// pipe (about two lanes per SM per clock on GB300) would otherwise hold every
// warp of the SM for ~1 us at the end of each item.
template <int I>
struct FFKeep {
    static constexpr int R = (8 * I + 31) / 32;   // rounds of 32 (particle, component) slots
    float h[R], l[R];
};

template <int I>
__device__ __forceinline__ void ff_keep(FFKeep<I> &k, int q, int c, float hi, float lo)
{
    const int slot = 8 * q + c;   // q, c are compile-time after unrolling
    if ((threadIdx.x & 31) == (slot & 31)) { k.h[slot >> 5] = hi; k.l[slot >> 5] = lo; }
}

// Bounds check of the end-of-item stores: output row i (-1 = no particle,
// skipped silently) of j-split sp.  Every stored index is in range by
// construction (rows come from positions < n_act of the active set, splits
// from the item number); a failure records DEV_BOUNDS in the status word and
// the store is skipped, so an indexing bug surfaces as a status, not as a
// stray write.
__device__ __forceinline__ bool row_ok(const ClusterDesc &d, int sp, int64_t i, int *status)
{
    if (i < 0) return false;
    if (i < d.n_act && sp >= 0 && sp < d.n_split) return true;
    atomicOr(status, DEV_BOUNDS);
    return false;
}

template <int I, int NC>
__device__ __forceinline__ void write_item_ff(const ClusterDesc &d, int sp, const FFKeep<I> &k, const int (&oi)[I],
                                              int *status)
{
    static_assert(NC <= 7, "F, J and the potential");
    const int lane = threadIdx.x & 31;
    const int c = lane & 7;
#pragma unroll
    for (int r = 0; r < FFKeep<I>::R; r++) {
        const int q = 4 * r + (lane >> 3);
        int i = -1;
#pragma unroll
        for (int qq = 4 * r; qq < I && qq < 4 * r + 4; qq++)
            if (qq == q) i = oi[qq];
        if (q >= I || c >= 7 || !row_ok(d, sp, i, status)) continue;
        const int64_t ii = i;
        const float h = c < NC ? k.h[r] : 0.f, l = c < NC ? k.l[r] : 0.f;
        if (d.n_split == 1) {
            if (c >= NC) continue;
            const double v = static_cast<double>(h) + static_cast<double>(l);
            if (c < 3) d.F[3 * ii + c] = v;
            else if (c < 6) d.J[3 * ii + c - 3] = v;
            else if (d.pot) d.pot[ii] = v;
        } else {
            float2 *slot = reinterpret_cast<float2 *>(d.pF + (static_cast<int64_t>(sp) * d.n_act + ii) * 8);
            slot[c] = make_float2(h, l);
        }
    }
}

// Float-float reduce-scatter of V = 8 I values over the 32 lanes of a warp
// (h[v], l[v]: this lane's part of value v = 8 q + c, component c of particle
// q as above, zero for c >= NC).  Each of the first log2 V rounds halves what
// a lane carries: of lanes L and L ^ b (b = 16, 8, ...), the one with bit b
// set keeps the upper half of the values and the other the lower half, and
// each adds the half it receives; the remaining rounds add the partner's
// whole value.  Lane L ends with the total of value L >> (5 - log2 V) in
// h[0], l[0], with the same bits on every lane that holds it (TwoSum's error
// term is exact in either operand order).  For V = 16 that is 32 shuffles and
// 16 float-float additions per lane, against 120 and 60 for a butterfly of
// every value, and the lanes are left holding one value each for the stores.
template <int V>
__device__ __forceinline__ void ff_reduce_scatter(float (&h)[V], float (&l)[V])
{
    static_assert(V == 8 || V == 16 || V == 32, "8 components of 1, 2 or 4 particles");
    constexpr int LV = V == 8 ? 3 : (V == 16 ? 4 : 5);
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int r = 0; r < LV; r++) {
        const int m = V >> (r + 1), b = 16 >> r;
        const bool up = (lane & b) != 0;
#pragma unroll
        for (int k = 0; k < m; k++) {
            const float sh = up ? h[k] : h[k + m], sl = up ? l[k] : l[k + m];
            float kh = up ? h[k + m] : h[k], kl = up ? l[k + m] : l[k];
            const float rh = __shfl_xor_sync(0xffffffffu, sh, b);
            const float rl = __shfl_xor_sync(0xffffffffu, sl, b);
            ff_add_ff(kh, kl, rh, rl);
            h[k] = kh;
            l[k] = kl;
        }
    }
#pragma unroll
    for (int b = 16 >> LV; b >= 1; b >>= 1) {
        const float rh = __shfl_xor_sync(0xffffffffu, h[0], b);
        const float rl = __shfl_xor_sync(0xffffffffu, l[0], b);
        ff_add_ff(h[0], l[0], rh, rl);
    }
}

// The stores of write_item_ff after ff_reduce_scatter: the first lane of
// each value's lane group stores it.
template <int I, int NC>
__device__ __forceinline__ void write_item_rs(const ClusterDesc &d, int sp, float h, float l, const int (&oi)[I],
                                              int *status)
{
    static_assert(NC <= 7, "F, J and the potential");
    constexpr int SH = I == 1 ? 2 : (I == 2 ? 1 : 0);   // 5 - log2(8 I)
    const int lane = threadIdx.x & 31;
    if (lane & ((1 << SH) - 1)) return;
    const int v = lane >> SH, q = v >> 3, c = v & 7;
    int i = -1;
#pragma unroll
    for (int qq = 0; qq < I; qq++)
        if (qq == q) i = oi[qq];
    if (c >= 7 || !row_ok(d, sp, i, status)) return;
    const int64_t ii = i;
    if (d.n_split == 1) {
        if (c >= NC) return;
        const double x = static_cast<double>(h) + static_cast<double>(l);
        if (c < 3) d.F[3 * ii + c] = x;
        else if (c < 6) d.J[3 * ii + c - 3] = x;
        else if (d.pot) d.pot[ii] = x;
    } else {
        float2 *slot = reinterpret_cast<float2 *>(d.pF + (static_cast<int64_t>(sp) * d.n_act + ii) * 8);
        slot[c] = c < NC ? make_float2(h, l) : make_float2(0.f, 0.f);
    }
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace nb
