// Thread-block-cluster variant of the j-pair regular-force kernel for small
// calls (tiling packed = 20): the pair arithmetic of nb_regf3.cuh (Sec. 3.3
// step (vi), criterion of Sec. 3.2), with the cross-split reduction and list
// gathering of Sec. 3.4 done inside the launch.
//
// A call with few active particles splits its j-range over many CTAs to
// occupy the GPU, and the persistent kernels then need split partials in
// global memory and a second (merge) launch.  Here the S j-splits of one
// block of active particles are the S CTAs of one thread-block cluster: each
// CTA stages its j-tiles in shared memory with asynchronous 16-byte copies
// (cp.async: every copy of a tile in flight at once, the next tile's issued
// before the current tile's list pass), runs the pair terms and the
// warp-wide list compaction,
// and leaves its float-float partial sums, its neighbour counts and its list
// segments in its own shared memory.  After a cluster barrier, warp w of CTA
// r reduces particle q = r + S w (+ S W, ...) of the block: it reads the S
// partials and counts from the CTAs' shared memory through the distributed
// shared-memory window (mapa + ld.shared::cluster), sums them in split order
// in float-float, and copies the list segments in split order (ascending j)
// into the caller's list row.  A second cluster barrier keeps every CTA's
// shared memory alive until its peers have read it.  There are no waits
// other than each thread's wait for its own copies and the block and cluster
// barriers, which every thread of every CTA reaches unconditionally.
#pragma once

#include "nb_regf3.cuh"

namespace nb {

__device__ __forceinline__ uint32_t cluster_ctarank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Barrier over every thread of every CTA of the cluster; the release /
// acquire pair orders the shared-memory writes before it with the
// distributed reads after it.
__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Address of the same shared-memory object in the CTA of rank `rank`.
__device__ __forceinline__ uint32_t peer_addr(const void *local, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(local)), "r"(rank));
    return r;
}
__device__ __forceinline__ float2 ld_peer_f2(uint32_t addr)
{
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
    return v;
}
// 16-byte asynchronous copy global -> shared, and the wait for all of this
// thread's copies (a wait on the thread's own copies, not on another thread).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
}

__device__ __forceinline__ int ld_peer_s32(uint32_t addr)
{
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

// Shared-memory layout of one CTA (cap: the call's list capacity).
template <class Fm, int W, int I, int JT>
struct ClLayout {
    static constexpr int NP = JT / 2;
    static constexpr int IPB = W * I;
    static constexpr int TILE = Fm::NS * 16 * NP;
    __host__ __device__ static constexpr int tot(bool pot) { return TILE; }
    __host__ __device__ static constexpr int part(bool pot) { return TILE + W * I * (pot ? 7 : 6) * 32 * 8; }
    __host__ __device__ static constexpr int cnt(bool pot) { return part(pot) + IPB * 8 * 8; }
    __host__ __device__ static constexpr int list(bool pot) { return cnt(pot) + IPB * 4; }
    __host__ __device__ static constexpr int bytes(bool pot, int cap) { return list(pot) + IPB * cap * 4; }
};

template <class Fm, int W, int I, int JT, int FLAGS>
__global__ void __launch_bounds__(W * 32, 1) regf_cl_kernel(const RegfParams p)
{
    using L = ClLayout<Fm, W, I, JT>;
    using JP = typename Fm::JP;
    using IB = typename Fm::IB;
    constexpr bool VC = (FLAGS & 1) != 0;
    constexpr bool POT = (FLAGS & 2) != 0;
    constexpr int NC = POT ? 7 : 6;
    constexpr int NP = L::NP;
    constexpr int STEPS = NP / 32;
    constexpr int IPB = L::IPB;
    constexpr int FOLD_STEPS_J = 64, FOLD_STEPS_F = 256;        // as in regf3_kernel
    constexpr int FOLD_TILES_J = STEPS >= FOLD_STEPS_J ? 1 : FOLD_STEPS_J / STEPS;
    constexpr int FOLD_TILES_F = STEPS >= FOLD_STEPS_F ? 1 : FOLD_STEPS_F / STEPS;
    using Bits = typename std::conditional<2 * STEPS <= 32, uint32_t, uint64_t>::type;

    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *tile = smem;
    float2 *s_tot = reinterpret_cast<float2 *>(smem + L::tot(POT));
    float2 *s_part = reinterpret_cast<float2 *>(smem + L::part(POT));   // [IPB][8] float-float partials
    int *s_cnt = reinterpret_cast<int *>(smem + L::cnt(POT));           // [IPB] neighbour counts
    int32_t *s_list = reinterpret_cast<int32_t *>(smem + L::list(POT)); // [IPB][cap] list segments

    const ClusterDesc &d = p.d0;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int S = d.n_split;                          // the cluster's size
    const int sp = static_cast<int>(cluster_ctarank());
    const int ib = static_cast<int>(blockIdx.x) / S;
    const int tb = sp * d.tiles_per_split;
    const int te = min(tb + d.tiles_per_split, d.n_tiles);
    const int cap = d.cap;

    // stage tile t: ceil(count / 2) j-pairs of each pair-interleaved stream
    auto issue_tile = [&](int t) {
        const int jt0 = t * JT;
        const int npairs = (min(JT, d.n_j - jt0) + 1) / 2;
        const int64_t first = (d.j_begin + static_cast<int64_t>(jt0)) / 2;
        for (int k = 0; k < Fm::NS; k++) {
            const float4 *src = static_cast<const float4 *>(p.js.s[k]) + first;
            const uint32_t dst = smem_u32(tile) + static_cast<uint32_t>(k * NP * 16);
            for (int e = tid; e < npairs; e += W * 32) cp_async16(dst + 16u * e, src + e);
        }
    };
    if (tb < te) issue_tile(tb);   // in flight while the i-values load

    // i-values of this warp's particles (block ib, slots warp * I + q)
    IB ipart[I];
    Acc2 acc[I];
    int gi[I], cnt[I];
    float2 *mytot = s_tot + warp * I * NC * 32 + lane;
    const Frame2 fr{};
#pragma unroll
    for (int q = 0; q < I; q++) {
        const int slot_i = ib * IPB + warp * I + q;
        int64_t slot = -1;
        float h2v = -1.f, dtv = 0.f;
        gi[q] = -1;
        if (slot_i < d.n_act) {
            const int a = d.act[slot_i];
            const double hv = d.h[slot_i];
            if (a >= 0 && a < d.n_j && hv >= 0.0 && hv <= DBL_MAX) {
                gi[q] = a;
                slot = d.j_begin + a;
                h2v = fmaxf(__double2float_rn(hv * hv), FLT_MIN);   // self (r2 = 0) is inside
                dtv = (VC && d.dtr) ? __double2float_rn(d.dtr[slot_i]) : 0.f;
            } else if (lane == 0 && sp == 0) {
                atomicOr(p.status, DEV_BAD_INPUT);
            }
        }
        Fm::set_i(ipart[q], p.soa, slot, h2v, dtv, fr);
        for (int c = 0; c < 3; c++) acc[q].f[c] = acc[q].j[c] = 0ull;
        acc[q].p = 0ull;
        cnt[q] = 0;
        for (int c = 0; c < NC; c++) mytot[(q * NC + c) * 32] = make_float2(0.f, 0.f);
    }

    for (int t = tb; t < te; ++t) {
        const int jt0 = t * JT;
        const int count = min(JT, d.n_j - jt0);
        cp_async_wait_all();
        __syncthreads();   // tile t has landed for every thread

        Bits bits[I];
#pragma unroll
        for (int q = 0; q < I; q++) bits[q] = 0u;
        auto step = [&](int k, auto tail_c) {
            constexpr bool tail = decltype(tail_c)::value;
            const int pl = k * 32 + lane;
            JP jp;
            Fm::template load_j<NP>(jp, tile, pl);
            if (tail) Fm::mask(jp, 2 * pl < count, 2 * pl + 1 < count);
#pragma unroll
            for (int q = 0; q < I; q++) {
                bool fa, fb;
                Fm::template pair<VC, POT>(ipart[q], jp, acc[q], fa, fb);
                bits[q] |= (fa ? Bits(1) << (2 * k) : Bits(0)) | (fb ? Bits(2) << (2 * k) : Bits(0));
            }
        };
        if (count == JT) {
#pragma unroll
            for (int k = 0; k < STEPS; ++k) step(k, std::false_type{});
        } else {
            // the last tile of the j-range: only the steps that hold a j
            const int whole = count >> 6;   // steps of 64 j with no padding
#pragma unroll 1
            for (int k = 0; k < whole; ++k) step(k, std::false_type{});
            if (count & 63) step(whole, std::true_type{});
        }
        __syncthreads();   // every warp is done with tile t
        if (t + 1 < te) issue_tile(t + 1);

        // neighbour lists of the tile into this CTA's segments, ascending j
        const unsigned lt = lanemask_lt();
#pragma unroll
        for (int q = 0; q < I; q++) {
            const Bits b = bits[q] & ~self_bit<Bits>(gi[q] - jt0, JT, lane);   // the particle itself
            Bits todo = reduce_or_bits(b);
            int32_t *row = s_list + (warp * I + q) * cap;
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

        auto fold = [&](int c) {
#pragma unroll
            for (int q = 0; q < I; q++) {
                f2 &part = c < 3 ? acc[q].f[c] : (c < 6 ? acc[q].j[c - 3] : acc[q].p);
                float2 *slot = mytot + (q * NC + c) * 32;
                float2 v = *slot;
                float pa, pb;
                up(part, pa, pb);
                ff_add(v.x, v.y, pa + pb);
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

    // this split's float-float partials (component c of particle q at
    // s_part[(warp I + q) 8 + c], zero for c >= NC) and counts, in shared memory
    {
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
        constexpr int SH = I == 1 ? 2 : (I == 2 ? 1 : 0);   // lane L holds value L >> SH
        if ((lane & ((1 << SH) - 1)) == 0) s_part[warp * I * 8 + (lane >> SH)] = make_float2(th[0], tl[0]);
#pragma unroll
        for (int q = 0; q < I; q++)
            if (lane == 0) s_cnt[warp * I + q] = cnt[q];
    }

    cluster_barrier();

    // reduction over the cluster's splits: warp w of CTA sp takes particles
    // sp + S w, sp + S (w + W), ... of the block
    for (int ql = sp + S * warp; ql < IPB; ql += S * W) {
        const int slot_i = ib * IPB + ql;
        if (slot_i >= d.n_act) continue;
        float sh[8] = {0, 0, 0, 0, 0, 0, 0, 0}, sl[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int c_s = 0;
        if (lane < S) {
            c_s = ld_peer_s32(peer_addr(s_cnt + ql, lane));
            const uint32_t pa = peer_addr(s_part + ql * 8, lane);
#pragma unroll
            for (int c = 0; c < 7; c++) {
                const float2 v = ld_peer_f2(pa + 8 * c);
                sh[c] = v.x;
                sl[c] = v.y;
            }
        }
        ff_reduce_scatter<8>(sh, sl);   // lane L: component L >> 2 summed over the splits
        // list segments in split order: exclusive prefix of the counts
        int incl = c_s;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int excl = incl - c_s;
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        const int ncopy = min(total, cap);
        int32_t *to = d.list + static_cast<int64_t>(slot_i) * cap;
        for (int r = 0; r < ncopy; r += 32) {
            const int e = r + lane;
            int src = 0;
            for (int stp = 16; stp > 0; stp >>= 1) {
                const int ex = __shfl_sync(0xffffffffu, excl, src + stp);
                if (ex <= e) src += stp;
            }
            const int off = e - __shfl_sync(0xffffffffu, excl, src);
            // off < min(count of split src, cap) and src < S by construction
            if (e < ncopy) {
                if (off >= 0 && off < cap && src < S)
                    to[e] = ld_peer_s32(peer_addr(s_list + ql * cap + off, src));
                else
                    atomicOr(p.status, DEV_BOUNDS);
            }
        }
        const double v = static_cast<double>(sh[0]) + static_cast<double>(sl[0]);
        const int64_t i = slot_i;
        const int a = d.act[slot_i];
        const double hv = d.h[slot_i];
        const int c = lane >> 2;
        if (a >= 0 && a < d.n_j && hv >= 0.0 && hv <= DBL_MAX) {
            if ((lane & 3) == 0) {
                if (c < 3) d.F[3 * i + c] = v;
                else if (c < 6) d.J[3 * i + c - 3] = v;
                else if (c == 6 && POT && d.pot) d.pot[i] = v;
            }
            if (lane == 0) {
                d.nnb[i] = total;
                d.ovf[i] = total > cap ? 1 : 0;
            }
        }
    }

    cluster_barrier();   // the peers have read this CTA's shared memory
}

}  // namespace nb
