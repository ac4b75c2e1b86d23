// j-pair regular-force kernel with separate list warps (tiling packed = 5 + NL).
//
// The same pair arithmetic as regf3_kernel (Sec. 3.3 step (vi), criterion of
// Sec. 3.2), but the CTA's warps are specialised: WC compute warps run the
// pair terms of their i-particles over the j-tiles (the TMA ring, the FP32
// partials and the float-float totals of regf3_kernel) and hand each tile's
// neighbour flags to shared memory; NL list warps turn
// those flags into the ascending neighbour lists (ballot + popc, as in
// regf3_kernel) and write the counts.  The compute warps thus never stop for
// the list compaction, which in regf3_kernel keeps the FMA pipe idle while
// every warp of a scheduler compacts its lists.  Flags pass through an FR-slot
// ring: a compute warp waits until the list warps have emptied the slot it
// fills (flag_empty), the list warps wait until every compute warp has filled
// it (flag_full).  The j-tile ring is refilled by list warp 0: a compute warp
// only arrives on the stage's `empty` barrier when its pair terms are done,
// and list warp 0 waits for that barrier and issues the copy NST tiles ahead.
// All waits are bounded.
#pragma once

#include "nb_regf3.cuh"

namespace nb {

template <class Fm, int WC, int NL, int I, int JT, int NST_, int FR_ = 2>
struct WsLayout {
    static constexpr int W = WC + NL;
    static constexpr int NST = NST_;
    static constexpr int FR = FR_;
    static constexpr int NP = JT / 2;
    static constexpr int STEPS = NP / 32;
    static constexpr int FLB = 2 * STEPS <= 32 ? 4 : 8;           // bytes of one lane's flags of a tile
    static constexpr int STAGE = Fm::NS * 16 * NP;
    static constexpr int HDR = 256;                               // barriers and counters
    static constexpr int TOT = HDR + NST * STAGE;
    __host__ __device__ static constexpr int tot_bytes(bool pot) { return WC * I * (pot ? 7 : 6) * 32 * 8; }
    __host__ __device__ static constexpr int fl(bool pot) { return TOT + tot_bytes(pot); }
    __host__ __device__ static constexpr int desc(bool pot) { return fl(pot) + FR * WC * I * 32 * FLB; }
    __host__ __device__ static constexpr int bytes(bool pot)
    {
        return desc(pot) + W * static_cast<int>(sizeof(ClusterDesc));
    }
};

template <class Fm, int WC, int NL, int I, int JT, int NST, int FR = 2>
constexpr int ws_smem_bytes(bool pot)
{
    return WsLayout<Fm, WC, NL, I, JT, NST, FR>::bytes(pot);
}

// FR_: slots of the flag ring between the compute and the list warps (a
// compute warp is at most FR_ tiles ahead of the list warps).
template <class Fm, int WC, int NL, int I, int JT, int NSTAGE, int FLAGS, int FR_ = 2>
__global__ void __launch_bounds__((WC + NL) * 32, 1) regf3ws_kernel(const RegfParams p)
{
    static_assert(WC % NL == 0, "each list warp serves the same number of compute warps");
    using L = WsLayout<Fm, WC, NL, I, JT, NSTAGE, FR_>;
    using P = Fm;
    using JP = typename P::JP;
    using IB = typename P::IB;
    constexpr bool VC = (FLAGS & 1) != 0;
    constexpr bool POT = (FLAGS & 2) != 0;
    constexpr int NC = POT ? 7 : 6;
    constexpr int NST = L::NST;
    constexpr int FR = L::FR;
    constexpr int NP = L::NP;
    constexpr int STEPS = L::STEPS;
    constexpr int FOLD_STEPS_J = 64, FOLD_STEPS_F = 256;          // as in regf3_kernel
    constexpr int FOLD_TILES_J = STEPS >= FOLD_STEPS_J ? 1 : FOLD_STEPS_J / STEPS;
    constexpr int FOLD_TILES_F = STEPS >= FOLD_STEPS_F ? 1 : FOLD_STEPS_F / STEPS;
    using Bits = typename std::conditional<2 * STEPS <= 32, uint32_t, uint64_t>::type;
    static_assert(sizeof(Bits) == L::FLB, "flag words");
    static_assert(16 * NST + 16 * FR <= L::HDR, "barriers fit the header");
    constexpr int NCW = WC / NL;                                  // compute warps per list warp
    static_assert(I * NC <= 32, "one lane per (particle, component) at the end of an item");

    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);          // tile landed (TMA)
    uint64_t *empty = full + NST;                                 // every compute warp is done with the stage
    uint64_t *flag_full = empty + NST;                            // every compute warp wrote its flags
    uint64_t *flag_empty = flag_full + FR;                        // every list warp read them
    unsigned char *stages = smem + L::HDR;
    float2 *s_tot = reinterpret_cast<float2 *>(smem + L::TOT);
    Bits *s_fl = reinterpret_cast<Bits *>(smem + L::fl(POT));     // [FR][WC][I][32]
    ClusterDesc *s_d = reinterpret_cast<ClusterDesc *>(smem + L::desc(POT));

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool lister = warp >= WC;
    TileCursor la;
    la.item = blockIdx.x;
    cursor_set(p, la);
    if (tid == 0) {
        for (int s = 0; s < NST; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], WC);
        }
        for (int f = 0; f < FR; f++) {
            mbar_init(&flag_full[f], WC);
            mbar_init(&flag_empty[f], NL);
        }
        fence_mbar_init();
        TileCursor c0 = la;
        for (int q = 0; q < NST && c0.item < p.n_items; ++q) {
            issue_pairs<Fm, JT, NST>(p, c0, q, full, stages);
            cursor_next(p, c0);
        }
    }
    uint32_t issued = 0;   // tiles issued so far (the prologue's, then list warp 0's)
    for (int q = 0; q < NST && la.item < p.n_items; ++q, ++issued) cursor_next(p, la);   // look-ahead = sequence NST
    __syncthreads();

    uint32_t g = 0;
    bool aborted = false;
    ClusterDesc &d = s_d[warp];

    if (!lister) {
        // ------------------------------------------------------------ compute warps
        float2 *mytot = s_tot + warp * I * NC * 32 + lane;   // + (i * NC + comp) * 32: (hi, lo)
        for (int64_t pos = blockIdx.x; pos < p.n_items && !aborted; pos += gridDim.x) {
            int cl, ib, sp;
            if (!item_at(p, pos, cl, ib, sp)) continue;
            if (lane == 0) d = p.work ? p.table[cl] : p.d0;
            __syncwarp();
            const int tb = sp * d.tiles_per_split;
            const int te = min(tb + d.tiles_per_split, d.n_tiles);
            IB ipart[I];
            Acc2 acc[I];
            int oidx[I];
            const Frame2 fr{};
#pragma unroll
            for (int k = 0; k < I; k++) {
                const int slot_i = (ib * WC + warp) * I + k;
                int idx = -1;
                int64_t slot = -1;
                float h2v = -1.f, dtv = 0.f;
                if (slot_i < d.n_act) {
                    const int a = d.act[slot_i];
                    const double hv = d.h[slot_i];
                    if (a >= 0 && a < d.n_j && hv >= 0.0 && hv <= DBL_MAX) {
                        idx = slot_i;
                        slot = d.j_begin + a;
                        h2v = fmaxf(__double2float_rn(hv * hv), FLT_MIN);   // self (r2 = 0) is inside
                        dtv = (VC && d.dtr) ? __double2float_rn(d.dtr[slot_i]) : 0.f;
                    } else if (lane == 0) {
                        atomicOr(p.status, DEV_BAD_INPUT);
                    }
                }
                oidx[k] = idx;
                P::set_i(ipart[k], p.soa, slot, h2v, dtv, fr);
                for (int c = 0; c < 3; c++) acc[k].f[c] = acc[k].j[c] = 0ull;
                acc[k].p = 0ull;
                for (int c = 0; c < NC; c++) mytot[(k * NC + c) * 32] = make_float2(0.f, 0.f);
            }
            __syncwarp();

            for (int t = tb; t < te; ++t, ++g) {
                const int s = g % NST;
                if (!mbar_wait_bounded(&full[s], (g / NST) & 1, p.wait_ns)) { aborted = true; break; }
                const unsigned char *st = stages + s * L::STAGE;
                const int count = min(JT, d.n_j - t * JT);
                Bits bits[I];
#pragma unroll
                for (int q = 0; q < I; q++) bits[q] = 0u;
                auto step = [&](int k, auto tail_c) {
                    constexpr bool tail = decltype(tail_c)::value;
                    const int pl = k * 32 + lane;
                    JP jp;
                    P::template load_j<NP>(jp, st, pl);
                    if (tail) P::mask(jp, 2 * pl < count, 2 * pl + 1 < count);
#pragma unroll
                    for (int q = 0; q < I; q++) {
                        bool fa, fb;
                        P::template pair<VC, POT>(ipart[q], jp, acc[q], fa, fb);
                        bits[q] |= (fa ? Bits(1) << (2 * k) : Bits(0)) | (fb ? Bits(2) << (2 * k) : Bits(0));
                    }
                };
                if (count == JT) {
#pragma unroll
                    for (int k = 0; k < STEPS; ++k) step(k, std::false_type{});
                } else {
                    // the last tile of a j-range: only the steps that hold a j
                    const int whole = count >> 6;   // steps of 64 j with no padding
#pragma unroll 1
                    for (int k = 0; k < whole; ++k) step(k, std::false_type{});
                    if (count & 63) step(whole, std::true_type{});
                }
                // this warp is done with the stage; list warp 0 refills it
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
                // hand the flags to the list warps
                const uint32_t fs = g % FR;
                if (!mbar_wait_bounded(&flag_empty[fs], ((g / FR) & 1) ^ 1, p.wait_ns)) { aborted = true; break; }
#pragma unroll
                for (int q = 0; q < I; q++) s_fl[((fs * WC + warp) * I + q) * 32 + lane] = bits[q];
                __syncwarp();
                if (lane == 0) mbar_arrive(&flag_full[fs]);

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
            if (aborted) break;

            // Reduce the float-float totals over the 32 lanes (a butterfly per
            // value), then write F, J and the potential; the list warps write
            // the counts and lists.  The two-float forms keep component c of
            // particle q on lane q NC + c after the butterflies: one FP64
            // conversion per lane instead of one per value on every lane (the
            // FP64 pipe is narrow; 0.6 % of the step at N = n_act = 131072, 2.4 %
            // at 16384 active, 2.5 % for the exact pair form), and a split slot
            // takes the float-float pair itself.  The plain FP32 form keeps the
            // all-lane conversion, which left its register allocation without
            // spills (the per-lane store cost that form 2.6 %).  A reduce-scatter
            // of the values, cheaper in shuffles, made the pair-term loop slower.
            if constexpr (!std::is_same<Fm, PairFP32>::value) {
                float vh = 0.f, vl = 0.f;
#pragma unroll
                for (int q = 0; q < I; q++) {
#pragma unroll
                    for (int c = 0; c < NC; c++) {
                        const float2 v = mytot[(q * NC + c) * 32];
                        float hi = v.x, lo = v.y;
                        for (int o = 16; o > 0; o >>= 1) {
                            const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
                            const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
                            ff_add_ff(hi, lo, h2, l2);
                        }
                        if (lane == q * NC + c) { vh = hi; vl = lo; }
                    }
                }
                const int q = lane / NC, c = lane - (lane / NC) * NC;
                int64_t i = -1;
#pragma unroll
                for (int qq = 0; qq < I; qq++)
                    if (qq == q) i = oidx[qq];
                if (lane < I * NC && row_ok(d, sp, i, p.status)) {
                    if (d.n_split == 1) {
                        const double v = static_cast<double>(vh) + static_cast<double>(vl);
                        if (c < 3) d.F[3 * i + c] = v;
                        else if (c < 6) d.J[3 * i + c - 3] = v;
                        else if (d.pot) d.pot[i] = v;
                    } else {
                        float2 *o8 = reinterpret_cast<float2 *>(d.pF + (static_cast<int64_t>(sp) * d.n_act + i) * 8);
                        o8[c] = make_float2(vh, vl);
                        if (c == NC - 1)
                            for (int cc = NC; cc < 7; cc++) o8[cc] = make_float2(0.f, 0.f);
                    }
                }
            } else {
#pragma unroll
                for (int q = 0; q < I; q++) {
                    double out[7] = {0, 0, 0, 0, 0, 0, 0};
                    for (int c = 0; c < NC; c++) {
                        const float2 v = mytot[(q * NC + c) * 32];
                        float hi = v.x, lo = v.y;
                        for (int o = 16; o > 0; o >>= 1) {
                            const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
                            const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
                            ff_add_ff(hi, lo, h2, l2);
                        }
                        out[c] = static_cast<double>(hi) + static_cast<double>(lo);
                    }
                    const int64_t i = oidx[q];
                    if (lane == 0 && row_ok(d, sp, i, p.status)) {
                        if (d.n_split == 1) {
                            for (int c = 0; c < 3; c++) { d.F[3 * i + c] = out[c]; d.J[3 * i + c] = out[3 + c]; }
                            if (POT && d.pot) d.pot[i] = out[6];
                        } else {
                            // the split slot holds float-float pairs, as written by write_item_ff
                            float2 *o8 = reinterpret_cast<float2 *>(d.pF + (static_cast<int64_t>(sp) * d.n_act + i) * 8);
                            for (int c = 0; c < 7; c++) {
                                const float h = c < NC ? __double2float_rn(out[c]) : 0.f;
                                const float l = c < NC ? __double2float_rn(out[c] - static_cast<double>(h)) : 0.f;
                                o8[c] = make_float2(h, l);
                            }
                        }
                    }
                }
            }
            __syncwarp();
        }
        if (aborted && lane == 0) atomicOr(p.status, DEV_TIMEOUT);
    } else {
        // --------------------------------------------------------------- list warps
        const int lw = warp - WC;   // serves compute warps lw, lw + NL, lw + 2 NL, ...
        for (int64_t pos = blockIdx.x; pos < p.n_items && !aborted; pos += gridDim.x) {
            int cl, ib, sp;
            if (!item_at(p, pos, cl, ib, sp)) continue;
            if (lane == 0) d = p.work ? p.table[cl] : p.d0;
            __syncwarp();
            const int tb = sp * d.tiles_per_split;
            const int te = min(tb + d.tiles_per_split, d.n_tiles);
            int32_t *row[NCW][I];
            int gi[NCW][I], cnt[NCW][I], oidx[NCW][I];
#pragma unroll
            for (int c = 0; c < NCW; c++) {
#pragma unroll
                for (int q = 0; q < I; q++) {
                    const int slot_i = (ib * WC + lw + NL * c) * I + q;
                    int a = -1, idx = -1;
                    if (slot_i < d.n_act) {
                        const int aa = d.act[slot_i];
                        const double hv = d.h[slot_i];
                        if (aa >= 0 && aa < d.n_j && hv >= 0.0 && hv <= DBL_MAX) { a = aa; idx = slot_i; }
                    }
                    gi[c][q] = a;
                    oidx[c][q] = idx;
                    cnt[c][q] = 0;
                    row[c][q] = idx < 0 ? nullptr
                                        : d.n_split == 1
                                              ? d.list + static_cast<int64_t>(idx) * d.cap
                                              : d.plist + (static_cast<int64_t>(sp) * d.n_act + idx) * d.cap;
                }
            }
            for (int t = tb; t < te; ++t, ++g) {
                const uint32_t fs = g % FR;
                if (!mbar_wait_bounded(&flag_full[fs], (g / FR) & 1, p.wait_ns)) { aborted = true; break; }
                if (lw == 0) {   // refill the stage of tile g with tile g + NST once every compute warp left it
                    if (lane == 0) {
                        const int s = g % NST;
                        if (!mbar_wait_bounded(&empty[s], (g / NST) & 1, p.wait_ns)) {
                            aborted = true;
                        } else if (la.item < p.n_items) {
                            issue_pairs<Fm, JT, NST>(p, la, g + NST, full, stages);
                            issued = g + NST + 1;
                        }
                    }
                    aborted = __shfl_sync(0xffffffffu, aborted, 0);
                    if (aborted) break;
                    cursor_next(p, la);
                }
                const int jt0 = t * JT;
#pragma unroll
                for (int c = 0; c < NCW; c++) {
#pragma unroll
                    for (int q = 0; q < I; q++) {
                        const Bits b = s_fl[((fs * WC + lw + NL * c) * I + q) * 32 + lane];
                        Bits todo = reduce_or_bits(b);
                        while (todo) {
                            const int unit = lowest_bit(todo) >> 1;
                            todo &= ~(Bits(3) << (2 * unit));
                            const int ja = jt0 + 2 * (unit * 32 + lane);
                            const bool fa = (b >> (2 * unit)) & 1u, fb = (b >> (2 * unit + 1)) & 1u;
                            const bool xa = fa && ja != gi[c][q], xb = fb && ja + 1 != gi[c][q];
                            const unsigned ma = __ballot_sync(0xffffffffu, xa);
                            const unsigned mb = __ballot_sync(0xffffffffu, xb);
                            const unsigned lt = lanemask_lt();
                            const int pa = cnt[c][q] + __popc(ma & lt) + __popc(mb & lt);
                            const int pb = pa + (xa ? 1 : 0);
                            if (xa && pa < d.cap) row[c][q][pa] = ja;
                            if (xb && pb < d.cap) row[c][q][pb] = ja + 1;
                            cnt[c][q] += __popc(ma) + __popc(mb);
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&flag_empty[fs]);
            }
            if (aborted) break;
            if (lane == 0) {
#pragma unroll
                for (int c = 0; c < NCW; c++) {
#pragma unroll
                    for (int q = 0; q < I; q++) {
                        const int64_t i = oidx[c][q];
                        if (!row_ok(d, sp, i, p.status)) continue;
                        if (d.n_split == 1) {
                            d.nnb[i] = cnt[c][q];
                            d.ovf[i] = cnt[c][q] > d.cap ? 1 : 0;
                        } else {
                            d.pcnt[static_cast<int64_t>(sp) * d.n_act + i] = cnt[c][q];
                        }
                    }
                }
            }
            __syncwarp();
        }
        if (aborted && lane == 0) {
            atomicOr(p.status, DEV_TIMEOUT);
            // let the copies this CTA issued land before its shared memory goes away
            if (lw == 0)
                for (uint32_t q = issued > NST ? issued - NST : 0; q < issued; ++q)
                    mbar_wait_bounded(&full[q % NST], (q / NST) & 1, p.wait_ns);
        }
    }
}

}  // namespace nb
