// f32x2 building blocks of the packed regular-force kernel (nb_regf3.cuh):
// Blackwell's add/sub/mul/fma.rn.f32x2 on two FP32 values held in a 64-bit
// register pair, the shared pair-term tail (r^2, R.V, neighbour test of
// Sec. 3.2, 1/r, force and jerk of Sec. 3.3 step (vi)), and the cursor that
// walks a CTA's sequence of j-tiles across work items.
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

// Warp-wide OR and lowest set bit of the per-lane neighbour flags of a tile.
__device__ __forceinline__ uint32_t reduce_or_bits(uint32_t b) { return __reduce_or_sync(0xffffffffu, b); }
__device__ __forceinline__ uint64_t reduce_or_bits(uint64_t b)
{
    const uint32_t lo = __reduce_or_sync(0xffffffffu, static_cast<uint32_t>(b));
    const uint32_t hi = __reduce_or_sync(0xffffffffu, static_cast<uint32_t>(b >> 32));
    return (static_cast<uint64_t>(hi) << 32) | lo;
}
__device__ __forceinline__ int lowest_bit(uint32_t b) { return __ffs(b) - 1; }

// The flag bit of j-offset o within a tile of JT j (bit 2 u + h of lane L for
// o = 2 (32 u + L) + h), on the lane that holds it, else 0: a particle's own
// slot is flagged by the pair terms (r^2 = 0 < h^2) and cleared with this.
template <class Bits>
__device__ __forceinline__ Bits self_bit(int o, int jt, int lane)
{
    return (o >= 0 && o < jt && ((o >> 1) & 31) == lane) ? (Bits(1) << (2 * (o >> 6) + (o & 1))) : Bits(0);
}
__device__ __forceinline__ int lowest_bit(uint64_t b) { return __ffsll(static_cast<long long>(b)) - 1; }

// Position in the CTA's sequence of j-tiles: the slot of the work item, the
// tile in it, the item's tile end, and the j-range the copies read.
struct TileCursor {
    int64_t item;
    int64_t jb;
    int nj, tile, te;
};

__device__ __forceinline__ void cursor_set(const RegfParams &p, TileCursor &c)
{
    int cl = 0, ib = 0, sp = 0;
    for (; c.item < p.n_items; c.item += gridDim.x)   // the consumers skip the same empty slots
        if (item_at(p, c.item, cl, ib, sp)) break;
    if (c.item >= p.n_items) return;
    const ClusterDesc &d = p.work ? p.table[cl] : p.d0;
    c.jb = d.j_begin;
    c.nj = d.n_j;
    c.tile = sp * d.tiles_per_split;
    c.te = min(c.tile + d.tiles_per_split, d.n_tiles);
}

__device__ __forceinline__ void cursor_next(const RegfParams &p, TileCursor &c)
{
    if (++c.tile < c.te) return;
    c.item += gridDim.x;
    cursor_set(p, c);
}

}  // namespace nb
