// Host side of libnbreg: the C-ABI declared in include/nbreg.h.
//
// The context owns the predicted j-set (three stored forms, SoA float4 /
// double4 streams), the split scratch, a device status word and the host-step
// staging buffers.  A regular-force call is one persistent kernel launch over
// work items (i-block x j-split) plus, when the j-range is split, one merge
// launch; nothing is copied between host and device inside a call.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <queue>
#include <tuple>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "nb_aux.cuh"
#include "nb_irr.cuh"
#include "nb_sort.cuh"
#include "nbreg.h"

using nb::ClusterDesc;
using nb::KernelEntry;

namespace {

constexpr uint64_t kDefaultWaitNs = 4000000000ull;   // 4 s bound on every copy wait

struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
            changed = cudaSetDevice(dev) == cudaSuccess;
        }
    }
    ~DeviceGuard()
    {
        if (changed) cudaSetDevice(prev);
    }
};

struct Registry {
    std::vector<KernelEntry> all;
    std::vector<int> occ;        // resident CTAs per SM, per entry (-1 = not yet queried)
    std::mutex mu;
};

Registry &registry()
{
    static Registry r;
    static std::once_flag once;
    std::call_once(once, [] {
        int n = 0;
        const KernelEntry *e = nb::kernels_fp64(&n);
        r.all.insert(r.all.end(), e, e + n);
        e = nb::kernels_mixed(&n);
        r.all.insert(r.all.end(), e, e + n);
        e = nb::kernels_fp32(&n);
        r.all.insert(r.all.end(), e, e + n);
        r.occ.assign(r.all.size(), -1);
    });
    return r;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

struct nb_ctx {
    int device = 0;
    int64_t n_max = 0;
    int sm_count = 0;
    double4_32a *pos64 = nullptr, *vel64 = nullptr;
    float4 *mx_hi = nullptr, *mx_lo = nullptr, *mv_hi = nullptr, *mv_lo = nullptr;
    float4 *pos32 = nullptr, *vel32 = nullptr;
    float4 *pim[7] = {};   // pair-interleaved two-float streams, (n_max + 1) / 2 j-pairs each
    float4 *pif[4] = {};   // pair-interleaved FP32 streams
    int forms_valid = 0;
    int *d_status = nullptr;
    double *d_frame = nullptr;   // [3] frame velocity of the float forms (device)
    // Frame under which each predicted slot range holds its float forms:
    // begin -> (end, frame epoch), disjoint ranges.  Every prediction that
    // computes a new frame starts a new epoch; NB_KEEP_FRAME and nb_set_frame
    // keep / start one explicitly.
    std::map<int64_t, std::pair<int64_t, uint64_t>> frames;
    uint64_t epoch = 0, epochs = 0;
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    nb_kcfg cfg[3];
    bool cfg_set[3] = {false, false, false};
    std::map<uint64_t, nb_tuned> tuned;   // autotuner table, by size class
    int last_launches = 0;
    uint64_t wait_ns = kDefaultWaitNs;
    uint32_t extra_tx = 0;
    void *stage = nullptr;   // nb_step_host device staging
    size_t stage_bytes = 0;
    cudaStream_t copy_st = nullptr;    // nb_step_host: result copies of finished chunks
    cudaEvent_t chunk_ev[4] = {};      // a chunk's kernels are done
    cudaEvent_t copy_done = nullptr;   // every result copy is done
    void *sort = nullptr;    // spatial sort and frames of the framed kernel
    size_t sort_bytes = 0;
    int *last_compact = nullptr;   // device count of compact blocks of the last framed call
    int last_blocks = 0;
    std::string err;
};

struct nb_plan {
    nb_ctx *ctx = nullptr;
    int mode = 0;
    const KernelEntry *e = nullptr;
    int entry = -1;
    int grid = 0;
    int64_t n_items = 0;
    std::vector<ClusterDesc> descs;
    ClusterDesc *d_table = nullptr;
    int64_t n_slots = 0;                  // slots of the work list (grid x the most items of a CTA)
    int4 *d_work = nullptr;               // [n_slots] (cluster, i-block, j-split, 0); cluster -1: empty
    int n_merge = 0;
    int64_t merge_total = 0;
    int64_t *d_act_begin = nullptr;
    int32_t *d_cluster_of = nullptr;
    void *scratch = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<nb_cluster> clusters;   // the caller's cluster table (for re-tiling by the autotuner)
    nb_kcfg cfg{};                      // the tiling the plan runs (split: tiles per j-split, 0 = heuristic)
    int flags = 0;                      // union of the clusters' flags
    int64_t act_sum = 0, j_max = 0;
};

namespace {

int cuda_fail(nb_ctx *ctx, cudaError_t e, const char *what)
{
    if (ctx) ctx->err = std::string(what) + ": " + cudaGetErrorString(e);
    return NB_ERR_CUDA;
}

#define NB_CUDA(ctx, call)                                                   \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);           \
    } while (0)

int mode_forms(int mode) { return mode == NB_FP64 ? NB_FORM_FP64 : mode == NB_MIXED ? NB_FORM_MIXED : NB_FORM_FP32; }

nb_kcfg default_cfg(int mode)
{
    Registry &r = registry();
    for (const auto &e : r.all)
        if (e.mode == mode && e.flags == 0) return nb_kcfg{e.warps, e.ipw, e.jtile, 0, e.packed};
    return nb_kcfg{0, 0, 0, 0, 0};
}

// Size class of the autotuner: (mode, flags, floor(log2 n_act), floor(log2 n_j)).
int log2_floor(int64_t n)
{
    int c = 0;
    while (n > 1) { n >>= 1; ++c; }
    return c;
}
uint64_t tune_key(int mode, int flags, int act_class, int j_class)
{
    return static_cast<uint64_t>(mode) | static_cast<uint64_t>(flags) << 4 |
           static_cast<uint64_t>(act_class) << 8 | static_cast<uint64_t>(j_class) << 16;
}

// Flag bit of the tuned table's batched classes (plans), beside the velocity
// criterion (1) and potential (2) bits of a call.
constexpr int kBatchedClass = 4;

// Tiling code of the thread-block-cluster kernel (nb_regf_cl.cuh) and its
// largest cluster (non-portable size; every CTA of a cluster sits in one GPC).
constexpr int kClusterPacked = 20;
constexpr int kMaxClusterSplits = 16;

// Tiling of a call: the one chosen with nb_set_kernel_config, else the tuned
// one of the call's size class, else the mode's default.
nb_kcfg pick_cfg(const nb_ctx *ctx, int mode, int flags, int64_t n_act, int64_t n_j)
{
    if (ctx->cfg_set[mode]) return ctx->cfg[mode];
    const auto it = ctx->tuned.find(tune_key(mode, flags, log2_floor(n_act), log2_floor(n_j)));
    return it != ctx->tuned.end() ? it->second.cfg : default_cfg(mode);
}

// Index of the kernel for (mode, cfg, flags); falls back to the mode's default
// tiling when this tiling has no instantiation with those flags.
int find_entry(int mode, const nb_kcfg &cfg, int flags)
{
    Registry &r = registry();
    for (size_t i = 0; i < r.all.size(); i++) {
        const auto &e = r.all[i];
        if (e.mode == mode && e.flags == flags && e.warps == cfg.warps && e.ipw == cfg.ipw &&
            e.jtile == cfg.jtile && e.packed == cfg.packed)
            return static_cast<int>(i);
    }
    for (size_t i = 0; i < r.all.size(); i++)
        if (r.all[i].mode == mode && r.all[i].flags == flags) return static_cast<int>(i);
    return -1;
}

int entry_occupancy(nb_ctx *ctx, int idx, int *occ)
{
    Registry &r = registry();
    std::lock_guard<std::mutex> lock(r.mu);
    if (r.occ[idx] < 0) {
        const KernelEntry &e = r.all[idx];
        if (e.packed == kClusterPacked) {
            // its list segments grow with the call's cap: allow up to the opt-in limit
            int optin = 0;
            NB_CUDA(ctx, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
            NB_CUDA(ctx, cudaFuncSetAttribute(e.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
            NB_CUDA(ctx, cudaFuncSetAttribute(e.fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
            r.occ[idx] = 1;
            *occ = 1;
            return NB_OK;
        }
        NB_CUDA(ctx, cudaFuncSetAttribute(e.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, e.smem));
        int o = 0;
        NB_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, e.fn, e.warps * 32, e.smem));
        if (o < 1) {
            ctx->err = "kernel does not fit on a multiprocessor";
            return NB_ERR_UNSUPPORTED;
        }
        r.occ[idx] = o;
    }
    *occ = r.occ[idx];
    return NB_OK;
}

// Fill the tiling fields of one cluster descriptor.
// Active particles per i-block of a kernel entry (its list warps own none).
int iblock_size(const KernelEntry &e) { return (e.warps - e.lists) * e.ipw; }

void tile_cluster(const KernelEntry &e, int occ, int sm, const nb_kcfg *cfg, ClusterDesc &d)
{
    const int ipb = iblock_size(e);
    d.n_iblk = (d.n_act + ipb - 1) / ipb;
    d.n_tiles = static_cast<int32_t>((static_cast<int64_t>(d.n_j) + e.jtile - 1) / e.jtile);
    int tps;
    if (cfg && cfg->split > 0) {
        tps = cfg->split;
    } else if (e.packed == kClusterPacked) {
        // thread-block-cluster kernel: as many splits as fit one cluster
        tps = std::max(1, (d.n_tiles + kMaxClusterSplits - 1) / kMaxClusterSplits);
    } else if (e.packed < 2) {
        // scalar kernels: enough work items for ~4 resident CTAs' worth of
        // items per slot, but at least two tiles per item
        const int64_t slots = static_cast<int64_t>(sm) * occ;
        const int64_t want = std::max<int64_t>(1, (4 * slots + d.n_iblk - 1) / std::max(d.n_iblk, 1));
        tps = static_cast<int>(std::max<int64_t>(2, (d.n_tiles + want - 1) / want));
    } else {
        // Packed kernels.  The persistent grid deals the work items round-robin
        // to its resident CTAs, so a call takes about ceil(items / slots)
        // rounds of one item's time.  Choose the tiles per split that minimise
        // that, counting an item's fixed cost (particle loads, lane reduction,
        // conversion and stores: ~6 us, measured at N = 16384) as 1.5 tiles and
        // a split call's merge as a launch plus its reads of the partials
        // (about 2e7 bytes per tile time); on a tie, fewer splits.  The split
        // scratch stays under 1 GiB.
        const int64_t slots = std::max<int64_t>(1, static_cast<int64_t>(sm) * occ);
        double best = 0.0;
        tps = d.n_tiles;
        for (int t = d.n_tiles; t >= 1; --t) {
            const int64_t ns = (d.n_tiles + t - 1) / t;
            if (ns > 1 && ns * d.n_act * (72 + 4 * static_cast<int64_t>(d.cap)) > (int64_t(1) << 30)) continue;
            const int64_t rounds = (static_cast<int64_t>(d.n_iblk) * ns + slots - 1) / slots;
            const double merge = ns > 1 ? 1.5 + static_cast<double>(ns) * d.n_act * (64.0 + 2.0 * d.cap) / 2e7 : 0.0;
            const double cost = static_cast<double>(rounds) * (t + 1.5) + merge;
            if (t == d.n_tiles || cost < best - 1e-9) { best = cost; tps = t; }
        }
    }
    d.tiles_per_split = std::max(1, tps);
    d.n_split = d.n_tiles == 0 ? 1 : (d.n_tiles + d.tiles_per_split - 1) / d.tiles_per_split;
}

// Bytes of split scratch one cluster needs, and the carving of it (the
// thread-block-cluster kernel keeps its partials in shared memory).
size_t cluster_scratch(const ClusterDesc &d, int packed = 0)
{
    if (d.n_split <= 1 || packed == kClusterPacked) return 0;
    const size_t cells = static_cast<size_t>(d.n_split) * d.n_act;
    return align_up(cells * 8 * sizeof(double), 256) + align_up(cells * sizeof(int32_t), 256) +
           align_up(cells * static_cast<size_t>(d.cap) * sizeof(int32_t), 256);
}

void carve_scratch(ClusterDesc &d, char *base, int packed = 0)
{
    if (d.n_split <= 1 || packed == kClusterPacked) { d.pF = nullptr; d.pcnt = nullptr; d.plist = nullptr; return; }
    const size_t cells = static_cast<size_t>(d.n_split) * d.n_act;
    d.pF = reinterpret_cast<double *>(base);
    base += align_up(cells * 8 * sizeof(double), 256);
    d.pcnt = reinterpret_cast<int32_t *>(base);
    base += align_up(cells * sizeof(int32_t), 256);
    d.plist = reinterpret_cast<int32_t *>(base);
}

// Per-particle (SoA) streams of a form.
nb::JSet jset(const nb_ctx *c, int mode)
{
    nb::JSet js{};
    if (mode == NB_FP64) { js.s[0] = c->pos64; js.s[1] = c->vel64; }
    else if (mode == NB_MIXED) { js.s[0] = c->mx_hi; js.s[1] = c->mx_lo; js.s[2] = c->mv_hi; js.s[3] = c->mv_lo; }
    else { js.s[0] = c->pos32; js.s[1] = c->vel32; }
    return js;
}

// Streams the j-tiles of kernel entry e are copied from.
nb::JSet tile_streams(const nb_ctx *c, int mode, const KernelEntry &e)
{
    if (e.packed < 2) return jset(c, mode);
    nb::JSet js{};
    if (mode == NB_MIXED) for (int k = 0; k < 7; k++) js.s[k] = c->pim[k];
    else for (int k = 0; k < 4; k++) js.s[k] = c->pif[k];
    return js;
}

// The j-pair kernels read pairs (2P, 2P+1); a j-range starting at an odd
// slot is served by the first compiled kernel of another layout.
int layout_fallback(int mode, int idx, int flags)
{
    Registry &r = registry();
    for (size_t i = 0; i < r.all.size(); i++)
        if (r.all[i].mode == mode && r.all[i].flags == flags && r.all[i].packed < 2) return static_cast<int>(i);
    return idx;
}

int grow_scratch(nb_ctx *ctx, size_t need, cudaStream_t st)
{
    if (need <= ctx->scratch_bytes) return NB_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
        ctx->err = "split scratch too small during stream capture (call nb_reserve first)";
        return NB_ERR_STATE;
    }
    NB_CUDA(ctx, cudaStreamSynchronize(st));
    if (ctx->scratch) cudaFree(ctx->scratch);
    ctx->scratch = nullptr;
    ctx->scratch_bytes = 0;
    if (cudaMalloc(&ctx->scratch, need) != cudaSuccess) {
        cudaGetLastError();
        ctx->err = "cannot allocate split scratch";
        return NB_ERR_NOMEM;
    }
    ctx->scratch_bytes = need;
    return NB_OK;
}

// Record that slots [a, b) now hold float forms predicted in frame epoch e.
void note_frame(nb_ctx *ctx, int64_t a, int64_t b, uint64_t e)
{
    if (a >= b) return;
    auto &f = ctx->frames;
    auto it = f.lower_bound(a);
    if (it != f.begin()) {
        auto pr = std::prev(it);
        if (pr->second.first > a) {   // a range that starts before a and reaches into [a, b)
            const auto tail = pr->second;
            pr->second.first = a;
            if (tail.first > b) f[b] = tail;
        }
    }
    it = f.lower_bound(a);
    while (it != f.end() && it->first < b) {
        const auto cur = *it;
        it = f.erase(it);
        if (cur.second.first > b) { f[b] = cur.second; break; }
    }
    f[a] = {b, e};
}

// A call's float-form arithmetic differences velocities stored relative to a
// frame velocity: every slot of its j-range must share one frame.
int check_frames(nb_ctx *ctx, int mode, int64_t a, int64_t n)
{
    if (mode == NB_FP64 || n <= 0) return NB_OK;
    const int64_t b = a + n;
    auto &f = ctx->frames;
    auto it = f.upper_bound(a);
    if (it != f.begin()) --it;
    bool seen = false;
    uint64_t e = 0;
    for (; it != f.end() && it->first < b; ++it) {
        if (it->second.first <= a) continue;
        if (seen && it->second.second != e) {
            ctx->err = "the j-range holds slots predicted in different velocity frames (predict it in one call, "
                       "or pass NB_KEEP_FRAME to the later predictions)";
            return NB_ERR_STATE;
        }
        seen = true;
        e = it->second.second;
    }
    return NB_OK;
}

struct Call {
    int64_t j_begin, n_j;
    int32_t n_act;
    const int32_t *act;
    const double *h, *dtr;
    int32_t cap;
    int mode;
    double *F, *J, *pot;
    int32_t *nnb, *list;
    uint8_t *ovf;
};

int check_call(nb_ctx *ctx, const Call &c)
{
    if (!ctx) return NB_ERR_ARG;
    if (c.mode < NB_FP64 || c.mode > NB_FP32) { ctx->err = "bad mode"; return NB_ERR_ARG; }
    if (c.j_begin < 0 || c.n_j < 0 || c.j_begin + c.n_j > ctx->n_max || c.n_j > INT32_MAX) {
        ctx->err = "j-range outside the context";
        return NB_ERR_ARG;
    }
    if (c.n_act < 0 || c.cap < 0) { ctx->err = "negative n_act or cap"; return NB_ERR_ARG; }
    if (c.n_act > 0) {
        if (c.n_j == 0) { ctx->err = "active particles with an empty j-range"; return NB_ERR_ARG; }
        if (!c.act || !c.h || !c.F || !c.J || !c.nnb || !c.ovf) { ctx->err = "NULL array"; return NB_ERR_ARG; }
        if (c.cap > 0 && !c.list) { ctx->err = "NULL list with cap > 0"; return NB_ERR_ARG; }
    }
    if (!(ctx->forms_valid & mode_forms(c.mode))) {
        ctx->err = "the requested form has not been predicted";
        return NB_ERR_STATE;
    }
    return check_frames(ctx, c.mode, c.j_begin, c.n_j);
}

ClusterDesc make_desc(const Call &c)
{
    ClusterDesc d{};
    d.j_begin = c.j_begin;
    d.n_j = static_cast<int32_t>(c.n_j);
    d.n_act = c.n_act;
    d.cap = c.cap;
    d.act = c.act;
    d.h = c.h;
    d.dtr = c.dtr;
    d.F = c.F;
    d.J = c.J;
    d.pot = c.pot;
    d.nnb = c.nnb;
    d.list = c.list;
    d.ovf = c.ovf;
    return d;
}

// Order the active set along a Morton curve and build one frame per block of
// `per_block` sorted particles (nb_sort.cu); fills d.perm and d.frames.
int sort_and_frames(nb_ctx *ctx, const Call &c, int per_block, ClusterDesc &d, cudaStream_t st)
{
    const int n_blocks = (c.n_act + per_block - 1) / per_block;
    const size_t need = nb::sort_scratch_bytes(c.n_act, n_blocks);
    if (need > ctx->sort_bytes) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
            ctx->err = "sort scratch too small during stream capture";
            return NB_ERR_STATE;
        }
        NB_CUDA(ctx, cudaStreamSynchronize(st));
        if (ctx->sort) cudaFree(ctx->sort);
        ctx->sort = nullptr;
        ctx->sort_bytes = 0;
        if (cudaMalloc(&ctx->sort, need) != cudaSuccess) {
            cudaGetLastError();
            ctx->err = "cannot allocate the sort scratch";
            return NB_ERR_NOMEM;
        }
        ctx->sort_bytes = need;
    }
    nb::SortParams sp{};
    sp.n_act = c.n_act;
    sp.n_j = static_cast<int>(c.n_j);
    sp.j_begin = c.j_begin;
    sp.act = c.act;
    sp.h = c.h;
    sp.pos_hi = ctx->mx_hi;
    sp.pos_lo = ctx->mx_lo;
    sp.vel_hi = ctx->mv_hi;
    sp.vel_lo = ctx->mv_lo;
    const nb::SortBuffers sb = nb::carve_sort(ctx->sort, c.n_act, n_blocks);
    d.perm = nb::launch_sort_and_frames(sp, sb, per_block, n_blocks, st);
    d.frames = sb.frames;
    NB_CUDA(ctx, cudaGetLastError());
    ctx->last_compact = sb.n_compact;
    ctx->last_blocks = n_blocks;
    return NB_OK;
}

// Dynamic shared memory of a kernel launch: the entry's, plus the list
// segments of the thread-block-cluster kernel.
size_t launch_smem(const KernelEntry &e, int cap)
{
    if (e.packed != kClusterPacked) return static_cast<size_t>(e.smem);
    return static_cast<size_t>(e.smem) + static_cast<size_t>(iblock_size(e)) * cap * sizeof(int32_t);
}

// Whether the thread-block-cluster kernel can run a call tiled as d: at most
// kMaxClusterSplits splits, shared memory within the opt-in limit, and at
// least one cluster of that size fits the GPU (answers cached per size).
bool cluster_fits(nb_ctx *ctx, int idx, const ClusterDesc &d)
{
    const KernelEntry &e = registry().all[idx];
    if (d.n_split < 1 || d.n_split > kMaxClusterSplits) return false;
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const size_t smem = launch_smem(e, d.cap);
    if (smem > static_cast<size_t>(optin)) return false;
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, size_t>, bool> known;
    const auto key = std::make_tuple(ctx->device, idx, static_cast<int>(d.n_split), smem);
    std::lock_guard<std::mutex> lock(mu);
    const auto it = known.find(key);
    if (it != known.end()) return it->second;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(static_cast<unsigned>(d.n_split));
    lc.blockDim = dim3(e.warps * 32);
    lc.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = static_cast<unsigned>(d.n_split);
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    int n = 0;
    const bool ok = cudaOccupancyMaxActiveClusters(&n, e.fn, &lc) == cudaSuccess && n > 0;
    if (!ok) cudaGetLastError();
    known[key] = ok;
    return ok;
}

// Launch the regular-force kernel of entry e over the work of p: persistent
// grid of `grid` CTAs, or, for the thread-block-cluster kernel, one cluster of
// d0.n_split CTAs per block of active particles.
int launch_regf(nb_ctx *ctx, const KernelEntry &e, const nb::RegfParams &p, int64_t grid, cudaStream_t st)
{
    nb::RegfParams q = p;
    void *args[] = {&q};
    if (e.packed != kClusterPacked) {
        NB_CUDA(ctx, cudaLaunchKernel(e.fn, dim3(static_cast<unsigned>(grid)), dim3(e.warps * 32), args, e.smem, st));
        return NB_OK;
    }
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(static_cast<unsigned>(static_cast<int64_t>(p.d0.n_iblk) * p.d0.n_split));
    lc.blockDim = dim3(e.warps * 32);
    lc.dynamicSmemBytes = launch_smem(e, p.d0.cap);
    lc.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = static_cast<unsigned>(p.d0.n_split);
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    NB_CUDA(ctx, cudaLaunchKernelExC(&lc, e.fn, args));
    return NB_OK;
}

// Kernel entry, resident CTAs per SM and tiling of a single call: the
// configuration chosen (cfg_override, else nb_set_kernel_config, else the
// tuned one of the call's size class, else the default), moved to a
// per-particle-layout kernel for a j-range at an odd slot, and to the mode's
// default when it names the cluster kernel for a split count, cap or cluster
// size that kernel cannot take.
int select_single(nb_ctx *ctx, const Call &c, const nb_kcfg *cfg_override, int *idx_out, int *occ_out,
                  ClusterDesc *d_out, bool *heuristic_out = nullptr)
{
    const int flags = (c.dtr ? 1 : 0) | (c.pot ? 2 : 0);
    nb_kcfg cfg = cfg_override ? *cfg_override : pick_cfg(ctx, c.mode, flags, c.n_act, c.n_j);
    for (int attempt = 0; attempt < 2; attempt++) {
        int idx = find_entry(c.mode, cfg, flags);
        if (idx < 0) { ctx->err = "no kernel for this mode"; return NB_ERR_UNSUPPORTED; }
        if (registry().all[idx].packed >= 2 && (c.j_begin & 1)) idx = layout_fallback(c.mode, idx, flags);
        if (registry().all[idx].packed >= 2 && (c.j_begin & 1)) {
            ctx->err = "no per-particle-layout kernel for a j-range at an odd slot with these flags";
            return NB_ERR_UNSUPPORTED;
        }
        int occ = 0;
        const int rc = entry_occupancy(ctx, idx, &occ);
        if (rc != NB_OK) return rc;
        ClusterDesc d = make_desc(c);
        tile_cluster(registry().all[idx], occ, ctx->sm_count, &cfg, d);
        if (registry().all[idx].packed == kClusterPacked && !cluster_fits(ctx, idx, d)) {
            cfg = default_cfg(c.mode);
            continue;
        }
        d.item_begin = 0;
        *idx_out = idx;
        *occ_out = occ;
        *d_out = d;
        if (heuristic_out) *heuristic_out = cfg.split <= 0;
        return NB_OK;
    }
    ctx->err = "no kernel for this call";
    return NB_ERR_UNSUPPORTED;
}

// A single call whose i-blocks fill at least one round of the persistent grid
// but not a whole number of rounds may run as two launches over consecutive
// rows of its active set: the i-blocks of the whole rounds with their j-ranges
// unsplit, then the remaining i-blocks with their j-ranges split so that they
// fill one round together (and a merge of their splits).  With the uniform
// split every i-block pays for the round that the remainder leaves part-filled
// (at 16384 of N = 16384 active, 512 i-blocks of 32 take four rounds of 152
// CTAs, the last 37 % full).  Taken only where the split is left to the
// heuristic and the cost model of tile_cluster (rounds x (tiles per item + 1.5)
// plus the merge, here plus half a tile for the second launch) puts it below
// the uniform split; not for the framed or the thread-block-cluster kernels.
// Returns the rows of the unsplit part (0: run the call whole) and the tiles
// per split of the rest.
struct TailSplit {
    int32_t rows;
    int32_t tps;
};

TailSplit tail_split(const KernelEntry &e, int occ, int sm, const ClusterDesc &d, bool heuristic)
{
    TailSplit t{0, 0};
    if (!heuristic || e.packed < 2 || e.packed == 4 || e.packed == kClusterPacked || d.n_tiles < 2) return t;
    const int64_t slots = std::max<int64_t>(1, static_cast<int64_t>(sm) * occ);
    const int64_t full = d.n_iblk / slots, rem = d.n_iblk - full * slots;
    if (full < 1 || rem == 0) return t;
    const int64_t ipb = iblock_size(e);
    const int64_t head_rows = full * slots * ipb, tail_rows = d.n_act - head_rows;
    const int S = static_cast<int>(std::min<int64_t>(std::max<int64_t>(slots / rem, 1), d.n_tiles));
    const int ts = (d.n_tiles + S - 1) / S;
    const int64_t ns = (d.n_tiles + ts - 1) / ts;
    if (tail_rows <= 0) return t;
    if (ns > 1 && ns * tail_rows * (72 + 4 * static_cast<int64_t>(d.cap)) > (int64_t(1) << 30)) return t;
    auto merge = [&](int64_t n_split, int64_t rows) {
        return n_split > 1 ? 1.5 + static_cast<double>(n_split) * rows * (64.0 + 2.0 * d.cap) / 2e7 : 0.0;
    };
    const int64_t items = static_cast<int64_t>(d.n_iblk) * d.n_split;
    const double uniform = static_cast<double>((items + slots - 1) / slots) * (d.tiles_per_split + 1.5) +
                           merge(d.n_split, d.n_act);
    const double tail = static_cast<double>(full) * (d.n_tiles + 1.5) + (ts + 1.5) + merge(ns, tail_rows) + 0.5;
    if (tail < uniform - 1e-9) {
        t.rows = static_cast<int32_t>(head_rows);
        t.tps = ts;
    }
    return t;
}

// The two parts of a tail-split call: rows [0, t.rows) with one split, the
// rest (the call's pointers moved on by t.rows rows) with t.tps tiles per split.
void tail_parts(const KernelEntry &e, int occ, int sm, const Call &c, const TailSplit &t, ClusterDesc &head,
                ClusterDesc &rest)
{
    Call ch = c;
    ch.n_act = t.rows;
    head = make_desc(ch);
    const int32_t n_tiles = static_cast<int32_t>((c.n_j + e.jtile - 1) / e.jtile);
    nb_kcfg fh{e.warps, e.ipw, e.jtile, std::max(1, n_tiles), e.packed};
    tile_cluster(e, occ, sm, &fh, head);
    Call cr = c;
    const int64_t r = t.rows;
    cr.n_act = c.n_act - t.rows;
    cr.act = c.act + r;
    cr.h = c.h + r;
    cr.dtr = c.dtr ? c.dtr + r : nullptr;
    cr.F = c.F + 3 * r;
    cr.J = c.J + 3 * r;
    cr.pot = c.pot ? c.pot + r : nullptr;
    cr.nnb = c.nnb + r;
    cr.list = c.list ? c.list + r * c.cap : nullptr;
    cr.ovf = c.ovf + r;
    rest = make_desc(cr);
    nb_kcfg fr{e.warps, e.ipw, e.jtile, t.tps, e.packed};
    tile_cluster(e, occ, sm, &fr, rest);
    head.item_begin = rest.item_begin = 0;
}

// Launch the force kernel of one part of a single call (its split scratch
// already carved), and the merge of its splits; counts the launches.
int launch_part(nb_ctx *ctx, const KernelEntry &e, int occ, const ClusterDesc &d, int mode, cudaStream_t st,
                int *launches)
{
    nb::RegfParams p{};
    p.js = tile_streams(ctx, mode, e);
    p.soa = jset(ctx, mode);
    p.d0 = d;
    p.table = nullptr;
    p.work = nullptr;
    p.n_clusters = 1;
    p.n_items = static_cast<int64_t>(d.n_iblk) * d.n_split;
    p.status = ctx->d_status;
    p.wait_ns = ctx->wait_ns;
    p.extra_tx = ctx->extra_tx;
    const int64_t grid = std::min<int64_t>(p.n_items, static_cast<int64_t>(ctx->sm_count) * occ);
    int rc = launch_regf(ctx, e, p, grid, st);
    if (rc != NB_OK) return rc;
    ++*launches;
    if (d.n_split > 1 && e.packed != kClusterPacked) {
        nb::MergeParams mp{};
        mp.d0 = d;
        mp.n_clusters = 1;
        mp.n_total = d.n_act;
        mp.ff = mode != NB_FP64;
        mp.status = ctx->d_status;
        nb::launch_merge(mp, st);
        NB_CUDA(ctx, cudaGetLastError());
        ++*launches;
    }
    return NB_OK;
}

int run_single(nb_ctx *ctx, const Call &c, const nb_kcfg *cfg_override, cudaStream_t st)
{
    int rc = check_call(ctx, c);
    if (rc != NB_OK) return rc;
    ctx->last_launches = 0;
    if (c.n_act == 0) return NB_OK;
    DeviceGuard guard(ctx->device);
    int idx = -1, occ = 0;
    ClusterDesc d{};
    bool heuristic = false;
    rc = select_single(ctx, c, cfg_override, &idx, &occ, &d, &heuristic);
    if (rc != NB_OK) return rc;
    const KernelEntry &e = registry().all[idx];
    const TailSplit tail = tail_split(e, occ, ctx->sm_count, d, heuristic);
    if (tail.rows > 0) {
        ClusterDesc head{}, rest{};
        tail_parts(e, occ, ctx->sm_count, c, tail, head, rest);
        rc = grow_scratch(ctx, cluster_scratch(rest, e.packed), st);
        if (rc != NB_OK) return rc;
        carve_scratch(head, nullptr, e.packed);
        carve_scratch(rest, static_cast<char *>(ctx->scratch), e.packed);
        int launches = 0;
        rc = launch_part(ctx, e, occ, head, c.mode, st, &launches);
        if (rc == NB_OK) rc = launch_part(ctx, e, occ, rest, c.mode, st, &launches);
        ctx->last_launches = launches;
        return rc;
    }
    rc = grow_scratch(ctx, cluster_scratch(d, e.packed), st);
    if (rc != NB_OK) return rc;
    carve_scratch(d, static_cast<char *>(ctx->scratch), e.packed);
    int sort_launches = 0;
    if (e.packed == 4) {   // framed kernel: spatial order of the active set and per-block frames
        rc = sort_and_frames(ctx, c, e.warps * e.ipw, d, st);
        if (rc != NB_OK) return rc;
        sort_launches = 10;
    }

    nb::RegfParams p{};
    p.js = tile_streams(ctx, c.mode, e);
    p.soa = jset(ctx, c.mode);
    p.d0 = d;
    p.table = nullptr;
    p.work = nullptr;
    p.n_clusters = 1;
    p.n_items = static_cast<int64_t>(d.n_iblk) * d.n_split;
    p.status = ctx->d_status;
    p.wait_ns = ctx->wait_ns;
    p.extra_tx = ctx->extra_tx;
    const int64_t grid = std::min<int64_t>(p.n_items, static_cast<int64_t>(ctx->sm_count) * occ);
    rc = launch_regf(ctx, e, p, grid, st);
    if (rc != NB_OK) return rc;
    ctx->last_launches = 1 + sort_launches;
    if (d.n_split > 1 && e.packed != kClusterPacked) {
        nb::MergeParams mp{};
        mp.d0 = d;
        mp.n_clusters = 1;
        mp.n_total = d.n_act;
        mp.ff = c.mode != NB_FP64;
        mp.status = ctx->d_status;
        nb::launch_merge(mp, st);
        NB_CUDA(ctx, cudaGetLastError());
        ctx->last_launches = 2 + sort_launches;
    }
    return NB_OK;
}

}  // namespace

extern "C" {

const char *nb_strerror(int s)
{
    switch (s) {
    case NB_OK: return "ok";
    case NB_ERR_ARG: return "invalid argument";
    case NB_ERR_CUDA: return "CUDA runtime error";
    case NB_ERR_NOMEM: return "out of memory";
    case NB_ERR_TIMEOUT: return "a bounded device wait ran out";
    case NB_ERR_STATE: return "invalid state (form not predicted, or scratch too small under capture)";
    case NB_ERR_UNSUPPORTED: return "unsupported configuration";
    case NB_ERR_DEVICE_INPUT: return "invalid active index or radius found on the device";
    case NB_ERR_INTERNAL: return "a device-side bounds check of the library's own indexing failed";
    default: return "unknown status";
    }
}

const char *nb_last_error(nb_ctx *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

int nb_create(nb_ctx **out, int device, int64_t n_max)
{
    if (!out) return NB_ERR_ARG;
    *out = nullptr;
    if (n_max <= 0 || n_max > INT32_MAX) return NB_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return NB_ERR_ARG;
    }
    DeviceGuard guard(device);
    nb_ctx *c = new nb_ctx();
    c->device = device;
    c->n_max = n_max;
    for (int m = 0; m < 3; m++) c->cfg[m] = default_cfg(m);
    int rc = NB_OK;
    auto alloc = [&](void **p, size_t bytes) {
        if (rc != NB_OK) return;
        if (cudaMalloc(p, bytes) != cudaSuccess) { cudaGetLastError(); rc = NB_ERR_NOMEM; }
    };
    const size_t n = static_cast<size_t>(n_max);
    alloc(reinterpret_cast<void **>(&c->pos64), n * sizeof(double4_32a));
    alloc(reinterpret_cast<void **>(&c->vel64), n * sizeof(double4_32a));
    alloc(reinterpret_cast<void **>(&c->mx_hi), n * sizeof(float4));
    alloc(reinterpret_cast<void **>(&c->mx_lo), n * sizeof(float4));
    alloc(reinterpret_cast<void **>(&c->mv_hi), n * sizeof(float4));
    alloc(reinterpret_cast<void **>(&c->mv_lo), n * sizeof(float4));
    alloc(reinterpret_cast<void **>(&c->pos32), n * sizeof(float4));
    alloc(reinterpret_cast<void **>(&c->vel32), n * sizeof(float4));
    const size_t npairs = (n + 1) / 2;
    for (int k = 0; k < 7; k++) alloc(reinterpret_cast<void **>(&c->pim[k]), npairs * sizeof(float4));
    for (int k = 0; k < 4; k++) alloc(reinterpret_cast<void **>(&c->pif[k]), npairs * sizeof(float4));
    alloc(reinterpret_cast<void **>(&c->d_status), sizeof(int));
    if (rc == NB_OK && cudaMemset(c->d_status, 0, sizeof(int)) != cudaSuccess) rc = NB_ERR_CUDA;
    alloc(reinterpret_cast<void **>(&c->d_frame), 4 * sizeof(double));
    if (rc == NB_OK && cudaMemset(c->d_frame, 0, 4 * sizeof(double)) != cudaSuccess) rc = NB_ERR_CUDA;
    if (rc == NB_OK && cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        rc = NB_ERR_CUDA;
    if (rc != NB_OK) {
        nb_destroy(c);
        return rc;
    }
    *out = c;
    return NB_OK;
}

void nb_destroy(nb_ctx *c)
{
    if (!c) return;
    DeviceGuard guard(c->device);
    cudaDeviceSynchronize();
    void *bufs[] = {c->pos64, c->vel64, c->mx_hi, c->mx_lo, c->mv_hi, c->mv_lo, c->pos32, c->vel32,
                    c->d_status, c->d_frame, c->scratch, c->stage, c->sort};
    for (void *b : bufs)
        if (b) cudaFree(b);
    for (float4 *b : c->pim)
        if (b) cudaFree(b);
    for (float4 *b : c->pif)
        if (b) cudaFree(b);
    for (cudaEvent_t e : c->chunk_ev)
        if (e) cudaEventDestroy(e);
    if (c->copy_done) cudaEventDestroy(c->copy_done);
    if (c->copy_st) cudaStreamDestroy(c->copy_st);
    delete c;
}

int nb_sm_count(nb_ctx *ctx) { return ctx ? ctx->sm_count : 0; }

static int predict_impl(nb_ctx *ctx, int64_t offset, int64_t n, const double *x0, const double *v0,
                        const double *a0, const double *adot0, const double *m, const double *t0,
                        double t, int forms, cudaStream_t st)
{
    if (!ctx) return NB_ERR_ARG;
    if (offset < 0 || n < 0 || offset + n > ctx->n_max) { ctx->err = "slots outside the context"; return NB_ERR_ARG; }
    if (n > 0 && (!x0 || !v0 || !m || (a0 && (!adot0 || !t0)))) { ctx->err = "NULL array"; return NB_ERR_ARG; }
    const bool keep = (forms & NB_KEEP_FRAME) != 0;
    forms &= ~NB_KEEP_FRAME;
    if (forms == 0) forms = NB_FORM_ALL;
    if (forms & ~NB_FORM_ALL) { ctx->err = "bad forms mask"; return NB_ERR_ARG; }
    DeviceGuard guard(ctx->device);
    nb::PredParams p{};
    p.offset = offset;
    p.n = n;
    p.x0 = x0; p.v0 = v0; p.a0 = a0; p.adot0 = adot0; p.m = m; p.t0 = t0; p.t = t;
    p.forms = forms;
    p.keep_frame = keep ? 1 : 0;
    p.frame = ctx->d_frame;
    p.pos64 = ctx->pos64; p.vel64 = ctx->vel64;
    p.mx_hi = ctx->mx_hi; p.mx_lo = ctx->mx_lo; p.mv_hi = ctx->mv_hi; p.mv_lo = ctx->mv_lo;
    p.pos32 = ctx->pos32; p.vel32 = ctx->vel32;
    for (int k = 0; k < 7; k++) p.pim[k] = ctx->pim[k];
    for (int k = 0; k < 4; k++) p.pif[k] = ctx->pif[k];
    nb::launch_predict(p, st);
    NB_CUDA(ctx, cudaGetLastError());
    ctx->forms_valid = forms;   // forms not rewritten are stale now
    if (n > 0) {
        if (!keep) ctx->epoch = ++ctx->epochs;
        note_frame(ctx, offset, offset + n, ctx->epoch);
    }
    return NB_OK;
}

int nb_predict(nb_ctx *ctx, int64_t offset, int64_t n, const double *x0, const double *v0,
               const double *a0, const double *adot0, const double *m, const double *t0, double t,
               int forms, nb_stream_t stream)
{
    if (n > 0 && (!a0 || !adot0 || !t0)) { if (ctx) ctx->err = "NULL array"; return NB_ERR_ARG; }
    return predict_impl(ctx, offset, n, x0, v0, a0, adot0, m, t0, t, forms,
                        static_cast<cudaStream_t>(stream));
}

int nb_set_predicted(nb_ctx *ctx, int64_t offset, int64_t n, const double *x, const double *v,
                     const double *m, int forms, nb_stream_t stream)
{
    return predict_impl(ctx, offset, n, x, v, nullptr, nullptr, m, nullptr, 0.0, forms,
                        static_cast<cudaStream_t>(stream));
}

int nb_get_predicted(nb_ctx *ctx, int64_t offset, int64_t n, double *x, double *v, double *m,
                     nb_stream_t stream)
{
    if (!ctx) return NB_ERR_ARG;
    if (offset < 0 || n < 0 || offset + n > ctx->n_max || (n > 0 && (!x || !v))) {
        ctx->err = "bad read-back range or NULL array";
        return NB_ERR_ARG;
    }
    if (!(ctx->forms_valid & NB_FORM_FP64)) { ctx->err = "FP64 form not predicted"; return NB_ERR_STATE; }
    if (n == 0) return NB_OK;
    DeviceGuard guard(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t w = sizeof(double4_32a);
    const char *p = reinterpret_cast<const char *>(ctx->pos64 + offset);
    const char *q = reinterpret_cast<const char *>(ctx->vel64 + offset);
    NB_CUDA(ctx, cudaMemcpy2DAsync(x, 3 * sizeof(double), p, w, 3 * sizeof(double), n, cudaMemcpyDeviceToDevice, st));
    NB_CUDA(ctx, cudaMemcpy2DAsync(v, 3 * sizeof(double), q, w, 3 * sizeof(double), n, cudaMemcpyDeviceToDevice, st));
    if (m)
        NB_CUDA(ctx, cudaMemcpy2DAsync(m, sizeof(double), p + 3 * sizeof(double), w, sizeof(double), n,
                                       cudaMemcpyDeviceToDevice, st));
    return NB_OK;
}

// The switch between needed-only and full prediction, from graph-replayed
// times on GB300 (two-float stored form): a full prediction of n slots takes
// about 2.06 us + 0.108 ns per slot (3.8 us at n = 16384, 16.2 us at 131072);
// a needed-only one about 4.3 us + 0.15 ns per list entry, and lists hold
// about half of their cap slots, i.e. ~0.075 ns per (active particle, list
// slot) thread.
static bool needed_not_worth_it(int64_t n, int32_t n_act, int32_t cap)
{
    const double threads = static_cast<double>(n_act) * (static_cast<double>(cap) + 1.0);
    return 4300.0 + 0.075 * threads >= 2060.0 + 0.108 * static_cast<double>(n);
}

int nb_predict_needed(nb_ctx *ctx, int64_t offset, int64_t n, int32_t n_act, const int32_t *act,
                      const int32_t *nnb, const int32_t *list, int32_t cap, const double *x0, const double *v0,
                      const double *a0, const double *adot0, const double *m, const double *t0, double t,
                      int forms, nb_stream_t stream)
{
    if (!ctx) return NB_ERR_ARG;
    if (offset < 0 || n < 0 || offset + n > ctx->n_max) { ctx->err = "slots outside the context"; return NB_ERR_ARG; }
    if (n_act < 0 || cap < 0) { ctx->err = "negative n_act or cap"; return NB_ERR_ARG; }
    if (n_act > 0 && n == 0) { ctx->err = "active particles with an empty range"; return NB_ERR_ARG; }
    if (n_act > 0 && (!act || !nnb || (cap > 0 && !list) || !x0 || !v0 || !a0 || !adot0 || !m || !t0)) {
        ctx->err = "NULL array";
        return NB_ERR_ARG;
    }
    const bool only = (forms & NB_NEEDED_ONLY) != 0;
    forms &= ~(NB_KEEP_FRAME | NB_NEEDED_ONLY);   // always the current frame
    if (forms == 0) forms = ctx->forms_valid;
    if (forms & ~NB_FORM_ALL) { ctx->err = "bad forms mask"; return NB_ERR_ARG; }
    if (forms == 0 || (forms & ~ctx->forms_valid)) {
        ctx->err = "needed-only prediction of a form the range's last prediction did not write";
        return NB_ERR_STATE;
    }
    // the slots it does not rewrite must already be in the current frame
    for (auto it = ctx->frames.begin(); it != ctx->frames.end(); ++it)
        if (it->first < offset + n && it->second.first > offset && it->second.second != ctx->epoch) {
            ctx->err = "the range was predicted in another velocity frame than the current one (predict it in "
                       "full, or set the frame, first)";
            return NB_ERR_STATE;
        }
    if (n_act == 0) return NB_OK;
    if (!only && needed_not_worth_it(n, n_act, cap))   // the NPACT switch: predict the whole range
        return predict_impl(ctx, offset, n, x0, v0, a0, adot0, m, t0, t, forms | NB_KEEP_FRAME,
                            static_cast<cudaStream_t>(stream));
    DeviceGuard guard(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    nb::NeededParams np{};
    nb::PredParams &p = np.pp;
    p.offset = offset;
    p.n = n;
    p.x0 = x0; p.v0 = v0; p.a0 = a0; p.adot0 = adot0; p.m = m; p.t0 = t0; p.t = t;
    p.forms = forms;
    p.keep_frame = 1;
    p.frame = ctx->d_frame;
    p.pos64 = ctx->pos64; p.vel64 = ctx->vel64;
    p.mx_hi = ctx->mx_hi; p.mx_lo = ctx->mx_lo; p.mv_hi = ctx->mv_hi; p.mv_lo = ctx->mv_lo;
    p.pos32 = ctx->pos32; p.vel32 = ctx->vel32;
    for (int k = 0; k < 7; k++) p.pim[k] = ctx->pim[k];
    for (int k = 0; k < 4; k++) p.pif[k] = ctx->pif[k];
    np.n_act = n_act;
    np.cap = cap;
    np.act = act;
    np.nnb = nnb;
    np.list = list;
    np.status = ctx->d_status;
    nb::launch_predict_needed(np, st);
    NB_CUDA(ctx, cudaGetLastError());
    ctx->forms_valid = forms;
    ctx->last_launches = 1;
    return NB_OK;
}

int nb_set_frame(nb_ctx *ctx, const double *u)
{
    if (!ctx || !u) return NB_ERR_ARG;
    DeviceGuard guard(ctx->device);
    NB_CUDA(ctx, cudaMemcpy(ctx->d_frame, u, 3 * sizeof(double), cudaMemcpyHostToDevice));
    ctx->epoch = ++ctx->epochs;
    return NB_OK;
}

int nb_get_frame(nb_ctx *ctx, double *u)
{
    if (!ctx || !u) return NB_ERR_ARG;
    DeviceGuard guard(ctx->device);
    NB_CUDA(ctx, cudaDeviceSynchronize());
    NB_CUDA(ctx, cudaMemcpy(u, ctx->d_frame, 3 * sizeof(double), cudaMemcpyDeviceToHost));
    return NB_OK;
}

int nb_regular_force(nb_ctx *ctx, int64_t j_begin, int64_t n_j, int32_t n_act, const int32_t *act,
                     const double *h, const double *dtr, int32_t cap, int mode, double *F, double *J,
                     double *pot, int32_t *nnb, int32_t *list, uint8_t *ovf, nb_stream_t stream)
{
    const Call c{j_begin, n_j, n_act, act, h, dtr, cap, mode, F, J, pot, nnb, list, ovf};
    return run_single(ctx, c, nullptr, static_cast<cudaStream_t>(stream));
}

int nb_last_launches(nb_ctx *ctx) { return ctx ? ctx->last_launches : 0; }

int nb_reserve(nb_ctx *ctx, size_t bytes)
{
    if (!ctx) return NB_ERR_ARG;
    DeviceGuard guard(ctx->device);
    return grow_scratch(ctx, bytes, nullptr);
}

size_t nb_scratch_bytes(nb_ctx *ctx, int64_t n_j, int32_t n_act, int32_t cap, int mode)
{
    if (!ctx || mode < 0 || mode > 2 || n_act <= 0 || n_j <= 0 || cap < 0) return 0;
    size_t best = 0;
    for (int flags = 0; flags < 4; flags++) {   // the largest over the flag variants
        const nb_kcfg cfg = pick_cfg(ctx, mode, flags, n_act, n_j);
        const int idx = find_entry(mode, cfg, flags);
        if (idx < 0) continue;
        int occ = 0;
        if (entry_occupancy(ctx, idx, &occ) != NB_OK) continue;
        ClusterDesc d{};
        d.n_j = static_cast<int32_t>(n_j);
        d.n_act = n_act;
        d.cap = cap;
        const KernelEntry &e = registry().all[idx];
        tile_cluster(e, occ, ctx->sm_count, &cfg, d);
        best = std::max(best, cluster_scratch(d, e.packed));
        const TailSplit t = tail_split(e, occ, ctx->sm_count, d, cfg.split <= 0);
        if (t.rows > 0) {   // the split part of a tail-split call
            ClusterDesc r{};
            r.n_j = d.n_j;
            r.n_act = n_act - t.rows;
            r.cap = cap;
            const nb_kcfg fr{e.warps, e.ipw, e.jtile, t.tps, e.packed};
            tile_cluster(e, occ, ctx->sm_count, &fr, r);
            best = std::max(best, cluster_scratch(r, e.packed));
        }
    }
    return best;
}

int nb_sync_status(nb_ctx *ctx, nb_stream_t stream)
{
    if (!ctx) return NB_ERR_ARG;
    DeviceGuard guard(ctx->device);
    NB_CUDA(ctx, cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    int h = 0;
    NB_CUDA(ctx, cudaMemcpy(&h, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (h != 0) NB_CUDA(ctx, cudaMemset(ctx->d_status, 0, sizeof(int)));
    if (h & nb::DEV_BOUNDS) {
        ctx->err = "a bounds check of the library's own output indexing failed on the device (store skipped)";
        return NB_ERR_INTERNAL;
    }
    if (h & nb::DEV_TIMEOUT) { ctx->err = "a bounded copy wait ran out on the device"; return NB_ERR_TIMEOUT; }
    if (h & nb::DEV_BAD_INPUT) { ctx->err = "invalid active index or radius on the device"; return NB_ERR_DEVICE_INPUT; }
    return NB_OK;
}

int nb_num_kernel_configs(int mode)
{
    int n = 0;
    for (const auto &e : registry().all)
        if (e.mode == mode && e.flags == 0) n++;
    return n;
}

int nb_get_kernel_config(int mode, int index, nb_kcfg *out)
{
    if (!out) return NB_ERR_ARG;
    int n = 0;
    for (const auto &e : registry().all)
        if (e.mode == mode && e.flags == 0) {
            if (n == index) { *out = nb_kcfg{e.warps, e.ipw, e.jtile, 0, e.packed}; return NB_OK; }
            n++;
        }
    return NB_ERR_ARG;
}

int nb_set_kernel_config(nb_ctx *ctx, int mode, const nb_kcfg *cfg)
{
    if (!ctx || mode < 0 || mode > 2) return NB_ERR_ARG;
    if (!cfg) { ctx->cfg_set[mode] = false; ctx->cfg[mode] = default_cfg(mode); return NB_OK; }
    if (cfg->split < 0) return NB_ERR_ARG;
    for (const auto &e : registry().all)
        if (e.mode == mode && e.flags == 0 && e.warps == cfg->warps && e.ipw == cfg->ipw &&
            e.jtile == cfg->jtile && e.packed == cfg->packed) {
            ctx->cfg[mode] = *cfg;
            ctx->cfg_set[mode] = true;
            return NB_OK;
        }
    return NB_ERR_UNSUPPORTED;
}

int nb_get_active_config(nb_ctx *ctx, int mode, nb_kcfg *out)
{
    if (!ctx || !out || mode < 0 || mode > 2) return NB_ERR_ARG;
    *out = ctx->cfg_set[mode] ? ctx->cfg[mode] : default_cfg(mode);
    return NB_OK;
}

int nb_time_regular_force(nb_ctx *ctx, const nb_kcfg *cfg, int64_t j_begin, int64_t n_j,
                          int32_t n_act, const int32_t *act, const double *h, const double *dtr,
                          int32_t cap, int mode, double *F, double *J, double *pot, int32_t *nnb,
                          int32_t *list, uint8_t *ovf, int reps, nb_stream_t stream, float *ms)
{
    if (!ctx || !cfg || !ms || reps <= 0) return NB_ERR_ARG;
    DeviceGuard guard(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Call c{j_begin, n_j, n_act, act, h, dtr, cap, mode, F, J, pot, nnb, list, ovf};
    int rc = run_single(ctx, c, cfg, st);   // warm-up (and scratch growth)
    if (rc != NB_OK) return rc;
    cudaEvent_t a, b;
    NB_CUDA(ctx, cudaEventCreate(&a));
    NB_CUDA(ctx, cudaEventCreate(&b));
    cudaEventRecord(a, st);
    for (int r = 0; r < reps && rc == NB_OK; r++) rc = run_single(ctx, c, cfg, st);
    cudaEventRecord(b, st);
    cudaError_t e = cudaEventSynchronize(b);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc != NB_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "timing events");
    *ms = t / reps;
    return NB_OK;
}

// ------------------------------------------------------------ irregular force

int nb_irregular_force(nb_ctx *ctx, int64_t j_begin, int64_t n_j, int32_t n_act, const int32_t *act,
                       const int32_t *nnb, const int32_t *list, int32_t cap, int mode, double *F,
                       double *J, double *pot, nb_stream_t stream)
{
    if (!ctx) return NB_ERR_ARG;
    if (mode < NB_FP64 || mode > NB_FP32) { ctx->err = "bad mode"; return NB_ERR_ARG; }
    if (j_begin < 0 || n_j < 0 || j_begin + n_j > ctx->n_max || n_j > INT32_MAX) {
        ctx->err = "j-range outside the context";
        return NB_ERR_ARG;
    }
    if (n_act < 0 || cap < 0) { ctx->err = "negative n_act or cap"; return NB_ERR_ARG; }
    if (n_act == 0) return NB_OK;
    if (n_j == 0) { ctx->err = "active particles with an empty j-range"; return NB_ERR_ARG; }
    if (!act || !nnb || !F || !J || (cap > 0 && !list)) { ctx->err = "NULL array"; return NB_ERR_ARG; }
    if (!(ctx->forms_valid & mode_forms(mode))) {
        ctx->err = "the requested form has not been predicted";
        return NB_ERR_STATE;
    }
    const int frc = check_frames(ctx, mode, j_begin, n_j);
    if (frc != NB_OK) return frc;
    DeviceGuard guard(ctx->device);
    nb::IrrParams p{};
    p.j_begin = j_begin;
    p.n_j = static_cast<int32_t>(n_j);
    p.n_act = n_act;
    p.cap = cap;
    p.act = act;
    p.nnb = nnb;
    p.list = list;
    p.js = jset(ctx, mode);
    p.F = F;
    p.J = J;
    p.pot = pot;
    p.status = ctx->d_status;
    NB_CUDA(ctx, nb::launch_irregular(p, mode, ctx->sm_count, static_cast<cudaStream_t>(stream)));
    ctx->last_launches = 1;
    return NB_OK;
}

// ------------------------------------------------------------ autotuner

int nb_autotune(nb_ctx *ctx, int64_t j_begin, int64_t n_j, int32_t n_act, const int32_t *act,
                const double *h, const double *dtr, int32_t cap, int mode, double *F, double *J,
                double *pot, int32_t *nnb, int32_t *list, uint8_t *ovf, int reps,
                nb_stream_t stream, nb_kcfg *best, float *best_ms)
{
    if (!ctx || reps <= 0) return NB_ERR_ARG;
    DeviceGuard guard(ctx->device);
    const Call c{j_begin, n_j, n_act, act, h, dtr, cap, mode, F, J, pot, nnb, list, ovf};
    int rc = check_call(ctx, c);
    if (rc != NB_OK) return rc;
    if (n_act <= 0) { ctx->err = "nothing to tune (n_act = 0)"; return NB_ERR_ARG; }
    const int flags = (dtr ? 1 : 0) | (pot ? 2 : 0);
    Registry &r = registry();
    nb_kcfg win{0, 0, 0, 0, 0};
    float win_ms = 0.f;
    for (size_t i = 0; i < r.all.size(); i++) {
        const KernelEntry &e = r.all[i];
        if (e.mode != mode || e.flags != flags) continue;
        if (e.packed >= 2 && (j_begin & 1)) continue;   // j-pair layouts need an even first slot
        int occ = 0;
        rc = entry_occupancy(ctx, static_cast<int>(i), &occ);
        if (rc != NB_OK) return rc;
        // j-split candidates: the default, one split, and ~1, 2, 4, 8 items per resident CTA
        ClusterDesc d{};
        d.n_j = static_cast<int32_t>(n_j);
        d.n_act = n_act;
        d.cap = cap;
        tile_cluster(e, occ, ctx->sm_count, nullptr, d);
        std::vector<int> splits{0, d.n_tiles};
        const int64_t slots = static_cast<int64_t>(ctx->sm_count) * occ;
        for (int k : {1, 2, 4, 8}) {
            const int64_t n_split = std::max<int64_t>(1, (k * slots + d.n_iblk - 1) / std::max(d.n_iblk, 1));
            splits.push_back(static_cast<int>(std::max<int64_t>(1, (d.n_tiles + n_split - 1) / n_split)));
        }
        std::vector<int> tried;
        for (int sp : splits) {
            const int tps = sp == 0 ? d.tiles_per_split : sp;
            if (std::find(tried.begin(), tried.end(), tps) != tried.end()) continue;
            tried.push_back(tps);
            if (e.packed == kClusterPacked) {   // only the splits one cluster can hold
                ClusterDesc dc = d;
                const nb_kcfg cc{e.warps, e.ipw, e.jtile, tps, e.packed};
                tile_cluster(e, occ, ctx->sm_count, &cc, dc);
                if (!cluster_fits(ctx, static_cast<int>(i), dc)) continue;
            }
            const nb_kcfg cfg{e.warps, e.ipw, e.jtile, sp, e.packed};
            float ms = 0.f;
            rc = nb_time_regular_force(ctx, &cfg, j_begin, n_j, n_act, act, h, dtr, cap, mode, F, J, pot, nnb,
                                       list, ovf, reps, stream, &ms);
            if (rc == NB_ERR_NOMEM) continue;   // this split's scratch does not fit: skip it
            if (rc != NB_OK) return rc;
            const int st = nb_sync_status(ctx, stream);
            if (st != NB_OK) return st;
            if (win.warps == 0 || ms < win_ms) { win = cfg; win_ms = ms; }
        }
    }
    if (win.warps == 0) { ctx->err = "no compiled kernel for this call"; return NB_ERR_UNSUPPORTED; }
    nb_tuned t{mode, flags, log2_floor(n_act), log2_floor(n_j), win, win_ms};
    ctx->tuned[tune_key(mode, flags, t.act_class, t.j_class)] = t;
    if (best) *best = win;
    if (best_ms) *best_ms = win_ms;
    return NB_OK;
}

int nb_num_tuned(nb_ctx *ctx) { return ctx ? static_cast<int>(ctx->tuned.size()) : 0; }

int nb_get_tuned(nb_ctx *ctx, int index, nb_tuned *out)
{
    if (!ctx || !out || index < 0 || index >= static_cast<int>(ctx->tuned.size())) return NB_ERR_ARG;
    auto it = ctx->tuned.begin();
    std::advance(it, index);
    *out = it->second;
    return NB_OK;
}

int nb_set_tuned(nb_ctx *ctx, const nb_tuned *t)
{
    if (!ctx || !t || t->mode < 0 || t->mode > 2 || t->flags < 0 || t->flags > 7 || t->act_class < 0 ||
        t->act_class > 62 || t->j_class < 0 || t->j_class > 62 || t->cfg.split < 0)
        return NB_ERR_ARG;
    const uint64_t key = tune_key(t->mode, t->flags, t->act_class, t->j_class);
    if (t->cfg.warps == 0) { ctx->tuned.erase(key); return NB_OK; }
    for (const auto &e : registry().all)
        if (e.mode == t->mode && e.flags == (t->flags & 3) && e.warps == t->cfg.warps && e.ipw == t->cfg.ipw &&
            e.jtile == t->cfg.jtile && e.packed == t->cfg.packed) {
            ctx->tuned[key] = *t;
            return NB_OK;
        }
    return NB_ERR_UNSUPPORTED;
}

// ------------------------------------------------------------ host step

int nb_step_host(nb_ctx *ctx, int64_t n, const double *x0, const double *v0, const double *a0,
                 const double *adot0, const double *m, const double *t0, double t, int32_t n_act,
                 const int32_t *act, const double *h, const double *dtr, int32_t cap, int mode,
                 double *F, double *J, double *pot, int32_t *nnb, int32_t *list, uint8_t *ovf,
                 nb_stream_t stream)
{
    if (!ctx) return NB_ERR_ARG;
    if (n <= 0 || n > ctx->n_max || n_act < 0 || cap < 0 || mode < 0 || mode > 2) {
        ctx->err = "bad sizes";
        return NB_ERR_ARG;
    }
    if (!x0 || !v0 || !a0 || !adot0 || !m || !t0) { ctx->err = "NULL host input"; return NB_ERR_ARG; }
    if (n_act > 0 && (!act || !h || !F || !J || !nnb || !ovf || (cap > 0 && !list))) {
        ctx->err = "NULL host array";
        return NB_ERR_ARG;
    }
    DeviceGuard guard(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t nn = static_cast<size_t>(n), na = static_cast<size_t>(n_act);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    const size_t o_in = take(nn * 14 * sizeof(double));
    const size_t o_act = take(na * sizeof(int32_t));
    const size_t o_h = take(na * sizeof(double));
    const size_t o_dtr = take(dtr ? na * sizeof(double) : 0);
    const size_t o_F = take(na * 3 * sizeof(double));
    const size_t o_J = take(na * 3 * sizeof(double));
    const size_t o_pot = take(pot ? na * sizeof(double) : 0);
    const size_t o_nnb = take(na * sizeof(int32_t));
    const size_t o_list = take(na * static_cast<size_t>(cap) * sizeof(int32_t));
    const size_t o_ovf = take(na);
    if (off > ctx->stage_bytes) {
        NB_CUDA(ctx, cudaStreamSynchronize(st));
        if (ctx->stage) cudaFree(ctx->stage);
        ctx->stage = nullptr;
        ctx->stage_bytes = 0;
        if (cudaMalloc(&ctx->stage, off) != cudaSuccess) {
            cudaGetLastError();
            ctx->err = "cannot allocate host-step staging";
            return NB_ERR_NOMEM;
        }
        ctx->stage_bytes = off;
    }
    char *s = static_cast<char *>(ctx->stage);
    double *d_in = reinterpret_cast<double *>(s + o_in);
    const size_t v3 = nn * 3 * sizeof(double);
    NB_CUDA(ctx, cudaMemcpyAsync(d_in, x0, v3, cudaMemcpyHostToDevice, st));
    NB_CUDA(ctx, cudaMemcpyAsync(d_in + 3 * nn, v0, v3, cudaMemcpyHostToDevice, st));
    NB_CUDA(ctx, cudaMemcpyAsync(d_in + 6 * nn, a0, v3, cudaMemcpyHostToDevice, st));
    NB_CUDA(ctx, cudaMemcpyAsync(d_in + 9 * nn, adot0, v3, cudaMemcpyHostToDevice, st));
    NB_CUDA(ctx, cudaMemcpyAsync(d_in + 12 * nn, m, nn * sizeof(double), cudaMemcpyHostToDevice, st));
    NB_CUDA(ctx, cudaMemcpyAsync(d_in + 13 * nn, t0, nn * sizeof(double), cudaMemcpyHostToDevice, st));
    if (n_act > 0) {
        NB_CUDA(ctx, cudaMemcpyAsync(s + o_act, act, na * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        NB_CUDA(ctx, cudaMemcpyAsync(s + o_h, h, na * sizeof(double), cudaMemcpyHostToDevice, st));
        if (dtr) NB_CUDA(ctx, cudaMemcpyAsync(s + o_dtr, dtr, na * sizeof(double), cudaMemcpyHostToDevice, st));
    }
    int rc = nb_predict(ctx, 0, n, d_in, d_in + 3 * nn, d_in + 6 * nn, d_in + 9 * nn, d_in + 12 * nn,
                        d_in + 13 * nn, t, mode_forms(mode), st);
    if (rc != NB_OK) return rc;
    int launches = 1;
    if (n_act > 0 && cap > 0)   // list slots past min(nnb, cap) come back as -1
        NB_CUDA(ctx, cudaMemsetAsync(s + o_list, 0xff, na * static_cast<size_t>(cap) * sizeof(int32_t), st));
    if (n_act > 0) {
        // A large active set is computed in up to four chunks of consecutive
        // active particles, in order on the caller's stream, all with the
        // tiling chosen for the whole call; each chunk's results go back to the
        // host on a second stream as soon as its kernels end, so only the last
        // chunk's copy follows the computation (at N = n_act = 131072 the
        // results are ~140 MB, 0.77 ms over the host link).  Chunks are whole
        // rounds of the persistent grid (resident CTAs x particles per CTA
        // block), so that no chunk ends in a part-filled round: up to three of
        // at least 8 rounds, then the last round alone, whose copy is the only
        // one left after the computation.  Every chunk takes the j-split of the
        // whole call, so the sums, and the results, are those of one call.
        const int flags = (dtr ? 1 : 0) | (pot ? 2 : 0);
        nb_kcfg cfg = pick_cfg(ctx, mode, flags, n_act, n);
        int64_t round = 0;
        {
            const int idx = find_entry(mode, cfg, flags);
            int occ = 0;
            if (idx >= 0 && entry_occupancy(ctx, idx, &occ) == NB_OK && occ > 0) {
                const KernelEntry &e = registry().all[idx];
                round = static_cast<int64_t>(ctx->sm_count) * occ * iblock_size(e);
                ClusterDesc whole{};
                whole.n_j = static_cast<int32_t>(n);
                whole.n_act = n_act;
                whole.cap = cap;
                tile_cluster(e, occ, ctx->sm_count, &cfg, whole);
                cfg.split = whole.tiles_per_split;
            }
        }
        const int64_t rounds = round > 0 ? (n_act + round - 1) / round : 1;
        const int KB = static_cast<int>(std::min<int64_t>(3, (rounds - 1) / 8));   // chunks before the last round
        const int K = KB > 0 ? KB + 1 : 1;
        if (K > 1 && !ctx->copy_st) {
            NB_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->copy_st, cudaStreamNonBlocking));
            for (cudaEvent_t &e : ctx->chunk_ev) NB_CUDA(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            NB_CUDA(ctx, cudaEventCreateWithFlags(&ctx->copy_done, cudaEventDisableTiming));
        }
        const auto dp = [&](size_t o) { return reinterpret_cast<double *>(s + o); };
        const auto ip = [&](size_t o) { return reinterpret_cast<int32_t *>(s + o); };
        const size_t capz = static_cast<size_t>(cap);
        for (int k = 0; k < K; k++) {
            const int64_t k0 = K == 1 ? 0 : round * ((rounds - 1) * std::min(k, KB) / KB);
            const int64_t k1 = k + 1 == K ? n_act : round * ((rounds - 1) * (k + 1) / KB);
            const size_t c0 = static_cast<size_t>(k0), cn = static_cast<size_t>(k1 - k0);
            const Call c{0, n, static_cast<int32_t>(k1 - k0), ip(o_act) + c0, dp(o_h) + c0,
                         dtr ? dp(o_dtr) + c0 : nullptr, cap, mode, dp(o_F) + 3 * c0, dp(o_J) + 3 * c0,
                         pot ? dp(o_pot) + c0 : nullptr, ip(o_nnb) + c0,
                         cap > 0 ? ip(o_list) + c0 * capz : nullptr, reinterpret_cast<uint8_t *>(s + o_ovf) + c0};
            rc = run_single(ctx, c, &cfg, st);
            if (rc != NB_OK) return rc;
            launches += ctx->last_launches;
            cudaStream_t cs = st;
            if (K > 1) {
                NB_CUDA(ctx, cudaEventRecord(ctx->chunk_ev[k], st));
                NB_CUDA(ctx, cudaStreamWaitEvent(ctx->copy_st, ctx->chunk_ev[k], 0));
                cs = ctx->copy_st;
            }
            NB_CUDA(ctx, cudaMemcpyAsync(F + 3 * c0, c.F, cn * 3 * sizeof(double), cudaMemcpyDeviceToHost, cs));
            NB_CUDA(ctx, cudaMemcpyAsync(J + 3 * c0, c.J, cn * 3 * sizeof(double), cudaMemcpyDeviceToHost, cs));
            if (pot) NB_CUDA(ctx, cudaMemcpyAsync(pot + c0, c.pot, cn * sizeof(double), cudaMemcpyDeviceToHost, cs));
            NB_CUDA(ctx, cudaMemcpyAsync(nnb + c0, c.nnb, cn * sizeof(int32_t), cudaMemcpyDeviceToHost, cs));
            if (cap > 0)
                NB_CUDA(ctx, cudaMemcpyAsync(list + c0 * capz, c.list, cn * capz * sizeof(int32_t),
                                             cudaMemcpyDeviceToHost, cs));
            NB_CUDA(ctx, cudaMemcpyAsync(ovf + c0, c.ovf, cn, cudaMemcpyDeviceToHost, cs));
        }
        if (K > 1) {   // the caller's stream (synchronised below) waits for the copies
            NB_CUDA(ctx, cudaEventRecord(ctx->copy_done, ctx->copy_st));
            NB_CUDA(ctx, cudaStreamWaitEvent(st, ctx->copy_done, 0));
        }
    }
    rc = nb_sync_status(ctx, stream);
    ctx->last_launches = launches;
    return rc;
}

// --------------------------------------------------------------- plans

void nb_plan_destroy(nb_plan *p)
{
    if (!p) return;
    DeviceGuard guard(p->ctx->device);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    void *bufs[] = {p->d_table, p->d_work, p->d_act_begin, p->d_cluster_of, p->scratch};
    for (void *b : bufs)
        if (b) cudaFree(b);
    delete p;
}

int nb_plan_create(nb_ctx *ctx, int32_t n_clusters, const nb_cluster *cl, int mode,
                   const nb_kcfg *cfg_in, nb_plan **out)
{
    if (!ctx || !out || n_clusters <= 0 || !cl) return NB_ERR_ARG;
    *out = nullptr;
    DeviceGuard guard(ctx->device);
    int flags = 0;
    int64_t act_sum = 0, j_max = 1;
    for (int c = 0; c < n_clusters; c++) {
        const Call call{cl[c].j_begin, cl[c].n_j, cl[c].n_act, cl[c].act, cl[c].h, cl[c].dtr, cl[c].cap,
                        mode, cl[c].F, cl[c].J, cl[c].pot, cl[c].nnb, cl[c].list, cl[c].ovf};
        const int rc = check_call(ctx, call);
        if (rc != NB_OK) return rc;
        flags |= (cl[c].dtr ? 1 : 0) | (cl[c].pot ? 2 : 0);
        act_sum += cl[c].n_act;
        j_max = std::max<int64_t>(j_max, cl[c].n_j);
    }
    // tiling: the caller's, else the one nb_plan_autotune found for this
    // batched size class, else that of a single call of the summed size
    nb_kcfg cfg;
    if (cfg_in) {
        cfg = *cfg_in;
    } else {
        const auto it = ctx->cfg_set[mode]
                            ? ctx->tuned.end()
                            : ctx->tuned.find(tune_key(mode, flags | kBatchedClass,
                                                       log2_floor(std::max<int64_t>(act_sum, 1)), log2_floor(j_max)));
        cfg = it != ctx->tuned.end() ? it->second.cfg : pick_cfg(ctx, mode, flags, std::max<int64_t>(act_sum, 1), j_max);
    }
    int idx = find_entry(mode, cfg, flags);
    if (idx >= 0 && registry().all[idx].packed == kClusterPacked)   // serves single calls only
        idx = find_entry(mode, default_cfg(mode), flags);
    if (idx < 0) return NB_ERR_UNSUPPORTED;
    bool odd = false;
    for (int c = 0; c < n_clusters; c++) odd |= (cl[c].j_begin & 1) != 0;
    if (registry().all[idx].packed >= 2 && odd) idx = layout_fallback(mode, idx, flags);
    if (registry().all[idx].packed >= 2 && odd) {
        ctx->err = "no per-particle-layout kernel for a j-range at an odd slot with these flags";
        return NB_ERR_UNSUPPORTED;
    }
    int occ = 0;
    int rc = entry_occupancy(ctx, idx, &occ);
    if (rc != NB_OK) return rc;
    nb_plan *p = new nb_plan();
    p->ctx = ctx;
    p->mode = mode;
    p->entry = idx;
    p->e = &registry().all[idx];
    p->clusters.assign(cl, cl + n_clusters);
    p->cfg = nb_kcfg{p->e->warps, p->e->ipw, p->e->jtile, cfg.split, p->e->packed};
    p->flags = flags;
    p->act_sum = act_sum;
    p->j_max = j_max;
    // Tile every cluster.  Splits are chosen for the whole batch: the number
    // of work items across clusters should cover the resident CTA slots.
    // The clusters are laid out by decreasing j-tile count (the order of equal
    // items in the work list below); every cluster keeps its own output
    // pointers.
    std::vector<int> order(n_clusters);
    for (int c = 0; c < n_clusters; c++) order[c] = c;
    const int64_t jt = p->e->jtile;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (cl[a].n_j + jt - 1) / jt > (cl[b].n_j + jt - 1) / jt;
    });
    std::vector<ClusterDesc> &ds = p->descs;
    int64_t iblk_total = 0;
    for (int c : order) {
        const Call call{cl[c].j_begin, cl[c].n_j, cl[c].n_act, cl[c].act, cl[c].h, cl[c].dtr, cl[c].cap,
                        mode, cl[c].F, cl[c].J, cl[c].pot, cl[c].nnb, cl[c].list, cl[c].ovf};
        ds.push_back(make_desc(call));
        ClusterDesc &d = ds.back();
        const int ipb = iblock_size(*p->e);
        d.n_iblk = (d.n_act + ipb - 1) / ipb;
        iblk_total += d.n_iblk;
    }
    // a common target length of a j-split (in tiles) for the batch
    int64_t work_tiles = 0;
    for (auto &d : ds) work_tiles += static_cast<int64_t>(d.n_iblk) * ((d.n_j + p->e->jtile - 1) / p->e->jtile);
    const int64_t slots = static_cast<int64_t>(ctx->sm_count) * occ;
    int tps = cfg.split > 0 ? cfg.split
                            : static_cast<int>(std::max<int64_t>(2, work_tiles / std::max<int64_t>(1, 8 * slots)));
    size_t scratch = 0;
    int64_t items = 0;
    for (auto &d : ds) {
        nb_kcfg fixed = cfg;
        fixed.split = tps;
        tile_cluster(*p->e, occ, ctx->sm_count, &fixed, d);
        d.item_begin = items;
        items += static_cast<int64_t>(d.n_iblk) * d.n_split;
        scratch += cluster_scratch(d);
    }
    p->n_items = items;
    p->grid = static_cast<int>(std::min<int64_t>(std::max<int64_t>(items, 1), slots));
    // The work list: the items are dealt to the grid's CTAs longest first,
    // each to the CTA with the least work so far (LPT); an item costs its
    // j-tiles plus one for its start and end, which take about one tile's
    // time.  CTA b runs slots b, b + grid, ... of the list; a CTA with fewer
    // items than the most loaded one leaves its last slots empty.
    std::vector<int4> work;
    {
        struct Item { int32_t cl, ib, sp, tiles; };
        std::vector<Item> its;
        its.reserve(static_cast<size_t>(items));
        for (int c = 0; c < static_cast<int>(ds.size()); c++) {
            const ClusterDesc &d = ds[c];
            for (int ib = 0; ib < d.n_iblk; ib++)
                for (int sp = 0; sp < d.n_split; sp++) {
                    const int tb = sp * d.tiles_per_split;
                    its.push_back({c, ib, sp, std::max(0, std::min(d.tiles_per_split, d.n_tiles - tb))});
                }
        }
        std::stable_sort(its.begin(), its.end(), [](const Item &a, const Item &b) { return a.tiles > b.tiles; });
        const int G = p->grid;
        std::vector<std::vector<int32_t>> per(G);
        using Load = std::pair<int64_t, int>;   // (cost so far, CTA): ties go to the lower CTA
        std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
        for (int b = 0; b < G; b++) heap.push({0, b});
        for (size_t k = 0; k < its.size(); k++) {
            const Load l = heap.top();
            heap.pop();
            per[l.second].push_back(static_cast<int32_t>(k));
            heap.push({l.first + its[k].tiles + 1, l.second});
        }
        // Each CTA runs its items alternately from the long and the short end.
        // A short item carries as many list entries per particle as a long
        // one in far fewer tiles; between two long items the list warps
        // catch up on it while the compute warps run on.
        for (auto &v : per) {
            std::vector<int32_t> alt;
            alt.reserve(v.size());
            for (size_t a = 0, b = v.size(); a < b;) {
                alt.push_back(v[a++]);
                if (a < b) alt.push_back(v[--b]);
            }
            v.swap(alt);
        }
        size_t most = 0;
        for (const auto &v : per) most = std::max(most, v.size());
        p->n_slots = static_cast<int64_t>(most) * G;
        work.assign(static_cast<size_t>(std::max<int64_t>(p->n_slots, 1)), make_int4(-1, 0, 0, 0));
        for (int b = 0; b < G; b++)
            for (size_t k = 0; k < per[b].size(); k++) {
                const Item &it = its[per[b][k]];
                work[k * G + b] = make_int4(it.cl, it.ib, it.sp, 0);
            }
    }
    auto fail = [&](int code) { nb_plan_destroy(p); return code; };
    if (scratch > 0) {
        if (cudaMalloc(&p->scratch, scratch) != cudaSuccess) { cudaGetLastError(); return fail(NB_ERR_NOMEM); }
    }
    char *base = static_cast<char *>(p->scratch);
    std::vector<int64_t> act_begin;
    std::vector<int32_t> cluster_of;
    int64_t merged = 0;
    for (int c = 0; c < n_clusters; c++) {
        ClusterDesc &d = ds[c];
        carve_scratch(d, base);
        base += cluster_scratch(d);
        if (d.n_split > 1 && d.n_act > 0) {
            act_begin.push_back(merged);
            cluster_of.push_back(c);
            merged += d.n_act;
        }
    }
    p->n_merge = static_cast<int>(cluster_of.size());
    p->merge_total = merged;
    if (cudaMalloc(&p->d_table, ds.size() * sizeof(ClusterDesc)) != cudaSuccess ||
        cudaMalloc(&p->d_work, work.size() * sizeof(int4)) != cudaSuccess) {
        cudaGetLastError();
        return fail(NB_ERR_NOMEM);
    }
    if (cudaMemcpy(p->d_table, ds.data(), ds.size() * sizeof(ClusterDesc), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->d_work, work.data(), work.size() * sizeof(int4),
                   cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(NB_ERR_CUDA);
    if (p->n_merge > 0) {
        if (cudaMalloc(&p->d_act_begin, act_begin.size() * sizeof(int64_t)) != cudaSuccess ||
            cudaMalloc(&p->d_cluster_of, cluster_of.size() * sizeof(int32_t)) != cudaSuccess) {
            cudaGetLastError();
            return fail(NB_ERR_NOMEM);
        }
        if (cudaMemcpy(p->d_act_begin, act_begin.data(), act_begin.size() * sizeof(int64_t),
                       cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(p->d_cluster_of, cluster_of.data(), cluster_of.size() * sizeof(int32_t),
                       cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(NB_ERR_CUDA);
    }
    *out = p;
    return NB_OK;
}

int nb_plan_launches(const nb_plan *p) { return p ? (p->n_items > 0 ? 1 : 0) + (p->n_merge > 0 ? 1 : 0) : 0; }

int nb_plan_run(nb_plan *p, nb_stream_t stream)
{
    if (!p) return NB_ERR_ARG;
    nb_ctx *ctx = p->ctx;
    if (!(ctx->forms_valid & mode_forms(p->mode))) { ctx->err = "form not predicted"; return NB_ERR_STATE; }
    DeviceGuard guard(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (p->n_items > 0) {
        nb::RegfParams rp{};
        rp.js = tile_streams(ctx, p->mode, *p->e);
        rp.soa = jset(ctx, p->mode);
        rp.table = p->d_table;
        rp.work = p->d_work;
        rp.n_clusters = static_cast<int32_t>(p->descs.size());
        rp.n_items = p->n_slots;
        rp.status = ctx->d_status;
        rp.wait_ns = ctx->wait_ns;
        rp.extra_tx = ctx->extra_tx;
        void *args[] = {&rp};
        NB_CUDA(ctx, cudaLaunchKernel(p->e->fn, dim3(p->grid), dim3(p->e->warps * 32), args, p->e->smem, st));
    }
    if (p->n_merge > 0) {
        nb::MergeParams mp{};
        mp.table = p->d_table;
        mp.act_begin = p->d_act_begin;
        mp.cluster_of = p->d_cluster_of;
        mp.n_clusters = p->n_merge;
        mp.n_total = p->merge_total;
        mp.ff = p->mode != NB_FP64;
        mp.status = ctx->d_status;
        nb::launch_merge(mp, st);
        NB_CUDA(ctx, cudaGetLastError());
    }
    return NB_OK;
}

int nb_plan_capture(nb_plan *p, nb_stream_t stream)
{
    if (!p) return NB_ERR_ARG;
    nb_ctx *ctx = p->ctx;
    DeviceGuard guard(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (p->exec) { cudaGraphExecDestroy(p->exec); p->exec = nullptr; }
    if (p->graph) { cudaGraphDestroy(p->graph); p->graph = nullptr; }
    NB_CUDA(ctx, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const int rc = nb_plan_run(p, stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &g);
    if (rc != NB_OK) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
    p->graph = g;
    NB_CUDA(ctx, cudaGraphInstantiate(&p->exec, g, 0));
    return NB_OK;
}

int nb_regular_force_batched(nb_ctx *ctx, int32_t n_clusters, const nb_cluster *clusters, int mode,
                             nb_stream_t stream)
{
    nb_plan *p = nullptr;
    int rc = nb_plan_create(ctx, n_clusters, clusters, mode, nullptr, &p);
    if (rc != NB_OK) return rc;
    rc = nb_plan_run(p, stream);
    const int st = nb_sync_status(ctx, stream);   // the plan's buffers outlive its kernels
    ctx->last_launches = rc == NB_OK ? nb_plan_launches(p) : 0;
    nb_plan_destroy(p);
    return rc != NB_OK ? rc : st;
}

int nb_plan_get_config(const nb_plan *p, nb_kcfg *out)
{
    if (!p || !out) return NB_ERR_ARG;
    *out = p->cfg;
    return NB_OK;
}

int nb_plan_autotune(nb_plan *p, int reps, nb_stream_t stream, nb_kcfg *best, float *best_ms)
{
    if (!p || reps <= 0) return NB_ERR_ARG;
    nb_ctx *ctx = p->ctx;
    if (!(ctx->forms_valid & mode_forms(p->mode))) { ctx->err = "form not predicted"; return NB_ERR_STATE; }
    DeviceGuard guard(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    bool odd = false;
    for (const auto &c : p->clusters) odd |= (c.j_begin & 1) != 0;
    const int nc = static_cast<int>(p->clusters.size());
    cudaEvent_t a, b;
    NB_CUDA(ctx, cudaEventCreate(&a));
    NB_CUDA(ctx, cudaEventCreate(&b));
    nb_kcfg win{0, 0, 0, 0, 0};
    float win_ms = 0.f;
    int rc = NB_OK;
    Registry &r = registry();
    for (size_t i = 0; i < r.all.size() && rc == NB_OK; i++) {
        const KernelEntry &e = r.all[i];
        if (e.mode != p->mode || e.flags != p->flags) continue;
        if (e.packed >= 2 && odd) continue;   // j-pair layouts need even first slots
        if (e.packed == kClusterPacked) continue;   // serves single calls only
        // j-split length in tiles: the plan's heuristic (0), powers of two up
        // to the largest cluster's tile count, and that count (no split)
        const int max_tiles = static_cast<int>((p->j_max + e.jtile - 1) / e.jtile);
        std::vector<int> tpss{0};
        for (int t = 1; t < max_tiles && t <= 64; t *= 2) tpss.push_back(t);
        tpss.push_back(std::max(1, max_tiles));
        for (int tps : tpss) {
            const nb_kcfg cfg{e.warps, e.ipw, e.jtile, tps, e.packed};
            nb_plan *q = nullptr;
            const int cr = nb_plan_create(ctx, nc, p->clusters.data(), p->mode, &cfg, &q);
            if (cr == NB_ERR_NOMEM) { cudaGetLastError(); continue; }   // this split's scratch does not fit
            if (cr != NB_OK) { rc = cr; break; }
            if (q->entry != static_cast<int>(i)) { nb_plan_destroy(q); continue; }
            rc = nb_plan_run(q, stream);   // warm-up
            if (rc == NB_OK) {
                cudaEventRecord(a, st);
                for (int k = 0; k < reps && rc == NB_OK; k++) rc = nb_plan_run(q, stream);
                cudaEventRecord(b, st);
                float t = 0.f;
                cudaError_t ce = cudaEventSynchronize(b);
                if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, a, b);
                if (ce != cudaSuccess) rc = cuda_fail(ctx, ce, "timing events");
                if (rc == NB_OK) {
                    const int s = nb_sync_status(ctx, stream);
                    if (s != NB_OK) rc = s;
                }
                t /= reps;
                if (rc == NB_OK && (win.warps == 0 || t < win_ms)) { win = cfg; win_ms = t; }
            }
            nb_plan_destroy(q);
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc != NB_OK) return rc;
    if (win.warps == 0) { ctx->err = "no compiled kernel for this plan"; return NB_ERR_UNSUPPORTED; }
    // rebuild the plan with the winner (its captured graph, if any, is dropped)
    nb_plan *q = nullptr;
    rc = nb_plan_create(ctx, nc, p->clusters.data(), p->mode, &win, &q);
    if (rc != NB_OK) return rc;
    std::swap(*p, *q);
    nb_plan_destroy(q);
    nb_tuned t{p->mode, p->flags | kBatchedClass, log2_floor(std::max<int64_t>(p->act_sum, 1)),
               log2_floor(p->j_max), win, win_ms};
    ctx->tuned[tune_key(t.mode, t.flags, t.act_class, t.j_class)] = t;
    if (best) *best = win;
    if (best_ms) *best_ms = win_ms;
    return NB_OK;
}

int nb_plan_launch(nb_plan *p, nb_stream_t stream)
{
    if (!p) return NB_ERR_ARG;
    if (!p->exec) { p->ctx->err = "plan has no captured graph"; return NB_ERR_STATE; }
    DeviceGuard guard(p->ctx->device);
    NB_CUDA(p->ctx, cudaGraphLaunch(p->exec, static_cast<cudaStream_t>(stream)));
    return NB_OK;
}

int nb_debug_frame_stats(nb_ctx *ctx, int *compact_blocks, int *blocks)
{
    if (!ctx || !compact_blocks || !blocks) return NB_ERR_ARG;
    *blocks = ctx->last_blocks;
    *compact_blocks = 0;
    if (ctx->last_compact) {
        DeviceGuard guard(ctx->device);
        NB_CUDA(ctx, cudaMemcpy(compact_blocks, ctx->last_compact, sizeof(int), cudaMemcpyDeviceToHost));
    }
    return NB_OK;
}

// Test hooks (not in the public header): bound of every device copy wait and
// extra transaction bytes that make every wait run out.
int nb_debug_set_wait(nb_ctx *ctx, uint64_t wait_ns, uint32_t extra_tx)
{
    if (!ctx) return NB_ERR_ARG;
    ctx->wait_ns = wait_ns ? wait_ns : kDefaultWaitNs;
    ctx->extra_tx = extra_tx & ~15u;
    return NB_OK;
}

}  // extern "C"

// ------------------------------------------------------ allocation-free call
//
// nb_regular_force_noalloc serves callers that may not allocate device memory
// while a step runs: code that runs inside a stream-capture region, real-time
// loops with a fixed memory budget reserved up front, or hosts whose device
// memory is handed out by another allocator that the library must not
// bypass.  nb_regular_force grows the context's split scratch with cudaMalloc
// when a call needs more; this variant instead uses one fixed device array,
// so it calls no cudaMalloc, cudaFree or allocating library routine.

// Split scratch of the allocation-free call: 32 MiB, resident on every device
// that loads the library, until the process exits.
static constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

std::mutex g_noalloc_mu;
void *g_noalloc_addr[256];   // device address of g_noalloc_scratch, per device (nullptr = not looked up)

// Device address of the fixed scratch on the current device.  The host-side
// name g_noalloc_scratch is only a stand-in for the symbol, never a device
// address, so the address is looked up once per device, with that device
// current.
int noalloc_scratch(nb_ctx *ctx, void **out)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (ctx->device < 0 || ctx->device >= 256) return NB_ERR_ARG;
    if (!g_noalloc_addr[ctx->device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(ctx, e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_addr[ctx->device] = p;
    }
    *out = g_noalloc_addr[ctx->device];
    return NB_OK;
}

}  // namespace

extern "C" int nb_regular_force_noalloc(nb_ctx *ctx, int64_t j_begin, int64_t n_j, int32_t n_act,
                                        const int32_t *act, const double *h, const double *dtr, int32_t cap,
                                        int mode, double *F, double *J, double *pot, int32_t *nnb,
                                        int32_t *list, uint8_t *ovf, nb_stream_t stream)
{
    const Call c{j_begin, n_j, n_act, act, h, dtr, cap, mode, F, J, pot, nnb, list, ovf};
    int rc = check_call(ctx, c);
    if (rc != NB_OK) return rc;
    ctx->last_launches = 0;
    if (c.n_act == 0) return NB_OK;
    DeviceGuard guard(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void *scratch = nullptr;
    rc = noalloc_scratch(ctx, &scratch);
    if (rc != NB_OK) return rc;
    // the tiling nb_regular_force would take: set by nb_set_kernel_config, else
    // the tuned one of the call's size class, else the default
    int idx = -1, occ = 0;
    ClusterDesc d{};
    bool heuristic = false;
    rc = select_single(ctx, c, nullptr, &idx, &occ, &d, &heuristic);
    if (rc != NB_OK) return rc;
    const KernelEntry &e = registry().all[idx];
    const TailSplit tail = tail_split(e, occ, ctx->sm_count, d, heuristic);
    ClusterDesc head{};
    if (tail.rows > 0) tail_parts(e, occ, ctx->sm_count, c, tail, head, d);   // d: the split part
    const size_t need = cluster_scratch(d, e.packed);
    if (need > kNoAllocScratchBytes) {
        ctx->err = "the call needs " + std::to_string(need) + " bytes of split scratch; the fixed array of "
                   "nb_regular_force_noalloc holds " + std::to_string(kNoAllocScratchBytes) +
                   " (use fewer active particles or a smaller cap per call, or nb_regular_force)";
        return NB_ERR_ARG;
    }
    // The array keeps the previous call's contents.  Nothing needs clearing:
    // every work item stores (does not add to) its own (split, particle)
    // partials, count and list slots, and the merge reads only those.
    carve_scratch(d, static_cast<char *>(scratch), e.packed);
    int launches = 0;
    if (tail.rows > 0) {   // the unsplit rounds first, as nb_regular_force runs them
        carve_scratch(head, nullptr, e.packed);
        rc = launch_part(ctx, e, occ, head, c.mode, st, &launches);
        if (rc != NB_OK) return rc;
    }
    rc = launch_part(ctx, e, occ, d, c.mode, st, &launches);
    ctx->last_launches = launches;
    return rc;
}
