/*
 * nbreg.h - C-ABI of the GB300 regular-force library (libnbreg.so).
 *
 * The library computes, for the active particles of one block step of an
 * Ahmad-Cohen (AC) neighbour-scheme N-body integrator, the regular force, its
 * time derivative (jerk) and the neighbour list, after predicting all
 * j-particles to the block time (Nitadori & Aarseth 2012, "Accelerating
 * NBODY6 with Graphics Processing Units"):
 *   - prediction of the j-particles: Sec. 3.3, step (iii);
 *   - neighbour criterion |R_ij| < h_i, or with the velocity term
 *     min(|R_ij|, |R_ij + dtr_i V_ij|) < h_i: Sec. 3.2;
 *   - regular force F_R,i = sum over j != i outside the sphere of
 *     m_j R_ij/|R_ij|^3, its derivative m_j [V_ij/|R_ij|^3
 *     - 3 (R_ij.V_ij) R_ij/|R_ij|^5], and the list
 *     L_i = { j != i : R_min < h_i }: Sec. 3.3, step (vi);
 *   - the library boundary itself mirrors the paper's GPUNB calls (send the
 *     predicted j-set, then compute blocks of i): Sec. 3.4 and Appendix C.
 * G = 1.  R_ij = x_j - x_i, V_ij = v_j - v_i.
 *
 * Conventions shared by every entry point:
 *   - Every pointer argument is a DEVICE pointer owned by the caller, unless
 *     the argument is documented as a host pointer.  The library never frees
 *     caller memory.  The context owns the predicted j-set and the scratch.
 *   - Vectors are row-major [n][3] FP64 (x, y, z of particle j at 3j..3j+2).
 *   - Indices are 0-based.  Active indices and list entries are relative to
 *     the first slot of the j-range a call is given.
 *   - Calls that take a stream are asynchronous on that stream (NULL is the
 *     legacy default stream).  They return at once with NB_OK or an argument
 *     error; errors raised on the device (bad index inside a device array,
 *     a bounded wait that ran out) are recorded in a device status word and
 *     surface through nb_sync_status().
 *   - No exception crosses the boundary; every entry point returns a status.
 *   - A context is bound to one device and must be used from one host thread
 *     at a time.
 */
#ifndef NBREG_H
#define NBREG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes returned by every entry point. */
enum nb_status {
    NB_OK = 0,
    NB_ERR_ARG = -1,         /* invalid argument (detected on the host)          */
    NB_ERR_CUDA = -2,        /* a CUDA runtime call failed                        */
    NB_ERR_NOMEM = -3,       /* device or pinned memory allocation failed         */
    NB_ERR_TIMEOUT = -4,     /* a bounded device wait ran out (device status)     */
    NB_ERR_STATE = -5,       /* e.g. the requested precision form was not predicted */
    NB_ERR_UNSUPPORTED = -6, /* no kernel for this combination                    */
    NB_ERR_DEVICE_INPUT = -7, /* invalid value found on the device (index, radius) */
    NB_ERR_INTERNAL = -8      /* a device-side bounds check of the library's own output
                               * indexing failed; the store was skipped (a library bug) */
};

/* Precision form of the pairwise arithmetic. */
enum nb_mode {
    NB_FP64 = 0,  /* FP64 differences, FP64 pair terms, FP64 sums                   */
    NB_MIXED = 1, /* two-float (hi+lo) position differences, FP32 pair terms,         *
                   * float-float sums per lane, across lanes and across j-splits,   *
                   * FP64 outputs; the default tilings (packed = 5, 9) difference   *
                   * FP32-rounded velocities, the exact pair tilings (packed = 2,   *
                   * 14) and the scalar kernels two-float velocities.  The float    *
                   * forms store velocities relative to a frame velocity u (see     *
                   * nb_predict), so an FP32 velocity difference has an absolute    *
                   * error of about 2^-24 (|v_i - u| + |v_j - u|): at the level of  *
                   * the pair term's other FP32 roundings as long as the predicted  *
                   * velocities spread about u by no more than a few velocity       *
                   * dispersions.  A cluster with any bulk velocity meets that when *
                   * it is predicted in a call of its own (u is then its own mean   *
                   * velocity); several clusters with different bulk velocities     *
                   * predicted in ONE call do not, and should be predicted one call *
                   * per cluster (or use the exact pair tilings).                   */
    NB_FP32 = 2   /* plain FP32 differences and pair terms, same sums as NB_MIXED    */
};

/* Bit mask of the predicted forms nb_predict()/nb_set_predicted() write, and
 * NB_KEEP_FRAME: store the float forms in the context's current frame
 * velocity instead of computing a new one (see nb_predict); NB_NEEDED_ONLY:
 * nb_predict_needed predicts only the slots it names (see there). */
enum nb_form_bits { NB_FORM_FP64 = 1, NB_FORM_MIXED = 2, NB_FORM_FP32 = 4, NB_FORM_ALL = 7,
                    NB_KEEP_FRAME = 8, NB_NEEDED_ONLY = 16 };

typedef struct nb_ctx nb_ctx;     /* opaque, library-owned */
typedef struct nb_plan nb_plan;   /* opaque, library-owned */
typedef void *nb_stream_t;        /* a cudaStream_t */

/* Kernel tiling of the regular-force kernel (chosen by the autotuner). */
typedef struct nb_kcfg {
    int32_t warps;      /* warps per CTA; each warp owns `ipw` active particles        */
    int32_t ipw;        /* active particles per warp (the i-tile of a warp)             */
    int32_t jtile;      /* j-particles per shared-memory tile                            */
    int32_t split;      /* j-tiles per work item; 0 = choose from the grid size          */
    int32_t packed;     /* float forms: 0 = one FP32 operation per pair term; 1 = two
                         * i-particles per f32x2 instruction; 2 = two j-particles per
                         * f32x2 instruction (pair-interleaved j-set); 3 = as 2 with two
                         * j-pairs per lane per step; 4 = as 2 (two-float form only)
                         * with the active set sorted along a Morton curve and compact
                         * blocks computed in FP32 offsets from a shared frame centre;
                         * 5 = as 2 (two-float form only) with two-float positions and
                         * FP32 velocity differences; 5 + NL (NL >= 1) = the arithmetic
                         * of 5 (two-float form) or 2 (FP32 form) with `warps` - NL
                         * compute warps and NL warps that build the neighbour lists;
                         * 10 + NL = the exact pair arithmetic of 2 (two-float form)
                         * with NL list warps.  FP64 form: 0.                            */
} nb_kcfg;

/* One independent cluster of a batched call (host struct; the pointers in it
 * are device pointers with the meaning of the nb_regular_force arguments). */
typedef struct nb_cluster {
    int64_t j_begin;       /* first slot of this cluster in the context's j-set */
    int64_t n_j;           /* number of j-particles of the cluster              */
    int32_t n_act;         /* active particles                                   */
    int32_t cap;           /* list capacity per active particle                  */
    const int32_t *act;    /* [n_act] indices in [0, n_j)                        */
    const double *h;       /* [n_act] neighbour radii, >= 0                      */
    const double *dtr;     /* [n_act] regular steps, or NULL (plain criterion)   */
    double *F;             /* [n_act][3] regular force                           */
    double *J;             /* [n_act][3] regular jerk                            */
    double *pot;           /* [n_act] sum of m_j/|R_ij| over the regular set, or NULL */
    int32_t *nnb;          /* [n_act] true neighbour count                       */
    int32_t *list;         /* [n_act][cap] ascending neighbour indices, or NULL if cap == 0 */
    uint8_t *ovf;          /* [n_act] 1 when nnb > cap                           */
} nb_cluster;

/* Open a context on CUDA device `device` for up to n_max j-particles
 * (~ GPUNB_OPEN, Appendix C).  Allocates the predicted j-set (248 bytes per
 * slot for all three forms and their pair-interleaved copies) and the device
 * status word.  *out is NULL on
 * failure.  Returns NB_ERR_ARG (n_max <= 0, bad device), NB_ERR_NOMEM or
 * NB_ERR_CUDA. */
int nb_create(nb_ctx **out, int device, int64_t n_max);

/* Release everything the context owns (~ GPUNB_CLOSE).  NULL is a no-op.
 * Synchronises the device first. */
void nb_destroy(nb_ctx *ctx);

/* Predict j-particles to the block time t and store them in slots
 * [offset, offset + n) of the context's j-set (Sec. 3.3 step (iii); the
 * paper's host predictor followed by GPUNB_SEND, here one kernel):
 *   dt = t - t0_j,  x = x0 + v0 dt + a0 dt^2/2 + adot0 dt^3/6,
 *                   v = v0 + a0 dt + adot0 dt^2/2       (FP64).
 * x0, v0, a0, adot0: [n][3]; m, t0: [n]; all device pointers.
 * forms: NB_FORM_* bits of the stored copies to write (0 = all): FP64
 * (x,y,z,m)+(vx,vy,vz,0) as double4; MIXED hi/lo float pairs of position and
 * velocity with the mass's hi and lo parts in the w of the position pair;
 * FP32 float4 copies; the j-pair kernels' pair-interleaved copies of the
 * MIXED and FP32 forms.
 * Velocity frame (no counterpart in the paper): the MIXED and FP32 copies
 * hold v - u, formed in FP64 before rounding, where the frame velocity u is
 * the mean start velocity v0 of 32 particles spread evenly over this call's
 * range (all of them if n < 32), computed on the device inside the same
 * launch; with NB_KEEP_FRAME in `forms` the context's current frame is used
 * instead (the last computed one, or the one given to nb_set_frame).  Only
 * velocity differences enter the results, so u changes no result beyond
 * rounding; it keeps the FP32 velocity differences accurate for clusters
 * that move through the caller's frame.  The FP64 copy holds v itself.  The
 * context records the frame of every predicted slot range: a force call
 * whose j-range holds slots predicted under different frames (e.g. a range
 * predicted in two calls without NB_KEEP_FRAME on the second) returns
 * NB_ERR_STATE instead of mixing them.
 * Errors: NB_ERR_ARG if offset < 0, n < 0, offset + n > n_max, a NULL array
 * with n > 0. */
int nb_predict(nb_ctx *ctx, int64_t offset, int64_t n, const double *x0, const double *v0,
               const double *a0, const double *adot0, const double *m, const double *t0,
               double t, int forms, nb_stream_t stream);

/* Needed-only prediction (Sec. 3.5: when few particles are needed the
 * paper's host library predicts only those, the NPACT switch between
 * GPUIRR_PRED_ACT and GPUIRR_PRED_ALL of Appendix C).  Predicts, with the
 * polynomial and stored forms of nb_predict, the slots of the range
 * [offset, offset + n) that an irregular-force call with the same act, nnb,
 * list and cap reads: act[k] and the first min(nnb[k], cap) entries of list
 * row k, for k < n_act.  One launch of one thread per (active particle, list
 * slot); a slot named several times is predicted by each thread naming it,
 * with identical results.  The input arrays are those of the whole range
 * ([n][3], [n], indexed like act).  The switch: the call predicts the whole
 * range instead (nb_predict with NB_KEEP_FRAME) when that is the cheaper
 * launch by a time model measured on GB300, i.e. when
 * 4.3 us + 0.075 ns * n_act * (cap + 1) >= 2.06 us + 0.108 ns * n (at n =
 * 16384 always; at n = 131072 with cap 256 from about 620 active particles);
 * NB_NEEDED_ONLY in `forms` turns the switch off, and then the slots it does
 * not name keep their values.  It uses the
 * context's current velocity frame, so every slot of the range must have been
 * predicted in that frame (NB_ERR_STATE otherwise: predict the range in full
 * first).  forms (0 = the forms valid now) must be forms the last prediction
 * wrote (NB_ERR_STATE otherwise); afterwards only those are valid.  Not a step
 * of the regular force, which needs every j-particle predicted.  An index
 * outside [0, n) or a negative count is skipped and reported as
 * NB_ERR_DEVICE_INPUT by nb_sync_status.  Holds no state between calls (it can
 * be captured in a CUDA graph).  Errors: NB_ERR_ARG for a range outside the
 * context, negative sizes or NULL arrays. */
int nb_predict_needed(nb_ctx *ctx, int64_t offset, int64_t n, int32_t n_act, const int32_t *act,
                      const int32_t *nnb, const int32_t *list, int32_t cap, const double *x0,
                      const double *v0, const double *a0, const double *adot0, const double *m,
                      const double *t0, double t, int forms, nb_stream_t stream);

/* Store already-predicted positions x, velocities v ([n][3]) and masses m
 * ([n]) in slots [offset, offset + n) (the bare GPUNB_SEND of the paper).
 * Same errors as nb_predict. */
int nb_set_predicted(nb_ctx *ctx, int64_t offset, int64_t n, const double *x, const double *v,
                     const double *m, int forms, nb_stream_t stream);

/* Read back slots [offset, offset + n) of the stored FP64 form: positions x
 * and velocities v ([n][3], device) and masses m ([n], device; may be NULL).
 * NB_ERR_STATE if the FP64 form was not written by the last prediction. */
int nb_get_predicted(nb_ctx *ctx, int64_t offset, int64_t n, double *x, double *v, double *m,
                     nb_stream_t stream);

/* The frame velocity of later predictions with NB_KEEP_FRAME: nb_set_frame
 * sets it from the host array u[3] (it starts a new frame, so slots predicted
 * before keep theirs); nb_get_frame waits for the device and copies the
 * current frame into u[3] (host).  NULL arguments: NB_ERR_ARG.  No
 * counterpart in the paper. */
int nb_set_frame(nb_ctx *ctx, const double *u);
int nb_get_frame(nb_ctx *ctx, double *u);

/* Regular force, jerk and neighbour list (Sec. 3.3 step (vi), criterion of
 * Sec. 3.2; ~ GPUNB_REGF).  The j-set is slots [j_begin, j_begin + n_j) of
 * the context; act[k] in [0, n_j) names active particle k within that range.
 *   h     [n_act] radii (>= 0, finite); dtr [n_act] regular steps or NULL
 *   cap   list capacity (>= 0); list is [n_act][cap], may be NULL if cap == 0
 *   F, J  [n_act][3]; pot [n_act] or NULL; nnb [n_act]; ovf [n_act]
 * Self is excluded by index.  The list holds the lowest min(nnb, cap)
 * neighbour indices in ascending order; entries past that are not written.
 * nnb is the true count, ovf[k] = (nnb[k] > cap).  A pair at exactly |R| = h
 * is not a neighbour.  Pairs with |R_ij| = 0 (j != i) outside the sphere are
 * undefined input.  mode: NB_FP64, NB_MIXED or NB_FP32; the matching form
 * must have been predicted (NB_ERR_STATE otherwise).  The call is one
 * persistent kernel launch, plus a merge launch when its j-range is split; a
 * call whose blocks of active particles fill some rounds of the grid and part
 * of another, with the split left to the library, may run as two launches
 * (the whole rounds unsplit, then the remaining rows with a split j-range and
 * their merge); nb_last_launches reports the count.  May grow the context's
 * split scratch with cudaMalloc (call nb_reserve() with nb_scratch_bytes()
 * first to avoid that, e.g. before stream capture).  Errors: NB_ERR_ARG for out-of-range sizes, NULL
 * outputs, mode; invalid act/h values found on the device set
 * NB_ERR_DEVICE_INPUT in the status word (those particles get no result). */
int nb_regular_force(nb_ctx *ctx, int64_t j_begin, int64_t n_j, int32_t n_act,
                     const int32_t *act, const double *h, const double *dtr, int32_t cap,
                     int mode, double *F, double *J, double *pot, int32_t *nnb,
                     int32_t *list, uint8_t *ovf, nb_stream_t stream);

/* Allocation-free variant of nb_regular_force (the paper has no counterpart;
 * it exists for the library's users).  Some callers cannot let a library
 * allocate device memory while a step runs: code that issues the step inside
 * a stream-capture region, real-time loops that reserve their memory once up
 * front, or programs whose device memory is handed out by another allocator.
 * nb_regular_force may call cudaMalloc to grow its split scratch; this call
 * never allocates or frees anything.  Instead its split partials live in one
 * fixed device array of 32 MiB (33554432 bytes) that every GPU loading the
 * library holds until the process exits.  A call with n_split j-splits needs
 * about n_split * n_act * (68 + 4 * cap) bytes of it (no split, no scratch;
 * for a call run as two parts, n_act is the rows of the split part).
 * Same arguments, outputs and errors as nb_regular_force, and the same tiling
 * (the one nb_set_kernel_config chose, else the tuned one of the call's size
 * class, else the default), so the two calls give bit-identical results; plus:
 * a call whose
 * split scratch would exceed the array returns NB_ERR_ARG with the sizes in
 * nb_last_error (fewer active particles per call or a smaller cap fit).
 * The first call on a device looks up the array's device address; make that
 * first call before any stream capture.  All calls share the one array and it
 * keeps the last call's contents (nothing needs clearing: a call writes every
 * partial it reads before reading it):
 * calls that may overlap on the GPU (other streams, other contexts on the same
 * device) race on it and must be serialised by the caller. */
int nb_regular_force_noalloc(nb_ctx *ctx, int64_t j_begin, int64_t n_j, int32_t n_act,
                             const int32_t *act, const double *h, const double *dtr, int32_t cap,
                             int mode, double *F, double *J, double *pot, int32_t *nnb,
                             int32_t *list, uint8_t *ovf, nb_stream_t stream);

/* Make sure the split scratch holds at least `bytes` (device memory). */
int nb_reserve(nb_ctx *ctx, size_t bytes);

/* Scratch bytes a call of nb_regular_force with these sizes needs (0 when the
 * call needs no split; for a call that runs as two parts, the larger of the
 * uniform split's need and the split part's).  Host only. */
size_t nb_scratch_bytes(nb_ctx *ctx, int64_t n_j, int32_t n_act, int32_t cap, int mode);

/* Batched form: the regular-force call for n_clusters independent clusters
 * (host array `clusters`), all in ONE persistent kernel launch plus one merge
 * launch.  A plan uploads the cluster table once and owns its scratch, so
 * nb_plan_run() allocates nothing and can be captured into a CUDA graph.
 * cfg NULL = the tiling nb_plan_autotune recorded for the plan's batched size
 * class, else the context's configuration for a single call of the summed
 * size (see nb_autotune).  The paper has no
 * counterpart (it runs one simulation per GPU); each cluster's outputs have
 * the meaning of nb_regular_force's.  Errors: those of nb_regular_force for
 * any cluster (NB_ERR_ARG, NB_ERR_STATE), NB_ERR_NOMEM for the plan's device
 * memory. */
int nb_plan_create(nb_ctx *ctx, int32_t n_clusters, const nb_cluster *clusters, int mode,
                   const nb_kcfg *cfg, nb_plan **out);
int nb_plan_run(nb_plan *plan, nb_stream_t stream);
/* Capture nb_plan_run on `stream` into a CUDA graph owned by the plan. */
int nb_plan_capture(nb_plan *plan, nb_stream_t stream);
/* Launch the captured graph (NB_ERR_STATE if nb_plan_capture was not called). */
int nb_plan_launch(nb_plan *plan, nb_stream_t stream);
void nb_plan_destroy(nb_plan *plan);
/* Kernel launches one nb_plan_run issues (host only). */
int nb_plan_launches(const nb_plan *plan);
/* The tiling the plan runs (split = j-tiles per j-split of every cluster, 0 =
 * the plan's heuristic).  Host only. */
int nb_plan_get_config(const nb_plan *plan, nb_kcfg *out);
/* Autotuner of a plan (no counterpart in the paper): times nb_plan_run of the
 * plan's own cluster table, `reps` runs after one warm-up (CUDA events on
 * `stream`; the clusters' outputs are overwritten), for every compiled tiling
 * of the plan's mode with its flags, each with the plan's j-split heuristic
 * and with fixed j-split lengths of 1, 2, 4, ... tiles up to the largest
 * cluster's tile count; rebuilds the plan with the fastest (a graph captured
 * from the plan is dropped: capture again) and records it in the context's
 * tuned table under the batched size class (mode, flags | 4, floor(log2 of the
 * summed n_act), floor(log2 of the largest n_j)), which later nb_plan_create
 * calls with cfg NULL use.  *best / *best_ms (either may be NULL) receive the
 * winner and its mean time per run.  Allocates, synchronises; not capturable. */
int nb_plan_autotune(nb_plan *plan, int reps, nb_stream_t stream, nb_kcfg *best, float *best_ms);

/* One-shot batched call: builds a plan for `clusters` (cfg = the context's
 * configuration for `mode`), runs it on `stream`, waits for the stream and
 * frees the plan.  Same outputs and errors as nb_plan_create followed by
 * nb_plan_run; returns the device status like nb_sync_status.  It allocates
 * and synchronises, so it cannot be captured: a batched step that repeats, or
 * runs inside a CUDA graph, keeps a plan (nb_plan_capture / nb_plan_launch). */
int nb_regular_force_batched(nb_ctx *ctx, int32_t n_clusters, const nb_cluster *clusters, int mode,
                             nb_stream_t stream);

/* One whole block step through HOST buffers (the paper's host-side loop of
 * prediction, GPUNB_SEND and GPUNB_REGF, Sec. 3.3 steps (iii)-(vi)): copy the j-set inputs and the
 * active set from host memory, predict (only the form `mode` needs), compute
 * the regular force, copy the results back into host memory and wait for
 * them.  All array arguments are HOST pointers (pinned memory gives
 * asynchronous copies).  List slots past min(nnb, cap) are returned as -1.  Same meaning and errors as nb_predict followed by
 * nb_regular_force on j-range [0, n); also returns the device status.  A large
 * active set is computed in a few chunks of consecutive active particles whose
 * results are copied back while the next chunk computes (same results as one
 * call). */
int nb_step_host(nb_ctx *ctx, int64_t n, const double *x0, const double *v0, const double *a0,
                 const double *adot0, const double *m, const double *t0, double t,
                 int32_t n_act, const int32_t *act, const double *h, const double *dtr,
                 int32_t cap, int mode, double *F, double *J, double *pot, int32_t *nnb,
                 int32_t *list, uint8_t *ovf, nb_stream_t stream);

/* Wait for `stream`, then read and clear the device status word.  Returns
 * NB_OK, NB_ERR_INTERNAL, NB_ERR_TIMEOUT, NB_ERR_DEVICE_INPUT or NB_ERR_CUDA. */
int nb_sync_status(nb_ctx *ctx, nb_stream_t stream);

/* Text for a status code (static storage). */
const char *nb_strerror(int status);

/* Text of the last error recorded on the context (valid until the next call). */
const char *nb_last_error(nb_ctx *ctx);

/* Kernel configurations compiled for a mode (the autotuner's search space). */
int nb_num_kernel_configs(int mode);
int nb_get_kernel_config(int mode, int index, nb_kcfg *out);
/* Select the configuration nb_regular_force uses for `mode` (NULL = back to
 * the autotuned tiling of each call's size class, else the built-in default).
 * NB_ERR_UNSUPPORTED if no compiled kernel matches.  nb_get_active_config
 * reports the configuration set here, or the built-in default. */
int nb_set_kernel_config(nb_ctx *ctx, int mode, const nb_kcfg *cfg);
int nb_get_active_config(nb_ctx *ctx, int mode, nb_kcfg *out);

/* Timing harness of the autotuner: run nb_regular_force with configuration
 * `cfg` `reps` times on `stream` after one warm-up and return the mean device
 * time per call in *ms (CUDA events on that stream). */
int nb_time_regular_force(nb_ctx *ctx, const nb_kcfg *cfg, int64_t j_begin, int64_t n_j,
                          int32_t n_act, const int32_t *act, const double *h,
                          const double *dtr, int32_t cap, int mode, double *F, double *J,
                          double *pot, int32_t *nnb, int32_t *list, uint8_t *ovf, int reps,
                          nb_stream_t stream, float *ms);

/* Irregular force (Sec. 3.3 step (iv); the paper computes it on the host):
 * for each active particle i, F_i, J_i (and, if pot != NULL, the potential
 * sum m_j/|R|) over the neighbour list row i, i.e. the first min(nnb[i], cap)
 * entries of list[i*cap ...], with R = x_j - x_i, V = v_j - v_i from the
 * predicted j-set in the form of `mode` (which must have been predicted).
 * act, nnb and list index the j-range [j_begin, j_begin + n_j) as for
 * nb_regular_force, whose outputs they usually are; with nnb[i] <= cap the sum
 * is the irregular force of the paper, and F_reg + F_irr is the full direct sum.
 * Outputs are FP64 (FP64 accumulation in every mode).  Device pointers,
 * asynchronous on `stream`; an active index outside the range, a negative
 * count, or a list entry outside the range or equal to i itself is skipped and
 * reported as NB_ERR_DEVICE_INPUT by nb_sync_status. */
int nb_irregular_force(nb_ctx *ctx, int64_t j_begin, int64_t n_j, int32_t n_act, const int32_t *act,
                       const int32_t *nnb, const int32_t *list, int32_t cap, int mode, double *F,
                       double *J, double *pot, nb_stream_t stream);

/* Autotuner (no counterpart in the paper, which fixes its tiling at compile
 * time).  A call's size class is (mode, flags, floor(log2 n_act),
 * floor(log2 n_j)), flags = 1 with a velocity criterion (dtr != NULL) | 2 with
 * a potential output.  nb_autotune times, on the caller's own call (the same
 * arguments as nb_regular_force; its outputs are overwritten), every compiled
 * tiling of the mode with exactly those flags, each with the default j-split
 * and with j-splits that give about 1, 2, 4 and 8 work items per resident CTA
 * and one split only, `reps` calls per candidate after one warm-up, and keeps
 * the fastest for the call's size class in the context.  Later calls of that
 * class (nb_regular_force, nb_step_host, nb_plan_create with the summed n_act
 * and the largest n_j) use the tuned tiling unless nb_set_kernel_config chose
 * one.  *best and *best_ms (either may be NULL) receive the winner and its
 * mean time.  Synchronises with the device.  Not a step of the paper's method:
 * it picks the i-tile, j-tile and j-split of the kernels. */
typedef struct {
    int32_t mode, flags, act_class, j_class;
    nb_kcfg cfg;
    float ms; /* mean device time per call measured by nb_autotune (0 if loaded) */
} nb_tuned;
int nb_autotune(nb_ctx *ctx, int64_t j_begin, int64_t n_j, int32_t n_act, const int32_t *act,
                const double *h, const double *dtr, int32_t cap, int mode, double *F, double *J,
                double *pot, int32_t *nnb, int32_t *list, uint8_t *ovf, int reps,
                nb_stream_t stream, nb_kcfg *best, float *best_ms);
/* The context's tuned table: entry count, entry `index` (in key order), and
 * insertion of an entry (e.g. one saved by an earlier run).  nb_set_tuned
 * checks that a kernel with the entry's tiling and flags is compiled
 * (NB_ERR_UNSUPPORTED otherwise); an entry with cfg.warps == 0 removes its
 * class from the table. */
int nb_num_tuned(nb_ctx *ctx);
int nb_get_tuned(nb_ctx *ctx, int index, nb_tuned *out);
int nb_set_tuned(nb_ctx *ctx, const nb_tuned *entry);

/* Number of kernels the last nb_regular_force call on this context launched. */
int nb_last_launches(nb_ctx *ctx);

/* Multiprocessor count of the context's device. */
int nb_sm_count(nb_ctx *ctx);

/* Test hook for the failure path: bound every device copy wait by wait_ns
 * nanoseconds (0 = the default of 4 s) and make each copy barrier expect
 * extra_tx more bytes than are copied (rounded down to a multiple of 16; 0 in
 * normal use).  With extra_tx > 0 no copy barrier completes, every wait runs
 * out after wait_ns, the kernels return early and nb_sync_status() reports
 * NB_ERR_TIMEOUT; the results of such calls are undefined. */
int nb_debug_set_wait(nb_ctx *ctx, uint64_t wait_ns, uint32_t extra_tx);

/* Diagnostic of the framed two-float kernel (tiling packed = 4, chosen with
 * nb_set_kernel_config): the number of blocks of the last framed call on the context and how many of
 * them were compact enough for frame coordinates (the rest ran the per-pair
 * two-float form).  Synchronises with the device. */
int nb_debug_frame_stats(nb_ctx *ctx, int *compact_blocks, int *blocks);

#ifdef __cplusplus
}
#endif
#endif /* NBREG_H */
