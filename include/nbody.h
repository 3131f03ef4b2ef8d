/*
 * libnbody: all-pairs softened-gravity N-body on one NVIDIA GB300 (sm_103a).
 *
 * The method is the case study of Milla & Rucci, "Performance Comparison of
 * Python Translators for a Multi-threaded CPU-bound Application"
 * (arXiv 2203.08263):
 *
 *   force (Section 2.3; the j-loops of the Section 3.2.4 and 3.3.5 figures)
 *     a_i = G * sum_j m_j (x_j - x_i) / (|x_j - x_i|^2 + eps^2)^(3/2),
 *     summed over every j including j = i (which contributes exactly 0);
 *   update (the Section 3.1.2 figure, split in two loops as in 3.2.3/3.3.5)
 *     all a_i from the positions at the start of the step; then
 *     v_i <- v_i + a_i dt / 2;  x_i <- x_i + v_i dt  (with the new v_i),
 *     positions moved only after every body has been kicked.
 *
 * The paper prints no values for G, eps (its SOFT = eps^2) or dt; they are
 * parameters here. eps must be > 0.
 *
 * Conventions for every entry point:
 *   - Arrays are contiguous, row-major: positions and velocities [n][3],
 *     masses [n]. Element type: float32 when precision == NB_FP32; float64
 *     when precision == NB_FP32_COMP_FP64_STATE (forces are then computed in
 *     FP32 with compensated accumulation; state, gradients and diagnostics
 *     stay FP64).
 *   - Array pointers are caller-owned device pointers (e.g. torch tensors on
 *     the context's device). nb_accel, nb_step and nb_run also accept host
 *     pointers (pageable or pinned); the library then copies in and out
 *     through its own device buffers and the call returns only after the
 *     results are back on the host. Every pointer must be 4-byte (float32)
 *     or 8-byte (float64) aligned.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *     default stream) unless stated. Argument errors return at once and
 *     launch nothing. Errors raised inside a kernel (a bounded wait that gave
 *     up) are recorded in the context and returned by nb_sync, and by the
 *     calls that wait for their own results (host-pointer calls, nb_energy,
 *     nb_autotune, nb_measure_peaks).
 *   - The context owns all scratch memory (packed bodies, split partials,
 *     trajectory segments, CUDA graphs, tuning tables). It grows that memory
 *     on demand with cudaMalloc, outside any stream capture.
 *   - A context is not thread-safe; use one per host thread. Its calls share
 *     its scratch, so calls issued on different streams must not overlap on
 *     the GPU: order the streams, or use one context per stream.
 *   - n == 0 is a valid no-op. No call aborts the process.
 */
#ifndef NBODY_H
#define NBODY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NB_ABI_VERSION 1

typedef struct nb_ctx nb_ctx;

typedef enum {
    NB_OK = 0,
    NB_ERR_INVALID = 1,     /* bad argument: NULL, n < 0, eps <= 0, misaligned ... */
    NB_ERR_CUDA = 2,        /* a CUDA runtime call failed; see nb_last_error */
    NB_ERR_NOMEM = 3,       /* device or host allocation failed */
    NB_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
    NB_ERR_UNSUPPORTED = 5  /* valid request this build does not implement */
} nb_status;

typedef enum {
    NB_FP32 = 0,                 /* FP32 state, FP32 forces */
    NB_FP32_COMP_FP64_STATE = 1  /* FP64 state; FP32 forces, compensated sums */
} nb_precision;

typedef enum {
    NB_SCHEME_PAPER = 0,  /* the printed update: half kick, then drift */
    NB_SCHEME_KDK = 1     /* velocity Verlet, named but not printed (3.2.3, 3.3.7) */
} nb_scheme;

typedef struct {
    double G;    /* gravitational constant (GRAVITY in the paper's listings) */
    double eps;  /* softening length; the listings add SOFT = eps^2 to r^2 */
    double dt;   /* time step (DT) */
    int precision;         /* nb_precision */
    int scheme;            /* nb_scheme; used by nb_step / nb_run */
    int tile_override[4];  /* {threads per CTA, bodies per thread, j-split,
                              j-tile bodies}; 0 = chosen by the autotuner */
} nb_params;

/* Library version; equals NB_ABI_VERSION of the header it was built from. */
int nb_abi_version(void);

/* Create a context on CUDA device `device` (cudaSetDevice is called). *out
 * receives the context, or NULL on failure. The params are copied. Returns
 * NB_ERR_INVALID for eps <= 0, a non-finite G/eps/dt or an unknown
 * precision/scheme. */
nb_status nb_create(nb_ctx **out, int device, const nb_params *p);

/* Wait for the context's work on every stream it used, release everything it
 * owns. NULL is ignored. */
void nb_destroy(nb_ctx *ctx);

/* Static, human-readable name of a status code. */
const char *nb_status_string(nb_status s);

/* Last error message recorded on ctx ("" if none); valid until the next call. */
const char *nb_last_error(const nb_ctx *ctx);

/* Replace G, eps and dt (precision and scheme are fixed at creation). */
nb_status nb_set_params(nb_ctx *ctx, double G, double eps, double dt);

/*
 * Accelerations only (Section 2.3 force sum):
 *   a[i][c] = G sum_j m_j (x_j - x_i)_c / (|x_j - x_i|^2 + eps^2)^(3/2).
 * x [n][3], m [n] in the state type; a [n][3] in the state type (float32 or
 * float64). Inputs are read-only.
 *
 * Force forms (the same sum in every form; nb_get_form tells which one
 * serves a size). A one-sided kernel sums over j for every i. From
 * n = 16384 up (or where nb_autotune finds it faster) a pair-symmetric
 * kernel evaluates each unordered pair {i, j} once and adds its term to both
 * bodies with opposite signs (Newton's third law), into per-block partials
 * that a second kernel adds in a fixed order: in FP32, and in the precision
 * form with FP32 pair terms and the partials two-summed before the FP64
 * update. One launch keeps nb x 3 x npad floats of partials in the context
 * (nb = npad / B blocks of B = 256, 512 or 1024 bodies, npad = n rounded up to a
 * block: about 12 n^2 / 1024 bytes, 0.2 GB at n = 131072). Above 512 MiB
 * of such partials (n = 262144: 0.8 GB; n = 2^20: 12.9 GB) the pair kernel
 * is launched tile by tile over w x w block pairs, each tile's partials
 * folded into running sums in the same order, with two tile buffers of at
 * most 28 MiB in all and the running sums (2 x 3 x npad floats): no size
 * limit, bit-identical results, the same speed. The VJP of nb_vjp and
 * nb_adjoint (FP32 and the precision form)
 * has the same forms (the pair-symmetric one from n = 8192, blocks of 256 or
 * 512 bodies, 8 sums per body: about 32 n^2 / 256 bytes in one launch at
 * n < 65536). Results are deterministic in every form.
 */
nb_status nb_accel(nb_ctx *ctx, int64_t n, const void *x, const void *m, void *a,
                   void *stream);

/* One step of the update selected by params.scheme, in place on x and v. */
nb_status nb_step(nb_ctx *ctx, int64_t n, void *x, void *v, const void *m, void *stream);

/*
 * `steps` steps in place on x, v (Section 3.1's loop over the update), by one
 * of three paths with the same arithmetic: a CUDA graph of one force launch
 * per step that the context captures once per (n, buffers, steps, checkpoint
 * layout) and caches; for systems of at most 4096 bodies, one kernel on one
 * thread-block cluster that keeps the positions in distributed shared memory
 * across all steps; for at most 8192 bodies, the same kernel on a cooperative
 * grid of up to one CTA per SM, exchanging positions through L2 with a
 * bounded grid barrier per step. nb_autotune picks the fastest path per size;
 * untuned, the cluster path serves n <= 512, the grid form n <= 4096 (FP32)
 * or n <= 8192 (precision form), and the graph path the rest. ckpt (nullable, device):
 * [steps/ckpt_every + 1][n][6] in the state type; slot k receives (x, v)
 * after k*ckpt_every steps (slot 0 = the input state). ckpt_every must divide
 * steps when ckpt != NULL. The paper scheme only when checkpointing.
 */
nb_status nb_run(nb_ctx *ctx, int64_t n, void *x, void *v, const void *m, int steps,
                 void *ckpt, int ckpt_every, void *stream);

/*
 * An ensemble of nsys independent systems, each advanced `steps` paper steps,
 * all in one persistent cooperative kernel launch (replayed from a cached CUDA
 * graph). System s owns bodies [offsets[s], offsets[s+1]); offsets (int64,
 * nsys+1 entries, offsets[0] = 0, non-decreasing) may be a host or a device
 * pointer. Systems do not interact. Each system's size must be at most
 * nb_batched_max_n(); steps at most 2^20 per call. Either precision and
 * either update scheme (params.precision, params.scheme), as nb_run; the
 * precision form runs items of at most 4 bodies per thread.
 * Inside the launch, work items are taken from one queue; a step of a
 * system starts when its previous step is done. Two forms (nb_get_batched_form):
 * one-sided items (system, step, chunk of T x R i-bodies for T threads per
 * CTA against all of the system's bodies; R = 8, 4, 2 or 1 per item: full
 * chunks at the shape's largest R, a system's ragged rest in smaller ones),
 * or pair-symmetric items: each system in groups of 256 bodies (zero-mass
 * padding), one item per pair of groups (each unordered pair of bodies
 * evaluated once for both), and one epilogue item per group that adds its
 * partials in group order and runs the update; a warp runs one item. In
 * FP32 the pair-symmetric form is the default when its work, padding
 * included, is below 0.85 of the one-sided form's (ensembles of systems of a
 * few hundred bodies and more) and its group-pair partials (sum over systems
 * of 12 x 256 x groups^2 bytes) fit in 16 GiB, and nb_autotune_batched times
 * both; the precision form runs it only when pinned (its FP32 partials are
 * longer sums than the one-sided tiles').
 */
nb_status nb_run_batched(nb_ctx *ctx, int nsys, const int64_t *offsets, void *x, void *v,
                         const void *m, int steps, void *stream);

/* Largest system size nb_run_batched accepts. */
int64_t nb_batched_max_n(void);

/*
 * Autotune nb_run_batched for this size profile (synchronous): times a few
 * steps of every candidate (bodies per thread, j-tile) on synthetic bodies
 * with the same system sizes and keeps the fastest for later nb_run_batched
 * calls with the same sizes.
 */
nb_status nb_autotune_batched(nb_ctx *ctx, int nsys, const int64_t *offsets);

/* The batched launch the context would use for these sizes: out[0..5] =
 * {threads per CTA, largest bodies per thread of an item, j-tile bodies, work
 * items per step, CTAs in the persistent grid, origin of the shape: 0 the
 * default, 1 nb_autotune_batched, 2 nb_set_batched_config or
 * nb_set_batched_form}. In the pair-symmetric form: {128, 8 bodies per lane,
 * 256 bodies per group, items per step, CTAs, origin}. */
nb_status nb_get_batched_config(nb_ctx *ctx, int nsys, const int64_t *offsets, int *out6);

/*
 * Pin the batched launch shape for this size profile (offsets as for
 * nb_run_batched): threads per CTA and the largest R of an item, one of
 * 128 or 256 x {1, 2, 4, 8} or 512 x {1, 2}, and jtile, the j-bodies per
 * streamed tile (32, 64, 128 or 256); the precision form takes R <= 4. All
 * three 0 removes a pinned or tuned shape (back to the default).
 * NB_ERR_INVALID for other values. Replaces
 * what nb_autotune_batched chose for these sizes. A tuning interface of this
 * library; the paper has no counterpart.
 */
nb_status nb_set_batched_config(nb_ctx *ctx, int nsys, const int64_t *offsets, int threads,
                                int bodies_per_thread, int jtile);

/* Force form of nb_run_batched for this size profile: 1 = one-sided items
 * (with a one-sided shape pinned or tuned before, else the default shape),
 * 2 = pair-symmetric items, 0 = remove a pinned or tuned choice (back to the
 * default). nb_set_batched_config pins the one-sided form. */
nb_status nb_set_batched_form(nb_ctx *ctx, int nsys, const int64_t *offsets, int form);
/* The form nb_run_batched would use for these sizes: *form = 1 one-sided,
 * 2 pair-symmetric. */
nb_status nb_get_batched_form(nb_ctx *ctx, int nsys, const int64_t *offsets, int *form);

/*
 * Reverse mode of nb_run with the paper scheme. Given the checkpoints written
 * by nb_run(..., ckpt, ckpt_every) over `steps` steps and the cotangents of
 * the final state (xbar_T, vbar_T: [n][3]), writes the gradients of the same
 * scalar loss w.r.t. the initial positions (xbar0 [n][3]), velocities
 * (vbar0 [n][3]) and masses (mbar [n]). Each segment of ckpt_every steps is
 * recomputed from its checkpoint and swept backwards:
 *   vbar' = vbar + dt xbar;  abar = dt/2 vbar';
 *   xbar += VJP_x(abar; x_t);  mbar += VJP_m(abar; x_t);  vbar = vbar'
 * with the all-pairs vector-Jacobian product
 *   VJP_x(abar)_k = G sum_j K(d_kj) (m_k abar_j - m_j abar_k),
 *   VJP_m(abar)_k = -G sum_j abar_j . d_kj / s_kj^(3/2),
 *   d_kj = x_j - x_k, s = |d|^2 + eps^2, K(d) = s^(-3/2) I - 3 s^(-5/2) d d^T.
 * All arrays device, in the state type. Inputs are read-only.
 */
nb_status nb_adjoint(nb_ctx *ctx, int64_t n, const void *m, int steps, const void *ckpt,
                     int ckpt_every, const void *xbar_T, const void *vbar_T, void *xbar0,
                     void *vbar0, void *mbar, void *stream);

/* One vector-Jacobian product of the acceleration at positions x:
 * xbar = VJP_x(abar), mbar = VJP_m(abar) (formulas as in nb_adjoint). */
nb_status nb_vjp(nb_ctx *ctx, int64_t n, const void *x, const void *m, const void *abar,
                 void *xbar, void *mbar, void *stream);

/*
 * Diagnostics (synchronous): out (host, 6 doubles) receives total momentum
 * P = sum m v (out[0..2]), kinetic energy KE = 1/2 sum m |v|^2 (out[3]), the
 * softened potential Phi = -G sum_{i<j} m_i m_j / sqrt(|x_j-x_i|^2 + eps^2)
 * (out[4]) and H' = KE + Phi/2 (out[5]), the energy the paper's half-kick
 * update conserves as dt -> 0. Pair terms in FP32, all sums in FP64.
 */
nb_status nb_energy(nb_ctx *ctx, int64_t n, const void *x, const void *v, const void *m,
                    double *out, void *stream);

/*
 * Time the candidate kernel shapes for problems of size n in mode `mode`
 * (0 = forward, 1 = adjoint VJP) and store the fastest in the context's
 * table (and in the JSON file named by $NB_AUTOTUNE_CACHE when set): every
 * compiled one-sided shape with its j-tile and split, and from n = 8192
 * (forward; 2048 for the FP32 VJP) the pair-symmetric kernels at each block
 * size. In mode 0 with n <= 8192 it also times nb_run's paths (graph of force
 * launches, one-cluster kernel, grid form) and records the fastest. Calls
 * that find no entry for their size bucket use a built-in heuristic instead.
 * Synchronous.
 */
nb_status nb_autotune(nb_ctx *ctx, int64_t n, int mode);

/* The launch shape the context would use for (n, mode):
 * out[0..4] = {threads per CTA, bodies per thread, j-split, j-tile bodies,
 * 1 if the shape came from a tuning run}. For the pair-symmetric forms the
 * block is threads x bodies per thread (also reported as the j-tile); the
 * forces' 256-body blocks come in two forms, 32 threads x 8 (one warp per
 * block pair) and 64 x 4 (two warps sharing the block pair's bodies, each
 * with half of its j-chunks; the untuned choice from 16384 to 32767 bodies). */
nb_status nb_get_config(nb_ctx *ctx, int64_t n, int mode, int *out5);

/* Force-sum forms (nb_get_form). */
typedef enum {
    NB_FORM_F32X2 = 0,           /* FP32, one-sided, packed f32x2 arithmetic */
    NB_FORM_SCALAR = 1,          /* FP32, one-sided, scalar arithmetic */
    NB_FORM_COMPENSATED = 2,     /* compensated FP32, FP64 state */
    NB_FORM_POTENTIAL = 3,       /* softened potential (nb_energy) */
    NB_FORM_VJP = 4,             /* adjoint VJP, FP32 */
    NB_FORM_VJP_COMPENSATED = 5, /* adjoint VJP, compensated, FP64 state */
    NB_FORM_SQRT_DIV = 6,        /* ablation: sqrt then division */
    NB_FORM_POW = 7,             /* ablation: powf */
    NB_FORM_PAIR_SYMMETRIC = 8,  /* FP32, each unordered pair once */
    NB_FORM_VJP_PAIR_SYMMETRIC = 9, /* adjoint VJP, FP32, each unordered pair once */
    NB_FORM_COMPENSATED_PAIR_SYMMETRIC = 10, /* compensated, FP64 state, each pair once */
    NB_FORM_VJP_COMPENSATED_PAIR_SYMMETRIC = 11 /* adjoint VJP, compensated, FP64 state, each pair once */
} nb_form;

/* The force-sum form (nb_form) the context would use for (n, mode), mode as
 * in nb_get_config (2 = the potential of nb_energy). */
nb_status nb_get_form(nb_ctx *ctx, int64_t n, int mode, int *form);

/* The nb_run path the context would use for n bodies: out[0] = 1 graph of
 * force launches, 2 one-cluster kernel, 3 its grid form; out[1] = the
 * cluster size or the grid's CTAs (0 for the graph path); out[2] = 1 if the
 * choice came from a tuning run. A query of this library's dispatch; the
 * paper has no counterpart. */
nb_status nb_get_run_path(nb_ctx *ctx, int64_t n, int *out3);

/* Wait for the context's work on `stream`, then report (and clear) any error
 * recorded by a kernel: NB_ERR_TIMEOUT if a bounded wait gave up. */
nb_status nb_sync(nb_ctx *ctx, void *stream);

/* Number of kernel launches the context issued (graph replays count each
 * kernel node once per replay). */
int64_t nb_launch_count(const nb_ctx *ctx);

/* Debug knobs. NB_DBG_WAIT_TIMEOUT_NS: give up a device-side wait after this
 * many nanoseconds (default 2e9; 0 gives up at the first poll that returns
 * without the phase complete). NB_DBG_STALL_PRODUCER (value 0/1): the
 * pair-sum kernels issue no j-tile copies, so every tile wait of nb_accel,
 * nb_step, nb_run, nb_vjp, nb_adjoint and nb_energy runs out, in
 * nb_run's grid form CTA 0 never arrives at the step barrier, so every
 * barrier wait runs out, and in nb_run_batched's pair-symmetric form one
 * warp never releases its first work item, so every item waiting for it runs
 * out its wait; with a short timeout this exercises the error path
 * without hanging (results are then invalid and nb_sync returns
 * NB_ERR_TIMEOUT). */
typedef enum {
    NB_DBG_WAIT_TIMEOUT_NS = 1,
    NB_DBG_STALL_PRODUCER = 2,
    /* FP32 forward denominator s^(3/2), s = r^2 + eps^2 (GPU analog of the
     * paper's math-operation experiment, Sections 3.2.6 and 3.3.6):
     * 0 = MUFU rsqrt cubed (default), 1 = IEEE sqrt then division,
     * 2 = powf(s, -1.5). Tuned shapes apply to 0 only. */
    NB_DBG_MATH_VARIANT = 3,
    /* nb_run path: 0 = chosen per size (default), 1 = graph of force
     * launches, 2 = one-cluster kernel, 3 = its grid form
     * (NB_ERR_UNSUPPORTED at nb_run when the system does not qualify). */
    NB_DBG_RUN_PATH = 4,
    /* Forward force form (FP32 and the precision form): 0 = chosen per size
     * (default), 1 = one-sided kernels only, 256, 512 or 1024 = the
     * pair-symmetric kernel with blocks of that many bodies, one warp per
     * 256 bodies of a block pair, at every size (nb_run's graph path; the
     * fused small-system paths keep their own kernel). */
    NB_DBG_FORM = 5,
    /* VJP form (nb_vjp, nb_adjoint; FP32 and the precision form): 0 =
     * chosen per size (default), 1 = one-sided only, 256 or 512 = the
     * pair-symmetric kernel with blocks of that many bodies at every size. */
    NB_DBG_VJP_FORM = 6,
    /* Pair-symmetric launches (forces, precision form, VJP): 0 = chosen per
     * size (default: one launch over all block pairs up to 512 MiB of
     * partials, above that one launch per tile of w x w block pairs with a
     * running sum of the partials, two tile buffers of at most 28 MiB in
     * all), -1 =
     * one launch always, w > 0 = tiles of w blocks whenever that makes more
     * than one tile. Results are bit-identical either way. */
    NB_DBG_SYM_TILE = 7,
    /* nb_adjoint with a pair-symmetric VJP: 0 = each reverse step's
     * preparation (v-bar update, the VJP's records) done by the previous
     * step's VJP epilogue inside a checkpoint segment (default), 1 = by a
     * kernel of its own every step. Results are bit-identical either way. */
    NB_DBG_ADJ_PREP = 8
} nb_debug_key;
nb_status nb_debug_set(nb_ctx *ctx, int key, int64_t value);

/*
 * Measurement of the roofline denominators on this device (synchronous):
 * out[0] = FP32 TFLOP/s issued as scalar FFMA, out[1] = FP32 TFLOP/s issued
 * as packed f32x2 FMA, out[2] = MUFU reciprocal square roots, Gop/s. Each is
 * one launch of independent FMA (or rsqrt) chains on every SM.
 */
nb_status nb_measure_peaks(nb_ctx *ctx, double *out3);

/*
 * nb_accel_noalloc: the FP32 force sum of nb_accel for callers that cannot
 * allocate device memory when they need it: processes whose device memory is
 * owned by a pooling allocator (a raw cudaMalloc there fails or fragments the
 * pool), and services whose footprint must be fixed when the library loads.
 * The paper has no counterpart; this is a deployment variant of nb_accel.
 *
 * Needs no context and calls no allocator: its working memory (packed
 * bodies, split partials, tickets) is a file-scope device array of about
 * 4.6 MB, reserved on every GPU that loads the library until the process
 * exits. n must be at most NB_NOALLOC_MAX_N (else NB_ERR_INVALID).
 * x [n][3], m [n], a [n][3]: float32 arrays in device (or managed) memory of
 * the current device, 4-byte aligned; anything else (NULL, host memory,
 * another device's memory, a misaligned address) returns NB_ERR_INVALID
 * before anything is launched, as do eps <= 0 and non-finite G or eps.
 * a = G sum_j m_j (x_j - x_i) / (|x_j - x_i|^2 + eps^2)^(3/2), asynchronous
 * on `stream`. The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) and the SM count, once per device (threads
 * making their first calls at the same time are serialised); make that first
 * call before any stream capture. A cudaDeviceReset after the first call is
 * not supported (the looked-up address is kept). Every call shares the one
 * array and clears its tickets at the start, so calls whose kernels overlap
 * on the GPU (different streams, or different host threads) race and must be
 * serialised by the caller. A device-side wait that gives up (a bulk copy
 * that has not landed after 2 s) leaves `a` partly written and is not
 * reported: there is no context to hold the error, and the next call clears
 * the error word.
 */
#define NB_NOALLOC_MAX_N 32768
nb_status nb_accel_noalloc(int64_t n, const float *x, const float *m, float *a, double G,
                           double eps, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* NBODY_H */
