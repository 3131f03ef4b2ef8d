// All-pairs tile engine: one kernel template serves every one-sided pair sum
// of the library (forces, compensated forces, potential, adjoint VJP); the
// pair-symmetric kernels (csrc/k_sym.cu) reuse its helpers and epilogues.
//
// Work decomposition. Bodies are packed in a "pair layout" (two bodies per
// 32-byte record for the force sums: {x0,x1,y0,y1}, {z0,z1,m0,m1}) and padded
// with zero-mass bodies to a multiple of the j-tile, so every j-tile is full
// and padding contributes exactly 0. CTA b handles i-block b / S and j-split
// b % S. Each of its NT threads owns R i-bodies in registers; thread 0 also
// streams the split's j-tiles into a ring of shared-memory slots with 1-D
// bulk async copies (cp.async.bulk, completion counted on an mbarrier per
// slot), refilling a slot one tile after every warp has released it through
// a second mbarrier per slot. (Built with NB_PRODUCER_WARP=1, a dedicated
// extra warp issues the copies instead; it costs a fifth more threads per
// CTA and, at 128 registers, one CTA per SM.) Every wait is bounded by a
// timeout and records an error bit instead of hanging.
//
// Split reduction. With S > 1 each CTA writes its partial sums, and the last
// CTA of an i-block to finish (atomic ticket) adds the S partials in split
// order 0..S-1, so the result does not depend on scheduling, then runs the
// policy's epilogue (write a, or kick + drift + repack for the next step).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ptx.cuh"

namespace nb {

// j-pairs per unrolled step of the tile loop, per policy (measured on GB300:
// 4 for the FP32 forces, 1 for the precision form, 2 elsewhere); a build
// flag NB_JP_UNROLL overrides all of them.
#ifdef NB_JP_UNROLL
#define NB_UNROLL_OR(n) NB_JP_UNROLL
#else
#define NB_UNROLL_OR(n) (n)
#endif

#ifndef NB_PRODUCER_WARP
#define NB_PRODUCER_WARP 0  // 0: consumer thread 0 issues the copies; 1: a dedicated warp does
#endif

#ifndef NB_COMP_NEWTON
// 1: one FP32 Newton step on the MUFU rsqrt in the precision-form kernels.
// Off by default: measured on the 2^20-body Plummer sphere it raises the
// force error (4.5e-8 vs 2.7e-8 relative L2; an FP32 Newton step cannot beat
// FP32 rounding and adds its own) and costs 4 FP32 ops per interaction.
#define NB_COMP_NEWTON 0
#endif

constexpr int kStages = 4;        // ring depth
constexpr int kProducerThreads = NB_PRODUCER_WARP ? 32 : 0;
constexpr int kPadBodies = 256;   // packed arrays hold a multiple of this
constexpr uint64_t kDrainTimeoutNs = 2000000000ull;

enum ErrBits : int {
    kErrFullWait = 1,   // consumer gave up waiting for a tile
    kErrEmptyWait = 2,  // producer gave up waiting for a free slot
    kErrDrain = 4,      // producer gave up waiting for its own copies
    kErrStepDep = 8,    // batched kernel: a system's previous step did not finish in time
};

enum DebugBits : int {
    kDbgStallProducer = 1,  // producer issues nothing: every consumer wait runs out
};

// Epilogue operations (runtime switch; never inside the pair loop).
enum EpiOp : int {
    kEpiAccel = 0,       // write a
    kEpiKickDrift = 1,   // paper: v += a dt/2; x += v dt
    kEpiKick2Drift = 2,  // velocity Verlet interior step: two half kicks, drift
    kEpiKick = 3,        // velocity Verlet closing half kick
    kEpiValue = 4,       // write the policy's per-body value (potential)
    kEpiVjp = 5,         // adjoint: accumulate xbar, mbar
};

struct ForceArgs {
    const float4 *src;    // j-records, pair layout; tile t at src + t * f4_per_tile
    int64_t n;            // real bodies
    int64_t npad;         // padded bodies (multiple of jt)
    int jt;               // j-tile bodies (even)
    int ntiles;           // npad / jt
    int split;            // S
    int iblocks;          // ceil(n / (NT * R))
    float eps2;
    double G;
    double dt;
    float4 *part;         // [S][iblocks * NT * R * PART_F4]
    unsigned *counters;   // [iblocks], zero between launches
    int *err;
    uint64_t timeout_ns;
    int op;               // EpiOp
    void *x;              // state positions [n][3]
    void *v;              // state velocities [n][3]
    void *out;            // kEpiAccel: a [n][3]; kEpiValue: [n] doubles
    float4 *xm_next;      // repacked positions for the next step (pair layout)
    void *ckpt;           // nullable: (x, v) [n][6] after this step
    // adjoint extras
    void *xbar;           // [n][3] accumulated
    void *mbar;           // [n] accumulated
    const void *abar64;   // [n][3] FP64 cotangent of a (precision form)
    const void *mass;     // [n] state-type masses (adjoint epilogue)
    int debug;            // bit 0: the producer issues no copies (timeout tests)
    int pdl;              // host: launched as a programmatic dependent of the previous kernel
    // pair-symmetric kernels launched tile by tile (csrc/k_sym.cu): the tile
    // side in blocks (0: one launch over all block pairs), this launch's
    // tile and the number of tiles; `part` then holds two tile buffers and
    // the bodies' running sums
    int tile_w;
    int tile;
    int ntile;
    // adjoint: the next reverse step's preparation fused into this VJP's
    // epilogue (pair-symmetric VJPs only, whose epilogue is a kernel of its
    // own that runs after every read of the records): vbar' = vbar + dt xbar
    // with the xbar just updated, abar = dt/2 vbar', and each body's half of
    // the next step's records from that step's positions
    int prep_next;
    const float4 *next_xm;   // FP32: the next step's packed positions
    const double *next_x64;  // precision form: the next step's FP64 (x, v) rows [n][6]
    void *vbar;              // [n][3] state-type, updated in place
};

// ---------------------------------------------------------------- helpers

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 dup(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// Scalar from the pair layout: record q = i >> 1, lane h = i & 1; within a
// record component c of body h sits at float 2c + h.
// Force records (2 float4 per pair): c = 0 x, 1 y, 2 z, 3 m.
__device__ __forceinline__ float pair_get(const float4 *base, int64_t i, int c) {
    const float *p = reinterpret_cast<const float *>(base + (i >> 1) * 2);
    return p[2 * c + (int)(i & 1)];
}
// Adjoint records (4 float4 per pair): c = 0..3 as above, 4..6 abar.
__device__ __forceinline__ float vrec_get(const float4 *base, int64_t i, int c) {
    const float *p = reinterpret_cast<const float *>(base + (i >> 1) * 4);
    return p[2 * c + (int)(i & 1)];
}
__device__ __forceinline__ void pair_put(float4 *base, int64_t i, float x, float y, float z,
                                         float m) {
    float *p = reinterpret_cast<float *>(base + (i >> 1) * 2);
    const int h = (int)(i & 1);
    p[0 + h] = x;
    p[2 + h] = y;
    p[4 + h] = z;
    p[6 + h] = m;
}

// Knuth's two-sum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// ------------------------------------------------------- the tile kernel

// One j-tile against the thread's R i-bodies. MASK drops the j == i pair
// (needed only where a pair term does not vanish at d = 0: the VJP).
template <int NT, int R, class P, bool MASK, class ACC>
__device__ __forceinline__ void tile_pass(const float4 *tile, int jpairs,
                                          const typename P::I (&ist)[R], ACC (&acc)[R],
                                          const typename P::C &cst, int64_t jbase, int64_t ibase,
                                          int tid) {
#pragma unroll(P::UNROLL)
    for (int jp = 0; jp < jpairs; ++jp) {
        float4 rec[P::REC_F4];
#pragma unroll
        for (int q = 0; q < P::REC_F4; ++q) rec[q] = tile[jp * P::REC_F4 + q];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if constexpr (MASK) {
                const int64_t k = ibase + r * NT + tid;
                const int64_t j0 = jbase + 2 * jp;
                const float2 keep = f2(j0 == k ? 0.f : 1.f, j0 + 1 == k ? 0.f : 1.f);
                P::interact_masked(rec, ist[r], acc[r], cst, keep);
            } else {
                P::interact(rec, ist[r], acc[r], cst);
            }
        }
    }
}

// Register caps: 512 resident threads per SM at R <= 4 (<= 128 registers).
// R = 8 stays uncapped: capping 128 x 8 tiles to 3 CTAs per SM (166
// registers) measured 5 % slower than 2 CTAs at 210 registers, and a 128 x 6
// shape at 3 CTAs per SM (168 registers, no spills) 2-3 % slower at N = 2^18
// and 10 % at 2^16: the reuse of each j-record across 8 i-bodies is worth
// more than the extra resident warps.
template <int NT, int R>
constexpr int min_blocks() {
    return (NB_PRODUCER_WARP || R > 4) ? 1 : 512 / NT;
}

template <int NT, int R, class P>
__global__ void __launch_bounds__(NT + kProducerThreads, (min_blocks<NT, R>())) force_kernel(const ForceArgs args) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw);
    uint64_t *empty = full + kStages;
    float4 *ring = reinterpret_cast<float4 *>(smem_raw + 128);
    __shared__ int s_last;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int ib = blockIdx.x / args.split;
    const int sp = blockIdx.x % args.split;
    const int t0 = (int)((int64_t)sp * args.ntiles / args.split);
    const int t1 = (int)((int64_t)(sp + 1) * args.ntiles / args.split);
    const int nt = t1 - t0;
    const int f4_per_tile = (args.jt >> 1) * P::REC_F4;
    const uint32_t tile_bytes = (uint32_t)f4_per_tile * 16u;
    const int64_t ibase = (int64_t)ib * NT * R;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NT / 32);
        }
        mbar_init_fence();
    }
    // Launched as a programmatic dependent (a step of nb_run after the
    // previous one), this grid may be scheduled while the previous kernel
    // finishes: wait until that grid has completed and its writes
    // (positions, partials, counters) are visible before touching global
    // memory. A no-op in an ordinary launch.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    __syncthreads();

    typename P::T tot[R];
#if NB_PRODUCER_WARP
    if (warp == NT / 32) {
        // ---------------- producer warp: one lane issues the bulk copies
        if (lane == 0) {
            int issued = 0;
            for (int k = 0; k < ((args.debug & kDbgStallProducer) ? 0 : nt); ++k) {
                const int slot = k % kStages;
                if (k >= kStages) {
                    if (!mbar_wait(&empty[slot], ((k / kStages) - 1) & 1, args.timeout_ns)) {
                        atomicOr(args.err, kErrEmptyWait);
                        break;
                    }
                }
                mbar_arrive_expect_tx(&full[slot], tile_bytes);
                bulk_g2s(ring + slot * f4_per_tile, args.src + (int64_t)(t0 + k) * f4_per_tile,
                         tile_bytes, &full[slot]);
                issued = k + 1;
            }
            // never leave while our own copies may still be landing
            for (int k = issued > kStages ? issued - kStages : 0; k < issued; ++k) {
                if (!mbar_wait(&full[k % kStages], (k / kStages) & 1, kDrainTimeoutNs))
                    atomicOr(args.err, kErrDrain);
            }
        }
        __syncwarp();
    } else {
        // ---------------- consumers
        typename P::I ist[R];
        typename P::C cst;
        P::consts(args, cst);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            int64_t i = ibase + r * NT + tid;
            P::load_i(args, i < args.npad ? i : 0, ist[r]);
            P::zero_total(tot[r]);
        }
        const int jpairs = args.jt >> 1;
        for (int k = 0; k < nt; ++k) {
            const int slot = k % kStages;
            if (!mbar_wait(&full[slot], (k / kStages) & 1, args.timeout_ns)) {
                atomicOr(args.err, kErrFullWait);
                break;
            }
            const float4 *tile = ring + slot * f4_per_tile;
            bool masked = false;
            (void)masked;
            if constexpr (P::SELF_MASK) {
                const int64_t jb = (int64_t)(t0 + k) * args.jt;
                masked = jb < ibase + (int64_t)NT * R && ibase < jb + args.jt;
            }
            if constexpr (P::PER_TILE) {
                typename P::A acc[R];
#pragma unroll
                for (int r = 0; r < R; ++r) P::zero_acc(acc[r]);
                if constexpr (P::SELF_MASK) {
                    if (masked)
                        tile_pass<NT, R, P, true>(tile, jpairs, ist, acc, cst,
                                                  (int64_t)(t0 + k) * args.jt, ibase, tid);
                    else
                        tile_pass<NT, R, P, false>(tile, jpairs, ist, acc, cst, 0, 0, tid);
                } else {
                    tile_pass<NT, R, P, false>(tile, jpairs, ist, acc, cst, 0, 0, tid);
                }
#pragma unroll
                for (int r = 0; r < R; ++r) P::tile_done(acc[r], tot[r]);
            } else {
                if constexpr (P::SELF_MASK) {
                    if (masked)
                        tile_pass<NT, R, P, true>(tile, jpairs, ist, tot, cst,
                                                  (int64_t)(t0 + k) * args.jt, ibase, tid);
                    else
                        tile_pass<NT, R, P, false>(tile, jpairs, ist, tot, cst, 0, 0, tid);
                } else {
                    tile_pass<NT, R, P, false>(tile, jpairs, ist, tot, cst, 0, 0, tid);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[slot]);
        }
    }

#else
    {
        // consumer thread 0 also streams the tiles: the first kStages up
        // front, then after tile k it refills the slot that tile k-1 used
        // (one tile of slack for the other warps to release it).
        int issued = 0;
        bool stop = (args.debug & kDbgStallProducer) != 0;
        if (tid == 0 && !stop) {
            for (int k = 0; k < nt && k < kStages; ++k) {
                mbar_arrive_expect_tx(&full[k], tile_bytes);
                bulk_g2s(ring + k * f4_per_tile, args.src + (int64_t)(t0 + k) * f4_per_tile,
                         tile_bytes, &full[k]);
                issued = k + 1;
            }
        }
        typename P::I ist[R];
        typename P::C cst;
        P::consts(args, cst);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            int64_t i = ibase + r * NT + tid;
            P::load_i(args, i < args.npad ? i : 0, ist[r]);
            P::zero_total(tot[r]);
        }
        const int jpairs = args.jt >> 1;
        for (int k = 0; k < nt; ++k) {
            const int slot = k % kStages;
            if (!mbar_wait(&full[slot], (k / kStages) & 1, args.timeout_ns)) {
                atomicOr(args.err, kErrFullWait);
                break;
            }
            const float4 *tile = ring + slot * f4_per_tile;
            bool masked = false;
            (void)masked;
            if constexpr (P::SELF_MASK) {
                const int64_t jb = (int64_t)(t0 + k) * args.jt;
                masked = jb < ibase + (int64_t)NT * R && ibase < jb + args.jt;
            }
            if constexpr (P::PER_TILE) {
                typename P::A acc[R];
#pragma unroll
                for (int r = 0; r < R; ++r) P::zero_acc(acc[r]);
                if constexpr (P::SELF_MASK) {
                    if (masked)
                        tile_pass<NT, R, P, true>(tile, jpairs, ist, acc, cst,
                                                  (int64_t)(t0 + k) * args.jt, ibase, tid);
                    else
                        tile_pass<NT, R, P, false>(tile, jpairs, ist, acc, cst, 0, 0, tid);
                } else {
                    tile_pass<NT, R, P, false>(tile, jpairs, ist, acc, cst, 0, 0, tid);
                }
#pragma unroll
                for (int r = 0; r < R; ++r) P::tile_done(acc[r], tot[r]);
            } else {
                if constexpr (P::SELF_MASK) {
                    if (masked)
                        tile_pass<NT, R, P, true>(tile, jpairs, ist, tot, cst,
                                                  (int64_t)(t0 + k) * args.jt, ibase, tid);
                    else
                        tile_pass<NT, R, P, false>(tile, jpairs, ist, tot, cst, 0, 0, tid);
                } else {
                    tile_pass<NT, R, P, false>(tile, jpairs, ist, tot, cst, 0, 0, tid);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[slot]);
            if (tid == 0 && !stop && k >= 1 && k - 1 + kStages < nt) {
                const int kp = k - 1, kr = k - 1 + kStages, rs = kp % kStages;
                if (!mbar_wait(&empty[rs], (kp / kStages) & 1, args.timeout_ns)) {
                    atomicOr(args.err, kErrEmptyWait);
                    stop = true;
                } else {
                    mbar_arrive_expect_tx(&full[rs], tile_bytes);
                    bulk_g2s(ring + rs * f4_per_tile, args.src + (int64_t)(t0 + kr) * f4_per_tile,
                             tile_bytes, &full[rs]);
                    issued = kr + 1;
                }
            }
        }
        if (tid == 0) {
            // never leave while our own copies may still be landing
            for (int k = issued > kStages ? issued - kStages : 0; k < issued; ++k) {
                if (!mbar_wait(&full[k % kStages], (k / kStages) & 1, kDrainTimeoutNs))
                    atomicOr(args.err, kErrDrain);
            }
        }
    }
#endif

    // ---------------- epilogue (all threads reach the barriers below)
    // The pair sums are done: once every CTA of this grid is here (or has
    // exited), the next step's grid may be scheduled and wait in its
    // prologue. Triggering at entry instead let the next grid's CTAs take
    // the first free SM slots and pile onto few SMs: 1.5-2x slower steps at
    // N = 3072-4096 (measured).
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const bool consumer = warp < NT / 32;
    if (args.split == 1) {
        if (consumer) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                int64_t i = ibase + r * NT + tid;
                if (i < args.n) {
                    typename P::F f;
                    P::from_total(f, tot[r]);
                    P::finish(args, i, f);
                }
            }
        }
        return;
    }
    const int64_t ni_pad = (int64_t)args.iblocks * NT * R;
    if (consumer) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            int64_t i = ibase + r * NT + tid;
            P::to_part(tot[r], args.part + ((int64_t)sp * ni_pad + i) * P::PART_F4);
        }
        __threadfence();
    }
    __syncthreads();
    if (tid == 0) {
        unsigned prev = atomicAdd(&args.counters[ib], 1u);
        s_last = (prev == (unsigned)(args.split - 1));
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (consumer) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            int64_t i = ibase + r * NT + tid;
            if (i < args.n) {
                typename P::F f;
                P::zero_final(f);
                for (int s = 0; s < args.split; ++s)
                    P::add_part(f, args.part + ((int64_t)s * ni_pad + i) * P::PART_F4);
                P::finish(args, i, f);
            }
        }
    }
    if (tid == 0) args.counters[ib] = 0u;
}

// ------------------------------------------------ shared force epilogues

// FP32 state: paper step, Verlet steps or plain output.
__device__ __forceinline__ void finish_fp32(const ForceArgs &args, int64_t i, float ax, float ay,
                                            float az) {
    if (args.op == kEpiAccel) {
        float *a = reinterpret_cast<float *>(args.out) + 3 * i;
        a[0] = ax;
        a[1] = ay;
        a[2] = az;
        return;
    }
    float *x = reinterpret_cast<float *>(args.x) + 3 * i;
    float *v = reinterpret_cast<float *>(args.v) + 3 * i;
    const float dt = (float)args.dt;
    float a3[3] = {ax, ay, az};
    float xs[3], vs[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float vc = v[c];
        // v <- v + a*dt/2 (the printed half kick), rounded step by step
        vc = __fadd_rn(vc, __fmul_rn(__fmul_rn(a3[c], dt), 0.5f));
        if (args.op == kEpiKick2Drift) vc = __fadd_rn(vc, __fmul_rn(__fmul_rn(a3[c], dt), 0.5f));
        vs[c] = vc;
        float xc = x[c];
        if (args.op != kEpiKick) xc = __fadd_rn(xc, __fmul_rn(vc, dt));  // dp = v*dt; x += dp
        xs[c] = xc;
        v[c] = vc;
        x[c] = xc;
    }
    if (args.op != kEpiKick)
        pair_put(args.xm_next, i, xs[0], xs[1], xs[2], pair_get(args.src, i, 3));
    if (args.ckpt) {
        float *ck = reinterpret_cast<float *>(args.ckpt) + 6 * i;
        ck[0] = xs[0]; ck[1] = xs[1]; ck[2] = xs[2];
        ck[3] = vs[0]; ck[4] = vs[1]; ck[5] = vs[2];
    }
}

// FP64 state (precision form): the update runs in double.
__device__ __forceinline__ void finish_fp64(const ForceArgs &args, int64_t i, double ax,
                                            double ay, double az) {
    if (args.op == kEpiAccel) {
        double *a = reinterpret_cast<double *>(args.out) + 3 * i;
        a[0] = ax;
        a[1] = ay;
        a[2] = az;
        return;
    }
    double *x = reinterpret_cast<double *>(args.x) + 3 * i;
    double *v = reinterpret_cast<double *>(args.v) + 3 * i;
    const double dt = args.dt;
    double a3[3] = {ax, ay, az};
    double xs[3], vs[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double vc = v[c];
        vc = __dadd_rn(vc, __dmul_rn(__dmul_rn(a3[c], dt), 0.5));
        if (args.op == kEpiKick2Drift) vc = __dadd_rn(vc, __dmul_rn(__dmul_rn(a3[c], dt), 0.5));
        vs[c] = vc;
        double xc = x[c];
        if (args.op != kEpiKick) xc = __dadd_rn(xc, __dmul_rn(vc, dt));
        xs[c] = xc;
        v[c] = vc;
        x[c] = xc;
    }
    if (args.op != kEpiKick)
        pair_put(args.xm_next, i, (float)xs[0], (float)xs[1], (float)xs[2],
                 pair_get(args.src, i, 3));
    if (args.ckpt) {
        double *ck = reinterpret_cast<double *>(args.ckpt) + 6 * i;
        ck[0] = xs[0]; ck[1] = xs[1]; ck[2] = xs[2];
        ck[3] = vs[0]; ck[4] = vs[1]; ck[5] = vs[2];
    }
}

// ------------------------------------------------------------ policies

// Plain FP32 force sum on the packed f32x2 pipe: each thread's i-body is held
// duplicated ({-x_i, -x_i}) and one record supplies two j-bodies, so one
// instruction evaluates the pair (i, j0), (i, j1). 12 FP32 operations and
// 1 MUFU rsqrt per interaction: 3 add (d), 3 fma (r^2 + eps^2), 3 mul
// (m y^3), 3 fma (accumulate).
struct AccelF32x2 {
    static constexpr int UNROLL = NB_UNROLL_OR(4);
    static constexpr bool SELF_MASK = false;
    static constexpr int REC_F4 = 2;
    static constexpr int PART_F4 = 1;
    static constexpr bool PER_TILE = false;
    struct I { float2 nx, ny, nz; };
    struct T { float2 x, y, z; };
    using A = T;
    struct F { float x, y, z; };
    struct C { float2 eps2; };
    __device__ static void consts(const ForceArgs &a, C &c) { c.eps2 = dup(a.eps2); }
    __device__ static void load_i(const ForceArgs &a, int64_t i, I &s) {
        s.nx = dup(-pair_get(a.src, i, 0));
        s.ny = dup(-pair_get(a.src, i, 1));
        s.nz = dup(-pair_get(a.src, i, 2));
    }
    __device__ static void zero_total(T &t) { t.x = t.y = t.z = f2(0.f, 0.f); }
    __device__ static void zero_acc(A &t) { zero_total(t); }
    __device__ static void tile_done(A &, T &) {}
    __device__ __forceinline__ static void interact(const float4 (&rec)[2], const I &s, T &t,
                                                    const C &c) {
        const float2 dx = __fadd2_rn(f2(rec[0].x, rec[0].y), s.nx);
        const float2 dy = __fadd2_rn(f2(rec[0].z, rec[0].w), s.ny);
        const float2 dz = __fadd2_rn(f2(rec[1].x, rec[1].y), s.nz);
        float2 q = __ffma2_rn(dx, dx, c.eps2);
        q = __ffma2_rn(dy, dy, q);
        q = __ffma2_rn(dz, dz, q);
        const float2 y = rsqrt_mufu2(q);
        const float2 y2 = __fmul2_rn(y, y);
        float2 w = __fmul2_rn(f2(rec[1].z, rec[1].w), y);
        w = __fmul2_rn(w, y2);
        t.x = __ffma2_rn(w, dx, t.x);
        t.y = __ffma2_rn(w, dy, t.y);
        t.z = __ffma2_rn(w, dz, t.z);
    }
    __device__ static void to_part(const T &t, float4 *dst) {
        *dst = make_float4(t.x.x + t.x.y, t.y.x + t.y.y, t.z.x + t.z.y, 0.f);
    }
    __device__ static void zero_final(F &f) { f.x = f.y = f.z = 0.f; }
    __device__ static void add_part(F &f, const float4 *src) {
        float4 p = __ldcg(src);
        f.x += p.x;
        f.y += p.y;
        f.z += p.z;
    }
    __device__ static void from_total(F &f, const T &t) {
        f.x = t.x.x + t.x.y;
        f.y = t.y.x + t.y.y;
        f.z = t.z.x + t.z.y;
    }
    __device__ static void finish(const ForceArgs &a, int64_t i, const F &f) {
        const float G = (float)a.G;
        finish_fp32(a, i, G * f.x, G * f.y, G * f.z);
    }
};

// Same sum with scalar FP32 instructions (one j-body at a time), kept as the
// baseline shape the autotuner can compare against.
struct AccelScalar {
    static constexpr int UNROLL = NB_UNROLL_OR(2);
    static constexpr bool SELF_MASK = false;
    static constexpr int REC_F4 = 2;
    static constexpr int PART_F4 = 1;
    static constexpr bool PER_TILE = false;
    struct I { float nx, ny, nz; };
    struct T { float x, y, z; };
    using A = T;
    using F = AccelF32x2::F;
    struct C { float eps2; };
    __device__ static void consts(const ForceArgs &a, C &c) { c.eps2 = a.eps2; }
    __device__ static void load_i(const ForceArgs &a, int64_t i, I &s) {
        s.nx = -pair_get(a.src, i, 0);
        s.ny = -pair_get(a.src, i, 1);
        s.nz = -pair_get(a.src, i, 2);
    }
    __device__ static void zero_total(T &t) { t.x = t.y = t.z = 0.f; }
    __device__ static void zero_acc(A &t) { zero_total(t); }
    __device__ static void tile_done(A &, T &) {}
    __device__ __forceinline__ static void one(float xj, float yj, float zj, float mj, const I &s,
                                               T &t, float eps2) {
        const float dx = xj + s.nx, dy = yj + s.ny, dz = zj + s.nz;
        float q = fmaf(dx, dx, eps2);
        q = fmaf(dy, dy, q);
        q = fmaf(dz, dz, q);
        const float y = rsqrt_mufu(q);
        const float w = (mj * y) * (y * y);
        t.x = fmaf(w, dx, t.x);
        t.y = fmaf(w, dy, t.y);
        t.z = fmaf(w, dz, t.z);
    }
    __device__ __forceinline__ static void interact(const float4 (&rec)[2], const I &s, T &t,
                                                    const C &c) {
        one(rec[0].x, rec[0].z, rec[1].x, rec[1].z, s, t, c.eps2);
        one(rec[0].y, rec[0].w, rec[1].y, rec[1].w, s, t, c.eps2);
    }
    __device__ static void to_part(const T &t, float4 *dst) { *dst = make_float4(t.x, t.y, t.z, 0.f); }
    __device__ static void zero_final(F &f) { f.x = f.y = f.z = 0.f; }
    __device__ static void add_part(F &f, const float4 *src) { AccelF32x2::add_part(f, src); }
    __device__ static void from_total(F &f, const T &t) {
        f.x = t.x;
        f.y = t.y;
        f.z = t.z;
    }
    __device__ static void finish(const ForceArgs &a, int64_t i, const F &f) {
        const float G = (float)a.G;
        finish_fp32(a, i, G * f.x, G * f.y, G * f.z);
    }
};

// Ablation of the denominator (s^(3/2) with s = |d|^2 + eps^2), the GPU
// analog of the paper's math-operation experiment (Sections 3.2.6, 3.3.6):
//   kMath = 1: power then divide, w = m / (s * sqrt(s)) with IEEE sqrt and
//              IEEE division (the listings' `dsquared ** -1.5` evaluated as
//              a positive power and a division);
//   kMath = 2: the power function, w = m * powf(s, -1.5).
// Scalar FP32; otherwise identical to AccelScalar.
template <int kMath>
struct AccelMath {
    static constexpr int UNROLL = NB_UNROLL_OR(2);
    static constexpr bool SELF_MASK = false;
    static constexpr int REC_F4 = 2;
    static constexpr int PART_F4 = 1;
    static constexpr bool PER_TILE = false;
    using I = AccelScalar::I;
    using T = AccelScalar::T;
    using A = T;
    using F = AccelScalar::F;
    using C = AccelScalar::C;
    __device__ static void consts(const ForceArgs &a, C &c) { c.eps2 = a.eps2; }
    __device__ static void load_i(const ForceArgs &a, int64_t i, I &s) { AccelScalar::load_i(a, i, s); }
    __device__ static void zero_total(T &t) { t.x = t.y = t.z = 0.f; }
    __device__ static void zero_acc(A &t) { zero_total(t); }
    __device__ static void tile_done(A &, T &) {}
    __device__ __forceinline__ static void one(float xj, float yj, float zj, float mj, const I &s,
                                               T &t, float eps2) {
        const float dx = xj + s.nx, dy = yj + s.ny, dz = zj + s.nz;
        float q = fmaf(dx, dx, eps2);
        q = fmaf(dy, dy, q);
        q = fmaf(dz, dz, q);
        float w;
        if constexpr (kMath == 1)
            w = __fdiv_rn(mj, __fmul_rn(q, __fsqrt_rn(q)));
        else
            w = mj * powf(q, -1.5f);
        t.x = fmaf(w, dx, t.x);
        t.y = fmaf(w, dy, t.y);
        t.z = fmaf(w, dz, t.z);
    }
    __device__ __forceinline__ static void interact(const float4 (&rec)[2], const I &s, T &t,
                                                    const C &c) {
        one(rec[0].x, rec[0].z, rec[1].x, rec[1].z, s, t, c.eps2);
        one(rec[0].y, rec[0].w, rec[1].y, rec[1].w, s, t, c.eps2);
    }
    __device__ static void to_part(const T &t, float4 *dst) { AccelScalar::to_part(t, dst); }
    __device__ static void zero_final(F &f) { AccelScalar::zero_final(f); }
    __device__ static void add_part(F &f, const float4 *src) { AccelScalar::add_part(f, src); }
    __device__ static void from_total(F &f, const T &t) { AccelScalar::from_total(f, t); }
    __device__ static void finish(const ForceArgs &a, int64_t i, const F &f) { AccelScalar::finish(a, i, f); }
};

// Precision form: FP32 pair terms (optionally one Newton-Raphson refinement
// of the MUFU reciprocal square root, y <- y (3/2 - s y^2 / 2), see
// NB_COMP_NEWTON), plain FP32 sums within a j-tile, and the per-tile sums
// folded into a (hi, lo) pair with Knuth's two-sum. Split partials carry
// (hi, lo) and are folded the same way in split order; the sum is widened to
// FP64 once, and the update runs in FP64.
struct AccelComp {
    static constexpr int UNROLL = NB_UNROLL_OR(1);
    static constexpr bool SELF_MASK = false;
    static constexpr int REC_F4 = 2;
    static constexpr int PART_F4 = 2;
    static constexpr bool PER_TILE = true;
    using I = AccelF32x2::I;
    struct A { float2 x, y, z; };
    struct T { float hx, hy, hz, lx, ly, lz; };
    using F = T;  // across splits: the same (hi, lo) two-sums, widened to FP64 once
    struct C { float2 eps2, mhalf, three_half; };
    __device__ static void consts(const ForceArgs &a, C &c) {
        c.eps2 = dup(a.eps2);
        c.mhalf = dup(-0.5f);
        c.three_half = dup(1.5f);
    }
    __device__ static void load_i(const ForceArgs &a, int64_t i, I &s) { AccelF32x2::load_i(a, i, s); }
    __device__ static void zero_total(T &t) { t.hx = t.hy = t.hz = t.lx = t.ly = t.lz = 0.f; }
    __device__ static void zero_acc(A &t) { t.x = t.y = t.z = f2(0.f, 0.f); }
    __device__ __forceinline__ static void interact(const float4 (&rec)[2], const I &s, A &t,
                                                    const C &c) {
        const float2 dx = __fadd2_rn(f2(rec[0].x, rec[0].y), s.nx);
        const float2 dy = __fadd2_rn(f2(rec[0].z, rec[0].w), s.ny);
        const float2 dz = __fadd2_rn(f2(rec[1].x, rec[1].y), s.nz);
        float2 q = __ffma2_rn(dx, dx, c.eps2);
        q = __ffma2_rn(dy, dy, q);
        q = __ffma2_rn(dz, dz, q);
        float2 y = rsqrt_mufu2(q);
#if NB_COMP_NEWTON
        // one Newton step for q^(-1/2): y <- y (3/2 - q y^2 / 2)
        const float2 tq = __fmul2_rn(__fmul2_rn(q, c.mhalf), y);
        y = __fmul2_rn(y, __ffma2_rn(tq, y, c.three_half));
#endif
        const float2 y2 = __fmul2_rn(y, y);
        float2 w = __fmul2_rn(f2(rec[1].z, rec[1].w), y);
        w = __fmul2_rn(w, y2);
        t.x = __ffma2_rn(w, dx, t.x);
        t.y = __ffma2_rn(w, dy, t.y);
        t.z = __ffma2_rn(w, dz, t.z);
    }
    __device__ static void tile_done(const A &a, T &t) {
        float s, e;
        two_sum(t.hx, a.x.x + a.x.y, s, e); t.hx = s; t.lx += e;
        two_sum(t.hy, a.y.x + a.y.y, s, e); t.hy = s; t.ly += e;
        two_sum(t.hz, a.z.x + a.z.y, s, e); t.hz = s; t.lz += e;
    }
    __device__ static void to_part(const T &t, float4 *dst) {
        dst[0] = make_float4(t.hx, t.hy, t.hz, 0.f);
        dst[1] = make_float4(t.lx, t.ly, t.lz, 0.f);
    }
    __device__ static void zero_final(F &f) { zero_total(f); }
    // One split's (hi, lo) partial into the running (hi, lo): the FP32
    // two-sum keeps about 2^-44 relative, and the FP64 pipe (slow on this
    // part) is left to the update.
    __device__ static void add_part(F &f, const float4 *src) {
        const float4 h = __ldcg(src), l = __ldcg(src + 1);
        float s, e;
        two_sum(f.hx, h.x, s, e); f.hx = s; f.lx = __fadd_rn(f.lx, __fadd_rn(l.x, e));
        two_sum(f.hy, h.y, s, e); f.hy = s; f.ly = __fadd_rn(f.ly, __fadd_rn(l.y, e));
        two_sum(f.hz, h.z, s, e); f.hz = s; f.lz = __fadd_rn(f.lz, __fadd_rn(l.z, e));
    }
    __device__ static void from_total(F &f, const T &t) { f = t; }
    __device__ static void finish(const ForceArgs &a, int64_t i, const F &f) {
        finish_fp64(a, i, a.G * ((double)f.hx + (double)f.lx), a.G * ((double)f.hy + (double)f.ly),
                    a.G * ((double)f.hz + (double)f.lz));
    }
};

// Softened potential per body, phi_i = sum_j m_j / sqrt(|d|^2 + eps^2) with
// FP32 pair terms, FP32 sums within a tile, FP64 sums across tiles. The
// epilogue removes the j = i term (m_i / eps, evaluated with the same FP32
// operations the loop used) and writes m_i * phi_i as a double.
struct Potential {
    static constexpr int UNROLL = NB_UNROLL_OR(2);
    static constexpr bool SELF_MASK = false;
    static constexpr int REC_F4 = 2;
    static constexpr int PART_F4 = 1;
    static constexpr bool PER_TILE = true;
    using I = AccelF32x2::I;
    struct A { float2 p; };
    struct T { double p; };
    struct F { double p; };
    struct C { float2 eps2; };
    __device__ static void consts(const ForceArgs &a, C &c) { c.eps2 = dup(a.eps2); }
    __device__ static void load_i(const ForceArgs &a, int64_t i, I &s) { AccelF32x2::load_i(a, i, s); }
    __device__ static void zero_total(T &t) { t.p = 0.0; }
    __device__ static void zero_acc(A &t) { t.p = f2(0.f, 0.f); }
    __device__ __forceinline__ static void interact(const float4 (&rec)[2], const I &s, A &t,
                                                    const C &c) {
        const float2 dx = __fadd2_rn(f2(rec[0].x, rec[0].y), s.nx);
        const float2 dy = __fadd2_rn(f2(rec[0].z, rec[0].w), s.ny);
        const float2 dz = __fadd2_rn(f2(rec[1].x, rec[1].y), s.nz);
        float2 q = __ffma2_rn(dx, dx, c.eps2);
        q = __ffma2_rn(dy, dy, q);
        q = __ffma2_rn(dz, dz, q);
        const float2 y = rsqrt_mufu2(q);
        t.p = __ffma2_rn(f2(rec[1].z, rec[1].w), y, t.p);
    }
    __device__ static void tile_done(const A &a, T &t) { t.p += (double)a.p.x + (double)a.p.y; }
    __device__ static void to_part(const T &t, float4 *dst) {
        *reinterpret_cast<double2 *>(dst) = make_double2(t.p, 0.0);
    }
    __device__ static void zero_final(F &f) { f.p = 0.0; }
    __device__ static void add_part(F &f, const float4 *src) {
        f.p += __ldcg(reinterpret_cast<const double2 *>(src)).x;
    }
    __device__ static void from_total(F &f, const T &t) { f.p = t.p; }
    __device__ static void finish(const ForceArgs &a, int64_t i, const F &f) {
        const float mi = pair_get(a.src, i, 3);
        const float self = __fmul_rn(mi, rsqrt_mufu(a.eps2));
        reinterpret_cast<double *>(a.out)[i] = (double)mi * (f.p - (double)self);
    }
};

// Adjoint vector-Jacobian product of the force sum. For the i-body k and
// every j (d = x_j - x_k, s = |d|^2 + eps^2, f = s^-3/2, h = s^-5/2,
// e = abar_j . d, g = abar_k . d):
//   U += f abar_j,  V += f m_j,  W += h (m_j g - m_k e) d,  P += f e
// and the epilogue forms
//   xbar_k += G (m_k U - V abar_k + 3 W),   mbar_k += -G P,
// which equals G sum_j K(d)(m_k abar_j - m_j abar_k) and
// -G sum_j f abar_j . d with K(d) = f I - 3 h d d^T. 27 FP32 operations and
// one MUFU rsqrt per pair. The j == k pair is masked (its f = eps^-3 terms
// would cancel only in the epilogue).
//
// Adjoint records, 4 float4 per pair of bodies:
//   {x0,x1,y0,y1} {z0,z1,m0,m1} {ax0,ax1,ay0,ay1} {az0,az1,0,0}
struct VjpF32x2 {
    static constexpr int UNROLL = NB_UNROLL_OR(2);
    static constexpr bool SELF_MASK = true;
    static constexpr int REC_F4 = 4;
    static constexpr int PART_F4 = 2;
    static constexpr bool PER_TILE = false;
    struct I { float2 nx, ny, nz, ax, ay, az, nm; };  // nm = -m_k
    struct T { float2 ux, uy, uz, v, wx, wy, wz, p; };
    using A = T;
    struct F { float ux, uy, uz, v, wx, wy, wz, p; };
    struct C { float2 eps2; };
    __device__ static void consts(const ForceArgs &a, C &c) { c.eps2 = dup(a.eps2); }
    __device__ static void load_i(const ForceArgs &a, int64_t i, I &s) {
        s.nx = dup(-vrec_get(a.src, i, 0));
        s.ny = dup(-vrec_get(a.src, i, 1));
        s.nz = dup(-vrec_get(a.src, i, 2));
        s.nm = dup(-vrec_get(a.src, i, 3));
        s.ax = dup(vrec_get(a.src, i, 4));
        s.ay = dup(vrec_get(a.src, i, 5));
        s.az = dup(vrec_get(a.src, i, 6));
    }
    __device__ static void zero_total(T &t) {
        t.ux = t.uy = t.uz = t.v = t.wx = t.wy = t.wz = t.p = f2(0.f, 0.f);
    }
    __device__ static void zero_acc(A &t) { zero_total(t); }
    __device__ static void tile_done(A &, T &) {}
    // Pair terms from the separation (dx, dy, dz); y = s^-1/2 (already masked).
    __device__ __forceinline__ static void terms(float2 dx, float2 dy, float2 dz, float2 y,
                                                 float2 mj, float2 ajx, float2 ajy, float2 ajz,
                                                 const I &s, T &t) {
        const float2 y2 = __fmul2_rn(y, y);
        const float2 f = __fmul2_rn(y, y2);
        const float2 h = __fmul2_rn(f, y2);
        float2 e = __fmul2_rn(ajx, dx);
        e = __ffma2_rn(ajy, dy, e);
        e = __ffma2_rn(ajz, dz, e);
        float2 g = __fmul2_rn(s.ax, dx);
        g = __ffma2_rn(s.ay, dy, g);
        g = __ffma2_rn(s.az, dz, g);
        const float2 c = __ffma2_rn(mj, g, __fmul2_rn(s.nm, e));  // m_j g - m_k e
        const float2 hc = __fmul2_rn(h, c);
        t.wx = __ffma2_rn(hc, dx, t.wx);
        t.wy = __ffma2_rn(hc, dy, t.wy);
        t.wz = __ffma2_rn(hc, dz, t.wz);
        t.ux = __ffma2_rn(f, ajx, t.ux);
        t.uy = __ffma2_rn(f, ajy, t.uy);
        t.uz = __ffma2_rn(f, ajz, t.uz);
        t.v = __ffma2_rn(f, mj, t.v);
        t.p = __ffma2_rn(f, e, t.p);
    }
    template <bool MASK>
    __device__ __forceinline__ static void pair(const float4 (&rec)[4], const I &s, T &t,
                                                float2 eps2, float2 keep) {
        const float2 dx = __fadd2_rn(f2(rec[0].x, rec[0].y), s.nx);
        const float2 dy = __fadd2_rn(f2(rec[0].z, rec[0].w), s.ny);
        const float2 dz = __fadd2_rn(f2(rec[1].x, rec[1].y), s.nz);
        float2 q = __ffma2_rn(dx, dx, eps2);
        q = __ffma2_rn(dy, dy, q);
        q = __ffma2_rn(dz, dz, q);
        float2 y = rsqrt_mufu2(q);
        if constexpr (MASK) y = __fmul2_rn(y, keep);
        terms(dx, dy, dz, y, f2(rec[1].z, rec[1].w), f2(rec[2].x, rec[2].y),
              f2(rec[2].z, rec[2].w), f2(rec[3].x, rec[3].y), s, t);
    }
    __device__ __forceinline__ static void interact(const float4 (&rec)[4], const I &s, T &t,
                                                    const C &c) {
        pair<false>(rec, s, t, c.eps2, dup(1.f));
    }
    __device__ __forceinline__ static void interact_masked(const float4 (&rec)[4], const I &s,
                                                           T &t, const C &c, float2 keep) {
        pair<true>(rec, s, t, c.eps2, keep);
    }
    __device__ static void to_part(const T &t, float4 *dst) {
        dst[0] = make_float4(t.ux.x + t.ux.y, t.uy.x + t.uy.y, t.uz.x + t.uz.y, t.v.x + t.v.y);
        dst[1] = make_float4(t.wx.x + t.wx.y, t.wy.x + t.wy.y, t.wz.x + t.wz.y, t.p.x + t.p.y);
    }
    __device__ static void zero_final(F &f) {
        f.ux = f.uy = f.uz = f.v = f.wx = f.wy = f.wz = f.p = 0.f;
    }
    __device__ static void add_part(F &f, const float4 *src) {
        const float4 a = __ldcg(src), b = __ldcg(src + 1);
        f.ux += a.x; f.uy += a.y; f.uz += a.z; f.v += a.w;
        f.wx += b.x; f.wy += b.y; f.wz += b.z; f.p += b.w;
    }
    __device__ static void from_total(F &f, const T &t) {
        float4 tmp[2];
        to_part(t, tmp);
        f.ux = tmp[0].x; f.uy = tmp[0].y; f.uz = tmp[0].z; f.v = tmp[0].w;
        f.wx = tmp[1].x; f.wy = tmp[1].y; f.wz = tmp[1].z; f.p = tmp[1].w;
    }
    __device__ static void finish(const ForceArgs &a, int64_t k, const F &f) {
        const float G = (float)a.G;
        const float mk = vrec_get(a.src, k, 3);
        const float ak[3] = {vrec_get(a.src, k, 4), vrec_get(a.src, k, 5), vrec_get(a.src, k, 6)};
        const float u[3] = {f.ux, f.uy, f.uz}, w[3] = {f.wx, f.wy, f.wz};
        float *xb = reinterpret_cast<float *>(a.xbar) + 3 * k;
#pragma unroll
        for (int c = 0; c < 3; ++c) xb[c] += G * (mk * u[c] - f.v * ak[c] + 3.f * w[c]);
        reinterpret_cast<float *>(a.mbar)[k] += -G * f.p;
        if (a.prep_next) {  // the next step's record half of body k (its mass stays)
            float *vb = reinterpret_cast<float *>(a.vbar) + 3 * k;
            const float dt = (float)a.dt;
            float an[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float vn = vb[c] + dt * xb[c];  // vbar' = vbar + dt xbar
                vb[c] = vn;
                an[c] = dt / 2.0f * vn;               // abar = dt/2 vbar'
            }
            float *p = reinterpret_cast<float *>(const_cast<float4 *>(a.src) + (k >> 1) * 4);
            const int h = (int)(k & 1);
            p[0 + h] = pair_get(a.next_xm, k, 0);
            p[2 + h] = pair_get(a.next_xm, k, 1);
            p[4 + h] = pair_get(a.next_xm, k, 2);
            p[8 + h] = an[0];
            p[10 + h] = an[1];
            p[12 + h] = an[2];
        }
    }
};

// Precision form of the VJP. Positions enter as FP32 (hi, lo) pairs of the
// FP64 state, and d = (x_j^hi - x_k^hi) + (x_j^lo - x_k^lo) keeps its
// relative error at FP32 rounding even for close pairs (whose terms weigh
// as |d|^-3); the rsqrt is refined only with NB_COMP_NEWTON; sums are FP32 within a tile
// and two-summed (hi, lo) across tiles and splits; the epilogue widens them
// and runs in FP64 with FP64 m_k and abar_k. Records, 5 float4 per pair of bodies:
//   {x0,x1,y0,y1} {z0,z1,m0,m1} {ax0,ax1,ay0,ay1} {az0,az1,xl0,xl1} {yl0,yl1,zl0,zl1}
struct VjpComp {
    static constexpr int UNROLL = NB_UNROLL_OR(2);
    static constexpr bool SELF_MASK = true;
    static constexpr int REC_F4 = 5;
    static constexpr int PART_F4 = 4;
    static constexpr bool PER_TILE = true;
    struct I {
        VjpF32x2::I b;
        float2 nlx, nly, nlz;
    };
    using A = VjpF32x2::T;
    struct T { float h[8], l[8]; };
    using F = T;  // across splits: the same (hi, lo) two-sums, widened to FP64 in finish
    struct C { float2 eps2, mhalf, three_half; };
    __device__ static void consts(const ForceArgs &a, C &c) {
        c.eps2 = dup(a.eps2);
        c.mhalf = dup(-0.5f);
        c.three_half = dup(1.5f);
    }
    __device__ static float get(const float4 *base, int64_t i, int c) {
        const float *p = reinterpret_cast<const float *>(base + (i >> 1) * 5);
        return p[2 * c + (int)(i & 1)];
    }
    __device__ static void load_i(const ForceArgs &a, int64_t i, I &s) {
        s.b.nx = dup(-get(a.src, i, 0));
        s.b.ny = dup(-get(a.src, i, 1));
        s.b.nz = dup(-get(a.src, i, 2));
        s.b.nm = dup(-get(a.src, i, 3));
        s.b.ax = dup(get(a.src, i, 4));
        s.b.ay = dup(get(a.src, i, 5));
        s.b.az = dup(get(a.src, i, 6));
        s.nlx = dup(-get(a.src, i, 7));
        s.nly = dup(-get(a.src, i, 8));
        s.nlz = dup(-get(a.src, i, 9));
    }
    __device__ static void zero_total(T &t) {
#pragma unroll
        for (int k = 0; k < 8; ++k) t.h[k] = t.l[k] = 0.f;
    }
    __device__ static void zero_acc(A &t) { VjpF32x2::zero_total(t); }
    template <bool MASK>
    __device__ __forceinline__ static void pair(const float4 (&rec)[5], const I &s, A &t,
                                                const C &c, float2 keep) {
        const float2 dx = __fadd2_rn(__fadd2_rn(f2(rec[0].x, rec[0].y), s.b.nx),
                                     __fadd2_rn(f2(rec[3].z, rec[3].w), s.nlx));
        const float2 dy = __fadd2_rn(__fadd2_rn(f2(rec[0].z, rec[0].w), s.b.ny),
                                     __fadd2_rn(f2(rec[4].x, rec[4].y), s.nly));
        const float2 dz = __fadd2_rn(__fadd2_rn(f2(rec[1].x, rec[1].y), s.b.nz),
                                     __fadd2_rn(f2(rec[4].z, rec[4].w), s.nlz));
        float2 q = __ffma2_rn(dx, dx, c.eps2);
        q = __ffma2_rn(dy, dy, q);
        q = __ffma2_rn(dz, dz, q);
        float2 y = rsqrt_mufu2(q);
#if NB_COMP_NEWTON
        const float2 tq = __fmul2_rn(__fmul2_rn(q, c.mhalf), y);
        y = __fmul2_rn(y, __ffma2_rn(tq, y, c.three_half));
#endif
        if constexpr (MASK) y = __fmul2_rn(y, keep);
        VjpF32x2::terms(dx, dy, dz, y, f2(rec[1].z, rec[1].w), f2(rec[2].x, rec[2].y),
                        f2(rec[2].z, rec[2].w), f2(rec[3].x, rec[3].y), s.b, t);
    }
    __device__ __forceinline__ static void interact(const float4 (&rec)[5], const I &s, A &t,
                                                    const C &c) {
        pair<false>(rec, s, t, c, dup(1.f));
    }
    __device__ __forceinline__ static void interact_masked(const float4 (&rec)[5], const I &s,
                                                           A &t, const C &c, float2 keep) {
        pair<true>(rec, s, t, c, keep);
    }
    __device__ static void tile_done(const A &a, T &t) {
        const float v[8] = {a.ux.x + a.ux.y, a.uy.x + a.uy.y, a.uz.x + a.uz.y, a.v.x + a.v.y,
                            a.wx.x + a.wx.y, a.wy.x + a.wy.y, a.wz.x + a.wz.y, a.p.x + a.p.y};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float s, e;
            two_sum(t.h[k], v[k], s, e);
            t.h[k] = s;
            t.l[k] += e;
        }
    }
    __device__ static void to_part(const T &t, float4 *dst) {
        dst[0] = make_float4(t.h[0], t.h[1], t.h[2], t.h[3]);
        dst[1] = make_float4(t.h[4], t.h[5], t.h[6], t.h[7]);
        dst[2] = make_float4(t.l[0], t.l[1], t.l[2], t.l[3]);
        dst[3] = make_float4(t.l[4], t.l[5], t.l[6], t.l[7]);
    }
    __device__ static void zero_final(F &f) { zero_total(f); }
    // One split's (hi, lo) partials into the running (hi, lo) with FP32
    // two-sums (about 2^-44 relative), in split order.
    __device__ static void add_part(F &f, const float4 *src) {
        const float4 h0 = __ldcg(src), h1 = __ldcg(src + 1), l0 = __ldcg(src + 2),
                     l1 = __ldcg(src + 3);
        const float hh[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
        const float ll[8] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float s, e;
            two_sum(f.h[k], hh[k], s, e);
            f.h[k] = s;
            f.l[k] = __fadd_rn(f.l[k], __fadd_rn(ll[k], e));
        }
    }
    __device__ static void from_total(F &f, const T &t) { f = t; }
    __device__ static void finish(const ForceArgs &a, int64_t k, const F &f) {
        double fs[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) fs[q] = (double)f.h[q] + (double)f.l[q];
        const double G = a.G;
        const double mk = reinterpret_cast<const double *>(a.mass)[k];
        const double *ak = reinterpret_cast<const double *>(a.abar64) + 3 * k;
        double *xb = reinterpret_cast<double *>(a.xbar) + 3 * k;
#pragma unroll
        for (int c = 0; c < 3; ++c) xb[c] += G * (mk * fs[c] - fs[3] * ak[c] + 3.0 * fs[4 + c]);
        reinterpret_cast<double *>(a.mbar)[k] += -G * fs[7];
        if (a.prep_next) {  // the next step's record half of body k (its mass stays)
            double *vb = reinterpret_cast<double *>(a.vbar) + 3 * k;
            double *an = const_cast<double *>(ak);
            const double dt = a.dt;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double vn = vb[c] + dt * xb[c];
                vb[c] = vn;
                an[c] = dt / 2.0 * vn;
            }
            float hi[3], lo[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double xc = a.next_x64[(int64_t)6 * k + c];
                hi[c] = (float)xc;
                lo[c] = (float)(xc - (double)hi[c]);
            }
            float *p = reinterpret_cast<float *>(const_cast<float4 *>(a.src) + (k >> 1) * 5);
            const int h = (int)(k & 1);
            p[0 + h] = hi[0];
            p[2 + h] = hi[1];
            p[4 + h] = hi[2];
            p[8 + h] = (float)an[0];
            p[10 + h] = (float)an[1];
            p[12 + h] = (float)an[2];
            p[14 + h] = lo[0];
            p[16 + h] = lo[1];
            p[18 + h] = lo[2];
        }
    }
};

}  // namespace nb
