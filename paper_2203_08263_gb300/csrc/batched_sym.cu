// Pair-symmetric ensemble kernel: every system of the batch advances `steps`
// steps inside one cooperative launch, each unordered pair of each system
// evaluated once for both bodies (the force terms of csrc/k_sym.cu).
//
// Work items, per system s and step t: every system is cut into groups of
// G = 256 bodies (padded with zero-mass bodies); a pair item (s, gi, gj),
// gi <= gj, sums the terms of all pairs between groups gi and gj into
// block-pair partials, and an epilogue item (s, g) adds group g's partials in
// group order and runs the update (half kick, drift, repack; the precision
// form two-sums the partials and updates in FP64). Items are numbered
// step-major; within a step the pair items come largest systems first, and
// each system's epilogue items follow its last pair item after a lag of
// about five times the grid's warps (in items), or at the step's end. A pair
// item of step t waits for every epilogue item of
// step t-1 of its system (the positions it reads), an epilogue item for every
// pair item of step t of its system (the partials it reads); both are lower
// numbers, so the oldest unfinished item is always ready and the queue always
// makes progress.
//
// A diagonal item (gi == gj) evaluates each unordered pair of its group about
// once (pair_item_diag: the off-diagonal 32 x 64 squares of the group take
// both sides of each pair, the 64 x 64 squares on the diagonal every ordered
// pair from the i side), 20 of the 32 squares an off-diagonal item evaluates.
//
// The unit of work is a warp: each warp of the persistent grid takes item
// numbers from one atomic counter, holds up to kHoldW of them (one by
// default) and runs the lowest-numbered ready one; it takes the next number
// while an item runs, so the atomic's latency is hidden, and keeps its queue
// state in shared memory, so the pair loop keeps its registers. In a pair item the warp holds the 256 bodies of
// group gi, 8 per lane, duplicated in f32x2 registers; group gj's 128 pair
// records go round the warp in four chunks of 32, one record per lane, for 32
// rounds each, carrying their running j-side sums with them (shuffles); after
// a chunk every record is home and its lane stores the sums. All reads of
// data written during the launch (positions, partials) go through L2.
#include <algorithm>
#include <cstring>

#include "batched.h"
#include "kernels.h"

namespace nb {

namespace {

// bodies per group: 32 lanes x kGR (groups of 128, 4 per lane: 105,902 items per step of the
// 512-system ensemble against 29,917, 3.04e12 interactions/s against 3.36e12 at 16 warps per SM,
// 2.93e12 at 20)
constexpr int kGrp = 256;
constexpr int kGR = 8;
constexpr int kSymWarps = 4;  // warps per CTA
#ifndef NB_SYMB_HOLD
#define NB_SYMB_HOLD 1  // measured on the 512-system ensemble: 3.15e12-3.17e12 interactions/s at 1, 2.99e12-3.01e12 at 2, 2.93e12 at 4, 2.92e12 at 8
#endif
constexpr int kHoldW = NB_SYMB_HOLD;  // items a warp may hold unstarted
constexpr unsigned kNone = 0xFFFFFFFFu;
#ifndef NB_SYMB_EPI_LAG
// measured on the 512-system ensemble (1,824 warps, 29,917 items per step):
// 3.37e12 interactions/s with every epilogue item after every pair item (0);
// 3.02e12 / 3.11e12 / 3.26e12 at lags of 0.5 / 1 / 2 grid-warps of items
// (epilogue items taken while their system's pair items still run wait for
// them), 3.37e12 at 3, 3.42e12 at 4 to 6, 3.41e12 at 8 and 11 (the partials
// read soon after they were written, from L2)
#define NB_SYMB_EPI_LAG 5.0
#endif
#ifndef NB_SYMB_MINB
#define NB_SYMB_MINB 3  // resident CTAs per SM the FP32 kernel's registers are sized for (4: 128 registers, 3.15e12 interactions/s on the 512-system ensemble against 3.37e12 at 3, even with the epilogue and diagonal items out of line and no record prefetch)
#endif

struct SymBatchArgs {
    const int64_t *off;    // [nsys + 1] body offsets
    const int64_t *poff;   // [nsys] offsets of the packed systems (bodies, multiples of kGrp)
    const int64_t *pofs;   // [nsys] offsets of the systems' partials (floats)
    const int *ng;         // [nsys] groups
    const int *npairs;     // [nsys] pair items per step
    const int4 *items;     // [items_per_step] {system, gi, gj, kind: 0 pair, 1 epilogue}
    unsigned *next;        // queue head
    unsigned *pair_done;   // [nsys] pair items completed, cumulative over steps
    unsigned *fin_done;    // [nsys] epilogue items completed, cumulative
    float4 *xm0, *xm1;
    float *part;
    void *x, *v;
    int steps, items_per_step, kdk;
    float eps2, G, dt;
    double Gd, dtd;
    int *err;
    uint64_t timeout_ns;
    int stall;  // debug: warp 0 of CTA 0 never releases its first item
};

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ float2 shfl2(float2 v, int src) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

__device__ __forceinline__ float pget_cg(const float4 *base, int64_t i, int c) {
    const float *p = reinterpret_cast<const float *>(base + (i >> 1) * 2);
    return __ldcg(p + 2 * c + (int)(i & 1));
}

// Pairs between groups gi and gj of one system (positions `src`, partials
// P[p][c][b] with npad bodies per row).
__device__ __forceinline__ void pair_item(const SymBatchArgs &a, const float4 *src, float *P,
                                          int64_t npad, int gi, int gj, int lane) {
    const int next = (lane + 1) & 31;
    const float2 eps2 = dup(a.eps2);
    float2 nx[kGR], ny[kGR], nz[kGR], mi[kGR], ax[kGR], ay[kGR], az[kGR];
    const int64_t ib = (int64_t)gi * kGrp + lane;
#pragma unroll
    for (int r = 0; r < kGR; ++r) {
        const int64_t i = ib + 32 * r;
        nx[r] = dup(-pget_cg(src, i, 0));
        ny[r] = dup(-pget_cg(src, i, 1));
        nz[r] = dup(-pget_cg(src, i, 2));
        mi[r] = dup(pget_cg(src, i, 3));
        ax[r] = ay[r] = az[r] = f2(0.f, 0.f);
    }
    // each lane's record of chunk ch + 1 is loaded while chunk ch runs
    const float4 *qsrc = src + 2 * ((int64_t)gj * (kGrp / 2) + lane);
    float4 n0 = __ldcg(qsrc), n1 = __ldcg(qsrc + 1);
    for (int ch = 0; ch < kGrp / 64; ++ch) {
        const float4 r0 = n0, r1 = n1;
        if (ch + 1 < kGrp / 64) {
            n0 = __ldcg(qsrc + 64 * (ch + 1));
            n1 = __ldcg(qsrc + 64 * (ch + 1) + 1);
        }
        float2 xj = f2(r0.x, r0.y), yj = f2(r0.z, r0.w), zj = f2(r1.x, r1.y), mj = f2(r1.z, r1.w);
        float2 bx = f2(0.f, 0.f), by = bx, bz = bx;
#pragma unroll 1
        for (int round = 0; round < 32; ++round) {
#pragma unroll
            for (int r = 0; r < kGR; ++r) {
                const float2 dx = __fadd2_rn(xj, nx[r]);
                const float2 dy = __fadd2_rn(yj, ny[r]);
                const float2 dz = __fadd2_rn(zj, nz[r]);
                float2 s = __ffma2_rn(dx, dx, eps2);
                s = __ffma2_rn(dy, dy, s);
                s = __ffma2_rn(dz, dz, s);
                const float2 y = rsqrt_mufu2(s);
                const float2 y3 = __fmul2_rn(__fmul2_rn(y, y), y);
                const float2 wi = __fmul2_rn(mj, y3);  // j on i: +m_j s^-3/2 d
                ax[r] = __ffma2_rn(wi, dx, ax[r]);
                ay[r] = __ffma2_rn(wi, dy, ay[r]);
                az[r] = __ffma2_rn(wi, dz, az[r]);
                const float2 wj = __fmul2_rn(mi[r], y3);  // i on j: -m_i s^-3/2 d (sign at the store)
                bx = __ffma2_rn(wj, dx, bx);
                by = __ffma2_rn(wj, dy, by);
                bz = __ffma2_rn(wj, dz, bz);
            }
            xj = shfl2(xj, next);
            yj = shfl2(yj, next);
            zj = shfl2(zj, next);
            mj = shfl2(mj, next);
            bx = shfl2(bx, next);
            by = shfl2(by, next);
            bz = shfl2(bz, next);
        }
        {  // j side: row gi of the partials, bodies of group gj
            float *p = P + (int64_t)gi * 3 * npad + (int64_t)gj * kGrp + ch * 64 + 2 * lane;
            __stcg(reinterpret_cast<float2 *>(p), f2(-bx.x, -bx.y));
            __stcg(reinterpret_cast<float2 *>(p + npad), f2(-by.x, -by.y));
            __stcg(reinterpret_cast<float2 *>(p + 2 * npad), f2(-bz.x, -bz.y));
        }
    }
    float *p = P + (int64_t)gj * 3 * npad + ib;  // i side: row gj, bodies of group gi
#pragma unroll
    for (int r = 0; r < kGR; ++r) {
        __stcg(p + 32 * r, ax[r].x + ax[r].y);
        __stcg(p + npad + 32 * r, ay[r].x + ay[r].y);
        __stcg(p + 2 * npad + 32 * r, az[r].x + az[r].y);
    }
}

// The diagonal item (gi == gj) with each unordered pair evaluated about
// once: in chunk CH (j-bodies 64 CH ... 64 CH + 63) the lane's i-bodies of
// sub-block r (bodies 32 r + lane) take both sides of the pair for r < 2 CH
// (all those j-bodies are higher), the i side only for r = 2 CH, 2 CH + 1
// (the 64 x 64 block on the diagonal, every ordered pair; the own pair adds
// 0), and nothing for r > 2 CH + 1 (those pairs are the mirror images of
// ones already taken). The j-side sums of a chunk wait in `stage` and join
// the i-side sums of the same bodies before the one partial of row gi is
// stored.
template <int CH>
__device__ __forceinline__ void diag_chunk(const float4 *src, int gi, int lane, float2 eps2,
                                           const float2 (&nx)[kGR], const float2 (&ny)[kGR],
                                           const float2 (&nz)[kGR], const float2 (&mi)[kGR],
                                           float2 (&ax)[kGR], float2 (&ay)[kGR], float2 (&az)[kGR],
                                           float *stage) {
    const int next = (lane + 1) & 31;
    const int64_t q = (int64_t)gi * (kGrp / 2) + CH * 32 + lane;
    const float4 r0 = __ldcg(src + 2 * q), r1 = __ldcg(src + 2 * q + 1);
    float2 xj = f2(r0.x, r0.y), yj = f2(r0.z, r0.w), zj = f2(r1.x, r1.y), mj = f2(r1.z, r1.w);
    float2 bx = f2(0.f, 0.f), by = bx, bz = bx;
#pragma unroll 1
    for (int round = 0; round < 32; ++round) {
#pragma unroll
        for (int r = 0; r < kGR; ++r) {
            if (r > 2 * CH + 1) continue;
            const float2 dx = __fadd2_rn(xj, nx[r]);
            const float2 dy = __fadd2_rn(yj, ny[r]);
            const float2 dz = __fadd2_rn(zj, nz[r]);
            float2 s = __ffma2_rn(dx, dx, eps2);
            s = __ffma2_rn(dy, dy, s);
            s = __ffma2_rn(dz, dz, s);
            const float2 y = rsqrt_mufu2(s);
            const float2 y3 = __fmul2_rn(__fmul2_rn(y, y), y);
            const float2 wi = __fmul2_rn(mj, y3);
            ax[r] = __ffma2_rn(wi, dx, ax[r]);
            ay[r] = __ffma2_rn(wi, dy, ay[r]);
            az[r] = __ffma2_rn(wi, dz, az[r]);
            if (r < 2 * CH) {
                const float2 wj = __fmul2_rn(mi[r], y3);
                bx = __ffma2_rn(wj, dx, bx);
                by = __ffma2_rn(wj, dy, by);
                bz = __ffma2_rn(wj, dz, bz);
            }
        }
        xj = shfl2(xj, next);
        yj = shfl2(yj, next);
        zj = shfl2(zj, next);
        mj = shfl2(mj, next);
        if (CH > 0) {
            bx = shfl2(bx, next);
            by = shfl2(by, next);
            bz = shfl2(bz, next);
        }
    }
    const int b = CH * 64 + 2 * lane;
    stage[b] = -bx.x;
    stage[b + 1] = -bx.y;
    stage[kGrp + b] = -by.x;
    stage[kGrp + b + 1] = -by.y;
    stage[2 * kGrp + b] = -bz.x;
    stage[2 * kGrp + b + 1] = -bz.y;
}

__device__ __forceinline__ void pair_item_diag(const float4 *src, float *P, int64_t npad, int gi,
                                               int lane, float2 eps2, float *stage) {
    float2 nx[kGR], ny[kGR], nz[kGR], mi[kGR], ax[kGR], ay[kGR], az[kGR];
    const int64_t ib = (int64_t)gi * kGrp + lane;
#pragma unroll
    for (int r = 0; r < kGR; ++r) {
        const int64_t i = ib + 32 * r;
        nx[r] = dup(-pget_cg(src, i, 0));
        ny[r] = dup(-pget_cg(src, i, 1));
        nz[r] = dup(-pget_cg(src, i, 2));
        mi[r] = dup(pget_cg(src, i, 3));
        ax[r] = ay[r] = az[r] = f2(0.f, 0.f);
    }
    static_assert(kGrp == 256 && kGR == 8, "the diagonal schedule assumes 4 chunks of 64 bodies");
    diag_chunk<0>(src, gi, lane, eps2, nx, ny, nz, mi, ax, ay, az, stage);
    diag_chunk<1>(src, gi, lane, eps2, nx, ny, nz, mi, ax, ay, az, stage);
    diag_chunk<2>(src, gi, lane, eps2, nx, ny, nz, mi, ax, ay, az, stage);
    diag_chunk<3>(src, gi, lane, eps2, nx, ny, nz, mi, ax, ay, az, stage);
    __syncwarp();
    float *p = P + (int64_t)gi * 3 * npad + ib;  // row gi, bodies of group gi
#pragma unroll
    for (int r = 0; r < kGR; ++r) {
        const int b = lane + 32 * r;
        __stcg(p + 32 * r, (ax[r].x + ax[r].y) + stage[b]);
        __stcg(p + npad + 32 * r, (ay[r].x + ay[r].y) + stage[kGrp + b]);
        __stcg(p + 2 * npad + 32 * r, (az[r].x + az[r].y) + stage[2 * kGrp + b]);
    }
    __syncwarp();  // the stage is free for the warp's next item
}

// Group g's bodies: partials in group order, then the update of step t.
template <bool F64>
__device__ __forceinline__ void epilogue_item(const SymBatchArgs &a, int s, int g, int t, int lane) {
    const int64_t b0 = a.off[s], n = a.off[s + 1] - b0;
    const int ngs = a.ng[s];
    const int64_t npad = (int64_t)ngs * kGrp;
    const float *P = a.part + a.pofs[s];
    const float4 *src = ((t & 1) ? a.xm1 : a.xm0) + a.poff[s];
    float4 *dst = ((t & 1) ? a.xm0 : a.xm1) + a.poff[s];
    const bool last_kick = a.kdk && t == a.steps;           // the closing half kick
    const bool double_kick = a.kdk && t > 0 && !last_kick;  // KDK between two drifts
    // The lane's bodies' sums, partner group by partner group, four bodies
    // at a time: the 12 loads of one partner group are independent, so they
    // are in flight together (one L2 round trip per partner group, not per
    // load), and the sums stay in few registers.
    constexpr int kHalf = kGR / 2;
    for (int r0 = 0; r0 < kGR; r0 += kHalf) {
        const int64_t i0 = (int64_t)g * kGrp + lane + 32 * r0;
        if (i0 >= n) break;
        float h[kHalf][3], l[kHalf][3];
#pragma unroll
        for (int r = 0; r < kHalf; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) h[r][c] = l[r][c] = 0.f;
        for (int p = 0; p < ngs; ++p) {
            const float *q = P + (int64_t)p * 3 * npad + i0;
            float v[kHalf][3];
#pragma unroll
            for (int r = 0; r < kHalf; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) v[r][c] = __ldcg(q + c * npad + 32 * r);  // padding rows included
#pragma unroll
            for (int r = 0; r < kHalf; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if constexpr (F64) {
                        float sum, e;
                        two_sum(h[r][c], v[r][c], sum, e);
                        h[r][c] = sum;
                        l[r][c] = __fadd_rn(l[r][c], e);
                    } else {
                        h[r][c] += v[r][c];
                    }
                }
        }
#pragma unroll
        for (int r = 0; r < kHalf; ++r) {
            const int64_t i = i0 + 32 * r;
            if (i >= n) break;
            if constexpr (!F64) {
                float *xp = reinterpret_cast<float *>(a.x) + 3 * (b0 + i);
                float *vp = reinterpret_cast<float *>(a.v) + 3 * (b0 + i);
                float xs[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float acc = a.G * h[r][c];
                    // v += a dt/2 (the printed half kick; twice between two drifts of KDK); x += v dt
                    float vc = __fadd_rn(__ldcg(vp + c), __fmul_rn(__fmul_rn(acc, a.dt), 0.5f));
                    if (double_kick) vc = __fadd_rn(vc, __fmul_rn(__fmul_rn(acc, a.dt), 0.5f));
                    vp[c] = vc;
                    if (!last_kick) {
                        xs[c] = __fadd_rn(__ldcg(xp + c), __fmul_rn(vc, a.dt));
                        xp[c] = xs[c];
                    }
                }
                if (!last_kick) pair_put(dst, i, xs[0], xs[1], xs[2], pget_cg(src, i, 3));
            } else {
                double *xp = reinterpret_cast<double *>(a.x) + 3 * (b0 + i);
                double *vp = reinterpret_cast<double *>(a.v) + 3 * (b0 + i);
                double xs[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const double acc = a.Gd * ((double)h[r][c] + (double)l[r][c]);
                    double vc = __dadd_rn(__ldcg(vp + c), __dmul_rn(__dmul_rn(acc, a.dtd), 0.5));
                    if (double_kick) vc = __dadd_rn(vc, __dmul_rn(__dmul_rn(acc, a.dtd), 0.5));
                    vp[c] = vc;
                    if (!last_kick) {
                        xs[c] = __dadd_rn(__ldcg(xp + c), __dmul_rn(vc, a.dtd));
                        xp[c] = xs[c];
                    }
                }
                if (!last_kick) pair_put(dst, i, (float)xs[0], (float)xs[1], (float)xs[2], pget_cg(src, i, 3));
            }
        }
    }
}

template <bool F64>
__global__ void __launch_bounds__(kSymWarps * 32, F64 ? 3 : NB_SYMB_MINB) batched_sym_kernel(const SymBatchArgs a) {
    const int lane = threadIdx.x & 31;
    // KDK adds one step of items that end in a kick only (the forces at the final positions)
    const unsigned total =
        (unsigned)a.items_per_step * (unsigned)(a.steps + (a.kdk && a.steps > 0 ? 1 : 0));
    // Each warp's queue state, in shared memory (lane 0 only) so that it holds
    // no registers across the items: the held items (number, counter to
    // watch, count it must reach), their count and whether the queue is
    // empty.
    struct WarpQueue {
        const unsigned *ctr[kHoldW];
        unsigned id[kHoldW], need[kHoldW];
        int nheld, exhausted;
    };
    __shared__ WarpQueue s_q[kSymWarps];
    __shared__ float s_stage[kSymWarps][3 * kGrp];  // a diagonal item's j-side sums
    WarpQueue &Q = s_q[threadIdx.x >> 5];
    if (lane == 0) {
        for (int k = 0; k < kHoldW; ++k) {
            Q.id[k] = kNone;
            Q.need[k] = 0;
            Q.ctr[k] = nullptr;
        }
        Q.nheld = 0;
        Q.exhausted = 0;
    }
    __syncwarp();
    unsigned *h_id = Q.id, *h_need = Q.need;
    const unsigned **h_ctr = Q.ctr;
    int &nheld = Q.nheld;
    int &exhausted = Q.exhausted;

    // File item number `id` (taken from the queue) into a free hold slot.
    auto file = [&](unsigned id) {
        if (id >= total) {
            exhausted = 1;
            return;
        }
        const unsigned t = id / (unsigned)a.items_per_step;
        const int4 it = a.items[id % (unsigned)a.items_per_step];
        unsigned need;
        const unsigned *ctr;
        if (it.w == 0) {  // pair item: every epilogue item of step t-1 of its system
            need = t * (unsigned)a.ng[it.x];
            ctr = a.fin_done + it.x;
        } else {  // epilogue item: every pair item of step t of its system
            need = (t + 1) * (unsigned)a.npairs[it.x];
            ctr = a.pair_done + it.x;
        }
#pragma unroll
        for (int k = 0; k < kHoldW; ++k)
            if (h_id[k] == kNone) {
                h_id[k] = id;
                h_need[k] = need;
                h_ctr[k] = ctr;
                ++nheld;
                return;
            }
    };
    auto claim = [&]() {
        if (exhausted || nheld >= kHoldW) return;
        file(atomicAdd(a.next, 1u));
    };

    // The lowest-numbered held item that is ready; takes more items while
    // none is and a hold slot is free; otherwise polls, bounded. On a
    // timeout the lowest held item is returned with abort set: skipped, but
    // released, so no other item waits for it forever.
    auto pick = [&](bool &abort) -> unsigned {
        abort = false;
        uint64_t t0 = 0;
        for (;;) {
            unsigned best = kNone;  // the lowest ready held item
#pragma unroll
            for (int k = 0; k < kHoldW; ++k)
                if (h_id[k] < best && (h_need[k] == 0 || ld_relaxed_u32(h_ctr[k]) >= h_need[k]))
                    best = h_id[k];
            if (best != kNone) {
#pragma unroll
                for (int k = 0; k < kHoldW; ++k)
                    if (h_id[k] == best) h_id[k] = kNone;
                --nheld;
                fence_acq_rel();  // the predecessors' writes happen before this item's reads
                return best;
            }
            if (!exhausted && nheld < kHoldW) {
                claim();
                continue;
            }
            if (nheld == 0) return total;
            const uint64_t now = global_ns();
            if (t0 == 0) t0 = now;
            if (now - t0 > a.timeout_ns) {
                unsigned low = kNone;
#pragma unroll
                for (int k = 0; k < kHoldW; ++k)
                    if (h_id[k] < low) low = h_id[k];
#pragma unroll
                for (int k = 0; k < kHoldW; ++k)
                    if (h_id[k] == low) h_id[k] = kNone;
                --nheld;
                atomicOr(a.err, kErrStepDep);
                abort = true;
                return low;
            }
            __nanosleep(64);
        }
    };

    bool hold_back = a.stall && blockIdx.x == 0 && threadIdx.x < 32;  // debug: skip the first release
    for (;;) {
        unsigned id = 0, pending = kNone;  // lane 0: a number taken during the item, filed after it
        int ab = 0;
        if (lane == 0) {
            bool abort;
            id = pick(abort);
            ab = abort ? 1 : 0;
            // take the next number now: the atomic's latency passes while the
            // item runs (the value is first needed when it is filed)
            if (id < total && !exhausted && nheld < kHoldW) pending = atomicAdd(a.next, 1u);
        }
        id = __shfl_sync(0xffffffffu, id, 0);
        ab = __shfl_sync(0xffffffffu, ab, 0);
        __syncwarp();  // lane 0's acquire orders the whole warp's reads of the item's inputs
        if (id >= total) break;
        const int t = (int)(id / (unsigned)a.items_per_step);
        const int4 it = a.items[id % (unsigned)a.items_per_step];
        const int s = it.x;
        if (!ab) {
            if (it.w == 0) {
                const float4 *src = ((t & 1) ? a.xm1 : a.xm0) + a.poff[s];
                if (it.y == it.z)
                    pair_item_diag(src, a.part + a.pofs[s], (int64_t)a.ng[s] * kGrp, it.y, lane,
                                   dup(a.eps2), s_stage[threadIdx.x >> 5]);
                else
                    pair_item(a, src, a.part + a.pofs[s], (int64_t)a.ng[s] * kGrp, it.y, it.z, lane);
            } else {
                epilogue_item<F64>(a, s, it.y, t, lane);
            }
        }
        // release: every lane's writes, then one count
        __threadfence();
        __syncwarp();
        if (lane == 0) {
            if (!hold_back) atomicAdd(it.w == 0 ? a.pair_done + s : a.fin_done + s, 1u);
            if (pending != kNone) file(pending);
        }
        hold_back = false;
    }
}

// Pack every system (zero-mass padding to whole groups) into both buffers'
// padding and buffer 0's bodies.
template <class TS>
__global__ void batched_sym_pack_kernel(const int64_t *off, const int64_t *poff, const int *ng,
                                        const TS *x, const TS *m, float4 *xm0, float4 *xm1) {
    const int s = blockIdx.x;
    const int64_t b0 = off[s], n = off[s + 1] - b0, p0 = poff[s];
    const int64_t npad = (int64_t)ng[s] * kGrp;
    for (int64_t i = threadIdx.x; i < npad; i += blockDim.x) {
        if (i < n) {
            pair_put(xm0 + p0, i, (float)x[3 * (b0 + i)], (float)x[3 * (b0 + i) + 1],
                     (float)x[3 * (b0 + i) + 2], (float)m[b0 + i]);
        } else {
            pair_put(xm0 + p0, i, 0.f, 0.f, 0.f, 0.f);
            pair_put(xm1 + p0, i, 0.f, 0.f, 0.f, 0.f);
        }
    }
}

struct SymLayout {
    size_t o_off, o_poff, o_pofs, o_ng, o_np, o_items, o_next, o_pdone, o_fdone, o_xm0, o_xm1, o_part,
        total;
};

SymLayout sym_layout_of(const BatchPlan &p) {
    SymLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o += (bytes + 255) / 256 * 256;
        return at;
    };
    L.o_off = take(p.off.size() * 8);
    L.o_poff = take(p.poff.size() * 8);
    L.o_pofs = take(p.sym_pofs.size() * 8);
    L.o_ng = take(p.sym_ng.size() * 4);
    L.o_np = take(p.sym_npairs.size() * 4);
    L.o_items = take(p.sym_items.size() * 4);
    L.o_next = take(4);                      // queue head ...
    L.o_pdone = take((size_t)p.nsys * 4);    // ... and completion counters: zeroed per launch
    L.o_fdone = take((size_t)p.nsys * 4);
    L.o_xm0 = take((size_t)p.total_pad * 16);
    L.o_xm1 = take((size_t)p.total_pad * 16);
    L.o_part = take((size_t)p.sym_part_floats * 4);
    L.total = o;
    return L;
}

}  // namespace

size_t batched_sym_part_bytes(const std::vector<int64_t> &off) {
    size_t floats = 0;
    for (size_t s = 0; s + 1 < off.size(); ++s) {
        const size_t g = (size_t)((off[s + 1] - off[s] + kGrp - 1) / kGrp);
        floats += g * 3 * g * kGrp;
    }
    return floats * 4;
}

double batched_sym_work_ratio(const std::vector<int64_t> &off) {
    // FP32 lane operations of the pair-symmetric items (16 per evaluated pair,
    // groups padded to kGrp) against the one-sided items' (12 per interaction)
    double sym = 0, one = 0;
    for (size_t s = 0; s + 1 < off.size(); ++s) {
        const int64_t n = off[s + 1] - off[s];
        const int64_t g = (n + kGrp - 1) / kGrp;
        // a diagonal item evaluates 20 of the 32 (sub-block, chunk) squares
        sym += 16.0 * ((double)(g * (g - 1) / 2) + 0.625 * (double)g) * kGrp * kGrp;
        one += 12.0 * (double)n * (double)n;
    }
    return one > 0 ? sym / one : 1e30;
}

bool batched_sym_plan(int num_sms, const std::vector<int64_t> &off, BatchPlan &p, std::string &why) {
    p.sym = 1;
    if (batched_sym_part_bytes(off) > kSymMaxPartBytes) {
        why = "the pair-symmetric form's partials for these sizes exceed 16 GiB";
        return false;
    }
    p.nsys = (int)off.size() - 1;
    p.nt = kSymWarps * 32;
    p.r = kGR;
    p.jt = kGrp;
    auto fn = p.f64 ? batched_sym_kernel<true> : batched_sym_kernel<false>;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, p.nt, 0) != cudaSuccess || occ <= 0) {
        why = "occupancy query failed";
        return false;
    }
    p.off = off;
    p.poff.assign(p.nsys, 0);
    p.sym_pofs.assign(p.nsys, 0);
    p.sym_ng.assign(p.nsys, 0);
    p.sym_npairs.assign(p.nsys, 0);
    p.total = off[p.nsys];
    int64_t acc = 0, pacc = 0;
    struct Pair { int s, gi, gj; int64_t g; };
    std::vector<Pair> pairs;
    for (int s = 0; s < p.nsys; ++s) {
        const int64_t n = off[s + 1] - off[s];
        const int g = (int)((n + kGrp - 1) / kGrp);
        p.sym_ng[s] = g;
        p.sym_npairs[s] = g * (g + 1) / 2;
        p.poff[s] = acc;
        p.sym_pofs[s] = pacc;
        acc += (int64_t)g * kGrp;
        pacc += (int64_t)g * 3 * g * kGrp;
        for (int gi = 0; gi < g; ++gi)
            for (int gj = gi; gj < g; ++gj) pairs.push_back({s, gi, gj, g});
    }
    p.total_pad = std::max<int64_t>(acc, kGrp);
    p.sym_part_floats = std::max<int64_t>(pacc, 1);
    // a step: pair items of the largest systems first; each system's epilogue
    // items follow its last pair item after a lag of about NB_SYMB_EPI_LAG x
    // the grid's warps (0: all epilogue items after all pair items), in the
    // same system order, so the next step's first pair items (the largest
    // systems') become ready first
    std::stable_sort(pairs.begin(), pairs.end(), [](const Pair &x, const Pair &y) { return x.g > y.g; });
    std::vector<int> order(p.nsys);
    for (int s = 0; s < p.nsys; ++s) order[s] = s;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return p.sym_ng[x] > p.sym_ng[y]; });
    int64_t nepi = 0;
    for (int s = 0; s < p.nsys; ++s) nepi += p.sym_ng[s];
    const int64_t nwarps =
        std::min<int64_t>((int64_t)occ * num_sms, ((int64_t)pairs.size() + nepi + kSymWarps - 1) / kSymWarps) *
        kSymWarps;
    const int64_t lag = (int64_t)(NB_SYMB_EPI_LAG * (double)nwarps);
    std::vector<int64_t> last(p.nsys, -1);  // each system's last pair item
    for (size_t k = 0; k < pairs.size(); ++k) last[pairs[k].s] = (int64_t)k;
    p.sym_items.clear();
    size_t next_epi = 0;  // systems in `order` whose epilogue items are out
    auto emit_epi = [&](int s) {
        for (int g = 0; g < p.sym_ng[s]; ++g) p.sym_items.insert(p.sym_items.end(), {s, g, 0, 1});
    };
    for (size_t k = 0; k < pairs.size(); ++k) {
        const Pair &q = pairs[k];
        p.sym_items.insert(p.sym_items.end(), {q.s, q.gi, q.gj, 0});
        if (NB_SYMB_EPI_LAG > 0)
            while (next_epi < order.size() && last[order[next_epi]] + lag <= (int64_t)k) emit_epi(order[next_epi++]);
    }
    while (next_epi < order.size()) emit_epi(order[next_epi++]);
    p.items_per_step = (int)(p.sym_items.size() / 4);
    p.ncta = (int)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)occ * num_sms, (p.items_per_step + kSymWarps - 1) / kSymWarps));
    SymLayout L = sym_layout_of(p);
    p.scratch_bytes = L.total;
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint64_t v) {
        for (int b = 0; b < 8; ++b) {
            h ^= (v >> (8 * b)) & 0xff;
            h *= 1099511628211ull;
        }
    };
    for (int64_t v : off) mix((uint64_t)v);
    mix(0x53594d4dull);  // the pair-symmetric form
    mix((uint64_t)p.ncta);
    mix((uint64_t)p.f64);
    p.signature = h;
    return true;
}

cudaError_t batched_sym_upload(const BatchPlan &p, void *scratch, cudaStream_t st) {
    SymLayout L = sym_layout_of(p);
    char *b = (char *)scratch;
    cudaError_t e;
#define NB_UP(field, o)                                                                      \
    if (!p.field.empty()) {                                                                  \
        e = cudaMemcpyAsync(b + (o), p.field.data(), p.field.size() * sizeof(p.field[0]),   \
                            cudaMemcpyHostToDevice, st);                                     \
        if (e != cudaSuccess) return e;                                                      \
    }
    NB_UP(off, L.o_off)
    NB_UP(poff, L.o_poff)
    NB_UP(sym_pofs, L.o_pofs)
    NB_UP(sym_ng, L.o_ng)
    NB_UP(sym_npairs, L.o_np)
    NB_UP(sym_items, L.o_items)
#undef NB_UP
    return cudaSuccess;
}

const int64_t *batched_sym_offsets(const BatchPlan &p, void *scratch) {
    return (const int64_t *)((char *)scratch + sym_layout_of(p).o_off);
}

cudaError_t batched_sym_enqueue(const BatchPlan &p, void *scratch, void *x, void *v, const void *m,
                                int steps, int kdk, float eps2, double G, double dt, int *err,
                                uint64_t timeout_ns, int stall, cudaStream_t st) {
    if ((uint64_t)p.items_per_step * (uint64_t)(steps + 1) + (uint64_t)p.ncta * kSymWarps * (kHoldW + 1) >=
        (1ull << 32))
        return cudaErrorInvalidValue;
    SymLayout L = sym_layout_of(p);
    char *b = (char *)scratch;
    SymBatchArgs a;
    a.off = (const int64_t *)(b + L.o_off);
    a.poff = (const int64_t *)(b + L.o_poff);
    a.pofs = (const int64_t *)(b + L.o_pofs);
    a.ng = (const int *)(b + L.o_ng);
    a.npairs = (const int *)(b + L.o_np);
    a.items = (const int4 *)(b + L.o_items);
    a.next = (unsigned *)(b + L.o_next);
    a.pair_done = (unsigned *)(b + L.o_pdone);
    a.fin_done = (unsigned *)(b + L.o_fdone);
    a.xm0 = (float4 *)(b + L.o_xm0);
    a.xm1 = (float4 *)(b + L.o_xm1);
    a.part = (float *)(b + L.o_part);
    a.x = x;
    a.v = v;
    a.steps = steps;
    a.items_per_step = p.items_per_step;
    a.kdk = kdk;
    a.eps2 = eps2;
    a.G = (float)G;
    a.dt = (float)dt;
    a.Gd = G;
    a.dtd = dt;
    a.err = err;
    a.timeout_ns = timeout_ns;
    a.stall = stall;
    cudaError_t e = cudaMemsetAsync(b + L.o_next, 0, L.o_xm0 - L.o_next, st);
    if (e != cudaSuccess) return e;
    if (p.f64)
        batched_sym_pack_kernel<double><<<p.nsys, 256, 0, st>>>(a.off, a.poff, a.ng, (const double *)x,
                                                               (const double *)m, a.xm0, a.xm1);
    else
        batched_sym_pack_kernel<float><<<p.nsys, 256, 0, st>>>(a.off, a.poff, a.ng, (const float *)x,
                                                              (const float *)m, a.xm0, a.xm1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = dim3((unsigned)p.ncta);
    cfg.blockDim = dim3((unsigned)p.nt);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (p.f64) return cudaLaunchKernelEx(&cfg, batched_sym_kernel<true>, a);
    return cudaLaunchKernelEx(&cfg, batched_sym_kernel<false>, a);
}

}  // namespace nb
