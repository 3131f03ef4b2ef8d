// Persistent ensemble kernel: every system of the batch advances `steps`
// paper steps inside one cooperative launch, as a dataflow over work items
// (system, step, i-chunk of NT x R bodies, R per item). Persistent CTAs take
// items from one atomic queue in step-major order (most work first within a
// step) and hold a few; an item is ready once every item of the previous
// step of its own system is done. A CTA runs its lowest-numbered ready item:
// the forces on its i-chunk from all j-bodies of the system (j-tiles streamed
// by 1-D bulk copies through a shared-memory ring), the half kick and the
// drift, the repacked positions written to the other buffer; then it
// releases the item. The lowest unfinished item is always ready, so the
// queue always makes progress, and load balance is within one item.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <numeric>
#include <type_traits>

#include "batched.h"
#include "engine.cuh"

namespace nb {

namespace {

struct BatchArgs {
    const int64_t *off, *poff;
    const int *item_sys, *item_lo, *item_r;  // per item of one step
    const int *nitems;                        // [nsys] items per step
    unsigned *next;  // queue head
    unsigned *done;  // [nsys] items completed, cumulative over steps
    float4 *xm0, *xm1;
    void *x, *v;  // [n][3] in the state type (float, or double in the precision form)
    int steps, jt, items_per_step;
    int kdk;  // 1: kick-drift-kick (kick twice between drifts; one closing half-kick step)
    float eps2, G, dt;
    double Gd, dtd;  // the precision form's FP64 update
    int *err;
    uint64_t timeout_ns;
};

__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Order this thread's earlier shared-memory accesses (and those it has
// acquired from other threads) before later bulk copies into shared memory.
__device__ __forceinline__ void fence_proxy_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Pair-layout scalar read through L2 only: another CTA may have written it
// earlier in this launch, and a line this SM cached before must not be used.
__device__ __forceinline__ float pair_get_cg(const float4 *base, int64_t i, int c) {
    const float *p = reinterpret_cast<const float *>(base + (i >> 1) * 2);
    return __ldcg(p + 2 * c + (int)(i & 1));
}

__device__ __forceinline__ unsigned ld_relaxed(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fence_acq_rel_gpu() {
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}


// Ring of the batched kernel: kBS slots. A slot is refilled by the lane 0 of
// the last warp to finish with it (a shared counter per slot), the moment it
// is free, with the tile kBS positions ahead; nobody waits for a free slot,
// and no warp's own progress decides when the others' tiles arrive.
constexpr int kBS = 8;
constexpr int kHold = 4;                  // items a CTA may hold unstarted
constexpr unsigned kNoItem = 0xFFFFFFFFu;

// Registers are allocated for the largest R the kernel holds. The occupancy
// hint asks for 512 resident threads per SM up to R = 2 (at most 128
// registers), 256 at R = 4 and 128 at R = 8 (as the single-system kernel of
// those shapes); a 512-thread CTA is then alone on its SM.
template <int NT, int RMAX>
constexpr int batched_min_blocks() {
    constexpr int per_sm = RMAX <= 2 ? 512 : (RMAX == 4 ? 256 : 128);
    return per_sm / NT > 1 ? per_sm / NT : 1;
}

// F64 = true: the precision form, FP64 state; FP32 pair terms summed per
// j-tile, two-summed into (hi, lo) across tiles, widened once for the FP64
// update (the arithmetic of the single-system precision form).
template <int NT, int RMAX, bool F64>
__global__ void __launch_bounds__(NT, (batched_min_blocks<NT, RMAX>())) batched_kernel(const BatchArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw);
    float4 *ring = reinterpret_cast<float4 *>(smem_raw + 128);
    __shared__ unsigned s_item;
    __shared__ int s_abort;
    __shared__ unsigned s_rel[kBS];  // warps done with the slot's current tile
    __shared__ unsigned s_issued;    // ring positions issued so far
    // Items this CTA has taken from the queue but not started (thread 0
    // only): number, system, and the completion count of the system that
    // makes it ready (0: ready at once).
    __shared__ unsigned h_id[kHold], h_need[kHold];
    __shared__ int h_sys[kHold];
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int f4_per_tile = a.jt;  // (jt / 2) records x 2 float4
    const uint32_t tile_bytes = (uint32_t)f4_per_tile * 16u;
    const float dt = a.dt;
    // KDK adds one step of items that only kick (the forces at the final positions)
    const unsigned total = (unsigned)a.items_per_step * (unsigned)(a.steps + (a.kdk && a.steps > 0 ? 1 : 0));

    if (tid == 0) {
        for (int s = 0; s < kBS; ++s) {
            mbar_init(&full[s], 1);
            s_rel[s] = 0;
        }
        for (int h = 0; h < kHold; ++h) h_id[h] = kNoItem;
        s_issued = 0;
        mbar_init_fence();
    }
    __syncthreads();

    // Ring position q (tiles streamed so far by this CTA) runs on across
    // items; slot q % kBS, phase q / kBS. Position q is issued only once
    // position q - kBS has been released by every warp: at the start of an
    // item (every earlier position is released then) or by the last warp to
    // release q - kBS.
    int nheld = 0;           // thread 0: items held
    bool exhausted = false;  // thread 0: the queue is empty
    uint32_t kk = 0;         // position of the current item's first tile
    bool give_up = false;  // a ring wait failed: stop streaming

    auto issue = [&](uint32_t q, const float4 *src_tile) {
        const int slot = q % kBS;
        mbar_arrive_expect_tx(&full[slot], tile_bytes);
        bulk_g2s(ring + slot * f4_per_tile, src_tile, tile_bytes, &full[slot]);
        atomicMax(&s_issued, q + 1);
    };

    // Thread 0: take one more item from the queue into a free hold slot.
    auto claim = [&]() {
        if (exhausted || nheld >= kHold) return;
        const unsigned id = atomicAdd(a.next, 1u);
        if (id >= total) {
            exhausted = true;
            return;
        }
        const unsigned t = id / (unsigned)a.items_per_step;
        const int sys = a.item_sys[id % (unsigned)a.items_per_step];
        for (int h = 0; h < kHold; ++h)
            if (h_id[h] == kNoItem) {
                h_id[h] = id;
                h_sys[h] = sys;
                h_need[h] = t * (unsigned)a.nitems[sys];  // step t needs all of step t-1
                ++nheld;
                return;
            }
    };

    // Thread 0: the next item to run. Runs the lowest-numbered held item
    // whose system has finished the previous step; while none is ready and a
    // hold slot is free, takes more items from the queue; otherwise polls,
    // bounded. Returns total when the queue is empty and nothing is held.
    // The lowest unfinished item of the whole launch is always ready (its
    // predecessors have lower numbers), and whoever holds it runs it at its
    // next pick, so the queue cannot stall; a CTA never idles on a system that
    // fell behind while later items of other systems are ready.
    auto pick = [&](bool &abort) -> unsigned {
        abort = false;
        uint64_t t0 = 0;
        for (;;) {
            int best = -1;
            for (int h = 0; h < kHold; ++h) {
                const unsigned id = h_id[h];
                if (id == kNoItem || (best >= 0 && id > h_id[best])) continue;
                if (h_need[h] == 0 || ld_relaxed(a.done + h_sys[h]) >= h_need[h]) best = h;
            }
            if (best >= 0) {
                const unsigned id = h_id[best];
                h_id[best] = kNoItem;
                --nheld;
                fence_acq_rel_gpu();  // the predecessors' writes happen before this item's reads
                return id;
            }
            if (!exhausted && nheld < kHold) {
                claim();
                continue;
            }
            if (nheld == 0) return total;
            const uint64_t now = global_ns();
            if (t0 == 0) t0 = now;
            if (now - t0 > a.timeout_ns) {
                // give up on the lowest held item: skipped, but released
                int low = -1;
                for (int h = 0; h < kHold; ++h)
                    if (h_id[h] != kNoItem && (low < 0 || h_id[h] < h_id[low])) low = h;
                const unsigned id = h_id[low];
                h_id[low] = kNoItem;
                --nheld;
                atomicOr(a.err, kErrStepDep);
                abort = true;
                return id;
            }
            __nanosleep(64);
        }
    };

    // One work item with R i-bodies per thread: forces on bodies [lo, hi)
    // of one system from its ntl j-tiles (Eq. 1 with softening), then the
    // printed update (half kick v += a dt/2, drift x += v dt with the new
    // v), and the repacked position written to the other buffer. A generic
    // lambda, instantiated for each R the kernel holds.
    auto run_item = [&](auto r_const, const float4 *src, float4 *dst, int64_t b0, int64_t lo,
                        int64_t hi, int ntl, int last_pairs, int t) {
        constexpr int R = decltype(r_const)::value;
        AccelF32x2::I ist[R];
        AccelF32x2::T tot[R];  // FP32: the sums; precision form: this tile's sums
        float hh[F64 ? R : 1][3], ll[F64 ? R : 1][3];  // precision form: (hi, lo) across tiles
        if constexpr (F64) {
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) hh[r][c] = ll[r][c] = 0.f;
        }
        AccelF32x2::C cst;
        cst.eps2 = dup(a.eps2);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            int64_t i = lo + r * NT + tid;
            if (i >= hi) i = lo;
            ist[r].nx = dup(-pair_get_cg(src, i, 0));
            ist[r].ny = dup(-pair_get_cg(src, i, 1));
            ist[r].nz = dup(-pair_get_cg(src, i, 2));
            AccelF32x2::zero_total(tot[r]);
        }
        for (int q = 0; q < ntl; ++q) {
            const uint32_t pos = kk + q;
            const int slot = pos % kBS;
            if (tid == 0 && q == ntl - 1) claim();  // queue latency hidden behind the last tile
            if (!give_up && !mbar_wait(&full[slot], (pos / kBS) & 1, a.timeout_ns)) {
                atomicOr(a.err, kErrFullWait);
                give_up = true;
            }
            if (!give_up) {
                const float4 *tile = ring + slot * f4_per_tile;
                // the system's last tile: only its real records (the rest are
                // zero-mass padding and would add exactly 0)
                const int jpairs = q == ntl - 1 ? last_pairs : (a.jt >> 1);
#pragma unroll(AccelF32x2::UNROLL)
                for (int jp = 0; jp < jpairs; ++jp) {
                    float4 rec[2] = {tile[2 * jp], tile[2 * jp + 1]};
#pragma unroll
                    for (int r = 0; r < R; ++r) AccelF32x2::interact(rec, ist[r], tot[r], cst);
                }
                if constexpr (F64) {
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const float b3[3] = {tot[r].x.x + tot[r].x.y, tot[r].y.x + tot[r].y.y,
                                             tot[r].z.x + tot[r].z.y};
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            float sum, err;
                            two_sum(hh[r][c], b3[c], sum, err);
                            hh[r][c] = sum;
                            ll[r][c] += err;
                        }
                        AccelF32x2::zero_total(tot[r]);
                    }
                }
                __syncwarp();
                if (lane == 0) {
                    // release the slot; the last warp refills it with position pos + kBS
                    __threadfence_block();
                    if (atomicAdd(&s_rel[slot], 1u) == NT / 32 - 1) {
                        s_rel[slot] = 0;
                        __threadfence_block();
                        fence_proxy_async_shared();
                        if (q + kBS < ntl) issue(pos + kBS, src + (int64_t)(q + kBS) * f4_per_tile);
                    }
                }
            }
        }
        kk += ntl;
        const bool last_kick = a.kdk && t == a.steps;             // the closing half kick
        const bool double_kick = a.kdk && t > 0 && !last_kick;    // KDK between two drifts
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int64_t i = lo + r * NT + tid;
            if (i < hi) {
                if constexpr (!F64) {
                    const float acc[3] = {a.G * (tot[r].x.x + tot[r].x.y), a.G * (tot[r].y.x + tot[r].y.y),
                                          a.G * (tot[r].z.x + tot[r].z.y)};
                    float *xp = reinterpret_cast<float *>(a.x) + 3 * (b0 + i);
                    float *vp = reinterpret_cast<float *>(a.v) + 3 * (b0 + i);
                    float xs[3];
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc) {
                        // v += a dt/2 (the printed half kick; twice between two drifts of KDK); x += v dt
                        float vc = __fadd_rn(__ldcg(vp + cc), __fmul_rn(__fmul_rn(acc[cc], dt), 0.5f));
                        if (double_kick) vc = __fadd_rn(vc, __fmul_rn(__fmul_rn(acc[cc], dt), 0.5f));
                        vp[cc] = vc;
                        if (!last_kick) {
                            xs[cc] = __fadd_rn(__ldcg(xp + cc), __fmul_rn(vc, dt));
                            xp[cc] = xs[cc];
                        }
                    }
                    if (!last_kick) pair_put(dst, i, xs[0], xs[1], xs[2], pair_get_cg(src, i, 3));
                } else {
                    double *xp = reinterpret_cast<double *>(a.x) + 3 * (b0 + i);
                    double *vp = reinterpret_cast<double *>(a.v) + 3 * (b0 + i);
                    double xs[3];
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc) {
                        const double acc = a.Gd * ((double)hh[r][cc] + (double)ll[r][cc]);
                        double vc = __dadd_rn(__ldcg(vp + cc), __dmul_rn(__dmul_rn(acc, a.dtd), 0.5));
                        if (double_kick) vc = __dadd_rn(vc, __dmul_rn(__dmul_rn(acc, a.dtd), 0.5));
                        vp[cc] = vc;
                        if (!last_kick) {
                            xs[cc] = __dadd_rn(__ldcg(xp + cc), __dmul_rn(vc, a.dtd));
                            xp[cc] = xs[cc];
                        }
                    }
                    if (!last_kick)
                        pair_put(dst, i, (float)xs[0], (float)xs[1], (float)xs[2], pair_get_cg(src, i, 3));
                }
            }
        }
    };

    for (;;) {
        if (tid == 0) {
            bool abort;
            const unsigned id = pick(abort);
            s_item = id;
            s_abort = abort ? 1 : 0;
            if (id < total && !abort && !give_up) {
                // the ring is free (the previous item ended with a barrier):
                // start streaming this item's first tiles before the broadcast
                const int t = (int)(id / (unsigned)a.items_per_step);
                const int sys = a.item_sys[id % (unsigned)a.items_per_step];
                const int64_t n = a.off[sys + 1] - a.off[sys];
                const int ntl = (int)((n + a.jt - 1) / a.jt);
                const float4 *src = ((t & 1) ? a.xm1 : a.xm0) + a.poff[sys];
                fence_proxy_async_global();
                for (int q = 0; q < ntl && q < kBS; ++q) issue(kk + q, src + (int64_t)q * f4_per_tile);
            }
        }
        __syncthreads();
        const unsigned id = s_item;
        if (id >= total) break;
        const int t = (int)(id / (unsigned)a.items_per_step);
        const int k = (int)(id % (unsigned)a.items_per_step);
        const int s = a.item_sys[k];
        const int r = a.item_r[k];
        const int64_t lo = a.item_lo[k];
        const int64_t b0 = a.off[s];
        const int64_t n = a.off[s + 1] - b0;
        const int64_t p0 = a.poff[s];
        const int ntl = (int)((n + a.jt - 1) / a.jt);
        const int last_pairs = (int)((n - (int64_t)(ntl - 1) * a.jt + 1) >> 1);
        const int64_t hi = lo + (int64_t)NT * r < n ? lo + (int64_t)NT * r : n;
        const float4 *src = ((t & 1) ? a.xm1 : a.xm0) + p0;  // one float4 per body
        float4 *dst = ((t & 1) ? a.xm0 : a.xm1) + p0;
        if (!s_abort && !give_up) {
            if constexpr (RMAX >= 8) {
                if (r == 8) run_item(std::integral_constant<int, 8>{}, src, dst, b0, lo, hi, ntl, last_pairs, t);
            }
            if constexpr (RMAX >= 4) {
                if (r == 4) run_item(std::integral_constant<int, 4>{}, src, dst, b0, lo, hi, ntl, last_pairs, t);
            }
            if constexpr (RMAX >= 2) {
                if (r == 2) run_item(std::integral_constant<int, 2>{}, src, dst, b0, lo, hi, ntl, last_pairs, t);
            }
            if (r == 1) run_item(std::integral_constant<int, 1>{}, src, dst, b0, lo, hi, ntl, last_pairs, t);
            fence_proxy_async_global();
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            atomicAdd(a.done + s, 1u);  // release this item to step t+1
        }
    }
    // never leave while our own copies may still be landing (the loop above
    // ended with a __syncthreads, so every issue is visible in s_issued)
    if (tid == 0) {
        const uint32_t issued = s_issued;
        for (uint32_t q = issued > (uint32_t)kBS ? issued - kBS : 0; q < issued; ++q) {
            if (!mbar_wait(&full[q % kBS], (q / kBS) & 1, kDrainTimeoutNs))
                atomicOr(a.err, kErrDrain);
        }
    }
}

// Pack every system into buffer 0 with zero-mass padding to whole j-tiles,
// and zero the padding of buffer 1 too: the steps' epilogues repack real
// bodies only, and the scratch may hold another plan's bodies (a tuning run
// with another j-tile, or other sizes) where this plan pads.
template <class TS>
__global__ void batched_pack_kernel(const int64_t *off, const int64_t *poff, int jt,
                                    const TS *x, const TS *m, float4 *xm, float4 *xm1) {
    const int s = blockIdx.x;
    const int64_t b0 = off[s], n = off[s + 1] - b0, p0 = poff[s];
    const int64_t npad = (n + jt - 1) / jt * jt;
    for (int64_t i = threadIdx.x; i < npad; i += blockDim.x) {
        if (i < n) {
            pair_put(xm + p0, i, (float)x[3 * (b0 + i)], (float)x[3 * (b0 + i) + 1],
                     (float)x[3 * (b0 + i) + 2], (float)m[b0 + i]);
        } else {
            pair_put(xm + p0, i, 0.f, 0.f, 0.f, 0.f);
            pair_put(xm1 + p0, i, 0.f, 0.f, 0.f, 0.f);
        }
    }
}

template <class TS>
__global__ void batched_fill_kernel(const int64_t *off, TS *x, TS *v, TS *m) {
    const int s = blockIdx.x;
    const int64_t b0 = off[s], n = off[s + 1] - b0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const int64_t g = b0 + i;
        for (int c = 0; c < 3; ++c) {
            uint32_t h = (uint32_t)(g * 3 + c) * 2654435761u;
            h ^= h >> 15;
            h *= 0x2c1b3c6dU;
            h ^= h >> 12;
            const float u = (float)(h >> 8) * (1.0f / 16777216.0f);
            x[3 * g + c] = (TS)(2.f * u - 1.f);
            v[3 * g + c] = (TS)(0.1f * (u - 0.5f));
        }
        m[g] = (TS)(1.0f / (float)n);
    }
}

size_t batched_smem(int jt) { return 128 + (size_t)kBS * jt * 16; }

using BatchedFn = void (*)(const BatchArgs);

// Shapes of the ensemble kernel: (threads, largest R). Up to R = 2 the
// registers fit 512 resident threads per SM; the 512-thread forms then run
// one CTA per SM.
BatchedFn batched_fn(int nt, int rmax, bool f64) {
    if (f64) {  // (hi, lo) per body on top of the sums: at most 4 bodies per thread
        switch (nt * 16 + rmax) {
            case 128 * 16 + 1: return batched_kernel<128, 1, true>;
            case 128 * 16 + 2: return batched_kernel<128, 2, true>;
            case 128 * 16 + 4: return batched_kernel<128, 4, true>;
            case 256 * 16 + 1: return batched_kernel<256, 1, true>;
            case 256 * 16 + 2: return batched_kernel<256, 2, true>;
            case 256 * 16 + 4: return batched_kernel<256, 4, true>;
            case 512 * 16 + 1: return batched_kernel<512, 1, true>;
            case 512 * 16 + 2: return batched_kernel<512, 2, true>;
            default: return nullptr;
        }
    }
    switch (nt * 16 + rmax) {
        case 128 * 16 + 1: return batched_kernel<128, 1, false>;
        case 128 * 16 + 2: return batched_kernel<128, 2, false>;
        case 128 * 16 + 4: return batched_kernel<128, 4, false>;
        case 128 * 16 + 8: return batched_kernel<128, 8, false>;
        case 256 * 16 + 1: return batched_kernel<256, 1, false>;
        case 256 * 16 + 2: return batched_kernel<256, 2, false>;
        case 256 * 16 + 4: return batched_kernel<256, 4, false>;
        case 256 * 16 + 8: return batched_kernel<256, 8, false>;
        case 512 * 16 + 1: return batched_kernel<512, 1, false>;
        case 512 * 16 + 2: return batched_kernel<512, 2, false>;
        default: return nullptr;
    }
}

// Device copy of the plan inside the scratch block.
struct Layout {
    size_t o_off, o_poff, o_isys, o_ilo, o_ir, o_nit, o_next, o_done, o_xm0, o_xm1, total;
};

Layout layout_of(const BatchPlan &p) {
    Layout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o += (bytes + 255) / 256 * 256;
        return at;
    };
    L.o_off = take(p.off.size() * 8);
    L.o_poff = take(p.poff.size() * 8);
    L.o_isys = take(p.item_sys.size() * 4);
    L.o_ilo = take(p.item_lo.size() * 4);
    L.o_ir = take(p.item_r.size() * 4);
    L.o_nit = take(p.nitems.size() * 4);
    L.o_next = take(4);                            // queue head ...
    L.o_done = take((size_t)p.nsys * 4);          // ... and completion counters: zeroed per launch
    L.o_xm0 = take((size_t)p.total_pad * 16);
    L.o_xm1 = take((size_t)p.total_pad * 16);
    L.total = o;
    return L;
}

}  // namespace

int64_t batched_max_n() { return int64_t(1) << 20; }

bool batched_plan(int device, int num_sms, const std::vector<int64_t> &off, BatchPlan &p,
                  std::string &why) {
    (void)device;
    if (p.sym) return batched_sym_plan(num_sms, off, p, why);
    p.nsys = (int)off.size() - 1;
    if (p.nt == 0) p.nt = 256;  // one CTA per SM: no co-resident CTA starves another
    if (p.r == 0) p.r = p.f64 ? 4 : 8;
    if (p.jt == 0) p.jt = 64;
    const BatchedFn fn = batched_fn(p.nt, p.r, p.f64 != 0);
    if (!fn || p.jt % 2 || kPadBodies % p.jt) {
        why = "unsupported batched shape";
        return false;
    }
    int occ = 0;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)batched_smem(p.jt));
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, p.nt, batched_smem(p.jt));
    if (e != cudaSuccess || occ <= 0) {
        why = "occupancy query failed";
        return false;
    }
    p.off = off;
    p.poff.assign(p.nsys, 0);
    p.nitems.assign(p.nsys, 0);
    p.total = off[p.nsys];
    // Items of a system: full chunks of NT x rmax i-bodies, then the ragged
    // rest as power-of-two items (its rows of NT in binary), so that a system
    // computes fewer than NT idle i-slots. Rounding 3 and 7 rows up to 4 and 8
    // saved items but cost a whole idle row against all of the system's
    // j-bodies: 5.0 % extra work on the C4 size mix against 3.3 %.
    struct Item { int sys, lo, r, ntl; };
    std::vector<Item> items;
    int64_t acc = 0;
    for (int s = 0; s < p.nsys; ++s) {
        const int64_t n = off[s + 1] - off[s];
        p.poff[s] = acc;
        acc += (n + p.jt - 1) / p.jt * p.jt;
        const int ntl = (int)((n + p.jt - 1) / p.jt);
        int64_t lo = 0;
        const int64_t full = (int64_t)p.nt * p.r;
        for (; lo + full <= n; lo += full) items.push_back({s, (int)lo, p.r, ntl});
        int rows = (int)((n - lo + p.nt - 1) / p.nt);
        for (int r = p.r; r >= 1 && rows > 0; r >>= 1)
            if (rows >= r) {
                items.push_back({s, (int)lo, r, ntl});
                lo += (int64_t)r * p.nt;
                rows -= r;
            }
    }
    for (int s = 0; s < p.nsys; ++s) p.nitems[s] = 0;
    for (const Item &it : items) p.nitems[it.sys]++;
    p.total_pad = std::max<int64_t>(acc, p.jt);
    // items of one step: most work first (R x tiles), then by system and row
    std::stable_sort(items.begin(), items.end(), [](const Item &x, const Item &y) {
        return (int64_t)x.r * x.ntl > (int64_t)y.r * y.ntl;
    });
    p.item_sys.clear();
    p.item_lo.clear();
    p.item_r.clear();
    for (const Item &it : items) {
        p.item_sys.push_back(it.sys);
        p.item_lo.push_back(it.lo);
        p.item_r.push_back(it.r);
    }
    p.items_per_step = (int)p.item_sys.size();
    p.ncta = std::max(1, std::min(occ * num_sms, std::max(p.items_per_step, 1)));
    Layout L = layout_of(p);
    p.scratch_bytes = L.total;
    // signature: FNV-1a over sizes and shape
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint64_t v) {
        for (int b = 0; b < 8; ++b) {
            h ^= (v >> (8 * b)) & 0xff;
            h *= 1099511628211ull;
        }
    };
    for (int64_t v : off) mix((uint64_t)v);
    mix((uint64_t)p.nt);
    mix((uint64_t)p.r);
    mix((uint64_t)p.jt);
    mix((uint64_t)p.ncta);
    p.signature = h;
    return true;
}

cudaError_t batched_upload(const BatchPlan &p, void *scratch, cudaStream_t st) {
    if (p.sym) return batched_sym_upload(p, scratch, st);
    Layout L = layout_of(p);
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
    NB_UP(item_sys, L.o_isys)
    NB_UP(item_lo, L.o_ilo)
    NB_UP(item_r, L.o_ir)
    NB_UP(nitems, L.o_nit)
#undef NB_UP
    return cudaSuccess;
}

cudaError_t batched_fill_synthetic(const BatchPlan &p, void *scratch, void *x, void *v, void *m,
                                   cudaStream_t st) {
    const int64_t *off = p.sym ? batched_sym_offsets(p, scratch)
                               : (const int64_t *)((char *)scratch + layout_of(p).o_off);
    if (p.f64)
        batched_fill_kernel<double><<<p.nsys, 256, 0, st>>>(off, (double *)x, (double *)v, (double *)m);
    else
        batched_fill_kernel<float><<<p.nsys, 256, 0, st>>>(off, (float *)x, (float *)v, (float *)m);
    return cudaGetLastError();
}

cudaError_t batched_enqueue(const BatchPlan &p, void *scratch, void *x, void *v, const void *m,
                            int steps, int kdk, float eps2, double G, double dt, int *err,
                            uint64_t timeout_ns, int stall, cudaStream_t st) {
    if (p.sym)
        return batched_sym_enqueue(p, scratch, x, v, m, steps, kdk, eps2, G, dt, err, timeout_ns, stall, st);
    if ((uint64_t)p.items_per_step * (uint64_t)(steps + 1) + (uint64_t)p.ncta * (kHold + 1) >= (1ull << 32))
        return cudaErrorInvalidValue;
    Layout L = layout_of(p);
    char *b = (char *)scratch;
    BatchArgs a;
    a.off = (const int64_t *)(b + L.o_off);
    a.poff = (const int64_t *)(b + L.o_poff);
    a.item_sys = (const int *)(b + L.o_isys);
    a.item_lo = (const int *)(b + L.o_ilo);
    a.item_r = (const int *)(b + L.o_ir);
    a.nitems = (const int *)(b + L.o_nit);
    a.next = (unsigned *)(b + L.o_next);
    a.done = (unsigned *)(b + L.o_done);
    a.xm0 = (float4 *)(b + L.o_xm0);
    a.xm1 = (float4 *)(b + L.o_xm1);
    a.x = x;
    a.v = v;
    a.steps = steps;
    a.kdk = kdk;
    a.jt = p.jt;
    a.items_per_step = p.items_per_step;
    a.eps2 = eps2;
    a.G = (float)G;
    a.dt = (float)dt;
    a.Gd = G;
    a.dtd = dt;
    a.err = err;
    a.timeout_ns = timeout_ns;
    cudaError_t e = cudaMemsetAsync(b + L.o_next, 0, L.o_xm0 - L.o_next, st);
    if (e != cudaSuccess) return e;
    if (p.f64)
        batched_pack_kernel<double><<<p.nsys, 256, 0, st>>>(a.off, a.poff, p.jt, (const double *)x,
                                                            (const double *)m, a.xm0, a.xm1);
    else
        batched_pack_kernel<float><<<p.nsys, 256, 0, st>>>(a.off, a.poff, p.jt, (const float *)x,
                                                           (const float *)m, a.xm0, a.xm1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = dim3((unsigned)p.ncta);
    cfg.blockDim = dim3((unsigned)p.nt);
    cfg.dynamicSmemBytes = batched_smem(p.jt);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    BatchedFn fn = batched_fn(p.nt, p.r, p.f64 != 0);
    if (!fn) return cudaErrorInvalidValue;
    return cudaLaunchKernelEx(&cfg, fn, a);
}

}  // namespace nb
