// Persistent ensemble kernel: every system of the batch advances `steps`
// paper steps inside one cooperative launch, as a dataflow over work items
// (system, step, i-chunk). Persistent CTAs pop items from one atomic queue in
// step-major order (largest systems first within a step); an item waits,
// bounded, until every item of the previous step of its own system is done,
// then computes the forces on its i-chunk from all j-bodies of the system
// (j-tiles streamed by 1-D bulk copies, issued by thread 0, through a
// shared-memory ring as in the single-system kernel), applies the half kick
// and the drift, writes the repacked positions to the other buffer and
// releases itself. The oldest unfinished item never waits, so the queue
// always makes progress, and load balance is within one item.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <numeric>

#include "batched.h"
#include "engine.cuh"

namespace nb {

namespace {

struct BatchArgs {
    const int64_t *off, *poff;
    const int *item_sys, *item_chunk, *nchunks;
    unsigned *next;  // queue head
    unsigned *done;  // [nsys] items completed, cumulative over steps
    float4 *xm0, *xm1;
    float *x, *v;
    int steps, jt, items_per_step;
    float eps2, G, dt;
    int *err;
    uint64_t timeout_ns;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Pair-layout scalar read through L2 only: another CTA may have written it
// earlier in this launch, and a line this SM cached before must not be used.
__device__ __forceinline__ float pair_get_cg(const float4 *base, int64_t i, int c) {
    const float *p = reinterpret_cast<const float *>(base + (i >> 1) * 2);
    return __ldcg(p + 2 * c + (int)(i & 1));
}

// Bounded wait until *p >= target; false on timeout.
__device__ bool wait_at_least(const unsigned *p, unsigned target, uint64_t timeout_ns) {
    if (ld_acquire(p) >= target) return true;
    const uint64_t t0 = global_ns();
    while (ld_acquire(p) < target) {
        __nanosleep(64);
        if (global_ns() - t0 > timeout_ns) return false;
    }
    return true;
}

// Ring of the batched kernel: deeper than the single-system kernel's, and
// refilled with a lag of two tiles, so that thread 0 rarely waits for the
// slowest warp on the short tiles of small systems.
constexpr int kBS = 8;           // slots
constexpr int kLead = kBS - 2;   // tiles issued ahead of the one being consumed

template <int NT, int R>
__global__ void __launch_bounds__(NT, (R <= 2 ? 4 : 2)) batched_kernel(const BatchArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw);
    uint64_t *empty = full + kBS;
    float4 *ring = reinterpret_cast<float4 *>(smem_raw + 128);
    __shared__ unsigned s_item;
    __shared__ int s_abort;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int f4_per_tile = a.jt;  // (jt / 2) records x 2 float4
    const uint32_t tile_bytes = (uint32_t)f4_per_tile * 16u;
    const float dt = a.dt;
    const unsigned total = (unsigned)a.items_per_step * (unsigned)a.steps;

    if (tid == 0) {
        for (int s = 0; s < kBS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NT / 32);
        }
        mbar_init_fence();
    }
    __syncthreads();

    // Ring position q (tiles streamed so far by this CTA) runs on across
    // items; slot q % kBS, phase q / kBS. Thread 0 issues position q
    // once position q - kBS has been released by every warp.
    uint32_t kk = 0;       // position of the current item's first tile
    uint32_t issued = 0;   // positions issued so far (thread 0)
    bool give_up = false;  // a ring wait failed: stop streaming

    auto issue = [&](uint32_t q, const float4 *src_tile) {
        const int slot = q % kBS;
        if (q >= (uint32_t)kBS &&
            !mbar_wait(&empty[slot], ((q / kBS) - 1) & 1, a.timeout_ns)) {
            atomicOr(a.err, kErrEmptyWait);
            give_up = true;
            return;
        }
        mbar_arrive_expect_tx(&full[slot], tile_bytes);
        bulk_g2s(ring + slot * f4_per_tile, src_tile, tile_bytes, &full[slot]);
        issued = q + 1;
    };

    // Thread 0 takes the next item number one item ahead, so the queue's
    // atomic latency overlaps the current item. Holding one unstarted item
    // cannot stall the queue: the lowest unfinished item is always one that
    // some CTA is running, and its dependencies are all finished.
    unsigned next_id = tid == 0 ? atomicAdd(a.next, 1u) : 0u;
    for (;;) {
        if (tid == 0) {
            s_item = next_id;
            s_abort = 0;
        }
        __syncthreads();
        const unsigned id = s_item;
        if (id >= total) break;
        const int t = (int)(id / (unsigned)a.items_per_step);
        const int k = (int)(id % (unsigned)a.items_per_step);
        const int s = a.item_sys[k];
        const int c = a.item_chunk[k];
        const int64_t b0 = a.off[s];
        const int64_t n = a.off[s + 1] - b0;
        const int64_t p0 = a.poff[s];
        const int ntl = (int)((n + a.jt - 1) / a.jt);
        const int64_t lo = (int64_t)c * NT * R;
        const int64_t hi = lo + (int64_t)NT * R < n ? lo + (int64_t)NT * R : n;
        const float4 *src = ((t & 1) ? a.xm1 : a.xm0) + p0;  // one float4 per body
        float4 *dst = ((t & 1) ? a.xm0 : a.xm1) + p0;
        if (tid == 0) {
            // step t of system s needs every item of its step t-1
            if (t > 0 && !wait_at_least(a.done + s, (unsigned)t * (unsigned)a.nchunks[s], a.timeout_ns)) {
                atomicOr(a.err, kErrGang);
                s_abort = 1;
            }
            fence_proxy_async_global();
            next_id = atomicAdd(a.next, 1u);
        }
        __syncthreads();
        const bool run = !s_abort && !give_up;
        if (tid == 0 && run)
            for (int q = 0; q < ntl && q < kLead && !give_up; ++q)
                issue(kk + q, src + (int64_t)q * f4_per_tile);
        AccelF32x2::I ist[R];
        AccelF32x2::T tot[R];
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
        if (run) {
            for (int q = 0; q < ntl; ++q) {
                const uint32_t pos = kk + q;
                const int slot = pos % kBS;
                if (!give_up && !mbar_wait(&full[slot], (pos / kBS) & 1, a.timeout_ns)) {
                    atomicOr(a.err, kErrFullWait);
                    give_up = true;
                }
                if (!give_up) {
                    const float4 *tile = ring + slot * f4_per_tile;
#pragma unroll(AccelF32x2::UNROLL)
                    for (int jp = 0; jp < (a.jt >> 1); ++jp) {
                        float4 rec[2] = {tile[2 * jp], tile[2 * jp + 1]};
#pragma unroll
                        for (int r = 0; r < R; ++r) AccelF32x2::interact(rec, ist[r], tot[r], cst);
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&empty[slot]);
                }
                // refill: position pos + kLead goes into the slot of pos - 2
                if (tid == 0 && !give_up && q + kLead < ntl)
                    issue(pos + kLead, src + (int64_t)(q + kLead) * f4_per_tile);
            }
            kk += ntl;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int64_t i = lo + r * NT + tid;
                if (i < hi) {
                    const float acc[3] = {a.G * (tot[r].x.x + tot[r].x.y), a.G * (tot[r].y.x + tot[r].y.y),
                                          a.G * (tot[r].z.x + tot[r].z.y)};
                    float *xp = a.x + 3 * (b0 + i);
                    float *vp = a.v + 3 * (b0 + i);
                    float xs[3];
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc) {
                        // v += a dt/2 (the printed half kick); x += v dt
                        const float vc = __fadd_rn(__ldcg(vp + cc), __fmul_rn(__fmul_rn(acc[cc], dt), 0.5f));
                        vp[cc] = vc;
                        xs[cc] = __fadd_rn(__ldcg(xp + cc), __fmul_rn(vc, dt));
                        xp[cc] = xs[cc];
                    }
                    pair_put(dst, i, xs[0], xs[1], xs[2], pair_get_cg(src, i, 3));
                }
            }
            fence_proxy_async_global();
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            atomicAdd(a.done + s, 1u);  // release this item to step t+1
        }
    }
    // never leave while our own copies may still be landing
    if (tid == 0) {
        for (uint32_t q = issued > (uint32_t)kBS ? issued - kBS : 0; q < issued; ++q) {
            if (!mbar_wait(&full[q % kBS], (q / kBS) & 1, kDrainTimeoutNs))
                atomicOr(a.err, kErrDrain);
        }
    }
}

__global__ void batched_pack_kernel(const int64_t *off, const int64_t *poff, int jt,
                                    const float *x, const float *m, float4 *xm) {
    const int s = blockIdx.x;
    const int64_t b0 = off[s], n = off[s + 1] - b0, p0 = poff[s];
    const int64_t npad = (n + jt - 1) / jt * jt;
    for (int64_t i = threadIdx.x; i < npad; i += blockDim.x) {
        if (i < n)
            pair_put(xm + p0, i, x[3 * (b0 + i)], x[3 * (b0 + i) + 1], x[3 * (b0 + i) + 2],
                     m[b0 + i]);
        else
            pair_put(xm + p0, i, 0.f, 0.f, 0.f, 0.f);
    }
}

__global__ void batched_fill_kernel(const int64_t *off, float *x, float *v, float *m) {
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
            x[3 * g + c] = 2.f * u - 1.f;
            v[3 * g + c] = 0.1f * (u - 0.5f);
        }
        m[g] = 1.0f / (float)n;
    }
}

template <int NT, int R>
size_t batched_smem(int jt) {
    return 128 + (size_t)kBS * jt * 16;
}

// Device copy of the plan inside the scratch block.
struct Layout {
    size_t o_off, o_poff, o_isys, o_ichunk, o_nch, o_next, o_done, o_xm0, o_xm1, total;
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
    L.o_ichunk = take(p.item_chunk.size() * 4);
    L.o_nch = take(p.nchunks.size() * 4);
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
    p.nsys = (int)off.size() - 1;
    if (p.nt == 0) p.nt = 128;
    if (p.r == 0) p.r = 2;
    if (p.jt == 0) p.jt = 64;
    if (p.nt != 128 || (p.r != 1 && p.r != 2 && p.r != 4) || p.jt % 2 || kPadBodies % p.jt) {
        why = "unsupported batched shape";
        return false;
    }
    int occ = 0;
    cudaError_t e;
    const size_t smem = batched_smem<128, 2>(p.jt);
    if (p.r == 1)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batched_kernel<128, 1>, 128, smem);
    else if (p.r == 2)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batched_kernel<128, 2>, 128, smem);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batched_kernel<128, 4>, 128, smem);
    if (e != cudaSuccess || occ <= 0) {
        why = "occupancy query failed";
        return false;
    }
    p.off = off;
    p.poff.assign(p.nsys, 0);
    p.nchunks.assign(p.nsys, 0);
    p.total = off[p.nsys];
    const int64_t chunk = (int64_t)p.nt * p.r;
    int64_t acc = 0;
    for (int s = 0; s < p.nsys; ++s) {
        const int64_t n = off[s + 1] - off[s];
        p.poff[s] = acc;
        acc += (n + p.jt - 1) / p.jt * p.jt;
        p.nchunks[s] = (int)((n + chunk - 1) / chunk);
    }
    p.total_pad = std::max<int64_t>(acc, p.jt);
    // items of one step: largest systems first, chunks in order
    std::vector<int> order(p.nsys);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return off[a + 1] - off[a] > off[b + 1] - off[b];
    });
    p.item_sys.clear();
    p.item_chunk.clear();
    for (int s : order)
        for (int c = 0; c < p.nchunks[s]; ++c) {
            p.item_sys.push_back(s);
            p.item_chunk.push_back(c);
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
    NB_UP(item_chunk, L.o_ichunk)
    NB_UP(nchunks, L.o_nch)
#undef NB_UP
    return cudaSuccess;
}

cudaError_t batched_fill_synthetic(const BatchPlan &p, void *scratch, float *x, float *v,
                                   float *m, cudaStream_t st) {
    Layout L = layout_of(p);
    batched_fill_kernel<<<p.nsys, 256, 0, st>>>((const int64_t *)((char *)scratch + L.o_off), x, v,
                                                m);
    return cudaGetLastError();
}

cudaError_t batched_enqueue(const BatchPlan &p, void *scratch, float *x, float *v, const float *m,
                            int steps, float eps2, float G, float dt, int *err,
                            uint64_t timeout_ns, cudaStream_t st) {
    if ((uint64_t)p.items_per_step * (uint64_t)steps + (uint64_t)p.ncta >= (1ull << 32))
        return cudaErrorInvalidValue;
    Layout L = layout_of(p);
    char *b = (char *)scratch;
    BatchArgs a;
    a.off = (const int64_t *)(b + L.o_off);
    a.poff = (const int64_t *)(b + L.o_poff);
    a.item_sys = (const int *)(b + L.o_isys);
    a.item_chunk = (const int *)(b + L.o_ichunk);
    a.nchunks = (const int *)(b + L.o_nch);
    a.next = (unsigned *)(b + L.o_next);
    a.done = (unsigned *)(b + L.o_done);
    a.xm0 = (float4 *)(b + L.o_xm0);
    a.xm1 = (float4 *)(b + L.o_xm1);
    a.x = x;
    a.v = v;
    a.steps = steps;
    a.jt = p.jt;
    a.items_per_step = p.items_per_step;
    a.eps2 = eps2;
    a.G = G;
    a.dt = dt;
    a.err = err;
    a.timeout_ns = timeout_ns;
    cudaError_t e = cudaMemsetAsync(b + L.o_next, 0, L.o_xm0 - L.o_next, st);
    if (e != cudaSuccess) return e;
    batched_pack_kernel<<<p.nsys, 256, 0, st>>>(a.off, a.poff, p.jt, x, m, a.xm0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = dim3((unsigned)p.ncta);
    cfg.blockDim = dim3((unsigned)p.nt);
    cfg.dynamicSmemBytes = batched_smem<128, 2>(p.jt);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (p.r == 1) return cudaLaunchKernelEx(&cfg, batched_kernel<128, 1>, a);
    if (p.r == 2) return cudaLaunchKernelEx(&cfg, batched_kernel<128, 2>, a);
    return cudaLaunchKernelEx(&cfg, batched_kernel<128, 4>, a);
}

}  // namespace nb
