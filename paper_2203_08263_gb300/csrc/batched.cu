// Persistent ensemble kernel: every system of the batch advances `steps`
// paper steps inside one cooperative launch. CTAs are grouped in gangs; a
// gang walks its list of systems, and for each step every member computes the
// forces on its slice of i-bodies from all j-bodies of the system (j-tiles
// streamed by 1-D bulk copies, issued by thread 0, through a shared-memory
// ring as in the single-system kernel), applies the half kick and the drift,
// writes the repacked positions to the other buffer and meets the rest of the
// gang at a bounded global-memory barrier before the next step.
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
    const int *work, *gang_first, *cta_gang, *cta_rank, *gang_size;
    unsigned *gang_ctr;
    float4 *xm0, *xm1;
    float *x, *v;
    int steps, jt;
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

// All gang members reach the barrier `epoch` times before anyone passes it
// the epoch-th time. The wait is bounded; on timeout an error bit is set and
// the CTA goes on (its results are then flagged invalid by the host).
__device__ void gang_barrier(unsigned *ctr, unsigned target, uint64_t timeout_ns, int *err) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1u);
        if (ld_acquire(ctr) < target) {
            const uint64_t t0 = global_ns();
            while (ld_acquire(ctr) < target) {
                __nanosleep(64);
                if (global_ns() - t0 > timeout_ns) {
                    atomicOr(err, kErrGang);
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
}

template <int NT, int R>
__global__ void __launch_bounds__(NT, (R <= 2 ? 4 : 2)) batched_kernel(const BatchArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw);
    uint64_t *empty = full + kStages;
    float4 *ring = reinterpret_cast<float4 *>(smem_raw + 128);
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int gang = a.cta_gang[blockIdx.x];
    const int rank = a.cta_rank[blockIdx.x];
    const int gsz = a.gang_size[gang];
    unsigned *ctr = a.gang_ctr + gang;
    const int f4_per_tile = a.jt;  // (jt / 2) records x 2 float4
    const uint32_t tile_bytes = (uint32_t)f4_per_tile * 16u;
    const float dt = a.dt;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NT / 32);
        }
        mbar_init_fence();
    }
    __syncthreads();

    // Ring position q (tiles streamed so far by this CTA) runs on across
    // passes, steps and systems; slot q % kStages, phase q / kStages. Thread 0
    // issues position q once position q - kStages has been released.
    uint32_t kk = 0;       // position of the current pass's first tile
    uint32_t issued = 0;   // positions issued so far (thread 0)
    unsigned epoch = 0;    // gang barriers passed
    bool give_up = false;  // a wait failed: stop streaming, keep the barriers

    auto issue = [&](uint32_t q, const float4 *src_tile) {
        const int slot = q % kStages;
        if (q >= (uint32_t)kStages &&
            !mbar_wait(&empty[slot], ((q / kStages) - 1) & 1, a.timeout_ns)) {
            atomicOr(a.err, kErrEmptyWait);
            give_up = true;
            return;
        }
        mbar_arrive_expect_tx(&full[slot], tile_bytes);
        bulk_g2s(ring + slot * f4_per_tile, src_tile, tile_bytes, &full[slot]);
        issued = q + 1;
    };

    for (int w = a.gang_first[gang]; w < a.gang_first[gang + 1]; ++w) {
        const int s = a.work[w];
        const int64_t b0 = a.off[s];
        const int64_t n = a.off[s + 1] - b0;
        const int64_t p0 = a.poff[s];
        const int64_t npad = (n + a.jt - 1) / a.jt * a.jt;
        const int ntl = (int)(npad / a.jt);
        const int64_t chunk = (n + gsz - 1) / gsz;
        const int64_t lo = (int64_t)rank * chunk;
        const int64_t hi = lo + chunk < n ? lo + chunk : n;
        const int passes = hi > lo ? (int)((hi - lo + (int64_t)NT * R - 1) / ((int64_t)NT * R)) : 0;
        for (int t = 0; t < a.steps; ++t) {
            const float4 *src = ((t & 1) ? a.xm1 : a.xm0) + p0;  // one float4 per body
            float4 *dst = ((t & 1) ? a.xm0 : a.xm1) + p0;
            if (tid == 0) fence_proxy_async_global();
            for (int ps = 0; ps < passes; ++ps) {
                if (tid == 0 && !give_up)
                    for (int k = 0; k < ntl && k < kStages - 1 && !give_up; ++k)
                        issue(kk + k, src + (int64_t)k * f4_per_tile);
                const int64_t ibase = lo + (int64_t)ps * NT * R;
                AccelF32x2::I ist[R];
                AccelF32x2::T tot[R];
                AccelF32x2::C cst;
                cst.eps2 = dup(a.eps2);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    int64_t i = ibase + r * NT + tid;
                    if (i >= hi) i = lo;
                    ist[r].nx = dup(-pair_get(src, i, 0));
                    ist[r].ny = dup(-pair_get(src, i, 1));
                    ist[r].nz = dup(-pair_get(src, i, 2));
                    AccelF32x2::zero_total(tot[r]);
                }
                for (int k = 0; k < ntl; ++k) {
                    const uint32_t q = kk + k;
                    const int slot = q % kStages;
                    if (!give_up && !mbar_wait(&full[slot], (q / kStages) & 1, a.timeout_ns)) {
                        atomicOr(a.err, kErrFullWait);
                        give_up = true;
                    }
                    if (!give_up) {
                        const float4 *tile = ring + slot * f4_per_tile;
#pragma unroll 2
                        for (int jp = 0; jp < (a.jt >> 1); ++jp) {
                            float4 rec[2] = {tile[2 * jp], tile[2 * jp + 1]};
#pragma unroll
                            for (int r = 0; r < R; ++r) AccelF32x2::interact(rec, ist[r], tot[r], cst);
                        }
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&empty[slot]);
                    }
                    // refill: position q + kStages - 1 goes into the slot of q - 1
                    if (tid == 0 && !give_up && k + kStages - 1 < ntl)
                        issue(q + kStages - 1, src + (int64_t)(k + kStages - 1) * f4_per_tile);
                }
                kk += ntl;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int64_t i = ibase + r * NT + tid;
                    if (i < hi) {
                        const float ax = a.G * (tot[r].x.x + tot[r].x.y);
                        const float ay = a.G * (tot[r].y.x + tot[r].y.y);
                        const float az = a.G * (tot[r].z.x + tot[r].z.y);
                        float *xp = a.x + 3 * (b0 + i);
                        float *vp = a.v + 3 * (b0 + i);
                        const float acc[3] = {ax, ay, az};
                        float xs[3];
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            // v += a dt/2 (the printed half kick); x += v dt
                            float vc = __fadd_rn(vp[c], __fmul_rn(__fmul_rn(acc[c], dt), 0.5f));
                            vp[c] = vc;
                            xs[c] = __fadd_rn(xp[c], __fmul_rn(vc, dt));
                            xp[c] = xs[c];
                        }
                        pair_put(dst, i, xs[0], xs[1], xs[2], pair_get(src, i, 3));
                    }
                }
            }
            // the whole system moves before anyone reads the next positions
            fence_proxy_async_global();
            ++epoch;
            gang_barrier(ctr, epoch * (unsigned)gsz, a.timeout_ns, a.err);
        }
    }
    // never leave while our own copies may still be landing
    if (tid == 0) {
        for (uint32_t q = issued > (uint32_t)kStages ? issued - kStages : 0; q < issued; ++q) {
            if (!mbar_wait(&full[q % kStages], (q / kStages) & 1, kDrainTimeoutNs))
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
    return 128 + (size_t)kStages * jt * 16;
}

// Device copy of the plan inside the scratch block.
struct Layout {
    size_t o_off, o_poff, o_work, o_gf, o_cg, o_cr, o_gs, o_ctr, o_xm0, o_xm1, total;
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
    L.o_work = take(p.work.size() * 4);
    L.o_gf = take(p.gang_first.size() * 4);
    L.o_cg = take(p.cta_gang.size() * 4);
    L.o_cr = take(p.cta_rank.size() * 4);
    L.o_gs = take(p.gang_size.size() * 4);
    L.o_ctr = take((size_t)p.ngang * 4);
    L.o_xm0 = take((size_t)p.total_pad * 16);
    L.o_xm1 = take((size_t)p.total_pad * 16);
    L.total = o;
    return L;
}

// per-CTA time of system (n) on a gang of g CTAs, in tile-pass units
double sys_time(int64_t n, int g, int nt, int r, int jt) {
    const int64_t chunk = (n + g - 1) / g;
    const int64_t passes = (chunk + (int64_t)nt * r - 1) / ((int64_t)nt * r);
    const int64_t ntl = (n + jt - 1) / jt;
    const double beta = 6.0;  // per-step latency: ring fill, epilogue, barrier
    return (double)passes * ntl + beta;
}

// Longest-processing-time-first packing of `items` (time, id) onto k bins.
double lpt(const std::vector<std::pair<double, int>> &items, int k, std::vector<int> *assign) {
    std::vector<double> load(k, 0.0);
    if (assign) assign->assign(items.size(), 0);
    for (size_t q = 0; q < items.size(); ++q) {
        int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[b] += items[q].first;
        if (assign) (*assign)[q] = b;
    }
    return *std::max_element(load.begin(), load.end());
}

}  // namespace

int64_t batched_max_n() { return int64_t(1) << 20; }

bool batched_plan(int device, int num_sms, const std::vector<int64_t> &off, BatchPlan &p,
                  std::string &why) {
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
    (void)device;
    const int P = occ * num_sms;
    p.off = off;
    p.poff.assign(p.nsys, 0);
    p.total = off[p.nsys];
    int64_t acc = 0;
    for (int s = 0; s < p.nsys; ++s) {
        p.poff[s] = acc;
        acc += (off[s + 1] - off[s] + p.jt - 1) / p.jt * p.jt;
    }
    p.total_pad = std::max<int64_t>(acc, p.jt);

    // gang sizes and LPT assignment under a makespan bound T (bisection)
    const int gmax = std::max(1, std::min(p.gmax > 0 ? p.gmax : 16, P));
    std::vector<int> sizes;
    for (int g = 1; g <= gmax; g *= 2) sizes.push_back(g);
    double lb = 0.0, work = 0.0;
    for (int s = 0; s < p.nsys; ++s) {
        const int64_t n = off[s + 1] - off[s];
        if (n == 0) continue;
        work += sys_time(n, 1, p.nt, p.r, p.jt);
        lb = std::max(lb, sys_time(n, gmax, p.nt, p.r, p.jt));
    }
    lb = std::max(lb, work / P);
    std::map<int, std::vector<std::pair<double, int>>> groups;
    std::map<int, int> kg;
    auto feasible = [&](double T, bool commit) -> bool {
        std::map<int, std::vector<std::pair<double, int>>> gr;
        for (int s = 0; s < p.nsys; ++s) {
            const int64_t n = off[s + 1] - off[s];
            if (n == 0) continue;
            int gs = gmax;
            for (int g : sizes)
                if (sys_time(n, g, p.nt, p.r, p.jt) <= T) { gs = g; break; }
            gr[gs].push_back({sys_time(n, gs, p.nt, p.r, p.jt), s});
        }
        int used = 0;
        std::map<int, int> kk;
        for (auto &kv : gr) {
            auto &items = kv.second;
            std::sort(items.begin(), items.end(), [](auto &A, auto &B) {
                return A.first > B.first || (A.first == B.first && A.second < B.second);
            });
            double tot = 0;
            for (auto &it : items) tot += it.first;
            int k = std::max(1, (int)std::ceil(tot / T));
            while (k < (int)items.size() && lpt(items, k, nullptr) > T) ++k;
            k = std::min<int>(k, (int)items.size());
            kk[kv.first] = k;
            used += k * kv.first;
        }
        if (used > P) return false;
        if (commit) {
            groups = gr;
            kg = kk;
        }
        return true;
    };
    double lo = lb, hi = lb;
    while (!feasible(hi, false)) {
        hi *= 1.5;
        if (hi > 1e15) { why = "no feasible schedule"; return false; }
    }
    for (int it = 0; it < 40; ++it) {
        double mid = 0.5 * (lo + hi);
        if (feasible(mid, false)) hi = mid; else lo = mid;
    }
    feasible(hi, true);
    p.makespan_tiles = hi;

    p.work.clear();
    p.gang_first.assign(1, 0);
    p.cta_gang.clear();
    p.cta_rank.clear();
    p.gang_size.clear();
    for (auto &kv : groups) {
        const int g = kv.first;
        const int k = kg[g];
        std::vector<int> assign;
        lpt(kv.second, k, &assign);
        for (int b = 0; b < k; ++b) {
            const int gang = (int)p.gang_size.size();
            p.gang_size.push_back(g);
            for (size_t q = 0; q < kv.second.size(); ++q)
                if (assign[q] == b) p.work.push_back(kv.second[q].second);
            p.gang_first.push_back((int)p.work.size());
            for (int rnk = 0; rnk < g; ++rnk) {
                p.cta_gang.push_back(gang);
                p.cta_rank.push_back(rnk);
            }
        }
    }
    if (p.work.empty()) {  // only empty systems: one idle gang
        p.gang_size.push_back(1);
        p.gang_first.push_back(0);
        p.cta_gang.push_back(0);
        p.cta_rank.push_back(0);
    }
    p.ngang = (int)p.gang_size.size();
    p.ncta = (int)p.cta_gang.size();
    Layout L = layout_of(p);
    p.plan_bytes = L.o_ctr;
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
    mix((uint64_t)p.gmax);
    p.signature = h;
    return true;
}

cudaError_t batched_upload(const BatchPlan &p, void *scratch, cudaStream_t st) {
    Layout L = layout_of(p);
    char *b = (char *)scratch;
    cudaError_t e;
#define NB_UP(field, o)                                                                      \
    e = cudaMemcpyAsync(b + (o), p.field.data(), p.field.size() * sizeof(p.field[0]),       \
                        cudaMemcpyHostToDevice, st);                                         \
    if (e != cudaSuccess) return e;
    NB_UP(off, L.o_off)
    NB_UP(poff, L.o_poff)
    NB_UP(work, L.o_work)
    NB_UP(gang_first, L.o_gf)
    NB_UP(cta_gang, L.o_cg)
    NB_UP(cta_rank, L.o_cr)
    NB_UP(gang_size, L.o_gs)
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
    Layout L = layout_of(p);
    char *b = (char *)scratch;
    BatchArgs a;
    a.off = (const int64_t *)(b + L.o_off);
    a.poff = (const int64_t *)(b + L.o_poff);
    a.work = (const int *)(b + L.o_work);
    a.gang_first = (const int *)(b + L.o_gf);
    a.cta_gang = (const int *)(b + L.o_cg);
    a.cta_rank = (const int *)(b + L.o_cr);
    a.gang_size = (const int *)(b + L.o_gs);
    a.gang_ctr = (unsigned *)(b + L.o_ctr);
    a.xm0 = (float4 *)(b + L.o_xm0);
    a.xm1 = (float4 *)(b + L.o_xm1);
    a.x = x;
    a.v = v;
    a.steps = steps;
    a.jt = p.jt;
    a.eps2 = eps2;
    a.G = G;
    a.dt = dt;
    a.err = err;
    a.timeout_ns = timeout_ns;
    cudaError_t e = cudaMemsetAsync(a.gang_ctr, 0, (size_t)p.ngang * 4, st);
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
