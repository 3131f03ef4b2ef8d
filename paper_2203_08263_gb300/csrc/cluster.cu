// Small systems: every step of nb_run in one launch of one thread-block
// cluster. The force sum (Eq. 1 with softening, as the single-system kernel)
// and the printed update (half kick v += a dt/2, drift x += v dt with the new
// v; or the kick-drift-kick variant) are the same arithmetic as the graph
// path; what differs is where the state lives between steps. Each CTA of the
// cluster keeps a full replica of the packed positions in its shared memory
// (two buffers), owns a contiguous slice of the bodies and keeps their x and v
// in registers. Per step it sums the forces on its slice against its own
// replica, updates the slice, writes the slice's new packed records into the
// other buffer of every CTA through distributed shared memory, and meets the
// others at one cluster barrier. No global memory is touched between the
// first load and the final store (checkpoints aside), and no kernel boundary
// separates the steps: at N of a few thousand the graph path's per-step
// launch, bulk-copy and split-reduction latencies dominate, and this path
// removes them. Its grid form (N <= 8192) spreads the slices over a
// cooperative grid of up to one CTA per SM instead of one cluster's 16: the
// records go through a global double buffer and a bounded grid barrier, and
// each CTA reloads all of them from L2 every step.
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "kernels.h"
#include "engine.cuh"

namespace nb {

namespace {

struct ClusterArgs {
    int n, npad, slice;  // bodies, cluster size x slice, bodies per CTA (even)
    int steps, kdk;      // paper steps; 1: kick-drift-kick scheme
    float eps2;
    double G, dt;
    void *x, *v;         // [n][3] in the state type, updated in place
    const void *m;       // [n] in the state type
    void *ckpt;          // nullable: slots of [n][6] (x, v), slot s after step s * ckpt_every
    int ckpt_every;
    // grid form only
    float4 *xm0, *xm1;   // packed positions in global memory, [npad] each, double-buffered
    unsigned *bar;       // grid barrier: [0] arrivals, cumulative over the launch; [1] CTAs done.
                         // Both zero at the start of a launch; the last CTA to finish zeroes them
    int *err;
    uint64_t timeout_ns;
    int stall;           // timeout tests: CTA 0 never arrives, so every barrier wait runs out
};

__device__ __forceinline__ unsigned ld_relaxed_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier of the grid form (all CTAs resident: cooperative
// launch). Arrivals accumulate over the launch; barrier number `epoch`
// completes when epoch x gridDim.x CTAs have arrived. Bounded: after
// timeout_ns the CTA records an error and returns false (it then leaves the
// step loop, so the others give up at their next barrier too).
__device__ __forceinline__ bool grid_barrier(const ClusterArgs &a, unsigned epoch, int *s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        // the writers fenced their records before the __syncthreads
        if (!(a.stall && blockIdx.x == 0)) atomicAdd(a.bar, 1u);
        const unsigned target = epoch * gridDim.x;
        int ok = 1;
        if (ld_relaxed_gpu(a.bar) < target) {
            const uint64_t t0 = global_ns();
            while (ld_relaxed_gpu(a.bar) < target) {
                __nanosleep(32);
                if (global_ns() - t0 > a.timeout_ns) {
                    atomicOr(a.err, kErrStepDep);
                    ok = 0;
                    break;
                }
            }
        }
        asm volatile("fence.acq_rel.gpu;" ::: "memory");  // the others' records after it
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t cluster_nctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_to_rank(uint32_t smem, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem), "r"(rank));
    return r;
}

__device__ __forceinline__ void st_cluster_f4(uint32_t addr, float4 v) {
    asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x),
                 "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

// Every thread of every CTA of the cluster arrives (release) and waits
// (acquire): remote shared-memory stores before it are visible after it.
__device__ __forceinline__ void cluster_barrier() {
    __syncwarp();  // the .aligned form wants the whole warp converged here
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::
                     : "memory");
}

// Pair-sum block of the precision form: FP32 packed partial sums over this
// many j-pairs of a lane, then a two-sum into the lane's (hi, lo) total, as
// the graph path does per 64-body tile.
constexpr int kCompBlockPairs = 32;

// F64 = false: FP32 state and forces (AccelF32x2). F64 = true: the precision
// form, FP64 state, FP32 pair terms summed in blocks, two-sums across blocks,
// FP64 across lanes and in the update (AccelComp's arithmetic).
// GRID = false: one thread-block cluster, replicas exchanged through
// distributed shared memory. GRID = true: a cooperative grid of up to one CTA
// per SM; each step every CTA writes its slice's records to a global buffer,
// meets the others at a grid barrier and reloads all records into its shared
// memory.
// RB = bodies per lane in the force sum (1, or 2 for slices of 64 or more:
// each j-record then feeds four interactions instead of two, halving the
// shared-memory traffic per interaction).
template <int NT, bool F64, bool GRID, int RB>
__global__ void __launch_bounds__(NT, 1) cluster_run_kernel(const ClusterArgs a) {
    using TS = typename std::conditional<F64, double, float>::type;
    extern __shared__ __align__(16) float4 rep[];  // cluster: [2][npad]; grid: [npad]
    const TS *xg = reinterpret_cast<const TS *>(a.x);
    const TS *vg = reinterpret_cast<const TS *>(a.v);
    const TS *mg = reinterpret_cast<const TS *>(a.m);
    TS *ckpt = reinterpret_cast<TS *>(a.ckpt);
    const int tid = threadIdx.x;
    const uint32_t rank = GRID ? blockIdx.x : cluster_ctarank();
    const uint32_t csize = GRID ? gridDim.x : cluster_nctarank();
    __shared__ int s_ok;
    const int S = a.slice;
    const int npad = a.npad;
    // Thread mapping of the force sum: lane l of warp w sums the RB bodies in
    // slots (w / Q) * 32 RB + r * 32 + l over the j-pairs jq, jq + Q, ... with
    // jq = w % Q, so all lanes of a warp read the same j-record (a broadcast
    // load: the j-split across lanes of one warp cost 8 shared-memory
    // wavefronts per 16-byte load). The Q partial sums of a body meet in
    // shared memory.
    constexpr int kRow = 32 * RB;                    // body slots per warp row
    const int spad = (S + kRow - 1) / kRow * kRow;   // body slots in whole rows
    const int rows = spad / kRow;
    const int Q = (NT / 32) / rows;                  // j-splits per body (>= 1)
    const int warp = tid >> 5, lane = tid & 31;
    const int jq = warp % Q;
    const bool in_row = warp < Q * rows;
    int il[RB], i[RB];  // body slots of this lane, their global indices
    bool act[RB];       // the slot holds a body of the slice
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        il[r] = (warp / Q) * kRow + r * 32 + lane;
        act[r] = in_row && il[r] < S;
        i[r] = (int)rank * S + (act[r] ? il[r] : 0);
    }
    const bool active = act[0];  // slot 0 of a lane is filled first
    // The thread that keeps body io's x and v and updates it: thread k of the
    // CTA for body k of the slice (the update's FP64 in the precision form is
    // slow on this part; compact owners fill ceil(S / 32) warps).
    const int io = (int)rank * S + tid;
    const bool owner = tid < S && io < a.n;
    __shared__ float s_red[NT * RB * (F64 ? 6 : 3)];  // per (split, body slot): partial sums (hi, lo)
    if constexpr (!GRID) {
        // both replicas: every body's record in buffer 0, zeros in buffer 1
        for (int k = tid; k < npad; k += NT) {
            if (k < a.n)
                pair_put(rep, k, (float)xg[3 * k], (float)xg[3 * k + 1], (float)xg[3 * k + 2], (float)mg[k]);
            else
                pair_put(rep, k, 0.f, 0.f, 0.f, 0.f);
            pair_put(rep + npad, k, 0.f, 0.f, 0.f, 0.f);
        }
    } else if (tid < S) {
        // this CTA's slice of both global buffers: records (zeros past n)
        const int k = (int)rank * S + tid;
        if (k < a.n)
            pair_put(a.xm0, k, (float)xg[3 * k], (float)xg[3 * k + 1], (float)xg[3 * k + 2], (float)mg[k]);
        else
            pair_put(a.xm0, k, 0.f, 0.f, 0.f, 0.f);
        pair_put(a.xm1, k, 0.f, 0.f, 0.f, 0.f);
        __threadfence();  // these records before the CTA's arrival at the barrier
    }
    TS xs[3] = {0, 0, 0}, vs[3] = {0, 0, 0};
    float mi = 0.f;
    if (owner) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            xs[c] = xg[3 * io + c];
            vs[c] = vg[3 * io + c];
        }
        mi = (float)mg[io];
        if (ckpt) {
            TS *ck = ckpt + 6 * (int64_t)io;
            ck[0] = xs[0]; ck[1] = xs[1]; ck[2] = xs[2];
            ck[3] = vs[0]; ck[4] = vs[1]; ck[5] = vs[2];
        }
    }
    // no CTA writes into another's buffer 1 before that one has zeroed it
    // (grid: no CTA reads buffer 0 before every slice of it is written)
    bool ok = true;
    if constexpr (GRID) ok = grid_barrier(a, 1u, &s_ok);
    else cluster_barrier();

    const int evals = a.steps + (a.kdk && a.steps > 0 ? 1 : 0);
    int cur = 0;
    for (int t = 0; ok && t < evals; ++t) {
        const float4 *src;
        float4 *dst;
        if constexpr (GRID) {
            const float4 *g = cur ? a.xm1 : a.xm0;
            for (int k = tid; k < npad; k += NT) rep[k] = __ldcg(g + k);  // all records, from L2
            __syncthreads();
            src = rep;
            dst = cur ? a.xm0 : a.xm1;
        } else {
            src = rep + cur * npad;
            dst = rep + (cur ^ 1) * npad;
        }
        TS ax = 0, ay = 0, az = 0;
        AccelF32x2::I ist[RB];
        AccelF32x2::C cst;
        cst.eps2 = dup(a.eps2);
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            ist[r].nx = dup(-pair_get(src, i[r], 0));
            ist[r].ny = dup(-pair_get(src, i[r], 1));
            ist[r].nz = dup(-pair_get(src, i[r], 2));
        }
        const int npairs = npad >> 1;
        if constexpr (!F64) {
            if (active) {
                AccelF32x2::T tot[RB];
#pragma unroll
                for (int r = 0; r < RB; ++r) AccelF32x2::zero_total(tot[r]);
#pragma unroll 4
                for (int p = jq; p < npairs; p += Q) {
                    const float4 rec[2] = {src[2 * p], src[2 * p + 1]};
#pragma unroll
                    for (int r = 0; r < RB; ++r) AccelF32x2::interact(rec, ist[r], tot[r], cst);
                }
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    if (!act[r]) continue;
                    float *rr = s_red + 3 * (jq * spad + il[r]);
                    rr[0] = tot[r].x.x + tot[r].x.y;
                    rr[1] = tot[r].y.x + tot[r].y.y;
                    rr[2] = tot[r].z.x + tot[r].z.y;
                }
            }
            __syncthreads();
            if (owner) {
                for (int q = 0; q < Q; ++q) {  // the body's splits in order
                    const float *rr = s_red + 3 * (q * spad + tid);
                    ax += rr[0];
                    ay += rr[1];
                    az += rr[2];
                }
            }
        } else {
            // blocks of FP32 partial sums two-summed into (hi, lo) per split ...
            if (active) {
                float h[RB][3], l[RB][3];
#pragma unroll
                for (int r = 0; r < RB; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c) h[r][c] = l[r][c] = 0.f;
                for (int p0 = jq; p0 < npairs; p0 += Q * kCompBlockPairs) {
                    AccelF32x2::T blk[RB];
#pragma unroll
                    for (int r = 0; r < RB; ++r) AccelF32x2::zero_total(blk[r]);
                    const int pend = min(npairs, p0 + Q * kCompBlockPairs);
#pragma unroll 4
                    for (int p = p0; p < pend; p += Q) {
                        const float4 rec[2] = {src[2 * p], src[2 * p + 1]};
#pragma unroll
                        for (int r = 0; r < RB; ++r) AccelF32x2::interact(rec, ist[r], blk[r], cst);
                    }
#pragma unroll
                    for (int r = 0; r < RB; ++r) {
                        const float b3[3] = {blk[r].x.x + blk[r].x.y, blk[r].y.x + blk[r].y.y,
                                             blk[r].z.x + blk[r].z.y};
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            float sum, err;
                            two_sum(h[r][c], b3[c], sum, err);
                            h[r][c] = sum;
                            l[r][c] += err;
                        }
                    }
                }
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    if (!act[r]) continue;
                    float *rr = s_red + 6 * (jq * spad + il[r]);
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        rr[c] = h[r][c];
                        rr[3 + c] = l[r][c];
                    }
                }
            }
            __syncthreads();
            // ... the splits folded with FP32 two-sums in order, widened once
            if (owner) {
                float h[3] = {0.f, 0.f, 0.f}, l[3] = {0.f, 0.f, 0.f};
                for (int q = 0; q < Q; ++q) {
                    const float *rr = s_red + 6 * (q * spad + tid);
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        float sum, err;
                        two_sum(h[c], rr[c], sum, err);
                        h[c] = sum;
                        l[c] = __fadd_rn(l[c], __fadd_rn(rr[3 + c], err));
                    }
                }
                ax = (double)h[0] + (double)l[0];
                ay = (double)h[1] + (double)l[1];
                az = (double)h[2] + (double)l[2];
            }
        }
        const bool last_kick = a.kdk && t == a.steps;  // the closing half kick of KDK
        if (owner) {
            const bool double_kick = a.kdk && t > 0 && !last_kick;
            if constexpr (!F64) {
                const float G = (float)a.G, dt = (float)a.dt;
                const float acc[3] = {G * ax, G * ay, G * az};
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    // v <- v + a*dt/2 (twice between two drifts of the KDK scheme), then x += v*dt
                    float vc = __fadd_rn(vs[c], __fmul_rn(__fmul_rn(acc[c], dt), 0.5f));
                    if (double_kick) vc = __fadd_rn(vc, __fmul_rn(__fmul_rn(acc[c], dt), 0.5f));
                    vs[c] = vc;
                    if (!last_kick) xs[c] = __fadd_rn(xs[c], __fmul_rn(vc, dt));
                }
            } else {
                const double acc[3] = {a.G * ax, a.G * ay, a.G * az};
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    double vc = __dadd_rn(vs[c], __dmul_rn(__dmul_rn(acc[c], a.dt), 0.5));
                    if (double_kick) vc = __dadd_rn(vc, __dmul_rn(__dmul_rn(acc[c], a.dt), 0.5));
                    vs[c] = vc;
                    if (!last_kick) xs[c] = __dadd_rn(xs[c], __dmul_rn(vc, a.dt));
                }
            }
            if (!last_kick) {
                pair_put(dst, io, (float)xs[0], (float)xs[1], (float)xs[2], mi);
                if constexpr (GRID) __threadfence();  // the record before the CTA's arrival
                if (ckpt && (t + 1) % a.ckpt_every == 0) {
                    TS *ck = ckpt + (int64_t)((t + 1) / a.ckpt_every) * 6 * a.n + 6 * (int64_t)io;
                    ck[0] = xs[0]; ck[1] = xs[1]; ck[2] = xs[2];
                    ck[3] = vs[0]; ck[4] = vs[1]; ck[5] = vs[2];
                }
            }
        }
        if (last_kick) break;
        if constexpr (GRID) {
            // every slice of dst written (global) before anyone reloads it
            ok = grid_barrier(a, (unsigned)t + 2u, &s_ok);
        } else {
            __syncthreads();  // this CTA's slice of dst is complete
            // The slice of S bodies is float4 [rank*S, rank*S + S) of the pair
            // layout (S even): copy it into the same place of every other CTA.
            const int base = (int)rank * S;
            for (int q = tid; q < (int)(csize - 1) * S; q += NT) {
                const uint32_t to = (rank + 1 + (uint32_t)(q / S)) % csize;
                const int k = base + q % S;
                st_cluster_f4(map_to_rank(smem_addr(&dst[k]), to), dst[k]);
            }
            cluster_barrier();
        }
        cur ^= 1;
    }
    if (owner) {
        TS *xw = reinterpret_cast<TS *>(a.x);
        TS *vw = reinterpret_cast<TS *>(a.v);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            xw[3 * io + c] = xs[c];
            vw[3 * io + c] = vs[c];
        }
    }
    if constexpr (GRID) {
        // Every CTA has passed its last barrier (or given up) before it counts
        // itself done, so once all have, nobody reads the arrivals again: the
        // last one zeroes both counters for the next launch (no memset launch
        // per call). A CTA that gave up at a barrier still gets here.
        __syncthreads();
        if (threadIdx.x == 0 && atomicAdd(a.bar + 1, 1u) == gridDim.x - 1) {
            atomicExch(a.bar, 0u);
            atomicExch(a.bar + 1, 0u);
        }
    }
}

constexpr int kClusterThreads = 512;

}  // namespace

using ClusterFn = void (*)(const ClusterArgs);

ClusterFn cluster_fn(bool f64, bool grid, int rb) {
    if (rb == 2) {
        if (grid)
            return f64 ? cluster_run_kernel<kClusterThreads, true, true, 2>
                       : cluster_run_kernel<kClusterThreads, false, true, 2>;
        return f64 ? cluster_run_kernel<kClusterThreads, true, false, 2>
                   : cluster_run_kernel<kClusterThreads, false, false, 2>;
    }
    if (grid)
        return f64 ? cluster_run_kernel<kClusterThreads, true, true, 1>
                   : cluster_run_kernel<kClusterThreads, false, true, 1>;
    return f64 ? cluster_run_kernel<kClusterThreads, true, false, 1>
               : cluster_run_kernel<kClusterThreads, false, false, 1>;
}

// Bodies per lane for a slice: two once a warp row of 64 slots is mostly filled.
int cluster_rb(int64_t slice) { return slice >= 64 ? 2 : 1; }

// Largest cluster this device can run the kernel with for n bodies (16 if
// non-portable clusters are allowed and fit, else 8), 0 if none: the two
// replicas must fit in shared memory.
int cluster_run_size(int64_t n, bool f64) {
    if (n <= 0 || n > kClusterMaxN) return 0;
    for (int c : {16, 8}) {
        const int64_t slice = ((n + c - 1) / c + 1) / 2 * 2;
        if (slice > kClusterThreads) continue;
        ClusterFn fn = cluster_fn(f64, false, cluster_rb(slice));
        const size_t smem = (size_t)2 * c * slice * 16;
        if (smem > 200 * 1024) continue;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            continue;
        if (c > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
            continue;
        cudaLaunchConfig_t cfg;
        memset(&cfg, 0, sizeof cfg);
        cfg.gridDim = dim3((unsigned)c);
        cfg.blockDim = dim3(kClusterThreads);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)c;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg) == cudaSuccess && clusters > 0) return c;
        cudaGetLastError();  // clear a refused query
    }
    cudaGetLastError();
    return 0;
}

cudaError_t launch_cluster_run(int cluster, int64_t n, bool f64, void *x, void *v, const void *m,
                               int steps, int kdk, float eps2, double G, double dt, void *ckpt,
                               int ckpt_every, cudaStream_t st) {
    if (cluster <= 0 || n <= 0 || n > kClusterMaxN) return cudaErrorInvalidValue;
    ClusterArgs a;
    a.n = (int)n;
    a.slice = (int)(((n + cluster - 1) / cluster + 1) / 2 * 2);
    ClusterFn fn = cluster_fn(f64, false, cluster_rb(a.slice));
    a.npad = cluster * a.slice;
    a.steps = steps;
    a.kdk = kdk;
    a.eps2 = eps2;
    a.G = G;
    a.dt = dt;
    a.x = x;
    a.v = v;
    a.m = m;
    a.ckpt = ckpt;
    a.ckpt_every = ckpt_every > 0 ? ckpt_every : 1;
    a.xm0 = a.xm1 = nullptr;
    a.bar = nullptr;
    a.err = nullptr;
    a.timeout_ns = 0;
    a.stall = 0;
    const size_t smem = (size_t)2 * a.npad * 16;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (cluster > 8) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = dim3((unsigned)cluster);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, a);
}

// Grid form: CTAs for n bodies with slices of at least min_slice bodies (even)
// and at most one CTA per SM, 0 if the path cannot run n bodies here.
int grid_run_ctas(int64_t n, int num_sms, int min_slice) {
    if (n <= 0 || n > kGridMaxN || num_sms <= 0) return 0;
    int64_t slice = std::max<int64_t>(min_slice, ((n + num_sms - 1) / num_sms + 1) / 2 * 2);
    slice = (slice + 1) / 2 * 2;
    if (slice > kClusterThreads) return 0;
    return (int)((n + slice - 1) / slice);
}

bool grid_run_ctas_valid(int64_t n, int num_sms, int ctas) {
    if (n <= 0 || n > kGridMaxN || ctas <= 0 || ctas > num_sms) return false;
    const int64_t slice = ((n + ctas - 1) / ctas + 1) / 2 * 2;
    return slice <= kClusterThreads;
}

cudaError_t launch_grid_run(int ctas, int64_t n, bool f64, void *x, void *v, const void *m, int steps,
                            int kdk, float eps2, double G, double dt, void *ckpt, int ckpt_every,
                            float4 *xm0, float4 *xm1, unsigned *bar, int *err, uint64_t timeout_ns,
                            int stall, cudaStream_t st) {
    if (ctas <= 0 || n <= 0 || n > kGridMaxN) return cudaErrorInvalidValue;
    ClusterArgs a;
    a.n = (int)n;
    a.slice = (int)(((n + ctas - 1) / ctas + 1) / 2 * 2);
    if (a.slice > kClusterThreads) return cudaErrorInvalidValue;
    ClusterFn fn = cluster_fn(f64, true, cluster_rb(a.slice));
    a.npad = ctas * a.slice;
    a.steps = steps;
    a.kdk = kdk;
    a.eps2 = eps2;
    a.G = G;
    a.dt = dt;
    a.x = x;
    a.v = v;
    a.m = m;
    a.ckpt = ckpt;
    a.ckpt_every = ckpt_every > 0 ? ckpt_every : 1;
    a.xm0 = xm0;
    a.xm1 = xm1;
    a.bar = bar;
    a.err = err;
    a.timeout_ns = timeout_ns;
    a.stall = stall;
    const size_t smem = (size_t)a.npad * 16;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = dim3((unsigned)ctas);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, a);
}

}  // namespace nb
