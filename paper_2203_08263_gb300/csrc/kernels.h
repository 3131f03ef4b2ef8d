// Internal launcher interface between the C-ABI layer (api.cu) and the
// kernel translation units. Host code only sees these declarations.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "engine.cuh"

namespace nb {

// Pair-sum policies compiled into the library.
enum Pol : int {
    kPolF32x2 = 0,   // plain FP32 forces, packed f32x2 arithmetic
    kPolScalar = 1,  // plain FP32 forces, scalar arithmetic
    kPolComp = 2,    // compensated FP32 forces, FP64 state
    kPolPot = 3,     // softened potential (diagnostics)
    kPolVjp = 4,     // adjoint VJP, FP32 state
    kPolVjpComp = 5, // adjoint VJP, compensated, FP64 state
    kPolDiv = 6,     // ablation: sqrt + division
    kPolPow = 7,     // ablation: powf
    kPolSym = 8,     // plain FP32 forces, each unordered pair once (csrc/k_sym.cu)
    kPolVjpSym = 9,  // adjoint VJP, FP32 state, each unordered pair once (csrc/k_sym.cu)
    kPolSymComp = 10,  // compensated forces, FP64 state, each unordered pair once (csrc/k_sym.cu)
    kPolVjpSymComp = 11,  // adjoint VJP, compensated, FP64 state, each unordered pair once (csrc/k_sym.cu)
    kPolCount = 12
};

// Bodies per lane of the pair-symmetric force policy; its table holds blocks
// of 32 x R x (1, 2 or 4 warps) = 256, 512 or 1024 bodies (Shape: nt = 32,
// 64 or 128, r = R, jt = the block, split = 1). The VJP's (FP32 and the
// precision form) hold R = 4, blocks of 256 or 512 bodies.
#ifndef NB_SYM_R
#define NB_SYM_R 8  // measured at N = 262144: 3.70e12 interactions/s at R = 6 (96 registers, 5 CTAs per SM), 3.98e12 at 8, 3.99e12 at 10
#endif
constexpr int kSymR = NB_SYM_R;
#ifndef NB_SYM_VJP_R
#define NB_SYM_VJP_R 4
#endif
constexpr int kSymVjpR = NB_SYM_VJP_R;
inline bool pol_is_sym(int pol) {
    return pol == kPolSym || pol == kPolVjpSym || pol == kPolSymComp || pol == kPolVjpSymComp;
}
// sums per body of a pair-symmetric policy (its partials: nb x sums x npad floats)
inline int sym_sums(int pol) { return pol == kPolVjpSym || pol == kPolVjpSymComp ? 8 : 3; }
// Above this many bytes of partials the ensemble's pair-symmetric form
// falls back to the one-sided items.
constexpr size_t kSymMaxPartBytes = (size_t)16 << 30;

// Pair t of the upper triangle of an n x n grid, row-major: rows r = 0..n-1
// holding columns c = r..n-1.
__host__ __device__ inline void tri_item(int64_t t, int n, int &r, int &c) {
    const double k = 2.0 * n + 1.0;
    int64_t q = (int64_t)((k - sqrt(k * k - 8.0 * (double)t)) * 0.5);
    if (q < 0) q = 0;
    if (q > n - 1) q = n - 1;
    auto start = [n](int64_t row) { return row * n - row * (row - 1) / 2; };
    while (q > 0 && start(q) > t) --q;
    while (q < n - 1 && start(q + 1) <= t) ++q;
    r = (int)q;
    c = (int)(q + (t - start(q)));
}

// Tiles of the pair-symmetric kernels' triangle of block pairs: the nb blocks
// are cut into strips of w; tile (I, J), I <= J, holds the block pairs
// (bi, bj), bi <= bj, with bi in strip I and bj in strip J. Tiles are numbered
// row-major over the triangle of strips: every body then meets its partner
// blocks p in ascending order across tiles (p < its block through the tiles
// of its column strip, top down, the rest through the tiles of its row
// strip, left to right), so a running sum over tiles adds the partials in
// the same order as one sum over all of them.
struct SymTile {
    int I, J;    // strips
    int r0, c0;  // first block of strip I, of strip J
    int hr, hc;  // blocks in strip I, in strip J
    __host__ __device__ int items() const { return I == J ? hr * (hr + 1) / 2 : hr * hc; }
};
__host__ __device__ inline int sym_tile_count(int nb, int w) {
    const int m = (nb + w - 1) / w;
    return m * (m + 1) / 2;
}
__host__ __device__ inline SymTile sym_tile(int t, int nb, int w) {
    SymTile g;
    tri_item(t, (nb + w - 1) / w, g.I, g.J);
    g.r0 = g.I * w;
    g.c0 = g.J * w;
    g.hr = nb - g.r0 < w ? nb - g.r0 : w;
    g.hc = nb - g.c0 < w ? nb - g.c0 : w;
    return g;
}
// Tiles of the pair-symmetric forms are used above this many bytes of
// partials for one launch over all block pairs; two tile buffers take at
// most kSymTileBufBytes. With the one-launch and the tile kernels running
// the same compiled pair loop, tiles cost nothing measurable: at N = 262144
// (805 MB of partials in one launch) 3.987e12 interactions/s in one launch
// against 3.984e12-3.991e12 by tiles of 16 to 49 blocks (3 steps per call),
// and 17.234 ms per bench step in one launch against 17.229 by tiles of 49;
// at N = 524288 4.009e12 against 4.017e12; at N = 131072 (201 MB, below the
// threshold) 3.916e12 against 3.908e12. The buffers' bound sets the tile
// side, and small tiles keep both buffers in L2: DRAM bytes written per
// N = 262144 step are 8 / 20 / 84 / 380 / 687 MB with tiles of 20 / 24 / 28 /
// 36 / 49 blocks (buffers of 19 / 28 / 38 / 62 / 118 MB), 774 MB in one
// launch, whose epilogue also reads 749 MB back. 28 MiB gives tiles of 24
// blocks for the forces (1024-body blocks) and of 21 for the VJP (512).
#ifndef NB_SYM_TILE_ABOVE_MIB
#define NB_SYM_TILE_ABOVE_MIB 512
#endif
#ifndef NB_SYM_TILE_BUF_MIB
#define NB_SYM_TILE_BUF_MIB 28
#endif
constexpr size_t kSymTileAbove = (size_t)NB_SYM_TILE_ABOVE_MIB << 20;
constexpr size_t kSymTileBufBytes = (size_t)NB_SYM_TILE_BUF_MIB << 20;

struct Shape {
    int pol, nt, r, split, jt;
};

struct ForceEntry {
    int nt, r;
    cudaError_t (*launch)(int jt, const ForceArgs &a, cudaStream_t st);
    int (*occupancy)(int jt);  // resident CTAs per SM
};

// Table of compiled (NT, R) instances of a policy.
const ForceEntry *force_table(int pol, int *count);
int pol_rec_f4(int pol);   // float4 per j-pair record
int pol_part_f4(int pol);  // float4 per i-body split partial

inline size_t force_smem_bytes(int rec_f4, int jt) {
    return 128 + (size_t)kStages * (size_t)(jt / 2) * rec_f4 * 16;
}

// ---- O(n) helpers (kern_misc.cu)
// Further packed buffers (count of them, `stride` float4 apart from `base`)
// whose padding records [n, npad) the pack also zeroes.
struct PadTargets {
    float4 *base = nullptr;
    int count = 0;
    int64_t stride = 0;
};
cudaError_t launch_pack_f32(int64_t n, int64_t npad, const float *x, const float *v,
                            const float *m, float4 *xm, float *ckpt0, PadTargets pads,
                            cudaStream_t st);
cudaError_t launch_pack_f64(int64_t n, int64_t npad, const double *x, const double *v,
                            const double *m, float4 *xm, double *ckpt0, PadTargets pads,
                            cudaStream_t st);
// synthetic bodies for tuning runs
cudaError_t launch_fill_synthetic(int64_t n, int64_t npad, float4 *xm, int rec_f4,
                                  cudaStream_t st);
// KE, P from (v, m) and sum of per-body potential terms; out[0..4] =
// {Px, Py, Pz, KE, sum_i vals[i]}. `scratch` holds blocks * 5 doubles.
cudaError_t launch_energy_reduce(int64_t n, const void *v, const void *m, int f64,
                                 const double *vals, double *scratch, int blocks, double *out,
                                 cudaStream_t st);
// adjoint: vbar' = vbar + dt xbar; abar = dt/2 vbar'; pack (x_t, m, abar) VJP
// records; restore/capture state helpers
// FP32: positions from the packed xm_t. FP64 (precision form): positions
// from x64 (row stride x_stride doubles), split into hi/lo records.
cudaError_t launch_adj_prepare(int64_t n, int64_t npad, int f64, const float4 *xm_t,
                               const double *x64, int x_stride, const void *m, void *vbar,
                               const void *xbar, double dt, float4 *rec, double *abar64,
                               cudaStream_t st);
cudaError_t launch_copy_ckpt_state(int64_t n, int f64, const void *ckpt_slot, void *x, void *v,
                                   cudaStream_t st);

// FP32 FFMA / f32x2 FMA TFLOP/s and MUFU rsqrt Gop/s micro-benchmarks
cudaError_t measure_peaks(int blocks, float *sink, cudaStream_t st, double out[3]);

// Small systems in one cluster launch (csrc/cluster.cu): every step of a run
// in one kernel, positions replicated in the shared memory of each CTA of one
// thread-block cluster and exchanged through distributed shared memory; FP32
// or the precision form.
constexpr int64_t kClusterMaxN = 4096;      // two replicas of 64 KiB
// Untuned choice of nb_run's path (one cluster up to kClusterDefault*, the
// grid form up to kGridDefault*, the graph of force launches above).
// Measured on GB300 at 100 steps, us per step graph / one cluster / grid:
//   FP32            N = 256: 4.6 / 1.9 / 2.9     1024: 5.6 / 6.1 / 4.4
//                   N = 4096: 12.8 / 74 / 10.8    8192: 33.8 / - / 33.5
//   precision form  N = 256: 8.6 / 3.1 / 4.2     1024: 10.8 / 7.3 / 5.8
//                   N = 4096: 24.2 / 80 / 12.7    8192: 44.4 / - / 37.1
// (one cluster has 16 SMs; the grid form all 152 but pays a grid barrier and
// an L2 reload per step; the graph path pays a kernel boundary and, in the
// precision form, an FP64 update spread over few CTAs.)
constexpr int64_t kClusterDefaultN = 512;
constexpr int64_t kClusterDefaultN64 = 512;
// Cluster size (16, or 8 where 16 cannot be scheduled) for n bodies; 0 if
// the path cannot run n bodies on this device.
// f64: the precision form (FP64 state, compensated FP32 forces).
int cluster_run_size(int64_t n, bool f64);
cudaError_t launch_cluster_run(int cluster, int64_t n, bool f64, void *x, void *v, const void *m,
                               int steps, int kdk, float eps2, double G, double dt, void *ckpt,
                               int ckpt_every, cudaStream_t st);
// The same step loop on a cooperative grid of up to one CTA per SM: slices
// written to a global double buffer (xm0, xm1: [npad] records each, npad =
// ctas x slice), a bounded grid barrier per step (bar: two counters, zero
// before the first launch; each launch leaves them zero), all records
// reloaded into shared memory.
constexpr int64_t kGridMaxN = 8192;  // one replica of 128 KiB
constexpr int64_t kGridDefaultN = 4096;
constexpr int64_t kGridDefaultN64 = 8192;
// CTAs for n bodies with slices of at least min_slice bodies (16 untuned;
// the tuner also tries 8, 32 and 64), 0 if the path cannot run n bodies here;
// and whether a tuned CTA count is runnable on this device.
int grid_run_ctas(int64_t n, int num_sms, int min_slice = 16);
bool grid_run_ctas_valid(int64_t n, int num_sms, int ctas);
cudaError_t launch_grid_run(int ctas, int64_t n, bool f64, void *x, void *v, const void *m, int steps,
                            int kdk, float eps2, double G, double dt, void *ckpt, int ckpt_every,
                            float4 *xm0, float4 *xm1, unsigned *bar, int *err, uint64_t timeout_ns,
                            int stall, cudaStream_t st);

}  // namespace nb
