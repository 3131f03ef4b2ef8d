// Pair-symmetric FP32 force sum: every unordered pair {i, j} is evaluated once
// and feeds both bodies (Newton's third law: the pair term of j on i is
// m_j s^-3/2 d and that of i on j is -m_i s^-3/2 d, d = x_j - x_i), so the
// force sum of Section 2.3 (counted at 20 flops per ordered interaction in
// Section 4.1) costs 16 FP32 lane operations per unordered pair, 8 per
// ordered interaction, against 12 in the one-sided policies.
//
// Work decomposition. Bodies are padded with zero-mass bodies to nb blocks of
// B = 32 x W x R. An item is a block pair (bi, bj), bi <= bj, one CTA each.
// Each warp of the CTA owns 32 x R bodies of block bi, R per lane, held
// duplicated in f32x2 registers as in the one-sided policy; block bj is
// walked in chunks of 32 records (64 bodies), one record per lane, and for
// 32 rounds every lane evaluates its R i-bodies against the two bodies of its
// current record, then passes the record and the record's running j-side sums
// to the next lane (shuffles). After 32 rounds each record is back home with
// its sums over the warp's i-bodies, which land in the warp's slice of shared
// memory; at the end the CTA adds the W slices in warp order. The diagonal
// item (bi == bj) evaluates every ordered pair of its block from the i side
// only (a body with itself contributes exactly 0: d = 0).
//
// Determinism. The partial sums land in P[p][c][b] (p = the partner block:
// bj for the i side of item (bi, bj), bi for its j side), which every body
// fills exactly once for each p; a second kernel adds P[0..nb-1][c][b] in
// that order and runs the shared epilogue (write a, or kick + drift + repack),
// so the result does not depend on scheduling.
#include <cstring>

#include "kernels.h"

namespace nb {
namespace {

__device__ __forceinline__ float2 shfl2(float2 v, int src) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// Item t of the upper triangle, rows bi = 0..nb-1 holding bj = bi..nb-1.
__device__ __forceinline__ void sym_item(int t, int nb, int &bi, int &bj) {
    const double c = 2.0 * nb + 1.0;
    int r = (int)((c - sqrt(c * c - 8.0 * t)) * 0.5);
    auto start = [nb](int row) { return row * nb - row * (row - 1) / 2; };
    if (r < 0) r = 0;
    if (r > nb - 1) r = nb - 1;
    while (r > 0 && start(r) > t) --r;
    while (r < nb - 1 && start(r + 1) <= t) ++r;
    bi = r;
    bj = r + (t - start(r));
}

template <int W>
__global__ void __launch_bounds__(W * 32) sym_force_kernel(const ForceArgs a) {
    constexpr int R = kSymR, B = W * 32 * R;
    extern __shared__ float acc_j[];  // [W][3][B]
    // the previous kernel on the stream (last step's epilogue reads P and
    // writes the records read here) must be complete
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int nb = (int)(a.npad / B);
    int bi, bj;
    sym_item(blockIdx.x, nb, bi, bj);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int next = (l + 1) & 31;
    const float2 eps2 = dup(a.eps2);
    float2 nx[R], ny[R], nz[R], mi[R], ax[R], ay[R], az[R];
    const int64_t gbase = (int64_t)bi * B + w * 32 * R;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t i = gbase + l + 32 * r;
        nx[r] = dup(-pair_get(a.src, i, 0));
        ny[r] = dup(-pair_get(a.src, i, 1));
        nz[r] = dup(-pair_get(a.src, i, 2));
        mi[r] = dup(pair_get(a.src, i, 3));
        ax[r] = ay[r] = az[r] = f2(0.f, 0.f);
    }
    const bool diag = bi == bj;
    float *mine = acc_j + w * 3 * B;
    for (int c = 0; c < B / 64; ++c) {
        const int64_t q = (int64_t)bj * (B / 2) + c * 32 + l;  // this lane's record
        const float4 r0 = __ldg(a.src + 2 * q), r1 = __ldg(a.src + 2 * q + 1);
        float2 xj = f2(r0.x, r0.y), yj = f2(r0.z, r0.w), zj = f2(r1.x, r1.y), mj = f2(r1.z, r1.w);
        float2 bx = f2(0.f, 0.f), by = bx, bz = bx;
#pragma unroll 1
        for (int round = 0; round < 32; ++round) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
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
                const float2 wj = __fmul2_rn(mi[r], y3);  // i on j: -m_i s^-3/2 d
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
        if (!diag) {
            const int k = c * 64 + 2 * l;
            mine[k] = -bx.x;
            mine[k + 1] = -bx.y;
            mine[B + k] = -by.x;
            mine[B + k + 1] = -by.y;
            mine[2 * B + k] = -bz.x;
            mine[2 * B + k + 1] = -bz.y;
        }
    }
    float *P = reinterpret_cast<float *>(a.part);
    const int64_t np = a.npad;
    {
        float *p = P + (int64_t)bj * 3 * np;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int64_t i = gbase + l + 32 * r;
            __stcg(p + i, ax[r].x + ax[r].y);
            __stcg(p + np + i, ay[r].x + ay[r].y);
            __stcg(p + 2 * np + i, az[r].x + az[r].y);
        }
    }
    if (!diag) {
        __syncthreads();
        float *p = P + (int64_t)bi * 3 * np + (int64_t)bj * B;
        for (int t = threadIdx.x; t < B; t += W * 32) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float s = 0.f;
#pragma unroll
                for (int k = 0; k < W; ++k) s += acc_j[k * 3 * B + c * B + t];
                __stcg(p + c * np + t, s);
            }
        }
    }
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Fixed-order sum of the nb partials of each body, then the shared epilogue.
__global__ void __launch_bounds__(256) sym_finish_kernel(const ForceArgs a) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.n) {
        const float *P = reinterpret_cast<const float *>(a.part);
        const int64_t np = a.npad;
        float fx = 0.f, fy = 0.f, fz = 0.f;
        for (int p = 0; p < a.ntiles; ++p) {
            const float *q = P + (int64_t)p * 3 * np + i;
            fx += __ldcs(q);
            fy += __ldcs(q + np);
            fz += __ldcs(q + 2 * np);
        }
        const float G = (float)a.G;
        finish_fp32(a, i, G * fx, G * fy, G * fz);
    }
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

cudaError_t launch_ex(const void *fn, dim3 grid, dim3 block, size_t smem, bool pdl,
                      const ForceArgs &a, cudaStream_t st) {
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    void *args[] = {const_cast<ForceArgs *>(&a)};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

template <int W>
cudaError_t launch_sym(int, const ForceArgs &a, cudaStream_t st) {
    constexpr int B = W * 32 * kSymR;
    const size_t smem = (size_t)W * 3 * B * 4;
    auto k = sym_force_kernel<W>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int64_t nb = a.npad / B;
    if (nb * B != a.npad || nb != a.ntiles) return cudaErrorInvalidValue;
    const unsigned items = (unsigned)(nb * (nb + 1) / 2);
    cudaError_t e = launch_ex((const void *)k, dim3(items), dim3(W * 32), smem, a.pdl != 0, a, st);
    if (e != cudaSuccess) return e;
    // the epilogue is a programmatic dependent of the pair kernel: its launch
    // overlaps the pair kernel's last wave, and it waits for its completion
    return launch_ex((const void *)sym_finish_kernel, dim3((unsigned)((a.n + 255) / 256)),
                     dim3(256), 0, true, a, st);
}

template <int W>
int occ_sym(int) {
    constexpr int B = W * 32 * kSymR;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, sym_force_kernel<W>, W * 32,
                                                      (size_t)W * 3 * B * 4) != cudaSuccess)
        return 0;
    return b;
}

const ForceEntry kTable[] = {
    {64, kSymR, &launch_sym<2>, &occ_sym<2>},   // blocks of 512 bodies
    {128, kSymR, &launch_sym<4>, &occ_sym<4>},  // blocks of 1024 bodies
};

}  // namespace

const ForceEntry *table_sym(int *count) {
    *count = (int)(sizeof(kTable) / sizeof(kTable[0]));
    return kTable;
}

}  // namespace nb
