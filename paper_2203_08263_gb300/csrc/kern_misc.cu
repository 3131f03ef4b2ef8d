// O(n) kernels around the pair sums: packing, diagnostics reductions and the
// adjoint's per-step preparation.
#include "kernels.h"

namespace nb {

namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    return (unsigned)(b > 0 ? b : 1);
}

template <class TS>
__global__ void pack_kernel(int64_t n, int64_t npad, const TS *__restrict__ x,
                            const TS *__restrict__ v, const TS *__restrict__ m, float4 *xm,
                            TS *ckpt0, PadTargets pads) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npad) return;
    // the step epilogues repack only real bodies, so the buffers they write
    // get their zero-mass padding here (a buffer reused from a larger system
    // would otherwise keep that system's bodies in its padding)
    if (i >= n)
        for (int s = 0; s < pads.count; ++s) pair_put(pads.base + s * pads.stride, i, 0.f, 0.f, 0.f, 0.f);
    if (i < n) {
        const TS x0 = x[3 * i], x1 = x[3 * i + 1], x2 = x[3 * i + 2];
        pair_put(xm, i, (float)x0, (float)x1, (float)x2, (float)m[i]);
        if (ckpt0) {
            TS *c = ckpt0 + 6 * i;
            c[0] = x0; c[1] = x1; c[2] = x2;
            c[3] = v[3 * i]; c[4] = v[3 * i + 1]; c[5] = v[3 * i + 2];
        }
    } else {
        pair_put(xm, i, 0.f, 0.f, 0.f, 0.f);
    }
}

__device__ __forceinline__ uint32_t mix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x7feb352dU;
    h ^= h >> 15;
    h *= 0x846ca68bU;
    h ^= h >> 16;
    return h;
}

// Arbitrary in-range bodies for tuning runs: values only steer timing.
__global__ void fill_synthetic_kernel(int64_t n, int64_t npad, float *rec, int floats_per_pair) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npad) return;
    float *p = rec + (i >> 1) * floats_per_pair;
    const int h = (int)(i & 1);
    for (int k = 0; k < floats_per_pair / 2; ++k) {
        uint32_t u = mix32((uint32_t)i * 2654435761u + (uint32_t)k * 40503u + 12345u);
        p[2 * k + h] = (float)u * (2.0f / 4294967296.0f) - 1.0f;
    }
    p[6 + h] = i < n ? 1.0f / (float)n : 0.0f;
}

template <class TS>
__global__ void energy_partial_kernel(int64_t n, const TS *__restrict__ v,
                                      const TS *__restrict__ m, const double *__restrict__ vals,
                                      double *scratch) {
    __shared__ double sh[5][kThreads];
    double acc[5] = {0, 0, 0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double mi = (double)m[i];
        const double v0 = (double)v[3 * i], v1 = (double)v[3 * i + 1], v2 = (double)v[3 * i + 2];
        acc[0] += mi * v0;
        acc[1] += mi * v1;
        acc[2] += mi * v2;
        acc[3] += 0.5 * mi * (v0 * v0 + v1 * v1 + v2 * v2);
        acc[4] += vals[i];
    }
    for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < 5; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 5) scratch[blockIdx.x * 5 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void energy_final_kernel(int blocks, const double *scratch, double *out) {
    if (threadIdx.x < 5) {
        double s = 0.0;
        for (int b = 0; b < blocks; ++b) s += scratch[b * 5 + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// FP32 adjoint records from the packed positions x_t (4 float4 per pair).
__global__ void adj_prepare_f32_kernel(int64_t n, int64_t npad, const float4 *__restrict__ xm_t,
                                       const float *__restrict__ m, float *vbar,
                                       const float *__restrict__ xbar, float dt, float4 *rec) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npad) return;
    float *p = reinterpret_cast<float *>(rec + (i >> 1) * 4);
    const int h = (int)(i & 1);
    if (i < n) {
        float a[3];
        for (int c = 0; c < 3; ++c) {
            const float vb = vbar[3 * i + c] + dt * xbar[3 * i + c];  // vbar' = vbar + dt xbar
            vbar[3 * i + c] = vb;
            a[c] = dt / 2.0f * vb;                                     // abar = dt/2 vbar'
        }
        p[0 + h] = pair_get(xm_t, i, 0);
        p[2 + h] = pair_get(xm_t, i, 1);
        p[4 + h] = pair_get(xm_t, i, 2);
        p[6 + h] = m[i];
        p[8 + h] = a[0];
        p[10 + h] = a[1];
        p[12 + h] = a[2];
        p[14 + h] = 0.f;
    } else {
        for (int k = 0; k < 8; ++k) p[2 * k + h] = 0.f;
    }
}

// Precision-form adjoint records (5 float4 per pair): FP64 positions split
// into FP32 hi + lo, FP32 abar, and the FP64 abar kept for the epilogue.
__global__ void adj_prepare_f64_kernel(int64_t n, int64_t npad, const double *__restrict__ x64,
                                       int x_stride, const double *__restrict__ m, double *vbar,
                                       const double *__restrict__ xbar, double dt, float4 *rec,
                                       double *abar64) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npad) return;
    float *p = reinterpret_cast<float *>(rec + (i >> 1) * 5);
    const int h = (int)(i & 1);
    if (i < n) {
        double a[3];
        for (int c = 0; c < 3; ++c) {
            const double vb = vbar[3 * i + c] + dt * xbar[3 * i + c];
            vbar[3 * i + c] = vb;
            a[c] = dt / 2.0 * vb;
            abar64[3 * i + c] = a[c];
        }
        float hi[3], lo[3];
        for (int c = 0; c < 3; ++c) {
            const double xc = x64[(int64_t)x_stride * i + c];
            hi[c] = (float)xc;
            lo[c] = (float)(xc - (double)hi[c]);
        }
        p[0 + h] = hi[0];
        p[2 + h] = hi[1];
        p[4 + h] = hi[2];
        p[6 + h] = (float)m[i];
        p[8 + h] = (float)a[0];
        p[10 + h] = (float)a[1];
        p[12 + h] = (float)a[2];
        p[14 + h] = lo[0];
        p[16 + h] = lo[1];
        p[18 + h] = lo[2];
    } else {
        for (int k = 0; k < 10; ++k) p[2 * k + h] = 0.f;
    }
}

template <class TS>
__global__ void copy_ckpt_kernel(int64_t n, const TS *__restrict__ slot, TS *x, TS *v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int c = 0; c < 3; ++c) {
        x[3 * i + c] = slot[6 * i + c];
        v[3 * i + c] = slot[6 * i + 3 + c];
    }
}

}  // namespace

cudaError_t launch_pack_f32(int64_t n, int64_t npad, const float *x, const float *v,
                            const float *m, float4 *xm, float *ckpt0, PadTargets pads,
                            cudaStream_t st) {
    pack_kernel<float><<<blocks_for(npad), kThreads, 0, st>>>(n, npad, x, v, m, xm, ckpt0, pads);
    return cudaGetLastError();
}

cudaError_t launch_pack_f64(int64_t n, int64_t npad, const double *x, const double *v,
                            const double *m, float4 *xm, double *ckpt0, PadTargets pads,
                            cudaStream_t st) {
    pack_kernel<double><<<blocks_for(npad), kThreads, 0, st>>>(n, npad, x, v, m, xm, ckpt0, pads);
    return cudaGetLastError();
}

cudaError_t launch_fill_synthetic(int64_t n, int64_t npad, float4 *xm, int rec_f4,
                                  cudaStream_t st) {
    fill_synthetic_kernel<<<blocks_for(npad), kThreads, 0, st>>>(
        n, npad, reinterpret_cast<float *>(xm), rec_f4 * 4);
    return cudaGetLastError();
}

cudaError_t launch_energy_reduce(int64_t n, const void *v, const void *m, int f64,
                                 const double *vals, double *scratch, int blocks, double *out,
                                 cudaStream_t st) {
    if (f64)
        energy_partial_kernel<double><<<blocks, kThreads, 0, st>>>(
            n, (const double *)v, (const double *)m, vals, scratch);
    else
        energy_partial_kernel<float><<<blocks, kThreads, 0, st>>>(
            n, (const float *)v, (const float *)m, vals, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    energy_final_kernel<<<1, 32, 0, st>>>(blocks, scratch, out);
    return cudaGetLastError();
}

cudaError_t launch_adj_prepare(int64_t n, int64_t npad, int f64, const float4 *xm_t,
                               const double *x64, int x_stride, const void *m, void *vbar,
                               const void *xbar, double dt, float4 *rec, double *abar64,
                               cudaStream_t st) {
    if (f64)
        adj_prepare_f64_kernel<<<blocks_for(npad), kThreads, 0, st>>>(
            n, npad, x64, x_stride, (const double *)m, (double *)vbar, (const double *)xbar, dt,
            rec, abar64);
    else
        adj_prepare_f32_kernel<<<blocks_for(npad), kThreads, 0, st>>>(
            n, npad, xm_t, (const float *)m, (float *)vbar, (const float *)xbar, (float)dt, rec);
    return cudaGetLastError();
}

cudaError_t launch_copy_ckpt_state(int64_t n, int f64, const void *slot, void *x, void *v,
                                   cudaStream_t st) {
    if (f64)
        copy_ckpt_kernel<double><<<blocks_for(n), kThreads, 0, st>>>(
            n, (const double *)slot, (double *)x, (double *)v);
    else
        copy_ckpt_kernel<float><<<blocks_for(n), kThreads, 0, st>>>(
            n, (const float *)slot, (float *)x, (float *)v);
    return cudaGetLastError();
}

}  // namespace nb
