// nb_accel_noalloc: the FP32 force sum without any allocation.
//
// Some callers cannot allocate device memory at the moment they need
// forces: processes whose device memory is entirely owned by a pooling
// allocator (a raw cudaMalloc there fails or fragments the pool), and
// services that must fix their memory footprint when the library loads. For
// them this entry point needs no context and reserves its working memory
// once, as a file-scope device array that every GPU loading the library
// holds until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/nbody.h"
#include "kernels.h"

namespace nb {
const ForceEntry *force_table(int pol, int *count);
}

using namespace nb;

namespace {

// Limits of the static working memory.
constexpr int64_t kMaxN = NB_NOALLOC_MAX_N;       // bodies
constexpr int kNT = 128, kR = 2;                  // launch shape (threads, bodies/thread)
constexpr int kMaxSplit = 8;                      // j-splits
constexpr int64_t kMaxNpad = (kMaxN + kPadBodies - 1) / kPadBodies * kPadBodies;
constexpr int64_t kMaxIBlocks = (kMaxN + kNT * kR - 1) / (kNT * kR);
constexpr size_t kXmBytes = (size_t)kMaxNpad * 16;
constexpr size_t kPartBytes = (size_t)kMaxSplit * kMaxIBlocks * kNT * kR * 16;
constexpr size_t kCtrBytes = 1024;
constexpr size_t kOffPart = kXmBytes;
constexpr size_t kOffCtr = kOffPart + kPartBytes;
constexpr size_t kOffErr = kOffCtr + kCtrBytes;
constexpr size_t kScratchBytes = kOffErr + 256;
static_assert(kMaxIBlocks * 4 <= (int64_t)kCtrBytes, "ticket area too small");

// Packed bodies, split partials, split tickets and the error word.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Per-device set-up, done once by the first call on the device: the device
// address of g_scratch and the SM count. `done` is published with release
// order after both are written, so a thread that reads it true (acquire)
// sees them; the first calls of concurrent threads serialise on g_setup_mu.
struct DeviceSetup {
    std::atomic<bool> done{false};
    unsigned char *scratch = nullptr;
    int num_sms = 0;
};
constexpr int kMaxDevices = 64;
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mu;

bool setup_device(int dev, DeviceSetup &su) {
    if (su.done.load(std::memory_order_acquire)) return true;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (su.done.load(std::memory_order_relaxed)) return true;
    // host code cannot use g_scratch's name as an address: ask the runtime
    // where the array lives on this (current) device
    void *p = nullptr;
    int sms = 0;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    su.scratch = static_cast<unsigned char *>(p);
    su.num_sms = sms;
    su.done.store(true, std::memory_order_release);
    return true;
}

// A caller array: device (or managed) memory of device `dev`, 4-byte aligned.
bool valid_array(const void *p, int dev) {
    if (!p || reinterpret_cast<uintptr_t>(p) % 4) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

}  // namespace

extern "C" nb_status nb_accel_noalloc(int64_t n, const float *x, const float *m, float *a,
                                      double G, double eps, void *stream) {
    if (n < 0 || n > kMaxN) return NB_ERR_INVALID;
    if (!std::isfinite(G) || !std::isfinite(eps) || !(eps > 0.0) ||
        !((float)(eps * eps) >= 1.17549435e-38f))
        return NB_ERR_INVALID;
    if (n == 0) return NB_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return NB_ERR_CUDA;
    }
    // argument errors return before anything is launched
    if (!valid_array(x, dev) || !valid_array(m, dev) || !valid_array(a, dev)) return NB_ERR_INVALID;
    DeviceSetup &su = g_setup[dev];
    if (!setup_device(dev, su)) return NB_ERR_CUDA;
    int cnt = 0;
    const ForceEntry *tab = force_table(kPolF32x2, &cnt);
    const ForceEntry *e = nullptr;
    for (int k = 0; k < cnt; ++k)
        if (tab[k].nt == kNT && tab[k].r == kR) e = &tab[k];
    if (!e) return NB_ERR_UNSUPPORTED;

    const int64_t npad = (n + kPadBodies - 1) / kPadBodies * kPadBodies;
    const int jt = npad >= 4096 ? 128 : 64;
    const int ntiles = (int)(npad / jt);
    const int iblocks = (int)((n + kNT * kR - 1) / (kNT * kR));
    // split: enough CTAs for one full wave, within the static partial area
    const int64_t slots = (int64_t)std::max(e->occupancy(jt), 1) * su.num_sms;
    int split = (int)std::min<int64_t>(std::max<int64_t>(1, slots / iblocks), kMaxSplit);
    split = std::min(split, ntiles);

    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    float4 *xm = reinterpret_cast<float4 *>(su.scratch);
    unsigned *ctr = reinterpret_cast<unsigned *>(su.scratch + kOffCtr);
    int *err = reinterpret_cast<int *>(su.scratch + kOffErr);
    // the tickets and the error word must start at zero on every call
    if (cudaMemsetAsync(su.scratch + kOffCtr, 0, kCtrBytes + 256, st) != cudaSuccess) {
        cudaGetLastError();
        return NB_ERR_CUDA;
    }
    if (launch_pack_f32(n, npad, x, nullptr, m, xm, nullptr, PadTargets(), st) != cudaSuccess) {
        cudaGetLastError();
        return NB_ERR_CUDA;
    }
    ForceArgs args;
    memset(&args, 0, sizeof args);
    args.src = xm;
    args.n = n;
    args.npad = npad;
    args.jt = jt;
    args.ntiles = ntiles;
    args.split = split;
    args.iblocks = iblocks;
    args.eps2 = (float)(eps * eps);
    args.G = G;
    args.part = reinterpret_cast<float4 *>(su.scratch + kOffPart);
    args.counters = ctr;
    args.err = err;
    args.timeout_ns = 2000000000ull;
    args.op = kEpiAccel;
    args.out = a;
    if (e->launch(jt, args, st) != cudaSuccess) {
        cudaGetLastError();
        return NB_ERR_CUDA;
    }
    return NB_OK;
}
