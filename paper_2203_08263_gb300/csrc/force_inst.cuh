// Instantiation helpers: one translation unit per policy keeps the build
// parallel. Each entry pairs a launcher with an occupancy query.
#pragma once
#include <cstring>

#include "kernels.h"

namespace nb {

template <class P, int NT, int R>
cudaError_t launch_force_inst(int jt, const ForceArgs &a, cudaStream_t st) {
    const size_t smem = force_smem_bytes(P::REC_F4, jt);
    auto k = force_kernel<NT, R, P>;
    if (smem > 48 * 1024) {
        cudaError_t e =
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (!a.pdl) {
        k<<<(unsigned)((int64_t)a.iblocks * a.split), NT + kProducerThreads, smem, st>>>(a);
        return cudaGetLastError();
    }
    // programmatic dependent launch: the grid may be scheduled before the
    // previous kernel on the stream completes; the kernel waits for it
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = dim3((unsigned)((int64_t)a.iblocks * a.split));
    cfg.blockDim = dim3(NT + kProducerThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, a);
}

template <class P, int NT, int R>
int occ_force_inst(int jt) {
    int b = 0;
    const size_t smem = force_smem_bytes(P::REC_F4, jt);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, force_kernel<NT, R, P>, NT + kProducerThreads, smem) !=
        cudaSuccess)
        return 0;
    return b;
}

#define NB_ENTRY(P, NT, R) {NT, R, &launch_force_inst<P, NT, R>, &occ_force_inst<P, NT, R>}

}  // namespace nb
