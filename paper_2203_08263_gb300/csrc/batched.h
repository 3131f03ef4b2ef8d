// Ensemble of independent systems in one persistent cooperative launch.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

namespace nb {

// Host-side schedule: CTAs form gangs; each gang advances its list of systems
// one after the other, every gang member holding a slice of the system's
// i-bodies and all of its j-bodies. Gang sizes and the system-to-gang
// assignment come from a longest-processing-time-first packing.
struct BatchPlan {
    int nsys = 0;
    int nt = 128, r = 2, jt = 64;   // kernel shape
    int gmax = 16;                  // largest gang (CTAs sharing one system)
    int ncta = 0, ngang = 0;
    int64_t total = 0, total_pad = 0;
    std::vector<int64_t> off, poff;
    std::vector<int> work, gang_first, cta_gang, cta_rank, gang_size;
    size_t plan_bytes = 0;     // device bytes for the arrays above
    size_t scratch_bytes = 0;  // plan + counters + two packed buffers
    uint64_t signature = 0;    // hash of sizes and shape
    int64_t launches = 3;      // memset, pack, persistent kernel
    double makespan_tiles = 0;
};

int64_t batched_max_n();

// Build the schedule for the given offsets on this device. Shape fields of
// `plan` (nt, r, jt) may be preset; 0 picks the default.
bool batched_plan(int device, int num_sms, const std::vector<int64_t> &off, BatchPlan &plan,
                  std::string &why);

// Upload the plan into `scratch` (on `st`) and enqueue: zero the gang
// counters, pack all systems, launch the persistent kernel.
cudaError_t batched_upload(const BatchPlan &plan, void *scratch, cudaStream_t st);
// Deterministic synthetic state for tuning runs (positions in [-1,1]^3,
// small velocities, masses 1/N_s): timing does not depend on the values.
cudaError_t batched_fill_synthetic(const BatchPlan &plan, void *scratch, float *x, float *v,
                                   float *m, cudaStream_t st);
cudaError_t batched_enqueue(const BatchPlan &plan, void *scratch, float *x, float *v,
                            const float *m, int steps, float eps2, float G, float dt, int *err,
                            uint64_t timeout_ns, cudaStream_t st);

}  // namespace nb
