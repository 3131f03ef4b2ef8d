// Ensemble of independent systems in one persistent cooperative launch.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

namespace nb {

// Host-side plan of the persistent ensemble kernel. The work of one step is
// split into items (system s, first i-body lo, R) of NT x R i-bodies each,
// against all of the system's j-bodies: full items use R = r (the plan's
// largest), the ragged rest of a system smaller powers of two. Items are
// numbered step-major (all items of step t before those of step t+1) and,
// within a step, by decreasing work. Persistent CTAs pop item numbers from
// one atomic counter; an item of step t waits only until every item of step
// t-1 of the same system is done (always lower numbers, so the oldest
// unfinished item can always run).
struct BatchPlan {
    int nsys = 0;
    int nt = 0, r = 0, jt = 0;      // kernel shape: threads, largest R, j-tile (0: the default)
    int ncta = 0;                   // persistent grid (resident CTAs)
    int items_per_step = 0;
    int origin = 0;                 // 0 default shape, 1 autotuned, 2 set by the caller
    int f64 = 0;                    // the precision form (FP64 state): shapes up to R = 4
    int64_t total = 0, total_pad = 0;
    std::vector<int64_t> off, poff;  // body offsets, packed offsets (per system)
    std::vector<int> item_sys, item_lo, item_r;  // per item of one step
    std::vector<int> nitems;                     // items per step of each system
    size_t scratch_bytes = 0;   // plan + counters + two packed buffers
    uint64_t signature = 0;     // hash of sizes and shape
    int64_t launches = 3;       // memset, pack, persistent kernel
    // The pair-symmetric form (csrc/batched_sym.cu): groups of 256 bodies,
    // block-pair items and one epilogue item per group (nt = 128, r = 8,
    // jt = the group; the plan fields above keep their meaning).
    int sym = 0;
    std::vector<int64_t> sym_pofs;         // per system: offset of its partials (floats)
    std::vector<int> sym_ng, sym_npairs;   // per system: groups, pair items per step
    std::vector<int> sym_items;            // per item of one step: {system, gi, gj, kind}
    int64_t sym_part_floats = 0;
};

int64_t batched_max_n();

// FP32 lane operations of the pair-symmetric form over those of the one-sided
// form for these system sizes (the padding to whole groups included).
double batched_sym_work_ratio(const std::vector<int64_t> &off);
// Bytes of group-pair partials the pair-symmetric form keeps for these sizes
// (sum over systems of groups^2 x 3 x 256 floats).
size_t batched_sym_part_bytes(const std::vector<int64_t> &off);
bool batched_sym_plan(int num_sms, const std::vector<int64_t> &off, BatchPlan &plan, std::string &why);
cudaError_t batched_sym_upload(const BatchPlan &plan, void *scratch, cudaStream_t st);
const int64_t *batched_sym_offsets(const BatchPlan &plan, void *scratch);
cudaError_t batched_sym_enqueue(const BatchPlan &plan, void *scratch, void *x, void *v,
                                const void *m, int steps, int kdk, float eps2, double G, double dt,
                                int *err, uint64_t timeout_ns, int stall, cudaStream_t st);

// Build the plan for the given offsets on this device. Shape fields of
// `plan` (nt, r, jt) may be preset; plan.sym = 1 builds the pair-symmetric
// form (and the functions below dispatch on it).
bool batched_plan(int device, int num_sms, const std::vector<int64_t> &off, BatchPlan &plan,
                  std::string &why);

// Copy the plan's arrays into `scratch` on `st`.
cudaError_t batched_upload(const BatchPlan &plan, void *scratch, cudaStream_t st);
// Deterministic synthetic state for tuning runs (positions in [-1,1]^3,
// small velocities, masses 1/N_s; float or double per plan.f64): timing does
// not depend on the values.
cudaError_t batched_fill_synthetic(const BatchPlan &plan, void *scratch, void *x, void *v, void *m,
                                   cudaStream_t st);
// Zero the queue and completion counters, pack every system, launch the
// persistent kernel for `steps` steps of the paper scheme (kdk = 0) or of
// kick-drift-kick (kdk = 1). stall (debug, the pair-symmetric form): one warp
// never releases its first item, so the items waiting for it run out their
// wait limit.
cudaError_t batched_enqueue(const BatchPlan &plan, void *scratch, void *x, void *v,
                            const void *m, int steps, int kdk, float eps2, double G, double dt,
                            int *err, uint64_t timeout_ns, int stall, cudaStream_t st);

}  // namespace nb
