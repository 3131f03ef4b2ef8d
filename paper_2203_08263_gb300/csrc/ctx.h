// Internal state of a libnbody context and the host-side helpers shared by
// the C-ABI translation units (api*.cu). Host code only.
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/nbody.h"
#include "batched.h"
#include "kernels.h"

namespace nb {
namespace detail {

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    int64_t nodes = 0;
    uint64_t stamp = 0;
};

struct TuneEntry {
    int pol, nt, r, jt, split_mode;  // split_mode: -1 half, 0 balanced, +1 double
};

}  // namespace detail
}  // namespace nb

struct nb_ctx {
    using DevBuf = nb::detail::DevBuf;
    int device = 0;
    nb_params p{};
    std::string err;
    int num_sms = 0;
    std::string dev_name;
    cudaStream_t side = nullptr;   // capture, tuning
    cudaStream_t side2 = nullptr;  // second branch of the adjoint graph
    int *err_word = nullptr;
    // scratch
    DevBuf xm[2], rec, part, counters, vals, red, st_v, abar64, stage[4], tune[6];
    DevBuf bat;      // batched-kernel scratch
    DevBuf gridbar;  // grid form of the step loop: barrier counter
    // adjoint: ping-pong segment buffers and the recompute stream's split scratch
    DevBuf adj_traj[2], adj_traj64[2], adj_x[2], adj_v[2], part2, counters2;
    std::map<std::string, nb::detail::GraphEntry> graphs;
    uint64_t stamp = 0;
    uint64_t timeout_ns = 2000000000ull;
    int debug = 0;
    int math = 0;  // ablation of the FP32 forward denominator (0 = MUFU rsqrt)
    int run_path = 0;  // nb_run: 0 chosen per size, 1 graph of force launches, 2 one cluster, 3 grid
    int form_pin = 0;  // FP32 forward: 0 chosen per size, 1 one-sided only, 512/1024 pair-symmetric blocks
    int vjp_form_pin = 0;  // FP32 VJP: 0 chosen per size, 1 one-sided only, 256/512 pair-symmetric blocks
    int sym_tile = 0;      // pair-symmetric tiles: 0 chosen per size, -1 never, w > 0 tiles of w blocks
    int adj_unfused = 0;   // nb_adjoint: 1 = every reverse step prepared by a kernel of its own
    std::map<int64_t, int> cluster_sizes;  // 2n + f64 -> cluster size of the one-cluster path (0: none)
    int64_t launches = 0;
    std::map<std::string, nb::detail::TuneEntry> tuned;
    std::map<uint64_t, nb::BatchPlan> batched_tuned;  // size profile -> tuned batched shape
    std::string tune_path;
};

namespace nb {
namespace detail {

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }
inline bool f64_state(const nb_ctx *ctx) { return ctx->p.precision == NB_FP32_COMP_FP64_STATE; }
inline size_t esize(const nb_ctx *ctx) { return f64_state(ctx) ? 8 : 4; }
inline int iblocks_of(int64_t n, int nt, int r) {
    return (int)((n + (int64_t)nt * r - 1) / ((int64_t)nt * r));
}

// Two timing events, destroyed on every exit path.
struct EventPair {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t create() {
        cudaError_t e = cudaEventCreate(&e0);
        return e != cudaSuccess ? e : cudaEventCreate(&e1);
    }
    ~EventPair() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

// One force launch: the shape and the sizes derived from it.
struct Plan {
    Shape s;
    const ForceEntry *e;
    int64_t npad;
    int iblocks, ntiles;
    size_t part_bytes;
    int tile_w = 0, ntile = 0;  // pair-symmetric forms launched by tiles of tile_w blocks (0: one launch)
};

// Record a formatted error message on ctx and return s.
nb_status fail(nb_ctx *ctx, nb_status s, const char *fmt, ...);
// Drop every cached CUDA graph.
void clear_graphs(nb_ctx *ctx);
// Grow a scratch buffer (waits for the device and drops cached graphs; not
// during a capture). zero: clear the new allocation.
nb_status ensure(nb_ctx *ctx, DevBuf &b, size_t bytes, bool zero = false);
// Validate a caller pointer: non-NULL, aligned, on the context's device, or
// host memory when `host` is non-NULL (then *host says which).
nb_status check_ptr(nb_ctx *ctx, const void *p, size_t align, const char *name, bool *host);
nb_status validate_params(nb_ctx *ctx, double G, double eps, double dt);

// Launch shapes.
int balanced_split(const nb_ctx *ctx, int iblocks, int ntiles, int occ);
const ForceEntry *find_entry(int pol, int nt, int r);
std::string tune_key(const nb_ctx *ctx, int mode, int64_t n);
int mode_pol(const nb_ctx *ctx, int mode);
Shape finish_shape(const nb_ctx *ctx, int pol, int nt, int r, int jt, int split_mode, int64_t n);
Shape heuristic_shape(const nb_ctx *ctx, int mode, int64_t n, bool allow_sym = true);
nb_status choose_shape(nb_ctx *ctx, int mode, int64_t n, Shape *out, bool *from_tune);
nb_status make_plan(nb_ctx *ctx, const Shape &s, int64_t n, Plan *p);
nb_status plan_scratch(nb_ctx *ctx, const Plan &p);

// Launches.
ForceArgs base_args(nb_ctx *ctx, const Plan &p, int64_t n, const float4 *src);
nb_status launch_force(nb_ctx *ctx, const Plan &p, const ForceArgs &a, cudaStream_t st);
// Pack (x, m) into xm (zero-mass padding up to npad); `pads` names the
// buffers the following step epilogues write, whose padding is zeroed too.
nb_status pack(nb_ctx *ctx, int64_t n, int64_t npad, const void *x, const void *v, const void *m,
               float4 *xm, void *ckpt0, cudaStream_t st, PadTargets pads = PadTargets());
GraphEntry *graph_lookup(nb_ctx *ctx, const std::string &key);
void graph_insert(nb_ctx *ctx, const std::string &key, cudaGraphExec_t ex, int64_t nodes);
// Which nb_run path serves n bodies: *path = 1 graph of force launches,
// 2 one-cluster kernel, 3 grid form of it; *size = the cluster size or the
// grid's CTAs.
nb_status choose_run_path(nb_ctx *ctx, int64_t n, int *path, int *size);
nb_status run_device(nb_ctx *ctx, int64_t n, void *x, void *v, const void *m, int steps,
                     void *ckpt, int ckpt_every, cudaStream_t st);
nb_status accel_device(nb_ctx *ctx, int64_t n, const void *x, const void *m, void *a_out,
                       cudaStream_t st);
// Wait for st, then report (and clear) a device-side error.
nb_status sync_and_check(nb_ctx *ctx, cudaStream_t st);

// Batched helpers and the tuning table.
uint64_t sizes_signature(const std::vector<int64_t> &off);
nb_status read_offsets(nb_ctx *ctx, int nsys, const int64_t *offsets, cudaStream_t st,
                       std::vector<int64_t> &off);
void load_tune_file(nb_ctx *ctx);
void save_tune_file(nb_ctx *ctx);

}  // namespace detail
}  // namespace nb

#define NB_CUDA(call)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return ::nb::detail::fail(ctx, e_ == cudaErrorMemoryAllocation ? NB_ERR_NOMEM   \
                                                                            : NB_ERR_CUDA,  \
                                      "%s: %s", #call, cudaGetErrorString(e_));            \
    } while (0)

#define NB_TRY(expr)                \
    do {                            \
        nb_status s_ = (expr);      \
        if (s_ != NB_OK) return s_; \
    } while (0)
