// libnbody C-ABI: context, scratch memory, launch-shape choice, CUDA-graph
// cache, host-pointer staging and the autotuner. Every step of the method
// runs in the kernels of this library; this file only validates, plans and
// launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/nbody.h"
#include "batched.h"
#include "kernels.h"

namespace nb {
const ForceEntry *table_f32x2(int *count);
const ForceEntry *table_scalar(int *count);
const ForceEntry *table_comp(int *count);
const ForceEntry *table_pot(int *count);
const ForceEntry *table_vjp(int *count);
const ForceEntry *table_vjp_comp(int *count);
const ForceEntry *table_div(int *count);
const ForceEntry *table_pow(int *count);

const ForceEntry *force_table(int pol, int *count) {
    switch (pol) {
        case kPolF32x2: return table_f32x2(count);
        case kPolScalar: return table_scalar(count);
        case kPolComp: return table_comp(count);
        case kPolPot: return table_pot(count);
        case kPolVjp: return table_vjp(count);
        case kPolVjpComp: return table_vjp_comp(count);
        case kPolDiv: return table_div(count);
        case kPolPow: return table_pow(count);
        default: *count = 0; return nullptr;
    }
}
int pol_rec_f4(int pol) { return pol == kPolVjp ? 4 : (pol == kPolVjpComp ? 5 : 2); }
int pol_part_f4(int pol) {
    switch (pol) {
        case kPolComp: return 2;
        case kPolVjp: return 2;
        case kPolVjpComp: return 4;
        default: return 1;
    }
}
}  // namespace nb

using namespace nb;

namespace {

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

int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

}  // namespace

struct nb_ctx {
    int device = 0;
    nb_params p{};
    std::string err;
    int num_sms = 0;
    std::string dev_name;
    cudaStream_t side = nullptr;
    int *err_word = nullptr;
    // scratch
    DevBuf xm[2], rec, part, counters, vals, red, traj, traj64, st_x, st_v, abar64, stage[4], tune[6];
    DevBuf bat;  // batched-kernel scratch
    // adjoint: ping-pong segment buffers and the recompute stream's split scratch
    DevBuf adj_traj[2], adj_traj64[2], adj_x[2], adj_v[2], part2, counters2;
    cudaStream_t side2 = nullptr;
    std::map<std::string, GraphEntry> graphs;
    uint64_t stamp = 0;
    uint64_t timeout_ns = 2000000000ull;
    int debug = 0;
    int math = 0;  // ablation of the FP32 forward denominator (0 = MUFU rsqrt)
    int64_t launches = 0;
    std::map<std::string, TuneEntry> tuned;
    std::map<uint64_t, BatchPlan> batched_tuned;  // size profile -> tuned batched shape
    std::string tune_path;
};

namespace {

nb_status fail(nb_ctx *ctx, nb_status s, const char *fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return s;
}

#define NB_CUDA(call)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? NB_ERR_NOMEM : NB_ERR_CUDA, \
                        "%s: %s", #call, cudaGetErrorString(e_));                           \
    } while (0)

#define NB_TRY(expr)                     \
    do {                                 \
        nb_status s_ = (expr);           \
        if (s_ != NB_OK) return s_;      \
    } while (0)

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

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

void clear_graphs(nb_ctx *ctx) {
    for (auto &kv : ctx->graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    ctx->graphs.clear();
}

// Grow a scratch buffer. Growth waits for the device and drops cached graphs
// (they may reference the old allocation), so it must not happen during a
// stream capture.
nb_status ensure(nb_ctx *ctx, DevBuf &b, size_t bytes, bool zero = false) {
    if (bytes == 0) bytes = 256;
    if (b.bytes >= bytes) return NB_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(ctx->side, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
        return fail(ctx, NB_ERR_INVALID, "scratch growth requested during stream capture");
    NB_CUDA(cudaDeviceSynchronize());
    clear_graphs(ctx);
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    size_t want = (size_t)round_up((int64_t)bytes, 1 << 20);
    NB_CUDA(cudaMalloc(&b.p, want));
    b.bytes = want;
    if (zero) NB_CUDA(cudaMemset(b.p, 0, want));
    return NB_OK;
}

nb_status check_ptr(nb_ctx *ctx, const void *p, size_t align, const char *name, bool *host) {
    if (!p) return fail(ctx, NB_ERR_INVALID, "%s is NULL", name);
    if (reinterpret_cast<uintptr_t>(p) % align)
        return fail(ctx, NB_ERR_INVALID, "%s is not %zu-byte aligned", name, align);
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, NB_ERR_INVALID, "%s: cannot query pointer (%s)", name,
                    cudaGetErrorString(e));
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
        if (at.device != ctx->device)
            return fail(ctx, NB_ERR_INVALID, "%s lives on device %d, context is on %d", name,
                        at.device, ctx->device);
        if (host) *host = false;
        return NB_OK;
    }
    if (!host) return fail(ctx, NB_ERR_INVALID, "%s must be a device pointer", name);
    *host = true;
    return NB_OK;
}

bool f64_state(const nb_ctx *ctx) { return ctx->p.precision == NB_FP32_COMP_FP64_STATE; }
size_t esize(const nb_ctx *ctx) { return f64_state(ctx) ? 8 : 4; }

nb_status validate_params(nb_ctx *ctx, double G, double eps, double dt) {
    if (!std::isfinite(G) || !std::isfinite(eps) || !std::isfinite(dt))
        return fail(ctx, NB_ERR_INVALID, "G, eps and dt must be finite");
    if (!(eps > 0.0) || !((float)(eps * eps) >= 1.17549435e-38f))
        return fail(ctx, NB_ERR_INVALID,
                    "eps must be > 0 with eps^2 a normal FP32 number (the j = i term is 0/0 otherwise)");
    return NB_OK;
}

// ----------------------------------------------------------- shape choice

int iblocks_of(int64_t n, int nt, int r) { return (int)((n + (int64_t)nt * r - 1) / ((int64_t)nt * r)); }

// Pick the j-split that minimises (waves x tiles per CTA + fixed cost per CTA).
int balanced_split(const nb_ctx *ctx, int iblocks, int ntiles, int occ) {
    const int64_t slots = (int64_t)std::max(occ, 1) * ctx->num_sms;
    int best = 1;
    double best_cost = 1e300;
    const int smax = std::min(ntiles, 1024);
    for (int s = 1; s <= smax; ++s) {
        int64_t ctas = (int64_t)iblocks * s;
        int64_t waves = (ctas + slots - 1) / slots;
        int per = (ntiles + s - 1) / s;
        double cost = (double)waves * (per + 1.5);
        if (cost < best_cost * 0.999) {
            best_cost = cost;
            best = s;
        }
    }
    return best;
}

const ForceEntry *find_entry(int pol, int nt, int r) {
    int cnt = 0;
    const ForceEntry *t = force_table(pol, &cnt);
    for (int k = 0; k < cnt; ++k)
        if (t[k].nt == nt && t[k].r == r) return &t[k];
    return nullptr;
}

std::string tune_key(const nb_ctx *ctx, int mode, int64_t n) {
    int bucket = 0;
    while ((int64_t(1) << bucket) < n) ++bucket;
    char buf[256];
    snprintf(buf, sizeof buf, "%s|%d|m%d|p%d|b%d", ctx->dev_name.c_str(), ctx->num_sms, mode,
             ctx->p.precision, bucket);
    return buf;
}

int mode_pol(const nb_ctx *ctx, int mode) {
    if (mode == 0 && !f64_state(ctx) && ctx->math == 1) return kPolDiv;
    if (mode == 0 && !f64_state(ctx) && ctx->math == 2) return kPolPow;
    if (mode == 0) return f64_state(ctx) ? kPolComp : kPolF32x2;
    if (mode == 1) return f64_state(ctx) ? kPolVjpComp : kPolVjp;
    return kPolPot;
}

Shape finish_shape(const nb_ctx *ctx, int pol, int nt, int r, int jt, int split_mode, int64_t n) {
    const ForceEntry *e = find_entry(pol, nt, r);
    const int64_t npad = round_up(std::max<int64_t>(n, 1), kPadBodies);
    const int ntiles = (int)(npad / jt);
    const int ib = iblocks_of(n, nt, r);
    const int occ = e ? e->occupancy(jt) : 1;
    int s = balanced_split(ctx, ib, ntiles, occ);
    if (split_mode < 0) s = std::max(1, s / 2);
    if (split_mode > 0) s = std::min(ntiles, s * 2);
    return Shape{pol, nt, r, s, jt};
}

// Built-in choice when no tuning entry exists.
Shape heuristic_shape(const nb_ctx *ctx, int mode, int64_t n) {
    const int pol = mode_pol(ctx, mode);
    int nt = 128, r = 1, jt = 64;
    if (pol == kPolF32x2) {
        if (n >= 32768) { r = 4; jt = 128; }
        else if (n >= 4096) { r = 2; jt = 128; }
    } else if (pol == kPolDiv || pol == kPolPow) {
        r = 4;
        if (n >= 4096) jt = 128;
    } else if (pol == kPolComp) {
        r = n >= 65536 ? 4 : 2;
        if (n >= 4096) jt = 128;
    } else if (pol == kPolPot) {
        r = 2;
        if (n >= 4096) jt = 128;
    } else {  // VJP (the precision form's R = 2 instance spills at the 128-register cap)
        r = (n >= 8192 && pol == kPolVjp) ? 2 : 1;
        if (n >= 4096) jt = 128;
    }
    return finish_shape(ctx, pol, nt, r, jt, 0, n);
}

nb_status choose_shape(nb_ctx *ctx, int mode, int64_t n, Shape *out, bool *from_tune) {
    if (from_tune) *from_tune = false;
    const int *o = ctx->p.tile_override;
    const int pol = mode_pol(ctx, mode);
    if (mode != 2 && (o[0] || o[1] || o[2] || o[3])) {
        Shape h = heuristic_shape(ctx, mode, n);
        int nt = o[0] ? o[0] : h.nt, r = o[1] ? o[1] : h.r, jt = o[3] ? o[3] : h.jt;
        if (!find_entry(pol, nt, r))
            return fail(ctx, NB_ERR_UNSUPPORTED, "no compiled kernel for %d threads x %d bodies", nt, r);
        if (jt < 2 || jt % 2 || kPadBodies % jt)
            return fail(ctx, NB_ERR_INVALID, "j-tile %d must be even and divide %d", jt, kPadBodies);
        Shape s = finish_shape(ctx, pol, nt, r, jt, 0, n);
        if (o[2] > 0) s.split = std::min<int>(o[2], (int)(round_up(std::max<int64_t>(n, 1), kPadBodies) / jt));
        *out = s;
        return NB_OK;
    }
    auto it = ctx->tuned.find(tune_key(ctx, mode, n));
    if (mode != 2 && ctx->math == 0 && it != ctx->tuned.end() &&
        find_entry(it->second.pol, it->second.nt, it->second.r)) {
        const TuneEntry &t = it->second;
        *out = finish_shape(ctx, t.pol, t.nt, t.r, t.jt, t.split_mode, n);
        if (from_tune) *from_tune = true;
        return NB_OK;
    }
    *out = heuristic_shape(ctx, mode, n);
    return NB_OK;
}

// ------------------------------------------------------------ force launch

struct Plan {
    Shape s;
    const ForceEntry *e;
    int64_t npad;
    int iblocks, ntiles;
    size_t part_bytes;
};

nb_status make_plan(nb_ctx *ctx, const Shape &s, int64_t n, Plan *p) {
    p->s = s;
    p->e = find_entry(s.pol, s.nt, s.r);
    if (!p->e) return fail(ctx, NB_ERR_UNSUPPORTED, "no kernel for shape");
    p->npad = round_up(std::max<int64_t>(n, 1), kPadBodies);
    p->iblocks = iblocks_of(std::max<int64_t>(n, 1), s.nt, s.r);
    p->ntiles = (int)(p->npad / s.jt);
    p->part_bytes = s.split > 1 ? (size_t)s.split * p->iblocks * s.nt * s.r *
                                      pol_part_f4(s.pol) * 16
                                : 0;
    return NB_OK;
}

nb_status plan_scratch(nb_ctx *ctx, const Plan &p) {
    NB_TRY(ensure(ctx, ctx->part, p.part_bytes));
    NB_TRY(ensure(ctx, ctx->counters, (size_t)p.iblocks * 4, true));
    return NB_OK;
}

ForceArgs base_args(nb_ctx *ctx, const Plan &p, int64_t n, const float4 *src) {
    ForceArgs a;
    memset(&a, 0, sizeof a);
    a.src = src;
    a.n = n;
    a.npad = p.npad;
    a.jt = p.s.jt;
    a.ntiles = p.ntiles;
    a.split = p.s.split;
    a.iblocks = p.iblocks;
    a.eps2 = (float)(ctx->p.eps * ctx->p.eps);
    a.G = ctx->p.G;
    a.dt = ctx->p.dt;
    a.part = reinterpret_cast<float4 *>(ctx->part.p);
    a.counters = reinterpret_cast<unsigned *>(ctx->counters.p);
    a.err = ctx->err_word;
    a.timeout_ns = ctx->timeout_ns;
    a.debug = ctx->debug;
    return a;
}

nb_status launch_force(nb_ctx *ctx, const Plan &p, const ForceArgs &a, cudaStream_t st) {
    NB_CUDA(p.e->launch(p.s.jt, a, st));
    ctx->launches += 1;
    return NB_OK;
}

nb_status pack(nb_ctx *ctx, int64_t n, int64_t npad, const void *x, const void *v, const void *m,
               float4 *xm, void *ckpt0, cudaStream_t st) {
    if (f64_state(ctx))
        NB_CUDA(launch_pack_f64(n, npad, (const double *)x, (const double *)v, (const double *)m,
                                xm, (double *)ckpt0, st));
    else
        NB_CUDA(launch_pack_f32(n, npad, (const float *)x, (const float *)v, (const float *)m, xm,
                                (float *)ckpt0, st));
    ctx->launches += 1;
    return NB_OK;
}

// ------------------------------------------------------------- graphs

GraphEntry *graph_lookup(nb_ctx *ctx, const std::string &key) {
    auto it = ctx->graphs.find(key);
    if (it == ctx->graphs.end()) return nullptr;
    it->second.stamp = ++ctx->stamp;
    return &it->second;
}

void graph_insert(nb_ctx *ctx, const std::string &key, cudaGraphExec_t ex, int64_t nodes) {
    if (ctx->graphs.size() >= 16) {
        auto victim = ctx->graphs.begin();
        for (auto it = ctx->graphs.begin(); it != ctx->graphs.end(); ++it)
            if (it->second.stamp < victim->second.stamp) victim = it;
        cudaGraphExecDestroy(victim->second.exec);
        ctx->graphs.erase(victim);
    }
    GraphEntry g;
    g.exec = ex;
    g.nodes = nodes;
    g.stamp = ++ctx->stamp;
    ctx->graphs[key] = g;
}

// ------------------------------------------------------- device run path

nb_status run_device(nb_ctx *ctx, int64_t n, void *x, void *v, const void *m, int steps,
                     void *ckpt, int ckpt_every, cudaStream_t st) {
    Shape s;
    NB_TRY(choose_shape(ctx, 0, n, &s, nullptr));
    Plan p;
    NB_TRY(make_plan(ctx, s, n, &p));
    NB_TRY(plan_scratch(ctx, p));
    NB_TRY(ensure(ctx, ctx->xm[0], (size_t)p.npad * 16));
    NB_TRY(ensure(ctx, ctx->xm[1], (size_t)p.npad * 16));
    const bool kdk = ctx->p.scheme == NB_SCHEME_KDK;
    char key[512];
    snprintf(key, sizeof key, "run|%lld|%p|%p|%p|%d|%p|%d|%d.%d.%d.%d.%d|%llu|%d|%a|%a|%a",
             (long long)n, x, v, m, steps, ckpt, ckpt_every, s.pol, s.nt, s.r, s.split, s.jt,
             (unsigned long long)ctx->timeout_ns * 16 + ctx->debug * 4 + ctx->math, ctx->p.scheme, ctx->p.G, ctx->p.eps, ctx->p.dt);
    GraphEntry *g = graph_lookup(ctx, key);
    if (!g) {
        NB_CUDA(cudaStreamBeginCapture(ctx->side, cudaStreamCaptureModeThreadLocal));
        int64_t saved = ctx->launches;
        float4 *xm[2] = {(float4 *)ctx->xm[0].p, (float4 *)ctx->xm[1].p};
        nb_status rs = pack(ctx, n, p.npad, x, v, m, xm[0], ckpt, ctx->side);
        const size_t slot_bytes = (size_t)n * 6 * esize(ctx);
        for (int t = 0; rs == NB_OK && t < steps; ++t) {
            ForceArgs a = base_args(ctx, p, n, xm[t & 1]);
            a.op = (kdk && t > 0) ? kEpiKick2Drift : kEpiKickDrift;
            a.x = x;
            a.v = v;
            a.xm_next = xm[(t + 1) & 1];
            if (ckpt && (t + 1) % ckpt_every == 0)
                a.ckpt = (char *)ckpt + (size_t)((t + 1) / ckpt_every) * slot_bytes;
            rs = launch_force(ctx, p, a, ctx->side);
        }
        if (rs == NB_OK && kdk && steps > 0) {
            ForceArgs a = base_args(ctx, p, n, xm[steps & 1]);
            a.op = kEpiKick;
            a.x = x;
            a.v = v;
            a.xm_next = xm[(steps + 1) & 1];
            rs = launch_force(ctx, p, a, ctx->side);
        }
        cudaGraph_t graph = nullptr;
        cudaError_t ce = cudaStreamEndCapture(ctx->side, &graph);
        int64_t nodes = ctx->launches - saved;
        ctx->launches = saved;
        if (rs != NB_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rs;
        }
        if (ce != cudaSuccess) return fail(ctx, NB_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ce));
        cudaGraphExec_t ex = nullptr;
        ce = cudaGraphInstantiate(&ex, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return fail(ctx, NB_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
        graph_insert(ctx, key, ex, nodes);
        g = graph_lookup(ctx, key);
    }
    NB_CUDA(cudaGraphLaunch(g->exec, st));
    ctx->launches += g->nodes;
    return NB_OK;
}

nb_status accel_device(nb_ctx *ctx, int64_t n, const void *x, const void *m, void *a_out,
                       cudaStream_t st) {
    Shape s;
    NB_TRY(choose_shape(ctx, 0, n, &s, nullptr));
    Plan p;
    NB_TRY(make_plan(ctx, s, n, &p));
    NB_TRY(plan_scratch(ctx, p));
    NB_TRY(ensure(ctx, ctx->xm[0], (size_t)p.npad * 16));
    float4 *xm = (float4 *)ctx->xm[0].p;
    NB_TRY(pack(ctx, n, p.npad, x, nullptr, m, xm, nullptr, st));
    ForceArgs a = base_args(ctx, p, n, xm);
    a.op = kEpiAccel;
    a.out = a_out;
    return launch_force(ctx, p, a, st);
}

// Wait for `st`, then report and clear a device-side error.
nb_status sync_and_check(nb_ctx *ctx, cudaStream_t st) {
    NB_CUDA(cudaStreamSynchronize(st));
    int h = 0;
    NB_CUDA(cudaMemcpy(&h, ctx->err_word, sizeof h, cudaMemcpyDeviceToHost));
    if (h) {
        NB_CUDA(cudaMemset(ctx->err_word, 0, sizeof(int)));
        return fail(ctx, NB_ERR_TIMEOUT,
                    "device-side wait gave up (error bits 0x%x: 1 tile wait, 2 slot wait, "
                    "4 copy drain, 8 batched step dependency); results of the affected calls are invalid",
                    h);
    }
    return NB_OK;
}

// FNV-1a over the system sizes: the key of the batched tuning table.
uint64_t sizes_signature(const std::vector<int64_t> &off) {
    uint64_t h = 1469598103934665603ull;
    for (size_t s = 1; s < off.size(); ++s) {
        uint64_t v = (uint64_t)(off[s] - off[s - 1]);
        for (int b = 0; b < 8; ++b) {
            h ^= (v >> (8 * b)) & 0xff;
            h *= 1099511628211ull;
        }
    }
    return h;
}

// Offsets may live on the host or the device; validate them.
nb_status read_offsets(nb_ctx *ctx, int nsys, const int64_t *offsets, cudaStream_t st,
                       std::vector<int64_t> &off) {
    off.assign((size_t)nsys + 1, 0);
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, offsets);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, NB_ERR_INVALID, "offsets: cannot query pointer");
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
        NB_CUDA(cudaStreamSynchronize(st));
        NB_CUDA(cudaMemcpy(off.data(), offsets, off.size() * 8, cudaMemcpyDeviceToHost));
    } else {
        memcpy(off.data(), offsets, off.size() * 8);
    }
    if (off[0] != 0) return fail(ctx, NB_ERR_INVALID, "offsets[0] must be 0");
    for (int s = 0; s < nsys; ++s) {
        const int64_t ns = off[s + 1] - off[s];
        if (ns < 0) return fail(ctx, NB_ERR_INVALID, "offsets must be non-decreasing");
        if (ns > batched_max_n())
            return fail(ctx, NB_ERR_INVALID, "system %d has %lld bodies, above the limit %lld", s,
                        (long long)ns, (long long)batched_max_n());
    }
    return NB_OK;
}

// ------------------------------------------------------------- tuner JSON

void load_tune_file(nb_ctx *ctx) {
    const char *path = getenv("NB_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    ctx->tune_path = path;
    FILE *f = fopen(path, "r");
    if (!f) return;
    std::string s;
    char buf[4096];
    size_t k;
    while ((k = fread(buf, 1, sizeof buf, f)) > 0) s.append(buf, k);
    fclose(f);
    // entries look like  "key": [pol, nt, r, jt, split_mode]
    size_t pos = 0;
    while ((pos = s.find('"', pos)) != std::string::npos) {
        size_t end = s.find('"', pos + 1);
        if (end == std::string::npos) break;
        std::string key = s.substr(pos + 1, end - pos - 1);
        size_t lb = s.find('[', end), rb = s.find(']', end);
        if (lb == std::string::npos || rb == std::string::npos || rb < lb) break;
        TuneEntry t;
        if (sscanf(s.c_str() + lb + 1, "%d , %d , %d , %d , %d", &t.pol, &t.nt, &t.r, &t.jt,
                   &t.split_mode) == 5)
            ctx->tuned[key] = t;
        pos = rb + 1;
    }
}

void save_tune_file(nb_ctx *ctx) {
    if (ctx->tune_path.empty()) return;
    std::string tmp = ctx->tune_path + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return;
    fprintf(f, "{\n");
    size_t i = 0;
    for (auto &kv : ctx->tuned) {
        const TuneEntry &t = kv.second;
        fprintf(f, "  \"%s\": [%d, %d, %d, %d, %d]%s\n", kv.first.c_str(), t.pol, t.nt, t.r, t.jt,
                t.split_mode, ++i < ctx->tuned.size() ? "," : "");
    }
    fprintf(f, "}\n");
    fclose(f);
    rename(tmp.c_str(), ctx->tune_path.c_str());
}

}  // namespace

// ======================================================================
//                                C-ABI
// ======================================================================

extern "C" {

int nb_abi_version(void) { return NB_ABI_VERSION; }

const char *nb_status_string(nb_status s) {
    switch (s) {
        case NB_OK: return "NB_OK";
        case NB_ERR_INVALID: return "NB_ERR_INVALID";
        case NB_ERR_CUDA: return "NB_ERR_CUDA";
        case NB_ERR_NOMEM: return "NB_ERR_NOMEM";
        case NB_ERR_TIMEOUT: return "NB_ERR_TIMEOUT";
        case NB_ERR_UNSUPPORTED: return "NB_ERR_UNSUPPORTED";
    }
    return "NB_ERR_UNKNOWN";
}

const char *nb_last_error(const nb_ctx *ctx) { return ctx ? ctx->err.c_str() : ""; }

nb_status nb_create(nb_ctx **out, int device, const nb_params *p) {
    if (!out) return NB_ERR_INVALID;
    *out = nullptr;
    if (!p) return NB_ERR_INVALID;
    if (!std::isfinite(p->G) || !std::isfinite(p->eps) || !std::isfinite(p->dt) || !(p->eps > 0) ||
        !((float)(p->eps * p->eps) >= 1.17549435e-38f))
        return NB_ERR_INVALID;
    if (p->precision != NB_FP32 && p->precision != NB_FP32_COMP_FP64_STATE) return NB_ERR_INVALID;
    if (p->scheme != NB_SCHEME_PAPER && p->scheme != NB_SCHEME_KDK) return NB_ERR_INVALID;
    for (int k = 0; k < 4; ++k)
        if (p->tile_override[k] < 0) return NB_ERR_INVALID;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return device < 0 ? NB_ERR_INVALID : NB_ERR_CUDA;
    }
    nb_ctx *ctx = new (std::nothrow) nb_ctx;
    if (!ctx) return NB_ERR_NOMEM;
    ctx->device = device;
    ctx->p = *p;
    cudaDeviceProp prop;
    if (cudaSetDevice(device) != cudaSuccess || cudaGetDeviceProperties(&prop, device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->side2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&ctx->err_word, sizeof(int)) != cudaSuccess ||
        cudaMemset(ctx->err_word, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        nb_destroy(ctx);
        return NB_ERR_CUDA;
    }
    ctx->num_sms = prop.multiProcessorCount;
    ctx->dev_name = prop.name;
    for (auto &ch : ctx->dev_name)
        if (ch == '"' || ch == '|') ch = '_';
    load_tune_file(ctx);
    *out = ctx;
    return NB_OK;
}

void nb_destroy(nb_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    clear_graphs(ctx);
    DevBuf *bufs[] = {&ctx->xm[0], &ctx->xm[1], &ctx->rec,      &ctx->part,     &ctx->counters,
                      &ctx->vals,  &ctx->red,   &ctx->traj,  &ctx->traj64,   &ctx->st_x,     &ctx->st_v,
                      &ctx->abar64, &ctx->stage[0], &ctx->stage[1], &ctx->stage[2], &ctx->stage[3],
                      &ctx->tune[0], &ctx->tune[1], &ctx->tune[2], &ctx->tune[3], &ctx->tune[4],
                      &ctx->tune[5], &ctx->bat, &ctx->adj_traj[0], &ctx->adj_traj[1],
                      &ctx->adj_traj64[0], &ctx->adj_traj64[1], &ctx->adj_x[0], &ctx->adj_x[1],
                      &ctx->adj_v[0], &ctx->adj_v[1], &ctx->part2, &ctx->counters2};
    for (DevBuf *b : bufs)
        if (b->p) cudaFree(b->p);
    if (ctx->err_word) cudaFree(ctx->err_word);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->side2) cudaStreamDestroy(ctx->side2);
    cudaGetLastError();
    delete ctx;
}

nb_status nb_set_params(nb_ctx *ctx, double G, double eps, double dt) {
    if (!ctx) return NB_ERR_INVALID;
    NB_TRY(validate_params(ctx, G, eps, dt));
    ctx->p.G = G;
    ctx->p.eps = eps;
    ctx->p.dt = dt;
    return NB_OK;
}

nb_status nb_accel(nb_ctx *ctx, int64_t n, const void *x, const void *m, void *a, void *stream) {
    if (!ctx) return NB_ERR_INVALID;
    if (n < 0) return fail(ctx, NB_ERR_INVALID, "n < 0");
    if (n == 0) return NB_OK;
    NB_CUDA(cudaSetDevice(ctx->device));
    const size_t es = esize(ctx);
    bool hx, hm, ha;
    NB_TRY(check_ptr(ctx, x, es, "x", &hx));
    NB_TRY(check_ptr(ctx, m, es, "m", &hm));
    NB_TRY(check_ptr(ctx, a, es, "a", &ha));
    cudaStream_t st = as_stream(stream);
    if (!hx && !hm && !ha) return accel_device(ctx, n, x, m, a, st);
    // host path: stage through context buffers, return when results are back
    const size_t b3 = (size_t)n * 3 * es, b1 = (size_t)n * es;
    NB_TRY(ensure(ctx, ctx->stage[0], b3));
    NB_TRY(ensure(ctx, ctx->stage[2], b1));
    NB_TRY(ensure(ctx, ctx->stage[3], b3));
    const void *dx = x, *dm = m;
    void *da = a;
    if (hx) { NB_CUDA(cudaMemcpyAsync(ctx->stage[0].p, x, b3, cudaMemcpyHostToDevice, st)); dx = ctx->stage[0].p; }
    if (hm) { NB_CUDA(cudaMemcpyAsync(ctx->stage[2].p, m, b1, cudaMemcpyHostToDevice, st)); dm = ctx->stage[2].p; }
    if (ha) da = ctx->stage[3].p;
    NB_TRY(accel_device(ctx, n, dx, dm, da, st));
    if (ha) NB_CUDA(cudaMemcpyAsync(a, da, b3, cudaMemcpyDeviceToHost, st));
    return sync_and_check(ctx, st);
}

nb_status nb_run(nb_ctx *ctx, int64_t n, void *x, void *v, const void *m, int steps, void *ckpt,
                 int ckpt_every, void *stream) {
    if (!ctx) return NB_ERR_INVALID;
    if (n < 0) return fail(ctx, NB_ERR_INVALID, "n < 0");
    if (steps < 0) return fail(ctx, NB_ERR_INVALID, "steps < 0");
    if (ckpt) {
        if (ckpt_every <= 0 || steps % ckpt_every)
            return fail(ctx, NB_ERR_INVALID, "ckpt_every must be > 0 and divide steps");
        if (ctx->p.scheme != NB_SCHEME_PAPER)
            return fail(ctx, NB_ERR_UNSUPPORTED, "checkpoints are written for the paper scheme only");
    }
    if (n == 0 || (steps == 0 && !ckpt)) return NB_OK;
    NB_CUDA(cudaSetDevice(ctx->device));
    const size_t es = esize(ctx);
    bool hx, hv, hm;
    NB_TRY(check_ptr(ctx, x, es, "x", &hx));
    NB_TRY(check_ptr(ctx, v, es, "v", &hv));
    NB_TRY(check_ptr(ctx, m, es, "m", &hm));
    if (ckpt) NB_TRY(check_ptr(ctx, ckpt, es, "ckpt", nullptr));
    cudaStream_t st = as_stream(stream);
    if (!hx && !hv && !hm) return run_device(ctx, n, x, v, m, steps, ckpt, ckpt_every, st);
    const size_t b3 = (size_t)n * 3 * es, b1 = (size_t)n * es;
    NB_TRY(ensure(ctx, ctx->stage[0], b3));
    NB_TRY(ensure(ctx, ctx->stage[1], b3));
    NB_TRY(ensure(ctx, ctx->stage[2], b1));
    void *dx = x, *dv = v;
    const void *dm = m;
    if (hx) { NB_CUDA(cudaMemcpyAsync(ctx->stage[0].p, x, b3, cudaMemcpyHostToDevice, st)); dx = ctx->stage[0].p; }
    if (hv) { NB_CUDA(cudaMemcpyAsync(ctx->stage[1].p, v, b3, cudaMemcpyHostToDevice, st)); dv = ctx->stage[1].p; }
    if (hm) { NB_CUDA(cudaMemcpyAsync(ctx->stage[2].p, m, b1, cudaMemcpyHostToDevice, st)); dm = ctx->stage[2].p; }
    NB_TRY(run_device(ctx, n, dx, dv, dm, steps, ckpt, ckpt_every, st));
    if (hx) NB_CUDA(cudaMemcpyAsync(x, dx, b3, cudaMemcpyDeviceToHost, st));
    if (hv) NB_CUDA(cudaMemcpyAsync(v, dv, b3, cudaMemcpyDeviceToHost, st));
    return sync_and_check(ctx, st);
}

nb_status nb_step(nb_ctx *ctx, int64_t n, void *x, void *v, const void *m, void *stream) {
    return nb_run(ctx, n, x, v, m, 1, nullptr, 0, stream);
}

nb_status nb_energy(nb_ctx *ctx, int64_t n, const void *x, const void *v, const void *m,
                    double *out, void *stream) {
    if (!ctx) return NB_ERR_INVALID;
    if (!out) return fail(ctx, NB_ERR_INVALID, "out is NULL");
    if (n < 0) return fail(ctx, NB_ERR_INVALID, "n < 0");
    for (int k = 0; k < 6; ++k) out[k] = 0.0;
    if (n == 0) return NB_OK;
    NB_CUDA(cudaSetDevice(ctx->device));
    const size_t es = esize(ctx);
    NB_TRY(check_ptr(ctx, x, es, "x", nullptr));
    NB_TRY(check_ptr(ctx, v, es, "v", nullptr));
    NB_TRY(check_ptr(ctx, m, es, "m", nullptr));
    cudaStream_t st = as_stream(stream);
    Shape s;
    NB_TRY(choose_shape(ctx, 2, n, &s, nullptr));
    Plan p;
    NB_TRY(make_plan(ctx, s, n, &p));
    NB_TRY(plan_scratch(ctx, p));
    NB_TRY(ensure(ctx, ctx->xm[0], (size_t)p.npad * 16));
    NB_TRY(ensure(ctx, ctx->vals, (size_t)n * 8));
    const int blocks = std::min<int64_t>(4 * ctx->num_sms, (n + 255) / 256);
    NB_TRY(ensure(ctx, ctx->red, (size_t)(blocks * 5 + 8) * 8));
    float4 *xm = (float4 *)ctx->xm[0].p;
    NB_TRY(pack(ctx, n, p.npad, x, nullptr, m, xm, nullptr, st));
    ForceArgs a = base_args(ctx, p, n, xm);
    a.op = kEpiValue;
    a.out = ctx->vals.p;
    NB_TRY(launch_force(ctx, p, a, st));
    double *red = (double *)ctx->red.p;
    NB_CUDA(launch_energy_reduce(n, v, m, f64_state(ctx) ? 1 : 0, (const double *)ctx->vals.p,
                                 red + 8, blocks, red, st));
    ctx->launches += 2;
    double h[5];
    NB_CUDA(cudaMemcpyAsync(h, red, sizeof h, cudaMemcpyDeviceToHost, st));
    NB_TRY(sync_and_check(ctx, st));
    out[0] = h[0];
    out[1] = h[1];
    out[2] = h[2];
    out[3] = h[3];
    out[4] = -0.5 * ctx->p.G * h[4];
    out[5] = out[3] + 0.5 * out[4];
    return NB_OK;
}

nb_status nb_vjp(nb_ctx *ctx, int64_t n, const void *x, const void *m, const void *abar,
                 void *xbar, void *mbar, void *stream) {
    if (!ctx) return NB_ERR_INVALID;
    if (n < 0) return fail(ctx, NB_ERR_INVALID, "n < 0");
    if (n == 0) return NB_OK;
    NB_CUDA(cudaSetDevice(ctx->device));
    const size_t es = esize(ctx);
    NB_TRY(check_ptr(ctx, x, es, "x", nullptr));
    NB_TRY(check_ptr(ctx, m, es, "m", nullptr));
    NB_TRY(check_ptr(ctx, abar, es, "abar", nullptr));
    NB_TRY(check_ptr(ctx, xbar, es, "xbar", nullptr));
    NB_TRY(check_ptr(ctx, mbar, es, "mbar", nullptr));
    cudaStream_t st = as_stream(stream);
    Shape s;
    NB_TRY(choose_shape(ctx, 1, n, &s, nullptr));
    Plan p;
    NB_TRY(make_plan(ctx, s, n, &p));
    NB_TRY(plan_scratch(ctx, p));
    NB_TRY(ensure(ctx, ctx->xm[0], (size_t)p.npad * 16));
    NB_TRY(ensure(ctx, ctx->rec, (size_t)p.npad * 8 * pol_rec_f4(s.pol)));
    NB_TRY(ensure(ctx, ctx->abar64, (size_t)n * 24));
    NB_TRY(ensure(ctx, ctx->st_v, (size_t)n * 3 * es));
    float4 *xm = (float4 *)ctx->xm[0].p;
    if (!f64_state(ctx)) NB_TRY(pack(ctx, n, p.npad, x, nullptr, m, xm, nullptr, st));
    // abar enters as vbar' with xbar = 0 and dt = 2: abar = dt/2 (vbar + dt*0)
    NB_CUDA(cudaMemcpyAsync(ctx->st_v.p, abar, (size_t)n * 3 * es, cudaMemcpyDeviceToDevice, st));
    NB_CUDA(cudaMemsetAsync(xbar, 0, (size_t)n * 3 * es, st));
    NB_CUDA(cudaMemsetAsync(mbar, 0, (size_t)n * es, st));
    NB_CUDA(launch_adj_prepare(n, p.npad, f64_state(ctx) ? 1 : 0, xm, (const double *)x, 3, m,
                               ctx->st_v.p, xbar, 2.0, (float4 *)ctx->rec.p,
                               (double *)ctx->abar64.p, st));
    ctx->launches += 1;
    ForceArgs a = base_args(ctx, p, n, (const float4 *)ctx->rec.p);
    a.op = kEpiVjp;
    a.xbar = xbar;
    a.mbar = mbar;
    a.abar64 = ctx->abar64.p;
    a.mass = m;
    return launch_force(ctx, p, a, st);
}

nb_status nb_adjoint(nb_ctx *ctx, int64_t n, const void *m, int steps, const void *ckpt,
                     int ckpt_every, const void *xbar_T, const void *vbar_T, void *xbar0,
                     void *vbar0, void *mbar, void *stream) {
    if (!ctx) return NB_ERR_INVALID;
    if (n < 0 || steps < 0) return fail(ctx, NB_ERR_INVALID, "n < 0 or steps < 0");
    if (ctx->p.scheme != NB_SCHEME_PAPER)
        return fail(ctx, NB_ERR_UNSUPPORTED, "the adjoint is implemented for the paper scheme");
    if (n == 0) return NB_OK;
    if (ckpt_every <= 0 || steps % ckpt_every)
        return fail(ctx, NB_ERR_INVALID, "ckpt_every must be > 0 and divide steps");
    NB_CUDA(cudaSetDevice(ctx->device));
    const size_t es = esize(ctx);
    NB_TRY(check_ptr(ctx, m, es, "m", nullptr));
    NB_TRY(check_ptr(ctx, ckpt, es, "ckpt", nullptr));
    NB_TRY(check_ptr(ctx, xbar_T, es, "xbar_T", nullptr));
    NB_TRY(check_ptr(ctx, vbar_T, es, "vbar_T", nullptr));
    NB_TRY(check_ptr(ctx, xbar0, es, "xbar0", nullptr));
    NB_TRY(check_ptr(ctx, vbar0, es, "vbar0", nullptr));
    NB_TRY(check_ptr(ctx, mbar, es, "mbar", nullptr));
    cudaStream_t st = as_stream(stream);
    const size_t b3 = (size_t)n * 3 * es;
    NB_CUDA(cudaMemcpyAsync(xbar0, xbar_T, b3, cudaMemcpyDeviceToDevice, st));
    NB_CUDA(cudaMemcpyAsync(vbar0, vbar_T, b3, cudaMemcpyDeviceToDevice, st));
    NB_CUDA(cudaMemsetAsync(mbar, 0, (size_t)n * es, st));
    if (steps == 0) return NB_OK;

    Shape sf, sv;
    NB_TRY(choose_shape(ctx, 0, n, &sf, nullptr));
    NB_TRY(choose_shape(ctx, 1, n, &sv, nullptr));
    Plan pf, pv;
    NB_TRY(make_plan(ctx, sf, n, &pf));
    NB_TRY(make_plan(ctx, sv, n, &pv));
    // the reverse sweep (stream side) and the recompute of the previous
    // segment (stream side2) run concurrently, each with its own split scratch
    NB_TRY(ensure(ctx, ctx->part, pv.part_bytes));
    NB_TRY(ensure(ctx, ctx->counters, (size_t)pv.iblocks * 4, true));
    NB_TRY(ensure(ctx, ctx->part2, pf.part_bytes));
    NB_TRY(ensure(ctx, ctx->counters2, (size_t)pf.iblocks * 4, true));
    const int64_t npad = pf.npad;
    const int k = ckpt_every;
    const bool f64 = f64_state(ctx);
    NB_TRY(ensure(ctx, ctx->rec, (size_t)npad * 8 * pol_rec_f4(sv.pol)));
    for (int b = 0; b < 2; ++b) {
        NB_TRY(ensure(ctx, ctx->adj_traj[b], (size_t)(k + 1) * npad * 16));
        if (f64) NB_TRY(ensure(ctx, ctx->adj_traj64[b], (size_t)k * n * 48));
        NB_TRY(ensure(ctx, ctx->adj_x[b], b3));
        NB_TRY(ensure(ctx, ctx->adj_v[b], b3));
    }
    NB_TRY(ensure(ctx, ctx->abar64, (size_t)n * 24));
    const size_t slot_bytes = (size_t)n * 6 * es;
    const int nseg = steps / k;

    char key[512];
    snprintf(key, sizeof key, "adj|%lld|%p|%d|%p|%d|%p|%p|%p|%d.%d.%d.%d.%d|%d.%d.%d.%d.%d|%llu|%a|%a|%a",
             (long long)n, m, steps, ckpt, k, xbar0, vbar0, mbar, sf.pol, sf.nt, sf.r, sf.split,
             sf.jt, sv.pol, sv.nt, sv.r, sv.split, sv.jt, (unsigned long long)ctx->timeout_ns * 4 + ctx->debug,
             ctx->p.G, ctx->p.eps, ctx->p.dt);
    GraphEntry *g = graph_lookup(ctx, key);
    if (!g) {
        NB_CUDA(cudaStreamBeginCapture(ctx->side, cudaStreamCaptureModeThreadLocal));
        int64_t saved = ctx->launches;
        nb_status rs = NB_OK;
        std::vector<cudaEvent_t> events;
        auto new_event = [&](cudaEvent_t *e) -> bool {
            if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return false;
            events.push_back(*e);
            return true;
        };
        auto cuda_ok = [&](cudaError_t ce) -> bool {
            if (ce == cudaSuccess) return true;
            rs = fail(ctx, NB_ERR_CUDA, "adjoint capture: %s", cudaGetErrorString(ce));
            return false;
        };
        std::vector<cudaEvent_t> ev_rec(nseg), ev_swp(nseg);
        auto traj_slot = [&](int b, int t) {
            return (float4 *)ctx->adj_traj[b].p + (size_t)t * (npad / 2) * 2;
        };
        // Recompute segment `seg` from its checkpoint on side2, keeping the
        // packed positions of every step (and FP64 ones in the precision form).
        auto recompute = [&](int seg) {
            const int b = seg & 1;
            const char *slot = (const char *)ckpt + (size_t)seg * slot_bytes;
            if (!cuda_ok(launch_copy_ckpt_state(n, f64 ? 1 : 0, slot, ctx->adj_x[b].p,
                                                ctx->adj_v[b].p, ctx->side2)))
                return;
            ctx->launches += 1;
            rs = pack(ctx, n, npad, ctx->adj_x[b].p, nullptr, m, traj_slot(b, 0), nullptr, ctx->side2);
            for (int t = 0; rs == NB_OK && t < k - 1; ++t) {
                ForceArgs a = base_args(ctx, pf, n, traj_slot(b, t));
                a.part = (float4 *)ctx->part2.p;
                a.counters = (unsigned *)ctx->counters2.p;
                a.op = kEpiKickDrift;
                a.x = ctx->adj_x[b].p;
                a.v = ctx->adj_v[b].p;
                a.xm_next = traj_slot(b, t + 1);
                if (f64) a.ckpt = (char *)ctx->adj_traj64[b].p + (size_t)(t + 1) * n * 48;
                rs = launch_force(ctx, pf, a, ctx->side2);
            }
            if (rs == NB_OK && (!new_event(&ev_rec[seg]) || !cuda_ok(cudaEventRecord(ev_rec[seg], ctx->side2))))
                if (rs == NB_OK) rs = fail(ctx, NB_ERR_CUDA, "adjoint capture: event");
        };
        // Sweep segment `seg` backwards on side.
        auto sweep = [&](int seg) {
            const int b = seg & 1;
            if (!cuda_ok(cudaStreamWaitEvent(ctx->side, ev_rec[seg], 0))) return;
            const char *slot = (const char *)ckpt + (size_t)seg * slot_bytes;
            for (int t = k - 1; rs == NB_OK && t >= 0; --t) {
                const double *x64 = !f64 ? nullptr
                                    : t == 0 ? (const double *)slot
                                             : (const double *)((char *)ctx->adj_traj64[b].p + (size_t)t * n * 48);
                if (!cuda_ok(launch_adj_prepare(n, npad, f64 ? 1 : 0, traj_slot(b, t), x64, 6, m, vbar0,
                                                xbar0, ctx->p.dt, (float4 *)ctx->rec.p,
                                                (double *)ctx->abar64.p, ctx->side)))
                    return;
                ctx->launches += 1;
                ForceArgs a = base_args(ctx, pv, n, (const float4 *)ctx->rec.p);
                a.op = kEpiVjp;
                a.xbar = xbar0;
                a.mbar = mbar;
                a.abar64 = ctx->abar64.p;
                a.mass = m;
                rs = launch_force(ctx, pv, a, ctx->side);
            }
            if (rs == NB_OK && (!new_event(&ev_swp[seg]) || !cuda_ok(cudaEventRecord(ev_swp[seg], ctx->side))))
                if (rs == NB_OK) rs = fail(ctx, NB_ERR_CUDA, "adjoint capture: event");
        };
        cudaEvent_t fork;
        if (!new_event(&fork) || !cuda_ok(cudaEventRecord(fork, ctx->side)) ||
            !cuda_ok(cudaStreamWaitEvent(ctx->side2, fork, 0))) {
            if (rs == NB_OK) rs = fail(ctx, NB_ERR_CUDA, "adjoint capture: fork");
        }
        if (rs == NB_OK) recompute(nseg - 1);
        for (int seg = nseg - 1; rs == NB_OK && seg >= 0; --seg) {
            if (seg >= 1) {
                // segment seg-1 reuses the buffers of segment seg+1
                if (seg + 1 <= nseg - 1 && !cuda_ok(cudaStreamWaitEvent(ctx->side2, ev_swp[seg + 1], 0)))
                    break;
                recompute(seg - 1);
                if (rs != NB_OK) break;
            }
            sweep(seg);
        }
        cudaGraph_t graph = nullptr;
        cudaError_t ce = cudaStreamEndCapture(ctx->side, &graph);
        for (cudaEvent_t e : events) cudaEventDestroy(e);
        int64_t nodes = ctx->launches - saved;
        ctx->launches = saved;
        if (rs != NB_OK) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return rs;
        }
        if (ce != cudaSuccess) return fail(ctx, NB_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ce));
        cudaGraphExec_t ex = nullptr;
        ce = cudaGraphInstantiate(&ex, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return fail(ctx, NB_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
        graph_insert(ctx, key, ex, nodes);
        g = graph_lookup(ctx, key);
    }
    NB_CUDA(cudaGraphLaunch(g->exec, st));
    ctx->launches += g->nodes;
    return NB_OK;
}

int64_t nb_batched_max_n(void) { return batched_max_n(); }

nb_status nb_run_batched(nb_ctx *ctx, int nsys, const int64_t *offsets, void *x, void *v,
                         const void *m, int steps, void *stream) {
    if (!ctx) return NB_ERR_INVALID;
    if (nsys < 0 || steps < 0) return fail(ctx, NB_ERR_INVALID, "nsys < 0 or steps < 0");
    if (nsys == 0 || steps == 0) return NB_OK;
    if (f64_state(ctx)) return fail(ctx, NB_ERR_UNSUPPORTED, "batched runs are FP32 only");
    if (ctx->p.scheme != NB_SCHEME_PAPER)
        return fail(ctx, NB_ERR_UNSUPPORTED, "batched runs use the paper scheme");
    if (!offsets) return fail(ctx, NB_ERR_INVALID, "offsets is NULL");
    NB_CUDA(cudaSetDevice(ctx->device));
    std::vector<int64_t> off;
    NB_TRY(read_offsets(ctx, nsys, offsets, as_stream(stream), off));
    const int64_t total = off[nsys];
    if (total == 0) return NB_OK;
    if (steps > (1 << 20)) return fail(ctx, NB_ERR_INVALID, "at most 2^20 steps per batched call");
    NB_TRY(check_ptr(ctx, x, 4, "x", nullptr));
    NB_TRY(check_ptr(ctx, v, 4, "v", nullptr));
    NB_TRY(check_ptr(ctx, m, 4, "m", nullptr));
    cudaStream_t st = as_stream(stream);
    BatchPlan plan;
    auto tuned = ctx->batched_tuned.find(sizes_signature(off));
    if (tuned != ctx->batched_tuned.end()) {
        plan.nt = tuned->second.nt;
        plan.r = tuned->second.r;
        plan.jt = tuned->second.jt;
    }
    std::string why;
    if (!batched_plan(ctx->device, ctx->num_sms, off, plan, why))
        return fail(ctx, NB_ERR_CUDA, "batched plan: %s", why.c_str());
    NB_TRY(ensure(ctx, ctx->bat, plan.scratch_bytes, false));
    NB_CUDA(batched_upload(plan, ctx->bat.p, st));
    char key[512];
    snprintf(key, sizeof key, "bat|%d|%p|%p|%p|%d|%lld|%llx|%llu|%a|%a|%a", nsys, x, v, m, steps,
             (long long)total, (unsigned long long)plan.signature,
             (unsigned long long)ctx->timeout_ns, ctx->p.G, ctx->p.eps, ctx->p.dt);
    GraphEntry *g = graph_lookup(ctx, key);
    if (!g) {
        NB_CUDA(cudaStreamBeginCapture(ctx->side, cudaStreamCaptureModeThreadLocal));
        cudaError_t ce = batched_enqueue(plan, ctx->bat.p, (float *)x, (float *)v, (const float *)m,
                                         steps, (float)(ctx->p.eps * ctx->p.eps), (float)ctx->p.G,
                                         (float)ctx->p.dt, ctx->err_word, ctx->timeout_ns, ctx->side);
        cudaGraph_t graph = nullptr;
        cudaError_t ce2 = cudaStreamEndCapture(ctx->side, &graph);
        if (ce != cudaSuccess || ce2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return fail(ctx, NB_ERR_CUDA, "batched capture: %s",
                        cudaGetErrorString(ce != cudaSuccess ? ce : ce2));
        }
        cudaGraphExec_t ex = nullptr;
        ce = cudaGraphInstantiate(&ex, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return fail(ctx, NB_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
        graph_insert(ctx, key, ex, plan.launches);
        g = graph_lookup(ctx, key);
    }
    NB_CUDA(cudaGraphLaunch(g->exec, st));
    ctx->launches += g->nodes;
    return NB_OK;
}

nb_status nb_autotune_batched(nb_ctx *ctx, int nsys, const int64_t *offsets) {
    if (!ctx) return NB_ERR_INVALID;
    if (nsys <= 0 || !offsets) return fail(ctx, NB_ERR_INVALID, "nsys must be > 0, offsets non-NULL");
    NB_CUDA(cudaSetDevice(ctx->device));
    std::vector<int64_t> off;
    NB_TRY(read_offsets(ctx, nsys, offsets, ctx->side, off));
    const int64_t total = off[nsys];
    if (total == 0) return NB_OK;
    NB_TRY(ensure(ctx, ctx->tune[1], (size_t)total * 12));
    NB_TRY(ensure(ctx, ctx->tune[2], (size_t)total * 12));
    NB_TRY(ensure(ctx, ctx->tune[3], (size_t)total * 4));
    cudaStream_t st = ctx->side;
    EventPair ev;
    NB_CUDA(ev.create());
    cudaEvent_t e0 = ev.e0, e1 = ev.e1;
    const int probe_steps = 4;
    float best_ms = 1e30f;
    BatchPlan best;
    for (int r : {1, 2, 4}) {
        for (int jt : {64, 128}) {
            BatchPlan plan;
            plan.r = r;
            plan.jt = jt;
            std::string why;
            if (!batched_plan(ctx->device, ctx->num_sms, off, plan, why)) continue;
            NB_TRY(ensure(ctx, ctx->bat, plan.scratch_bytes, false));
            NB_CUDA(batched_upload(plan, ctx->bat.p, st));
            float *x = (float *)ctx->tune[1].p, *v = (float *)ctx->tune[2].p, *m = (float *)ctx->tune[3].p;
            NB_CUDA(batched_fill_synthetic(plan, ctx->bat.p, x, v, m, st));
            const float eps2 = (float)(ctx->p.eps * ctx->p.eps);
            NB_CUDA(batched_enqueue(plan, ctx->bat.p, x, v, m, 1, eps2, (float)ctx->p.G,
                                    (float)ctx->p.dt, ctx->err_word, ctx->timeout_ns, st));
            NB_CUDA(cudaEventRecord(e0, st));
            NB_CUDA(batched_enqueue(plan, ctx->bat.p, x, v, m, probe_steps, eps2, (float)ctx->p.G,
                                    (float)ctx->p.dt, ctx->err_word, ctx->timeout_ns, st));
            NB_CUDA(cudaEventRecord(e1, st));
            NB_CUDA(cudaEventSynchronize(e1));
            ctx->launches += 6;
            float ms = 0.f;
            NB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best_ms) {
                best_ms = ms;
                best = plan;
            }
        }
    }
    NB_TRY(sync_and_check(ctx, st));
    if (best_ms >= 1e30f) return fail(ctx, NB_ERR_CUDA, "no batched shape could be planned");
    ctx->batched_tuned[sizes_signature(off)] = best;
    clear_graphs(ctx);
    return NB_OK;
}

nb_status nb_get_batched_config(nb_ctx *ctx, int nsys, const int64_t *offsets, int *out6) {
    if (!ctx || !out6) return NB_ERR_INVALID;
    if (nsys <= 0 || !offsets) return fail(ctx, NB_ERR_INVALID, "nsys must be > 0, offsets non-NULL");
    NB_CUDA(cudaSetDevice(ctx->device));
    std::vector<int64_t> off;
    NB_TRY(read_offsets(ctx, nsys, offsets, ctx->side, off));
    BatchPlan plan;
    auto tuned = ctx->batched_tuned.find(sizes_signature(off));
    const bool from_tune = tuned != ctx->batched_tuned.end();
    if (from_tune) {
        plan.r = tuned->second.r;
        plan.jt = tuned->second.jt;
    }
    std::string why;
    if (!batched_plan(ctx->device, ctx->num_sms, off, plan, why))
        return fail(ctx, NB_ERR_CUDA, "batched plan: %s", why.c_str());
    out6[0] = plan.nt;
    out6[1] = plan.r;
    out6[2] = plan.jt;
    out6[3] = plan.items_per_step;
    out6[4] = plan.ncta;
    out6[5] = from_tune ? 1 : 0;
    return NB_OK;
}

nb_status nb_autotune(nb_ctx *ctx, int64_t n, int mode) {
    if (!ctx) return NB_ERR_INVALID;
    if (n <= 0) return fail(ctx, NB_ERR_INVALID, "n must be > 0");
    if (mode != 0 && mode != 1) return fail(ctx, NB_ERR_INVALID, "mode must be 0 or 1");
    NB_CUDA(cudaSetDevice(ctx->device));
    std::vector<int> pols;
    if (mode == 0) {
        if (f64_state(ctx)) pols = {kPolComp};
        else pols = {kPolF32x2, kPolScalar};
    } else {
        pols = {f64_state(ctx) ? kPolVjpComp : kPolVjp};
    }
    const int64_t npad = round_up(n, kPadBodies);
    const size_t es = esize(ctx);
    NB_TRY(ensure(ctx, ctx->tune[0], (size_t)npad * 40));          // records
    NB_TRY(ensure(ctx, ctx->tune[1], (size_t)n * 3 * 8, true));    // out / xbar
    NB_TRY(ensure(ctx, ctx->tune[2], (size_t)n * 8, true));        // mbar
    NB_TRY(ensure(ctx, ctx->tune[3], (size_t)n * 8, true));        // mass
    NB_TRY(ensure(ctx, ctx->tune[4], (size_t)n * 3 * 8, true));    // abar64
    (void)es;
    cudaStream_t st = ctx->side;
    EventPair ev;
    NB_CUDA(ev.create());
    cudaEvent_t e0 = ev.e0, e1 = ev.e1;
    auto time_shape = [&](const Shape &s, float *ms) -> nb_status {
        Plan p;
        NB_TRY(make_plan(ctx, s, n, &p));
        if (p.part_bytes > ((size_t)1 << 31)) { *ms = 1e30f; return NB_OK; }
        NB_TRY(plan_scratch(ctx, p));
        NB_CUDA(launch_fill_synthetic(n, npad, (float4 *)ctx->tune[0].p, pol_rec_f4(s.pol), st));
        ForceArgs a = base_args(ctx, p, n, (const float4 *)ctx->tune[0].p);
        a.op = mode == 0 ? kEpiAccel : kEpiVjp;
        a.out = ctx->tune[1].p;
        a.xbar = ctx->tune[1].p;
        a.mbar = ctx->tune[2].p;
        a.mass = ctx->tune[3].p;
        a.abar64 = ctx->tune[4].p;
        NB_CUDA(p.e->launch(s.jt, a, st));  // warm-up
        float best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            NB_CUDA(cudaEventRecord(e0, st));
            NB_CUDA(p.e->launch(s.jt, a, st));
            NB_CUDA(cudaEventRecord(e1, st));
            NB_CUDA(cudaEventSynchronize(e1));
            float t = 0;
            NB_CUDA(cudaEventElapsedTime(&t, e0, e1));
            best = std::min(best, t);
        }
        *ms = best;
        return NB_OK;
    };
    TuneEntry best{};
    float best_ms = 1e30f;
    for (int pol : pols) {
        int cnt = 0;
        const ForceEntry *tab = force_table(pol, &cnt);
        for (int k = 0; k < cnt; ++k) {
            const int jt = npad >= 4096 ? 128 : 64;
            Shape s = finish_shape(ctx, pol, tab[k].nt, tab[k].r, jt, 0, n);
            float ms;
            NB_TRY(time_shape(s, &ms));
            // a later candidate must win by more than 1 % (keeps the choice
            // stable against timing noise)
            if (ms < best_ms * 0.99f) { best_ms = ms; best = TuneEntry{pol, tab[k].nt, tab[k].r, jt, 0}; }
        }
    }
    // refine the tile and split around the winner
    const TuneEntry base = best;
    for (int jt : {64, 128, 256}) {
        for (int sm : {-1, 0, 1}) {
            if (jt == base.jt && sm == 0) continue;
            if (npad % jt) continue;
            Shape s = finish_shape(ctx, base.pol, base.nt, base.r, jt, sm, n);
            float ms;
            NB_TRY(time_shape(s, &ms));
            if (ms < best_ms * 0.99f) { best_ms = ms; best = TuneEntry{base.pol, base.nt, base.r, jt, sm}; }
        }
    }
    NB_TRY(sync_and_check(ctx, st));
    ctx->tuned[tune_key(ctx, mode, n)] = best;
    clear_graphs(ctx);
    save_tune_file(ctx);
    return NB_OK;
}

nb_status nb_get_config(nb_ctx *ctx, int64_t n, int mode, int *out5) {
    if (!ctx || !out5) return NB_ERR_INVALID;
    if (mode < 0 || mode > 2) return fail(ctx, NB_ERR_INVALID, "mode must be 0, 1 or 2");
    Shape s;
    bool tuned = false;
    NB_TRY(choose_shape(ctx, mode, std::max<int64_t>(n, 1), &s, &tuned));
    out5[0] = s.nt;
    out5[1] = s.r;
    out5[2] = s.split;
    out5[3] = s.jt;
    out5[4] = tuned ? 1 : 0;
    return NB_OK;
}

nb_status nb_measure_peaks(nb_ctx *ctx, double *out3) {
    if (!ctx || !out3) return NB_ERR_INVALID;
    NB_CUDA(cudaSetDevice(ctx->device));
    NB_TRY(ensure(ctx, ctx->tune[5], 256));
    NB_CUDA(measure_peaks(ctx->num_sms * 8, (float *)ctx->tune[5].p, ctx->side, out3));
    ctx->launches += 6;
    return sync_and_check(ctx, ctx->side);
}

nb_status nb_sync(nb_ctx *ctx, void *stream) {
    if (!ctx) return NB_ERR_INVALID;
    NB_CUDA(cudaSetDevice(ctx->device));
    return sync_and_check(ctx, as_stream(stream));
}

int64_t nb_launch_count(const nb_ctx *ctx) { return ctx ? ctx->launches : 0; }

nb_status nb_debug_set(nb_ctx *ctx, int key, int64_t value) {
    if (!ctx) return NB_ERR_INVALID;
    if (key == NB_DBG_WAIT_TIMEOUT_NS) {
        if (value < 0) return fail(ctx, NB_ERR_INVALID, "timeout must be >= 0");
        ctx->timeout_ns = (uint64_t)value;
        return NB_OK;
    }
    if (key == NB_DBG_MATH_VARIANT) {
        if (value < 0 || value > 2) return fail(ctx, NB_ERR_INVALID, "math variant must be 0, 1 or 2");
        ctx->math = (int)value;
        clear_graphs(ctx);
        return NB_OK;
    }
    if (key == NB_DBG_STALL_PRODUCER) {
        if (value != 0 && value != 1) return fail(ctx, NB_ERR_INVALID, "value must be 0 or 1");
        ctx->debug = value ? (ctx->debug | kDbgStallProducer) : (ctx->debug & ~kDbgStallProducer);
        return NB_OK;
    }
    return fail(ctx, NB_ERR_INVALID, "unknown debug key %d", key);
}

}  // extern "C"
