// libnbody C-ABI: ensembles of independent systems in one persistent launch,
// and their tuner.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"

using namespace nb;
using namespace nb::detail;

namespace {

// The plan's preset fields for these sizes: the tuned or pinned entry, else
// the default shape, in FP32 in the pair-symmetric form when it needs less
// than 0.85 of the one-sided form's FP32 work (groups of 256 bodies waste
// little on systems of a few hundred bodies and more). Untuned, the
// precision form keeps the one-sided items: the pair-symmetric items sum up
// to 256 terms per FP32 partial against the one-sided tiles' 32 to 128
// (measured on 30 cube systems of 64 to 2048 bodies, eps = 0.01: 1.5e-11 in
// x after 4 steps in both forms); the tuner times both. Sizes whose partials
// would exceed kSymMaxPartBytes keep the one-sided items.
void preset_plan(nb_ctx *ctx, const std::vector<int64_t> &off, BatchPlan &plan) {
    plan.f64 = f64_state(ctx) ? 1 : 0;
    auto tuned = ctx->batched_tuned.find(sizes_signature(off));
    if (tuned != ctx->batched_tuned.end()) {
        plan.nt = tuned->second.nt;
        plan.r = tuned->second.r;
        plan.jt = tuned->second.jt;
        plan.origin = tuned->second.origin;
        plan.sym = tuned->second.sym;
        return;
    }
    plan.sym = !plan.f64 && batched_sym_work_ratio(off) < 0.85 && batched_sym_part_bytes(off) <= kSymMaxPartBytes
                   ? 1
                   : 0;
}

}  // namespace

extern "C" {

int64_t nb_batched_max_n(void) { return batched_max_n(); }

nb_status nb_run_batched(nb_ctx *ctx, int nsys, const int64_t *offsets, void *x, void *v,
                         const void *m, int steps, void *stream) {
    if (!ctx) return NB_ERR_INVALID;
    if (nsys < 0 || steps < 0) return fail(ctx, NB_ERR_INVALID, "nsys < 0 or steps < 0");
    if (nsys == 0 || steps == 0) return NB_OK;
    if (!offsets) return fail(ctx, NB_ERR_INVALID, "offsets is NULL");
    NB_CUDA(cudaSetDevice(ctx->device));
    std::vector<int64_t> off;
    NB_TRY(read_offsets(ctx, nsys, offsets, as_stream(stream), off));
    const int64_t total = off[nsys];
    if (total == 0) return NB_OK;
    if (steps > (1 << 20)) return fail(ctx, NB_ERR_INVALID, "at most 2^20 steps per batched call");
    const size_t es = esize(ctx);
    NB_TRY(check_ptr(ctx, x, es, "x", nullptr));
    NB_TRY(check_ptr(ctx, v, es, "v", nullptr));
    NB_TRY(check_ptr(ctx, m, es, "m", nullptr));
    cudaStream_t st = as_stream(stream);
    BatchPlan plan;
    preset_plan(ctx, off, plan);
    std::string why;
    if (!batched_plan(ctx->device, ctx->num_sms, off, plan, why))
        return fail(ctx, NB_ERR_CUDA, "batched plan: %s", why.c_str());
    NB_TRY(ensure(ctx, ctx->bat, plan.scratch_bytes, false));
    NB_CUDA(batched_upload(plan, ctx->bat.p, st));
    char key[512];
    const int kdk = ctx->p.scheme == NB_SCHEME_KDK ? 1 : 0;
    snprintf(key, sizeof key, "bat|%d|%p|%p|%p|%d|%d|%lld|%llx|%llu|%d|%a|%a|%a", nsys, x, v, m, steps,
             kdk, (long long)total, (unsigned long long)plan.signature,
             (unsigned long long)ctx->timeout_ns, ctx->debug, ctx->p.G, ctx->p.eps, ctx->p.dt);
    GraphEntry *g = graph_lookup(ctx, key);
    if (!g) {
        NB_CUDA(cudaStreamBeginCapture(ctx->side, cudaStreamCaptureModeThreadLocal));
        cudaError_t ce = batched_enqueue(plan, ctx->bat.p, x, v, m, steps, kdk,
                                         (float)(ctx->p.eps * ctx->p.eps), ctx->p.G, ctx->p.dt,
                                         ctx->err_word, ctx->timeout_ns,
                                         (ctx->debug & kDbgStallProducer) ? 1 : 0, ctx->side);
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
    const size_t es = esize(ctx);
    NB_TRY(ensure(ctx, ctx->tune[1], (size_t)total * 3 * es));
    NB_TRY(ensure(ctx, ctx->tune[2], (size_t)total * 3 * es));
    NB_TRY(ensure(ctx, ctx->tune[3], (size_t)total * es));
    cudaStream_t st = ctx->side;
    EventPair ev;
    NB_CUDA(ev.create());
    cudaEvent_t e0 = ev.e0, e1 = ev.e1;
    const int probe_steps = 4;
    float best_ms = 1e30f;
    BatchPlan best;
    // (threads, largest R) of the one-sided form at two j-tiles, then the
    // pair-symmetric form (shape {0, 0}: its own)
    static const int kShapes[][2] = {{128, 1}, {128, 2}, {128, 4}, {128, 8}, {256, 1}, {256, 2},
                                     {256, 4}, {256, 8}, {512, 1}, {512, 2}, {0, 0}};
    for (const auto &shape : kShapes) {
        for (int jt : {64, 128}) {
            if (f64_state(ctx) && shape[1] > 4) continue;  // the precision form: R <= 4
            if (shape[0] == 0 && jt != 64) continue;  // the pair-symmetric form: its own shape
            BatchPlan plan;
            plan.f64 = f64_state(ctx) ? 1 : 0;
            plan.nt = shape[0];
            plan.r = shape[1];
            plan.jt = jt;
            plan.sym = shape[0] == 0 ? 1 : 0;
            std::string why;
            if (!batched_plan(ctx->device, ctx->num_sms, off, plan, why)) continue;
            NB_TRY(ensure(ctx, ctx->bat, plan.scratch_bytes, false));
            NB_CUDA(batched_upload(plan, ctx->bat.p, st));
            void *x = ctx->tune[1].p, *v = ctx->tune[2].p, *m = ctx->tune[3].p;
            NB_CUDA(batched_fill_synthetic(plan, ctx->bat.p, x, v, m, st));
            const float eps2 = (float)(ctx->p.eps * ctx->p.eps);
            NB_CUDA(batched_enqueue(plan, ctx->bat.p, x, v, m, 1, 0, eps2, ctx->p.G,
                                    ctx->p.dt, ctx->err_word, ctx->timeout_ns, 0, st));
            NB_CUDA(cudaEventRecord(e0, st));
            NB_CUDA(batched_enqueue(plan, ctx->bat.p, x, v, m, probe_steps, 0, eps2, ctx->p.G,
                                    ctx->p.dt, ctx->err_word, ctx->timeout_ns, 0, st));
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
    best.origin = 1;
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
    preset_plan(ctx, off, plan);
    std::string why;
    if (!batched_plan(ctx->device, ctx->num_sms, off, plan, why))
        return fail(ctx, NB_ERR_CUDA, "batched plan: %s", why.c_str());
    out6[0] = plan.nt;
    out6[1] = plan.r;
    out6[2] = plan.jt;
    out6[3] = plan.items_per_step;
    out6[4] = plan.ncta;
    out6[5] = plan.origin;
    return NB_OK;
}

nb_status nb_set_batched_config(nb_ctx *ctx, int nsys, const int64_t *offsets, int threads,
                                int bodies_per_thread, int jtile) {
    if (!ctx) return NB_ERR_INVALID;
    if (nsys <= 0 || !offsets) return fail(ctx, NB_ERR_INVALID, "nsys must be > 0, offsets non-NULL");
    NB_CUDA(cudaSetDevice(ctx->device));
    std::vector<int64_t> off;
    NB_TRY(read_offsets(ctx, nsys, offsets, ctx->side, off));
    const uint64_t sig = sizes_signature(off);
    if (threads == 0 && bodies_per_thread == 0 && jtile == 0) {
        ctx->batched_tuned.erase(sig);
        clear_graphs(ctx);
        return NB_OK;
    }
    const bool r_any = bodies_per_thread == 1 || bodies_per_thread == 2 || bodies_per_thread == 4 ||
                       bodies_per_thread == 8;
    const bool shape_ok = ((threads == 128 || threads == 256) && r_any) ||
                          (threads == 512 && (bodies_per_thread == 1 || bodies_per_thread == 2));
    if (!shape_ok)
        return fail(ctx, NB_ERR_INVALID,
                    "threads x bodies_per_thread must be 128 or 256 x {1,2,4,8}, or 512 x {1,2}");
    if (jtile != 32 && jtile != 64 && jtile != 128 && jtile != 256)
        return fail(ctx, NB_ERR_INVALID, "jtile must be 32, 64, 128 or 256");
    if (f64_state(ctx) && bodies_per_thread > 4)
        return fail(ctx, NB_ERR_INVALID, "the precision form takes at most 4 bodies per thread");
    BatchPlan plan;
    plan.f64 = f64_state(ctx) ? 1 : 0;
    plan.nt = threads;
    plan.r = bodies_per_thread;
    plan.jt = jtile;
    plan.sym = 0;
    std::string why;
    if (!batched_plan(ctx->device, ctx->num_sms, off, plan, why))
        return fail(ctx, NB_ERR_CUDA, "batched plan: %s", why.c_str());
    plan.origin = 2;
    ctx->batched_tuned[sig] = plan;
    clear_graphs(ctx);
    return NB_OK;
}

nb_status nb_set_batched_form(nb_ctx *ctx, int nsys, const int64_t *offsets, int form) {
    if (!ctx) return NB_ERR_INVALID;
    if (nsys <= 0 || !offsets) return fail(ctx, NB_ERR_INVALID, "nsys must be > 0, offsets non-NULL");
    if (form < 0 || form > 2) return fail(ctx, NB_ERR_INVALID, "form must be 0, 1 or 2");
    NB_CUDA(cudaSetDevice(ctx->device));
    std::vector<int64_t> off;
    NB_TRY(read_offsets(ctx, nsys, offsets, ctx->side, off));
    const uint64_t sig = sizes_signature(off);
    clear_graphs(ctx);
    if (form == 0) {
        ctx->batched_tuned.erase(sig);
        return NB_OK;
    }
    BatchPlan plan;
    plan.f64 = f64_state(ctx) ? 1 : 0;
    auto it = ctx->batched_tuned.find(sig);
    if (form == 1 && it != ctx->batched_tuned.end() && !it->second.sym) {  // keep a one-sided shape
        plan.nt = it->second.nt;
        plan.r = it->second.r;
        plan.jt = it->second.jt;
    }
    plan.sym = form == 2 ? 1 : 0;
    std::string why;
    if (!batched_plan(ctx->device, ctx->num_sms, off, plan, why))
        return fail(ctx, NB_ERR_CUDA, "batched plan: %s", why.c_str());
    plan.origin = 2;
    ctx->batched_tuned[sig] = plan;
    return NB_OK;
}

nb_status nb_get_batched_form(nb_ctx *ctx, int nsys, const int64_t *offsets, int *form) {
    if (!ctx || !form) return NB_ERR_INVALID;
    if (nsys <= 0 || !offsets) return fail(ctx, NB_ERR_INVALID, "nsys must be > 0, offsets non-NULL");
    NB_CUDA(cudaSetDevice(ctx->device));
    std::vector<int64_t> off;
    NB_TRY(read_offsets(ctx, nsys, offsets, ctx->side, off));
    BatchPlan plan;
    preset_plan(ctx, off, plan);
    *form = plan.sym ? 2 : 1;
    return NB_OK;
}

}  // extern "C"
