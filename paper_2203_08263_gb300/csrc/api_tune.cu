// libnbody C-ABI: the launch-shape tuner and shape queries.
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

extern "C" {

nb_status nb_autotune(nb_ctx *ctx, int64_t n, int mode) {
    if (!ctx) return NB_ERR_INVALID;
    if (n <= 0) return fail(ctx, NB_ERR_INVALID, "n must be > 0");
    if (mode != 0 && mode != 1) return fail(ctx, NB_ERR_INVALID, "mode must be 0 or 1");
    NB_CUDA(cudaSetDevice(ctx->device));
    std::vector<int> pols;
    if (mode == 0) {
        if (f64_state(ctx)) pols = n >= 8192 ? std::vector<int>{kPolComp, kPolSymComp} : std::vector<int>{kPolComp};
        else if (ctx->math == 0 && n >= 8192) pols = {kPolF32x2, kPolScalar, kPolSym};
        else pols = {kPolF32x2, kPolScalar};
    } else if (f64_state(ctx)) {
        pols = n >= 2048 ? std::vector<int>{kPolVjpComp, kPolVjpSymComp} : std::vector<int>{kPolVjpComp};
    } else {
        pols = n >= 2048 ? std::vector<int>{kPolVjp, kPolVjpSym} : std::vector<int>{kPolVjp};
    }
    const int64_t npad = round_up(n, kPadBodies);
    const size_t es = esize(ctx);
    // records, up to the pair-symmetric policy's padding to 1024 bodies
    NB_TRY(ensure(ctx, ctx->tune[0], (size_t)round_up(n, 1024) * 40));
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
        const nb_status ps = make_plan(ctx, s, n, &p);
        if (ps == NB_ERR_UNSUPPORTED && pol_is_sym(s.pol)) {  // partials above the cap: not a candidate
            ctx->err.clear();
            *ms = 1e30f;
            return NB_OK;
        }
        NB_TRY(ps);
        const size_t cap = pol_is_sym(s.pol) ? kSymMaxPartBytes : ((size_t)1 << 31);
        if (p.part_bytes > cap) { *ms = 1e30f; return NB_OK; }
        NB_TRY(plan_scratch(ctx, p));
        NB_CUDA(launch_fill_synthetic(n, p.npad, (float4 *)ctx->tune[0].p, pol_rec_f4(s.pol), st));
        ForceArgs a = base_args(ctx, p, n, (const float4 *)ctx->tune[0].p);
        a.op = mode == 0 ? kEpiAccel : kEpiVjp;
        a.out = ctx->tune[1].p;
        a.xbar = ctx->tune[1].p;
        a.mbar = ctx->tune[2].p;
        a.mass = ctx->tune[3].p;
        a.abar64 = ctx->tune[4].p;
        // warm-up, and a first estimate that sets how many back-to-back
        // launches one timing covers (about 1 ms: a launch of a few
        // microseconds alone is within the events' jitter)
        NB_CUDA(cudaEventRecord(e0, st));
        NB_CUDA(p.e->launch(s.jt, a, st));
        NB_CUDA(cudaEventRecord(e1, st));
        NB_CUDA(cudaEventSynchronize(e1));
        float t1 = 0;
        NB_CUDA(cudaEventElapsedTime(&t1, e0, e1));
        const int batch = std::max(1, std::min(64, (int)(1.0f / std::max(t1, 1e-3f))));
        float best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            NB_CUDA(cudaEventRecord(e0, st));
            for (int b = 0; b < batch; ++b) NB_CUDA(p.e->launch(s.jt, a, st));
            NB_CUDA(cudaEventRecord(e1, st));
            NB_CUDA(cudaEventSynchronize(e1));
            float t = 0;
            NB_CUDA(cudaEventElapsedTime(&t, e0, e1));
            best = std::min(best, t / batch);
        }
        *ms = best;
        return NB_OK;
    };
    TuneEntry best{};
    float best_ms = 1e30f;
    for (int pol : pols) {
        int cnt = 0;
        const ForceEntry *tab = force_table(pol, &cnt);
        // pair-symmetric blocks largest first: a smaller block (more block
        // pairs, twice the partials) must then win by the margin below
        // (measured at N = 262144: 1024-body blocks 0.7 % faster than 512,
        // inside the margin when 512 came first)
        for (int kk = 0; kk < cnt; ++kk) {
            const int k = pol_is_sym(pol) ? cnt - 1 - kk : kk;
            const int jt = npad >= 4096 ? 128 : 64;
            Shape s = finish_shape(ctx, pol, tab[k].nt, tab[k].r, jt, 0, n);
            float ms;
            NB_TRY(time_shape(s, &ms));
            // a later candidate must win by more than 1 % (keeps the choice
            // stable against timing noise)
            if (ms < best_ms * 0.99f) { best_ms = ms; best = TuneEntry{pol, tab[k].nt, tab[k].r, jt, 0}; }
        }
    }
    // refine the tile and split around the winner (the pair-symmetric
    // policy has neither: its table entries are its shapes)
    const TuneEntry base = best;
    for (int jt : {64, 128, 256}) {
        if (pol_is_sym(base.pol)) break;
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
    // nb_run's paths for small systems: the graph of force launches (with the
    // shape just chosen), the one-cluster kernel and its grid form, 20 steps
    // each on zeroed state (timing does not depend on the values)
    const bool f64 = f64_state(ctx);
    const bool fused = mode == 0 && (f64 || ctx->math == 0);
    const int cluster = fused && n <= kClusterMaxN ? cluster_run_size(n, f64) : 0;
    const int grid = fused ? grid_run_ctas(n, ctx->num_sms, 8) : 0;
    if (cluster || grid) {
        void *x = ctx->tune[1].p, *v = ctx->tune[4].p, *m = ctx->tune[3].p;
        NB_CUDA(cudaMemsetAsync(x, 0, (size_t)n * 3 * esize(ctx), st));
        NB_CUDA(cudaMemsetAsync(v, 0, (size_t)n * 3 * esize(ctx), st));
        NB_CUDA(cudaMemsetAsync(m, 0, (size_t)n * esize(ctx), st));
        const int steps = 20;
        const int saved_path = ctx->run_path;
        const std::string run_key = tune_key(ctx, mode, n) + "|run";
        // candidates: graph, one cluster, and the grid form at slices of at
        // least 8, 16, 32 and 64 bodies (distinct CTA counts only; 64 takes the
        // two-bodies-per-lane form); the grid form
        // runs with the CTA count of a provisional "|run" entry
        struct Cand { int path, size; };
        std::vector<Cand> cands = {{1, 0}};
        if (cluster) cands.push_back({2, cluster});
        for (int ms : {8, 16, 32, 64}) {
            const int g = grid_run_ctas(n, ctx->num_sms, ms);
            bool seen = false;
            for (const Cand &c : cands) seen = seen || (c.path == 3 && c.size == g);
            if (g && !seen) cands.push_back({3, g});
        }
        const auto saved_entry = ctx->tuned.find(run_key);
        const bool had_entry = saved_entry != ctx->tuned.end();
        const TuneEntry old_entry = had_entry ? saved_entry->second : TuneEntry{};
        float best_ms = 1e30f;
        Cand best_c = {1, 0};
        nb_status rs = NB_OK;
        for (const Cand &cd : cands) {
            if (rs != NB_OK) break;
            ctx->run_path = cd.path == 3 ? 0 : cd.path;
            if (cd.path == 3) ctx->tuned[run_key] = TuneEntry{2, cd.size, 0, 0, 0};
            float ms = 1e30f;
            rs = run_device(ctx, n, x, v, m, steps, nullptr, 0, st);  // warm-up (and graph capture)
            for (int rep = 0; rs == NB_OK && rep < 3; ++rep) {
                if (cudaEventRecord(e0, st) != cudaSuccess) { rs = NB_ERR_CUDA; break; }
                rs = run_device(ctx, n, x, v, m, steps, nullptr, 0, st);
                if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                    rs = NB_ERR_CUDA;
                    break;
                }
                float t = 0;
                cudaEventElapsedTime(&t, e0, e1);
                ms = std::min(ms, t);
            }
            if (ms < best_ms) {
                best_ms = ms;
                best_c = cd;
            }
        }
        ctx->run_path = saved_path;
        if (had_entry) ctx->tuned[run_key] = old_entry;
        else ctx->tuned.erase(run_key);
        NB_TRY(rs);
        NB_TRY(sync_and_check(ctx, st));
        // stored: 0 graph, 1 one cluster, 2 grid; the cluster size or the grid's CTAs
        ctx->tuned[run_key] = TuneEntry{best_c.path - 1, best_c.size, 0, 0, 0};
        clear_graphs(ctx);
    }
    save_tune_file(ctx);
    return NB_OK;
}

nb_status nb_get_run_path(nb_ctx *ctx, int64_t n, int *out3) {
    if (!ctx || !out3) return NB_ERR_INVALID;
    if (n <= 0) return fail(ctx, NB_ERR_INVALID, "n must be > 0");
    NB_CUDA(cudaSetDevice(ctx->device));
    int path = 1, size = 0;
    NB_TRY(choose_run_path(ctx, n, &path, &size));
    out3[0] = path;
    out3[1] = size;
    out3[2] = ctx->run_path == 0 && ctx->tuned.count(tune_key(ctx, 0, n) + "|run") ? 1 : 0;
    return NB_OK;
}

nb_status nb_get_form(nb_ctx *ctx, int64_t n, int mode, int *form) {
    if (!ctx || !form) return NB_ERR_INVALID;
    if (mode < 0 || mode > 2) return fail(ctx, NB_ERR_INVALID, "mode must be 0, 1 or 2");
    Shape s;
    NB_TRY(choose_shape(ctx, mode, std::max<int64_t>(n, 1), &s, nullptr));
    *form = s.pol;  // the policy ids are the nb_form values
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

}  // extern "C"
