// Host-side machinery of a libnbody context: scratch memory, launch-shape
// choice, force launches, the CUDA-graph cache and the tuning table.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "ctx.h"

namespace nb {
const ForceEntry *table_f32x2(int *count);
const ForceEntry *table_scalar(int *count);
const ForceEntry *table_comp(int *count);
const ForceEntry *table_pot(int *count);
const ForceEntry *table_vjp(int *count);
const ForceEntry *table_vjp_comp(int *count);
const ForceEntry *table_div(int *count);
const ForceEntry *table_pow(int *count);
const ForceEntry *table_sym(int *count);
const ForceEntry *table_vjp_sym(int *count);
const ForceEntry *table_comp_sym(int *count);
const ForceEntry *table_vjp_comp_sym(int *count);

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
        case kPolSym: return table_sym(count);
        case kPolVjpSym: return table_vjp_sym(count);
        case kPolSymComp: return table_comp_sym(count);
        case kPolVjpSymComp: return table_vjp_comp_sym(count);
        default: *count = 0; return nullptr;
    }
}
int pol_rec_f4(int pol) {
    if (pol == kPolVjp || pol == kPolVjpSym) return 4;
    return (pol == kPolVjpComp || pol == kPolVjpSymComp) ? 5 : 2;
}
int pol_part_f4(int pol) {
    switch (pol) {
        case kPolComp: return 2;
        case kPolVjp: return 2;
        case kPolVjpComp: return 4;
        default: return 1;
    }
}
}  // namespace nb

namespace nb {
namespace detail {

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



void clear_graphs(nb_ctx *ctx) {
    for (auto &kv : ctx->graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    ctx->graphs.clear();
}

// Grow a scratch buffer. Growth waits for the device and drops cached graphs
// (they may reference the old allocation), so it must not happen during a
// stream capture.
nb_status ensure(nb_ctx *ctx, DevBuf &b, size_t bytes, bool zero) {
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


nb_status validate_params(nb_ctx *ctx, double G, double eps, double dt) {
    if (!std::isfinite(G) || !std::isfinite(eps) || !std::isfinite(dt))
        return fail(ctx, NB_ERR_INVALID, "G, eps and dt must be finite");
    if (!(eps > 0.0) || !((float)(eps * eps) >= 1.17549435e-38f))
        return fail(ctx, NB_ERR_INVALID,
                    "eps must be > 0 with eps^2 a normal FP32 number (the j = i term is 0/0 otherwise)");
    return NB_OK;
}

// ----------------------------------------------------------- shape choice


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
    if (pol_is_sym(pol)) return Shape{pol, nt, r, 1, nt * r};  // no split: items are block pairs
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
Shape heuristic_shape(const nb_ctx *ctx, int mode, int64_t n, bool allow_sym) {
    const int pol = mode_pol(ctx, mode);
    int nt = 128, r = 1, jt = 64;
    if ((pol == kPolF32x2 || pol == kPolComp) && allow_sym && n >= 16384) {
        // each unordered pair once, blocks of 1024 bodies from 2^17 up (enough
        // block pairs to fill the GPU), 512 below, and below 2^15 blocks of
        // 256 whose block pairs two warps share (64 threads x kSymR / 2: more
        // resident warps where the block pairs are few)
        const int sp = pol == kPolComp ? kPolSymComp : kPolSym;
        if (n < 32768) return Shape{sp, 64, kSymR / 2, 1, 64 * (kSymR / 2)};
        const int snt = n >= 131072 ? 128 : 64;
        const int64_t b = (int64_t)snt * kSymR;
        return Shape{sp, snt, kSymR, 1, (int)b};
    }
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
    } else if ((pol == kPolVjp || pol == kPolVjpComp) && allow_sym && n >= 8192) {
        // each unordered pair once: blocks of 256 bodies below 2^16, 512 from there
        const int snt = n >= 65536 ? 128 : 64;
        const int64_t b = (int64_t)snt * kSymVjpR;
        return Shape{pol == kPolVjp ? kPolVjpSym : kPolVjpSymComp, snt, kSymVjpR, 1, (int)b};
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
        Shape h = heuristic_shape(ctx, mode, n, false);  // overrides address the one-sided kernels
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
    if ((pol == kPolF32x2 || pol == kPolComp) && ctx->form_pin > 1) {
        *out = Shape{pol == kPolComp ? kPolSymComp : kPolSym, ctx->form_pin / kSymR, kSymR, 1,
                     ctx->form_pin};
        return NB_OK;
    }
    if ((pol == kPolVjp || pol == kPolVjpComp) && ctx->vjp_form_pin > 1) {
        *out = Shape{pol == kPolVjp ? kPolVjpSym : kPolVjpSymComp, ctx->vjp_form_pin / kSymVjpR, kSymVjpR, 1,
                     ctx->vjp_form_pin};
        return NB_OK;
    }
    const int pin = mode == 1 ? ctx->vjp_form_pin : ctx->form_pin;
    auto it = ctx->tuned.find(tune_key(ctx, mode, n));
    if (mode != 2 && ctx->math == 0 && it != ctx->tuned.end() &&
        find_entry(it->second.pol, it->second.nt, it->second.r) &&
        !(pin == 1 && pol_is_sym(it->second.pol))) {
        const TuneEntry &t = it->second;
        *out = finish_shape(ctx, t.pol, t.nt, t.r, t.jt, t.split_mode, n);
        if (from_tune) *from_tune = true;
        return NB_OK;
    }
    *out = heuristic_shape(ctx, mode, n, pin != 1);
    return NB_OK;
}

// ------------------------------------------------------------ force launch


nb_status make_plan(nb_ctx *ctx, const Shape &s, int64_t n, Plan *p) {
    p->s = s;
    p->e = find_entry(s.pol, s.nt, s.r);
    if (!p->e) return fail(ctx, NB_ERR_UNSUPPORTED, "no kernel for shape");
    if (pol_is_sym(s.pol)) {
        // blocks of nt x r bodies; partials P[nb][sums][npad] (csrc/k_sym.cu)
        const int64_t b = (int64_t)s.nt * s.r;
        p->npad = round_up(std::max<int64_t>(n, 1), b);
        p->iblocks = (int)(p->npad / b);
        p->ntiles = p->iblocks;
        const int na = sym_sums(s.pol);
        p->part_bytes = (size_t)p->iblocks * na * (size_t)p->npad * 4;
        // above kSymTileAbove bytes of partials for one launch, launches by
        // tiles of w x w block pairs: two tile buffers (within
        // kSymTileBufBytes, about four waves of CTAs per tile) and the
        // running sums [2][sums][npad]
        int w = ctx->sym_tile > 0 ? ctx->sym_tile : 0;
        if (ctx->sym_tile == 0 && p->part_bytes > kSymTileAbove) {
            const int64_t slots = (int64_t)std::max(p->e->occupancy((int)b), 1) * ctx->num_sms;
            const double slot_bytes = 2.0 * na * (double)b * 4;
            const int w_waves = (int)std::sqrt(4.0 * (double)slots);
            const int w_buf = (int)std::sqrt((double)kSymTileBufBytes / (2.0 * slot_bytes));
            w = std::max(1, std::min(w_waves, w_buf));
        }
        if (w > 0 && w < p->iblocks) {
            p->tile_w = w;
            p->ntile = sym_tile_count(p->iblocks, w);
            p->part_bytes = 2 * (size_t)w * w * 2 * na * (size_t)b * 4 + 2 * (size_t)na * p->npad * 4;
        }
        return NB_OK;
    }
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
    a.tile_w = p.tile_w;
    a.ntile = p.ntile;
    return a;
}

nb_status launch_force(nb_ctx *ctx, const Plan &p, const ForceArgs &a, cudaStream_t st) {
    NB_CUDA(p.e->launch(p.s.jt, a, st));
    // the pair kernel (one per tile) and its fixed-order sum with the epilogue
    ctx->launches += pol_is_sym(p.s.pol) ? (p.ntile > 0 ? p.ntile + 1 : 2) : 1;
    return NB_OK;
}

nb_status pack(nb_ctx *ctx, int64_t n, int64_t npad, const void *x, const void *v, const void *m,
               float4 *xm, void *ckpt0, cudaStream_t st, PadTargets pads) {
    if (f64_state(ctx))
        NB_CUDA(launch_pack_f64(n, npad, (const double *)x, (const double *)v, (const double *)m,
                                xm, (double *)ckpt0, pads, st));
    else
        NB_CUDA(launch_pack_f32(n, npad, (const float *)x, (const float *)v, (const float *)m, xm,
                                (float *)ckpt0, pads, st));
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

nb_status choose_run_path(nb_ctx *ctx, int64_t n, int *path, int *size) {
    *path = 1;
    *size = 0;
    if (ctx->run_path == 1) return NB_OK;
    const bool f64 = f64_state(ctx);
    const bool eligible = f64 || ctx->math == 0;  // the math-variant ablation has no fused form
    int c = 0, g = 0;
    if (eligible && n <= kClusterMaxN) {
        const int64_t key = 2 * n + (f64 ? 1 : 0);
        auto it = ctx->cluster_sizes.find(key);
        if (it == ctx->cluster_sizes.end()) {
            c = cluster_run_size(n, f64);
            ctx->cluster_sizes[key] = c;
        } else {
            c = it->second;
        }
    }
    if (eligible) g = grid_run_ctas(n, ctx->num_sms);
    if (ctx->run_path == 2 || ctx->run_path == 3) {
        const int want = ctx->run_path == 2 ? c : g;
        if (!want)
            return fail(ctx, NB_ERR_UNSUPPORTED,
                        "the %s path runs systems of at most %lld bodies (FP32 with the MUFU "
                        "denominator, or the precision form)%s",
                        ctx->run_path == 2 ? "one-cluster" : "grid",
                        (long long)(ctx->run_path == 2 ? kClusterMaxN : kGridMaxN),
                        ctx->run_path == 2 ? " that fit a cluster on this device" : "");
        *path = ctx->run_path;
        *size = want;
        return NB_OK;
    }
    auto t = ctx->tuned.find(tune_key(ctx, 0, n) + "|run");
    if (t != ctx->tuned.end()) {
        // tuned: 0 graph, 1 one cluster, 2 grid with the tuned CTA count (a
        // choice this device cannot run falls back to the graph path)
        if (t->second.pol == 1 && c) { *path = 2; *size = c; }
        if (t->second.pol == 2 && g) {
            *path = 3;
            *size = grid_run_ctas_valid(n, ctx->num_sms, t->second.nt) ? t->second.nt : g;
        }
        return NB_OK;
    }
    if (c && n <= (f64 ? kClusterDefaultN64 : kClusterDefaultN)) {
        *path = 2;
        *size = c;
    } else if (g && n <= (f64 ? kGridDefaultN64 : kGridDefaultN)) {
        *path = 3;
        *size = g;
    }
    return NB_OK;
}

nb_status run_device(nb_ctx *ctx, int64_t n, void *x, void *v, const void *m, int steps,
                     void *ckpt, int ckpt_every, cudaStream_t st) {
    int path = 1, size = 0;
    NB_TRY(choose_run_path(ctx, n, &path, &size));
    const int kdk_flag = ctx->p.scheme == NB_SCHEME_KDK ? 1 : 0;
    const float eps2 = (float)(ctx->p.eps * ctx->p.eps);
    if (path == 2) {
        NB_CUDA(launch_cluster_run(size, n, f64_state(ctx), x, v, m, steps, kdk_flag, eps2, ctx->p.G,
                                   ctx->p.dt, ckpt, ckpt_every, st));
        ctx->launches += 1;
        return NB_OK;
    }
    if (path == 3) {
        const int64_t slice = ((n + size - 1) / size + 1) / 2 * 2;
        const size_t bytes = (size_t)size * slice * 16;
        NB_TRY(ensure(ctx, ctx->xm[0], bytes));
        NB_TRY(ensure(ctx, ctx->xm[1], bytes));
        NB_TRY(ensure(ctx, ctx->gridbar, 256, true));  // the barrier's counters start at zero
        NB_CUDA(launch_grid_run(size, n, f64_state(ctx), x, v, m, steps, kdk_flag, eps2, ctx->p.G,
                                ctx->p.dt, ckpt, ckpt_every, (float4 *)ctx->xm[0].p,
                                (float4 *)ctx->xm[1].p, (unsigned *)ctx->gridbar.p, ctx->err_word,
                                ctx->timeout_ns, (ctx->debug & kDbgStallProducer) ? 1 : 0, st));
        ctx->launches += 1;
        return NB_OK;
    }
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
        PadTargets pads;
        pads.base = xm[1];
        pads.count = 1;
        nb_status rs = pack(ctx, n, p.npad, x, v, m, xm[0], ckpt, ctx->side, pads);
        const size_t slot_bytes = (size_t)n * 6 * esize(ctx);
        for (int t = 0; rs == NB_OK && t < steps; ++t) {
            ForceArgs a = base_args(ctx, p, n, xm[t & 1]);
            a.pdl = 1;
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
            a.pdl = 1;
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

}  // namespace detail
}  // namespace nb
