// libnbody C-ABI: the vector-Jacobian product of the forces and the
// checkpoint-and-recompute adjoint of a trajectory.
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
    // the records of both kernels live in buffers of the larger padding
    const int64_t npad = std::max(pf.npad, pv.npad);
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
             sf.jt, sv.pol, sv.nt, sv.r, sv.split, sv.jt,
             (unsigned long long)ctx->timeout_ns * 8 + ctx->adj_unfused * 4 + ctx->debug,
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
            PadTargets pads;  // the recomputed steps' records
            pads.base = traj_slot(b, 1);
            pads.count = k - 1;
            pads.stride = traj_slot(b, 1) - traj_slot(b, 0);
            rs = pack(ctx, n, npad, ctx->adj_x[b].p, nullptr, m, traj_slot(b, 0), nullptr, ctx->side2,
                      pads);
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
        // With a pair-symmetric VJP each step's epilogue (a kernel of its own,
        // after every read of the records) also prepares the next step of
        // the segment; the first step of a segment is prepared on its own.
        const bool fuse = pol_is_sym(sv.pol) && !ctx->adj_unfused;
        auto sweep = [&](int seg) {
            const int b = seg & 1;
            if (!cuda_ok(cudaStreamWaitEvent(ctx->side, ev_rec[seg], 0))) return;
            const char *slot = (const char *)ckpt + (size_t)seg * slot_bytes;
            auto x64_of = [&](int t) -> const double * {
                return !f64 ? nullptr
                            : t == 0 ? (const double *)slot
                                     : (const double *)((char *)ctx->adj_traj64[b].p + (size_t)t * n * 48);
            };
            for (int t = k - 1; rs == NB_OK && t >= 0; --t) {
                if (!fuse || t == k - 1) {
                    if (!cuda_ok(launch_adj_prepare(n, npad, f64 ? 1 : 0, traj_slot(b, t), x64_of(t), 6, m,
                                                    vbar0, xbar0, ctx->p.dt, (float4 *)ctx->rec.p,
                                                    (double *)ctx->abar64.p, ctx->side)))
                        return;
                    ctx->launches += 1;
                }
                ForceArgs a = base_args(ctx, pv, n, (const float4 *)ctx->rec.p);
                a.op = kEpiVjp;
                a.xbar = xbar0;
                a.mbar = mbar;
                a.abar64 = ctx->abar64.p;
                a.mass = m;
                if (fuse && t > 0) {
                    a.prep_next = 1;
                    a.next_xm = traj_slot(b, t - 1);
                    a.next_x64 = x64_of(t - 1);
                    a.vbar = vbar0;
                }
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

}  // extern "C"
