// libnbody C-ABI: context lifetime, forces, steps, diagnostics and control.
// Every step of the method runs in the kernels of this library; these entry
// points validate, plan and launch.
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
    DevBuf *bufs[] = {&ctx->xm[0],     &ctx->xm[1],     &ctx->rec,        &ctx->part,
                      &ctx->counters,  &ctx->vals,      &ctx->red,        &ctx->st_v,
                      &ctx->abar64,    &ctx->stage[0],  &ctx->stage[1],   &ctx->stage[2],
                      &ctx->stage[3],  &ctx->tune[0],   &ctx->tune[1],    &ctx->tune[2],
                      &ctx->tune[3],   &ctx->tune[4],   &ctx->tune[5],    &ctx->bat,
                      &ctx->adj_traj[0], &ctx->adj_traj[1], &ctx->adj_traj64[0],
                      &ctx->adj_traj64[1], &ctx->adj_x[0], &ctx->adj_x[1], &ctx->adj_v[0],
                      &ctx->adj_v[1],  &ctx->part2,     &ctx->counters2,  &ctx->gridbar};
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
    if (key == NB_DBG_RUN_PATH) {
        if (value < 0 || value > 3) return fail(ctx, NB_ERR_INVALID, "run path must be 0, 1, 2 or 3");
        ctx->run_path = (int)value;
        return NB_OK;
    }
    if (key == NB_DBG_FORM) {
        if (value != 0 && value != 1 &&
            !(value % kSymR == 0 && find_entry(kPolSym, (int)(value / kSymR), kSymR)))
            return fail(ctx, NB_ERR_INVALID, "force form must be 0, 1 or a compiled pair-symmetric block (256, 512, 1024)");
        ctx->form_pin = (int)value;
        clear_graphs(ctx);
        return NB_OK;
    }
    if (key == NB_DBG_VJP_FORM) {
        if (value != 0 && value != 1 &&
            !(value % kSymVjpR == 0 && find_entry(kPolVjpSym, (int)(value / kSymVjpR), kSymVjpR)))
            return fail(ctx, NB_ERR_INVALID, "VJP form must be 0, 1 or a compiled pair-symmetric block (256, 512)");
        ctx->vjp_form_pin = (int)value;
        clear_graphs(ctx);
        return NB_OK;
    }
    if (key == NB_DBG_SYM_TILE) {
        if (value < -1 || value > (1 << 20))
            return fail(ctx, NB_ERR_INVALID, "tile side must be -1, 0 or a block count");
        ctx->sym_tile = (int)value;
        clear_graphs(ctx);
        return NB_OK;
    }
    if (key == NB_DBG_ADJ_PREP) {
        if (value != 0 && value != 1) return fail(ctx, NB_ERR_INVALID, "value must be 0 or 1");
        ctx->adj_unfused = (int)value;
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
