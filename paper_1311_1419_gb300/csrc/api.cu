// The C ABI (include/csvc.h): contexts, plans, argument checking, dispatch of
// the encode/decode/metrics kernels, compression-ratio accounting and the
// serving tickets.  No torch type crosses this boundary; every call reports
// failure through its return code.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <new>
#include <string>

#include "internal.h"

namespace csvc {

namespace {
thread_local std::string g_last_error;
}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int status, const std::string& msg) {
    g_last_error = msg;
    return status;
}

int cuda_fail(cudaError_t err, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorName(err) + " (" +
                   cudaGetErrorString(err) + ")";
    return err == cudaErrorMemoryAllocation ? CS_ENOMEM : CS_ECUDA;
}

cudaError_t slot_ring_init(SlotRing* r, int n) {
    for (int i = 0; i < n; ++i) {
        cudaEvent_t e = nullptr;
        cudaError_t err = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        if (err != cudaSuccess) return err;
        r->ev.push_back(e);
    }
    return cudaSuccess;
}

void slot_ring_destroy(SlotRing* r) {
    for (cudaEvent_t e : r->ev) cudaEventDestroy(e);
    r->ev.clear();
}

static bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &st) == cudaSuccess && st == cudaStreamCaptureStatusActive;
}

cudaError_t slot_take(SlotRing* r, cudaStream_t s, int* slot) {
    if (r->ev.empty()) return cudaErrorInvalidValue;
    const int i = (int)(r->next++ % r->ev.size());
    *slot = i;
    return cudaStreamWaitEvent(s, r->ev[i], capturing(s) ? cudaEventWaitExternal : 0);
}

cudaError_t slot_done(SlotRing* r, int slot, cudaStream_t s) {
    return capturing(s) ? cudaEventRecordWithFlags(r->ev[slot], s, cudaEventRecordExternal)
                        : cudaEventRecord(r->ev[slot], s);
}

cudaStream_t fork_stream(const cs_ctx* ctx, cudaStream_t s, int which) {
    int set = 0;
    for (size_t i = 0; i < ctx->streams.size(); ++i)
        if (ctx->streams[i] == s) set = (int)i + 1;
    return ctx->fork_streams[(size_t)set * kForkStreams + which];
}

// Device scratch of the decode kernels counts against the context's HBM
// budget: with a budget it may take at most half of it, and no more than the
// serving pool (once it exists) and earlier scratch leave.
static size_t scratch_room(const cs_ctx* ctx) {
    if (!ctx->hbm_budget) return SIZE_MAX;
    const size_t used = ctx->scratch_bytes + serving_pool_bytes(ctx);
    const size_t room = ctx->hbm_budget > used ? ctx->hbm_budget - used : 0;
    const size_t half = ctx->hbm_budget / 2;
    return std::min(room, half > ctx->scratch_bytes ? half - ctx->scratch_bytes : (size_t)0);
}

size_t scratch_room_of(const cs_ctx* ctx) { return scratch_room(ctx); }

// Validate a call's parameters against the plan and derive the GOP shape.
int make_shape(const cs_plan* plan, const cs_params* p, GopShape* gs) {
    if (!plan || !p) return fail(CS_EINVAL, "null plan or params");
    if (p->height < 1 || p->width < 1) return fail(CS_EINVAL, "frame size must be >= 1");
    if (p->gop < 2) return fail(CS_EINVAL, "gop must be >= 2 (one key + at least one CS frame)");
    if (p->n_gops < 0) return fail(CS_EINVAL, "n_gops must be >= 0");
    if (p->block != plan->b) return fail(CS_EINVAL, "block*block does not match the plan's N");
    if (p->m != plan->m) return fail(CS_EINVAL, "m does not match the plan's M");
    gs->h = p->height;
    gs->w = p->width;
    gs->g = p->gop;
    gs->n_gops = p->n_gops == 0 ? 1 : p->n_gops;
    gs->b = plan->b;
    gs->n = plan->n;
    gs->m = plan->m;
    gs->nbr = (p->height + plan->b - 1) / plan->b;
    gs->nbc = (p->width + plan->b - 1) / plan->b;
    gs->nblk = gs->nbr * gs->nbc;
    const long long n_cs = (long long)gs->n_gops * (p->gop - 1);
    if (n_cs * gs->nblk > (1ll << 31) - 1) return fail(CS_EINVAL, "too many blocks in one call");
    gs->n_cs = (int)n_cs;
    return CS_OK;
}

namespace {

int check_decode_params(const cs_params* p) {
    if (p->iters < 0 || p->iters > kMaxIters) return fail(CS_EINVAL, "iters out of range");
    if (p->fp32_tail_iters < 0) return fail(CS_EINVAL, "fp32_tail_iters must be >= 0");
    if (!(p->lambda_rel >= 0.f) || !isfinite(p->lambda_rel))
        return fail(CS_EINVAL, "lambda_rel must be finite and >= 0");
    if (p->precision < CS_FP32 || p->precision > CS_FP16) return fail(CS_EINVAL, "bad precision");
    if (p->engine < CS_ENGINE_AUTO || p->engine > CS_ENGINE_TC_CHUNK) return fail(CS_EINVAL, "bad engine");
    return CS_OK;
}

// Check one decode request and fill its launch arguments; *engine gets the
// kernel that will run it.
int prepare_decode(cs_plan* plan, const cs_params* params, const uint8_t* key, const float* y,
                   float* out_f32, uint8_t* out_u8, DecodeArgs* d, int* engine) {
    GopShape gs;
    int st = make_shape(plan, params, &gs);
    if (st) return st;
    st = check_decode_params(params);
    if (st) return st;
    if (!out_f32 && !out_u8) return fail(CS_EINVAL, "both outputs are NULL");
    if (gs.n_cs > 0 && (!key || !y)) return fail(CS_EINVAL, "null input pointer");
    d->plan = plan;
    d->gs = gs;
    d->key = key;
    d->y = y;
    d->out_f32 = out_f32;
    d->out_u8 = out_u8;
    d->iters = params->iters;
    d->tail_iters = params->fp32_tail_iters;
    d->lambda_rel = params->lambda_rel;
    d->precision = params->precision;
    d->beta = plan->ctx->beta_dev;
    d->plain_threads = 0;
    d->plain_blocks = 0;
    int eng = params->engine;
    const bool tc_ok = tc_supported(plan, params->precision);
    const bool tcs_ok = tcs_supported(plan);
    const bool tcz_ok = tcz_supported(plan);
    if (eng == CS_ENGINE_TC_CHUNK && !tcz_ok)
        return fail(CS_EINVAL, "chunked tensor-core decode does not support this (N, M)");
    if (eng == CS_ENGINE_TC && !tc_ok)
        return fail(CS_EINVAL, "on-chip tensor-core decode does not support this (N, M)");
    if (eng == CS_ENGINE_TC_STREAM && !tcs_ok)
        return fail(CS_EINVAL, "streaming tensor-core decode does not support this (N, M)");
    {   // the autotuned shape of this (N, M), if cs_autotune has run for it
        std::lock_guard<std::mutex> lock(plan->ctx->tune_mu);
        auto it = plan->ctx->tuned.find({plan->n, plan->m});
        if (it != plan->ctx->tuned.end()) {
            // (the plain kernel computes in FP32 only: mixed precision keeps the default order then)
            if (eng == CS_ENGINE_AUTO && (params->precision == CS_FP32 || it->second[0] != CS_ENGINE_PLAIN))
                eng = it->second[0];
            d->plain_threads = it->second[1];
            d->plain_blocks = it->second[2];
        }
    }
    if (eng == CS_ENGINE_AUTO) eng = tc_ok ? CS_ENGINE_TC : tcs_ok ? CS_ENGINE_TC_STREAM : CS_ENGINE_PLAIN;
    if (eng == CS_ENGINE_PLAIN && params->precision != CS_FP32)
        return fail(CS_EINVAL, "the plain engine computes in FP32 only");
    *engine = eng;
    return CS_OK;
}

}  // namespace

int prepare_decode_args(cs_plan* plan, const cs_params* params, const uint8_t* key, const float* y,
                        float* out_f32, uint8_t* out_u8, DecodeArgs* d, int* engine) {
    return prepare_decode(plan, params, key, y, out_f32, out_u8, d, engine);
}

int decode_enqueue(cs_plan* plan, const cs_params* params, const uint8_t* key, const float* y,
                   float* out_f32, uint8_t* out_u8, cudaStream_t stream) {
    DecodeArgs d;
    int engine = 0;
    int st = prepare_decode(plan, params, key, y, out_f32, out_u8, &d, &engine);
    if (st) return st;
    cudaError_t e = engine == CS_ENGINE_TC          ? launch_decode_tc(d, stream)
                    : engine == CS_ENGINE_TC_STREAM ? launch_decode_tcs(d, stream)
                    : engine == CS_ENGINE_TC_CHUNK  ? launch_decode_tcz(d, stream)
                                                    : launch_decode_plain(d, stream);
    if (e != cudaSuccess) return cuda_fail(e, "decode launch");
    return CS_OK;
}

}  // namespace csvc

using namespace csvc;

extern "C" {

int cs_ctx_create(cs_ctx** out, int device, size_t hbm_budget_bytes) {
    if (!out) return fail(CS_EINVAL, "out is NULL");
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || count == 0) return fail(CS_ENODEV, "no CUDA device");
    if (device < 0 || device >= count) return fail(CS_EINVAL, "device index out of range");
    CS_CUDA_TRY(cudaSetDevice(device));
    cudaDeviceProp prop;
    CS_CUDA_TRY(cudaGetDeviceProperties(&prop, device));
    if (prop.major != 10 || prop.minor != 3)
        return fail(CS_ENODEV, "this library is built for sm_103 (GB300) only");
    cs_ctx* ctx = new (std::nothrow) cs_ctx();
    if (!ctx) return fail(CS_ENOMEM, "host allocation failed");
    ctx->device = device;
    ctx->sm_count = prop.multiProcessorCount;
    ctx->hbm_budget = hbm_budget_bytes;
    // FISTA momentum schedule: t_1 = 1, t_{k+1} = (1 + sqrt(1 + 4 t_k^2))/2,
    // beta_k = (t_k - 1)/t_{k+1}; a data-independent scalar sequence, in FP64.
    std::vector<float> beta(kMaxIters);
    double t = 1.0;
    for (int k = 0; k < kMaxIters; ++k) {
        const double tn = (1.0 + sqrt(1.0 + 4.0 * t * t)) / 2.0;
        beta[k] = (float)((t - 1.0) / tn);
        t = tn;
    }
    e = cudaMalloc(&ctx->beta_dev, sizeof(float) * kMaxIters);
    if (e == cudaSuccess)
        e = cudaMemcpy(ctx->beta_dev, beta.data(), sizeof(float) * kMaxIters, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->err_dev, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->err_dev, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->counters_dev, sizeof(int) * kTileCounters);
    if (e == cudaSuccess) e = slot_ring_init(&ctx->counter_ring, kTileCounters);
    if (e == cudaSuccess) e = slot_ring_init(&ctx->stage_ring, 1);
    for (int i = 0; e == cudaSuccess && i < 8; ++i) {
        cudaStream_t s;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) ctx->streams.push_back(s);
    }
    if (e == cudaSuccess) e = tcsq_create(ctx);
    int prio_least = 0, prio_greatest = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
    // one fork set for callers' streams and one per serving stream
    for (int i = 0; e == cudaSuccess && i < kForkStreams * (1 + (int)ctx->streams.size()); ++i) {
        cudaStream_t s;
        e = cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking,
                                         i % kForkStreams == kForkTc8Head ? prio_greatest : prio_least);
        if (e == cudaSuccess) ctx->fork_streams.push_back(s);
    }
    if (e != cudaSuccess) {
        int st = cuda_fail(e, "context setup");
        cs_ctx_destroy(ctx);
        return st;
    }
    *out = ctx;
    return CS_OK;
}

int cs_ctx_destroy(cs_ctx* ctx) {
    if (!ctx) return CS_OK;
    cudaSetDevice(ctx->device);
    for (cudaStream_t s : ctx->streams) cudaStreamSynchronize(s);
    tcsq_destroy(ctx);
    serving_destroy(ctx);
    for (cudaStream_t s : ctx->streams) cudaStreamDestroy(s);
    for (cudaStream_t s : ctx->fork_streams) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    if (ctx->beta_dev) cudaFree(ctx->beta_dev);
    if (ctx->err_dev) cudaFree(ctx->err_dev);
    if (ctx->counters_dev) cudaFree(ctx->counters_dev);
    if (ctx->tc8_scratch) cudaFree(ctx->tc8_scratch);
    if (ctx->tcs_scratch) cudaFree(ctx->tcs_scratch);
    if (ctx->tv_scratch) cudaFree(ctx->tv_scratch);
    slot_ring_destroy(&ctx->counter_ring);
    slot_ring_destroy(&ctx->tc8_ring);
    slot_ring_destroy(&ctx->tcs_ring);
    slot_ring_destroy(&ctx->tv_ring);
    slot_ring_destroy(&ctx->stage_ring);
    if (ctx->stage) cudaFree(ctx->stage);
    delete ctx;
    return CS_OK;
}

int cs_make_phi(cs_ctx* ctx, int32_t n, int32_t m, uint64_t seed, cs_plan** out) {
    if (!ctx || !out) return fail(CS_EINVAL, "null ctx or out");
    *out = nullptr;
    int b = (int)lround(sqrt((double)n));
    if (n < 1 || n > kMaxN || b * b != n) return fail(CS_EINVAL, "N must be a perfect square <= 4096");
    if (m < 1 || m > n || m > 1024) return fail(CS_EINVAL, "need 1 <= M <= min(N, 1024)");
    CS_CUDA_TRY(cudaSetDevice(ctx->device));
    cs_plan* p = new (std::nothrow) cs_plan();
    if (!p) return fail(CS_ENOMEM, "host allocation failed");
    p->ctx = ctx;
    p->n = n;
    p->m = m;
    p->b = b;
    p->seed = seed;
    double* gram = nullptr;
    double* lam_dev = nullptr;
    float* ranges_dev = nullptr;
    float ranges[3] = {0.f, 0.f, 0.f};
    cudaStream_t s = nullptr;
    double lam = 0.0;
    const bool tc_chip = tc_plan_supported(n, m), tcs = tcs_plan_supported(n, m);
    const bool tc = tc_chip || tcs;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    const size_t mn = (size_t)m * n;
    if (e == cudaSuccess) e = cudaMalloc(&p->phi, mn * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&p->a, mn * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&p->dct, (size_t)b * b * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&gram, (size_t)m * m * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&lam_dev, sizeof(double));
    if (e == cudaSuccess && tc) e = cudaMalloc(&ranges_dev, 3 * sizeof(float));
    if (e == cudaSuccess) e = launch_phi(p->phi, n, m, seed, s);
    if (e == cudaSuccess) e = launch_form_a(p->phi, p->a, p->dct, n, m, b, s);
    if (e == cudaSuccess) e = launch_lambda_max(p->phi, n, m, gram, lam_dev, s);
    if (e == cudaSuccess && tc) e = launch_tc_ranges(p->a, p->phi, n, m, ranges_dev, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&lam, lam_dev, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && tc)
        e = cudaMemcpyAsync(ranges, ranges_dev, sizeof(ranges), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && tc && ranges[0] > 0.f) {
        // fp16 operands: A scaled so that max |A| lands near 2^14; the residual
        // operand scaled down only if 4 * 255 * max_m ||Phi_m||_1 could pass 2^14
        p->tc_ea = (int)floor(log2(16384.0 / (double)ranges[0]));
        const double pbound = 4.0 * 255.0 * (double)ranges[1];
        p->tc_ep = pbound > 16384.0 ? (int)floor(log2(16384.0 / pbound)) : 0;
        if (tc_chip) {
            e = cudaMalloc(&p->a_tc, tc_operand_bytes(n, m));
            if (e == cudaSuccess)
                e = n == 1024 ? launch_tc8_images(p->a, p->a_tc, m, p->tc_ea, s)
                              : launch_tc_images(p->a, p->a_tc, n, m, p->tc_ea, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        }
        if (e == cudaSuccess && tcs) {
            e = cudaMalloc(&p->a_tcs, tcs_operand_bytes(n, m));
            if (e == cudaSuccess) e = launch_tcs_images(p->a, p->a_tcs, n, m, p->tc_ea, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e == cudaSuccess) {
                // the streaming decode's per-CTA iterates, one ring per context, as
                // many per-launch areas (up to kTcsSlotsMax) as the budget allows;
                // none fits: this context decodes these shapes without the
                // streaming kernel
                std::lock_guard<std::mutex> lock(ctx->mu);
                if (!ctx->tcs_scratch) {
                    const size_t slot = tcs_slot_bytes(ctx->sm_count);
                    const int n = (int)std::min<size_t>(kTcsSlotsMax, scratch_room(ctx) / slot);
                    if (n > 0) {
                        e = cudaMalloc(&ctx->tcs_scratch, (size_t)n * slot);
                        if (e == cudaSuccess) e = slot_ring_init(&ctx->tcs_ring, n);
                        if (e == cudaSuccess) {
                            ctx->tcs_slots = n;
                            ctx->scratch_bytes += (size_t)n * slot;
                        }
                    }
                }
            }
        }
        if (ranges[2] > 0.f) p->tc_ephi = (int)floor(log2(16384.0 / (double)ranges[2]));   // max |Phi| near 2^14
        if (e == cudaSuccess && tcs && ranges[2] > 0.f) {
            // the streaming TV decode's images of Phi (the streaming decode's layouts)
            e = cudaMalloc(&p->phi_tcs, tcs_operand_bytes(n, m));
            if (e == cudaSuccess) e = launch_tcs_images(p->phi, p->phi_tcs, n, m, p->tc_ephi, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        }
        if (e == cudaSuccess && tc_chip && n == 256 && ranges[2] > 0.f) {
            // the 16 x 16 tensor-core encode's Phi images
            e = cudaMalloc(&p->phi_tc, tc_operand_bytes(n, m));
            if (e == cudaSuccess) e = launch_tc_images(p->phi, p->phi_tc, n, m, p->tc_ephi, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        } else if (e == cudaSuccess && encode_tcg_plan_supported(n, m) && ranges[2] > 0.f) {
            // the general tensor-core encode's Phi images (every other block size and M)
            e = cudaMalloc(&p->phi_tcg, encode_tcg_image_bytes(n, m));
            if (e == cudaSuccess) e = launch_phi_images_g(p->phi, p->phi_tcg, n, m, p->tc_ephi, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        }
        if (e == cudaSuccess && tc_chip && n == 1024) {
            // the cluster decode's s^K all-gather, one ring per context (when the
            // budget has no room for it, 32 x 32 blocks skip the cluster kernel)
            std::lock_guard<std::mutex> lock(ctx->mu);
            const size_t bytes = (size_t)kScratchSlots * tc8_slot_bytes(ctx->sm_count);
            if (!ctx->tc8_scratch && bytes <= scratch_room(ctx)) {
                e = cudaMalloc(&ctx->tc8_scratch, bytes);
                if (e == cudaSuccess) e = slot_ring_init(&ctx->tc8_ring, kScratchSlots);
                if (e == cudaSuccess) ctx->scratch_bytes += bytes;
            }
        }
    }
    if (gram) cudaFree(gram);
    if (lam_dev) cudaFree(lam_dev);
    if (ranges_dev) cudaFree(ranges_dev);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess) {
        int st = cuda_fail(e, "cs_make_phi");
        cs_plan_destroy(p);
        return st;
    }
    if (!(lam > 0.0) || !isfinite(lam)) {
        cs_plan_destroy(p);
        return fail(CS_ECUDA, "power iteration returned a non-positive lambda_max");
    }
    p->lipschitz = 1.0001 * lam;
    *out = p;
    return CS_OK;
}

int cs_plan_destroy(cs_plan* p) {
    if (!p) return CS_OK;
    cudaSetDevice(p->ctx->device);
    if (p->phi) cudaFree(p->phi);
    if (p->a) cudaFree(p->a);
    if (p->dct) cudaFree(p->dct);
    if (p->a_tc) cudaFree(p->a_tc);
    if (p->a_tcs) cudaFree(p->a_tcs);
    if (p->phi_tcs) cudaFree(p->phi_tcs);
    if (p->phi_tc) cudaFree(p->phi_tc);
    if (p->phi_tcg) cudaFree(p->phi_tcg);
    delete p;
    return CS_OK;
}

int cs_plan_phi(const cs_plan* p, const float** phi_dev) {
    if (!p || !phi_dev) return fail(CS_EINVAL, "null argument");
    *phi_dev = p->phi;
    return CS_OK;
}

int cs_plan_a(const cs_plan* p, const float** a_dev) {
    if (!p || !a_dev) return fail(CS_EINVAL, "null argument");
    *a_dev = p->a;
    return CS_OK;
}

int cs_plan_lipschitz(const cs_plan* p, double* lipschitz) {
    if (!p || !lipschitz) return fail(CS_EINVAL, "null argument");
    *lipschitz = p->lipschitz;
    return CS_OK;
}

int cs_encode_gop(cs_plan* plan, const cs_params* params, const uint8_t* frames_dev, float* y_dev,
                  cs_stream_t stream) {
    GopShape gs;
    int st = make_shape(plan, params, &gs);
    if (st) return st;
    if (gs.n_cs > 0 && (!frames_dev || !y_dev)) return fail(CS_EINVAL, "null buffer");
    if (params->engine < CS_ENGINE_AUTO || params->engine > CS_ENGINE_TC_CHUNK) return fail(CS_EINVAL, "bad engine");
    // the tensor-core encode where the plan has Phi images for it, unless the plain
    // engine is asked for
    const bool tc = params->engine != CS_ENGINE_PLAIN && encode_tcg_supported(plan);
    cudaError_t e = tc ? launch_encode_tcg(plan, gs, frames_dev, y_dev, (cudaStream_t)stream)
                       : launch_encode(plan, gs, frames_dev, y_dev, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "encode launch");
    return CS_OK;
}

int cs_encode_batch(cs_ctx* ctx, int32_t n_plans, cs_plan* const* plans, const cs_params* params,
                    const uint8_t* frames_dev, float* const* y_dev, cs_stream_t stream) {
    if (!ctx || n_plans < 0 || (n_plans > 0 && (!plans || !params || !y_dev)))
        return fail(CS_EINVAL, "null argument");
    if (n_plans == 0) return CS_OK;
    std::vector<GopShape> gs(n_plans);
    for (int i = 0; i < n_plans; ++i) {
        if (!plans[i] || plans[i]->ctx != ctx) return fail(CS_EINVAL, "plan of another context");
        const int st = make_shape(plans[i], &params[i], &gs[i]);
        if (st) return st;
        if (params[i].engine < CS_ENGINE_AUTO || params[i].engine > CS_ENGINE_TC_CHUNK)
            return fail(CS_EINVAL, "bad engine");
        if (gs[i].h != gs[0].h || gs[i].w != gs[0].w || gs[i].g != gs[0].g || gs[i].n_gops != gs[0].n_gops ||
            gs[i].b != gs[0].b)
            return fail(CS_EINVAL, "every plan's call must describe the same clip and block size");
        if (gs[i].n_cs > 0 && (!frames_dev || !y_dev[i])) return fail(CS_EINVAL, "null buffer");
    }
    CS_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    // the plans the tensor-core encode takes share launches (the clip is read once
    // per launch); the rest run on the plain kernel one by one
    std::vector<const cs_plan*> tc_plans;
    std::vector<float*> tc_y;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n_plans && e == cudaSuccess; ++i) {
        if (params[i].engine != CS_ENGINE_PLAIN && encode_tcg_supported(plans[i])) {
            tc_plans.push_back(plans[i]);
            tc_y.push_back(y_dev[i]);
        } else {
            e = launch_encode(plans[i], gs[i], frames_dev, y_dev[i], s);
        }
    }
    if (e == cudaSuccess && !tc_plans.empty())
        e = launch_encode_tcg_multi(tc_plans.data(), tc_y.data(), (int)tc_plans.size(), gs[0], frames_dev, s);
    if (e != cudaSuccess) return cuda_fail(e, "encode launch");
    return CS_OK;
}

int cs_decode_gop(cs_plan* plan, const cs_params* params, const uint8_t* key_dev, const float* y_dev,
                  float* frames_f32_dev, uint8_t* frames_u8_dev, cs_stream_t stream) {
    return decode_enqueue(plan, params, key_dev, y_dev, frames_f32_dev, frames_u8_dev,
                          (cudaStream_t)stream);
}

int cs_decode_batch(cs_ctx* ctx, int32_t n_jobs, cs_plan* const* plans, const cs_params* params,
                    const uint8_t* const* key_dev, const float* const* y_dev,
                    float* const* frames_f32_dev, uint8_t* const* frames_u8_dev,
                    cs_stream_t stream) {
    if (!ctx || n_jobs < 0 || (n_jobs > 0 && (!plans || !params || !key_dev || !y_dev)))
        return fail(CS_EINVAL, "null argument");
    std::vector<DecodeArgs> tc_jobs, tcs_jobs, tcz_jobs, plain_jobs;
    tc_jobs.reserve(n_jobs);
    for (int i = 0; i < n_jobs; ++i) {
        if (!plans[i] || plans[i]->ctx != ctx) return fail(CS_EINVAL, "plan of another context");
        DecodeArgs d;
        int engine = 0;
        int st = prepare_decode(plans[i], &params[i], key_dev[i], y_dev[i],
                                frames_f32_dev ? frames_f32_dev[i] : nullptr,
                                frames_u8_dev ? frames_u8_dev[i] : nullptr, &d, &engine);
        if (st) return fail(st, std::string("job ") + std::to_string(i) + ": " + cs_last_error());
        (engine == CS_ENGINE_TC          ? tc_jobs
         : engine == CS_ENGINE_TC_STREAM ? tcs_jobs
         : engine == CS_ENGINE_TC_CHUNK  ? tcz_jobs
                                         : plain_jobs)
            .push_back(d);
    }
    cudaError_t e = cudaSuccess;
    cudaStream_t s = (cudaStream_t)stream;
    if (!tcs_jobs.empty() && !tc_jobs.empty()) {
        // the streaming kernel's launch on its own fork stream, joined back on s:
        // its CTAs take SMs as the on-chip launches' tails drain
        cudaStream_t fs = fork_stream(ctx, s, kForkTcs);
        cudaEvent_t fork = nullptr, join = nullptr;
        e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(fs, fork, 0);
        if (e == cudaSuccess) e = launch_decode_tcs_batch(tcs_jobs.data(), (int)tcs_jobs.size(), fs);
        if (e == cudaSuccess) e = cudaEventRecord(join, fs);
        if (e == cudaSuccess) e = launch_decode_tc_batch(tc_jobs.data(), (int)tc_jobs.size(), s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, join, 0);
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
    } else if (!tc_jobs.empty()) {
        e = launch_decode_tc_batch(tc_jobs.data(), (int)tc_jobs.size(), s);
    } else if (!tcs_jobs.empty()) {
        e = launch_decode_tcs_batch(tcs_jobs.data(), (int)tcs_jobs.size(), s);
    }
    // the chunked kernel's launch takes every SM: after the others on s
    if (e == cudaSuccess && !tcz_jobs.empty()) e = launch_decode_tcz_batch(tcz_jobs.data(), (int)tcz_jobs.size(), s);
    for (size_t i = 0; e == cudaSuccess && i < plain_jobs.size(); ++i)
        e = launch_decode_plain(plain_jobs[i], s);
    if (e != cudaSuccess) return cuda_fail(e, "batched decode launch");
    return CS_OK;
}

int cs_psnr(const uint8_t* ref_dev, const float* test_dev, int32_t n_frames, int32_t height,
            int32_t width, double* psnr_dev, cs_stream_t stream) {
    if (n_frames < 0 || height < 1 || width < 1) return fail(CS_EINVAL, "bad shape");
    if (n_frames > 0 && (!ref_dev || !test_dev || !psnr_dev)) return fail(CS_EINVAL, "null buffer");
    cudaError_t e = launch_psnr(ref_dev, test_dev, n_frames, height, width, psnr_dev,
                                (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "psnr launch");
    return CS_OK;
}

double cs_total_cr(int32_t gop, double cr_key, double cr_cs) {
    if (gop < 1 || !(cr_key > 0.0) || !(cr_cs > 0.0)) return NAN;
    return gop / (1.0 / cr_key + (gop - 1) / cr_cs);
}

double cs_raw_key_cr(int32_t gop, int32_t height, int32_t width, int32_t block, int32_t m) {
    if (gop < 1 || height < 1 || width < 1 || block < 1 || m < 1) return NAN;
    const double nblk = (double)((height + block - 1) / block) * ((width + block - 1) / block);
    const double px = (double)height * width;
    return gop * px / (px + (gop - 1) * nblk * m);
}

int cs_ctx_set_debug(cs_ctx* ctx, int32_t flags) {
    if (!ctx) return fail(CS_EINVAL, "null ctx");
    if (flags & ~CS_DEBUG_DROP_ARRIVAL) return fail(CS_EINVAL, "unknown debug flag");
    ctx->debug_flags.store(flags);
    return CS_OK;
}

int cs_ctx_set_serving(cs_ctx* ctx, int32_t mode) {
    if (!ctx) return fail(CS_EINVAL, "null ctx");
    if (mode != CS_SERVING_QUEUE && mode != CS_SERVING_LAUNCH) return fail(CS_EINVAL, "bad serving mode");
    std::lock_guard<std::mutex> lock(ctx->mu);
    ctx->serving_queue = mode == CS_SERVING_QUEUE;
    return CS_OK;
}

int cs_ctx_status(cs_ctx* ctx) {
    if (!ctx) return fail(CS_EINVAL, "null ctx");
    CS_CUDA_TRY(cudaSetDevice(ctx->device));
    CS_CUDA_TRY(cudaDeviceSynchronize());
    int flag = 0;
    CS_CUDA_TRY(cudaMemcpy(&flag, ctx->err_dev, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        CS_CUDA_TRY(cudaMemset(ctx->err_dev, 0, sizeof(int)));
        return fail(CS_ETIMEDOUT, "a decode kernel gave up a bounded device-side wait");
    }
    return CS_OK;
}

const char* cs_strerror(int status) {
    switch (status) {
        case CS_OK: return "ok";
        case CS_EINVAL: return "invalid argument";
        case CS_ENOMEM: return "out of device memory or HBM budget";
        case CS_EAGAIN: return "not admitted now, retry";
        case CS_ETIMEDOUT: return "bounded device wait timed out";
        case CS_ECUDA: return "CUDA error";
        case CS_ENOTFOUND: return "unknown ticket";
        case CS_ENODEV: return "no usable sm_103 device";
        default: return "unknown status";
    }
}

const char* cs_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
