// Autotuner of the decode's launch shape per (N, M).
//
// The recovery of a plan's blocks can run on the persistent tensor-core kernel
// with the iterates on chip (where the shape has one), on the streaming
// tensor-core kernel (where the shape has one) or on the plain kernel with 64 to 1024 threads
// and 1, 2, 4, 8 or 16 measured blocks per CTA.  cs_autotune times the candidates the plan's
// shape admits on a synthetic call of the same N and M (random measurements, a
// zero key, a few thousand blocks, a short fixed iteration count) and records
// the fastest in the context; FP32 decodes with engine CS_ENGINE_AUTO then use
// it.  The plain kernel's sweep stops after its default shape when that is more
// than 4x slower than a tensor-core kernel of the shape.
// Timing synchronises the device, so it runs once per (N, M), before serving
// or before a decode is captured into a CUDA graph.
#include <algorithm>
#include <vector>

#include "internal.h"

namespace csvc {
namespace {

struct Candidate {
    int engine;
    int threads;
    int blocks;
};

// Uniform values in [-0.5, 0.5) from a 64-bit LCG (Knuth's MMIX constants):
// inputs only, their distribution does not change the kernels' timing.
void fill_uniform(std::vector<float>& v, uint64_t seed) {
    uint64_t x = seed * 0x9E3779B97F4A7C15ull + 1;
    for (float& f : v) {
        x = x * 6364136223846793005ull + 1442695040888963407ull;
        f = (float)((double)(x >> 11) * (1.0 / 9007199254740992.0) - 0.5);
    }
}

}  // namespace
}  // namespace csvc

using namespace csvc;

extern "C" int cs_autotune(cs_ctx* ctx, cs_plan* plan, int32_t* engine, int32_t* plain_threads,
                           int32_t* plain_blocks_per_cta, float* ns_per_block_iter) {
    if (!ctx || !plan) return fail(CS_EINVAL, "null argument");
    if (plan->ctx != ctx) return fail(CS_EINVAL, "plan belongs to another context");
    CS_CUDA_TRY(cudaSetDevice(ctx->device));
    const int b = plan->b, n = plan->n, m = plan->m;
    const int cols = 64;
    // two tiles of 128 blocks per SM (the throughput of a call that fills the GPU;
    // a kernel that gives a tile one SM needs it), at most 40 M pixels out
    long long rows = std::min<long long>(2ll * ctx->sm_count * 128, (40ll << 20) / n);
    rows = std::max<long long>(cols, rows / cols * cols);
    GopShape gs;
    gs.b = b;
    gs.n = n;
    gs.m = m;
    gs.nbr = (int)(rows / cols);
    gs.nbc = cols;
    gs.nblk = (int)rows;
    gs.h = b * gs.nbr;
    gs.w = b * gs.nbc;
    gs.g = 2;
    gs.n_gops = 1;
    gs.n_cs = 1;

    // tensor-core kernels first, then the plain kernel's default shape, then the rest
    // of its sweep; the rest is skipped when the default is over 4x slower than a
    // tensor-core kernel, a wider margin than the spread between the plain shapes
    std::vector<Candidate> cands;
    if (tc_supported(plan, CS_FP32)) cands.push_back({CS_ENGINE_TC, 0, 0});
    if (tcs_supported(plan)) cands.push_back({CS_ENGINE_TC_STREAM, 0, 0});
    if (tcz_supported(plan)) cands.push_back({CS_ENGINE_TC_CHUNK, 0, 0});
    const size_t n_tc = cands.size();
    int t_def = 0, r_def = 0;
    plain_default_shape(n, m, &t_def, &r_def);
    cands.push_back({CS_ENGINE_PLAIN, t_def, r_def});
    for (int t : {64, 128, 256, 512, 1024})
        for (int r : {1, 2, 4, 8, 16})
            if (plain_shape_valid(t, r, n, m) && !(t == t_def && r == r_def))
                cands.push_back({CS_ENGINE_PLAIN, t, r});

    std::vector<float> y_host((size_t)rows * m);
    fill_uniform(y_host, plan->seed);
    float *y = nullptr, *out = nullptr;
    uint8_t* key = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const size_t px = (size_t)gs.h * gs.w;
    cudaError_t e = cudaMalloc(&y, y_host.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&out, px * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&key, px);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(y, y_host.data(), y_host.size() * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(key, 0, px, s);

    const int iters = 16;
    Candidate best{0, 0, 0};
    float best_ms = -1.f, plain_default_ms = 0.f;
    for (size_t i = 0; e == cudaSuccess && i < cands.size(); ++i) {
        if (i == n_tc + 1 && n_tc > 0 && best.engine != CS_ENGINE_PLAIN && plain_default_ms > 4.f * best_ms)
            break;
        DecodeArgs d;
        d.plan = plan;
        d.gs = gs;
        d.key = key;
        d.y = y;
        d.out_f32 = out;
        d.out_u8 = nullptr;
        d.iters = iters;
        d.tail_iters = 0;
        d.lambda_rel = 0.01f;
        d.precision = CS_FP32;
        d.beta = ctx->beta_dev;
        d.plain_threads = cands[i].threads;
        d.plain_blocks = cands[i].blocks;
        auto launch = [&]() {
            return cands[i].engine == CS_ENGINE_TC          ? launch_decode_tc(d, s)
                   : cands[i].engine == CS_ENGINE_TC_STREAM ? launch_decode_tcs(d, s)
                   : cands[i].engine == CS_ENGINE_TC_CHUNK  ? launch_decode_tcz(d, s)
                                                            : launch_decode_plain(d, s);
        };
        e = launch();   // warm-up (and first-launch attribute set-up)
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        for (int r = 0; e == cudaSuccess && r < 2; ++r) e = launch();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && i == n_tc) plain_default_ms = ms;
        if (e == cudaSuccess && (best_ms < 0.f || ms < best_ms)) {
            best_ms = ms;
            best = cands[i];
        }
    }
    if (y) cudaFree(y);
    if (out) cudaFree(out);
    if (key) cudaFree(key);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess) return cuda_fail(e, "cs_autotune");
    if (best_ms < 0.f) return fail(CS_EINVAL, "no decode kernel for this (N, M)");
    {
        std::lock_guard<std::mutex> lock(ctx->tune_mu);
        ctx->tuned[{n, m}] = {best.engine, best.threads, best.blocks};
    }
    if (engine) *engine = best.engine;
    if (plain_threads) *plain_threads = best.threads;
    if (plain_blocks_per_cta) *plain_blocks_per_cta = best.blocks;
    if (ns_per_block_iter) *ns_per_block_iter = (float)(1e6 * best_ms / 2.0 / ((double)rows * iters));
    return CS_OK;
}
