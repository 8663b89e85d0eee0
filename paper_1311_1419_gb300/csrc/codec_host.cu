// cs_codec_host: the whole codec of one clip from and to host memory.
//
// The clip (key frames and CS frames, Sec. 3) is copied to the device once;
// every plan measures it (Sec. 3.1, y = Phi r per block of every residual; the
// plans of one block size in one encode launch that reads the clip once);
// the measurements of all plans are recovered in one batched decode (Sec. 3.2,
// Eqs. 1-4); every decoded CS frame is scored by PSNR against the original
// (Sec. 4); the uint8 decoded frames and the PSNRs go back to the host.  The
// device staging belongs to the context: one buffer, grown when a call needs
// more, handed from call to call through a one-slot ring so that calls on
// different streams take turns.
#include <string>
#include <vector>

#include "internal.h"

namespace csvc {
int make_shape(const cs_plan* plan, const cs_params* p, GopShape* gs);
}  // namespace csvc

using namespace csvc;

namespace {
constexpr size_t kStageAlign = 256;
size_t up(size_t x) { return (x + kStageAlign - 1) / kStageAlign * kStageAlign; }
}  // namespace

extern "C" int cs_codec_host(cs_ctx* ctx, int32_t n_plans, cs_plan* const* plans,
                             const cs_params* params, const uint8_t* clip_host,
                             uint8_t* const* frames_u8_host, double* const* psnr_host,
                             cs_stream_t stream) {
    if (!ctx || n_plans < 1 || !plans || !params || !clip_host || !frames_u8_host || !psnr_host)
        return fail(CS_EINVAL, "null argument or no plan");
    std::vector<GopShape> gs(n_plans);
    for (int i = 0; i < n_plans; ++i) {
        if (!plans[i] || plans[i]->ctx != ctx) return fail(CS_EINVAL, "plan of another context");
        if (!frames_u8_host[i] || !psnr_host[i]) return fail(CS_EINVAL, "null output buffer");
        const int st = make_shape(plans[i], &params[i], &gs[i]);
        if (st) return st;
        if (gs[i].h != gs[0].h || gs[i].w != gs[0].w || gs[i].g != gs[0].g ||
            gs[i].n_gops != gs[0].n_gops)
            return fail(CS_EINVAL, "every plan's call must describe the same clip shape");
    }
    const GopShape& g0 = gs[0];
    const size_t px = (size_t)g0.h * g0.w;
    const size_t clip_b = px * g0.n_gops * g0.g, keys_b = px * g0.n_gops, cs_b = px * g0.n_cs;
    // staging: clip | keys | CS frames | per plan: y, float frames, uint8 frames, PSNR
    size_t total = up(clip_b) + up(keys_b) + up(cs_b);
    std::vector<size_t> off_y(n_plans), off_f(n_plans), off_u(n_plans), off_p(n_plans);
    for (int i = 0; i < n_plans; ++i) {
        off_y[i] = total;
        total += up((size_t)gs[i].n_cs * gs[i].nblk * gs[i].m * sizeof(float));
        off_f[i] = total;
        total += up(cs_b * sizeof(float));
        off_u[i] = total;
        total += up(cs_b);
        off_p[i] = total;
        total += up((size_t)g0.n_cs * sizeof(double));
    }
    std::lock_guard<std::mutex> lock(ctx->stage_mu);
    CS_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    if (ctx->stage_bytes < total) {
        // the previous holder must be done with the old buffer before it goes
        CS_CUDA_TRY(cudaEventSynchronize(ctx->stage_ring.ev[0]));
        if (ctx->stage) cudaFree(ctx->stage);
        ctx->stage = nullptr;
        ctx->stage_bytes = 0;
        CS_CUDA_TRY(cudaMalloc(&ctx->stage, total));
        ctx->stage_bytes = total;
    }
    int slot = 0;
    CS_CUDA_TRY(slot_take(&ctx->stage_ring, s, &slot));
    uint8_t* base = ctx->stage;
    uint8_t* clip = base;
    uint8_t* keys = base + up(clip_b);
    uint8_t* csf = keys + up(keys_b);
    const size_t gop_b = px * g0.g;
    cudaError_t e = cudaMemcpyAsync(clip, clip_host, clip_b, cudaMemcpyHostToDevice, s);
    // the key of GOP k is frame k G; its CS frames k G + 1 .. k G + G - 1 are contiguous
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(keys, px, clip, gop_b, px, g0.n_gops, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(csf, px * (g0.g - 1), clip + px, gop_b, px * (g0.g - 1), g0.n_gops,
                              cudaMemcpyDeviceToDevice, s);
    int st = e == cudaSuccess ? CS_OK : cuda_fail(e, "cs_codec_host copy-in");
    std::vector<const uint8_t*> key_p(n_plans, keys);
    std::vector<const float*> y_p(n_plans);
    std::vector<float*> f_p(n_plans);
    std::vector<uint8_t*> u_p(n_plans);
    for (int i = 0; i < n_plans; ++i) {
        y_p[i] = reinterpret_cast<const float*>(base + off_y[i]);
        f_p[i] = reinterpret_cast<float*>(base + off_f[i]);
        u_p[i] = base + off_u[i];
    }
    // one pass over the clip for the plans of one block size, else plan by plan
    bool one_b = true;
    for (int i = 1; i < n_plans; ++i) one_b = one_b && gs[i].b == gs[0].b;
    if (st == CS_OK && one_b) {
        std::vector<float*> y_w(n_plans);
        for (int i = 0; i < n_plans; ++i) y_w[i] = const_cast<float*>(y_p[i]);
        st = cs_encode_batch(ctx, n_plans, plans, params, clip, y_w.data(), stream);
    }
    for (int i = 0; st == CS_OK && !one_b && i < n_plans; ++i)
        st = cs_encode_gop(plans[i], &params[i], clip, const_cast<float*>(y_p[i]), stream);
    if (st == CS_OK)
        st = cs_decode_batch(ctx, n_plans, plans, params, key_p.data(), y_p.data(), f_p.data(),
                             u_p.data(), stream);
    for (int i = 0; st == CS_OK && i < n_plans; ++i)
        st = cs_psnr(csf, f_p[i], g0.n_cs, g0.h, g0.w, reinterpret_cast<double*>(base + off_p[i]),
                     stream);
    for (int i = 0; st == CS_OK && i < n_plans; ++i) {
        e = cudaMemcpyAsync(frames_u8_host[i], u_p[i], cs_b, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(psnr_host[i], base + off_p[i], (size_t)g0.n_cs * sizeof(double),
                                cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) st = cuda_fail(e, "cs_codec_host copy-out");
    }
    // the slot is released even on failure: whatever was enqueued runs first
    e = slot_done(&ctx->stage_ring, slot, s);
    if (st == CS_OK && e != cudaSuccess) st = cuda_fail(e, "cs_codec_host");
    return st;
}
