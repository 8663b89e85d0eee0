// TV recovery of every measured block (Eq. 1 with the total variation, the
// regulariser of the paper's TVAL3 decoder, Sec. 4), followed by the key
// add-back of Eq. (4).  Per block, min ||D r||_1 s.t. Phi r = y by the
// augmented Lagrangian / alternating-direction scheme (Li, Yin, Jiang, Zhang,
// Comput. Optim. Appl. 2013): with the splitting w = D r (D the forward
// differences along rows and columns, zero at the last column / row), each
// iteration takes
//   w   = shrink(D r - nu / beta, 1 / beta)
//   r  -= alpha (D^T (beta (D r - w) - nu) + Phi^T (mu (Phi r - y) - lam))
//   nu -= beta (D r - w),  lam -= mu (Phi r - y)
// with alpha = 1 / (8 beta + mu L) (8 bounds ||D||^2, L the plan's Lipschitz
// constant of Phi Phi^T), from r = nu = lam = 0, for a fixed count.  One CTA
// per block; the residual works in the pixel domain, so the reconstruction is
// the add-back alone.  Phi is read from global memory (L1/L2 resident).
#include <math.h>

#include "internal.h"

namespace csvc {

int make_shape(const cs_plan* plan, const cs_params* p, GopShape* gs);

namespace {

constexpr int kT = 256;

__device__ __forceinline__ float shrink(float v, float t) { return v - fminf(fmaxf(v, -t), t); }

__global__ void __launch_bounds__(kT) k_tv_plain(const float* __restrict__ phi,
                                                 const float* __restrict__ yall,
                                                 const uint8_t* __restrict__ keys,
                                                 float* __restrict__ out_f32,
                                                 uint8_t* __restrict__ out_u8, GopShape gs, int iters,
                                                 float beta, float mu, float alpha) {
    extern __shared__ float sm[];
    const int n = gs.n, m = gs.m, b = gs.b;
    float* r = sm;              // [N] residual block
    float* dr = r + n;          // [2N] D r: row differences, then column differences
    float* nu = dr + 2 * n;     // [2N] multiplier of D r = w
    float* wv = nu + 2 * n;     // [2N] w
    float* tv = wv + 2 * n;     // [2N] beta (D r - w) - nu
    float* ys = tv + 2 * n;     // [M]
    float* lam = ys + m;        // [M] multiplier of Phi r = y
    float* rho = lam + m;       // [M] Phi r - y, then mu rho - lam
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long row = blockIdx.x;
    const float* y = yall + row * m;
    for (int i = tid; i < n; i += kT) r[i] = 0.f;
    for (int e = tid; e < 2 * n; e += kT) dr[e] = nu[e] = 0.f;
    for (int i = tid; i < m; i += kT) {
        ys[i] = y[i];
        lam[i] = 0.f;
        rho[i] = -y[i];
    }
    __syncthreads();
    const float ib = 1.f / beta;
    for (int k = 0; k < iters; ++k) {
        // w-step and the difference-side term of the gradient
        for (int e = tid; e < 2 * n; e += kT) {
            const float w = shrink(dr[e] - nu[e] * ib, ib);
            wv[e] = w;
            tv[e] = beta * (dr[e] - w) - nu[e];
        }
        for (int i = tid; i < m; i += kT) rho[i] = mu * rho[i] - lam[i];
        __syncthreads();
        // r-step: one gradient step of length alpha
        for (int j = tid; j < n; j += kT) {
            const int pr = j / b, pc = j % b;
            float g = 0.f;
            if (pc > 0) g += tv[j - 1];
            if (pc < b - 1) g -= tv[j];
            if (pr > 0) g += tv[n + j - b];
            if (pr < b - 1) g -= tv[n + j];
            for (int i = 0; i < m; ++i) g = fmaf(phi[(size_t)i * n + j], rho[i], g);
            r[j] -= alpha * g;
        }
        __syncthreads();
        // D r and Phi r - y at the new r
        for (int e = tid; e < 2 * n; e += kT) {
            const int j = e < n ? e : e - n;
            const int pr = j / b, pc = j % b;
            float v = 0.f;
            if (e < n) {
                if (pc < b - 1) v = r[j + 1] - r[j];
            } else {
                if (pr < b - 1) v = r[j + b] - r[j];
            }
            dr[e] = v;
        }
        for (int i = warp; i < m; i += kT / 32) {
            const float* prow = phi + (size_t)i * n;
            float acc = 0.f;
            for (int col = lane; col < n; col += 32) acc = fmaf(prow[col], r[col], acc);
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if (lane == 0) rho[i] = acc - ys[i];
        }
        __syncthreads();
        // multipliers (each entry by the thread that reads it in the next w-step)
        for (int e = tid; e < 2 * n; e += kT) nu[e] -= beta * (dr[e] - wv[e]);
        for (int i = tid; i < m; i += kT) lam[i] -= mu * rho[i];
        __syncthreads();
    }
    // add back the key (Eq. 4), crop
    const int c = (int)(row / gs.nblk), blk = (int)(row % gs.nblk);
    const int g = c / (gs.g - 1);
    const int bi = blk / gs.nbc, bj = blk % gs.nbc;
    const size_t frame_px = (size_t)gs.h * gs.w;
    for (int j = tid; j < n; j += kT) {
        const int py = bi * b + j / b, px = bj * b + j % b;
        if (py >= gs.h || px >= gs.w) continue;
        const size_t off = (size_t)py * gs.w + px;
        const float v = (float)keys[(size_t)g * frame_px + off] + r[j];
        if (out_f32) out_f32[(size_t)c * frame_px + off] = v;
        if (out_u8) out_u8[(size_t)c * frame_px + off] = (uint8_t)fminf(fmaxf(rintf(v), 0.f), 255.f);
    }
}

}  // namespace
}  // namespace csvc

using namespace csvc;

extern "C" int cs_decode_gop_tv(cs_plan* plan, const cs_params* params, float beta, float mu,
                                const uint8_t* key_dev, const float* y_dev, float* frames_f32_dev,
                                uint8_t* frames_u8_dev, cs_stream_t stream) {
    if (!plan || !params) return fail(CS_EINVAL, "null argument");
    if (!(beta > 0.f) || !(mu > 0.f) || !isfinite(beta) || !isfinite(mu))
        return fail(CS_EINVAL, "beta and mu must be finite and > 0");
    if (params->iters < 0 || params->iters > kMaxIters) return fail(CS_EINVAL, "iters out of range");
    if (params->precision != CS_FP32) return fail(CS_EINVAL, "TV recovery computes in FP32 only");
    if (params->engine == CS_ENGINE_TC || params->engine == CS_ENGINE_TC_STREAM)
        return fail(CS_EINVAL, "TV recovery has no tensor-core kernel");
    GopShape gs;
    int st = make_shape(plan, params, &gs);
    if (st) return st;
    if (!frames_f32_dev && !frames_u8_dev) return fail(CS_EINVAL, "both outputs are NULL");
    const long long rows = (long long)gs.n_cs * gs.nblk;
    if (rows == 0) return CS_OK;
    if (!key_dev || !y_dev) return fail(CS_EINVAL, "null input pointer");
    const size_t smem = (size_t)(9 * gs.n + 3 * gs.m) * sizeof(float);
    if (smem > 227 * 1024) return fail(CS_EINVAL, "block too large for the TV kernel");
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_tv_plain, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return cuda_fail(e, "cs_decode_gop_tv");
    }
    const float alpha = (float)(1.0 / (8.0 * (double)beta + (double)mu * plan->lipschitz));
    k_tv_plain<<<(unsigned)rows, kT, smem, (cudaStream_t)stream>>>(
        plan->phi, y_dev, key_dev, frames_f32_dev, frames_u8_dev, gs, params->iters, beta, mu, alpha);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "cs_decode_gop_tv");
    return CS_OK;
}
