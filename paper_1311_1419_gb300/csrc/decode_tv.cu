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
// constant of Phi Phi^T), from r = nu = lam = 0, for a fixed count.  A CTA
// recovers R blocks with their state in shared memory; the residual works in
// the pixel domain, so the reconstruction is the add-back alone.  Phi is read
// from global memory (L1/L2 resident), once per R blocks.
#include <math.h>

#include "internal.h"

namespace csvc {

int make_shape(const cs_plan* plan, const cs_params* p, GopShape* gs);

namespace {

constexpr int kT = 256;

__device__ __forceinline__ float shrink(float v, float t) { return v - fminf(fmaxf(v, -t), t); }

// R blocks per CTA share every load of Phi (the two Phi products are each
// register-blocked: 4 rows of Phi against the R blocks' vectors per pass), and
// each block's iteration is the one above.
template <int R>
__global__ void __launch_bounds__(kT) k_tv_plain(const float* __restrict__ phi,
                                                 const float* __restrict__ yall,
                                                 const uint8_t* __restrict__ keys,
                                                 float* __restrict__ out_f32,
                                                 uint8_t* __restrict__ out_u8, GopShape gs, int iters,
                                                 float beta, float mu, float alpha) {
    extern __shared__ float sm[];
    const int n = gs.n, m = gs.m, b = gs.b;
    const int mp = (m + 3) & ~3;                // rows of the M-vectors, 16-byte aligned
    float* r = sm;                  // [R][N] residual blocks
    float* dr = r + R * n;          // [R][2N] D r: row differences, then column differences
    float* nu = dr + 2 * R * n;     // [R][2N] multiplier of D r = w
    float* wv = nu + 2 * R * n;     // [R][2N] w
    float* tv = wv + 2 * R * n;     // [R][2N] beta (D r - w) - nu
    float* ys = sm + ((9 * R * n + 3) & ~3);    // [R][mp] y (zero beyond M)
    float* lam = ys + R * mp;       // [R][mp] multiplier of Phi r = y
    float* rho = lam + R * mp;      // [R][mp] Phi r - y, then mu rho - lam
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long total = (long long)gs.n_cs * gs.nblk;
    const long long row0 = (long long)blockIdx.x * R;
    for (int e = tid; e < R * n; e += kT) r[e] = 0.f;
    for (int e = tid; e < 2 * R * n; e += kT) dr[e] = nu[e] = 0.f;
    for (int e = tid; e < R * mp; e += kT) {
        const int q = e / mp, i = e % mp;
        // blocks beyond the call's last measure nothing: their iterates stay 0
        const float v = (i < m && row0 + q < total) ? yall[(row0 + q) * m + i] : 0.f;
        ys[e] = v;
        lam[e] = 0.f;
        rho[e] = -v;
    }
    __syncthreads();
    const float ib = 1.f / beta;
    for (int k = 0; k < iters; ++k) {
        // w-step and the difference-side term of the gradient
        for (int e = tid; e < 2 * R * n; e += kT) {
            const float w = shrink(dr[e] - nu[e] * ib, ib);
            wv[e] = w;
            tv[e] = beta * (dr[e] - w) - nu[e];
        }
        for (int e = tid; e < R * mp; e += kT) rho[e] = mu * rho[e] - lam[e];
        __syncthreads();
        // r-step: one gradient step of length alpha; D^T tv, then Phi^T rho, 4 rows of
        // Phi per pass against every block's rho (rows m .. mp - 1 of rho are zero)
        for (int j = tid; j < n; j += kT) {
            const int pr = j / b, pc = j % b;
            float g[R];
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const float* t = tv + 2 * q * n;
                float v = 0.f;
                if (pc > 0) v += t[j - 1];
                if (pc < b - 1) v -= t[j];
                if (pr > 0) v += t[n + j - b];
                if (pr < b - 1) v -= t[n + j];
                g[q] = v;
            }
            for (int i = 0; i < m; i += 4) {
                float pv[4];
#pragma unroll
                for (int rr = 0; rr < 4; ++rr) pv[rr] = i + rr < m ? phi[(size_t)(i + rr) * n + j] : 0.f;
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const float4 rv = *reinterpret_cast<const float4*>(rho + q * mp + i);
                    g[q] = fmaf(pv[0], rv.x, g[q]);
                    g[q] = fmaf(pv[1], rv.y, g[q]);
                    g[q] = fmaf(pv[2], rv.z, g[q]);
                    g[q] = fmaf(pv[3], rv.w, g[q]);
                }
            }
#pragma unroll
            for (int q = 0; q < R; ++q) r[q * n + j] -= alpha * g[q];
        }
        __syncthreads();
        // D r at the new r
        for (int e = tid; e < 2 * R * n; e += kT) {
            const int q = e / (2 * n), e2 = e % (2 * n);
            const float* rq = r + q * n;
            const int j = e2 < n ? e2 : e2 - n;
            const int pr = j / b, pc = j % b;
            float v = 0.f;
            if (e2 < n) {
                if (pc < b - 1) v = rq[j + 1] - rq[j];
            } else {
                if (pr < b - 1) v = rq[j + b] - rq[j];
            }
            dr[e] = v;
        }
        // Phi r - y at the new r: a warp takes 4 rows of Phi against the R blocks
        for (int i0 = warp * 4; i0 < m; i0 += (kT / 32) * 4) {
            float acc[4][R];
#pragma unroll
            for (int rr = 0; rr < 4; ++rr)
#pragma unroll
                for (int q = 0; q < R; ++q) acc[rr][q] = 0.f;
            const int nrow = m - i0 < 4 ? m - i0 : 4;
            for (int col = lane; col < n; col += 32) {
                float rv[R];
#pragma unroll
                for (int q = 0; q < R; ++q) rv[q] = r[q * n + col];
#pragma unroll
                for (int rr = 0; rr < 4; ++rr) {
                    if (rr < nrow) {
                        const float pv = phi[(size_t)(i0 + rr) * n + col];
#pragma unroll
                        for (int q = 0; q < R; ++q) acc[rr][q] = fmaf(pv, rv[q], acc[rr][q]);
                    }
                }
            }
#pragma unroll
            for (int rr = 0; rr < 4; ++rr) {
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    float v = acc[rr][q];
                    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                    if (lane == 0 && rr < nrow) rho[q * mp + i0 + rr] = v - ys[q * mp + i0 + rr];
                }
            }
        }
        __syncthreads();
        // multipliers (each entry by the thread that reads it in the next w-step)
        for (int e = tid; e < 2 * R * n; e += kT) nu[e] -= beta * (dr[e] - wv[e]);
        for (int e = tid; e < R * mp; e += kT) lam[e] -= mu * rho[e];
        __syncthreads();
    }
    // add back the key (Eq. 4), crop
    const size_t frame_px = (size_t)gs.h * gs.w;
    for (int e = tid; e < R * n; e += kT) {
        const int q = e / n, j = e % n;
        const long long row = row0 + q;
        if (row >= total) continue;
        const int c = (int)(row / gs.nblk), blk = (int)(row % gs.nblk);
        const int g = c / (gs.g - 1);
        const int bi = blk / gs.nbc, bj = blk % gs.nbc;
        const int py = bi * b + j / b, px = bj * b + j % b;
        if (py >= gs.h || px >= gs.w) continue;
        const size_t off = (size_t)py * gs.w + px;
        const float v = (float)keys[(size_t)g * frame_px + off] + r[e];
        if (out_f32) out_f32[(size_t)c * frame_px + off] = v;
        if (out_u8) out_u8[(size_t)c * frame_px + off] = (uint8_t)fminf(fmaxf(rintf(v), 0.f), 255.f);
    }
}

size_t tv_smem(int n, int m, int nr) {
    const int mp = (m + 3) & ~3;
    return (size_t)(((9 * nr * n + 3) & ~3) + 3 * nr * mp) * sizeof(float);
}

template <int R>
cudaError_t launch_tv(const float* phi, const float* y, const uint8_t* key, float* f32, uint8_t* u8,
                      const GopShape& gs, int iters, float beta, float mu, float alpha, cudaStream_t s) {
    const size_t smem = tv_smem(gs.n, gs.m, R);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_tv_plain<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    const long long rows = (long long)gs.n_cs * gs.nblk;
    k_tv_plain<R><<<(unsigned)((rows + R - 1) / R), kT, smem, s>>>(phi, y, key, f32, u8, gs, iters, beta,
                                                                    mu, alpha);
    return cudaGetLastError();
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
    if (params->engine == CS_ENGINE_TC_STREAM)
        return fail(CS_EINVAL, "TV recovery has no streaming tensor-core kernel");
    GopShape gs;
    int st = make_shape(plan, params, &gs);
    if (st) return st;
    if (!frames_f32_dev && !frames_u8_dev) return fail(CS_EINVAL, "both outputs are NULL");
    const long long rows = (long long)gs.n_cs * gs.nblk;
    if (rows == 0) return CS_OK;
    if (!key_dev || !y_dev) return fail(CS_EINVAL, "null input pointer");
    const float alpha = (float)(1.0 / (8.0 * (double)beta + (double)mu * plan->lipschitz));
    cudaStream_t s = (cudaStream_t)stream;
    const int it = params->iters;
    if (params->engine != CS_ENGINE_PLAIN && tv_tc_supported(plan)) {
        const cudaError_t e = launch_decode_tv_tc(plan, gs, it, beta, mu, alpha, key_dev, y_dev, frames_f32_dev,
                                                  frames_u8_dev, s);
        return e == cudaSuccess ? CS_OK : cuda_fail(e, "cs_decode_gop_tv");
    }
    if (params->engine == CS_ENGINE_TC)
        return fail(CS_EINVAL, "TV recovery's tensor-core kernel takes 16 x 16 blocks with M <= 128");
    if (tv_smem(gs.n, gs.m, 1) > 227 * 1024) return fail(CS_EINVAL, "block too large for the TV kernel");
    // as many blocks per CTA (8, 4, 2 or 1) as keep the state under 100 KB, so that
    // two CTAs share an SM
    int nr = 1;
    for (int r : {8, 4, 2})
        if (tv_smem(gs.n, gs.m, r) <= 100 * 1024) {
            nr = r;
            break;
        }
    cudaError_t e;
    switch (nr) {
        case 8: e = launch_tv<8>(plan->phi, y_dev, key_dev, frames_f32_dev, frames_u8_dev, gs, it, beta, mu, alpha, s); break;
        case 4: e = launch_tv<4>(plan->phi, y_dev, key_dev, frames_f32_dev, frames_u8_dev, gs, it, beta, mu, alpha, s); break;
        case 2: e = launch_tv<2>(plan->phi, y_dev, key_dev, frames_f32_dev, frames_u8_dev, gs, it, beta, mu, alpha, s); break;
        default: e = launch_tv<1>(plan->phi, y_dev, key_dev, frames_f32_dev, frames_u8_dev, gs, it, beta, mu, alpha, s); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cs_decode_gop_tv");
    return CS_OK;
}
