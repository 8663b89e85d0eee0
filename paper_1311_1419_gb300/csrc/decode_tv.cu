// TV recovery of every measured block (Eq. 1 with the total variation, the
// regulariser of the paper's TVAL3 decoder, Sec. 4), followed by the key
// add-back of Eq. (4).  Per block, min ||D r||_1 s.t. Phi r = y by the augmented
// Lagrangian / alternating-direction scheme (Li, Yin, Jiang, Zhang, Comput.
// Optim. Appl. 2013): with the splitting w = D r (D the forward differences
// along rows and columns, zero at the last column / row), each iteration takes
//   w   = shrink(D r - nu / beta, 1 / beta)
//   r  -= alpha (D^T (beta (D r - w) - nu) + Phi^T (mu (Phi r - y) - lam))
//   nu -= beta (D r - w),  lam -= mu (Phi r - y)
// with alpha = 1 / (8 beta + mu L) (8 bounds ||D||^2, L the plan's Lipschitz
// constant of Phi Phi^T), from r = nu = lam = 0, for a fixed count.  This file's
// kernel is the plain one (SIMT FP32, every shape; 16 x 16 blocks with M <= 128
// run on the tensor cores, decode_tc.cu).  It keeps q = nu + beta w instead of
// nu and w: the difference term of the gradient is D^T (beta D r - q) and the
// multiplier step is nu' = q - beta D r', so a block's state is r, r' (the next
// iterate), q (2 N), y, lam and Phi r - y: 4 N + 3 M values, and a CTA recovers
// R blocks (up to 12 of 32 x 32) sharing every load of Phi (read from L2).
#include <math.h>

#include "internal.h"

namespace csvc {

int make_shape(const cs_plan* plan, const cs_params* p, GopShape* gs);

namespace {

__device__ __forceinline__ float shrink(float v, float t) { return v - fminf(fmaxf(v, -t), t); }

// R blocks per CTA of kT threads, JB pixels per thread in the Phi^T product (n =
// JB x kT for 32 x 32 blocks: 512 threads, 2 pixels each; else 256 threads, one
// pixel each).
template <int R, int JB, int kT>
__global__ void __launch_bounds__(kT) k_tv_plain(const float* __restrict__ phi,
                                                 const float* __restrict__ yall,
                                                 const uint8_t* __restrict__ keys,
                                                 float* __restrict__ out_f32,
                                                 uint8_t* __restrict__ out_u8, GopShape gs, int iters,
                                                 float beta, float mu, float alpha) {
    extern __shared__ float sm[];
    const int n = gs.n, m = gs.m, b = gs.b;
    const int mp = (m + 3) & ~3;                // rows of the M-vectors, 16-byte aligned
    float* ra = sm;                             // [R][N] r
    float* rb = ra + R * n;                     // [R][N] the next r
    float* qs = rb + R * n;                     // [R][2N] q: row differences, then column differences
    float* ys = qs + 2 * R * n;                 // [R][mp] y (zero beyond M)
    float* lam = ys + R * mp;                   // [R][mp] multiplier of Phi r = y
    float* rho = lam + R * mp;                  // [R][mp] Phi r - y, then mu (Phi r - y) - lam
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long total = (long long)gs.n_cs * gs.nblk;
    const long long row0 = (long long)blockIdx.x * R;
    for (int e = tid; e < R * n; e += kT) ra[e] = 0.f;
    for (int e = tid; e < 2 * R * n; e += kT) qs[e] = 0.f;
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
        for (int e = tid; e < R * mp; e += kT) rho[e] = mu * rho[e] - lam[e];
        __syncthreads();
        // r' = r - alpha (D^T (beta D r - q) + Phi^T P): the Phi^T P term for the
        // thread's JB pixels of all R blocks, 4 rows of Phi per pass (rows >= m zero)
        for (int j0 = tid; j0 < n; j0 += JB * kT) {
            float g[JB][R];
#pragma unroll
            for (int t = 0; t < JB; ++t)
#pragma unroll
                for (int q = 0; q < R; ++q) g[t][q] = 0.f;
            for (int i = 0; i < m; i += 4) {
                float pv[JB][4];
#pragma unroll
                for (int t = 0; t < JB; ++t)
#pragma unroll
                    for (int rr = 0; rr < 4; ++rr)
                        pv[t][rr] = (i + rr < m && j0 + t * kT < n) ? __ldg(phi + (size_t)(i + rr) * n + j0 + t * kT) : 0.f;
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const float4 pq = *reinterpret_cast<const float4*>(rho + q * mp + i);
#pragma unroll
                    for (int t = 0; t < JB; ++t) {
                        g[t][q] = fmaf(pv[t][0], pq.x, g[t][q]);
                        g[t][q] = fmaf(pv[t][1], pq.y, g[t][q]);
                        g[t][q] = fmaf(pv[t][2], pq.z, g[t][q]);
                        g[t][q] = fmaf(pv[t][3], pq.w, g[t][q]);
                    }
                }
            }
#pragma unroll
            for (int t = 0; t < JB; ++t) {
                const int j = j0 + t * kT;
                if (j >= n) continue;
                const int pr = j / b, pc = j % b;
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const float* rq = ra + q * n;
                    const float* q0 = qs + 2 * q * n;
                    const float* q1 = q0 + n;
                    const float rj = rq[j];
                    // t_h and t_v at j and at the neighbours left and above
                    const float th = pc < b - 1 ? beta * (rq[j + 1] - rj) - q0[j] : 0.f;
                    const float tl = pc > 0 ? beta * (rj - rq[j - 1]) - q0[j - 1] : 0.f;
                    const float tv = pr < b - 1 ? beta * (rq[j + b] - rj) - q1[j] : 0.f;
                    const float tu = pr > 0 ? beta * (rj - rq[j - b]) - q1[j - b] : 0.f;
                    rb[q * n + j] = rj - alpha * (tl - th + tu - tv + g[t][q]);
                }
            }
        }
        __syncthreads();
        float* tmp = ra;
        ra = rb;
        rb = tmp;
        // q' = nu' + beta w' with nu' = q - beta D r', w' = shrink(D r' - nu' / beta, 1 / beta)
        for (int e = tid; e < 2 * R * n; e += kT) {
            const int q = e / (2 * n), e2 = e % (2 * n);
            const float* rq = ra + q * n;
            const int j = e2 < n ? e2 : e2 - n;
            const int pr = j / b, pc = j % b;
            float d = 0.f;
            if (e2 < n) {
                if (pc < b - 1) d = rq[j + 1] - rq[j];
            } else {
                if (pr < b - 1) d = rq[j + b] - rq[j];
            }
            const float nu = qs[e] - beta * d;
            qs[e] = nu + beta * shrink(d - nu * ib, ib);
        }
        // Phi r' - y and lam -= mu (Phi r' - y): a warp takes 4 rows of Phi against
        // the R blocks, its lanes 4 pixels at a time
        for (int i0 = warp * 4; i0 < m; i0 += (kT / 32) * 4) {
            float acc[4][R];
#pragma unroll
            for (int rr = 0; rr < 4; ++rr)
#pragma unroll
                for (int q = 0; q < R; ++q) acc[rr][q] = 0.f;
            const int nrow = m - i0 < 4 ? m - i0 : 4;
            for (int c4 = lane; c4 < n / 4; c4 += 32) {
                float4 pv[4];
#pragma unroll
                for (int rr = 0; rr < 4; ++rr)
                    pv[rr] = rr < nrow ? __ldg(reinterpret_cast<const float4*>(phi + (size_t)(i0 + rr) * n) + c4)
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const float4 rv = *reinterpret_cast<const float4*>(ra + q * n + 4 * c4);
#pragma unroll
                    for (int rr = 0; rr < 4; ++rr) {
                        acc[rr][q] = fmaf(pv[rr].x, rv.x, acc[rr][q]);
                        acc[rr][q] = fmaf(pv[rr].y, rv.y, acc[rr][q]);
                        acc[rr][q] = fmaf(pv[rr].z, rv.z, acc[rr][q]);
                        acc[rr][q] = fmaf(pv[rr].w, rv.w, acc[rr][q]);
                    }
                }
            }
#pragma unroll
            for (int rr = 0; rr < 4; ++rr) {
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    float v = acc[rr][q];
                    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                    if (lane == 0 && rr < nrow) {
                        const int e = q * mp + i0 + rr;
                        const float rh = v - ys[e];
                        rho[e] = rh;
                        lam[e] -= mu * rh;
                    }
                }
            }
        }
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
        const float v = (float)keys[(size_t)g * frame_px + off] + ra[e];
        if (out_f32) out_f32[(size_t)c * frame_px + off] = v;
        if (out_u8) out_u8[(size_t)c * frame_px + off] = (uint8_t)fminf(fmaxf(rintf(v), 0.f), 255.f);
    }
}

size_t tv_smem(int n, int m, int nr) {
    const int mp = (m + 3) & ~3;
    return (size_t)nr * (size_t)(4 * n + 3 * mp) * sizeof(float);
}

template <int R, int JB, int kT>
cudaError_t launch_tv(const float* phi, const float* y, const uint8_t* key, float* f32, uint8_t* u8,
                      const GopShape& gs, int iters, float beta, float mu, float alpha, cudaStream_t s) {
    const size_t smem = tv_smem(gs.n, gs.m, R);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_tv_plain<R, JB, kT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    const long long rows = (long long)gs.n_cs * gs.nblk;
    k_tv_plain<R, JB, kT><<<(unsigned)((rows + R - 1) / R), kT, smem, s>>>(phi, y, key, f32, u8, gs, iters,
                                                                            beta, mu, alpha);
    return cudaGetLastError();
}

template <int R>
cudaError_t launch_tv_r(const float* phi, const float* y, const uint8_t* key, float* f32, uint8_t* u8,
                        const GopShape& gs, int iters, float beta, float mu, float alpha, cudaStream_t s) {
    return gs.n >= 1024 ? launch_tv<R, 2, 512>(phi, y, key, f32, u8, gs, iters, beta, mu, alpha, s)
                        : launch_tv<R, 1, 256>(phi, y, key, f32, u8, gs, iters, beta, mu, alpha, s);
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
    // the on-chip tensor-core kernel (16 x 16 blocks, M <= 128), else the streaming
    // one, else (or when the budget leaves no room for the streaming state) the
    // plain kernel; an explicit engine insists on its kernel
    if (params->engine == CS_ENGINE_TC_CHUNK) return fail(CS_EINVAL, "TV recovery has no chunked tensor-core kernel");
    if ((params->engine == CS_ENGINE_AUTO || params->engine == CS_ENGINE_TC) && tv_tc_supported(plan)) {
        const cudaError_t e = launch_decode_tv_tc(plan, gs, it, beta, mu, alpha, key_dev, y_dev, frames_f32_dev,
                                                  frames_u8_dev, s);
        return e == cudaSuccess ? CS_OK : cuda_fail(e, "cs_decode_gop_tv");
    }
    if (params->engine == CS_ENGINE_TC)
        return fail(CS_EINVAL, "TV recovery's on-chip tensor-core kernel takes 16 x 16 blocks with M <= 128");
    if ((params->engine == CS_ENGINE_AUTO || params->engine == CS_ENGINE_TC_STREAM) && tv_tcs_supported(plan)) {
        const cudaError_t e = launch_decode_tv_tcs(plan, gs, it, beta, mu, alpha, key_dev, y_dev, frames_f32_dev,
                                                   frames_u8_dev, s);
        if (e == cudaSuccess) return CS_OK;
        if (e != cudaErrorMemoryAllocation || params->engine == CS_ENGINE_TC_STREAM)
            return cuda_fail(e, "cs_decode_gop_tv");
    }
    if (params->engine == CS_ENGINE_TC_STREAM)
        return fail(CS_EINVAL, "TV recovery's streaming tensor-core kernel takes N = 64, 256, 1024 with M <= 512");
    if (tv_smem(gs.n, gs.m, 1) > 227 * 1024) return fail(CS_EINVAL, "block too large for the TV kernel");
    // as many blocks per CTA (12 for 32 x 32 blocks, else up to 8: at 12 the
    // 256-thread CTA's registers would allow only two per SM; then 4, 2 or 1) as
    // fit the shared memory and still give every SM two CTAs' worth of work
    int nr = 1;
    for (int r : {12, 8, 4, 2})
        if ((r < 12 || gs.n >= 1024) && tv_smem(gs.n, gs.m, r) <= 227 * 1024 &&
            rows >= 2ll * r * plan->ctx->sm_count) {
            nr = r;
            break;
        }
    cudaError_t e;
    const float* ph = plan->phi;
    switch (nr) {
        case 12: e = launch_tv_r<12>(ph, y_dev, key_dev, frames_f32_dev, frames_u8_dev, gs, it, beta, mu, alpha, s); break;
        case 8: e = launch_tv_r<8>(ph, y_dev, key_dev, frames_f32_dev, frames_u8_dev, gs, it, beta, mu, alpha, s); break;
        case 4: e = launch_tv_r<4>(ph, y_dev, key_dev, frames_f32_dev, frames_u8_dev, gs, it, beta, mu, alpha, s); break;
        case 2: e = launch_tv_r<2>(ph, y_dev, key_dev, frames_f32_dev, frames_u8_dev, gs, it, beta, mu, alpha, s); break;
        default: e = launch_tv_r<1>(ph, y_dev, key_dev, frames_f32_dev, frames_u8_dev, gs, it, beta, mu, alpha, s); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cs_decode_gop_tv");
    return CS_OK;
}
