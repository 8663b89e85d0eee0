// K5 + K7: plain FP32 per-block decode.  One CTA recovers one measured block
// by fixed-count FISTA on 1/2 ||A s - y||^2 + lambda ||s||_1 (Eq. 1 with an
// l1 regulariser in the DCT basis; Beck & Teboulle 2009), then reconstructs
// the residual r = Psi s (separable inverse DCT, R = C^T S C) and adds it back
// to the GOP's key frame (Eq. 4).  A is read from global memory (L1/L2
// resident) every iteration; the iterates stay in registers and shared memory.
// This kernel is the simple SIMT baseline of the decode, and the path for the
// (N, M) shapes the tensor-core kernel does not take.  Its thread count per
// block (T) is a launch-time choice: the autotuner times the candidates.
#include "internal.h"

namespace csvc {
namespace {

__device__ __forceinline__ float soft_threshold(float v, float tau) {
    return v - fminf(fmaxf(v, -tau), tau);
}

template <int T, int PER>
__global__ void __launch_bounds__(T) k_fista_plain(
    const float* __restrict__ a, const float* __restrict__ dct, const float* __restrict__ yall,
    const uint8_t* __restrict__ keys, float* __restrict__ out_f32, uint8_t* __restrict__ out_u8,
    GopShape gs, int iters, float lambda_rel, float inv_l, const float* __restrict__ beta) {
    extern __shared__ float sm[];
    const int n = gs.n, m = gs.m, b = gs.b;
    float* zs = sm;           // [N] current z (then s^K for recon)
    float* rho = zs + n;      // [M] A z - y
    float* ys = rho + m;      // [M]
    float* cs = ys + m;       // [B][B] DCT matrix
    float* tmp = cs + b * b;  // [N] recon scratch
    __shared__ float red[T / 32];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long r = blockIdx.x;
    const float* y = yall + r * m;
    for (int i = tid; i < m; i += T) ys[i] = y[i];
    for (int i = tid; i < b * b; i += T) cs[i] = dct[i];
    for (int i = tid; i < n; i += T) zs[i] = 0.f;
    for (int i = tid; i < m; i += T) rho[i] = ys[i];
    __syncthreads();

    // lambda_b = lambda_rel * ||A^T y||_inf
    float amax = 0.f;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int col = tid + j * T;
        if (col < n) {
            float g = 0.f;
            for (int i = 0; i < m; ++i) g = fmaf(a[(size_t)i * n + col], rho[i], g);
            amax = fmaxf(amax, fabsf(g));
        }
    }
    for (int off = 16; off > 0; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, off));
    if (lane == 0) red[warp] = amax;
    __syncthreads();
    amax = 0.f;
    for (int w = 0; w < T / 32; ++w) amax = fmaxf(amax, red[w]);
    const float tau = lambda_rel * amax * inv_l;

    float z[PER], sp[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) z[j] = sp[j] = 0.f;

    for (int k = 0; k < iters; ++k) {
        // rho = A z - y, one warp per measurement row
        for (int i = warp; i < m; i += T / 32) {
            const float* arow = a + (size_t)i * n;
            float acc = 0.f;
            for (int col = lane; col < n; col += 32) acc = fmaf(arow[col], zs[col], acc);
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if (lane == 0) rho[i] = acc - ys[i];
        }
        __syncthreads();
        const float bk = beta[k];
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const int col = tid + j * T;
            if (col < n) {
                float g = 0.f;
                for (int i = 0; i < m; ++i) g = fmaf(a[(size_t)i * n + col], rho[i], g);
                const float s = soft_threshold(z[j] - g * inv_l, tau);
                z[j] = s + bk * (s - sp[j]);
                sp[j] = s;
                zs[col] = z[j];  // every read of zs happened before the barrier above
            }
        }
        __syncthreads();
    }

    // recon: S = s^K as B x B, T = S C, R = C^T T
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int col = tid + j * T;
        if (col < n) zs[col] = sp[j];
    }
    __syncthreads();
    for (int idx = tid; idx < n; idx += T) {
        const int k = idx / b, q = idx % b;
        float acc = 0.f;
        for (int l = 0; l < b; ++l) acc = fmaf(zs[k * b + l], cs[l * b + q], acc);
        tmp[idx] = acc;
    }
    __syncthreads();
    const int c = (int)(r / gs.nblk), blk = (int)(r % gs.nblk);
    const int g = c / (gs.g - 1);
    const int bi = blk / gs.nbc, bj = blk % gs.nbc;
    const size_t frame_px = (size_t)gs.h * gs.w;
    for (int idx = tid; idx < n; idx += T) {
        const int p = idx / b, q = idx % b;
        const int py = bi * b + p, px = bj * b + q;
        if (py >= gs.h || px >= gs.w) continue;
        float acc = 0.f;
        for (int k = 0; k < b; ++k) acc = fmaf(cs[k * b + p], tmp[k * b + q], acc);
        const size_t off = (size_t)py * gs.w + px;
        const float v = (float)keys[(size_t)g * frame_px + off] + acc;
        if (out_f32) out_f32[(size_t)c * frame_px + off] = v;
        if (out_u8) out_u8[(size_t)c * frame_px + off] = (uint8_t)fminf(fmaxf(rintf(v), 0.f), 255.f);
    }
}

template <int T, int PER>
cudaError_t launch_per(const DecodeArgs& d, size_t smem, long long rows, cudaStream_t s) {
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_fista_plain<T, PER>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const float inv_l = (float)(1.0 / d.plan->lipschitz);
    k_fista_plain<T, PER><<<(unsigned)rows, T, smem, s>>>(
        d.plan->a, d.plan->dct, d.y, d.key, d.out_f32, d.out_u8, d.gs, d.iters, d.lambda_rel,
        inv_l, d.beta);
    return cudaGetLastError();
}

template <int T>
cudaError_t launch_threads(const DecodeArgs& d, size_t smem, long long rows, cudaStream_t s) {
    const int per = (d.gs.n + T - 1) / T;
    if (per <= 1) return launch_per<T, 1>(d, smem, rows, s);
    if (per <= 2) return launch_per<T, 2>(d, smem, rows, s);
    if (per <= 4) return launch_per<T, 4>(d, smem, rows, s);
    if (per <= 8) return launch_per<T, 8>(d, smem, rows, s);
    if (per <= 16) return launch_per<T, 16>(d, smem, rows, s);
    return cudaErrorInvalidValue;
}

}  // namespace

bool plain_threads_valid(int threads, int n) {
    return (threads == 64 || threads == 128 || threads == 256 || threads == 512 ||
            threads == 1024) && (n + threads - 1) / threads <= 16;
}

int plain_threads_default(int n) { return n <= 64 ? 64 : n <= 4096 ? 256 : 1024; }

cudaError_t launch_decode_plain(const DecodeArgs& d, cudaStream_t s) {
    const GopShape& gs = d.gs;
    const long long rows = (long long)gs.n_cs * gs.nblk;
    if (rows == 0) return cudaSuccess;
    const size_t smem = (size_t)(2 * gs.n + 2 * gs.m + gs.b * gs.b) * sizeof(float);
    const int t = d.plain_threads ? d.plain_threads : plain_threads_default(gs.n);
    if (!plain_threads_valid(t, gs.n)) return cudaErrorInvalidValue;
    switch (t) {
        case 64: return launch_threads<64>(d, smem, rows, s);
        case 128: return launch_threads<128>(d, smem, rows, s);
        case 256: return launch_threads<256>(d, smem, rows, s);
        case 512: return launch_threads<512>(d, smem, rows, s);
        default: return launch_threads<1024>(d, smem, rows, s);
    }
}

}  // namespace csvc
