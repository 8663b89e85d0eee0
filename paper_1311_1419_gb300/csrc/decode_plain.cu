// K5 + K7: plain FP32 decode.  A CTA recovers R measured blocks by
// fixed-count FISTA on 1/2 ||A s - y||^2 + lambda ||s||_1 (Eq. 1 with an l1
// regulariser in the DCT basis; Beck & Teboulle 2009), then reconstructs each
// residual r = Psi s (separable inverse DCT, R = C^T S C) and adds it back to
// its GOP's key frame (Eq. 4).  A is read from global memory (L2 resident)
// every iteration, once for all R blocks of the CTA: each loaded element of A
// feeds R multiply-adds, so R divides the L2 traffic of A, which dominates
// once A (M x N floats) no longer fits L1.  The iterates of the R blocks live
// in shared memory.  This kernel is the simple SIMT baseline of the decode
// and the path of the (N, M) shapes the tensor-core kernels do not take; its
// launch shape (threads per CTA T, blocks per CTA R = 1, 2, 4, 8 or 16) is
// chosen by the autotuner.
#include <math.h>

#include "internal.h"

namespace csvc {
namespace {


__device__ __forceinline__ float soft_threshold(float v, float tau) {
    return v - fminf(fmaxf(v, -tau), tau);
}

template <int T, int R>
__global__ void __launch_bounds__(T) k_fista_plain(
    const float* __restrict__ a, const float* __restrict__ dct, const float* __restrict__ yall,
    const uint8_t* __restrict__ keys, float* __restrict__ out_f32, uint8_t* __restrict__ out_u8,
    GopShape gs, int iters, float lambda_rel, float inv_l, const float* __restrict__ beta) {
    constexpr int nr = R;
    extern __shared__ float sm[];
    const int n = gs.n, m = gs.m, b = gs.b;
    const int mp = (m + 3) & ~3;  // row stride of rho / ys: 16-byte aligned rows
    float* zs = sm;               // [R][N] current z (then s^K for recon)
    float* sps = zs + nr * n;     // [R][N] s^{k-1}
    float* rho = sm + ((2 * nr * n + 3) & ~3);   // [R][mp] A z - y (zero beyond M), 16-byte aligned
    float* ys = rho + nr * mp;    // [R][mp]
    float* cs = ys + nr * mp;     // [B][B] DCT matrix
    float* tmp = zs;              // recon scratch: T = S C over z once s^K is in sps
    __shared__ float red[R][T / 32];
    __shared__ float taus[R];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long total = (long long)gs.n_cs * gs.nblk;
    const long long row0 = (long long)blockIdx.x * nr;
    // blocks beyond the call's last measure nothing (y = 0): their iterates stay 0
    for (int e = tid; e < nr * mp; e += T) {
        const int q = e / mp, i = e % mp;
        const float v = (i < m && row0 + q < total) ? yall[(row0 + q) * m + i] : 0.f;
        ys[e] = v;
        rho[e] = v;
    }
    for (int i = tid; i < b * b; i += T) cs[i] = dct[i];
    for (int e = tid; e < nr * n; e += T) zs[e] = sps[e] = 0.f;
    __syncthreads();

    // lambda_b = lambda_rel * ||A^T y_b||_inf
    {
        float amax[R];
#pragma unroll
        for (int q = 0; q < R; ++q) amax[q] = 0.f;
        for (int col = tid; col < n; col += T) {
            float g[R];
#pragma unroll
            for (int q = 0; q < R; ++q) g[q] = 0.f;
            for (int i = 0; i < m; ++i) {
                const float av = a[(size_t)i * n + col];
#pragma unroll
                for (int q = 0; q < R; ++q) g[q] = fmaf(av, rho[q * mp + i], g[q]);
            }
#pragma unroll
            for (int q = 0; q < R; ++q) amax[q] = fmaxf(amax[q], fabsf(g[q]));
        }
#pragma unroll
        for (int q = 0; q < R; ++q) {
            float v = amax[q];
            for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
            if (lane == 0) red[q][warp] = v;
        }
        __syncthreads();
        if (tid < nr) {
            float v = 0.f;
            for (int w = 0; w < T / 32; ++w) v = fmaxf(v, red[tid][w]);
            taus[tid] = lambda_rel * v * inv_l;
        }
        __syncthreads();
    }

    for (int k = 0; k < iters; ++k) {
        // rho = A z - y: a warp takes 4 measurement rows at a time, so each value
        // of z loaded from shared memory feeds 4 rows x R blocks of multiply-adds
        for (int i0 = warp * 4; i0 < m; i0 += (T / 32) * 4) {
            float acc[4][R];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < R; ++q) acc[r][q] = 0.f;
            const int nrow = m - i0 < 4 ? m - i0 : 4;
            for (int col = lane; col < n; col += 32) {
                float zv[R];
#pragma unroll
                for (int q = 0; q < R; ++q) zv[q] = zs[q * n + col];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    if (r < nrow) {
                        const float av = a[(size_t)(i0 + r) * n + col];
#pragma unroll
                        for (int q = 0; q < R; ++q) acc[r][q] = fmaf(av, zv[q], acc[r][q]);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    float v = acc[r][q];
                    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                    if (lane == 0 && r < nrow) rho[q * mp + i0 + r] = v - ys[q * mp + i0 + r];
                }
            }
        }
        __syncthreads();
        const float bk = beta[k];
        for (int col = tid; col < n; col += T) {
            float g[R];
#pragma unroll
            for (int q = 0; q < R; ++q) g[q] = 0.f;
            // 4 rows of rho per 16-byte (broadcast) load; rows m .. mp - 1 of rho are
            // zero, and A is read only below m
            for (int i = 0; i < m; i += 4) {
                float av[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) av[r] = i + r < m ? a[(size_t)(i + r) * n + col] : 0.f;
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const float4 rv = *reinterpret_cast<const float4*>(rho + q * mp + i);
                    g[q] = fmaf(av[0], rv.x, g[q]);
                    g[q] = fmaf(av[1], rv.y, g[q]);
                    g[q] = fmaf(av[2], rv.z, g[q]);
                    g[q] = fmaf(av[3], rv.w, g[q]);
                }
            }
#pragma unroll
            for (int q = 0; q < R; ++q) {
                // every read of zs happened before the barrier above
                const float s = soft_threshold(zs[q * n + col] - g[q] * inv_l, taus[q]);
                zs[q * n + col] = s + bk * (s - sps[q * n + col]);
                sps[q * n + col] = s;
            }
        }
        __syncthreads();
    }

    // recon: S = s^K as B x B, T = S C (into zs), R = C^T T
    for (int e = tid; e < nr * n; e += T) {
        const int q = e / n, idx = e % n;
        const int kk = idx / b, qq = idx % b;
        const float* srow = sps + q * n + kk * b;
        float acc = 0.f;
        for (int l = 0; l < b; ++l) acc = fmaf(srow[l], cs[l * b + qq], acc);
        tmp[e] = acc;
    }
    __syncthreads();
    const size_t frame_px = (size_t)gs.h * gs.w;
    for (int e = tid; e < nr * n; e += T) {
        const int q = e / n, idx = e % n;
        const long long r = row0 + q;
        if (r >= total) continue;
        const int c = (int)(r / gs.nblk), blk = (int)(r % gs.nblk);
        const int g = c / (gs.g - 1);
        const int bi = blk / gs.nbc, bj = blk % gs.nbc;
        const int p = idx / b, qq = idx % b;
        const int py = bi * b + p, px = bj * b + qq;
        if (py >= gs.h || px >= gs.w) continue;
        float acc = 0.f;
        for (int kk = 0; kk < b; ++kk) acc = fmaf(cs[kk * b + p], tmp[q * n + kk * b + qq], acc);
        const size_t off = (size_t)py * gs.w + px;
        const float v = (float)keys[(size_t)g * frame_px + off] + acc;
        if (out_f32) out_f32[(size_t)c * frame_px + off] = v;
        if (out_u8) out_u8[(size_t)c * frame_px + off] = (uint8_t)fminf(fmaxf(rintf(v), 0.f), 255.f);
    }
}

template <int T, int R>
cudaError_t launch_tr(const DecodeArgs& d, size_t smem, long long rows, cudaStream_t s) {
    // the opt-in covers dynamic + static shared memory (red, taus: under 2 KB)
    if (smem + 2048 > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_fista_plain<T, R>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const float inv_l = (float)(1.0 / d.plan->lipschitz);
    const long long ctas = (rows + R - 1) / R;
    k_fista_plain<T, R><<<(unsigned)ctas, T, smem, s>>>(d.plan->a, d.plan->dct, d.y, d.key, d.out_f32,
                                                        d.out_u8, d.gs, d.iters, d.lambda_rel, inv_l,
                                                        d.beta);
    return cudaGetLastError();
}

template <int T>
cudaError_t launch_t(const DecodeArgs& d, int nr, size_t smem, long long rows, cudaStream_t s) {
    switch (nr) {
        case 1: return launch_tr<T, 1>(d, smem, rows, s);
        case 2: return launch_tr<T, 2>(d, smem, rows, s);
        case 4: return launch_tr<T, 4>(d, smem, rows, s);
        case 8: return launch_tr<T, 8>(d, smem, rows, s);
        default: return launch_tr<T, 16>(d, smem, rows, s);
    }
}

size_t plain_smem(int n, int m, int b, int nr) {
    const int mp = (m + 3) & ~3;
    return (size_t)(((2 * nr * n + 3) & ~3) + 2 * nr * mp + b * b) * sizeof(float);
}

}  // namespace

bool plain_shape_valid(int threads, int blocks_per_cta, int n, int m) {
    const int b = (int)lround(sqrt((double)n));
    return (threads == 64 || threads == 128 || threads == 256 || threads == 512 || threads == 1024) &&
           (blocks_per_cta == 1 || blocks_per_cta == 2 || blocks_per_cta == 4 || blocks_per_cta == 8 ||
            (blocks_per_cta == 16 && threads <= 512)) &&
           plain_smem(n, m, b, blocks_per_cta) <= 200 * 1024;
}

bool plain_threads_valid(int threads, int n) { return plain_shape_valid(threads, 1, n, 1); }

int plain_threads_default(int n) { return n >= 1024 ? 1024 : n >= 256 ? 256 : 128; }

// The launch shape of an (N, M) that cs_autotune has not timed: as many blocks
// per CTA as shared memory allows (up to 8, or 16 when A reaches 256 KB and L2
// bandwidth bounds the kernel).
static int plain_blocks_default(int t, int n, int m) {
    if ((long long)n * m >= 65536 && plain_shape_valid(t <= 512 ? t : 512, 16, n, m)) return 16;
    for (int r : {8, 4, 2})
        if (plain_shape_valid(t, r, n, m)) return r;
    return 1;
}

void plain_default_shape(int n, int m, int* threads, int* blocks_per_cta) {
    int t = plain_threads_default(n);
    const int nr = plain_blocks_default(t, n, m);
    if (nr == 16 && t > 512) t = 512;
    *threads = t;
    *blocks_per_cta = nr;
}

cudaError_t launch_decode_plain(const DecodeArgs& d, cudaStream_t s) {
    const GopShape& gs = d.gs;
    const long long rows = (long long)gs.n_cs * gs.nblk;
    if (rows == 0) return cudaSuccess;
    int t = d.plain_threads ? d.plain_threads : plain_threads_default(gs.n);
    const int nr = d.plain_blocks ? d.plain_blocks : plain_blocks_default(t, gs.n, gs.m);
    if (!d.plain_threads && nr == 16 && t > 512) t = 512;
    if (!plain_shape_valid(t, nr, gs.n, gs.m)) return cudaErrorInvalidValue;
    const size_t smem = plain_smem(gs.n, gs.m, gs.b, nr);
    switch (t) {
        case 64: return launch_t<64>(d, nr, smem, rows, s);
        case 128: return launch_t<128>(d, nr, smem, rows, s);
        case 256: return launch_t<256>(d, nr, smem, rows, s);
        case 512: return launch_t<512>(d, nr, smem, rows, s);
        default: return launch_t<1024>(d, nr, smem, rows, s);
    }
}

}  // namespace csvc
