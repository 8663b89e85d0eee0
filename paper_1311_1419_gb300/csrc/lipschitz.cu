// The FISTA step constant of a plan: L = 1.0001 * lambda_max(A^T A) and, Psi
// being orthonormal, lambda_max(A^T A) = lambda_max(Phi Phi^T), the largest
// eigenvalue of the M x M Gram matrix G, by FP64 power iteration (1000 steps
// from v0 = 1/sqrt(M), then the Rayleigh quotient v^T G v).
//
// FP64 is scarce on this part (a few FP64 operations per clock per SM), and a
// power iteration is a chain of M x M matrix-vector products, so it runs on a
// cluster of 8 CTAs: CTA q owns rows [q R, (q + 1) R) of w = G v (R =
// ceil(M / 8), the rows in its shared memory when they fit) and keeps a full
// copy of v.  Each step it writes its rows of w into every CTA's next copy of v
// (distributed shared memory) and its partial ||w||^2 into its own slot; one
// cluster barrier later every CTA adds the 8 partials in rank order and scales
// its copy, so all copies stay identical and every run gives the same bits.
// The sums take a different order from the oracle's, so L agrees with it to
// rounding (about 1e-15 relative), not bit for bit.
#include <math.h>

#include "internal.h"

namespace csvc {
namespace {

constexpr int kPowCl = 8;          // CTAs per cluster
constexpr int kPowThreads = 512;

// K3a: Gram matrix G = Phi Phi^T in FP64, one CTA per row.
__global__ void k_gram(const float* __restrict__ phi, double* __restrict__ g, int n, int m) {
    extern __shared__ double rowi[];
    const int i = blockIdx.x;
    for (int k = threadIdx.x; k < n; k += blockDim.x) rowi[k] = (double)phi[(size_t)i * n + k];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int j = warp; j < m; j += nwarps) {
        double acc = 0.0;
        for (int k = lane; k < n; k += 32) acc += rowi[k] * (double)phi[(size_t)j * n + k];
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) g[(size_t)i * m + j] = acc;
    }
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t mapa(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" :::
                     "memory");
}

// Sum over the CTA's threads in a fixed order (warp tree, then warps in order).
__device__ double cta_sum(double v, double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double tot = 0.0;
    for (int w = 0; w < kPowThreads / 32; ++w) tot += red[w];
    return tot;
}

// K3b: the power iteration on a cluster of 8 CTAs (see the file comment).
__global__ void __cluster_dims__(kPowCl, 1, 1) __launch_bounds__(kPowThreads)
    k_power8(const double* __restrict__ gram, int m, int iters, bool g_in_smem, double* result) {
    extern __shared__ double sh[];
    double* v0 = sh;              // [M] v of even steps
    double* v1 = v0 + m;          // [M] v of odd steps
    double* part = v1 + m;        // [2] this CTA's partial sum, by step parity
    double* red = part + 2;       // [kPowThreads / 32]
    double* gs = red + kPowThreads / 32;   // [R][M] this CTA's rows of G, when they fit
    const uint32_t rank = cluster_rank();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = kPowThreads / 32;
    const int rows = (m + kPowCl - 1) / kPowCl;
    const int r0 = (int)rank * rows, r1 = min(m, r0 + rows);
    const double* g = gram + (size_t)r0 * m;
    if (g_in_smem) {
        for (int e = threadIdx.x; e < (r1 - r0) * m; e += kPowThreads) gs[e] = g[e];
        g = gs;
    }
    for (int j = threadIdx.x; j < m; j += kPowThreads) v0[j] = 1.0 / sqrt((double)m);
    cluster_sync();   // every copy of v0 set, every CTA's shared memory live
    for (int it = 0; it <= iters; ++it) {
        const double* v = (it & 1) ? v1 : v0;
        double* vn = (it & 1) ? v0 : v1;
        const bool last = it == iters;
        double psum = 0.0;
        for (int i = r0 + warp; i < r1; i += nwarps) {
            const double* grow = g + (size_t)(i - r0) * m;
            double acc = 0.0;
            for (int j = lane; j < m; j += 32) acc += grow[j] * v[j];
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            // last step: the Rayleigh quotient v^T (G v); else ||G v||^2 and w into every copy
            psum += last ? v[i] * acc : acc * acc;
            if (!last && lane < kPowCl) {
                const uint32_t remote = mapa(smem_addr(&vn[i]), (uint32_t)lane);
                asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(remote), "d"(acc) : "memory");
            }
        }
        const double tot = cta_sum(lane == 0 ? psum : 0.0, red);
        if (threadIdx.x == 0) part[it & 1] = tot;
        cluster_sync();   // every w row and every partial of this step in place
        double total = 0.0;
        for (uint32_t q = 0; q < kPowCl; ++q) {
            double pq;
            asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(pq) : "r"(mapa(smem_addr(&part[it & 1]), q))
                         : "memory");
            total += pq;
        }
        if (last) {
            if (rank == 0 && threadIdx.x == 0) *result = total;
            break;
        }
        const double inv = 1.0 / sqrt(total);
        for (int j = threadIdx.x; j < m; j += kPowThreads) vn[j] *= inv;
        __syncthreads();  // this copy of v is scaled before the next step reads it
    }
    cluster_sync();       // no CTA leaves while a peer may still read its partials
}

}  // namespace

cudaError_t launch_lambda_max(const float* phi, int n, int m, double* gram, double* result,
                              cudaStream_t s) {
    size_t smem = (size_t)n * sizeof(double);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_gram, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_gram<<<m, 256, smem, s>>>(phi, gram, n, m);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int rows = (m + kPowCl - 1) / kPowCl;
    smem = (2 * (size_t)m + 2 + kPowThreads / 32) * sizeof(double);
    const size_t g_bytes = (size_t)rows * m * sizeof(double);
    const bool g_in_smem = smem + g_bytes <= 160 * 1024;
    if (g_in_smem) smem += g_bytes;
    e = cudaFuncSetAttribute(k_power8, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_power8<<<kPowCl, kPowThreads, smem, s>>>(gram, m, 1000, g_in_smem, result);
    return cudaGetLastError();
}

}  // namespace csvc
