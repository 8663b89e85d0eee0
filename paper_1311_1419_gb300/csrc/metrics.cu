// K8: per-frame PSNR (the paper's quality measure, Sec. 4 and Table I),
// 10 log10(255^2 / MSE), with the squared error summed in FP64.
//
// A cluster of 8 CTAs takes one frame: each CTA sums the squared errors of an
// eighth of the pixels (vector loads when the frame is 16-byte aligned), and
// CTA 0 adds the 8 partial sums in rank order from distributed shared memory,
// so the result does not depend on scheduling.  d = t - r is exact in FP64
// (r an 8-bit integer, t a float32), and d^2 accumulates by FMA in FP64.
#include <math.h>

#include "internal.h"

namespace csvc {
namespace {

constexpr int kPsnrCta = 8;
constexpr int kPsnrThreads = 512;

__device__ __forceinline__ double sq_err(uint8_t r, float t) {
    return (double)t - (double)r;
}

__global__ void __cluster_dims__(kPsnrCta, 1, 1) __launch_bounds__(kPsnrThreads)
    k_psnr(const uint8_t* __restrict__ ref, const float* __restrict__ test, long long px,
           bool vec, double* __restrict__ out) {
    __shared__ double red[kPsnrThreads / 32];
    __shared__ double partial;
    uint32_t rank;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
    const long long f = blockIdx.x / kPsnrCta;
    const long long chunk = (px + 4 * kPsnrCta - 1) / (4 * kPsnrCta) * 4;   // multiple of 4
    const long long begin = (long long)rank * chunk;
    const long long end = begin + chunk < px ? begin + chunk : px;
    const uint8_t* r = ref + f * px;
    const float* t = test + f * px;
    double acc = 0.0;
    long long i = begin + threadIdx.x * 4;
    if (vec) {
        // 4 pixels per thread and step: 4-byte uint8 and 16-byte float32 loads
        for (; i + 3 < end; i += 4 * kPsnrThreads) {
            const uchar4 rv = *reinterpret_cast<const uchar4*>(r + i);
            const float4 tv = __ldg(reinterpret_cast<const float4*>(t + i));
            double d = sq_err(rv.x, tv.x);
            acc = fma(d, d, acc);
            d = sq_err(rv.y, tv.y);
            acc = fma(d, d, acc);
            d = sq_err(rv.z, tv.z);
            acc = fma(d, d, acc);
            d = sq_err(rv.w, tv.w);
            acc = fma(d, d, acc);
        }
    } else {
        for (long long j = begin + threadIdx.x; j < end; j += kPsnrThreads) {
            const double d = sq_err(r[j], t[j]);
            acc = fma(d, d, acc);
        }
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < kPsnrThreads / 32; ++w) tot += red[w];
        partial = tot;
    }
    // every CTA's partial is in its shared memory before CTA 0 reads them
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" :::
                     "memory");
    if (rank == 0 && threadIdx.x == 0) {
        const uint32_t local = (uint32_t)__cvta_generic_to_shared(&partial);
        double tot = 0.0;
        for (uint32_t q = 0; q < kPsnrCta; ++q) {
            uint32_t remote;
            double v;
            asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(q));
            asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(remote) : "memory");
            tot += v;
        }
        const double mse = tot / (double)px;
        out[f] = (mse == 0.0) ? INFINITY : 10.0 * log10(255.0 * 255.0 / mse);
    }
    // no CTA leaves while CTA 0 may still read its shared memory
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" :::
                     "memory");
}

}  // namespace

cudaError_t launch_psnr(const uint8_t* ref, const float* test, int n_frames, int h, int w,
                        double* out, cudaStream_t s) {
    if (n_frames == 0) return cudaSuccess;
    const long long px = (long long)h * w;
    const bool vec = px % 4 == 0 && (reinterpret_cast<uintptr_t>(ref) & 3) == 0 &&
                     (reinterpret_cast<uintptr_t>(test) & 15) == 0;
    k_psnr<<<(unsigned)n_frames * kPsnrCta, kPsnrThreads, 0, s>>>(ref, test, px, vec, out);
    return cudaGetLastError();
}

}  // namespace csvc
