// K8: per-frame PSNR (the paper's quality measure, Sec. 4 and Table I),
// 10 log10(255^2 / MSE); the squared errors are summed with about 48 significant bits.
//
// A cluster of 8 CTAs takes one frame: each CTA sums the squared errors of an
// eighth of the pixels (vector loads when the frame is 16-byte aligned), and
// CTA 0 adds the 8 partial sums in rank order from distributed shared memory,
// so the result does not depend on scheduling.  FP64 is scarce on this part,
// so a thread keeps its sum in float-float (about 48 significant bits) with
// error-free transformations in FP32: d = t - r exactly as a pair s + e
// (Knuth's TwoSum), s^2 exactly as p + q (the FMA TwoProduct), d^2 = p + (q +
// 2 s e) up to e^2 < 2^-48 s^2, and each term added to the pair (hi, lo) by
// TwoSum.  The per-thread pairs are combined in FP64.
#include <math.h>

#include "internal.h"

namespace csvc {
namespace {

constexpr int kPsnrCta = 8;
constexpr int kPsnrThreads = 512;

// a + b = s + e exactly (round to nearest, no reassociation)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (hi, lo) += (t - r)^2
__device__ __forceinline__ void add_sq_err(uint8_t r, float t, float& hi, float& lo) {
    float s, e;
    two_sum(t, -(float)r, s, e);                    // d = s + e exactly
    const float p = __fmul_rn(s, s);
    const float q = __fmaf_rn(s, s, -p);            // s^2 = p + q exactly
    const float tail = __fmaf_rn(__fmul_rn(2.f, s), e, q);
    float h, c;
    two_sum(hi, p, h, c);
    hi = h;
    lo = __fadd_rn(lo, __fadd_rn(c, tail));
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
    float hi = 0.f, lo = 0.f;
    long long i = begin + threadIdx.x * 4;
    if (vec) {
        // 4 pixels per thread and step: 4-byte uint8 and 16-byte float32 loads
        for (; i + 3 < end; i += 4 * kPsnrThreads) {
            const uchar4 rv = *reinterpret_cast<const uchar4*>(r + i);
            const float4 tv = __ldg(reinterpret_cast<const float4*>(t + i));
            add_sq_err(rv.x, tv.x, hi, lo);
            add_sq_err(rv.y, tv.y, hi, lo);
            add_sq_err(rv.z, tv.z, hi, lo);
            add_sq_err(rv.w, tv.w, hi, lo);
        }
    } else {
        for (long long j = begin + threadIdx.x; j < end; j += kPsnrThreads) add_sq_err(r[j], t[j], hi, lo);
    }
    double acc = (double)hi + (double)lo;
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
