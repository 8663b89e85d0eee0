// K8: per-frame PSNR (the paper's quality measure, Sec. 4 and Table I),
// 10 log10(255^2 / MSE), with the squared error summed in FP64.
#include <math.h>

#include "internal.h"

namespace csvc {
namespace {

__global__ void k_psnr(const uint8_t* __restrict__ ref, const float* __restrict__ test,
                       long long px, double* __restrict__ out) {
    __shared__ double red[32];
    const long long f = blockIdx.x;
    const uint8_t* r = ref + f * px;
    const float* t = test + f * px;
    double acc = 0.0;
    for (long long i = threadIdx.x; i < px; i += blockDim.x) {
        const double d = (double)r[i] - (double)t[i];
        acc += d * d;
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        const double mse = tot / (double)px;
        out[f] = (mse == 0.0) ? INFINITY : 10.0 * log10(255.0 * 255.0 / mse);
    }
}

}  // namespace

cudaError_t launch_psnr(const uint8_t* ref, const float* test, int n_frames, int h, int w,
                        double* out, cudaStream_t s) {
    if (n_frames == 0) return cudaSuccess;
    k_psnr<<<n_frames, 1024, 0, s>>>(ref, test, (long long)h * w, out);
    return cudaGetLastError();
}

}  // namespace csvc
