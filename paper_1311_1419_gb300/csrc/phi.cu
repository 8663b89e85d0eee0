// Plan construction on the device: the Gaussian measurement matrix Phi
// (Sec. 3.1 and Sec. 4: "a Gaussian random matrix") and A = Phi Psi with Psi
// the orthonormal 2-D DCT of a block (the step constant L is in lipschitz.cu).
//
// Phi must be identical bit for bit wherever it is generated, so every double
// operation on its path is an explicit round-to-nearest intrinsic (never
// contracted into an FMA), and this file is also compiled with -fmad=false.
// log and sincos are written here from textbook methods (an atanh series after
// an exponent split, and a Taylor series after an exact quarter-turn
// reduction) rather than calling the CUDA math library, whose last-bit
// behaviour is not specified.
#include <math.h>

#include "internal.h"

namespace csvc {
namespace {

// ---- Philox4x64-10 (Salmon, Moraes, Dror, Shaw; SC'11) ---------------------
constexpr uint64_t kPhiloxM0 = 0xD2E7470EE14C6C93ull;
constexpr uint64_t kPhiloxM1 = 0xCA5A826395121157ull;
constexpr uint64_t kPhiloxW0 = 0x9E3779B97F4A7C15ull;  // golden ratio
constexpr uint64_t kPhiloxW1 = 0xBB67AE8584CAA73Bull;  // sqrt(3) - 1

__device__ __forceinline__ void philox4x64_10(uint64_t x[4], uint64_t k0, uint64_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t lo0 = kPhiloxM0 * x[0], hi0 = __umul64hi(kPhiloxM0, x[0]);
        const uint64_t lo1 = kPhiloxM1 * x[2], hi1 = __umul64hi(kPhiloxM1, x[2]);
        const uint64_t n0 = hi1 ^ x[1] ^ k0;
        const uint64_t n2 = hi0 ^ x[3] ^ k1;
        x[0] = n0;
        x[1] = lo1;
        x[2] = n2;
        x[3] = lo0;
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
}

// ---- elementary functions in plain IEEE double ----------------------------
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }

// ln 2 split so that e * kLn2Hi is exact for |e| < 2^13 (kLn2Hi has 40 bits).
__device__ __forceinline__ double ln2_hi() { return __longlong_as_double(0x3FE62E42FEFA2000ll); }
__device__ __forceinline__ double ln2_lo() { return __longlong_as_double(0x3D69EF35793C7673ll); }
__device__ __forceinline__ double sqrt2_d() { return __longlong_as_double(0x3FF6A09E667F3BCDll); }
__device__ __forceinline__ double pio2_d() { return __longlong_as_double(0x3FF921FB54442D18ll); }

// 1/k! rounded to nearest; k! itself is exact in a double for k <= 22.
__device__ __forceinline__ double inv_factorial(int k) {
    uint64_t f = 1;
    for (int i = 2; i <= k; ++i) f *= (uint64_t)i;
    return ddiv(1.0, __ull2double_rn(f));
}

// Natural log of a positive normal double.  x = 2^e f, f in [1,2); if
// f > sqrt 2, halve f and bump e.  s = (f-1)/(f+1), ln f = 2 atanh s =
// 2s + 2s (s^2 q(s^2)) with q(w) = sum_{j=1..11} w^(j-1)/(2j+1) by Horner,
// ln x = e ln2_hi + (ln f + e ln2_lo).
__device__ double log_fp64(double x) {
    const long long bits = __double_as_longlong(x);
    double e = (double)(int)(((bits >> 52) & 0x7FF) - 1023);
    double f = __longlong_as_double((bits & 0x000FFFFFFFFFFFFFll) | 0x3FF0000000000000ll);
    if (f > sqrt2_d()) {
        f = dmul(f, 0.5);
        e = dadd(e, 1.0);
    }
    const double s = ddiv(dsub(f, 1.0), dadd(f, 1.0));
    const double s2 = dmul(s, s);
    constexpr int kTerms = 11;
    double q = ddiv(1.0, (double)(2 * kTerms + 1));
    for (int j = kTerms - 1; j >= 1; --j) q = dadd(dmul(q, s2), ddiv(1.0, (double)(2 * j + 1)));
    const double two_s = dmul(2.0, s);
    const double ln_f = dadd(two_s, dmul(two_s, dmul(s2, q)));
    return dadd(dmul(e, ln2_hi()), dadd(ln_f, dmul(e, ln2_lo())));
}

// sin and cos of 2 pi u for u in [0,1) holding at most 53 significant bits.
// t = 4u and d = t - rint(t) are exact; theta = d pi/2 in [-pi/4, pi/4];
// sin theta = theta + theta (theta^2 p), p the Taylor tail to theta^19;
// cos theta = 1 + theta^2 q, q the Taylor tail to theta^20; rotate by the
// quadrant rint(t) mod 4.
__device__ void sincos_2pi(double u, double* sn, double* cs) {
    const double t = dmul(4.0, u);
    const double n = rint(t);
    const double d = dsub(t, n);
    const double th = dmul(d, pio2_d());
    const double th2 = dmul(th, th);
    constexpr int kSin = 9, kCos = 10;
    double p = (kSin & 1) ? -inv_factorial(2 * kSin + 1) : inv_factorial(2 * kSin + 1);
    for (int k = kSin - 1; k >= 1; --k) {
        const double c = inv_factorial(2 * k + 1);
        p = dadd(dmul(p, th2), (k & 1) ? -c : c);
    }
    const double s = dadd(th, dmul(th, dmul(th2, p)));
    double q = (kCos & 1) ? -inv_factorial(2 * kCos) : inv_factorial(2 * kCos);
    for (int k = kCos - 1; k >= 1; --k) {
        const double c = inv_factorial(2 * k);
        q = dadd(dmul(q, th2), (k & 1) ? -c : c);
    }
    const double c = dadd(1.0, dmul(th2, q));
    switch (((long long)n) & 3) {
        case 0: *sn = s; *cs = c; break;
        case 1: *sn = c; *cs = -s; break;
        case 2: *sn = -s; *cs = -c; break;
        default: *sn = -c; *cs = s; break;
    }
}

// K1: one thread per pair q of row-major entries (2q, 2q+1).
__global__ void k_phi(float* __restrict__ phi, long long total, uint64_t tag, uint64_t seed,
                      double sqrt_m) {
    const long long pairs = (total + 1) / 2;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < pairs;
         q += (long long)gridDim.x * blockDim.x) {
        uint64_t x[4] = {(uint64_t)q, tag, 0ull, 0ull};
        philox4x64_10(x, seed, 0ull);
        const double two_m53 = 1.1102230246251565e-16;  // 2^-53, exact
        const double u1 = dmul(__ull2double_rn((x[0] >> 11) + 1ull), two_m53);
        const double u2 = dmul(__ull2double_rn(x[1] >> 11), two_m53);
        const double rad = __dsqrt_rn(dmul(-2.0, log_fp64(u1)));
        double sn, cs;
        sincos_2pi(u2, &sn, &cs);
        phi[2 * q] = __double2float_rn(ddiv(dmul(rad, cs), sqrt_m));
        if (2 * q + 1 < total) phi[2 * q + 1] = __double2float_rn(ddiv(dmul(rad, sn), sqrt_m));
    }
}

// K2: A = Phi Psi row by row.  Row i of A is the 2-D DCT C Phi_i C^T of row i
// of Phi viewed as a B x B block (r = Psi s <=> R = C^T S C, so s = Psi^T r and
// A = Phi Psi maps Phi_i to C Phi_i C^T).  FP64 throughout, one rounding at
// the end.  Block 0 also writes the float32 DCT matrix used by recon.
__global__ void k_form_a(const float* __restrict__ phi, float* __restrict__ a,
                         float* __restrict__ dct_out, int n, int b) {
    extern __shared__ double sm[];
    double* c = sm;             // [B][B]
    double* row = c + b * b;    // [B][B] Phi_i
    double* tmp = row + b * b;  // [B][B] C Phi_i
    const int i = blockIdx.x;
    for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) {
        const int k = idx / b, j = idx % b;
        const double alpha = (k == 0) ? sqrt(1.0 / b) : sqrt(2.0 / b);
        c[idx] = alpha * cospi((double)((2 * j + 1) * k) / (double)(2 * b));
        row[idx] = (double)phi[(size_t)i * n + idx];
        if (i == 0) dct_out[idx] = (float)c[idx];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) {
        const int k = idx / b, q = idx % b;
        double acc = 0.0;
        for (int p = 0; p < b; ++p) acc += c[k * b + p] * row[p * b + q];
        tmp[idx] = acc;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) {
        const int k = idx / b, l = idx % b;
        double acc = 0.0;
        for (int q = 0; q < b; ++q) acc += tmp[k * b + q] * c[l * b + q];
        a[(size_t)i * n + idx] = (float)acc;
    }
}

}  // namespace

cudaError_t launch_phi(float* phi, int n, int m, uint64_t seed, cudaStream_t s) {
    const long long total = (long long)n * m;
    const long long pairs = (total + 1) / 2;
    const int threads = 256;
    const int blocks = (int)((pairs + threads - 1) / threads);
    const uint64_t tag = ((uint64_t)n << 16) | (uint64_t)m;
    k_phi<<<blocks, threads, 0, s>>>(phi, total, tag, seed, sqrt((double)m));
    return cudaGetLastError();
}

cudaError_t launch_form_a(const float* phi, float* a, float* dct, int n, int m, int b,
                          cudaStream_t s) {
    const size_t smem = 3ull * b * b * sizeof(double);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_form_a, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_form_a<<<m, 256, smem, s>>>(phi, a, dct, n, b);
    return cudaGetLastError();
}

}  // namespace csvc
