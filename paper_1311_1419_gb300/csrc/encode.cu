// K4: block-CS measurement of every CS frame of one or more GOPs (Sec. 3.1).
// For CS frame t, residual r = int(F_t) - int(F_key), key = floor(t/G) G (the
// same key for every CS frame of the GOP, Sec. 3.2), zero-padded to whole
// B x B blocks; y_b = Phi r_b for every block b.  This is one batched GEMM
// Y[rows][M] = R[rows][N] Phi^T over rows = n_cs * nblk blocks, with the
// residual formed on the fly from the uint8 frames (never materialised).
#include "internal.h"

namespace csvc {
namespace {

constexpr int kRowsPerCta = 64;
constexpr int kMPerCta = 64;
constexpr int kKChunk = 32;

__global__ void __launch_bounds__(256) k_encode(const uint8_t* __restrict__ frames,
                                                const float* __restrict__ phi,
                                                float* __restrict__ y, GopShape gs, int lb) {
    __shared__ float rs[kKChunk][kRowsPerCta];
    __shared__ float ps[kKChunk][kMPerCta + 4];
    // per block row of the tile: offsets of its top-left pixel in the CS frame and
    // in the key frame, and its valid extent (blocks at the right / bottom edge
    // are cropped; the padding is zero)
    __shared__ long long row_cur[kRowsPerCta], row_key[kRowsPerCta];
    __shared__ int row_vr[kRowsPerCta], row_vc[kRowsPerCta];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int row0 = blockIdx.x * kRowsPerCta;
    const int m0 = blockIdx.y * kMPerCta;
    const long long total_rows = (long long)gs.n_cs * gs.nblk;
    const size_t frame_px = (size_t)gs.h * gs.w;
    if (tid < kRowsPerCta) {
        const long long row = row0 + tid;
        int vr = 0, vc = 0;
        long long cur = 0, key = 0;
        if (row < total_rows) {
            const int c = (int)(row / gs.nblk), blk = (int)(row % gs.nblk);
            const int g = c / (gs.g - 1), j = c % (gs.g - 1) + 1;
            const int bi = blk / gs.nbc, bj = blk % gs.nbc;
            const long long off = (long long)bi * gs.b * gs.w + (long long)bj * gs.b;
            cur = (long long)(g * gs.g + j) * (long long)frame_px + off;
            key = (long long)(g * gs.g) * (long long)frame_px + off;
            vr = min(gs.b, gs.h - bi * gs.b);
            vc = min(gs.b, gs.w - bj * gs.b);
        }
        row_cur[tid] = cur;
        row_key[tid] = key;
        row_vr[tid] = vr;
        row_vc[tid] = vc;
    }
    __syncthreads();

    float acc[4][4] = {};
    for (int k0 = 0; k0 < gs.n; k0 += kKChunk) {
        // residual chunk: rows row0.., pixels k0..k0+31 of each block
        for (int e = tid; e < kRowsPerCta * kKChunk; e += 256) {
            const int rr = e / kKChunk, kk = e % kKChunk;
            const int k = k0 + kk;
            const int ky = lb >= 0 ? k >> lb : k / gs.b, kx = lb >= 0 ? k & (gs.b - 1) : k % gs.b;
            float v = 0.f;
            if (k < gs.n && ky < row_vr[rr] && kx < row_vc[rr]) {
                const long long o = (long long)ky * gs.w + kx;
                v = (float)((int)frames[row_cur[rr] + o] - (int)frames[row_key[rr] + o]);
            }
            rs[kk][rr] = v;
        }
        for (int e = tid; e < kMPerCta * kKChunk; e += 256) {
            const int mm = e / kKChunk, kk = e % kKChunk;
            const int m = m0 + mm, k = k0 + kk;
            ps[kk][mm] = (m < gs.m && k < gs.n) ? phi[(size_t)m * gs.n + k] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < kKChunk; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = rs[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = ps[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const long long row = row0 + ty * 4 + i;
        if (row >= total_rows) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + tx * 4 + j;
            if (m < gs.m) y[(size_t)row * gs.m + m] = acc[i][j];
        }
    }
}

}  // namespace

cudaError_t launch_encode(const cs_plan* plan, const GopShape& gs, const uint8_t* frames,
                          float* y, cudaStream_t s) {
    const long long rows = (long long)gs.n_cs * gs.nblk;
    if (rows == 0) return cudaSuccess;
    dim3 grid((unsigned)((rows + kRowsPerCta - 1) / kRowsPerCta),
              (unsigned)((gs.m + kMPerCta - 1) / kMPerCta));
    int lb = -1;   // log2 of the block side when it is a power of two
    for (int i = 0; i < 7; ++i)
        if ((1 << i) == gs.b) lb = i;
    k_encode<<<grid, 256, 0, s>>>(frames, plan->phi, y, gs, lb);
    return cudaGetLastError();
}

}  // namespace csvc
