// K4 on the tensor cores for every block size: block-CS measurement of every
// CS frame (Sec. 3.1), y_b = Phi r_b, for 8 x 8, 16 x 16 and 32 x 32 blocks
// (N = 64, 256, 1024) and M <= 256.
//
// One GEMM across the blocks of the call, Y [rows x M] = R [rows x N] Phi^T,
// as in the 16 x 16 kernel (encode_tc.cu): residuals are integers in
// [-255, 255], exact in fp16, and Phi * 2^e is split into fp16 hi + lo, so two
// MMAs per K step give FP32-grade products.  Phi does not fit on chip for
// N = 1024, so here it streams: per tile of 128 blocks, K runs in chunks of 64
// pixels (two rows of a 32 x 32 block, four of a 16 x 16, a whole 8 x 8 block);
// thread 0 bulk-copies each chunk of the Phi images (contiguous in their
// K-chunk-major layout, and resident in L2) into a two-stage ring while all
// threads form the residual chunk from the uint8 frames (8-byte loads) into a
// double-buffered 128-byte-swizzled operand; one commit per chunk frees both
// buffers of its stage.  The accumulator (M16 columns of tensor memory) is read
// back as y = D 2^-e.  Every mbarrier wait is bounded and reports through the
// context's error word.
#include <cuda_fp16.h>

#include "internal.h"
#include "tc_ptx.h"

namespace csvc {
namespace {

using namespace tc;

constexpr int kT = 256;
constexpr int kTile = 128;
constexpr int kChunk = 64;                          // K per chunk: one 128-byte swizzle atom column
constexpr int kMaxM16 = 256;
constexpr uint32_t kRStage = kTile * kChunk * 2;           // 16 KB
constexpr uint64_t kWaitNs = 1000000000ull;
// Shared memory for M16 rows of Phi: two stages of a hi + lo chunk (m16 x 64 x 2
// bytes each), two residual chunks, barriers.  Up to M16 = 112 two CTAs share an
// SM (one's residual chunk forms while the other's copies and MMAs run).
__host__ __device__ constexpr uint32_t phi_stage_bytes(int m16) { return 2u * (uint32_t)m16 * kChunk * 2u; }
__host__ __device__ constexpr uint32_t off_r(int m16) { return 2u * phi_stage_bytes(m16); }
__host__ __device__ constexpr uint32_t off_bar(int m16) { return off_r(m16) + 2u * kRStage; }
__host__ __device__ constexpr uint32_t smem_bytes(int m16) { return off_bar(m16) + 128u + 1024u; }
constexpr int kTwoPerSmM16 = 112;
static_assert(smem_bytes(kTwoPerSmM16) <= 232448 / 2 - 1024, "two CTAs per SM");

// Byte offset of pixels k .. k + 7 (k % 8 == 0, k < 64) of block row `row` in a
// chunk operand (K-major, 16 row groups of 1 KB, 128-byte swizzle).
__device__ __forceinline__ uint32_t rchunk_off(uint32_t row, uint32_t k) {
    const uint32_t r = row & 7;
    return (row >> 3) * 1024u + r * 128u + (((k >> 3) ^ r) << 4);
}

__device__ __forceinline__ bool wait_e(uint64_t* bar, uint32_t parity, int* abort, int* err) {
    if (*(volatile int*)abort) return false;
    if (mbar_wait(bar, parity, kWaitNs)) return true;
    *(volatile int*)abort = 1;
    atomicExch(err, 1);
    return false;
}

__global__ void __launch_bounds__(kT, 2) k_encode_tcg(const uint8_t* __restrict__ frames,
                                                       const uint8_t* __restrict__ phi_img, float* __restrict__ y,
                                                       GopShape gs, int m16, float scale_out, bool vec,
                                                       int* err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
    const uint32_t kOffPhi = 0, kPhiStage = phi_stage_bytes(m16), kOffR = off_r(m16);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + off_bar(m16));
    uint64_t* phi_full = bar;          // [2]: the stage's Phi chunk has landed
    uint64_t* mma_done = bar + 2;      // [2]: the stage's MMAs have read both its buffers
    uint64_t* acc_full = bar + 4;      // the tile's accumulator is complete
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 5);
    int* abort = reinterpret_cast<int*>(bar + 6);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n = gs.n, bsz = gs.b, nch = n / kChunk;
    const uint32_t ncols = m16 <= 128 ? 128u : 256u;
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&phi_full[s], 1);
            mbar_init(&mma_done[s], 1);
        }
        mbar_init(acc_full, 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        __syncwarp();
        tmem_alloc(tmem_slot, ncols);
        tmem_relinquish();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const uint32_t s_base = smem_u32(sm);
    const uint32_t img = (uint32_t)m16 * (uint32_t)n * 2;      // one fp16 image of Phi
    const uint32_t cbytes = (uint32_t)m16 * kChunk * 2;         // one chunk of one image
    const long long rows = (long long)gs.n_cs * gs.nblk;
    const long long tiles = (rows + kTile - 1) / kTile;
    const size_t frame_px = (size_t)gs.h * gs.w;
    const int rows_per_chunk = kChunk / bsz;                    // block rows in a chunk
    const int segs = bsz / 8;                                   // 8-pixel segments per block row
    uint32_t g = 0;                                             // chunks issued so far
    uint32_t ph_acc = 0;
    bool ok = true;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        for (int c = 0; c < nch; ++c, ++g) {
            const uint32_t s = g & 1;
            // the MMAs of chunk g - 2 have read this stage's buffers
            if (g >= 2) ok = wait_e(&mma_done[s], ((g >> 1) & 1) ^ 1, abort, err) && ok;
            if (tid == 0 && ok) {
                uint8_t* dst = sm + kOffPhi + s * kPhiStage;
                mbar_arrive_expect_tx(&phi_full[s], 2 * cbytes);
                bulk_g2s(dst, phi_img + (size_t)c * cbytes, cbytes, &phi_full[s]);
                bulk_g2s(dst + cbytes, phi_img + img + (size_t)c * cbytes, cbytes, &phi_full[s]);
            }
            // the residual chunk: block b, block row c * rows_per_chunk + rr, segment sg
            uint8_t* rbuf = sm + kOffR + s * kRStage;
            for (int item = tid; item < kTile * kChunk / 8; item += kT) {
                const int b = item / (kChunk / 8), kseg = item % (kChunk / 8);
                const int rr = kseg / segs, sg = kseg % segs;
                const long long row = tile * kTile + b;
                float v[8];
#pragma unroll
                for (int x = 0; x < 8; ++x) v[x] = 0.f;
                if (row < rows) {
                    const int ci = (int)(row / gs.nblk), blk = (int)(row % gs.nblk);
                    const int gg = ci / (gs.g - 1), j = ci % (gs.g - 1) + 1;
                    const int fy = (blk / gs.nbc) * bsz + c * rows_per_chunk + rr;
                    const int fx0 = (blk % gs.nbc) * bsz + 8 * sg;
                    if (fy < gs.h) {
                        const uint8_t* cur = frames + (size_t)(gg * gs.g + j) * frame_px + (size_t)fy * gs.w + fx0;
                        const uint8_t* key = frames + (size_t)(gg * gs.g) * frame_px + (size_t)fy * gs.w + fx0;
                        if (vec) {
                            const uint2 cv = __ldg(reinterpret_cast<const uint2*>(cur));
                            const uint2 kv = __ldg(reinterpret_cast<const uint2*>(key));
                            const uint8_t* cb = reinterpret_cast<const uint8_t*>(&cv);
                            const uint8_t* kb = reinterpret_cast<const uint8_t*>(&kv);
#pragma unroll
                            for (int x = 0; x < 8; ++x) v[x] = (float)((int)cb[x] - (int)kb[x]);
                        } else {
#pragma unroll
                            for (int x = 0; x < 8; ++x)
                                if (fx0 + x < gs.w) v[x] = (float)((int)cur[x] - (int)key[x]);
                        }
                    }
                }
                uint4 pk;
                uint32_t* w = reinterpret_cast<uint32_t*>(&pk);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    __half2 h2 = __floats2half2_rn(v[2 * e], v[2 * e + 1]);
                    w[e] = *reinterpret_cast<uint32_t*>(&h2);
                }
                *reinterpret_cast<uint4*>(rbuf + rchunk_off((uint32_t)b, (uint32_t)(8 * kseg))) = pk;
            }
            fence_proxy_async_smem();
            fence_before_sync();
            __syncthreads();
            fence_after_sync();
            if (tid == 0) {
                ok = wait_e(&phi_full[s], (g >> 1) & 1, abort, err) && ok;
                fence_after_sync();
                if (ok) {
                    const uint64_t da = desc_sw128(s_base + kOffR + s * kRStage, 16, 1024);
                    const uint64_t dh = desc_sw128(s_base + kOffPhi + s * kPhiStage, 16, 1024);
                    const uint64_t dl = desc_sw128(s_base + kOffPhi + s * kPhiStage + cbytes, 16, 1024);
                    const uint32_t id = idesc_f16(128, (uint32_t)m16, 0u, 0u, 0u);
#pragma unroll
                    for (uint32_t ks = 0; ks < kChunk / 16; ++ks) {
                        mma_f16(tmem, da + 2 * ks, dh + 2 * ks, id, (c > 0 || ks > 0) ? 1u : 0u);
                        mma_f16(tmem, da + 2 * ks, dl + 2 * ks, id, 1u);
                    }
                }
                mma_commit(&mma_done[s]);
                if (c == nch - 1) mma_commit(acc_full);
            }
        }
        // y = D 2^-e: warp w reads lanes 32 (w % 4) .. of columns half (w / 4) of M16
        ok = wait_e(acc_full, ph_acc, abort, err) && ok;
        ph_acc ^= 1;
        fence_after_sync();
        {
            const int q = warp & 3, hf = warp >> 2;
            const int b = 32 * q + lane;
            const long long row = tile * kTile + b;
            const int c0 = hf * (m16 / 2);
            for (int cc = c0; cc < c0 + m16 / 2; cc += 8) {
                uint32_t d[8];
                tmem_ld8(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)cc, d);
                tmem_wait_ld();
                if (ok && row < rows) {
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (cc + i < gs.m) y[row * gs.m + cc + i] = __uint_as_float(d[i]) * scale_out;
                }
            }
        }
        fence_before_sync();
        __syncthreads();   // the accumulator is reused by the next tile
        fence_after_sync();
    }
    if (tid == 0) {
        // copies and MMAs still in flight after a wait gave up: wait for them (bounded)
        for (uint32_t s = 0; s < 2 && g > s; ++s) {
            const uint32_t last = g - 1 - ((g - 1 - s) & 1);    // the last chunk of stage s
            mbar_wait(&phi_full[s], (last >> 1) & 1, kWaitNs);
            mbar_wait(&mma_done[s], (last >> 1) & 1, kWaitNs);
        }
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 0) tmem_dealloc(tmem, ncols);
}

// The images of Phi * 2^e for this kernel: fp16 hi then fp16 lo, each m16 x n,
// rows >= M zero, 128-byte-swizzled atoms of 8 rows x 64 columns, atom
// (col / 64, row / 8) at ((col / 64) * m16 / 8 + row / 8) * 1024: a 64-column
// K chunk of all rows is one contiguous range.
__global__ void k_phi_images_g(const float* __restrict__ phi, uint8_t* __restrict__ img, int n, int m, int m16,
                               float scale) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m16 * n) return;
    const int row = idx / n, col = idx % n;
    const float v = row < m ? phi[(size_t)row * n + col] * scale : 0.f;
    const __half hh = __float2half_rn(v);
    const __half hl = __float2half_rn(v - __half2float(hh));
    const uint32_t off = sw128_offset((uint32_t)row, (uint32_t)col, (uint32_t)m16 / 8);
    *reinterpret_cast<__half*>(img + off) = hh;
    *reinterpret_cast<__half*>(img + (size_t)m16 * n * 2 + off) = hl;
}

}  // namespace

bool encode_tcg_plan_supported(int n, int m) {
    return (n == 64 || n == 256 || n == 1024) && m >= 1 && (m + 15) / 16 * 16 <= kMaxM16;
}
size_t encode_tcg_image_bytes(int n, int m) { return 2ull * (size_t)((m + 15) / 16 * 16) * (size_t)n * 2; }

cudaError_t launch_phi_images_g(const float* phi, uint8_t* img, int n, int m, int e, cudaStream_t s) {
    const int m16 = (m + 15) / 16 * 16;
    const int total = m16 * n;
    k_phi_images_g<<<(total + 255) / 256, 256, 0, s>>>(phi, img, n, m, m16, ldexpf(1.f, e));
    return cudaGetLastError();
}

cudaError_t launch_encode_tcg(const cs_plan* plan, const GopShape& gs, const uint8_t* frames, float* y,
                              cudaStream_t s) {
    const long long rows = (long long)gs.n_cs * gs.nblk;
    if (rows == 0) return cudaSuccess;
    const int m16 = (plan->m + 15) / 16 * 16;
    const long long tiles = (rows + kTile - 1) / kTile;
    const int per_sm = m16 <= kTwoPerSmM16 ? 2 : 1;
    const int grid = (int)(tiles < per_sm * plan->ctx->sm_count ? tiles : per_sm * plan->ctx->sm_count);
    // 8-byte frame loads when every block row segment starts on an 8-byte
    // boundary and no block is cropped at the right edge
    const bool vec = gs.w % 8 == 0 && gs.w % gs.b == 0 && (reinterpret_cast<uintptr_t>(frames) & 7) == 0;
    cudaError_t e = cudaFuncSetAttribute(k_encode_tcg, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_bytes(kMaxM16));
    if (e != cudaSuccess) return e;
    k_encode_tcg<<<grid, kT, smem_bytes(m16), s>>>(frames, plan->phi_tcg, y, gs, m16, ldexpf(1.f, -plan->tc_ephi),
                                              vec, plan->ctx->err_dev);
    return cudaGetLastError();
}

}  // namespace csvc
