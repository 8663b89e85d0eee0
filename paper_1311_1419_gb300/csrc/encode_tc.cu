// K4 on the tensor cores: block-CS measurement of every CS frame (Sec. 3.1),
// y_b = Phi r_b, for 16 x 16 blocks (N = 256) and M <= 128.
//
// Across the blocks of a call this is one GEMM, Y [rows x M] = R [rows x 256]
// Phi^T.  The residual r = int(F_t) - int(F_key) of the same key frame for
// every CS frame of the GOP (Sec. 3.2) is an integer in [-255, 255], exact in
// fp16; Phi * 2^e is split into fp16 hi + lo images (22 significant bits), so
// two MMAs per K step give products as accurate as FP32.  A persistent CTA
// keeps both Phi images in shared memory (loaded once by the bulk-copy engine)
// and, per tile of 128 blocks: forms the residual tile from the uint8 frames
// with 16-byte loads straight into the 128-byte-swizzled K-major operand,
// issues the 32 MMAs into tensor memory, and writes y = D 2^-e.  Every
// mbarrier wait is bounded and reports through the context's error word.
#include <cuda_fp16.h>

#include "internal.h"
#include "tc_ptx.h"

namespace csvc {
namespace {

using namespace tc;

constexpr int kT = 256;
constexpr int kTile = 128;
constexpr int kN = 256;
constexpr int kMaxM16 = 128;
constexpr uint32_t kPhiImg = kMaxM16 * kN * 2;    // 64 KB per fp16 image
constexpr uint32_t kOffHi = 0, kOffLo = kPhiImg, kOffR = 2 * kPhiImg;
constexpr uint32_t kRImg = kTile * kN * 2;        // 64 KB
constexpr uint32_t kOffBar = kOffR + kRImg;
constexpr uint32_t kSmemBytes = kOffBar + 64 + 1024;
constexpr uint64_t kWaitNs = 1000000000ull;

// Byte offset of elements k .. k + 7 (k % 8 == 0) of row `row` in a K-major
// operand of 16 row groups, 128-byte swizzle.
__device__ __forceinline__ uint32_t rtile_off(uint32_t row, uint32_t k) {
    const uint32_t r = row & 7;
    return ((k >> 6) * (kTile / 8) + (row >> 3)) * 1024u + r * 128u + ((((k & 63) >> 3) ^ r) << 4);
}

__global__ void __launch_bounds__(kT, 1) k_encode_tc(const uint8_t* __restrict__ frames,
                                                      const uint8_t* __restrict__ phi_img, float* __restrict__ y,
                                                      GopShape gs, int m16, float scale_out, bool vec,
                                                      int* err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
    uint64_t* bar_load = reinterpret_cast<uint64_t*>(sm + kOffBar);
    uint64_t* bar_mma = bar_load + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar_load + 2);
    int* abort = reinterpret_cast<int*>(bar_load + 3);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t img = (uint32_t)m16 * kN * 2;
    if (tid == 0) {
        mbar_init(bar_load, 1);
        mbar_init(bar_mma, 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        __syncwarp();
        tmem_alloc(tmem_slot, 128);
        tmem_relinquish();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    if (tid == 0) {
        mbar_arrive_expect_tx(bar_load, 2 * img);
        bulk_g2s(sm + kOffHi, phi_img, img, bar_load);
        bulk_g2s(sm + kOffLo, phi_img + img, img, bar_load);
    }
    bool ok = mbar_wait(bar_load, 0, kWaitNs);
    if (!ok && tid == 0) {
        *(volatile int*)abort = 1;
        atomicExch(err, 1);
    }
    const long long rows = (long long)gs.n_cs * gs.nblk;
    const long long tiles = (rows + kTile - 1) / kTile;
    const size_t frame_px = (size_t)gs.h * gs.w;
    uint32_t ph = 0;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        // residual tile: block b of the tile, pixel row py -> 16 fp16 at k = 16 py ..
        for (int item = tid; item < kTile * 16; item += kT) {
            const int b = item >> 4, py = item & 15;
            const long long row = tile * kTile + b;
            float v[16];
#pragma unroll
            for (int x = 0; x < 16; ++x) v[x] = 0.f;
            if (row < rows) {
                const int c = (int)(row / gs.nblk), blk = (int)(row % gs.nblk);
                const int g = c / (gs.g - 1), j = c % (gs.g - 1) + 1;
                const int fy = (blk / gs.nbc) * 16 + py, fx0 = (blk % gs.nbc) * 16;
                if (fy < gs.h) {
                    const uint8_t* cur = frames + (size_t)(g * gs.g + j) * frame_px + (size_t)fy * gs.w + fx0;
                    const uint8_t* key = frames + (size_t)(g * gs.g) * frame_px + (size_t)fy * gs.w + fx0;
                    if (vec) {
                        const uint4 cv = __ldg(reinterpret_cast<const uint4*>(cur));
                        const uint4 kv = __ldg(reinterpret_cast<const uint4*>(key));
                        const uint8_t* cb = reinterpret_cast<const uint8_t*>(&cv);
                        const uint8_t* kb = reinterpret_cast<const uint8_t*>(&kv);
#pragma unroll
                        for (int x = 0; x < 16; ++x) v[x] = (float)((int)cb[x] - (int)kb[x]);
                    } else {
#pragma unroll
                        for (int x = 0; x < 16; ++x)
                            if (fx0 + x < gs.w) v[x] = (float)((int)cur[x] - (int)key[x]);
                    }
                }
            }
#pragma unroll
            for (int hf = 0; hf < 2; ++hf) {
                uint4 pk;
                uint32_t* w = reinterpret_cast<uint32_t*>(&pk);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    __half2 h2 = __floats2half2_rn(v[8 * hf + 2 * e], v[8 * hf + 2 * e + 1]);
                    w[e] = *reinterpret_cast<uint32_t*>(&h2);
                }
                *reinterpret_cast<uint4*>(sm + kOffR + rtile_off((uint32_t)b, (uint32_t)(16 * py + 8 * hf))) = pk;
            }
        }
        fence_proxy_async_smem();
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
        if (tid == 0 && !*(volatile int*)abort) {
            const uint32_t s_base = smem_u32(sm);
            const uint32_t rg = (uint32_t)(m16 / 8);
            const uint64_t da = desc_sw128(s_base + kOffR, 16, 1024);
            const uint64_t dh = desc_sw128(s_base + kOffHi, 16, 1024);
            const uint64_t dl = desc_sw128(s_base + kOffLo, 16, 1024);
            const uint32_t id = idesc_f16(128, (uint32_t)m16, 0u, 0u, 0u);
#pragma unroll 1
            for (uint32_t ks = 0; ks < kN / 16; ++ks) {
                const uint32_t k0 = 16 * ks;
                const uint32_t a16 = ((k0 >> 6) * (kTile / 8) * 1024 + ((k0 & 63) >> 4) * 32) >> 4;
                const uint32_t b16 = ((k0 >> 6) * rg * 1024 + ((k0 & 63) >> 4) * 32) >> 4;
                mma_f16(tmem, da + a16, dh + b16, id, ks > 0);
                mma_f16(tmem, da + a16, dl + b16, id, 1);
            }
            mma_commit(bar_mma);
        }
        if (!*(volatile int*)abort) {
            if (!mbar_wait(bar_mma, ph, kWaitNs)) {
                *(volatile int*)abort = 1;
                atomicExch(err, 1);
            }
        }
        ph ^= 1;
        fence_after_sync();
        // y = D 2^-e: warp w reads lanes 32 (w % 4) .. of columns half (w / 4) of M16
        {
            const int q = warp & 3, hf = warp >> 2;
            const int b = 32 * q + lane;
            const long long row = tile * kTile + b;
            const int c0 = hf * (m16 / 2);
            for (int c = c0; c < c0 + m16 / 2; c += 8) {
                uint32_t d[8];
                tmem_ld8(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c, d);
                tmem_wait_ld();
                if (row < rows) {
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (c + i < gs.m) y[row * gs.m + c + i] = __uint_as_float(d[i]) * scale_out;
                }
            }
        }
        fence_before_sync();
        __syncthreads();   // the residual tile and the accumulator are reused
        fence_after_sync();
    }
    if (tid == 0) {
        // an abandoned Phi copy or MMA may still be in flight: wait for both (bounded)
        if (!ok) mbar_wait(bar_load, 0, kWaitNs);
        mma_commit(bar_mma);
        mbar_wait(bar_mma, ph, kWaitNs);
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 0) tmem_dealloc(tmem, 128);
}

}  // namespace

bool encode_tc_supported(const cs_plan* plan) {
    return plan->phi_tc != nullptr && plan->n == kN && plan->m >= 1 && plan->m <= kMaxM16;
}

cudaError_t launch_encode_tc(const cs_plan* plan, const GopShape& gs, const uint8_t* frames, float* y,
                             cudaStream_t s) {
    const long long rows = (long long)gs.n_cs * gs.nblk;
    if (rows == 0) return cudaSuccess;
    const int m16 = (plan->m + 15) / 16 * 16;
    const long long tiles = (rows + kTile - 1) / kTile;
    const int grid = (int)(tiles < plan->ctx->sm_count ? tiles : plan->ctx->sm_count);
    // 16-byte frame loads when every block row starts on a 16-byte boundary and
    // no block is cropped at the right edge
    const bool vec = gs.w % 16 == 0 && (reinterpret_cast<uintptr_t>(frames) & 15) == 0;
    cudaError_t e = cudaFuncSetAttribute(k_encode_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    k_encode_tc<<<grid, kT, kSmemBytes, s>>>(frames, plan->phi_tc, y, gs, m16,
                                             ldexpf(1.f, -plan->tc_ephi), vec, plan->ctx->err_dev);
    return cudaGetLastError();
}

}  // namespace csvc
