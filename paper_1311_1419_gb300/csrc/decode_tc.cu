// K6 + K7: persistent tensor-core decode on tcgen05.
//
// Recovery of every measured block by fixed-count FISTA on
// 1/2 ||A s - y||^2 + lambda ||s||_1 (Eq. 1 with an l1 regulariser in the DCT
// basis; Beck & Teboulle 2009), followed by r = Psi s and the key add-back of
// Eq. (4).  Across blocks the two products of every iteration are dense
// contractions, so a tile of 64 blocks runs them on the tensor cores:
//
//   GEMM1  U^T [M x 64] = A [M x N]   . Z^T [N x 64]     (u = A z per block)
//   GEMM2  G^T [N x 64] = A^T [N x M] . P^T [M x 64]     (g = A^T (u - y))
//
// One CTA per SM holds A (hi and lo halves of a 2-term split, fp16 or bf16,
// 128-byte swizzled) in shared memory for its whole life, loaded once by the
// bulk-copy engine.  The iterates never leave the SM: Y, Z and S_prev live in
// tensor memory next to the accumulators; the epilogue warps apply the soft
// threshold and the momentum step and write the next MMA operand (Z, or the
// residual P) back to shared memory as MN-major swizzled rows.  FP32-grade
// products use three MMAs (hi.hi + hi.lo + lo.hi); the mixed-precision modes
// run one MMA (hi.hi) until their FP32-grade tail.
//
// Roles: warps 0-7 are the epilogue (TMEM lane quarter = warp % 4, column
// half = warp / 4); warp 8 allocates TMEM, loads A and issues the MMAs.  Every
// wait on an mbarrier is bounded; a wait that gives up sets the context's
// error word and the CTA drains and exits without further work.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include "internal.h"
#include "tc_ptx.h"

namespace csvc {
namespace {

using namespace tc;

constexpr int kN = 256;              // coefficients per block (16 x 16 blocks)
constexpr int kMPad = 128;           // rows of A kept on chip (M <= 128)
constexpr int kTileBlocks = 64;      // blocks per tile = MMA N dimension
constexpr int kEpiWarps = 8;
constexpr int kThreads = (kEpiWarps + 1) * 32;
constexpr uint32_t kImgBytes = kMPad * kN * 2;          // one 16-bit image of A: 64 KB
constexpr uint32_t kZBytes = kN * kTileBlocks * 2;      // 32 KB
constexpr uint32_t kPBytes = kMPad * kTileBlocks * 2;   // 16 KB
constexpr uint32_t kOffAHi = 0, kOffALo = kImgBytes;
constexpr uint32_t kOffZHi = 2 * kImgBytes, kOffZLo = kOffZHi + kZBytes;
constexpr uint32_t kOffPHi = kOffZLo + kZBytes, kOffPLo = kOffPHi + kPBytes;
constexpr uint32_t kOffMisc = kOffPLo + kPBytes;        // 224 KB
constexpr uint32_t kSmemBytes = kOffMisc + 1024 + 1024; // misc + alignment slack
// TMEM columns
constexpr uint32_t kColU = 0, kColY = 64, kColG = 128, kColZ = 256, kColS = 384;
constexpr uint64_t kWaitNs = 2000000000ull;             // 2 s per wait

struct TcArgs {
    const uint8_t* a_img;   // hi image then lo image, 2 x 64 KB
    const float* y;
    const uint8_t* keys;
    float* out_f32;
    uint8_t* out_u8;
    const float* dct;       // [16][16]
    const float* beta;
    int* err;
    GopShape gs;
    long long rows;         // measured blocks in the call
    int n_tiles;
    int iters;
    int split_from;         // iterations k >= split_from use the 3-MMA split
    float lambda_rel;
    float inv_l;
    float su;               // U = acc * su
    float sg;               // G = acc * sg
    float sp;               // P operand = P * sp
};

struct Misc {
    uint64_t bar_load, bar_u, bar_g, bar_p, bar_z, bar_end;
    uint32_t tmem_base;
    int abort;
    uint32_t colmax[kTileBlocks];
    float tau[kTileBlocks];
};

template <bool BF>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
    if constexpr (BF) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    } else {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    }
}
template <bool BF>
__device__ __forceinline__ float2 unpack2(uint32_t v) {
    if constexpr (BF) {
        __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&v);
        return __bfloat1622float2(h);
    } else {
        __half2 h = *reinterpret_cast<__half2*>(&v);
        return __half22float2(h);
    }
}

// Write 32 values (blocks 32h .. 32h+31) of operand row `row` (8-row swizzle
// atoms, one 128-byte row of 64 blocks) as hi and, if wanted, lo halves.
template <bool BF>
__device__ __forceinline__ void write_operand_row(uint8_t* hi_base, uint8_t* lo_base, int row,
                                                  int half, const float (&v)[32], bool want_lo) {
    const uint32_t r = row & 7;
    uint8_t* hrow = hi_base + (row >> 3) * 1024 + r * 128;
    uint8_t* lrow = lo_base + (row >> 3) * 1024 + r * 128;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const uint32_t chunk = (uint32_t)(4 * half + c);
        uint32_t h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float a = v[8 * c + 2 * e], b = v[8 * c + 2 * e + 1];
            h[e] = pack2<BF>(a, b);
            if (want_lo) {
                const float2 hf = unpack2<BF>(h[e]);
                l[e] = pack2<BF>(a - hf.x, b - hf.y);
            }
        }
        const uint32_t off = ((chunk ^ r) << 4);
        *reinterpret_cast<uint4*>(hrow + off) = make_uint4(h[0], h[1], h[2], h[3]);
        if (want_lo) *reinterpret_cast<uint4*>(lrow + off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

__device__ __forceinline__ void epi_barrier() {
    asm volatile("bar.sync 1, %0;" ::"r"(kEpiWarps * 32) : "memory");
}

// Bounded wait; once any wait in the CTA has given up, later waits return at
// once so that every role drains through the same control flow.
__device__ __forceinline__ bool wait_bar(Misc* ms, uint64_t* bar, uint32_t parity, int* err) {
    if (*(volatile int*)&ms->abort) return false;
    if (mbar_wait(bar, parity, kWaitNs)) return true;
    *(volatile int*)&ms->abort = 1;
    atomicExch(err, 1);
    return false;
}

template <bool BF>
__global__ void __launch_bounds__(kThreads, 1) k_fista_tc(const TcArgs args) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
    Misc* ms = reinterpret_cast<Misc*>(sm + kOffMisc);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const GopShape& gs = args.gs;
    const int m_rows = gs.m;
    const int k_steps2 = (m_rows + 15) / 16;

    if (warp == kEpiWarps) {
        if (lane == 0) {
            mbar_init(&ms->bar_load, 1);
            mbar_init(&ms->bar_u, 1);
            mbar_init(&ms->bar_g, 1);
            mbar_init(&ms->bar_p, kEpiWarps);
            mbar_init(&ms->bar_z, kEpiWarps);
            mbar_init(&ms->bar_end, 1);
            ms->abort = 0;
            fence_mbar_init();
        }
        __syncwarp();
        tmem_alloc(&ms->tmem_base, 512);
        tmem_relinquish();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tbase = ms->tmem_base;

    if (warp == kEpiWarps) {
        // ------------------------------ MMA issuer ------------------------------
        if (lane == 0) {
            mbar_arrive_expect_tx(&ms->bar_load, 2 * kImgBytes);
            for (uint32_t off = 0; off < 2 * kImgBytes; off += 32768)
                bulk_g2s(sm + kOffAHi + off, args.a_img + off, 32768, &ms->bar_load);
            bool ok = wait_bar(ms, &ms->bar_load, 0, args.err);
            const uint32_t s_base = smem_u32(sm);
            const uint32_t id1 = idesc_f16(128, kTileBlocks, BF ? 1u : 0u, 0u, 1u);
            const uint32_t id2 = idesc_f16(128, kTileBlocks, BF ? 1u : 0u, 1u, 1u);
            uint32_t phase_z = 0, phase_p = 0;
            for (int tile = blockIdx.x; tile < args.n_tiles; tile += gridDim.x) {
                for (int k = 0; k < args.iters; ++k) {
                    const bool split = k >= args.split_from;
                    ok = wait_bar(ms, &ms->bar_z, phase_z, args.err) && ok;
                    phase_z ^= 1;
                    fence_after_sync();
                    if (ok) {
                        for (int ks = 0; ks < kN / 16; ++ks) {
                            const int n0 = 16 * ks;
                            const uint32_t a_off = (n0 / 64) * (kMPad / 8) * 1024 + ((n0 % 64) / 16) * 32;
                            const uint32_t z_off = (n0 / 8) * 1024;
                            const uint64_t ahi = desc_sw128(s_base + kOffAHi + a_off, 16, 1024);
                            const uint64_t zhi = desc_sw128(s_base + kOffZHi + z_off, 1024, 1024);
                            mma_f16(tbase + kColU, ahi, zhi, id1, ks > 0);
                            if (split) {
                                const uint64_t alo = desc_sw128(s_base + kOffALo + a_off, 16, 1024);
                                const uint64_t zlo = desc_sw128(s_base + kOffZLo + z_off, 1024, 1024);
                                mma_f16(tbase + kColU, ahi, zlo, id1, 1);
                                mma_f16(tbase + kColU, alo, zhi, id1, 1);
                            }
                        }
                        mma_commit(&ms->bar_u);
                    }
                    ok = wait_bar(ms, &ms->bar_p, phase_p, args.err) && ok;
                    phase_p ^= 1;
                    fence_after_sync();
                    if (ok) {
                        for (int slab = 0; slab < kN / 128; ++slab) {
                            for (int ks = 0; ks < k_steps2; ++ks) {
                                const uint32_t a_off = (2 * slab) * (kMPad / 8) * 1024 + (2 * ks) * 1024;
                                const uint32_t p_off = (2 * ks) * 1024;
                                const uint64_t ahi =
                                    desc_sw128(s_base + kOffAHi + a_off, (kMPad / 8) * 1024, 1024);
                                const uint64_t phi = desc_sw128(s_base + kOffPHi + p_off, 1024, 1024);
                                const uint32_t d = tbase + kColG + 64 * slab;
                                mma_f16(d, ahi, phi, id2, ks > 0);
                                if (split) {
                                    const uint64_t alo =
                                        desc_sw128(s_base + kOffALo + a_off, (kMPad / 8) * 1024, 1024);
                                    const uint64_t plo = desc_sw128(s_base + kOffPLo + p_off, 1024, 1024);
                                    mma_f16(d, ahi, plo, id2, 1);
                                    mma_f16(d, alo, phi, id2, 1);
                                }
                            }
                        }
                        mma_commit(&ms->bar_g);
                    }
                }
            }
            // drain: every MMA issued so far has completed before TMEM is freed
            mma_commit(&ms->bar_end);
            mbar_wait(&ms->bar_end, 0, kWaitNs);
            if (!ok) mbar_wait(&ms->bar_load, 0, kWaitNs);  // the A copy, if it never landed
        }
        __syncwarp();
    } else {
        // ------------------------------ epilogue ------------------------------
        const int q = warp & 3, half = warp >> 2;
        const int lrow = 32 * q + lane;                     // TMEM lane of this thread
        const uint32_t lane_addr = tbase + ((uint32_t)(32 * q) << 16);
        uint8_t* z_hi = sm + kOffZHi;
        uint8_t* z_lo = sm + kOffZLo;
        uint8_t* p_hi = sm + kOffPHi;
        uint8_t* p_lo = sm + kOffPLo;
        const float ginv = args.sg * args.inv_l;
        uint32_t phase_u = 0, phase_g = 0;
        for (int tile = blockIdx.x; tile < args.n_tiles; tile += gridDim.x) {
            const long long row0 = (long long)tile * kTileBlocks;
            // --- tile init: Y, Z = S = 0 in TMEM, Z operand = 0 ---
            {
                uint32_t r[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const long long row = row0 + 32 * half + j;
                    float v = 0.f;
                    if (lrow < m_rows && row < args.rows) v = args.y[row * m_rows + lrow];
                    r[j] = __float_as_uint(v);
                }
                tmem_st32(lane_addr + kColY + 32 * half, r);
#pragma unroll
                for (int j = 0; j < 32; ++j) r[j] = 0u;
                for (int slab = 0; slab < 2; ++slab) {
                    tmem_st32(lane_addr + kColZ + 64 * slab + 32 * half, r);
                    tmem_st32(lane_addr + kColS + 64 * slab + 32 * half, r);
                }
                const float zero[32] = {};
                for (int slab = 0; slab < 2; ++slab)
                    write_operand_row<BF>(z_hi, z_lo, 128 * slab + lrow, half, zero, true);
                if (threadIdx.x < kTileBlocks) ms->colmax[threadIdx.x] = 0u;
                tmem_wait_st();
            }
            fence_proxy_async_smem();
            fence_before_sync();
            epi_barrier();
            if (args.iters > 0) {
                __syncwarp();
                if (lane == 0) mbar_arrive(&ms->bar_z);
            }
            for (int k = 0; k < args.iters; ++k) {
                // --- P = U - Y, as the MMA operand of GEMM2 ---
                const bool ok_u = wait_bar(ms, &ms->bar_u, phase_u, args.err);
                phase_u ^= 1;
                fence_after_sync();
                {
                    uint32_t u[32], yv[32];
                    tmem_ld32(lane_addr + kColU + 32 * half, u);
                    tmem_ld32(lane_addr + kColY + 32 * half, yv);
                    tmem_wait_ld();
                    float p[32];
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        p[j] = (__uint_as_float(u[j]) * args.su - __uint_as_float(yv[j])) * args.sp;
                    if (ok_u) write_operand_row<BF>(p_hi, p_lo, lrow, half, p, k >= args.split_from);
                }
                fence_proxy_async_smem();
                fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(&ms->bar_p);

                // --- gradient step, soft threshold, momentum ---
                const bool ok_g = wait_bar(ms, &ms->bar_g, phase_g, args.err);
                phase_g ^= 1;
                fence_after_sync();
                if (k == 0) {
                    // lambda_b = lambda_rel ||A^T y_b||_inf; here G = -A^T y
                    for (int slab = 0; slab < 2; ++slab) {
                        uint32_t g[32];
                        tmem_ld32(lane_addr + kColG + 64 * slab + 32 * half, g);
                        tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const float a = fabsf(__uint_as_float(g[j]) * args.sg);
                            const uint32_t mx = __reduce_max_sync(0xffffffffu, __float_as_uint(a));
                            if (lane == 0) atomicMax(&ms->colmax[32 * half + j], mx);
                        }
                    }
                    epi_barrier();
                    if (threadIdx.x < kTileBlocks)
                        ms->tau[threadIdx.x] =
                            args.lambda_rel * __uint_as_float(ms->colmax[threadIdx.x]) * args.inv_l;
                    epi_barrier();
                }
                const float bk = args.beta[k];
                const bool want_z = k + 1 < args.iters;
                const bool z_split = k + 1 >= args.split_from;
                for (int slab = 0; slab < 2; ++slab) {
                    uint32_t g[32], z[32], s[32];
                    tmem_ld32(lane_addr + kColG + 64 * slab + 32 * half, g);
                    tmem_ld32(lane_addr + kColZ + 64 * slab + 32 * half, z);
                    tmem_ld32(lane_addr + kColS + 64 * slab + 32 * half, s);
                    tmem_wait_ld();
                    float zn[32];
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float tau = ms->tau[32 * half + j];
                        const float v = fmaf(-__uint_as_float(g[j]), ginv, __uint_as_float(z[j]));
                        const float sv = v - fminf(fmaxf(v, -tau), tau);
                        const float znew = fmaf(bk, sv - __uint_as_float(s[j]), sv);
                        zn[j] = znew;
                        z[j] = __float_as_uint(znew);
                        s[j] = __float_as_uint(sv);
                    }
                    tmem_st32(lane_addr + kColZ + 64 * slab + 32 * half, z);
                    tmem_st32(lane_addr + kColS + 64 * slab + 32 * half, s);
                    if (want_z && ok_g) write_operand_row<BF>(z_hi, z_lo, 128 * slab + lrow, half, zn, z_split);
                }
                tmem_wait_st();
                if (want_z) {
                    fence_proxy_async_smem();
                    fence_before_sync();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&ms->bar_z);
                }
            }
            // --- reconstruct: S (= s^K) -> R = C^T S C, add the key, store ---
            epi_barrier();   // the operand area is free: no MMA is pending for this tile
            float* s_f = reinterpret_cast<float*>(sm + kOffZHi);          // [64][256]
            float* c_s = reinterpret_cast<float*>(sm + kOffPHi);          // [16][16]
            float* t_w = c_s + 256 + warp * 256;                          // per-warp [16][16]
            for (int slab = 0; slab < 2; ++slab) {
                uint32_t s[32];
                tmem_ld32(lane_addr + kColS + 64 * slab + 32 * half, s);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    s_f[(32 * half + j) * kN + 128 * slab + lrow] = __uint_as_float(s[j]);
            }
            for (int i = threadIdx.x; i < 256; i += kEpiWarps * 32) c_s[i] = args.dct[i];
            epi_barrier();
            const size_t frame_px = (size_t)gs.h * gs.w;
            for (int bl = warp; bl < kTileBlocks; bl += kEpiWarps) {
                const long long row = row0 + bl;
                if (row >= args.rows) break;
                const float* sb = s_f + bl * kN;
                const int qc = lane & 15, r0 = lane >> 4;
                // T = S C (rows k = r0, r0+2, ...)
#pragma unroll
                for (int kk = r0; kk < 16; kk += 2) {
                    float acc = 0.f;
#pragma unroll
                    for (int l = 0; l < 16; ++l) acc = fmaf(sb[kk * 16 + l], c_s[l * 16 + qc], acc);
                    t_w[kk * 16 + qc] = acc;
                }
                __syncwarp();
                const int c = (int)(row / gs.nblk), blk = (int)(row % gs.nblk);
                const int g = c / (gs.g - 1);
                const int bi = blk / gs.nbc, bj = blk % gs.nbc;
#pragma unroll
                for (int pp = r0; pp < 16; pp += 2) {
                    float acc = 0.f;
#pragma unroll
                    for (int kk = 0; kk < 16; ++kk) acc = fmaf(c_s[kk * 16 + pp], t_w[kk * 16 + qc], acc);
                    const int py = bi * 16 + pp, px = bj * 16 + qc;
                    if (py < gs.h && px < gs.w) {
                        const size_t off = (size_t)py * gs.w + px;
                        const float v = (float)args.keys[(size_t)g * frame_px + off] + acc;
                        if (args.out_f32) args.out_f32[(size_t)c * frame_px + off] = v;
                        if (args.out_u8)
                            args.out_u8[(size_t)c * frame_px + off] =
                                (uint8_t)fminf(fmaxf(rintf(v), 0.f), 255.f);
                    }
                }
                __syncwarp();
            }
            epi_barrier();   // s_f / c_s are overwritten by the next tile's init
        }
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == kEpiWarps) tmem_dealloc(tbase, 512);
}

// Scales of the fp16 operands: max |A| and max_m sum_n |Phi[m][n]|.
__global__ void k_tc_ranges(const float* __restrict__ a, const float* __restrict__ phi, int n, int m,
                            float* __restrict__ out) {
    __shared__ float red_a[32], red_l[32];
    float amax = 0.f, lmax = 0.f;
    for (int row = threadIdx.x >> 5; row < m; row += blockDim.x >> 5) {
        float l1 = 0.f;
        for (int c = threadIdx.x & 31; c < n; c += 32) {
            amax = fmaxf(amax, fabsf(a[(size_t)row * n + c]));
            l1 += fabsf(phi[(size_t)row * n + c]);
        }
        for (int off = 16; off > 0; off >>= 1) l1 += __shfl_xor_sync(0xffffffffu, l1, off);
        lmax = fmaxf(lmax, l1);
    }
    for (int off = 16; off > 0; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, off));
    if ((threadIdx.x & 31) == 0) {
        red_a[threadIdx.x >> 5] = amax;
        red_l[threadIdx.x >> 5] = lmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float x = 0.f, y = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            x = fmaxf(x, red_a[w]);
            y = fmaxf(y, red_l[w]);
        }
        out[0] = x;
        out[1] = y;
    }
}

// The four 64 KB shared-memory images of A * 2^ea: fp16 hi, fp16 lo, bf16 hi,
// bf16 lo, rows >= M zero, 128-byte swizzled as in the kernel.
__global__ void k_tc_images(const float* __restrict__ a, uint8_t* __restrict__ img, int n, int m,
                            float scale) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= kMPad * kN) return;
    const int row = idx / kN, col = idx % kN;
    const float v = row < m ? a[(size_t)row * n + col] * scale : 0.f;
    const uint32_t off = sw128_offset((uint32_t)row, (uint32_t)col, kMPad / 8);
    const __half hh = __float2half_rn(v);
    const __half hl = __float2half_rn(v - __half2float(hh));
    const __nv_bfloat16 bh = __float2bfloat16_rn(v);
    const __nv_bfloat16 bl = __float2bfloat16_rn(v - __bfloat162float(bh));
    *reinterpret_cast<__half*>(img + off) = hh;
    *reinterpret_cast<__half*>(img + kImgBytes + off) = hl;
    *reinterpret_cast<__nv_bfloat16*>(img + 2 * kImgBytes + off) = bh;
    *reinterpret_cast<__nv_bfloat16*>(img + 3 * kImgBytes + off) = bl;
}

}  // namespace

bool tc_plan_supported(int n, int m) { return n == kN && m >= 1 && m <= kMPad; }
size_t tc_operand_bytes() { return 4ull * kImgBytes; }

cudaError_t launch_tc_ranges(const float* a, const float* phi, int n, int m, float* out,
                             cudaStream_t s) {
    k_tc_ranges<<<1, 1024, 0, s>>>(a, phi, n, m, out);
    return cudaGetLastError();
}

cudaError_t launch_tc_images(const float* a, uint8_t* img, int n, int m, int ea, cudaStream_t s) {
    const int total = kMPad * kN;
    k_tc_images<<<(total + 255) / 256, 256, 0, s>>>(a, img, n, m, ldexpf(1.f, ea));
    return cudaGetLastError();
}

bool tc_supported(const cs_plan* plan, int precision) {
    (void)precision;
    return plan->a_tc != nullptr && tc_plan_supported(plan->n, plan->m);
}

cudaError_t launch_decode_tc(const DecodeArgs& d, cudaStream_t s) {
    const GopShape& gs = d.gs;
    const long long rows = (long long)gs.n_cs * gs.nblk;
    if (rows == 0) return cudaSuccess;
    const cs_plan* p = d.plan;
    TcArgs a;
    const bool bf = d.precision == CS_BF16 || d.precision == CS_BF16X2;
    a.a_img = p->a_tc + (bf ? 2 * kImgBytes : 0);
    a.y = d.y;
    a.keys = d.key;
    a.out_f32 = d.out_f32;
    a.out_u8 = d.out_u8;
    a.dct = p->dct;
    a.beta = d.beta;
    a.err = p->ctx->err_dev;
    a.gs = gs;
    a.rows = rows;
    a.n_tiles = (int)((rows + kTileBlocks - 1) / kTileBlocks);
    a.iters = d.iters;
    const bool mixed = d.precision == CS_BF16 || d.precision == CS_FP16;
    a.split_from = mixed ? (d.iters > d.tail_iters ? d.iters - d.tail_iters : 0) : 0;
    a.lambda_rel = d.lambda_rel;
    a.inv_l = (float)(1.0 / p->lipschitz);
    a.su = ldexpf(1.f, -p->tc_ea);
    a.sg = ldexpf(1.f, -(p->tc_ea + p->tc_ep));
    a.sp = ldexpf(1.f, p->tc_ep);
    const int sms = p->ctx->sm_count;
    const int grid = a.n_tiles < sms ? a.n_tiles : sms;
    cudaError_t e;
    if (bf) {
        e = cudaFuncSetAttribute(k_fista_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSmemBytes);
        if (e != cudaSuccess) return e;
        k_fista_tc<true><<<grid, kThreads, kSmemBytes, s>>>(a);
    } else {
        e = cudaFuncSetAttribute(k_fista_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSmemBytes);
        if (e != cudaSuccess) return e;
        k_fista_tc<false><<<grid, kThreads, kSmemBytes, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace csvc
