// Tensor-core FISTA for 16 x 16 and 32 x 32 blocks with up to 128 measurements:
// A streamed from L2, the iterates in global memory at 12 bytes of traffic per
// coefficient and iteration.
//
// The recovery is the fixed-count FISTA of the other decode kernels (Eq. 1 with
// an l1 regulariser in the DCT basis; Beck & Teboulle 2009), then r = Psi s and
// the key add-back of Eq. 4.  A tile of 128 blocks (the MMA's M dimension, one
// block per TMEM lane) is one CTA's work, one CTA per SM.  An iteration runs
// over chunks c of 128 coefficients:
//
//   GEMM2  G_c [128 x 128]  = P [128 x M16] . A[:, c]
//   step   s^k_c = soft(z^k_c - G_c / L),  z^{k+1}_c = s^k_c + beta_k (s^k_c - s^{k-1}_c)
//   GEMM1  U [128 x M16]   += Z^{k+1}_c . A[:, c]^T        (Z^{k+1}_c from tensor memory)
//
// and ends with P = U - y, the next iteration's GEMM2 operand.  GEMM1 is split
// along K into the chunks of GEMM2: each chunk's part is issued as soon as the
// step has put that chunk of z^{k+1} (fp16 hi and lo) into tensor memory, so z
// never goes to global memory.  The step recomputes z^k = s^{k-1} +
// beta_{k-1} (s^{k-1} - s^{k-2}) in FP32 from the two previous iterates, which
// stay in global memory (the new s^k is written over s^{k-2}): 8 bytes read and
// 4 written per coefficient and iteration, the reads past L1 so that L1 keeps the
// tile's y rows, which every iteration's residual reads again.  P stays in shared
// memory; only the slices of A's two images stream, through a six-stage ring fed
// by a copy warp.
// Tensor memory: two 128-column G accumulators (the step of chunk c overlaps
// GEMM2 of chunk c + 1), U (M16 columns) and the Z chunk's hi and lo halves.
// Mixed precision: a split product uses three MMAs (hi.hi + lo.hi + hi.lo), a
// bulk one hi.hi only.  Every mbarrier wait is bounded and reports through the
// context's error word; a CTA that gives up drains its copies and MMAs.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "tc_ptx.h"

namespace csvc {
namespace {

using namespace tc;

constexpr int kTile = 128;                  // blocks per tile = TMEM lanes = MMA M
constexpr int kCc = 128;                    // coefficients per chunk
constexpr int kMaxM16z = 128;
constexpr int kEpiWarps = 16;               // 4 TMEM lane quarters x 4 column groups
constexpr int kColGroups = kEpiWarps / 4;
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kThreads = 64 + kEpiThreads;  // warp 0 MMAs, warp 1 copies, warps 2 .. 17 epilogue
constexpr int kPerThread = kCc / kColGroups;  // coefficients of a chunk per epilogue thread
constexpr int kSliceK = 32;                 // K per ring slot: one 64-byte swizzle atom
constexpr uint32_t kHalfBytes = 8192;       // one slice of A, hi or lo: 32 x 128 or M16 x 32 fp16
constexpr uint32_t kStageBytes = 2 * kHalfBytes;
constexpr int kStages = 6;
constexpr uint32_t kTBytes = kTile * 64;    // one 32-wide K slice of P (8 KB)
constexpr uint32_t kPBytes = (kMaxM16z / kSliceK) * kTBytes;   // P hi (or lo): 32 KB
constexpr uint32_t kOffP = kStages * kStageBytes;              // P hi, then P lo
constexpr uint32_t kOffMisc = kOffP + 2 * kPBytes;
// 162 KB in all: with the SM's 1 KB reserve it fits the 164 KB shared-memory split, which
// leaves about 92 KB of L1 for the tile's y rows, read again every iteration (the DCT
// matrix waits in the P area, idle during reconstruction)
constexpr uint32_t kSmemBytes = kOffMisc + 1024 + 1024;        // + alignment slack
constexpr uint32_t kColG = 0;               // two G accumulators of 128 columns
constexpr uint32_t kColU = 256;             // U: M16 <= 128 columns
// the Z chunk in two halves: half h holds coefficients 32 j + 16 h .. 32 j + 16 h + 15 of
// the chunk (j = 0 .. 3), hi then lo, 32 columns each
constexpr uint32_t kColZ = 384;
__host__ __device__ constexpr uint32_t zcol_hi(int h) { return kColZ + 64u * (uint32_t)h; }
__host__ __device__ constexpr uint32_t zcol_lo(int h) { return kColZ + 64u * (uint32_t)h + 32u; }
// per-CTA scratch: two s buffers (N floats per block, [N / 4][128 blocks] float4),
// then the tile's y ([M16 / 4][128] float4)
constexpr size_t kScrS = (size_t)1024 * kTile * 4;
constexpr size_t kScrY = 2 * kScrS;
constexpr size_t kScrBytesZ = kScrY + (size_t)kMaxM16z * kTile * 4;
constexpr uint64_t kWaitNs = 1000000000ull;  // 1 s per wait
constexpr uint32_t kBarEpi = 1;              // named barrier of the epilogue
constexpr int kMaxJobsZ = 48;

}  // namespace

// One job of a launch: the blocks of one cs_decode_gop call (or a range of them).
struct TczJob {
    const uint8_t* a1_img;  // GEMM1 image of A 2^ea (32-column K slices): hi then lo
    const uint8_t* a2_img;  // GEMM2 image (32-row K slices, MN-major): hi then lo
    const float* y;
    const uint8_t* keys;
    float* out_f32;
    uint8_t* out_u8;
    const float* dct;       // [B][B]
    GopShape gs;
    long long row0;         // first measured block of the job
    long long rows;         // end (exclusive)
    int tile_begin;
    int n, m16, iters;
    int split_from;         // iterations k >= split_from use the 3-MMA split
    float lambda_rel, inv_l;
    float su, sg, sp;       // U = acc su, G = acc sg, P operand = P sp
};
struct TczLaunch {
    const float* beta;
    int* err;
    int* tile_counter;
    uint8_t* scratch;       // gridDim.x areas of kScrBytesZ
    int drop_arrival;       // test hook: CTA 0 withholds one epilogue warp's first P-ready arrival
    int n_jobs;
    int n_tiles;
    TczJob jobs[kMaxJobsZ];
};

namespace {

struct MiscZ {
    uint64_t full[kStages], empty[kStages];
    uint64_t acc_full[2], acc_empty[2];
    uint64_t z_full[2], z_empty[2], u_full, p_ready, drain;
    uint32_t tmem_base;
    int abort;
    int next_tile;
    int job;
    uint32_t colmax[kTile];
};
static_assert(sizeof(MiscZ) <= 1024, "barrier block");
static_assert(kOffMisc + sizeof(MiscZ) + 1024 <= kSmemBytes, "shared memory layout");

template <bool BF>
__device__ __forceinline__ uint32_t pack2z(float2 v) {
    if constexpr (BF) {
        __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
        return *reinterpret_cast<uint32_t*>(&h);
    } else {
        __half2 h = __floats2half2_rn(v.x, v.y);
        return *reinterpret_cast<uint32_t*>(&h);
    }
}
template <bool BF>
__device__ __forceinline__ float2 unpack2z(uint32_t v) {
    if constexpr (BF) {
        __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&v);
        return __bfloat1622float2(h);
    } else {
        __half2 h = *reinterpret_cast<__half2*>(&v);
        return __half22float2(h);
    }
}

__device__ __forceinline__ bool wait_z(MiscZ* ms, uint64_t* bar, uint32_t parity, int* err) {
    if (*(volatile int*)&ms->abort) return false;
    if (mbar_wait(bar, parity, kWaitNs)) return true;
    *(volatile int*)&ms->abort = 1;
    atomicExch(err, 1);
    return false;
}
__device__ __forceinline__ void cta_sync_z() {
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
}
// The CTA's next tile (thread 0 claims it; every thread gets it): -1 when none is left.
__device__ __forceinline__ int fetch_tile_z(const TczLaunch& L, MiscZ* ms) {
    if (threadIdx.x == 0) {
        const int t = atomicAdd(L.tile_counter, 1);
        int j = -1;
        if (t < L.n_tiles) {
            j = 0;
            while (j + 1 < L.n_jobs && L.jobs[j + 1].tile_begin <= t) ++j;
        }
        ms->job = j;
        ms->next_tile = t < L.n_tiles ? t : -1;
    }
    __syncthreads();
    return ms->next_tile;
}

__device__ __forceinline__ int p_slices_z(int m16) { return (m16 + kSliceK - 1) / kSliceK; }

// The ring's sequence of A slices for one chunk step of GEMM2 (K = M16 in 32-row
// slices) and of GEMM1 (K = the chunk's 128 coefficients in 32-column slices).
// Passes of a tile: 0 = GEMM2 over every chunk for lambda; then, per iteration k,
// for each chunk c: GEMM2 of chunk c, then GEMM1 of chunk c - 1 (and, after the
// last chunk, GEMM1 of the last chunk) while k + 1 < K.

// One A slice into a ring stage: GEMM2 slice ks of chunk c (rows 32 ks .. of
// coefficients 128 c ..: 8 KB, contiguous in the GEMM2 image) or GEMM1 slice ks
// of chunk c (columns 128 c + 32 ks .., every row: M16 x 64 bytes, contiguous in
// the GEMM1 image); the lo half 8 KB after the hi half when split.
__device__ __forceinline__ void copy_slice_z(const TczJob& J, uint8_t* stg, uint64_t* full, bool g2, int c, int ks,
                                             bool split) {
    const int n = J.n, m16 = J.m16;
    const uint32_t bytes = g2 ? (uint32_t)kCc * 64u : (uint32_t)m16 * 64u;
    const size_t img1 = (size_t)m16 * n * 2, img2 = (size_t)((m16 + 31) / 32 * 32) * n * 2;
    const size_t off = g2 ? ((size_t)ks * (n / 32) + (size_t)c * (kCc / 32)) * 2048
                          : (size_t)(c * (kCc / kSliceK) + ks) * (size_t)(m16 / 8) * 512;
    const uint8_t* src = g2 ? J.a2_img : J.a1_img;
    mbar_arrive_expect_tx(full, (split ? 2u : 1u) * bytes);
    bulk_g2s(stg, src + off, bytes, full);
    if (split) bulk_g2s(stg + kHalfBytes, src + (g2 ? img2 : img1) + off, bytes, full);
}

// Warp 1: streams the A slices of every pass into the stage ring, in the order
// the MMA warp takes them.  A is constant, so the warp runs ahead as far as the
// ring allows.
__device__ __forceinline__ void copy_role_z(const TczLaunch& L, MiscZ* ms, uint8_t* sm, int lane) {
    uint32_t st = 0, last_par = 0, issued = 0;   // per stage, one bit each
    bool ok = true;
    for (;;) {
        const int tile = fetch_tile_z(L, ms);
        if (tile < 0) break;
        const TczJob& J = L.jobs[ms->job];
        cta_sync_z();   // B
        const int K = J.iters, nch = J.n / kCc, ns2 = p_slices_z(J.m16), ns1 = kCc / kSliceK;
        auto put = [&](bool g2, int c, bool split) {
            const int ns = g2 ? ns2 : ns1;
            for (int ks = 0; ks < ns; ++ks) {
                const uint32_t s = st % kStages, par = (st / kStages) & 1;
                ok = wait_z(ms, &ms->empty[s], par ^ 1, L.err) && ok;
                if (ok && lane == 0) {
                    copy_slice_z(J, sm + s * kStageBytes, &ms->full[s], g2, c, ks, split);
                    last_par = (last_par & ~(1u << s)) | (par << s);
                    issued |= 1u << s;
                }
                __syncwarp();
                ++st;
            }
        };
        if (K > 0) {
            for (int c = 0; c < nch; ++c) put(true, c, 0 >= J.split_from);   // lambda
            for (int k = 0; k < K; ++k) {
                const bool split = k >= J.split_from, want_z = k + 1 < K, zsplit = k + 1 >= J.split_from;
                for (int c = 0; c < nch; ++c) {
                    put(true, c, split);
                    if (want_z && c > 0) put(false, c - 1, zsplit);
                }
                if (want_z) put(false, nch - 1, zsplit);
            }
        }
        cta_sync_z();   // C
    }
    if (lane == 0) {
        // copies whose consumer gave up may still be in flight (bounded)
        for (int s = 0; s < kStages; ++s)
            if ((issued >> s) & 1u) mbar_wait(&ms->full[s], (last_par >> s) & 1u, kWaitNs);
    }
    __syncwarp();
}

// Warp 0: issues every MMA (lane 0).  GEMM2 of a chunk goes into the next of the
// two G accumulators.  GEMM1 of a chunk adds into U in two halves: the first K
// step of every 32-coefficient slice once the epilogue has put the chunk's half-A Z
// into tensor memory (z_full[0]), then the second once half B is there (z_full[1]);
// each half frees its Z columns again (z_empty[h]).  A slice serves both halves, so
// its ring stage is released after half B.  The last chunk's GEMM1 also completes U
// (u_full).  GEMM1 of z^{k+1} is split (or not) as iteration k + 1's products are.
template <bool BF>
__device__ __forceinline__ void mma_role_z(const TczLaunch& L, MiscZ* ms, uint8_t* sm, uint32_t tbase, int lane) {
    const uint32_t s_base = smem_u32(sm);
    uint32_t st = 0, acc = 0, zt = 0, pc = 0;
    bool ok = true;
    for (;;) {
        const int tile = fetch_tile_z(L, ms);
        if (tile < 0) break;
        const TczJob& J = L.jobs[ms->job];
        cta_sync_z();   // B
        const int K = J.iters, nch = J.n / kCc, m16 = J.m16;
        const uint32_t id2 = idesc_f16(128, kCc, BF ? 1u : 0u, 0u, 1u);
        const uint32_t id1 = idesc_f16(128, (uint32_t)m16, BF ? 1u : 0u, 0u, 0u);
        auto gemm2 = [&](bool split) {
            const uint32_t a = acc & 1;
            ok = wait_z(ms, &ms->acc_empty[a], ((acc >> 1) & 1) ^ 1, L.err) && ok;
            fence_after_sync();
            const uint32_t d = tbase + kColG + a * kCc;
            const int ns = p_slices_z(m16);
#pragma unroll 1
            for (int ks = 0; ks < ns; ++ks) {
                const uint32_t s = st % kStages, par = (st / kStages) & 1;
                ok = wait_z(ms, &ms->full[s], par, L.err) && ok;
                fence_after_sync();
                if (ok && lane == 0) {
                    const uint32_t stg = s_base + s * kStageBytes;
                    // P: K-major, 8-row groups 512 bytes apart; the A slice: MN-major,
                    // 32-column atoms 2 KB apart, 8-row K groups 512 bytes apart
                    const uint64_t p_hi = desc_sw64(s_base + kOffP + (uint32_t)ks * kTBytes, 16, 512);
                    const uint64_t p_lo = desc_sw64(s_base + kOffP + kPBytes + (uint32_t)ks * kTBytes, 16, 512);
                    const uint64_t b_hi = desc_sw64(stg, 2048, 512);
                    const uint64_t b_lo = desc_sw64(stg + kHalfBytes, 2048, 512);
                    const int nk = min(2, m16 / 16 - 2 * ks);
                    for (int kk = 0; kk < nk; ++kk) {
                        const uint32_t to = (uint32_t)kk * 2u, bo = (uint32_t)kk * 64u;
                        mma_f16(d, p_hi + to, b_hi + bo, id2, (ks > 0 || kk > 0) ? 1u : 0u);
                        if (split) {
                            mma_f16(d, p_lo + to, b_hi + bo, id2, 1u);
                            mma_f16(d, p_hi + to, b_lo + bo, id2, 1u);
                        }
                    }
                    mma_commit(&ms->empty[s]);
                }
                __syncwarp();
                ++st;
            }
            if (ok && lane == 0) mma_commit(&ms->acc_full[a]);
            __syncwarp();
            ++acc;
        };
        uint32_t g1_stage[kCc / kSliceK];   // the ring stages of the chunk's GEMM1 slices
        auto gemm1 = [&](int c, int h, bool split, bool last) {
            ok = wait_z(ms, &ms->z_full[h], zt & 1, L.err) && ok;
            fence_after_sync();
#pragma unroll
            for (int ks = 0; ks < kCc / kSliceK; ++ks) {
                if (h == 0) {   // the slices arrive for half A and stay for half B
                    const uint32_t s = st % kStages, par = (st / kStages) & 1;
                    ok = wait_z(ms, &ms->full[s], par, L.err) && ok;
                    fence_after_sync();
                    g1_stage[ks] = s;
                    ++st;
                }
                if (ok && lane == 0) {
                    const uint32_t s = g1_stage[ks];
                    const uint32_t stg = s_base + s * kStageBytes;
                    const uint64_t b_hi = desc_sw64(stg, 16, 512);   // K-major: M16 rows of 32 columns
                    const uint64_t b_lo = desc_sw64(stg + kHalfBytes, 16, 512);
                    const uint32_t zc = (uint32_t)(8 * ks);           // 16 coefficients = 8 columns
                    const uint32_t bo = (uint32_t)h * 2u;             // the slice's K step h
                    const uint32_t accum = (c > 0 || ks > 0 || h > 0) ? 1u : 0u;
                    mma_f16_tmem_a(tbase + kColU, tbase + zcol_hi(h) + zc, b_hi + bo, id1, accum);
                    if (split) {
                        mma_f16_tmem_a(tbase + kColU, tbase + zcol_lo(h) + zc, b_hi + bo, id1, 1u);
                        mma_f16_tmem_a(tbase + kColU, tbase + zcol_hi(h) + zc, b_lo + bo, id1, 1u);
                    }
                    if (h == 1) mma_commit(&ms->empty[s]);
                }
                __syncwarp();
            }
            if (ok && lane == 0) {
                mma_commit(&ms->z_empty[h]);
                if (last && h == 1) mma_commit(&ms->u_full);
            }
            __syncwarp();
            if (h == 1) ++zt;
        };
        if (K > 0) {
            ok = wait_z(ms, &ms->p_ready, pc & 1, L.err) && ok;   // P_0 = -y
            ++pc;
            for (int c = 0; c < nch; ++c) gemm2(0 >= J.split_from);   // lambda
            for (int k = 0; k < K; ++k) {
                const bool split = k >= J.split_from, want_z = k + 1 < K, zsplit = k + 1 >= J.split_from;
                if (k > 0) {
                    ok = wait_z(ms, &ms->p_ready, pc & 1, L.err) && ok;
                    ++pc;
                }
                for (int c = 0; c < nch; ++c) {
                    gemm2(split);
                    if (want_z && c > 0) {
                        gemm1(c - 1, 0, zsplit, false);
                        gemm1(c - 1, 1, zsplit, false);
                    }
                }
                if (want_z) {
                    gemm1(nch - 1, 0, zsplit, true);
                    gemm1(nch - 1, 1, zsplit, true);
                }
            }
        }
        cta_sync_z();   // C
    }
    if (lane == 0) {
        // every MMA issued so far has completed before tensor memory is freed
        mma_commit(&ms->drain);
        mbar_wait(&ms->drain, 0, kWaitNs);
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// Epilogue pieces.  Thread: TMEM lane / tile row r = 32 q + lane (q = warp % 4),
// column group cg: a quarter of U's columns and 32 coefficients of every chunk.

// P = (U su - y) sp for the thread's quarter of the M16 columns (U = 0 at k = 0)
// into the shared P operand (64-byte-swizzled K-major slices of 32 columns), fp16
// (bf16) hi and, when split, lo.
template <bool BF>
__device__ __forceinline__ void residual_z(const TczJob& J, uint8_t* p_hi, uint8_t* p_lo, uint32_t lane_addr,
                                           int cg, int r, const float4* __restrict__ y4, bool use_u, bool split) {
    const int w4 = J.m16 / kColGroups;   // a multiple of 4
    const int i0 = cg * w4;
    for (int c0 = 0; c0 < w4; c0 += 16) {
        uint32_t u[4][4];
        float4 yv[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
#pragma unroll
            for (int e = 0; e < 4; ++e) u[t][e] = 0u;
            if (use_u && c0 + 4 * t < w4) tmem_ld4(lane_addr + kColU + (uint32_t)(i0 + c0 + 4 * t), u[t]);
            yv[t] = c0 + 4 * t < w4 ? y4[(size_t)((i0 + c0) / 4 + t) * kTile + r] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (use_u) tmem_wait_ld();
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if (c0 + 4 * t >= w4) break;
            const int i = i0 + c0 + 4 * t;
            const float yy[4] = {yv[t].x, yv[t].y, yv[t].z, yv[t].w};
            float p[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) p[e] = (__uint_as_float(u[t][e]) * J.su - yy[e]) * J.sp;
            const uint32_t h0 = pack2z<BF>(make_float2(p[0], p[1])), h1 = pack2z<BF>(make_float2(p[2], p[3]));
            const uint32_t off = sw64_offset((uint32_t)r, (uint32_t)i, kTile / 8);
            *reinterpret_cast<uint2*>(p_hi + off) = make_uint2(h0, h1);
            if (split) {
                const float2 d0 = unpack2z<BF>(h0), d1 = unpack2z<BF>(h1);
                *reinterpret_cast<uint2*>(p_lo + off) =
                    make_uint2(pack2z<BF>(make_float2(p[0] - d0.x, p[1] - d0.y)),
                               pack2z<BF>(make_float2(p[2] - d1.x, p[3] - d1.y)));
            }
        }
    }
}

// lambda pass: max |G| over the thread's 32 columns from gaddr.
__device__ __forceinline__ float gmax_z(uint32_t gaddr, float mx) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t g0[8], g1[8];
        tmem_ld8(gaddr + 16 * h, g0);
        tmem_ld8(gaddr + 16 * h + 8, g1);
        tmem_wait_ld();
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            mx = fmaxf(mx, fabsf(__uint_as_float(g0[e])));
            mx = fmaxf(mx, fabsf(__uint_as_float(g1[e])));
        }
    }
    return mx;
}

// The thread's s^{k-1} (a) and s^{k-2} (c) for 16 coefficients at float4 index v0 ..
// (each 128 float4 apart): zero where iteration k has none (k < 1, k < 2).  The
// loads skip L1, which keeps y's rows there.
__device__ __forceinline__ void load_s_z(const float4* __restrict__ s1, const float4* __restrict__ s2, size_t v0,
                                         int k, float4 (&a)[4], float4 (&c)[4]) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        a[v] = k >= 1 ? ld_stream4(s1 + v0 + (size_t)v * kTile) : make_float4(0.f, 0.f, 0.f, 0.f);
        c[v] = k >= 2 ? ld_stream4(s2 + v0 + (size_t)v * kTile) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// The step for the thread's 32 coefficients of one chunk, 16 at a time (G from
// accumulator columns gaddr ..; the coefficients' s values at float4 index v0 ..
// v0 + 7, each 128 float4 apart): z^k = s^{k-1} + beta_{k-1} (s^{k-1} - s^{k-2})
// (0 at k = 0), s^k = soft(z^k - g / L, tau) written over s^{k-2}, and, when
// want_z, z^{k+1} = s^k + beta_k (s^k - s^{k-1}) as hi / lo pairs into tensor
// memory: 16 coefficients h into Z half h at column zoff of its hi and lo parts,
// once GEMM1 has finished with that half of the previous chunk (z_empty[h]), each
// half announced at once (z_full[h]) so that its GEMM1 runs beside the rest of the
// step.  The first 16 coefficients' s values arrive loaded in (pa, pc);
// when nk >= 0 the step leaves there the first 16 of the next chunk's (iteration
// nk, index nv0 in n1 / n2), so that their loads overlap the hand-over between
// chunks.
template <bool BF>
__device__ __forceinline__ void step_z(const TczJob& J, const TczLaunch& L, MiscZ* ms, const float4* __restrict__ s1,
                                       float4* __restrict__ s2, size_t v0, uint32_t gaddr, uint32_t zoff, int k,
                                       float tau, bool want_z, uint32_t& zw, int lane, float4 (&pa)[4], float4 (&pc)[4],
                                       const float4* __restrict__ n1, const float4* __restrict__ n2, size_t nv0,
                                       int nk) {
    const float2 ginv2 = make_float2(-J.sg * J.inv_l, -J.sg * J.inv_l);
    const float bk = L.beta[k], bkm1 = k > 0 ? L.beta[k - 1] : 0.f;
    const float2 b2 = make_float2(bk, bk), bm2 = make_float2(bkm1, bkm1);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t g[2][8];
        tmem_ld8(gaddr + 16 * h, g[0]);
        tmem_ld8(gaddr + 16 * h + 8, g[1]);
        if (h == 1) load_s_z(s1, s2, v0 + 4 * kTile, k, pa, pc);
        tmem_wait_ld();
        uint32_t zh[8], zl[8];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const float2 a2[2] = {make_float2(pa[v].x, pa[v].y), make_float2(pa[v].z, pa[v].w)};
            const float2 c2[2] = {make_float2(pc[v].x, pc[v].y), make_float2(pc[v].z, pc[v].w)};
            float2 sk[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float2 z = fma2(bm2, sub2(a2[e], c2[e]), a2[e]);
                const float2 gv = make_float2(__uint_as_float(g[v >> 1][4 * (v & 1) + 2 * e]),
                                              __uint_as_float(g[v >> 1][4 * (v & 1) + 2 * e + 1]));
                const float2 x = fma2(gv, ginv2, z);
                const float2 cl = make_float2(fminf(fmaxf(x.x, -tau), tau), fminf(fmaxf(x.y, -tau), tau));
                sk[e] = sub2(x, cl);
                const float2 zn = fma2(b2, sub2(sk[e], a2[e]), sk[e]);
                zh[2 * v + e] = pack2z<BF>(zn);
                zl[2 * v + e] = pack2z<BF>(sub2(zn, unpack2z<BF>(zh[2 * v + e])));
            }
            s2[v0 + (size_t)(4 * h + v) * kTile] = make_float4(sk[0].x, sk[0].y, sk[1].x, sk[1].y);
        }
        if (h == 1 && nk >= 0) load_s_z(n1, n2, nv0, nk, pa, pc);
        if (want_z) {
            // GEMM1 of the previous chunk has read this half's Z columns
            wait_z(ms, &ms->z_empty[h], (zw & 1) ^ 1, L.err);
            fence_after_sync();
            tmem_st8(zoff + zcol_hi(h), zh);
            tmem_st8(zoff + zcol_lo(h), zl);
            tmem_wait_st();
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&ms->z_full[h]);
        }
    }
    if (want_z) ++zw;
}

// Warps 2 .. 17.
template <bool BF>
__device__ __forceinline__ void epi_role_z(const TczLaunch& L, MiscZ* ms, uint8_t* sm, uint32_t tbase, int warp,
                                           int lane) {
    const int ew = warp - 2, q = warp & 3, cg = ew >> 2;
    const int r = 32 * q + lane;                      // TMEM lane = tile row
    const int et = threadIdx.x - 64;                  // 0 .. kEpiThreads - 1
    const uint32_t lane_addr = tbase + ((uint32_t)(32 * q) << 16);
    uint8_t* scr = L.scratch + (size_t)blockIdx.x * kScrBytesZ;
    float4* buf0 = reinterpret_cast<float4*>(scr);
    float4* buf1 = reinterpret_cast<float4*>(scr + kScrS);
    float4* y4 = reinterpret_cast<float4*>(scr + kScrY);
    uint8_t* p_hi = sm + kOffP;
    uint8_t* p_lo = p_hi + kPBytes;
    uint32_t acc = 0, zw = 0, uc = 0;
    bool first_tile = true;
    for (;;) {
        const int tile = fetch_tile_z(L, ms);
        if (tile < 0) break;
        const TczJob& J = L.jobs[ms->job];
        const GopShape& gs = J.gs;
        const int n = J.n, m16 = J.m16, K = J.iters, bsz = gs.b, nch = n / kCc;
        if (cg == 0) ms->colmax[r] = 0u;
        cta_sync_z();   // B
        const long long tile_row0 = J.row0 + (long long)(tile - J.tile_begin) * kTile;
        if (K > 0) {
            {   // the tile's y, read once (coalesced), as [m16 / 4][128] float4, zero beyond M
                // and beyond the job's last block
                const int m = gs.m;
                const long long rows_left = J.rows - tile_row0;
                float* yf = reinterpret_cast<float*>(y4);
                const float* src = J.y + tile_row0 * m;
                for (int e = et; e < kTile * m16; e += kEpiThreads) {
                    const int rr = e / m16, i = e % m16;
                    const float v = (i < m && rr < rows_left) ? src[(size_t)rr * m + i] : 0.f;
                    yf[((size_t)(i / 4) * kTile + rr) * 4 + (i & 3)] = v;
                }
                __threadfence_block();
                named_sync(kBarEpi, kEpiThreads);
            }
            // P_0 = -y (z^0 = 0, so U = 0): the operand of the lambda pass and of k = 0
            residual_z<BF>(J, p_hi, p_lo, lane_addr, cg, r, y4, false, 0 >= J.split_from);
            fence_proxy_async_smem();
            fence_before_sync();
            __syncwarp();
            // (the test hook withholds one warp's arrival in CTA 0: the MMA warp's
            // bounded wait then gives up and the CTA drains)
            if (lane == 0 && !(L.drop_arrival && blockIdx.x == 0 && ew == 1 && first_tile))
                mbar_arrive(&ms->p_ready);
            // lambda_b = lambda_rel ||A^T y_b||_inf from G = -A^T y
            float mx = 0.f;
            for (int c = 0; c < nch; ++c, ++acc) {
                wait_z(ms, &ms->acc_full[acc & 1], (acc >> 1) & 1, L.err);
                fence_after_sync();
                mx = gmax_z(lane_addr + kColG + (acc & 1) * kCc + (uint32_t)(kPerThread * cg), mx);
                fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(&ms->acc_empty[acc & 1]);
            }
            atomicMax(&ms->colmax[r], __float_as_uint(mx * J.sg));
            named_sync(kBarEpi, kEpiThreads);
            const float tau = J.lambda_rel * __uint_as_float(ms->colmax[r]) * J.inv_l;
            // the thread's first s index of chunk c; s^k goes over s^{k-2}: even k into
            // buf0, odd k into buf1
            auto vidx = [&](int c) { return (size_t)(c * (kCc / 4) + cg * (kPerThread / 4)) * kTile + r; };
            float4 pa[4], pc[4];   // the next chunk's first 16 s^{k-1} and s^{k-2}: none at k = 0
#pragma unroll
            for (int v = 0; v < 4; ++v) pa[v] = pc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int k = 0; k < K; ++k) {
                const bool want_z = k + 1 < K;
                const float4* s1 = (k & 1) ? buf0 : buf1;
                float4* s2 = (k & 1) ? buf1 : buf0;
                for (int c = 0; c < nch; ++c, ++acc) {
                    wait_z(ms, &ms->acc_full[acc & 1], (acc >> 1) & 1, L.err);
                    fence_after_sync();
                    // the next chunk: c + 1 of this iteration, else chunk 0 of the next one
                    const int kn = c + 1 < nch ? k : k + 1, cn = c + 1 < nch ? c + 1 : 0;
                    step_z<BF>(J, L, ms, s1, s2, vidx(c),
                               lane_addr + kColG + (acc & 1) * kCc + (uint32_t)(kPerThread * cg),
                               lane_addr + (uint32_t)(8 * cg), k, tau, want_z, zw, lane, pa, pc,
                               (kn & 1) ? buf0 : buf1, (kn & 1) ? buf1 : buf0, vidx(cn), kn < K ? kn : -1);
                    fence_before_sync();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&ms->acc_empty[acc & 1]);
                }
                if (want_z) {
                    // U of z^{k+1} is complete: P for iteration k + 1
                    wait_z(ms, &ms->u_full, uc & 1, L.err);
                    ++uc;
                    fence_after_sync();
                    residual_z<BF>(J, p_hi, p_lo, lane_addr, cg, r, y4, true, k + 1 >= J.split_from);
                    fence_proxy_async_smem();
                    fence_before_sync();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&ms->p_ready);
                }
            }
        }
        // --- reconstruct: R = C^T S C per block, S = s^{K-1}, one block at a time
        // (four for 16 x 16), through the idle P area of shared memory ---
        float* s_s = reinterpret_cast<float*>(sm + kOffP);
        float* t_s = s_s + 1024;
        float* c_s = t_s + 1024;                      // the DCT matrix, <= 32 x 32
        for (int i = et; i < bsz * bsz; i += kEpiThreads) c_s[i] = J.dct[i];
        __threadfence_block();
        named_sync(kBarEpi, kEpiThreads);
        const float4* sK = (K > 0 && ((K - 1) & 1)) ? buf1 : buf0;
        const int gb = 1024 / n;
        const size_t frame_px = (size_t)gs.h * gs.w;
        for (int b0 = 0; b0 < kTile; b0 += gb) {
            for (int e = et; e < gb * n; e += kEpiThreads) {
                const int bl = e / n, j = e % n;
                s_s[e] = K > 0 ? reinterpret_cast<const float*>(sK + (size_t)(j / 4) * kTile + b0 + bl)[j & 3] : 0.f;
            }
            named_sync(kBarEpi, kEpiThreads);
            for (int e = et; e < gb * n; e += kEpiThreads) {
                const int bl = e / n, idx = e % n, kk = idx / bsz, qq = idx % bsz;
                const float* srow = s_s + bl * n + kk * bsz;
                float a = 0.f;
                for (int l = 0; l < bsz; ++l) a = fmaf(srow[l], c_s[l * bsz + qq], a);
                t_s[e] = a;
            }
            named_sync(kBarEpi, kEpiThreads);
            for (int e = et; e < gb * n; e += kEpiThreads) {
                const int bl = e / n, idx = e % n, p = idx / bsz, qq = idx % bsz;
                const long long grow = tile_row0 + b0 + bl;
                if (grow >= J.rows) continue;
                const int c_idx = (int)(grow / gs.nblk), blk = (int)(grow % gs.nblk);
                const int g_key = c_idx / (gs.g - 1);
                const int py = (blk / gs.nbc) * bsz + p, px = (blk % gs.nbc) * bsz + qq;
                if (py >= gs.h || px >= gs.w) continue;
                float a = 0.f;
                for (int kk = 0; kk < bsz; ++kk) a = fmaf(c_s[kk * bsz + p], t_s[bl * n + kk * bsz + qq], a);
                const size_t off = (size_t)py * gs.w + px;
                const float v = (float)J.keys[(size_t)g_key * frame_px + off] + a;
                if (J.out_f32) J.out_f32[(size_t)c_idx * frame_px + off] = v;
                if (J.out_u8) J.out_u8[(size_t)c_idx * frame_px + off] = (uint8_t)fminf(fmaxf(rintf(v), 0.f), 255.f);
            }
            named_sync(kBarEpi, kEpiThreads);
        }
        cta_sync_z();   // C
        first_tile = false;
    }
}

template <bool BF>
__global__ void __maxnreg__(96) k_fista_tcz(const __grid_constant__ TczLaunch L) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
    MiscZ* ms = reinterpret_cast<MiscZ*>(sm + kOffMisc);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        if (lane == 0) {
            for (int s = 0; s < kStages; ++s) {
                mbar_init(&ms->full[s], 1);
                mbar_init(&ms->empty[s], 1);
            }
            for (int a = 0; a < 2; ++a) {
                mbar_init(&ms->acc_full[a], 1);
                mbar_init(&ms->acc_empty[a], kEpiWarps);
            }
            for (int h = 0; h < 2; ++h) {
                mbar_init(&ms->z_full[h], kEpiWarps);
                mbar_init(&ms->z_empty[h], 1);
            }
            mbar_init(&ms->u_full, 1);
            mbar_init(&ms->p_ready, kEpiWarps);
            mbar_init(&ms->drain, 1);
            ms->abort = 0;
            fence_mbar_init();
        }
        __syncwarp();
        tmem_alloc(&ms->tmem_base, 512);
        tmem_relinquish();
    }
    cta_sync_z();
    const uint32_t tbase = ms->tmem_base;
    if (warp == 0)
        mma_role_z<BF>(L, ms, sm, tbase, lane);
    else if (warp == 1)
        copy_role_z(L, ms, sm, lane);
    else
        epi_role_z<BF>(L, ms, sm, tbase, warp, lane);
    cta_sync_z();
    if (warp == 0) tmem_dealloc(tbase, 512);
}

int m16_of_z(int m) { return (m + 15) / 16 * 16; }

}  // namespace

bool tcz_plan_supported(int n, int m) {
    return (n == 256 || n == 1024) && m >= 1 && m16_of_z(m) <= kMaxM16z;
}

bool tcz_supported(const cs_plan* plan) {
    const cs_ctx* ctx = plan->ctx;
    return plan->a_tcs != nullptr && ctx->tcs_scratch != nullptr && tcz_plan_supported(plan->n, plan->m) &&
           (size_t)ctx->sm_count * kScrBytesZ <= tcs_slot_bytes(ctx->sm_count);
}

namespace {

void fill_job_z(const DecodeArgs& d, int tile_begin, TczJob* J) {
    const cs_plan* p = d.plan;
    const bool bf = d.precision == CS_BF16 || d.precision == CS_BF16X2;
    const int m16 = m16_of_z(p->m), m32 = (p->m + 31) / 32 * 32;
    const size_t img1 = (size_t)m16 * p->n * 2, img2 = (size_t)m32 * p->n * 2;
    // the streaming decode's images: GEMM1 fp16 hi, lo, bf16 hi, lo; then GEMM2's
    J->a1_img = p->a_tcs + (bf ? 2 * img1 : 0);
    J->a2_img = p->a_tcs + 4 * img1 + (bf ? 2 * img2 : 0);
    J->y = d.y;
    J->keys = d.key;
    J->out_f32 = d.out_f32;
    J->out_u8 = d.out_u8;
    J->dct = p->dct;
    J->gs = d.gs;
    const long long total = (long long)d.gs.n_cs * d.gs.nblk;
    J->row0 = d.row_begin;
    J->rows = d.row_end < 0 ? total : d.row_end;
    J->tile_begin = tile_begin;
    J->n = p->n;
    J->m16 = m16;
    J->iters = d.iters;
    const bool mixed = d.precision == CS_BF16 || d.precision == CS_FP16;
    J->split_from = mixed ? (d.iters > d.tail_iters ? d.iters - d.tail_iters : 0) : 0;
    J->lambda_rel = d.lambda_rel;
    J->inv_l = (float)(1.0 / p->lipschitz);
    J->su = ldexpf(1.f, -p->tc_ea);
    J->sg = ldexpf(1.f, -(p->tc_ea + p->tc_ep));
    J->sp = ldexpf(1.f, p->tc_ep);
}

long long job_rows_z(const DecodeArgs& d) {
    const long long total = (long long)d.gs.n_cs * d.gs.nblk;
    return (d.row_end < 0 ? total : d.row_end) - d.row_begin;
}

// One launch for up to kMaxJobsZ jobs of one operand type, heaviest first: one
// CTA per SM, the per-CTA state in a slot of the streaming decode's scratch.
cudaError_t launch_group_z(const DecodeArgs* const* jobs, int n_jobs, bool bf, cudaStream_t s) {
    cs_ctx* ctx = jobs[0]->plan->ctx;
    if (!ctx->tcs_scratch) return cudaErrorInvalidValue;
    TczLaunch L{};
    L.beta = jobs[0]->beta;
    L.err = ctx->err_dev;
    int tiles = 0;
    for (int i = 0; i < n_jobs; ++i) {
        fill_job_z(*jobs[i], tiles, &L.jobs[i]);
        tiles += (int)((L.jobs[i].rows - L.jobs[i].row0 + kTile - 1) / kTile);
    }
    L.n_jobs = n_jobs;
    L.n_tiles = tiles;
    const void* fn = bf ? (const void*)k_fista_tcz<true> : (const void*)k_fista_tcz<false>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(ctx->launch_mu);
    int cslot = 0, sslot = 0;
    e = slot_take(&ctx->counter_ring, s, &cslot);
    if (e == cudaSuccess) e = slot_take(&ctx->tcs_ring, s, &sslot);
    if (e != cudaSuccess) return e;
    L.tile_counter = ctx->counters_dev + cslot;
    L.drop_arrival = ctx->debug_flags.exchange(0) & CS_DEBUG_DROP_ARRIVAL;
    L.scratch = ctx->tcs_scratch + (size_t)sslot * tcs_slot_bytes(ctx->sm_count);
    e = cudaMemsetAsync(L.tile_counter, 0, sizeof(int), s);
    const int grid = std::min(tiles, ctx->sm_count);
    if (e == cudaSuccess) {
        if (bf)
            k_fista_tcz<true><<<grid, kThreads, kSmemBytes, s>>>(L);
        else
            k_fista_tcz<false><<<grid, kThreads, kSmemBytes, s>>>(L);
        e = cudaGetLastError();
    }
    const cudaError_t e1 = slot_done(&ctx->counter_ring, cslot, s);
    const cudaError_t e2 = slot_done(&ctx->tcs_ring, sslot, s);
    return e != cudaSuccess ? e : e1 != cudaSuccess ? e1 : e2;
}

}  // namespace

// A 32 x 32 job with more tiles than SMs leaves a last round of (tiles mod SMs)
// tiles on as many SMs, which takes as long as a full round.  When that remainder is
// at most four rounds of the cluster kernel's co-resident clusters (a tile-iteration
// there takes about a fifth of one here, on eight SMs), the cluster kernel decodes
// the job's first `remainder` tiles and this kernel the rest in whole rounds, one
// after the other on the call's stream.  The split depends on the job and the
// device alone, so a job decodes to the same bits in any batch.
static long long cluster_head_rows(const DecodeArgs& d) {
    if (d.plan->n != 1024 || d.row_begin != 0 || !tc_supported(d.plan, d.precision)) return 0;
    const long long tiles = (job_rows_z(d) + kTile - 1) / kTile;
    const int sm = d.plan->ctx->sm_count;
    const long long rem = tiles % sm;
    if (tiles <= sm || rem == 0) return 0;
    const int clusters = tc8_clusters(d.precision == CS_BF16 || d.precision == CS_BF16X2);
    return rem <= 4ll * clusters ? rem * kTile : 0;
}

cudaError_t launch_decode_tcz_batch(const DecodeArgs* jobs, int n_jobs, cudaStream_t s) {
    std::vector<DecodeArgs> own, heads;
    own.reserve(n_jobs);
    for (int i = 0; i < n_jobs; ++i) {
        if (job_rows_z(jobs[i]) <= 0) continue;
        const long long h = cluster_head_rows(jobs[i]);
        DecodeArgs d = jobs[i];
        if (h > 0) {
            DecodeArgs dh = d;
            dh.row_end = h;
            heads.push_back(dh);
            d.row_begin = h;
        }
        own.push_back(d);
    }
    if (!heads.empty()) {
        const cudaError_t e = launch_decode_tc8_batch(heads.data(), (int)heads.size(), s);
        if (e != cudaSuccess) return e;
    }
    std::vector<const DecodeArgs*> groups[2];
    for (const DecodeArgs& d : own) {
        const bool bf = d.precision == CS_BF16 || d.precision == CS_BF16X2;
        groups[bf ? 1 : 0].push_back(&d);
    }
    for (int bf = 0; bf < 2; ++bf) {
        std::vector<const DecodeArgs*>& g = groups[bf];
        std::stable_sort(g.begin(), g.end(), [](const DecodeArgs* a, const DecodeArgs* b) {
            return (double)job_rows_z(*a) * a->iters * a->plan->n > (double)job_rows_z(*b) * b->iters * b->plan->n;
        });
        for (size_t i = 0; i < g.size(); i += kMaxJobsZ) {
            const int nj = (int)std::min(g.size() - i, (size_t)kMaxJobsZ);
            const cudaError_t e = launch_group_z(g.data() + i, nj, bf == 1, s);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

cudaError_t launch_decode_tcz(const DecodeArgs& d, cudaStream_t s) { return launch_decode_tcz_batch(&d, 1, s); }

}  // namespace csvc
