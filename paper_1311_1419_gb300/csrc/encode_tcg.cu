// K4 on the tensor cores: block-CS measurement of every CS frame (Sec. 3.1),
// y_b = Phi r_b, for 8 x 8, 16 x 16 and 32 x 32 blocks (N = 64, 256, 1024),
// for one plan or for several plans of the same N over the same clip in one
// launch, which then reads the clip once.
//
// One GEMM across the blocks of the call per plan, Y_p [rows x M_p] = R [rows x
// N] Phi_p^T, with R shared by the plans: residuals are integers in [-255, 255],
// exact in fp16, and Phi * 2^e is split into fp16 hi + lo, which gives
// FP32-grade products.  Where the accumulators fit, a plan's hi and lo images
// form one B operand of 2 M16 rows (Y_hi and Y_lo side by side in tensor
// memory, added at the end), so a K step is one MMA of N = 2 M16; otherwise
// each is its own MMA.  A tile is 128 blocks (one per TMEM lane); K runs in
// chunks of 64 pixels (two rows of a 32 x 32 block, four of a 16 x 16, a whole
// 8 x 8 block).  Per CTA (one per SM) the work is a pipeline over its chunks,
// with mbarrier hand-offs and no CTA-wide barrier per chunk:
//   - warps 1 .. 16 (the converters): warp w owns TMEM lane quarter w % 4 (32
//     blocks of the tile) and pixels 16 ((w - 1) / 4) .. + 15 of every chunk;
//     each thread loads its block's current and key bytes four chunks ahead into
//     registers, forms current - key as fp16 (exact) and stores it into a TMEM
//     stage, the MMA's A operand;
//   - warp 17 (one thread): bulk-copies every plan's Phi chunk (hi and lo,
//     contiguous in the images' K-chunk-major layout, resident in L2) into an
//     S-stage ring, as soon as the stage's last MMAs are done;
//   - warp 0 (one thread): issues each plan's MMAs into the plan's accumulator
//     columns;
//   - the converters, after a tile's last chunk: y = D 2^-e through shared
//     memory in slices of 64 columns, so that rows of y are stored
//     contiguously.
// Every mbarrier wait is bounded and reports through the context's error word.
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>

#include "internal.h"
#include "tc_ptx.h"

namespace csvc {

constexpr int kMaxEncPlans = 4;
struct EncPlan {
    const uint8_t* img;   // Phi * 2^e: fp16 hi image then fp16 lo image, m16 x n each
    float* y;             // [rows][m]
    int m, m16;           // measurements, rounded up to 16
    int col;              // first accumulator column (hi; lo at col + m16 in paired mode)
    int phi_off;          // byte offset of the plan's hi chunk in a Phi stage (lo follows it)
    float scale;          // 2^-e
};
struct EncLaunch {
    const uint8_t* frames;
    GopShape gs;          // the clip (its m is not used)
    int* err;
    int n_plans;
    int m16_total;        // rows of all plans' images
    int paired;           // hi and lo as one B operand of 2 m16 rows
    int r_col;            // first TMEM column of the residual stages (32 columns each)
    int ncols;            // TMEM columns allocated
    int vec;              // 1: 8-byte frame loads, 2: 16-byte, 0: byte loads
    EncPlan p[kMaxEncPlans];
};

namespace {

using namespace tc;

constexpr int kTile = 128;
constexpr int kChunk = 64;                          // K per chunk: one 128-byte swizzle atom column
constexpr int kConvWarps = 16;                      // warps 1 .. 16: four per TMEM lane quarter
constexpr int kThreadsE = (2 + kConvWarps) * 32;    // + warp 0 (MMAs) and warp 17 (Phi copies)
constexpr int kPhiWarp = kConvWarps + 1;
constexpr int kDepth = 4;                           // chunks of frame bytes in flight per thread
constexpr int kMaxM16 = 256;                        // per plan (one MMA's N)
constexpr int kMaxM16Total = 320;                   // per launch
constexpr uint32_t kYStage = kTile * 64 * 4;        // y staging: 128 rows x 64 columns
constexpr uint32_t kBarConv = 1;                    // named barrier of the converter warps
constexpr uint64_t kWaitNs = 1000000000ull;

__host__ __device__ constexpr uint32_t phi_stage_bytes(int m16_total) {
    return 2u * (uint32_t)m16_total * kChunk * 2u;
}
__host__ __device__ constexpr uint32_t off_y(int s, int m16_total) { return (uint32_t)s * phi_stage_bytes(m16_total); }
__host__ __device__ constexpr uint32_t off_bar(int s, int m16_total) { return off_y(s, m16_total) + kYStage; }
// (at least 116 KB: one CTA per SM, so that no CTA waits for another's tensor memory)
__host__ __device__ constexpr uint32_t smem_bytes(int s, int m16_total) {
    return off_bar(s, m16_total) + 256u + 1024u > 116u * 1024u ? off_bar(s, m16_total) + 256u + 1024u : 116u * 1024u;
}
constexpr uint32_t kSmemMax = 232448;
static_assert(smem_bytes(2, kMaxM16Total) <= kSmemMax, "the widest launch fits");

__device__ __forceinline__ bool wait_e(uint64_t* bar, uint32_t parity, int* abort, int* err) {
    if (*(volatile int*)abort) return false;
    if (mbar_wait(bar, parity, kWaitNs)) return true;
    *(volatile int*)abort = 1;
    atomicExch(err, 1);
    return false;
}

// A converter thread's block of a tile: byte offsets of its first chunk's two
// 8-pixel segments in the current frame (the key at key_off from them), the
// frame rows of the two segments (-1: no block), and the frame column.
struct Src {
    long long off0, off1, key_d;
    int fy0, fy1, fx;
};

// Thread (lane quarter q = block 32 q + lane of the tile, pixel group cg = 16
// pixels of a chunk).  The 16 pixels: a half row of a 32 x 32 block, a row of a
// 16 x 16 block, two rows of an 8 x 8 block.
__device__ __forceinline__ void src_of(const EncLaunch& L, int tile, int rows, int b, int cg, Src& sr) {
    const GopShape& gs = L.gs;
    const int bsz = gs.b;
    const int row = tile * kTile + b;
    sr.fy0 = sr.fy1 = -1;
    sr.fx = 0;
    sr.off0 = sr.off1 = sr.key_d = 0;
    if (row >= rows) return;
    const int ci = row / gs.nblk, blk = row - ci * gs.nblk;
    const int gg = ci / (gs.g - 1), j = ci - gg * (gs.g - 1) + 1;
    const int bi = blk / gs.nbc, bj = blk - bi * gs.nbc;
    int r0, c0, r1, c1;
    if (bsz == 32) { r0 = r1 = cg >> 1; c0 = 16 * (cg & 1); c1 = c0 + 8; }
    else if (bsz == 16) { r0 = r1 = cg; c0 = 0; c1 = 8; }
    else { r0 = 2 * cg; r1 = r0 + 1; c0 = c1 = 0; }
    const long long frame_px = (long long)gs.h * gs.w;
    const long long cur = (long long)(gg * gs.g + j) * frame_px;
    sr.fy0 = bi * bsz + r0;
    sr.fy1 = bi * bsz + r1;
    sr.fx = bj * bsz + c0;
    sr.off0 = cur + (long long)sr.fy0 * gs.w + bj * bsz + c0;
    sr.off1 = cur + (long long)sr.fy1 * gs.w + bj * bsz + c1;
    sr.key_d = -(long long)j * frame_px;
}

// The thread's 16 current and 16 key bytes of chunk c (zero outside the frame).
__device__ __forceinline__ void load_bytes(const EncLaunch& L, const Src& sr, int c, uint4& cv, uint4& kv) {
    const GopShape& gs = L.gs;
    const int dy = c * (kChunk / gs.b);
    const long long step = (long long)dy * gs.w;
    const bool v0 = sr.fy0 >= 0 && sr.fy0 + dy < gs.h, v1 = sr.fy1 >= 0 && sr.fy1 + dy < gs.h;
    cv = kv = make_uint4(0u, 0u, 0u, 0u);
    const uint8_t* p0 = L.frames + sr.off0 + step;
    const uint8_t* p1 = L.frames + sr.off1 + step;
    if (L.vec == 2) {          // both segments in one 16-byte row piece
        if (v0) {
            cv = __ldg(reinterpret_cast<const uint4*>(p0));
            kv = __ldg(reinterpret_cast<const uint4*>(p0 + sr.key_d));
        }
    } else if (L.vec == 1) {
        if (v0) {
            const uint2 a = __ldg(reinterpret_cast<const uint2*>(p0));
            const uint2 k = __ldg(reinterpret_cast<const uint2*>(p0 + sr.key_d));
            cv.x = a.x; cv.y = a.y; kv.x = k.x; kv.y = k.y;
        }
        if (v1) {
            const uint2 a = __ldg(reinterpret_cast<const uint2*>(p1));
            const uint2 k = __ldg(reinterpret_cast<const uint2*>(p1 + sr.key_d));
            cv.z = a.x; cv.w = a.y; kv.z = k.x; kv.w = k.y;
        }
    } else {
        // cropped right edge or unaligned rows: byte loads, zero beyond the frame
        uint32_t cw[4] = {0u, 0u, 0u, 0u}, kw[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int x = 0; x < 16; ++x) {
            const bool seg1 = x >= 8;
            const int xx = x & 7;
            const bool in = (seg1 ? v1 : v0) && sr.fx + (seg1 && gs.b >= 16 ? 8 : 0) + xx < gs.w;
            const uint8_t* p = (seg1 ? p1 : p0) + xx;
            if (in) {
                cw[x >> 2] |= (uint32_t)p[0] << (8 * (x & 3));
                kw[x >> 2] |= (uint32_t)p[sr.key_d] << (8 * (x & 3));
            }
        }
        cv = make_uint4(cw[0], cw[1], cw[2], cw[3]);
        kv = make_uint4(kw[0], kw[1], kw[2], kw[3]);
    }
}

// current - key for 16 pixels as 8 fp16 pairs.  A byte b placed under the
// exponent byte 0x64 is the fp16 value 1024 + b, exactly; the difference of two
// such values is cur - key, exactly (|cur - key| <= 255 < 2^11).
__device__ __forceinline__ void residual16(const uint4& cv, const uint4& kv, uint32_t (&r)[8]) {
    const uint32_t cw[4] = {cv.x, cv.y, cv.z, cv.w}, kw[4] = {kv.x, kv.y, kv.z, kv.w};
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const uint32_t sel = (e & 1) ? 0x4342u : 0x4140u;
        const uint32_t ch = __byte_perm(cw[e >> 1], 0x64646464u, sel);
        const uint32_t kh = __byte_perm(kw[e >> 1], 0x64646464u, sel);
        const __half2 d = __hsub2(*reinterpret_cast<const __half2*>(&ch), *reinterpret_cast<const __half2*>(&kh));
        r[e] = *reinterpret_cast<const uint32_t*>(&d);
    }
}

// Every plan's hi and lo chunk c into a Phi stage (plan q's hi chunk at
// phi_off_q, its lo chunk m16_q x 128 bytes after it).
__device__ __forceinline__ void load_phi(const EncLaunch& L, uint8_t* stage, uint64_t* full, int c) {
    mbar_arrive_expect_tx(full, phi_stage_bytes(L.m16_total));
    for (int q = 0; q < L.n_plans; ++q) {
        const EncPlan& P = L.p[q];
        const uint32_t cb = (uint32_t)P.m16 * kChunk * 2;                  // one chunk of one image
        const size_t img = (size_t)P.m16 * L.gs.n * 2;
        uint8_t* dst = stage + P.phi_off;
        bulk_g2s(dst, P.img + (size_t)c * cb, cb, full);
        bulk_g2s(dst + cb, P.img + img + (size_t)c * cb, cb, full);
    }
}

// After a tile's last chunk: y = D 2^-e (paired: D_hi + D_lo) through shared
// memory, 64 columns at a time; row r's column x sits at [r][x ^ (r % 32)], so
// that the TMEM-side writes (one row per lane) and the row-contiguous reads both
// avoid bank conflicts.  Converter warp (q, h) reads lanes 32 q .. and 16
// columns of each slice.
__device__ __forceinline__ void write_y(const EncLaunch& L, float* ys, uint32_t tmem, int tile, int rows, int q,
                                        int h, int warp, int lane, bool ok) {
    const int r = 32 * q + lane;
    const int live = min(kTile, rows - tile * kTile);
    const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
    for (int pi = 0; pi < L.n_plans; ++pi) {
        const EncPlan& P = L.p[pi];
        for (int s0 = 0; s0 < P.m16; s0 += 64) {
#pragma unroll
            for (int cc = 0; cc < 16; cc += 8) {
                const int col = s0 + 16 * h + cc;
                if (col < P.m16) {
                    uint32_t d[8], dl[8];
                    tmem_ld8(lane_base + (uint32_t)(P.col + col), d);
                    if (L.paired) tmem_ld8(lane_base + (uint32_t)(P.col + P.m16 + col), dl);
                    tmem_wait_ld();
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float v = __uint_as_float(d[i]) + (L.paired ? __uint_as_float(dl[i]) : 0.f);
                        ys[r * 64 + ((16 * h + cc + i) ^ (r & 31))] = v * P.scale;
                    }
                }
            }
            named_sync(kBarConv, kConvWarps * 32);
            // a warp stores whole row segments: rows w - 1, w + 15, ..., lanes along
            // the slice's columns
            const int width = min(64, P.m - s0);
            float* yt = P.y + (size_t)tile * kTile * P.m + s0;
            if (ok)
                for (int rr = warp - 1; rr < live; rr += kConvWarps)
                    for (int cl = lane; cl < width; cl += 32) yt[rr * P.m + cl] = ys[rr * 64 + (cl ^ (rr & 31))];
            named_sync(kBarConv, kConvWarps * 32);
        }
    }
}

template <int S>
__global__ void __maxnreg__(96) k_encode_tcg(const __grid_constant__ EncLaunch L) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
    const int mt = L.m16_total;
    const uint32_t kPhiStage = phi_stage_bytes(mt);
    float* ys = reinterpret_cast<float*>(sm + off_y(S, mt));
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + off_bar(S, mt));
    uint64_t* phi_full = bar;              // [S]: the stage's Phi chunks have landed
    uint64_t* r_full = bar + S;            // [S]: the converters have stored the stage's residual chunk
    uint64_t* mma_done = bar + 2 * S;      // [S]: the stage's MMAs are done (Phi and residual stage free)
    uint64_t* acc_full = bar + 3 * S;      // the tile's accumulators are complete
    uint64_t* acc_empty = bar + 3 * S + 1; // the converters have read them out
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 3 * S + 2);
    int* abort = reinterpret_cast<int*>(bar + 3 * S + 3);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nch = L.gs.n / kChunk;                        // 1, 4 or 16
    const int lg_nch = nch == 1 ? 0 : nch == 4 ? 2 : 4;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&phi_full[s], 1);
            mbar_init(&r_full[s], kConvWarps);
            mbar_init(&mma_done[s], 1);
        }
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, kConvWarps);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        __syncwarp();
        tmem_alloc(tmem_slot, (uint32_t)L.ncols);
        tmem_relinquish();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const int rows = L.gs.n_cs * L.gs.nblk;                 // < 2^31 (checked by the host)
    const int tiles = (rows + kTile - 1) / kTile;
    const int my_tiles = tiles > (int)blockIdx.x ? (tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int total = my_tiles * nch;                       // this CTA's chunks, tile-major
    auto tile_of = [&](int g) { return (int)blockIdx.x + (g >> lg_nch) * (int)gridDim.x; };
    if (warp == 0) {
        if (lane == 0) {
            // ---- every MMA ----
            const uint32_t s_base = smem_u32(sm);
            bool ok = true;
            int mma_last[S];
#pragma unroll
            for (int s = 0; s < S; ++s) mma_last[s] = -1;
            for (int g = 0; g < total; ++g) {
                const int s = g % S, c = g & (nch - 1);
                const uint32_t u = (uint32_t)(g / S);
                // a tile's first chunk overwrites the accumulators: the previous tile's y is out
                if (c == 0 && g > 0) ok = wait_e(acc_empty, (uint32_t)(((g >> lg_nch) - 1) & 1), abort, L.err) && ok;
                ok = wait_e(&phi_full[s], u & 1, abort, L.err) && ok;
                ok = wait_e(&r_full[s], u & 1, abort, L.err) && ok;
                fence_after_sync();
                if (ok) {
                    const uint32_t a0 = tmem + (uint32_t)(L.r_col + 32 * s);
                    for (int q = 0; q < L.n_plans; ++q) {
                        const EncPlan& P = L.p[q];
                        const uint32_t po = (uint32_t)s * kPhiStage + (uint32_t)P.phi_off;
                        const uint64_t dh = desc_sw128(s_base + po, 16, 1024);
                        const uint32_t d = tmem + (uint32_t)P.col;
                        if (L.paired) {
                            // hi and lo rows as one B operand: D_hi, D_lo side by side
                            const uint32_t id = idesc_f16(128, 2u * (uint32_t)P.m16, 0u, 0u, 0u);
#pragma unroll
                            for (uint32_t ks = 0; ks < kChunk / 16; ++ks)
                                mma_f16_tmem_a(d, a0 + 8 * ks, dh + 2 * ks, id, (c > 0 || ks > 0) ? 1u : 0u);
                        } else {
                            const uint64_t dl = desc_sw128(s_base + po + (uint32_t)P.m16 * kChunk * 2u, 16, 1024);
                            const uint32_t id = idesc_f16(128, (uint32_t)P.m16, 0u, 0u, 0u);
#pragma unroll
                            for (uint32_t ks = 0; ks < kChunk / 16; ++ks) {
                                mma_f16_tmem_a(d, a0 + 8 * ks, dh + 2 * ks, id, (c > 0 || ks > 0) ? 1u : 0u);
                                mma_f16_tmem_a(d, a0 + 8 * ks, dl + 2 * ks, id, 1u);
                            }
                        }
                    }
                    mma_commit(&mma_done[s]);
                    mma_last[s] = g;
                    if (c == nch - 1) mma_commit(acc_full);
                }
            }
            // MMAs still in flight after a wait gave up: wait for them (bounded)
#pragma unroll
            for (int s = 0; s < S; ++s)
                if (mma_last[s] >= 0) mbar_wait(&mma_done[s], (uint32_t)((mma_last[s] / S) & 1), kWaitNs);
        }
        __syncwarp();
    } else if (warp == kPhiWarp) {
        if (lane == 0) {
            // ---- Phi chunks, S ahead: stage s once its previous MMAs are done ----
            bool ok = true;
            int phi_last[S];
#pragma unroll
            for (int s = 0; s < S; ++s) phi_last[s] = -1;
            for (int g = 0; g < total && ok; ++g) {
                const int s = g % S;
                if (g >= S) ok = wait_e(&mma_done[s], (uint32_t)((g / S - 1) & 1), abort, L.err) && ok;
                if (ok) {
                    load_phi(L, sm + (uint32_t)s * kPhiStage, &phi_full[s], g & (nch - 1));
                    phi_last[s] = g;
                }
            }
            // copies still in flight after a wait gave up: wait for them (bounded)
#pragma unroll
            for (int s = 0; s < S; ++s)
                if (phi_last[s] >= 0) mbar_wait(&phi_full[s], (uint32_t)((phi_last[s] / S) & 1), kWaitNs);
        }
        __syncwarp();
    } else {
        // ---- converters: residual chunks into tensor memory, then y ----
        // warp (q, h): blocks 32 q + lane, pixel group h (16 pixels)
        const int q = warp & 3, h = (warp - 1) >> 2;
        const int b = 32 * q + lane;                       // the thread's block of every tile
        const uint32_t r_lane = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(L.r_col + 8 * h);
        bool ok = true;
        Src pf;                                            // the prefetch's tile
        int pf_tile = -1;
        uint4 cv[kDepth], kv[kDepth];                      // chunk g in slot g % kDepth
        auto fetch = [&](int gp, uint4& c_, uint4& k_) {
            const int tp = tile_of(gp);
            if (tp != pf_tile) {
                src_of(L, tp, rows, b, h, pf);
                pf_tile = tp;
            }
            load_bytes(L, pf, gp & (nch - 1), c_, k_);
        };
#pragma unroll
        for (int j = 0; j < kDepth; ++j)
            if (j < total) fetch(j, cv[j], kv[j]);
        uint32_t ph_acc = 0;
        for (int g0 = 0; g0 < total; g0 += kDepth) {
#pragma unroll
            for (int j = 0; j < kDepth; ++j) {
                const int g = g0 + j;
                if (g < total) {
                    const int s = g % S, c = g & (nch - 1);
                    const uint32_t u = (uint32_t)(g / S);
                    uint32_t r[8];
                    residual16(cv[j], kv[j], r);
                    if (g + kDepth < total) fetch(g + kDepth, cv[j], kv[j]);
                    // the stage's previous MMAs are done before it is overwritten
                    if (g >= S) ok = wait_e(&mma_done[s], (u - 1) & 1, abort, L.err) && ok;
                    fence_after_sync();
                    tmem_st8(r_lane + (uint32_t)(32 * s), r);
                    tmem_wait_st();
                    fence_before_sync();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&r_full[s]);
                    if (c == nch - 1) {
                        ok = wait_e(acc_full, ph_acc, abort, L.err) && ok;
                        ph_acc ^= 1;
                        fence_after_sync();
                        write_y(L, ys, tmem, tile_of(g), rows, q, h, warp, lane, ok);
                        // this warp's accumulator reads are done: the next tile may overwrite them
                        fence_before_sync();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(acc_empty);
                    }
                }
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 0) tmem_dealloc(tmem, (uint32_t)L.ncols);
}

// The images of Phi * 2^e for this kernel: fp16 hi then fp16 lo, each m16 x n,
// rows >= M zero, 128-byte-swizzled atoms of 8 rows x 64 columns, atom
// (col / 64, row / 8) at ((col / 64) * m16 / 8 + row / 8) * 1024: a 64-column
// K chunk of all rows is one contiguous range.  (The on-chip kernels' images of
// 16 x 16 plans with M <= 128 have this layout too, with the bf16 images after.)
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

template <int S>
cudaError_t launch_shape(const EncLaunch& L, int grid, cudaStream_t s) {
    // the shared-memory limit is raised to the device maximum once per shape and
    // device (a driver call per launch would cost microseconds of host time)
    static std::atomic<uint64_t> raised{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = 1ull << (dev & 63);
    if (!(raised.load(std::memory_order_acquire) & bit)) {
        e = cudaFuncSetAttribute(k_encode_tcg<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax);
        if (e != cudaSuccess) return e;
        raised.fetch_or(bit, std::memory_order_acq_rel);
    }
    k_encode_tcg<S><<<grid, kThreadsE, smem_bytes(S, L.m16_total), s>>>(L);
    return cudaGetLastError();
}

int m16_of_e(int m) { return (m + 15) / 16 * 16; }

// A plan's images for this kernel: its own, or for 16 x 16 plans with M <= 128
// the on-chip kernels' (the same layout, fp16 hi and lo first).
const uint8_t* enc_images(const cs_plan* p) { return p->phi_tcg ? p->phi_tcg : p->phi_tc; }

}  // namespace

bool encode_tcg_plan_supported(int n, int m) {
    return (n == 64 || n == 256 || n == 1024) && m >= 1 && m16_of_e(m) <= kMaxM16;
}
size_t encode_tcg_image_bytes(int n, int m) { return 2ull * (size_t)m16_of_e(m) * (size_t)n * 2; }
bool encode_tcg_supported(const cs_plan* plan) {
    return enc_images(plan) != nullptr && encode_tcg_plan_supported(plan->n, plan->m);
}

cudaError_t launch_phi_images_g(const float* phi, uint8_t* img, int n, int m, int e, cudaStream_t s) {
    const int m16 = m16_of_e(m);
    const int total = m16 * n;
    k_phi_images_g<<<(total + 255) / 256, 256, 0, s>>>(phi, img, n, m, m16, ldexpf(1.f, e));
    return cudaGetLastError();
}

cudaError_t launch_encode_tcg_multi(const cs_plan* const* plans, float* const* ys, int n_plans, const GopShape& gs,
                                    const uint8_t* frames, cudaStream_t s) {
    const long long rows = (long long)gs.n_cs * gs.nblk;
    if (rows == 0 || n_plans <= 0) return cudaSuccess;
    if (rows > (1ll << 31) - kTile) return cudaErrorInvalidValue;   // block indices are 32-bit
    const long long tiles = (rows + kTile - 1) / kTile;
    const int sms = plans[0]->ctx->sm_count;
    const int grid = (int)(tiles < sms ? tiles : sms);
    // frame loads: 16 bytes when a thread's 16 pixels are one aligned row piece
    // (16 x 16 and 32 x 32 blocks), else 8 bytes, when every segment starts on
    // its boundary and no block is cropped at the right edge; else bytes
    const uintptr_t fa = reinterpret_cast<uintptr_t>(frames);
    const bool whole = gs.w % gs.b == 0;
    const int vec = whole && gs.b >= 16 && gs.w % 16 == 0 && (fa & 15) == 0 ? 2
                    : whole && gs.w % 8 == 0 && (fa & 7) == 0           ? 1
                                                                         : 0;
    // consecutive plans whose images fit one launch share it
    for (int i = 0; i < n_plans;) {
        EncLaunch L{};
        L.frames = frames;
        L.gs = gs;
        L.err = plans[i]->ctx->err_dev;
        L.vec = vec;
        int mt = 0, k = 0;
        bool pair_ok = true;
        while (i + k < n_plans && k < kMaxEncPlans) {
            const cs_plan* p = plans[i + k];
            const int m16 = m16_of_e(p->m);
            if (k > 0 && mt + m16 > kMaxM16Total) break;
            EncPlan& P = L.p[k];
            P.img = enc_images(p);
            P.y = ys[i + k];
            P.m = p->m;
            P.m16 = m16;
            P.phi_off = 2 * mt * kChunk * 2;
            P.scale = ldexpf(1.f, -p->tc_ephi);
            pair_ok = pair_ok && 2 * m16 <= kMaxM16;
            mt += m16;
            ++k;
        }
        L.n_plans = k;
        L.m16_total = mt;
        // the deepest Phi ring whose shared memory and tensor-memory columns fit,
        // hi and lo paired where their accumulators fit beside the residual stages
        int stages = 0;
        for (int st : {4, 3, 2}) {
            if (smem_bytes(st, mt) > kSmemMax) continue;
            const bool paired = pair_ok && 2 * mt + 32 * st <= 512;
            const int acc = paired ? 2 * mt : mt;
            const int r_col = (acc + 31) / 32 * 32;
            if (r_col + 32 * st > 512) continue;
            stages = st;
            L.paired = paired;
            L.r_col = r_col;
            int nc = 32;
            while (nc < r_col + 32 * st) nc *= 2;
            L.ncols = nc;
            break;
        }
        if (!stages) return cudaErrorInvalidConfiguration;
        int col = 0;
        for (int q = 0; q < k; ++q) {
            L.p[q].col = col;
            col += L.paired ? 2 * L.p[q].m16 : L.p[q].m16;
        }
        const cudaError_t e = stages == 4 ? launch_shape<4>(L, grid, s)
                              : stages == 3 ? launch_shape<3>(L, grid, s)
                                            : launch_shape<2>(L, grid, s);
        if (e != cudaSuccess) return e;
        i += k;
    }
    return cudaSuccess;
}

cudaError_t launch_encode_tcg(const cs_plan* plan, const GopShape& gs, const uint8_t* frames, float* y,
                              cudaStream_t s) {
    return launch_encode_tcg_multi(&plan, &y, 1, gs, frames, s);
}

}  // namespace csvc
