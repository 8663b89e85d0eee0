// K4 on the tensor cores: block-CS measurement of every CS frame (Sec. 3.1),
// y_b = Phi r_b, for 8 x 8, 16 x 16 and 32 x 32 blocks (N = 64, 256, 1024),
// for one plan or for several plans of the same N over the same clip in one
// launch, which then reads the clip once.
//
// One GEMM across the blocks of the call per plan, Y_p [rows x M_p] = R [rows x
// N] Phi_p^T, with R shared by the plans: residuals are integers in [-255, 255],
// exact in fp16, and Phi * 2^e is split into fp16 hi + lo, so two MMAs per K
// step give FP32-grade products.  A tile is 128 blocks (one per TMEM lane); K
// runs in chunks of 64 pixels (two rows of a 32 x 32 block, four of a 16 x 16,
// a whole 8 x 8 block).  Per CTA (one per SM) the work is a pipeline over its
// chunks, with mbarrier hand-offs and no CTA-wide barrier per chunk:
//   - warps 1 .. 16, residual bytes: every thread copies the current and key
//     bytes of its own two 8-pixel items of a chunk with asynchronous 8-byte
//     copies, D chunks ahead, into a ring in shared memory (no other thread
//     reads them, so the copies need no barrier);
//   - warps 1 .. 16, residual chunks: current - key (fp16, exact) into an
//     S-stage ring of 128-byte-swizzled operands, one arrival per warp;
//   - warp 0 (one thread): bulk-copies every plan's Phi chunk (hi and lo,
//     contiguous in the images' K-chunk-major layout, resident in L2) S - 1
//     chunks ahead into an S-stage ring, and issues each plan's MMAs into the
//     plan's own accumulator columns;
//   - warps 1 .. 16, after a tile's last chunk: y = D 2^-e through shared memory
//     (the residual ring, idle then) in slices of 64 columns, so that rows of y
//     are stored contiguously.
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
    int m, m16, col;      // measurements, rounded up to 16, first accumulator column
    float scale;          // 2^-e
};
struct EncLaunch {
    const uint8_t* frames;
    GopShape gs;          // the clip (its m is not used)
    int* err;
    int n_plans;
    int m16_total;        // accumulator columns of all plans
    int vec;              // 8-byte frame loads are aligned and never cross the right edge
    EncPlan p[kMaxEncPlans];
};

namespace {

using namespace tc;

constexpr int kT = 512;                             // converter threads (16 warps)
constexpr int kTile = 128;
constexpr int kChunk = 64;                          // K per chunk: one 128-byte swizzle atom column
constexpr int kItems = kTile * kChunk / 8;          // 8-pixel items of a chunk: 1024
constexpr int kItemsPerThread = kItems / kT;        // 2
constexpr uint32_t kRStage = kTile * kChunk * 2;    // fp16 residual operand of a chunk: 16 KB
constexpr uint32_t kRawSlot = 2u * kItems * 8u;     // current then key bytes of a chunk: 16 KB
constexpr int kMaxM16 = 256;                        // per plan (one MMA's N)
constexpr int kMaxM16Total = 320;                   // per launch
constexpr uint64_t kWaitNs = 1000000000ull;

__host__ __device__ constexpr uint32_t phi_stage_bytes(int m16_total) {
    return 2u * (uint32_t)m16_total * kChunk * 2u;
}
__host__ __device__ constexpr uint32_t off_r(int s, int m16_total) { return (uint32_t)s * phi_stage_bytes(m16_total); }
__host__ __device__ constexpr uint32_t off_raw(int s, int m16_total) {
    return off_r(s, m16_total) + (uint32_t)s * kRStage;
}
__host__ __device__ constexpr uint32_t off_bar(int s, int d, int m16_total) {
    return off_raw(s, m16_total) + (uint32_t)d * kRawSlot;
}
__host__ __device__ constexpr uint32_t smem_bytes(int s, int d, int m16_total) {
    return off_bar(s, d, m16_total) + 256u + 1024u;
}
constexpr uint32_t kSmemMax = 232448;
static_assert(smem_bytes(2, 2, kMaxM16Total) <= kSmemMax, "the widest launch fits");

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

// Where a converter thread's items of a tile come from.  Thread t's items are
// blocks b_i = t / 8 + 64 i of the tile (i = 0, 1), all at segment kseg = t % 8
// of a chunk (block row rr = kseg / segs of the chunk's rows, 8-pixel segment sg
// = kseg % segs), so per tile it keeps each block's byte offsets of its first
// chunk in the current and key frames; chunk c adds c (64 / B) rows.
struct ItemBase {
    long long cur[kItemsPerThread], key[kItemsPerThread];
    int fy[kItemsPerThread];   // frame row of the first chunk (>= H: outside; -1: no block)
    int fx[kItemsPerThread];   // frame column of the segment
};

__device__ __forceinline__ void item_bases(const EncLaunch& L, int tile, int rows, int t, ItemBase& ib) {
    const GopShape& gs = L.gs;
    const int bsz = gs.b, segs = bsz / 8;
    const int kseg = t % (kChunk / 8), rr = kseg / segs, sg = kseg % segs;
    const long long frame_px = (long long)gs.h * gs.w;
#pragma unroll
    for (int i = 0; i < kItemsPerThread; ++i) {
        const int b = t / (kChunk / 8) + (kT / (kChunk / 8)) * i;
        const int row = tile * kTile + b;
        ib.fy[i] = -1;
        ib.fx[i] = 0;
        ib.cur[i] = ib.key[i] = 0;
        if (row < rows) {
            const int r32 = row;
            const int ci = r32 / gs.nblk, blk = r32 - ci * gs.nblk;
            const int gg = ci / (gs.g - 1), j = ci - gg * (gs.g - 1) + 1;
            const int bi = blk / gs.nbc, bj = blk - bi * gs.nbc;
            const int fy = bi * bsz + rr, fx = bj * bsz + 8 * sg;
            ib.fy[i] = fy;
            ib.fx[i] = fx;
            ib.cur[i] = (long long)(gg * gs.g + j) * frame_px + (long long)fy * gs.w + fx;
            ib.key[i] = (long long)(gg * gs.g) * frame_px + (long long)fy * gs.w + fx;
        }
    }
}

// The residual bytes of this thread's items of chunk c (of the tile ib describes)
// into a raw slot: item i at 8 (t + 512 i) (current frame) and 8192 + 8 (t + 512
// i) (its key).  Items outside the frame or beyond the last block read as zero.
__device__ __forceinline__ void load_raw(const EncLaunch& L, uint8_t* raw, const ItemBase& ib, int c, int t) {
    const GopShape& gs = L.gs;
    const int dy = c * (kChunk / gs.b);
#pragma unroll
    for (int i = 0; i < kItemsPerThread; ++i) {
        const int item = t + kT * i;
        uint8_t* dc = raw + 8 * item;
        uint8_t* dk = raw + kItems * 8 + 8 * item;
        const bool valid = ib.fy[i] >= 0 && ib.fy[i] + dy < gs.h;
        const long long step = (long long)dy * gs.w;
        const uint8_t* cur = valid ? L.frames + ib.cur[i] + step : L.frames;
        const uint8_t* key = valid ? L.frames + ib.key[i] + step : L.frames;
        if (L.vec) {
            cp_async8(dc, cur, valid);
            cp_async8(dk, key, valid);
        } else {
            // cropped right edge or unaligned rows: plain byte loads, zero beyond the frame
#pragma unroll
            for (int x = 0; x < 8; ++x) {
                const bool in = valid && ib.fx[i] + x < gs.w;
                dc[x] = in ? cur[x] : (uint8_t)0;
                dk[x] = in ? key[x] : (uint8_t)0;
            }
        }
    }
}

// current - key of the thread's items into the fp16 residual operand.  A byte b
// placed under the exponent byte 0x64 is the fp16 value 1024 + b, exactly; the
// difference of two such values is cur - key, exactly (|cur - key| <= 255 <
// 2^11), so a pixel pair costs two byte permutes and one half2 subtract.
__device__ __forceinline__ void form_residual(const uint8_t* raw, uint8_t* rbuf, int t) {
#pragma unroll
    for (int i = 0; i < kItemsPerThread; ++i) {
        const int item = t + kT * i;
        const uint2 cv = *reinterpret_cast<const uint2*>(raw + 8 * item);
        const uint2 kv = *reinterpret_cast<const uint2*>(raw + kItems * 8 + 8 * item);
        const uint32_t cw[2] = {cv.x, cv.y}, kw[2] = {kv.x, kv.y};
        uint4 pk;
        uint32_t* w = reinterpret_cast<uint32_t*>(&pk);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            // bytes 2 (e & 1), 2 (e & 1) + 1 of the word, each under 0x64
            const uint32_t sel = (e & 1) ? 0x4342u : 0x4140u;
            const uint32_t ch = __byte_perm(cw[e >> 1], 0x64646464u, sel);
            const uint32_t kh = __byte_perm(kw[e >> 1], 0x64646464u, sel);
            const __half2 d = __hsub2(*reinterpret_cast<const __half2*>(&ch), *reinterpret_cast<const __half2*>(&kh));
            w[e] = *reinterpret_cast<const uint32_t*>(&d);
        }
        const int b = item / (kChunk / 8), kseg = item % (kChunk / 8);
        *reinterpret_cast<uint4*>(rbuf + rchunk_off((uint32_t)b, (uint32_t)(8 * kseg))) = pk;
    }
}

// Thread 0: every plan's hi and lo chunk c into a Phi stage (plan q's hi chunk at
// 256 col_q bytes, its lo chunk m16_q x 128 bytes after it).
__device__ __forceinline__ void load_phi(const EncLaunch& L, uint8_t* stage, uint64_t* full, int c) {
    mbar_arrive_expect_tx(full, phi_stage_bytes(L.m16_total));
    for (int q = 0; q < L.n_plans; ++q) {
        const EncPlan& P = L.p[q];
        const uint32_t cb = (uint32_t)P.m16 * kChunk * 2;                  // one chunk of one image
        const size_t img = (size_t)P.m16 * L.gs.n * 2;
        uint8_t* dst = stage + 2u * (uint32_t)P.col * kChunk * 2u;
        bulk_g2s(dst, P.img + (size_t)c * cb, cb, full);
        bulk_g2s(dst + cb, P.img + img + (size_t)c * cb, cb, full);
    }
}

constexpr int kConvWarps = kT / 32;                 // warps 1 .. 16: residual chunks and y
constexpr int kThreadsE = 32 + kT;                  // warp 0: Phi copies and MMAs
constexpr uint32_t kBarConv = 1;                    // named barrier of the converter warps

template <int S, int D>
__global__ void __launch_bounds__(kThreadsE, 1) k_encode_tcg(const __grid_constant__ EncLaunch L) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
    const int mt = L.m16_total;
    const uint32_t kPhiStage = phi_stage_bytes(mt);
    uint8_t* phi_s = sm;
    uint8_t* r_s = sm + off_r(S, mt);
    uint8_t* raw_s = sm + off_raw(S, mt);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + off_bar(S, D, mt));
    uint64_t* phi_full = bar;              // [S]: the stage's Phi chunks have landed
    uint64_t* r_full = bar + S;            // [S]: the converter warps have formed the stage's residual chunk
    uint64_t* mma_done = bar + 2 * S;      // [S]: the stage's MMAs have read both its buffers
    uint64_t* acc_full = bar + 3 * S;      // the tile's accumulators are complete
    uint64_t* acc_empty = bar + 3 * S + 1; // the converter warps have read them out
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 3 * S + 2);
    int* abort = reinterpret_cast<int*>(bar + 3 * S + 3);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nch = L.gs.n / kChunk;                      // 1, 4 or 16
    const int lg_nch = nch == 1 ? 0 : nch == 4 ? 2 : 4;
    const uint32_t ncols = mt <= 32 ? 32u : mt <= 64 ? 64u : mt <= 128 ? 128u : mt <= 256 ? 256u : 512u;
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
        tmem_alloc(tmem_slot, ncols);
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
            // ---- Phi copies, S - 1 chunks ahead, and every MMA ----
            const uint32_t s_base = smem_u32(sm);
            bool ok = true;
            int phi_last[S], mma_last[S];   // each stage's last copy and commit (for the drain)
#pragma unroll
            for (int s = 0; s < S; ++s) phi_last[s] = mma_last[s] = -1;
#pragma unroll
            for (int g = 0; g < S - 1; ++g)
                if (g < total) {
                    load_phi(L, phi_s + (uint32_t)g * kPhiStage, &phi_full[g], g & (nch - 1));
                    phi_last[g] = g;
                }
            for (int g = 0; g < total; ++g) {
                const int s = g % S, c = g & (nch - 1);
                const uint32_t u = (uint32_t)(g / S);
                // a tile's first chunk overwrites the accumulators: the previous tile's y is out
                if (c == 0 && g > 0) ok = wait_e(acc_empty, (uint32_t)(((g >> lg_nch) - 1) & 1), abort, L.err) && ok;
                ok = wait_e(&phi_full[s], u & 1, abort, L.err) && ok;
                ok = wait_e(&r_full[s], u & 1, abort, L.err) && ok;
                fence_after_sync();
                if (ok) {
                    const uint64_t da = desc_sw128(s_base + off_r(S, mt) + (uint32_t)s * kRStage, 16, 1024);
                    for (int q = 0; q < L.n_plans; ++q) {
                        const EncPlan& P = L.p[q];
                        const uint32_t po = (uint32_t)s * kPhiStage + 2u * (uint32_t)P.col * kChunk * 2u;
                        const uint64_t dh = desc_sw128(s_base + po, 16, 1024);
                        const uint64_t dl = desc_sw128(s_base + po + (uint32_t)P.m16 * kChunk * 2u, 16, 1024);
                        const uint32_t id = idesc_f16(128, (uint32_t)P.m16, 0u, 0u, 0u);
#pragma unroll
                        for (uint32_t ks = 0; ks < kChunk / 16; ++ks) {
                            mma_f16(tmem + (uint32_t)P.col, da + 2 * ks, dh + 2 * ks, id, (c > 0 || ks > 0) ? 1u : 0u);
                            mma_f16(tmem + (uint32_t)P.col, da + 2 * ks, dl + 2 * ks, id, 1u);
                        }
                    }
                    mma_commit(&mma_done[s]);
                    mma_last[s] = g;
                    if (c == nch - 1) mma_commit(acc_full);
                }
                // Phi for chunk g + S - 1, into the stage whose last reader was chunk g - 1
                const int gn = g + S - 1;
                if (gn < total) {
                    const int sn = gn % S;
                    if (gn >= S) ok = wait_e(&mma_done[sn], (uint32_t)((gn / S - 1) & 1), abort, L.err) && ok;
                    if (ok) {
                        load_phi(L, phi_s + (uint32_t)sn * kPhiStage, &phi_full[sn], gn & (nch - 1));
                        phi_last[sn] = gn;
                    }
                }
            }
            // copies and MMAs still in flight after a wait gave up: wait for each
            // stage's last ones (bounded; they have completed on the normal path)
#pragma unroll
            for (int s = 0; s < S; ++s) {
                if (phi_last[s] >= 0) mbar_wait(&phi_full[s], (uint32_t)((phi_last[s] / S) & 1), kWaitNs);
                if (mma_last[s] >= 0) mbar_wait(&mma_done[s], (uint32_t)((mma_last[s] / S) & 1), kWaitNs);
            }
        }
        __syncwarp();
    } else {
        // ---- residual chunks (D chunks of bytes in flight) and y ----
        const int t = threadIdx.x - 32;
        bool ok = true;
        ItemBase pf;                 // the item bases of the tile the prefetch is in
        int pf_tile = -1;
        auto prefetch = [&](int gp, uint8_t* slot) {
            const int tp = tile_of(gp);
            if (tp != pf_tile) {
                item_bases(L, tp, rows, t, pf);
                pf_tile = tp;
            }
            load_raw(L, slot, pf, gp & (nch - 1), t);
        };
#pragma unroll
        for (int g = 0; g < D; ++g) {
            if (g < total) prefetch(g, raw_s + (uint32_t)g * kRawSlot);
            cp_async_commit();
        }
        uint32_t ph_acc = 0;
        for (int g = 0; g < total; ++g) {
            const int s = g % S, c = g & (nch - 1);
            const uint32_t u = (uint32_t)(g / S);
            uint8_t* raw = raw_s + (uint32_t)(g % D) * kRawSlot;
            cp_async_wait_group<D - 1>();                   // this thread's bytes of chunk g
            if (g >= S) ok = wait_e(&mma_done[s], (u - 1) & 1, abort, L.err) && ok;   // R stage s is free
            form_residual(raw, r_s + (uint32_t)s * kRStage, t);
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&r_full[s]);
            if (g + D < total) prefetch(g + D, raw);
            cp_async_commit();
            if (c == nch - 1) {
                // y = D 2^-e through shared memory (the residual ring: every MMA of
                // the tile has completed), 64 columns at a time; row r's column x
                // sits at [r][x ^ (r % 32)], so that the TMEM-side writes (one row
                // per lane) and the row-contiguous reads both avoid bank conflicts
                ok = wait_e(acc_full, ph_acc, abort, L.err) && ok;
                ph_acc ^= 1;
                fence_after_sync();
                const int tile = tile_of(g);
                float* ys = reinterpret_cast<float*>(r_s);
                // four warps per TMEM lane quarter, 16 columns of a slice each
                const int q4 = warp & 3, qc = (warp - 1) >> 2;
                const int r = 32 * q4 + lane;
                const int live = min(kTile, rows - tile * kTile);
                for (int q = 0; q < L.n_plans; ++q) {
                    const EncPlan& P = L.p[q];
                    for (int s0 = 0; s0 < P.m16; s0 += 64) {
#pragma unroll
                        for (int cc = 0; cc < 16; cc += 8) {
                            const int col = s0 + 16 * qc + cc;
                            if (col < P.m16) {
                                uint32_t d[8];
                                tmem_ld8(tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(P.col + col), d);
                                tmem_wait_ld();
#pragma unroll
                                for (int i = 0; i < 8; ++i)
                                    ys[r * 64 + ((16 * qc + cc + i) ^ (r & 31))] = __uint_as_float(d[i]) * P.scale;
                            }
                        }
                        named_sync(kBarConv, kT);
                        // a warp stores whole row segments: rows w, w + 16, ..., lanes
                        // along the slice's columns
                        const int width = min(64, P.m - s0);
                        float* yt = P.y + (size_t)tile * kTile * P.m + s0;
                        if (ok)
                            for (int rr = warp - 1; rr < live; rr += kConvWarps)
                                for (int cl = lane; cl < width; cl += 32)
                                    yt[rr * P.m + cl] = ys[rr * 64 + (cl ^ (rr & 31))];
                        named_sync(kBarConv, kT);
                    }
                }
                // this warp's accumulator reads are done: the next tile may overwrite them
                fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(acc_empty);
            }
        }
        cp_async_wait_all();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 0) tmem_dealloc(tmem, ncols);
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

template <int S, int D>
cudaError_t launch_shape(const EncLaunch& L, int grid, cudaStream_t s) {
    // the shared-memory limit is raised to the device maximum once per shape and
    // device (a driver call per launch would cost microseconds of host time)
    static std::atomic<uint64_t> raised{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = 1ull << (dev & 63);
    if (!(raised.load(std::memory_order_acquire) & bit)) {
        e = cudaFuncSetAttribute(k_encode_tcg<S, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax);
        if (e != cudaSuccess) return e;
        raised.fetch_or(bit, std::memory_order_acq_rel);
    }
    k_encode_tcg<S, D><<<grid, kThreadsE, smem_bytes(S, D, L.m16_total), s>>>(L);
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
    // 8-byte frame loads when every block row segment starts on an 8-byte
    // boundary and no block is cropped at the right edge
    const int vec = gs.w % 8 == 0 && gs.w % gs.b == 0 && (reinterpret_cast<uintptr_t>(frames) & 7) == 0;
    // consecutive plans whose accumulators fit one launch share it
    for (int i = 0; i < n_plans;) {
        EncLaunch L{};
        L.frames = frames;
        L.gs = gs;
        L.err = plans[i]->ctx->err_dev;
        L.vec = vec;
        int mt = 0, k = 0;
        while (i + k < n_plans && k < kMaxEncPlans) {
            const cs_plan* p = plans[i + k];
            const int m16 = m16_of_e(p->m);
            if (k > 0 && mt + m16 > kMaxM16Total) break;
            EncPlan& P = L.p[k];
            P.img = enc_images(p);
            P.y = ys[i + k];
            P.m = p->m;
            P.m16 = m16;
            P.col = mt;
            P.scale = ldexpf(1.f, -p->tc_ephi);
            mt += m16;
            ++k;
        }
        L.n_plans = k;
        L.m16_total = mt;
        // the deepest pipeline that fits
        cudaError_t e;
        if (smem_bytes(3, 4, mt) <= kSmemMax) e = launch_shape<3, 4>(L, grid, s);
        else if (smem_bytes(2, 4, mt) <= kSmemMax) e = launch_shape<2, 4>(L, grid, s);
        else if (smem_bytes(2, 3, mt) <= kSmemMax) e = launch_shape<2, 3>(L, grid, s);
        else e = launch_shape<2, 2>(L, grid, s);
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
