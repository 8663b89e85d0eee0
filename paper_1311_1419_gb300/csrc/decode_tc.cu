// K6 + K7: persistent tensor-core decode on tcgen05.
//
// Recovery of every measured block by fixed-count FISTA on
// 1/2 ||A s - y||^2 + lambda ||s||_1 (Eq. 1 with an l1 regulariser in the DCT
// basis; Beck & Teboulle 2009), followed by r = Psi s and the key add-back of
// Eq. (4).  Across blocks the two products of every iteration are dense
// contractions; a tile of 128 blocks runs them on the tensor cores with the
// blocks on the 128 TMEM lanes:
//
//   GEMM1  U [128 x M16] = Z [128 x 256]   . A^T [256 x M16]   (u = A z per block)
//   GEMM2  G [128 x 256] = P [128 x M16]   . A   [M16 x 256]   (g = A^T (u - y))
//
// A tcgen05.mma costs about the same number of cycles whatever its N when an
// operand comes from shared memory, so GEMM2 is issued at the full N = 256 and
// GEMM1 takes its A operand (Z) straight from tensor memory, where it runs at
// the tensor cores' rate.  Per CTA (one per SM):
//   shared memory : A (hi and lo 16-bit images, 128-byte swizzled, loaded by the
//                   bulk-copy engine), the residual operand P (hi, lo), the DCT
//   tensor memory : the accumulator (U, then G), Z hi and Z lo (GEMM1's A)
//   registers     : s^{k-1} of the thread's 64 coefficients (the momentum state;
//                   16 of them in shared memory, interleaved by thread)
// y is re-read from L2 each iteration, by coalesced asynchronous copies into the
// P operand's slots while the tensor cores and the gradient step run.  The iterate z is kept as its hi + lo
// halves (22 significant bits with fp16).  FP32-grade products use three MMAs
// (hi.hi + lo.hi + hi.lo); mixed precision runs one (hi.hi) until its tail.
//
// Roles: 16 warps; lane quarter (32 blocks) = warp % 4, column group = warp / 4
// (64 coefficients of the gradient step in two slices of 32, a quarter of M16
// in the residual step).  Thread 0 also loads A and issues the MMAs, between its own epilogue
// phases (every phase waits on the previous one anyway); GEMM1 starts on the
// first half of every column group as soon as all warps have written it.  One launch may carry several jobs (plans / GOP
// calls of the same operand type); tiles are numbered across jobs and A is
// reloaded when a CTA moves to another job.  Every mbarrier wait is bounded;
// a wait that gives up sets the context's error word and the CTA drains.
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

constexpr int kN = 256;               // coefficients per block (16 x 16 blocks)
constexpr int kMaxM16 = 128;          // measurement rows kept on chip
constexpr int kTile = 128;            // blocks per tile = TMEM lanes = MMA M
constexpr int kEpiWarps = 16;         // warps 4 .. 19
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kProdWarps = 4;         // warp 0 issues MMAs and copies A, warps 1 .. 3 stage y
constexpr int kStageWarps = kProdWarps - 1;
constexpr int kThreads = (kProdWarps + kEpiWarps) * 32;
// registers per thread: at launch, then the producer and epilogue warpgroups
constexpr int kLaunchRegs = 96, kProdRegs = 32, kEpiRegs = 112;
static_assert(kProdWarps * 32 * kProdRegs + kEpiThreads * kEpiRegs <= kThreads * kLaunchRegs,
              "register split exceeds the launch allocation");
constexpr uint32_t kBarEpi = 1, kBarStage = 2;          // named barriers
constexpr int kPerThread = kN / 4;    // coefficients per epilogue thread
constexpr uint32_t kPImg = kTile * kMaxM16 * 2;         // 32 KB per 16-bit P image (2 K atoms)
// Shared-memory layout of a kernel instance for M16 <= MX: the A images take
// MX x 512 bytes each, and the momentum pairs that do not stay in registers
// take the rest (MX = 128: 24 pairs in registers, 8 in shared memory; MX = 96:
// 16 and 16), so that the epilogue does not spill.
template <int MX>
struct Lay {
    static constexpr int kMax = MX;
    static constexpr int kSpReg = MX > 96 ? 24 : 16;   // momentum pairs in registers
    static constexpr uint32_t kAImg = (uint32_t)MX * kN * 2;
    static constexpr uint32_t kOffAHi = 0, kOffALo = kAImg;
    static constexpr uint32_t kOffPHi = 2 * kAImg, kOffPLo = kOffPHi + kPImg;
    static constexpr uint32_t kOffC = kOffPLo + kPImg;             // DCT matrix, 1 KB
    static constexpr uint32_t kOffMisc = kOffC + 1024;
    static constexpr uint32_t kOffSp = kOffMisc + 1024;             // [32 - kSpReg][kEpiThreads] float2
    static constexpr uint32_t kSmemBytes = kOffSp + (kPerThread / 2 - kSpReg) * kEpiThreads * 8 + 1024;
    static_assert(kSmemBytes <= 232448, "shared memory per CTA");
};
constexpr uint32_t kColAcc = 0, kColZHi = 256, kColZLo = 384;
constexpr uint64_t kWaitNs = 1000000000ull;             // 1 s per wait

struct Misc {
    uint64_t bar_load, bar_u, bar_g, bar_p, bar_z0, bar_z1, bar_y, bar_drain;
    uint32_t tmem_base;
    int abort;
    int next_tile;
    int load_failed;
    uint32_t colmax[kTile];
};

}  // namespace

// One job of a launch: the blocks of one cs_decode_gop call.
struct TcJob {
    const uint8_t* a_img;   // hi image then lo image, m16 x 512 bytes each
    const float* y;
    const uint8_t* keys;
    float* out_f32;
    uint8_t* out_u8;
    const float* dct;       // [16][16]
    GopShape gs;
    long long rows;         // measured blocks
    int tile_begin;         // first global tile of the job
    int m16;                // M rounded up to 16
    int iters;
    int split_from;         // iterations k >= split_from use the 3-MMA split
    float lambda_rel, inv_l;
    float su, sg, sp;       // U = acc su, G = acc sg, P operand = P sp
    float tv_beta, tv_mu, tv_alpha;   // TV recovery (k_tv_tc): the splitting's penalties, step
};

constexpr int kMaxJobs = 48;
struct TcLaunch {
    const float* beta;
    int* err;
    int* tile_counter;      // zeroed before the launch; tiles are handed out in order
    uint8_t* scratch;       // TV recovery: per-CTA state (q and lambda), kTvScrBytes each
    int drop_arrival;       // test hook: CTA 0 withholds its first residual-ready arrival
    int n_jobs;
    int n_tiles;
    TcJob jobs[kMaxJobs];
};

namespace {

__device__ __forceinline__ int job_of(const TcLaunch& L, int tile) {
    int j = 0;
    while (j + 1 < L.n_jobs && L.jobs[j + 1].tile_begin <= tile) ++j;
    return j;
}

template <bool BF>
__device__ __forceinline__ uint32_t pack2(float2 v) {
    if constexpr (BF) {
        __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
        return *reinterpret_cast<uint32_t*>(&h);
    } else {
        __half2 h = __floats2half2_rn(v.x, v.y);
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

// Bounded wait; once any wait in the CTA has given up, later waits return at
// once so that every role drains through the same control flow.
__device__ __forceinline__ bool wait_bar(Misc* ms, uint64_t* bar, uint32_t parity, int* err) {
    if (*(volatile int*)&ms->abort) return false;
    if (mbar_wait(bar, parity, kWaitNs)) return true;
    *(volatile int*)&ms->abort = 1;
    atomicExch(err, 1);
    return false;
}

// Coefficients of an epilogue thread: two slices of 32, 32 c .. 32 c + 31 (half
// 0) and 128 + 32 c .. (half 1), in chunks of 8.  Half 0 of all column groups
// covers accumulator columns 0 .. 127, so once it is done GEMM1 may overwrite
// them (U needs at most M16 <= 128 columns) while half 1 is still being read.
__device__ __forceinline__ int coef_of(int cgrp, int half, int chunk) {
    return 128 * half + 32 * cgrp + 8 * chunk;
}

__device__ __forceinline__ float2 u2f2(uint32_t a, uint32_t b) {
    return make_float2(__uint_as_float(a), __uint_as_float(b));
}

// Byte offset of the 8-byte granule holding elements k..k+3 (k % 4 == 0) of
// row `row` in a K-major operand of `row_groups` 8-row groups, 128-byte swizzle.
__device__ __forceinline__ uint32_t kmajor_off(uint32_t row, uint32_t k, uint32_t row_groups) {
    const uint32_t r = row & 7;
    return ((k >> 6) * row_groups + (row >> 3)) * 1024u + r * 128u + ((((k & 63) >> 3) ^ r) << 4) +
           ((k & 7) << 1);
}

// Stage the tile's y in the slots of the P operand, which are free between
// GEMM2's completion and the next residual step.  y[b][m] goes to the slot the
// residual step of block b later overwrites with P[b][m]: elements m, m+1 of
// each 4-element granule to the P hi granule, m+2, m+3 to the P lo granule.
// Warp wi of nw copies rows wi, wi + nw, ...; its lanes read consecutive m.
__device__ __forceinline__ void stage_y(uint8_t* p_hi, uint8_t* p_lo, const float* y_tile,
                                        long long rows_left, int m_rows, int wi, int lane, int nw) {
    const int nrows = rows_left < kTile ? (int)rows_left : kTile;
    // slot of (b, m) = kmajor_off(b, m & ~3) + 4 (m & 1) in P hi (m & 2 == 0) or P lo.
    // With m = lane + 32 j the low five bits of m are the lane's, so the slot is
    //   row(b) + lane_col + (j / 2) * 16 KB + ((lane_chunk ^ 16 (b & 7)) ^ 64 (j & 1)),
    // row(b) = (b / 8) * 1024 + (b % 8) * 128 and lane_chunk = 16 (lane / 8): the
    // 16-byte chunk index XORed with b & 7 is the 128-byte swizzle.
    const uint32_t lane_col = (((uint32_t)lane & 4u) << 1) + 4u * ((uint32_t)lane & 1u) +
                              (((uint32_t)lane & 2u) ? kPImg : 0u);
    const uint32_t lane_chunk = ((uint32_t)lane >> 3) << 4;
    for (int b = wi; b < nrows; b += nw) {
        const float* src = y_tile + (long long)b * m_rows;
        uint8_t* row = p_hi + (uint32_t)(b >> 3) * 1024u + (uint32_t)(b & 7) * 128u + lane_col;
        const uint32_t x = lane_chunk ^ ((uint32_t)(b & 7) << 4);
#pragma unroll
        for (int j = 0; j < kMaxM16 / 32; ++j) {
            const int m = lane + 32 * j;
            if (m < m_rows)
                cp_async4(row + (uint32_t)(j >> 1) * (kTile / 8) * 1024u + (x ^ (64u * (j & 1))),
                          src + m, true);
        }
    }
    (void)p_lo;   // P lo follows P hi at kPImg
    cp_async_commit();
}

// GEMM1 K-steps ks0 .. ks0 + nks - 1 (16 coefficients each; steps 0 .. 7 read
// coefficients 0 .. 127, steps 8 .. 15 the rest), issued by the single MMA thread.
template <bool BF, int MX>
__device__ __forceinline__ void issue_gemm1_steps(uint32_t tbase, uint32_t s_base, int m16, int ks0,
                                                  int nks, bool split) {
    const uint32_t rg = (uint32_t)(m16 / 8);
    const uint64_t d_hi = desc_sw128(s_base + Lay<MX>::kOffAHi, 16, 1024);
    const uint64_t d_lo = desc_sw128(s_base + Lay<MX>::kOffALo, 16, 1024);
    const uint32_t id1 = idesc_f16(128, (uint32_t)m16, BF ? 1u : 0u, 0u, 0u);
#pragma unroll 1
    for (int j = 0; j < nks; ++j) {
        const uint32_t ks = (uint32_t)(ks0 + j);
        const uint32_t n0 = 16 * ks;
        const uint32_t b16 = ((n0 >> 6) * rg * 1024 + ((n0 & 63) >> 4) * 32) >> 4;
        const uint32_t zh = tbase + kColZHi + 8 * ks;
        const uint32_t zl = tbase + kColZLo + 8 * ks;
        mma_f16_tmem_a(tbase + kColAcc, zh, d_hi + b16, id1, ks != 0);
        if (split) {
            mma_f16_tmem_a(tbase + kColAcc, zl, d_hi + b16, id1, 1);
            mma_f16_tmem_a(tbase + kColAcc, zh, d_lo + b16, id1, 1);
        }
    }
}

// GEMM2: G = P A at N = 256, K = m16.
template <bool BF, int MX>
__device__ __forceinline__ void issue_gemm2(uint32_t tbase, uint32_t s_base, int m16, bool split) {
    const uint64_t dp_hi = desc_sw128(s_base + Lay<MX>::kOffPHi, 16, 1024);
    const uint64_t dp_lo = desc_sw128(s_base + Lay<MX>::kOffPLo, 16, 1024);
    const uint64_t da_hi = desc_sw128(s_base + Lay<MX>::kOffAHi, (uint32_t)(m16 / 8) * 1024, 1024);
    const uint64_t da_lo = desc_sw128(s_base + Lay<MX>::kOffALo, (uint32_t)(m16 / 8) * 1024, 1024);
    const uint32_t id2 = idesc_f16(128, kN, BF ? 1u : 0u, 0u, 1u);
#pragma unroll 1
    for (int ks = 0; ks < m16 / 16; ++ks) {
        const uint32_t m0 = 16 * (uint32_t)ks;
        const uint32_t a16 = ((m0 >> 6) * (kTile / 8) * 1024 + ((m0 & 63) >> 4) * 32) >> 4;
        const uint32_t b16 = ((m0 >> 3) * 1024) >> 4;
        mma_f16(tbase + kColAcc, dp_hi + a16, da_hi + b16, id2, ks > 0);
        if (split) {
            mma_f16(tbase + kColAcc, dp_lo + a16, da_hi + b16, id2, 1);
            mma_f16(tbase + kColAcc, dp_hi + a16, da_lo + b16, id2, 1);
        }
    }
}

// The tile loop every role runs: a CTA-wide barrier after the tile is fetched
// (A), after the tile's set-up (B) and after its reconstruction (C).  Roles
// are warp-uniform, so each warp meets the same barriers at its own code.
__device__ __forceinline__ int fetch_tile(const TcLaunch& L, Misc* ms) {
    if (threadIdx.x == 0) ms->next_tile = atomicAdd(L.tile_counter, 1);
    __syncthreads();   // A
    return ms->next_tile;
}
__device__ __forceinline__ void cta_sync() {
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
}

// The job's operand image (hi, then lo) into shared memory, by the MMA warp when
// the CTA moves to another job.  Returns false when the wait gave up.
template <int MX>
__device__ __forceinline__ bool load_images(const TcLaunch& L, const TcJob& J, Misc* ms, uint8_t* sm,
                                            int lane, uint32_t& ph_load) {
    if (lane == 0) {
        const uint32_t img = (uint32_t)J.m16 * kN * 2;
        mbar_arrive_expect_tx(&ms->bar_load, 2 * img);
        bulk_g2s(sm + Lay<MX>::kOffAHi, J.a_img, img, &ms->bar_load);
        bulk_g2s(sm + Lay<MX>::kOffALo, J.a_img + img, img, &ms->bar_load);
    }
    __syncwarp();
    const bool loaded = wait_bar(ms, &ms->bar_load, ph_load, L.err);
    if (!loaded) ms->load_failed = 1;
    ph_load ^= 1;
    return loaded;
}

// Warp 0: loads A when the CTA moves to another job and issues every MMA.  Only
// lane 0 issues; the warp waits together.
template <bool BF, int MX>
__device__ __forceinline__ void mma_role(const TcLaunch& L, Misc* ms, uint8_t* sm, uint32_t tbase,
                                         uint32_t s_base, int lane) {
    uint32_t ph_p = 0, ph_z0 = 0, ph_z1 = 0, ph_load = 0;
    int cur_job = -1;
    bool ok = true;
    for (;;) {
        const int tile = fetch_tile(L, ms);
        if (tile >= L.n_tiles) break;
        const int jid = job_of(L, tile);
        const TcJob& J = L.jobs[jid];
        if (jid != cur_job) {
            ok = load_images<MX>(L, J, ms, sm, lane, ph_load) && ok;
            cur_job = jid;
        }
        cta_sync();   // B: Z = 0 is in tensor memory
        if (J.iters > 0 && ok && lane == 0) {
            issue_gemm1_steps<BF, MX>(tbase, s_base, J.m16, 0, 16, 0 >= J.split_from);
            mma_commit(&ms->bar_u);
        }
        __syncwarp();
        for (int k = 0; k < J.iters; ++k) {
            ok = wait_bar(ms, &ms->bar_p, ph_p, L.err) && ok;
            ph_p ^= 1;
            fence_after_sync();
            if (ok && lane == 0) {
                issue_gemm2<BF, MX>(tbase, s_base, J.m16, k >= J.split_from);
                mma_commit(&ms->bar_g);
            }
            __syncwarp();
            if (k + 1 < J.iters) {
                const bool z_split = k + 1 >= J.split_from;
                ok = wait_bar(ms, &ms->bar_z0, ph_z0, L.err) && ok;
                ph_z0 ^= 1;
                fence_after_sync();
                if (ok && lane == 0) issue_gemm1_steps<BF, MX>(tbase, s_base, J.m16, 0, 8, z_split);
                __syncwarp();
                ok = wait_bar(ms, &ms->bar_z1, ph_z1, L.err) && ok;
                ph_z1 ^= 1;
                fence_after_sync();
                if (ok && lane == 0) {
                    issue_gemm1_steps<BF, MX>(tbase, s_base, J.m16, 8, 8, z_split);
                    mma_commit(&ms->bar_u);
                }
                __syncwarp();
            }
        }
        cta_sync();   // C
    }
    if (lane == 0) {
        // drain: every MMA issued so far has completed before TMEM is freed
        mma_commit(&ms->bar_drain);
        mbar_wait(&ms->bar_drain, 0, kWaitNs);
        // an A copy whose wait gave up may still be in flight: wait for it (bounded)
        if (ms->load_failed) mbar_wait(&ms->bar_load, ph_load ^ 1, kWaitNs);
    }
    __syncwarp();
}

// Warps 1..3: zero the P operand at a tile's start and stage y into its slots
// for every iteration, as soon as GEMM2 of the previous iteration has consumed P.
template <int MX>
__device__ __forceinline__ void stage_role(const TcLaunch& L, Misc* ms, uint8_t* sm, int wi, int lane) {
    uint8_t* p_hi = sm + Lay<MX>::kOffPHi;
    uint8_t* p_lo = sm + Lay<MX>::kOffPLo;
    const int st = wi * 32 + lane;
    uint32_t ph_g = 0;
    for (;;) {
        const int tile = fetch_tile(L, ms);
        if (tile >= L.n_tiles) break;
        const TcJob& J = L.jobs[job_of(L, tile)];
        const long long tile_row0 = (long long)(tile - J.tile_begin) * kTile;
        const long long rows_left = J.rows - tile_row0;
        const float* y_tile = J.y + tile_row0 * J.gs.m;
        // padding rows m >= M and absent blocks stay zero: their U and y are zero
        for (int i = st; i < (int)(2 * kPImg / 16); i += kStageWarps * 32)
            reinterpret_cast<uint4*>(p_hi)[i] = make_uint4(0u, 0u, 0u, 0u);
        named_sync(kBarStage, kStageWarps * 32);
        if (J.iters > 0) {
            stage_y(p_hi, p_lo, y_tile, rows_left, J.gs.m, wi, lane, kStageWarps);
            cp_async_arrive_noinc(&ms->bar_y);
        }
        cta_sync();   // B
        for (int k = 0; k < J.iters; ++k) {
            wait_bar(ms, &ms->bar_g, ph_g, L.err);   // GEMM2 of iteration k has read P
            ph_g ^= 1;
            if (k + 1 < J.iters) {
                stage_y(p_hi, p_lo, y_tile, rows_left, J.gs.m, wi, lane, kStageWarps);
                cp_async_arrive_noinc(&ms->bar_y);
            }
        }
        cta_sync();   // C
    }
    cp_async_wait_all();
}

// Warps 4..19: the residual step, the gradient / soft-threshold / momentum step
// and the reconstruction, on the tile's TMEM lanes.
template <bool BF, int MX>
__device__ __forceinline__ void epi_role(const TcLaunch& L, Misc* ms, uint8_t* sm, uint32_t tbase,
                                         int warp, int lane) {
    using Y = Lay<MX>;
    constexpr int kSpReg = Y::kSpReg;
    const float* c_s = reinterpret_cast<const float*>(sm + Y::kOffC);
    const int ew = warp - kProdWarps;
    const int q = warp & 3, cgrp = ew >> 2;                 // TMEM lane quarter = warp % 4
    const int blk = 32 * q + lane;                          // TMEM lane = block of the tile
    const uint32_t lane_addr = tbase + ((uint32_t)(32 * q) << 16);
    uint8_t* p_hi = sm + Y::kOffPHi;
    uint8_t* p_lo = sm + Y::kOffPLo;
    float2* sp_smem = reinterpret_cast<float2*>(sm + Y::kOffSp) + (ew * 32 + lane);
    uint32_t ph_u = 0, ph_g = 0, ph_y = 0;
    bool first_tile = true;
    for (;;) {
        const int tile = fetch_tile(L, ms);
        if (tile >= L.n_tiles) break;
        const int jid = job_of(L, tile);
        const TcJob& J = L.jobs[jid];
        const GopShape& gs = J.gs;
        const long long row = (long long)(tile - J.tile_begin) * kTile + blk;
        const bool live = row < J.rows;
        const int mq = J.m16 / 4;                           // residual rows of this thread
        const int mbase = cgrp * mq;
        const float2 ginv2 = make_float2(-J.sg * J.inv_l, -J.sg * J.inv_l);
        // s^{k-1}: pairs 0 .. kSpReg-1 in registers, the rest in shared memory
        float2 sp[kSpReg];
#pragma unroll
        for (int i = 0; i < kSpReg; ++i) sp[i] = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = kSpReg; i < kPerThread / 2; ++i)
            sp_smem[(i - kSpReg) * kEpiThreads] = make_float2(0.f, 0.f);
        float tau = 0.f;
        {   // Z = 0 in TMEM
            uint32_t zr[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) zr[i] = 0u;
            tmem_st32(lane_addr + kColZHi + 32 * cgrp, zr);
            tmem_st32(lane_addr + kColZLo + 32 * cgrp, zr);
            if (cgrp == 0) ms->colmax[blk] = 0u;
            tmem_wait_st();
        }
        cta_sync();   // B
        for (int k = 0; k < J.iters; ++k) {
            const float bk = L.beta[k];
            // --- residual P = U - y (this thread: rows mbase .. mbase + mq) ---
            const bool ok_u = wait_bar(ms, &ms->bar_u, ph_u, L.err);
            ph_u ^= 1;
            fence_after_sync();
            wait_bar(ms, &ms->bar_y, ph_y, L.err);          // y is in the P slots
            ph_y ^= 1;
            const float2 su2 = make_float2(J.su, J.su), sp2 = make_float2(J.sp, J.sp);
            const bool p_split = k >= J.split_from;
#pragma unroll
            for (int g4 = 0; g4 < kMaxM16 / 16; ++g4) {
                if (4 * g4 < mq) {
                    uint32_t u[4];
                    tmem_ld4(lane_addr + kColAcc + mbase + 4 * g4, u);
                    const uint32_t off =
                        kmajor_off((uint32_t)blk, (uint32_t)(mbase + 4 * g4), kTile / 8);
                    const float2 y01 = *reinterpret_cast<const float2*>(p_hi + off);
                    const float2 y23 = *reinterpret_cast<const float2*>(p_lo + off);
                    tmem_wait_ld();
                    const float2 p0 = mul2(sub2(mul2(u2f2(u[0], u[1]), su2), y01), sp2);
                    const float2 p1 = mul2(sub2(mul2(u2f2(u[2], u[3]), su2), y23), sp2);
                    const uint32_t h0 = pack2<BF>(p0), h1 = pack2<BF>(p1);
                    if (ok_u) {
                        *reinterpret_cast<uint2*>(p_hi + off) = make_uint2(h0, h1);
                        if (p_split) {
                            const uint32_t l0 = pack2<BF>(sub2(p0, unpack2<BF>(h0)));
                            const uint32_t l1 = pack2<BF>(sub2(p1, unpack2<BF>(h1)));
                            *reinterpret_cast<uint2*>(p_lo + off) = make_uint2(l0, l1);
                        }
                    }
                }
            }
            fence_proxy_async_smem();
            fence_before_sync();
            __syncwarp();
            // (the test hook withholds one warp's first arrival in CTA 0: the MMA
            // warp's bounded wait then gives up and the CTA drains)
            const bool withhold = L.drop_arrival && blockIdx.x == 0 && ew == 1 && k == 0 &&
                                  first_tile;
            if (lane == 0 && !withhold) mbar_arrive(&ms->bar_p);

            // --- gradient step, soft threshold, momentum ---
            const bool ok_g = wait_bar(ms, &ms->bar_g, ph_g, L.err);
            ph_g ^= 1;
            fence_after_sync();
            if (k == 0) {
                // lambda_b = lambda_rel ||A^T y_b||_inf; at k = 0, G = -A^T y
                float mx = 0.f;
#pragma unroll
                for (int ch = 0; ch < kPerThread / 8; ++ch) {
                    uint32_t g[8];
                    tmem_ld8(lane_addr + kColAcc + coef_of(cgrp, ch >> 2, ch & 3), g);
                    tmem_wait_ld();
#pragma unroll
                    for (int i = 0; i < 8; ++i) mx = fmaxf(mx, fabsf(__uint_as_float(g[i])));
                }
                atomicMax(&ms->colmax[blk], __float_as_uint(mx * J.sg));
                named_sync(kBarEpi, kEpiThreads);
                tau = J.lambda_rel * __uint_as_float(ms->colmax[blk]) * J.inv_l;
            }
            const bool want_z = k + 1 < J.iters;
            const float2 b2 = make_float2(bk, bk);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
#pragma unroll
                for (int ch = 0; ch < 4; ++ch) {
                    const int o = coef_of(cgrp, h, ch);               // first coefficient
                    uint32_t g[8], zh[4], zl[4];
                    tmem_ld8(lane_addr + kColAcc + o, g);
                    tmem_ld4(lane_addr + kColZHi + o / 2, zh);
                    tmem_ld4(lane_addr + kColZLo + o / 2, zl);
                    tmem_wait_ld();
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int si = 16 * h + 4 * ch + e;
                        const float2 zhf = unpack2<BF>(zh[e]), zlf = unpack2<BF>(zl[e]);
                        const float2 z2 = make_float2(zhf.x + zlf.x, zhf.y + zlf.y);
                        const float2 v = fma2(u2f2(g[2 * e], g[2 * e + 1]), ginv2, z2);
                        const float2 cl = make_float2(fminf(fmaxf(v.x, -tau), tau),
                                                      fminf(fmaxf(v.y, -tau), tau));
                        const float2 sv = sub2(v, cl);
                        float2& spv = si < kSpReg ? sp[si < kSpReg ? si : 0]
                                                  : sp_smem[(si - kSpReg) * kEpiThreads];
                        const float2 zn = fma2(b2, sub2(sv, spv), sv);
                        spv = sv;
                        zh[e] = pack2<BF>(zn);
                        zl[e] = pack2<BF>(sub2(zn, unpack2<BF>(zh[e])));
                    }
                    if (want_z && ok_g) {
                        tmem_st4(lane_addr + kColZHi + o / 2, zh);
                        tmem_st4(lane_addr + kColZLo + o / 2, zl);
                    }
                }
                if (want_z) {
                    tmem_wait_st();
                    fence_before_sync();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(h ? &ms->bar_z1 : &ms->bar_z0);
                }
            }
        }
        // --- reconstruct: R = C^T S C, S = s^K (rows 4 cgrp .. 4 cgrp + 3 here) ---
        // every MMA of the tile has completed (the last G was waited); the other
        // warps of this lane quarter have read their last G columns
        fence_before_sync();
        named_sync(kBarEpi, kEpiThreads);
        fence_after_sync();
#pragma unroll
        for (int kr = 0; kr < 4; ++kr) {
            // this thread holds S rows 2 cgrp, 2 cgrp + 1, 8 + 2 cgrp, 9 + 2 cgrp;
            // row (kr) = slice kr / 2, chunks 2 (kr % 2) and 2 (kr % 2) + 1
            uint32_t t[16];
#pragma unroll
            for (int qq = 0; qq < 16; ++qq) {
                float acc = 0.f;
#pragma unroll
                for (int l = 0; l < 16; l += 2) {
                    const int si = 16 * (kr >> 1) + 8 * (kr & 1) + l / 2;
                    const float2 s2 = si < kSpReg ? sp[si < kSpReg ? si : 0]
                                                  : sp_smem[(si - kSpReg) * kEpiThreads];
                    acc = fmaf(s2.x, c_s[l * 16 + qq], acc);
                    acc = fmaf(s2.y, c_s[(l + 1) * 16 + qq], acc);
                }
                t[qq] = __float_as_uint(acc);
            }
            const int krow = 8 * (kr >> 1) + 2 * cgrp + (kr & 1);
            tmem_st16(lane_addr + kColAcc + 16 * krow, t);
        }
        tmem_wait_st();
        fence_before_sync();
        named_sync(kBarEpi, kEpiThreads);
        fence_after_sync();
        const int c_idx = live ? (int)(row / gs.nblk) : 0, bl = live ? (int)(row % gs.nblk) : 0;
        const int g_key = c_idx / (gs.g - 1);
        const int bi = bl / gs.nbc, bj = bl % gs.nbc;
        const size_t frame_px = (size_t)gs.h * gs.w;
        for (int pr = 0; pr < 4; ++pr) {                   // output rows 4 cgrp + pr
            float r[16];
#pragma unroll
            for (int qq = 0; qq < 16; ++qq) r[qq] = 0.f;
            for (int kr = 0; kr < 16; ++kr) {
                uint32_t t[16];
                tmem_ld16(lane_addr + kColAcc + 16 * kr, t);
                tmem_wait_ld();
                const float cv = c_s[kr * 16 + 4 * cgrp + pr];
#pragma unroll
                for (int qq = 0; qq < 16; ++qq) r[qq] = fmaf(cv, __uint_as_float(t[qq]), r[qq]);
            }
            const int py = bi * 16 + 4 * cgrp + pr;
            if (!live || py >= gs.h) continue;
#pragma unroll
            for (int qq = 0; qq < 16; ++qq) {
                const int px = bj * 16 + qq;
                if (px >= gs.w) continue;
                const size_t off = (size_t)py * gs.w + px;
                const float v = (float)J.keys[(size_t)g_key * frame_px + off] + r[qq];
                if (J.out_f32) J.out_f32[(size_t)c_idx * frame_px + off] = v;
                if (J.out_u8)
                    J.out_u8[(size_t)c_idx * frame_px + off] = (uint8_t)fminf(fmaxf(rintf(v), 0.f), 255.f);
            }
        }
        cta_sync();   // C: the accumulator (holding T) is reused by the next tile
        first_tile = false;
    }
}

template <bool BF, int MX>
__global__ void __launch_bounds__(kThreads, 1) k_fista_tc(const __grid_constant__ TcLaunch L) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
    Misc* ms = reinterpret_cast<Misc*>(sm + Lay<MX>::kOffMisc);
    float* c_s = reinterpret_cast<float*>(sm + Lay<MX>::kOffC);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == 0) {
        if (lane == 0) {
            mbar_init(&ms->bar_load, 1);
            mbar_init(&ms->bar_u, 1);
            mbar_init(&ms->bar_g, 1);
            mbar_init(&ms->bar_p, kEpiWarps);
            mbar_init(&ms->bar_z0, kEpiWarps);
            mbar_init(&ms->bar_z1, kEpiWarps);
            mbar_init(&ms->bar_y, kStageWarps * 32);
            mbar_init(&ms->bar_drain, 1);
            ms->abort = 0;
            ms->load_failed = 0;
            fence_mbar_init();
        }
        __syncwarp();
        tmem_alloc(&ms->tmem_base, 512);
        tmem_relinquish();
    }
    for (int i = threadIdx.x; i < 256; i += kThreads) c_s[i] = L.jobs[0].dct[i];
    cta_sync();
    const uint32_t tbase = ms->tmem_base;

    // registers move from the producer warpgroup to the four epilogue warpgroups
    // (the launch holds kThreads x kLaunchRegs; the split below sums to at most that)
    if (warp < kProdWarps) {
        regs_dec<kProdRegs>();
        if (warp == 0)
            mma_role<BF, MX>(L, ms, sm, tbase, smem_u32(sm), lane);
        else
            stage_role<MX>(L, ms, sm, warp - 1, lane);
    } else {
        regs_inc<kEpiRegs>();
        epi_role<BF, MX>(L, ms, sm, tbase, warp, lane);
    }
    cta_sync();
    if (warp == 0) tmem_dealloc(tbase, 512);
}

// ---------------------------------------------------------------------------
// TV recovery on the same tiles (16 x 16 blocks, M16 <= 128): Eq. 1 with the
// total variation, min ||D r||_1 s.t. Phi r = y, by the augmented-Lagrangian
// alternating-direction iteration of the plain TV kernel (decode_tv.cu), with
// the two Phi products of every iteration on the tensor cores:
//
//   GEMM1  U [128 x M16] = R [128 x 256] . Phi^T     (Phi r per block; R read from TMEM)
//   GEMM2  G [128 x 256] = P [128 x M16] . Phi       (Phi^T P per block)
//
// with P = mu (Phi r - y) - lam.  The iterate r stays in tensor memory as its
// fp16 hi + lo halves (GEMM1's A operand, where FISTA keeps Z), and the rest of
// the state goes through a per-CTA global scratch small enough to stay in L2:
// q = nu + beta w (2 N per block; with it the difference-side gradient is
// D^T (beta D r - q) and the multiplier step is nu' = q - beta D r') and lam
// (M16 per block).  lam -= mu (Phi r' - y) needs Phi r', which is the next
// GEMM1, so it is taken there: P_k = 2 mu (U_k - y) - lam_{k-1} and lam_k =
// lam_{k-1} - mu (U_k - y), with P_0 = -mu y.  An epilogue thread (block = TMEM
// lane, column group cg) owns pixel rows 4 cg .. 4 cg + 3 of its block; the
// differences reach one row into the neighbouring column groups, whose TMEM
// columns of the same lane it reads after a barrier of the four warps of its
// lane quarter.  Per iteration k:
//   residual : P, lam                                   (after GEMM1; none at k = 0)
//   r step   : r' = r - alpha (D^T (beta D r - q) + G), staged in the
//              accumulator columns of the thread's own pixels (after GEMM2)
//   to R     : r' split into R hi / lo, then GEMM1 of r' starts
//   q step   : nu' = q - beta D r', w' = shrink(D r' - nu' / beta, 1 / beta),
//              q' = nu' + beta w'                       (while GEMM1 runs)
// Every product is FP32-grade (three MMAs per K step).
constexpr size_t kTvScrQ = 2ull * kN * kTile * 4;                   // q: [2][N / 4][128] float4
constexpr size_t kTvScrBytes = kTvScrQ + (size_t)kMaxM16 * kTile * 4;   // lam: [M16 / 4][128] float4
constexpr uint32_t kBarQuarter = 3;                                 // named barriers 3 .. 6
constexpr uint32_t kTvSmemBytes = Lay<kMaxM16>::kOffMisc + 1024 + 1024;

__device__ __forceinline__ void quarter_sync(int q) { named_sync(kBarQuarter + (uint32_t)q, 128); }

__device__ __forceinline__ float shrink_tv(float v, float t) { return v - fminf(fmaxf(v, -t), t); }

// Row p (16 pixels) of r: its R hi and lo columns, unpacked after the wait.
__device__ __forceinline__ void tv_ld_row(uint32_t lane_addr, int p, uint32_t (&hi)[8], uint32_t (&lo)[8]) {
    tmem_ld8(lane_addr + kColZHi + 8 * p, hi);
    tmem_ld8(lane_addr + kColZLo + 8 * p, lo);
}
__device__ __forceinline__ void tv_unpack_row(const uint32_t (&hi)[8], const uint32_t (&lo)[8], float (&r)[16]) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const float2 h = unpack2<false>(hi[e]), l = unpack2<false>(lo[e]);
        r[2 * e] = h.x + l.x;
        r[2 * e + 1] = h.y + l.y;
    }
}
// q of plane pl (0: differences along the row, 1: down the column) at row p, as
// float4 index v = 0 .. 3 of block blk: a warp's 32 blocks read 512 contiguous bytes.
__device__ __forceinline__ size_t tv_q_index(int pl, int p, int v, int blk) {
    return (size_t)(pl * (kN / 4) + 4 * p + v) * kTile + blk;
}
__device__ __forceinline__ void tv_ld_q(const float4* __restrict__ q4, int pl, int p, int blk, float (&o)[16]) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const float4 x = q4[tv_q_index(pl, p, v, blk)];
        o[4 * v] = x.x;
        o[4 * v + 1] = x.y;
        o[4 * v + 2] = x.z;
        o[4 * v + 3] = x.w;
    }
}
__device__ __forceinline__ void tv_st_q(float4* __restrict__ q4, int pl, int p, int blk, const float (&o)[16]) {
#pragma unroll
    for (int v = 0; v < 4; ++v)
        q4[tv_q_index(pl, p, v, blk)] = make_float4(o[4 * v], o[4 * v + 1], o[4 * v + 2], o[4 * v + 3]);
}

// Residual step of iteration k for measurements mbase .. mbase + mq - 1 of the
// thread's block: rho = U su - y (U = 0 at k = 0), P = c mu rho - lam (c = 1 at
// k = 0, else 2; lam = lam_{k-1}), lam_k = lam_{k-1} - mu rho, and P sp written
// as fp16 hi / lo over the staged y.
__device__ __forceinline__ void tv_residual(const TcJob& J, uint8_t* p_hi, uint8_t* p_lo, uint32_t lane_addr,
                                            float4* __restrict__ lam4, int blk, int mbase, int mq, int k,
                                            bool write_p) {
    const float mu = J.tv_mu, cmu = k == 0 ? mu : 2.f * mu;
    const bool use_u = k > 0, read_lam = k > 1, write_lam = k > 0 && k + 1 < J.iters;
    const float2 sp2 = make_float2(J.sp, J.sp);
#pragma unroll
    for (int g4 = 0; g4 < kMaxM16 / 16; ++g4) {
        if (4 * g4 < mq) {
            const int m = mbase + 4 * g4;
            uint32_t u[4] = {0u, 0u, 0u, 0u};
            if (use_u) tmem_ld4(lane_addr + kColAcc + m, u);
            const uint32_t off = kmajor_off((uint32_t)blk, (uint32_t)m, kTile / 8);
            const float2 y01 = *reinterpret_cast<const float2*>(p_hi + off);
            const float2 y23 = *reinterpret_cast<const float2*>(p_lo + off);
            const size_t li = (size_t)(m / 4) * kTile + blk;
            const float4 lv = read_lam ? lam4[li] : make_float4(0.f, 0.f, 0.f, 0.f);
            if (use_u) tmem_wait_ld();
            const float yy[4] = {y01.x, y01.y, y23.x, y23.y};
            float l[4] = {lv.x, lv.y, lv.z, lv.w};
            float p[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float rho = __uint_as_float(u[e]) * J.su - yy[e];
                p[e] = cmu * rho - l[e];
                l[e] -= mu * rho;
            }
            if (write_lam) lam4[li] = make_float4(l[0], l[1], l[2], l[3]);
            const float2 p0 = mul2(make_float2(p[0], p[1]), sp2), p1 = mul2(make_float2(p[2], p[3]), sp2);
            const uint32_t h0 = pack2<false>(p0), h1 = pack2<false>(p1);
            if (write_p) {
                *reinterpret_cast<uint2*>(p_hi + off) = make_uint2(h0, h1);
                const uint32_t l0 = pack2<false>(sub2(p0, unpack2<false>(h0)));
                const uint32_t l1 = pack2<false>(sub2(p1, unpack2<false>(h1)));
                *reinterpret_cast<uint2*>(p_lo + off) = make_uint2(l0, l1);
            }
        }
    }
}

// r step for rows p0 .. p0 + 3: r' = r - alpha (D^T t + G sg), t = beta D r - q
// (t_h in the row, t_v down the column; both zero where the difference leaves the
// block), r' written as fp32 into the accumulator columns of the same pixels.
// At k = 0 (first) r = q = 0.
__device__ __forceinline__ void tv_r_step(const TcJob& J, uint32_t lane_addr, const float4* __restrict__ q4,
                                          int blk, int p0, bool first) {
    const float beta = J.tv_beta, alpha = J.tv_alpha, sg = J.sg;
    float rc[16], tvp[16];   // r of the current row; t_v of the row above
#pragma unroll
    for (int c = 0; c < 16; ++c) rc[c] = tvp[c] = 0.f;
    if (!first) {
        uint32_t h0[8], l0[8];
        tv_ld_row(lane_addr, p0, h0, l0);
        if (p0 > 0) {
            uint32_t h1[8], l1[8];
            tv_ld_row(lane_addr, p0 - 1, h1, l1);
            float qv[16];
            tv_ld_q(q4, 1, p0 - 1, blk, qv);
            tmem_wait_ld();
            float ra[16];
            tv_unpack_row(h1, l1, ra);
            tv_unpack_row(h0, l0, rc);
#pragma unroll
            for (int c = 0; c < 16; ++c) tvp[c] = beta * (rc[c] - ra[c]) - qv[c];
        } else {
            tmem_wait_ld();
            tv_unpack_row(h0, l0, rc);
        }
    }
#pragma unroll 1
    for (int i = 0; i < 4; ++i) {
        const int p = p0 + i;
        uint32_t g[16];
        tmem_ld16(lane_addr + kColAcc + 16 * p, g);
        float rn[16], qh[16], qv[16];
        if (first) {
#pragma unroll
            for (int c = 0; c < 16; ++c) rn[c] = qh[c] = qv[c] = 0.f;
            tmem_wait_ld();
        } else {
            uint32_t hn[8], ln[8];
            tv_ld_row(lane_addr, p < 15 ? p + 1 : p, hn, ln);
            tv_ld_q(q4, 0, p, blk, qh);
            tv_ld_q(q4, 1, p, blk, qv);
            tmem_wait_ld();
            tv_unpack_row(hn, ln, rn);
        }
        float th[16], tv[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            th[c] = c < 15 ? beta * (rc[c + 1] - rc[c]) - qh[c] : 0.f;
            tv[c] = p < 15 ? beta * (rn[c] - rc[c]) - qv[c] : 0.f;
        }
        uint32_t o[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const float dt = (c > 0 ? th[c - 1] : 0.f) - th[c] + tvp[c] - tv[c];
            o[c] = __float_as_uint(rc[c] - alpha * fmaf(__uint_as_float(g[c]), sg, dt));
        }
        tmem_st16(lane_addr + kColAcc + 16 * p, o);
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            rc[c] = rn[c];
            tvp[c] = tv[c];
        }
    }
}

// r' (staged in the accumulator) into R hi / lo, rows p0 .. p0 + 3.
__device__ __forceinline__ void tv_to_r(uint32_t lane_addr, int p0) {
#pragma unroll
    for (int i = 0; i < 4; i += 2) {
        uint32_t v0[16], v1[16];
        tmem_ld16(lane_addr + kColAcc + 16 * (p0 + i), v0);
        tmem_ld16(lane_addr + kColAcc + 16 * (p0 + i + 1), v1);
        tmem_wait_ld();
        uint32_t hi[2][8], lo[2][8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const float2 x0 = u2f2(v0[2 * e], v0[2 * e + 1]), x1 = u2f2(v1[2 * e], v1[2 * e + 1]);
            hi[0][e] = pack2<false>(x0);
            lo[0][e] = pack2<false>(sub2(x0, unpack2<false>(hi[0][e])));
            hi[1][e] = pack2<false>(x1);
            lo[1][e] = pack2<false>(sub2(x1, unpack2<false>(hi[1][e])));
        }
        tmem_st8(lane_addr + kColZHi + 8 * (p0 + i), hi[0]);
        tmem_st8(lane_addr + kColZLo + 8 * (p0 + i), lo[0]);
        tmem_st8(lane_addr + kColZHi + 8 * (p0 + i + 1), hi[1]);
        tmem_st8(lane_addr + kColZLo + 8 * (p0 + i + 1), lo[1]);
    }
}

// q step for rows p0 .. p0 + 3 with r' from R: nu' = q - beta d, w' = shrink(d -
// nu' / beta, 1 / beta), q' = nu' + beta w', d = D r'.  At k = 0 (first) q = 0.
__device__ __forceinline__ void tv_q_step(const TcJob& J, uint32_t lane_addr, float4* __restrict__ q4, int blk,
                                          int p0, bool first) {
    const float beta = J.tv_beta, ib = 1.f / beta;
    float rc[16];
    {
        uint32_t h[8], l[8];
        tv_ld_row(lane_addr, p0, h, l);
        tmem_wait_ld();
        tv_unpack_row(h, l, rc);
    }
#pragma unroll 1
    for (int i = 0; i < 4; ++i) {
        const int p = p0 + i;
        uint32_t hn[8], ln[8];
        tv_ld_row(lane_addr, p < 15 ? p + 1 : p, hn, ln);
        float qh[16], qv[16];
        if (first) {
#pragma unroll
            for (int c = 0; c < 16; ++c) qh[c] = qv[c] = 0.f;
        } else {
            tv_ld_q(q4, 0, p, blk, qh);
            tv_ld_q(q4, 1, p, blk, qv);
        }
        tmem_wait_ld();
        float rn[16];
        tv_unpack_row(hn, ln, rn);
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const float dh = c < 15 ? rc[c + 1] - rc[c] : 0.f;
            const float dv = p < 15 ? rn[c] - rc[c] : 0.f;
            const float nh = qh[c] - beta * dh, nv = qv[c] - beta * dv;
            qh[c] = nh + beta * shrink_tv(dh - nh * ib, ib);
            qv[c] = nv + beta * shrink_tv(dv - nv * ib, ib);
        }
        tv_st_q(q4, 0, p, blk, qh);
        tv_st_q(q4, 1, p, blk, qv);
#pragma unroll
        for (int c = 0; c < 16; ++c) rc[c] = rn[c];
    }
}

// Warp 0 of the TV kernel: loads Phi's image when the CTA moves to another job
// and issues GEMM1 (from k = 1) and GEMM2 of every iteration.
template <int MX>
__device__ __forceinline__ void mma_role_tv(const TcLaunch& L, Misc* ms, uint8_t* sm, uint32_t tbase,
                                            uint32_t s_base, int lane) {
    uint32_t ph_p = 0, ph_z = 0, ph_load = 0;
    int cur_job = -1;
    bool ok = true;
    for (;;) {
        const int tile = fetch_tile(L, ms);
        if (tile >= L.n_tiles) break;
        const int jid = job_of(L, tile);
        const TcJob& J = L.jobs[jid];
        if (jid != cur_job) {
            ok = load_images<MX>(L, J, ms, sm, lane, ph_load) && ok;
            cur_job = jid;
        }
        cta_sync();   // B
        for (int k = 0; k < J.iters; ++k) {
            if (k > 0) {
                ok = wait_bar(ms, &ms->bar_z0, ph_z, L.err) && ok;   // r^k is in R
                ph_z ^= 1;
                fence_after_sync();
                if (ok && lane == 0) {
                    issue_gemm1_steps<false, MX>(tbase, s_base, J.m16, 0, 16, true);
                    mma_commit(&ms->bar_u);
                }
                __syncwarp();
            }
            ok = wait_bar(ms, &ms->bar_p, ph_p, L.err) && ok;
            ph_p ^= 1;
            fence_after_sync();
            if (ok && lane == 0) {
                issue_gemm2<false, MX>(tbase, s_base, J.m16, true);
                mma_commit(&ms->bar_g);
            }
            __syncwarp();
        }
        cta_sync();   // C
    }
    if (lane == 0) {
        mma_commit(&ms->bar_drain);
        mbar_wait(&ms->bar_drain, 0, kWaitNs);
        if (ms->load_failed) mbar_wait(&ms->bar_load, ph_load ^ 1, kWaitNs);
    }
    __syncwarp();
}

// Warps 4 .. 19 of the TV kernel: every step of the iteration but the products,
// then r^K plus the key (Eq. 4).
template <int MX>
__device__ __forceinline__ void epi_role_tv(const TcLaunch& L, Misc* ms, uint8_t* sm, uint32_t tbase, int warp,
                                            int lane) {
    const int ew = warp - kProdWarps;
    const int q = warp & 3, cgrp = ew >> 2;
    const int blk = 32 * q + lane;
    const int p0 = 4 * cgrp;
    const uint32_t lane_addr = tbase + ((uint32_t)(32 * q) << 16);
    uint8_t* p_hi = sm + Lay<MX>::kOffPHi;
    uint8_t* p_lo = sm + Lay<MX>::kOffPLo;
    uint8_t* scr = L.scratch + (size_t)blockIdx.x * kTvScrBytes;
    float4* q4 = reinterpret_cast<float4*>(scr);
    float4* lam4 = reinterpret_cast<float4*>(scr + kTvScrQ);
    uint32_t ph_u = 0, ph_g = 0, ph_y = 0;
    bool first_tile = true;
    for (;;) {
        const int tile = fetch_tile(L, ms);
        if (tile >= L.n_tiles) break;
        const TcJob& J = L.jobs[job_of(L, tile)];
        const GopShape& gs = J.gs;
        const long long row = (long long)(tile - J.tile_begin) * kTile + blk;
        const bool live = row < J.rows;
        const int mq = J.m16 / 4, mbase = cgrp * mq;
        cta_sync();   // B
        for (int k = 0; k < J.iters; ++k) {
            bool ok_u = true;
            if (k > 0) {
                ok_u = wait_bar(ms, &ms->bar_u, ph_u, L.err);
                ph_u ^= 1;
                fence_after_sync();
            }
            wait_bar(ms, &ms->bar_y, ph_y, L.err);          // y is in the P slots
            ph_y ^= 1;
            tv_residual(J, p_hi, p_lo, lane_addr, lam4, blk, mbase, mq, k, ok_u);
            fence_proxy_async_smem();
            fence_before_sync();
            __syncwarp();
            // (the test hook withholds one warp's first arrival in CTA 0)
            const bool withhold = L.drop_arrival && blockIdx.x == 0 && ew == 1 && k == 0 && first_tile;
            if (lane == 0 && !withhold) mbar_arrive(&ms->bar_p);

            wait_bar(ms, &ms->bar_g, ph_g, L.err);
            ph_g ^= 1;
            fence_after_sync();
            if (k > 0) quarter_sync(q);                     // the neighbours' q^k is written
            tv_r_step(J, lane_addr, q4, blk, p0, k == 0);
            tmem_wait_st();
            fence_before_sync();
            quarter_sync(q);                                // every read of r^k is done
            fence_after_sync();
            if (k + 1 < J.iters) {
                tv_to_r(lane_addr, p0);
                tmem_wait_st();
                fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(&ms->bar_z0);
                quarter_sync(q);                            // the neighbours' rows of r' are in R
                fence_after_sync();
                tv_q_step(J, lane_addr, q4, blk, p0, k == 0);
            }
        }
        // r^K (in the accumulator; zero when there are no iterations) plus the key
        const int c_idx = live ? (int)(row / gs.nblk) : 0, bl = live ? (int)(row % gs.nblk) : 0;
        const int g_key = c_idx / (gs.g - 1);
        const int bi = bl / gs.nbc, bj = bl % gs.nbc;
        const size_t frame_px = (size_t)gs.h * gs.w;
        for (int i = 0; i < 4; ++i) {
            const int p = p0 + i;
            uint32_t v[16];
            tmem_ld16(lane_addr + kColAcc + 16 * p, v);
            tmem_wait_ld();
            const int py = bi * 16 + p;
            if (!live || py >= gs.h) continue;
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const int px = bj * 16 + c;
                if (px >= gs.w) continue;
                const size_t off = (size_t)py * gs.w + px;
                const float rv = J.iters > 0 ? __uint_as_float(v[c]) : 0.f;
                const float x = (float)J.keys[(size_t)g_key * frame_px + off] + rv;
                if (J.out_f32) J.out_f32[(size_t)c_idx * frame_px + off] = x;
                if (J.out_u8) J.out_u8[(size_t)c_idx * frame_px + off] = (uint8_t)fminf(fmaxf(rintf(x), 0.f), 255.f);
            }
        }
        cta_sync();   // C: the accumulator is reused by the next tile
        first_tile = false;
    }
}

template <int MX>
__global__ void __launch_bounds__(kThreads, 1) k_tv_tc(const __grid_constant__ TcLaunch L) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
    Misc* ms = reinterpret_cast<Misc*>(sm + Lay<MX>::kOffMisc);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        if (lane == 0) {
            mbar_init(&ms->bar_load, 1);
            mbar_init(&ms->bar_u, 1);
            mbar_init(&ms->bar_g, 1);
            mbar_init(&ms->bar_p, kEpiWarps);
            mbar_init(&ms->bar_z0, kEpiWarps);
            mbar_init(&ms->bar_z1, kEpiWarps);
            mbar_init(&ms->bar_y, kStageWarps * 32);
            mbar_init(&ms->bar_drain, 1);
            ms->abort = 0;
            ms->load_failed = 0;
            fence_mbar_init();
        }
        __syncwarp();
        tmem_alloc(&ms->tmem_base, 512);
        tmem_relinquish();
    }
    cta_sync();
    const uint32_t tbase = ms->tmem_base;
    if (warp < kProdWarps) {
        regs_dec<kProdRegs>();
        if (warp == 0)
            mma_role_tv<MX>(L, ms, sm, tbase, smem_u32(sm), lane);
        else
            stage_role<MX>(L, ms, sm, warp - 1, lane);
    } else {
        regs_inc<kEpiRegs>();
        epi_role_tv<MX>(L, ms, sm, tbase, warp, lane);
    }
    cta_sync();
    if (warp == 0) tmem_dealloc(tbase, 512);
}

// Scales of the fp16 operands: max |A|, max_m sum_n |Phi[m][n]| and max |Phi|.
__global__ void k_tc_ranges(const float* __restrict__ a, const float* __restrict__ phi, int n, int m,
                            float* __restrict__ out) {
    __shared__ float red_a[32], red_l[32], red_p[32];
    float amax = 0.f, lmax = 0.f, pmax = 0.f;
    for (int row = threadIdx.x >> 5; row < m; row += blockDim.x >> 5) {
        float l1 = 0.f;
        for (int c = threadIdx.x & 31; c < n; c += 32) {
            amax = fmaxf(amax, fabsf(a[(size_t)row * n + c]));
            l1 += fabsf(phi[(size_t)row * n + c]);
            pmax = fmaxf(pmax, fabsf(phi[(size_t)row * n + c]));
        }
        for (int off = 16; off > 0; off >>= 1) l1 += __shfl_xor_sync(0xffffffffu, l1, off);
        lmax = fmaxf(lmax, l1);
    }
    for (int off = 16; off > 0; off >>= 1) {
        amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, off));
        pmax = fmaxf(pmax, __shfl_xor_sync(0xffffffffu, pmax, off));
    }
    if ((threadIdx.x & 31) == 0) {
        red_a[threadIdx.x >> 5] = amax;
        red_l[threadIdx.x >> 5] = lmax;
        red_p[threadIdx.x >> 5] = pmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float x = 0.f, y = 0.f, z = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            x = fmaxf(x, red_a[w]);
            y = fmaxf(y, red_l[w]);
            z = fmaxf(z, red_p[w]);
        }
        out[0] = x;
        out[1] = y;
        out[2] = z;
    }
}

// The four shared-memory images of A * 2^ea: fp16 hi, fp16 lo, bf16 hi, bf16
// lo, each m16 rows x 256, rows >= M zero, 128-byte swizzled atoms of 8 rows x
// 64 columns (atom (col/64, row/8) at ((col/64) * m16/8 + row/8) * 1024).
__global__ void k_tc_images(const float* __restrict__ a, uint8_t* __restrict__ img, int n, int m,
                            int m16, float scale) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m16 * kN) return;
    const int row = idx / kN, col = idx % kN;
    const float v = row < m ? a[(size_t)row * n + col] * scale : 0.f;
    const uint32_t off = sw128_offset((uint32_t)row, (uint32_t)col, (uint32_t)m16 / 8);
    const size_t img_bytes = (size_t)m16 * kN * 2;
    const __half hh = __float2half_rn(v);
    const __half hl = __float2half_rn(v - __half2float(hh));
    const __nv_bfloat16 bh = __float2bfloat16_rn(v);
    const __nv_bfloat16 bl = __float2bfloat16_rn(v - __bfloat162float(bh));
    *reinterpret_cast<__half*>(img + off) = hh;
    *reinterpret_cast<__half*>(img + img_bytes + off) = hl;
    *reinterpret_cast<__nv_bfloat16*>(img + 2 * img_bytes + off) = bh;
    *reinterpret_cast<__nv_bfloat16*>(img + 3 * img_bytes + off) = bl;
}

int m16_of(int m) { return (m + 15) / 16 * 16; }

}  // namespace

// 16 x 16 blocks on this file's kernel, 32 x 32 blocks on the cluster kernel
bool tc_plan_supported(int n, int m) { return (n == kN || n == 1024) && m >= 1 && m <= kMaxM16; }
size_t tc_operand_bytes(int n, int m) { return 4ull * (size_t)m16_of(m) * (size_t)n * 2; }

cudaError_t launch_tc_ranges(const float* a, const float* phi, int n, int m, float* out,
                             cudaStream_t s) {
    k_tc_ranges<<<1, 1024, 0, s>>>(a, phi, n, m, out);
    return cudaGetLastError();
}

cudaError_t launch_tc_images(const float* a, uint8_t* img, int n, int m, int ea, cudaStream_t s) {
    const int m16 = m16_of(m);
    const int total = m16 * kN;
    k_tc_images<<<(total + 255) / 256, 256, 0, s>>>(a, img, n, m, m16, ldexpf(1.f, ea));
    return cudaGetLastError();
}

bool tc_supported(const cs_plan* plan, int precision) {
    (void)precision;
    return plan->a_tc != nullptr && tc_plan_supported(plan->n, plan->m) &&
           (plan->n != 1024 || plan->ctx->tc8_scratch != nullptr);
}

static void fill_job(const DecodeArgs& d, int tile_begin, TcJob* J, bool* bf) {
    const cs_plan* p = d.plan;
    const GopShape& gs = d.gs;
    *bf = d.precision == CS_BF16 || d.precision == CS_BF16X2;
    const int m16 = m16_of(p->m);
    const size_t img = (size_t)m16 * kN * 2;
    J->a_img = p->a_tc + (*bf ? 2 * img : 0);
    J->y = d.y;
    J->keys = d.key;
    J->out_f32 = d.out_f32;
    J->out_u8 = d.out_u8;
    J->dct = p->dct;
    J->gs = gs;
    J->rows = (long long)gs.n_cs * gs.nblk;
    J->tile_begin = tile_begin;
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

// One launch for up to kMaxJobs jobs of one operand type (fp16 or bf16).  Jobs
// are laid out heaviest first (iterations x work per iteration) so that the
// dynamic tile order approximates longest-processing-time scheduling.
template <bool BF, int MX>
static cudaError_t launch_kernel(const TcLaunch& L, int grid, cudaStream_t s) {
    const void* fn = (const void*)k_fista_tc<BF, MX>;
    // The epilogue warpgroups' setmaxnreg.inc draws on the registers the CTA was
    // launched with: never launch unless that allocation covers the split.
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    if (fa.numRegs < kLaunchRegs || fa.maxThreadsPerBlock < kThreads)
        return cudaErrorInvalidConfiguration;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Lay<MX>::kSmemBytes);
    if (e != cudaSuccess) return e;
    k_fista_tc<BF, MX><<<grid, kThreads, Lay<MX>::kSmemBytes, s>>>(L);
    return cudaGetLastError();
}

// One launch for up to kMaxJobs jobs of one operand type (fp16 or bf16) and
// one layout (M16 <= mx).  Jobs are laid out heaviest first (iterations x
// work per iteration) so that the dynamic tile order approximates
// longest-processing-time scheduling.
static cudaError_t launch_group(const DecodeArgs* const* jobs, int n_jobs, bool bf, int mx,
                                cudaStream_t s) {
    TcLaunch L{};
    L.beta = jobs[0]->beta;
    L.err = jobs[0]->plan->ctx->err_dev;
    cs_ctx* ctx = jobs[0]->plan->ctx;
    std::lock_guard<std::mutex> lock(ctx->launch_mu);
    int cslot = 0;
    cudaError_t e = slot_take(&ctx->counter_ring, s, &cslot);
    if (e != cudaSuccess) return e;
    L.tile_counter = ctx->counters_dev + cslot;
    L.drop_arrival = ctx->debug_flags.exchange(0) & CS_DEBUG_DROP_ARRIVAL;
    e = cudaMemsetAsync(L.tile_counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    int tiles = 0;
    for (int i = 0; i < n_jobs; ++i) {
        bool jbf = false;
        fill_job(*jobs[i], tiles, &L.jobs[i], &jbf);
        tiles += (int)((L.jobs[i].rows + kTile - 1) / kTile);
    }
    L.n_jobs = n_jobs;
    L.n_tiles = tiles;
    const int sms = ctx->sm_count;
    const int grid = tiles < sms ? tiles : sms;
    if (mx <= 96) e = bf ? launch_kernel<true, 96>(L, grid, s) : launch_kernel<false, 96>(L, grid, s);
    else e = bf ? launch_kernel<true, 128>(L, grid, s) : launch_kernel<false, 128>(L, grid, s);
    if (e != cudaSuccess) return e;
    return slot_done(&ctx->counter_ring, cslot, s);
}

static double job_cost(const DecodeArgs& d) {
    const bool mixed = d.precision == CS_BF16 || d.precision == CS_FP16;
    const double split_iters = mixed ? (double)(d.tail_iters < d.iters ? d.tail_iters : d.iters)
                                     : (double)d.iters;
    const double m16 = (double)m16_of(d.plan->m);
    // per iteration: 16 GEMM1 steps + m16/16 GEMM2 steps, x3 when split, plus the epilogue
    const double per = 16.0 + m16 / 16.0 + 24.0;
    return (double)d.iters * per + 2.0 * split_iters * (16.0 + m16 / 16.0);
}

cudaError_t launch_decode_tc_batch(const DecodeArgs* jobs, int n_jobs, cudaStream_t s) {
    // groups by operand type and shared-memory layout (M16 <= 96: more of the
    // momentum state in shared memory, no register spills)
    std::vector<const DecodeArgs*> groups[2][2];
    std::vector<DecodeArgs> big;   // 32 x 32 blocks: the cluster kernel
    for (int i = 0; i < n_jobs; ++i) {
        if (jobs[i].plan->n != kN) {
            big.push_back(jobs[i]);
            continue;
        }
        if ((long long)jobs[i].gs.n_cs * jobs[i].gs.nblk == 0) continue;
        const bool bf = jobs[i].precision == CS_BF16 || jobs[i].precision == CS_BF16X2;
        const bool wide = m16_of(jobs[i].plan->m) > 96;
        groups[bf ? 1 : 0][wide ? 1 : 0].push_back(&jobs[i]);
    }
    struct Launch {
        const DecodeArgs* const* jobs;
        int n;
        bool bf;
        int mx;
    };
    std::vector<Launch> launches;
    for (int bf = 0; bf < 2; ++bf)
        for (int w = 1; w >= 0; --w) {
            std::vector<const DecodeArgs*>& g = groups[bf][w];
            std::stable_sort(g.begin(), g.end(), [](const DecodeArgs* a, const DecodeArgs* b) {
                return job_cost(*a) > job_cost(*b);
            });
            for (size_t i = 0; i < g.size(); i += kMaxJobs)
                launches.push_back({g.data() + i, (int)std::min(g.size() - i, (size_t)kMaxJobs),
                                    bf == 1, w ? 128 : 96});
        }
    cudaError_t e = cudaSuccess;
    if (launches.size() <= 1) {
        if (!launches.empty())
            e = launch_group(launches[0].jobs, launches[0].n, launches[0].bf, launches[0].mx, s);
    } else {
        // several persistent launches: fork them onto the context's own streams so
        // that one's tail overlaps the next one's start, then join on s
        cs_ctx* ctx = jobs[0].plan->ctx;
        cudaEvent_t fork = nullptr;
        e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(fork, s);
        std::vector<cudaEvent_t> joins;
        for (size_t i = 0; e == cudaSuccess && i < launches.size(); ++i) {
            cudaStream_t fs = i == 0 ? s : fork_stream(ctx, s, (int)((i - 1) % kForkTcGroups));
            if (i > 0) e = cudaStreamWaitEvent(fs, fork, 0);
            if (e == cudaSuccess) e = launch_group(launches[i].jobs, launches[i].n, launches[i].bf,
                                                   launches[i].mx, fs);
            if (e == cudaSuccess && i > 0) {
                cudaEvent_t j = nullptr;
                e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
                if (e == cudaSuccess) e = cudaEventRecord(j, fs);
                if (e == cudaSuccess) joins.push_back(j);
                else if (j) cudaEventDestroy(j);
            }
        }
        for (cudaEvent_t j : joins) {
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, j, 0);
            cudaEventDestroy(j);
        }
        if (fork) cudaEventDestroy(fork);
    }
    if (e == cudaSuccess && !big.empty()) e = launch_decode_tc8_batch(big.data(), (int)big.size(), s);
    return e;
}

cudaError_t launch_decode_tc(const DecodeArgs& d, cudaStream_t s) {
    return launch_decode_tc_batch(&d, 1, s);
}

bool tv_tc_supported(const cs_plan* plan) {
    const cs_ctx* ctx = plan->ctx;
    return plan->n == kN && plan->phi_tc != nullptr && m16_of(plan->m) <= kMaxM16 && ctx->tcs_scratch &&
           (size_t)ctx->sm_count * kTvScrBytes <= tcs_slot_bytes(ctx->sm_count);
}

// TV recovery of one call's blocks on the tensor cores: one persistent launch,
// one CTA per SM, its state in a slot of the context's streaming-decode scratch.
cudaError_t launch_decode_tv_tc(const cs_plan* plan, const GopShape& gs, int iters, float beta, float mu,
                                float alpha, const uint8_t* key, const float* y, float* out_f32,
                                uint8_t* out_u8, cudaStream_t s) {
    cs_ctx* ctx = plan->ctx;
    TcLaunch L{};
    L.err = ctx->err_dev;
    TcJob& J = L.jobs[0];
    J.a_img = plan->phi_tc;   // Phi 2^tc_ephi: fp16 hi, then fp16 lo
    J.y = y;
    J.keys = key;
    J.out_f32 = out_f32;
    J.out_u8 = out_u8;
    J.dct = plan->dct;
    J.gs = gs;
    J.rows = (long long)gs.n_cs * gs.nblk;
    J.tile_begin = 0;
    J.m16 = m16_of(plan->m);
    J.iters = iters;
    J.split_from = 0;
    // P = 2 mu (U - y) - lam in fp16: FISTA's residual scale, halved once more
    // and again for every doubling of mu above 1
    const int ep = plan->tc_ep - 1 - (mu > 1.f ? (int)ceil(log2((double)mu)) : 0);
    J.su = ldexpf(1.f, -plan->tc_ephi);
    J.sg = ldexpf(1.f, -(plan->tc_ephi + ep));
    J.sp = ldexpf(1.f, ep);
    J.tv_beta = beta;
    J.tv_mu = mu;
    J.tv_alpha = alpha;
    L.n_jobs = 1;
    L.n_tiles = (int)((J.rows + kTile - 1) / kTile);
    const void* fn = (const void*)k_tv_tc<kMaxM16>;
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    if (fa.numRegs < kLaunchRegs || fa.maxThreadsPerBlock < kThreads) return cudaErrorInvalidConfiguration;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTvSmemBytes);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(ctx->launch_mu);
    int cslot = 0, sslot = 0;
    e = slot_take(&ctx->counter_ring, s, &cslot);
    if (e == cudaSuccess) e = slot_take(&ctx->tcs_ring, s, &sslot);
    if (e != cudaSuccess) return e;
    L.tile_counter = ctx->counters_dev + cslot;
    L.scratch = ctx->tcs_scratch + (size_t)sslot * tcs_slot_bytes(ctx->sm_count);
    L.drop_arrival = ctx->debug_flags.exchange(0) & CS_DEBUG_DROP_ARRIVAL;
    e = cudaMemsetAsync(L.tile_counter, 0, sizeof(int), s);
    const int grid = L.n_tiles < ctx->sm_count ? L.n_tiles : ctx->sm_count;
    if (e == cudaSuccess) {
        k_tv_tc<kMaxM16><<<grid, kThreads, kTvSmemBytes, s>>>(L);
        e = cudaGetLastError();
    }
    // the slots are handed back even on failure: whatever was enqueued runs first
    const cudaError_t e1 = slot_done(&ctx->counter_ring, cslot, s);
    const cudaError_t e2 = slot_done(&ctx->tcs_ring, sslot, s);
    return e != cudaSuccess ? e : e1 != cudaSuccess ? e1 : e2;
}

}  // namespace csvc
