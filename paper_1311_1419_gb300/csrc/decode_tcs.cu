// K6 for the (N, M) shapes whose iterates do not fit on one SM: tensor-core
// FISTA with streamed operands and the iterates in global memory.
//
// The recovery is the same fixed-count FISTA on 1/2 ||A s - y||^2 +
// lambda ||s||_1 (Eq. 1 with an l1 regulariser in the DCT basis; Beck &
// Teboulle 2009) followed by r = Psi s and the key add-back of Eq. (4), for
// 8 x 8, 16 x 16 and 32 x 32 blocks (N = 64, 256, 1024) with up to 512
// measurements.  A tile of 128 blocks is one CTA's work (the MMA's M
// dimension).  Per FISTA iteration of a tile, two GEMMs run on the tensor cores:
//
//   GEMM1  U [128 x M16] = Z [128 x N] . A^T   in one or two column chunks of <= 256
//   GEMM2  G [128 x N]   = P [128 x M16] . A   in column chunks of min(N, 256)
//
// Neither A (up to 2 MB as fp16 hi + lo at N = 1024, M = 512) nor the tile's
// iterates (Z and s^{k-1}: 1 MB) fit on chip, so the operands stream: a copy
// warp feeds a two-slot ring of 32-wide K slices (64-byte-swizzled operands,
// 48 KB per slot) through the bulk-copy engine (the tile operand Z or P from
// this CTA's global scratch, the A slice from one of the plan's two swizzled
// images of A, which stay in L2 and make every slice one contiguous copy), one
// thread issues the MMAs into a 256-column accumulator in tensor memory, and
// two CTAs share an SM (half its shared and tensor memory each), so that one
// tile's epilogue, bound by the iterates' global-memory traffic, overlaps the
// other tile's MMAs.  The epilogue (8 warps: TMEM lane quarter = warp % 4, two
// column groups) forms P = U - y (y staged once per tile in the scratch, laid
// out for coalesced reads) into the scratch's P image and runs the gradient /
// soft-threshold / momentum step, reading and writing s^{k-1} (fp32) and Z
// (fp16 hi + lo, the next GEMM1's operand image) in the scratch.  lambda_b needs max |A^T y_b| over all N
// coefficients before the first step, so GEMM2 runs once more at k = 0 for it.
// Mixed precision: a split product uses three MMAs (hi.hi + lo.hi + hi.lo),
// a bulk one hi.hi only.  Every mbarrier wait is bounded and reports through
// the context's error word; a CTA that gives up drains its copies and MMAs.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <vector>

#include "internal.h"
#include "tc_ptx.h"

namespace csvc {
namespace {

using namespace tc;

constexpr int kTile = 128;                 // blocks per tile = TMEM lanes = MMA M
constexpr int kMaxNs = 1024, kMaxM16s = 512;
constexpr int kEpiWarps = 8;                // 4 TMEM lane quarters x 2 column groups
constexpr int kColGroups = kEpiWarps / 4;
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kThreads = 64 + kEpiThreads;  // warp 0 MMA, warp 1 copies, warps 2 .. 9 epilogue
constexpr int kCtasPerSm = 2;               // two tiles per SM: one's epilogue overlaps the other's MMAs
constexpr int kChunk = 256;                 // accumulator columns per chunk (the CTA's TMEM)
constexpr int kSliceK = 32;                 // K per ring slot: one 64-byte swizzle atom
constexpr uint32_t kTBytes = kTile * 64;    // one K slice of the tile operand (8 KB)
constexpr uint32_t kBBytes = kChunk * 64;   // one K slice of up to 256 rows of A (16 KB)
constexpr int kStages = 2;
constexpr uint32_t kStageBytes = 2 * (kTBytes + kBBytes);   // hi and lo of both: 48 KB
constexpr uint32_t kOffC = kStages * kStageBytes;           // DCT matrix, <= 32 x 32 floats
constexpr uint32_t kOffMisc = kOffC + 4096;
constexpr uint32_t kSmemBytes = kOffMisc + 1024 + 1024;     // + alignment slack
// per-CTA global scratch: Z image (hi, lo), P image (hi, lo), s^{k-1}, the tile's y
constexpr size_t kScrZ = 0, kScrP = 512 * 1024, kScrS = 768 * 1024, kScrY = 1280 * 1024,
                 kScrBytes = 1536 * 1024;
constexpr uint64_t kWaitNs = 1000000000ull;                 // 1 s per wait
constexpr uint32_t kBarEpi = 1;                             // named barrier of the epilogue



}  // namespace

// One job of a launch: the blocks of one cs_decode_gop call.
struct TcsJob {
    const uint8_t* a1_img;  // GEMM1's image of A * 2^ea: hi then lo, m16 x n x 2 bytes each
    const uint8_t* a2_img;  // GEMM2's image: hi then lo, m32 x n x 2 bytes each
    const float* y;
    const uint8_t* keys;
    float* out_f32;
    uint8_t* out_u8;
    const float* dct;       // [B][B]
    GopShape gs;
    long long row0;         // first measured block of this launch's share of the call
    long long rows;         // end (exclusive) of that share
    int tile_begin;
    int n, m16;
    int iters;
    int split_from;         // iterations k >= split_from use the 3-MMA split
    int y_vec;              // rows of y start on 16-byte boundaries
    float lambda_rel, inv_l;
    float su, sg, sp;       // U = acc su, G = acc sg, P operand = P sp
};

// The device work queue of the serving path (see TcsQueue below): one entry per
// tile, published by the host in any order; a CTA claims position h once its
// entry's seq reads h + 1.
constexpr int kQJobs = 64;
constexpr int kQRing = 16384;
struct QEntry {
    unsigned long long seq;  // position + 1 once published (0: empty)
    int job;                 // job slot
    int tile;                // tile of the job
};
struct QJob {
    TcsJob job;
    unsigned int done_target;  // the slot's cumulative tile count when this job is done
    unsigned int seq;          // written to done_seq[slot] by the job's last tile
};
// Host-mapped (pinned) memory: the host writes jobs and entries, the CTAs claim
// positions (system-scope CAS on head) and report finished jobs.
struct QShared {
    unsigned long long head;   // next position to claim
    int closing;               // set by a CTA that found nothing to do for the idle limit
    int pad;
    unsigned int done_seq[kQJobs];
    QJob jobs[kQJobs];
    QEntry ring[kQRing];
};

constexpr int kMaxJobsS = 48;
struct TcsLaunch {
    const float* beta;
    int* err;
    int* tile_counter;
    QShared* q;               // non-null: take tiles from the device work queue
    unsigned int* q_done;     // per job slot, tiles finished (cumulative), device memory
    unsigned long long q_idle_ns;
    uint8_t* scratch;       // this launch's area: gridDim.x x kScrBytes
    int drop_arrival;       // test hook: CTA 0 withholds one epilogue warp's first P-ready arrival
    int n_jobs;
    int n_tiles;
    TcsJob jobs[kMaxJobsS];
};

namespace {

struct MiscS {
    uint64_t full[kStages], empty[kStages];
    uint64_t acc_full, acc_empty;
    uint64_t p_ready, z_ready, drain;
    uint32_t tmem_base;
    int abort;
    int next_tile;          // >= 0: a tile was claimed; -1: no more tiles
    int qjob;               // device-queue job slot of the claimed tile (-1: a launch's own job)
    long long tile_in_job;  // the claimed tile's index within its job
    uint32_t q_target, q_seq;
    TcsJob job;             // the claimed tile's job
    uint32_t colmax[kTile];
};
static_assert(sizeof(MiscS) <= 1024, "barrier block");

template <bool BF>
__device__ __forceinline__ uint32_t pack2s(float2 v) {
    if constexpr (BF) {
        __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
        return *reinterpret_cast<uint32_t*>(&h);
    } else {
        __half2 h = __floats2half2_rn(v.x, v.y);
        return *reinterpret_cast<uint32_t*>(&h);
    }
}
template <bool BF>
__device__ __forceinline__ float2 unpack2s(uint32_t v) {
    if constexpr (BF) {
        __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&v);
        return __bfloat1622float2(h);
    } else {
        __half2 h = *reinterpret_cast<__half2*>(&v);
        return __half22float2(h);
    }
}

__device__ __forceinline__ bool wait_s(MiscS* ms, uint64_t* bar, uint32_t parity, int* err) {
    if (*(volatile int*)&ms->abort) return false;
    if (mbar_wait(bar, parity, kWaitNs)) return true;
    *(volatile int*)&ms->abort = 1;
    atomicExch(err, 1);
    return false;
}

__device__ __forceinline__ int job_of_s(const TcsLaunch& L, int tile) {
    int j = 0;
    while (j + 1 < L.n_jobs && L.jobs[j + 1].tile_begin <= tile) ++j;
    return j;
}

__device__ __forceinline__ unsigned long long ld_acquire_sys_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_acquire_sys_s32(const int* p) {
    int v;
    asm volatile("ld.acquire.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys_u32(unsigned int* p, unsigned int v) {
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// The CTA's next tile, claimed by thread 0 and shared through shared memory
// (job descriptor included): from the launch's own jobs by an atomic counter, or
// from the device work queue, waiting (bounded by the idle limit) for the host
// to publish one.  Returns -1 when there is none: every role then leaves.
__device__ __forceinline__ int fetch_tile_s(const TcsLaunch& L, MiscS* ms) {
    if (threadIdx.x == 0) {
        int got = -1;
        if (L.q == nullptr) {
            const int t = atomicAdd(L.tile_counter, 1);
            if (t < L.n_tiles) {
                const int j = job_of_s(L, t);
                ms->job = L.jobs[j];
                ms->tile_in_job = t - L.jobs[j].tile_begin;
                ms->qjob = -1;
                got = 0;
            }
        } else {
            const uint64_t t0 = globaltimer_ns();
            while (!ld_acquire_sys_s32(&L.q->closing)) {
                const unsigned long long h = *(volatile unsigned long long*)&L.q->head;
                const QEntry* e = &L.q->ring[h % kQRing];
                if (ld_acquire_sys_u64(&e->seq) == h + 1) {
                    // read the entry before claiming it: once claimed, the host may
                    // reuse it for position h + kQRing
                    const int js = *(volatile const int*)&e->job;
                    const int tl = *(volatile const int*)&e->tile;
                    if (atomicCAS_system(&L.q->head, h, h + 1) == h) {
                        const QJob& qj = L.q->jobs[js];
                        ms->job = qj.job;
                        ms->q_target = qj.done_target;
                        ms->q_seq = qj.seq;
                        ms->tile_in_job = tl;
                        ms->qjob = js;
                        got = 0;
                        break;
                    }
                    continue;   // another CTA took it: look again at once
                }
                if (globaltimer_ns() - t0 > L.q_idle_ns) {
                    // idle for the limit: close the launch (every CTA leaves; tiles
                    // published from now on wait for the host's next launch)
                    atomicCAS_system(&L.q->closing, 0, 1);
                    break;
                }
                __nanosleep(1000);
            }
        }
        ms->next_tile = got;
    }
    __syncthreads();
    return ms->next_tile;
}

// After a queue tile's outputs are written: count it, and let the job's last
// tile tell the host (outputs first visible, then the job's sequence number).
__device__ __forceinline__ void finish_tile_s(const TcsLaunch& L, MiscS* ms) {
    if (threadIdx.x == 0 && ms->qjob >= 0) {
        __threadfence_system();
        const unsigned int done = atomicAdd(&L.q_done[ms->qjob], 1u) + 1u;
        if (done == ms->q_target) st_release_sys_u32(&L.q->done_seq[ms->qjob], ms->q_seq);
    }
}
__device__ __forceinline__ void cta_sync_s() {
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
}

// Chunk geometry.  GEMM1: U in one chunk of m16 columns, or two of about m16 / 2
// (multiples of 16).  GEMM2: G in n / nc chunks of nc = min(n, 256) columns.
__device__ __forceinline__ int g1_chunks(int m16) { return m16 > kChunk ? 2 : 1; }
__device__ __forceinline__ int g1_width(int m16, int c) {
    if (m16 <= kChunk) return m16;
    const int w0 = (m16 / 2 + 15) / 16 * 16;
    return c == 0 ? w0 : m16 - w0;
}
__device__ __forceinline__ int g1_base(int m16, int c) { return c == 0 ? 0 : g1_width(m16, 0); }
__device__ __forceinline__ int g2_width(int n) { return n < kChunk ? n : kChunk; }
__device__ __forceinline__ int p_slices(int m16) { return (m16 + kSliceK - 1) / kSliceK; }

// Passes of a tile with K iterations: 0 = GEMM2 for lambda, 1 = GEMM2 of k = 0,
// then GEMM1 (even) and GEMM2 (odd) of k = pass / 2.
__device__ __forceinline__ bool pass_is_g2(int pass) { return pass < 2 || (pass & 1); }
__device__ __forceinline__ int pass_iter(int pass) { return pass < 2 ? 0 : pass / 2; }

// Index (in float4) of s^{k-1} values 4 v .. 4 v + 3 of the column group cg of
// GEMM2 chunk jc for tile row r: each epilogue warp reads 512 contiguous bytes.
__device__ __forceinline__ size_t s_index4(int jc, int cg, int v, int r, int nc) {
    return ((size_t)(jc * kColGroups + cg) * (nc / (4 * kColGroups)) + v) * kTile + r;
}

// ---------------------------------------------------------------------------
// Warp 1: streams the operands of every pass into the stage ring.
template <bool BF>
__device__ __forceinline__ void copy_role(const TcsLaunch& L, MiscS* ms, uint8_t* sm, int lane) {
    uint8_t* scr = L.scratch + (size_t)blockIdx.x * kScrBytes;
    uint32_t st = 0, pc = 0, zc = 0;
    uint32_t last_par[kStages] = {};
    bool issued[kStages] = {};
    bool ok = true;
    for (;;) {
        const int tile = fetch_tile_s(L, ms);
        if (tile < 0) break;
        const TcsJob& J = ms->job;
        cta_sync_s();   // B
        const int n = J.n, m16 = J.m16;
        const size_t img1 = (size_t)m16 * n * 2, img2 = (size_t)((m16 + 31) / 32 * 32) * n * 2;
        const uint8_t* z_hi = scr + kScrZ;
        const uint8_t* z_lo = z_hi + (size_t)n * 256;
        const uint8_t* p_hi = scr + kScrP;
        const uint8_t* p_lo = p_hi + (size_t)p_slices(m16) * kTBytes;
        for (int pass = 0; pass < 2 * J.iters; ++pass) {
            const bool g2 = pass_is_g2(pass);
            const int k = pass_iter(pass);
            const bool split = k >= J.split_from;
            if (pass != 1) {   // P (GEMM2) or Z (GEMM1) written by the epilogue
                if (g2) {
                    ok = wait_s(ms, &ms->p_ready, pc & 1, L.err) && ok;
                    ++pc;
                } else {
                    ok = wait_s(ms, &ms->z_ready, zc & 1, L.err) && ok;
                    ++zc;
                }
            }
            const int nch = g2 ? n / g2_width(n) : g1_chunks(m16);
            const int nst = g2 ? p_slices(m16) : n / kSliceK;
            for (int c = 0; c < nch; ++c) {
                for (int ks = 0; ks < nst; ++ks) {
                    const uint32_t s = st % kStages, par = (st / kStages) & 1;
                    ok = wait_s(ms, &ms->empty[s], par ^ 1, L.err) && ok;
                    if (ok && lane == 0) {
                        uint8_t* stg = sm + s * kStageBytes;
                        const int reps = split ? 2 : 1;
                        // GEMM2: slice ks of P and of A's rows 32 ks .., columns of chunk c
                        // (contiguous in the GEMM2 image); GEMM1: slice ks of Z and of A's
                        // columns 32 ks .., rows of chunk c (contiguous in the GEMM1 image)
                        const uint32_t bbytes = g2 ? (uint32_t)g2_width(n) * 64u
                                                   : (uint32_t)g1_width(m16, c) * 64u;
                        mbar_arrive_expect_tx(&ms->full[s], (uint32_t)reps * (kTBytes + bbytes));
                        for (int h = 0; h < reps; ++h) {
                            uint8_t* t_dst = stg + h * kTBytes;
                            uint8_t* b_dst = stg + 2 * kTBytes + h * kBBytes;
                            if (g2) {
                                const uint8_t* aimg = J.a2_img + (h ? img2 : 0);
                                bulk_g2s(t_dst, (h ? p_lo : p_hi) + (size_t)ks * kTBytes, kTBytes, &ms->full[s]);
                                bulk_g2s(b_dst, aimg + ((size_t)ks * (n / 32) + (size_t)c * (g2_width(n) / 32)) * 2048,
                                         bbytes, &ms->full[s]);
                            } else {
                                const uint8_t* aimg = J.a1_img + (h ? img1 : 0);
                                bulk_g2s(t_dst, (h ? z_lo : z_hi) + (size_t)ks * kTBytes, kTBytes, &ms->full[s]);
                                bulk_g2s(b_dst, aimg + ((size_t)ks * (m16 / 8) + g1_base(m16, c) / 8) * 512,
                                         bbytes, &ms->full[s]);
                            }
                        }
                        last_par[s] = par;
                        issued[s] = true;
                    }
                    __syncwarp();
                    ++st;
                }
            }
        }
        cta_sync_s();   // C
    }
    if (lane == 0) {
        // copies whose consumer gave up may still be in flight (bounded)
        for (int s = 0; s < kStages; ++s)
            if (issued[s]) mbar_wait(&ms->full[s], last_par[s], kWaitNs);
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// Warp 0: issues every MMA (lane 0), chunk by chunk into the two accumulators.
template <bool BF>
__device__ __forceinline__ void mma_role_s(const TcsLaunch& L, MiscS* ms, uint8_t* sm, uint32_t tbase,
                                           int lane) {
    const uint32_t s_base = smem_u32(sm);
    uint32_t st = 0, acc = 0;
    bool ok = true;
    for (;;) {
        const int tile = fetch_tile_s(L, ms);
        if (tile < 0) break;
        const TcsJob& J = ms->job;
        cta_sync_s();   // B
        const int n = J.n, m16 = J.m16;
        for (int pass = 0; pass < 2 * J.iters; ++pass) {
            const bool g2 = pass_is_g2(pass);
            const bool split = pass_iter(pass) >= J.split_from;
            const int nch = g2 ? n / g2_width(n) : g1_chunks(m16);
            const int nst = g2 ? p_slices(m16) : n / kSliceK;
            for (int c = 0; c < nch; ++c) {
                ok = wait_s(ms, &ms->acc_empty, (acc & 1) ^ 1, L.err) && ok;
                fence_after_sync();
                const uint32_t d = tbase;
                const int width = g2 ? g2_width(n) : g1_width(m16, c);
                const uint32_t id = idesc_f16(128, (uint32_t)width, BF ? 1u : 0u, 0u, g2 ? 1u : 0u);
#pragma unroll 1
                for (int ks = 0; ks < nst; ++ks) {
                    const uint32_t s = st % kStages, par = (st / kStages) & 1;
                    ok = wait_s(ms, &ms->full[s], par, L.err) && ok;
                    fence_after_sync();
                    if (ok && lane == 0) {
                        const uint32_t stg = s_base + s * kStageBytes;
                        // K-major operands: 8-row groups 512 bytes apart; GEMM2's A slice
                        // is MN-major: 32-column atoms 2 KB apart, 8-row K groups 512 bytes
                        const uint64_t t_hi = desc_sw64(stg, 16, 512);
                        const uint64_t t_lo = desc_sw64(stg + kTBytes, 16, 512);
                        const uint64_t b_hi = g2 ? desc_sw64(stg + 2 * kTBytes, 2048, 512)
                                                 : desc_sw64(stg + 2 * kTBytes, 16, 512);
                        const uint64_t b_lo = g2 ? desc_sw64(stg + 2 * kTBytes + kBBytes, 2048, 512)
                                                 : desc_sw64(stg + 2 * kTBytes + kBBytes, 16, 512);
                        // K steps of 16 in this slice: 32 bytes along a K-major row; two
                        // 8-row K groups (1 KB) in GEMM2's MN-major A slice
                        const int nk = g2 ? min(2, m16 / 16 - 2 * ks) : 2;
                        for (int kk = 0; kk < nk; ++kk) {
                            const uint32_t to = (uint32_t)kk * 2u;
                            const uint32_t bo = g2 ? (uint32_t)kk * 64u : (uint32_t)kk * 2u;
                            const uint32_t accum = (ks > 0 || kk > 0) ? 1u : 0u;
                            mma_f16(d, t_hi + to, b_hi + bo, id, accum);
                            if (split) {
                                mma_f16(d, t_lo + to, b_hi + bo, id, 1u);
                                mma_f16(d, t_hi + to, b_lo + bo, id, 1u);
                            }
                        }
                        mma_commit(&ms->empty[s]);
                    }
                    __syncwarp();
                    ++st;
                }
                if (ok && lane == 0) mma_commit(&ms->acc_full);
                __syncwarp();
                ++acc;
            }
        }
        cta_sync_s();   // C: the epilogue has written the tile's outputs
        finish_tile_s(L, ms);
    }
    if (lane == 0) {
        // every MMA issued so far has completed before tensor memory is freed
        mma_commit(&ms->drain);
        mbar_wait(&ms->drain, 0, kWaitNs);
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// Epilogue pieces.  Thread: TMEM lane / tile row r = 32 q + lane, column
// group cg of the chunk.

// P = (U su - y) sp for the thread's columns of GEMM1 chunk c (U = 0 at k = 0),
// written as fp16/bf16 hi (and lo) into the scratch's P image.  Columns go in
// groups of 16: the group's y values (from the staged copy: 4 measurements of
// 128 rows per 2 KB, so a warp reads 512 contiguous bytes) and accumulator
// columns are requested together.
template <bool BF>
__device__ __forceinline__ void epi_residual(const TcsJob& J, uint8_t* __restrict__ p_hi, uint8_t* __restrict__ p_lo,
                                             uint32_t lane_addr, int c, int cg, int r,
                                             const float4* __restrict__ y4, bool use_u, bool split) {
    const int w4 = g1_width(J.m16, c) / kColGroups;
    const int i0 = g1_base(J.m16, c) + cg * w4;
    for (int c0 = 0; c0 < w4; c0 += 16) {
        uint32_t u[4][4];
        float4 yv[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
#pragma unroll
            for (int e = 0; e < 4; ++e) u[t][e] = 0u;
            if (use_u && c0 + 4 * t < w4) tmem_ld4(lane_addr + (uint32_t)(cg * w4 + c0 + 4 * t), u[t]);
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
            const uint32_t h0 = pack2s<BF>(make_float2(p[0], p[1])), h1 = pack2s<BF>(make_float2(p[2], p[3]));
            const uint32_t off = sw64_offset((uint32_t)r, (uint32_t)i, kTile / 8);
            *reinterpret_cast<uint2*>(p_hi + off) = make_uint2(h0, h1);
            if (split) {
                const float2 d0 = unpack2s<BF>(h0), d1 = unpack2s<BF>(h1);
                const uint32_t l0 = pack2s<BF>(make_float2(p[0] - d0.x, p[1] - d0.y));
                const uint32_t l1 = pack2s<BF>(make_float2(p[2] - d1.x, p[3] - d1.y));
                *reinterpret_cast<uint2*>(p_lo + off) = make_uint2(l0, l1);
            }
        }
    }
}

// lambda pass: max |G| over the thread's columns of GEMM2 chunk jc.
__device__ __forceinline__ float epi_gmax(uint32_t lane_addr, int w, int cg, float mx) {
    for (int c0 = 0; c0 < w; c0 += 16) {
        uint32_t g0[8], g1[8];
        tmem_ld8(lane_addr + (uint32_t)(cg * w + c0), g0);
        tmem_ld8(lane_addr + (uint32_t)(cg * w + c0 + 8), g1);
        tmem_wait_ld();
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            mx = fmaxf(mx, fabsf(__uint_as_float(g0[e])));
            mx = fmaxf(mx, fabsf(__uint_as_float(g1[e])));
        }
    }
    return mx;
}

// Gradient step, soft threshold and momentum for the thread's columns of GEMM2
// chunk jc: s^k = soft(z^k - g / L, tau), z^{k+1} = s^k + beta_k (s^k - s^{k-1}).
// 16 coefficients at a time: their z (hi, lo) and s^{k-1} are requested
// together (eight independent 16-byte loads per round trip).
struct UpdIn {
    uint4 zh[2], zl[2];
    float4 sp[4];
};
template <bool BF>
__device__ __forceinline__ void epi_update(const TcsJob& J, uint8_t* __restrict__ scr, uint32_t lane_addr,
                                           int jc, int cg, int r, int k, float tau, float bk, bool want_z) {
    const int n = J.n, nc = g2_width(n), w = nc / kColGroups;
    uint8_t* __restrict__ z_hi = scr + kScrZ;
    uint8_t* __restrict__ z_lo = z_hi + (size_t)n * 256;
    float4* __restrict__ s4 = reinterpret_cast<float4*>(scr + kScrS);
    const float2 ginv2 = make_float2(-J.sg * J.inv_l, -J.sg * J.inv_l);
    const float2 b2 = make_float2(bk, bk);
    const int jb = jc * nc + cg * w;                                   // the thread's first coefficient
    auto load_in = [&](int c0, UpdIn& in) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t zoff = sw64_offset((uint32_t)r, (uint32_t)(jb + c0 + 8 * h), kTile / 8);
            in.zh[h] = *reinterpret_cast<const uint4*>(z_hi + zoff);
            in.zl[h] = *reinterpret_cast<const uint4*>(z_lo + zoff);
        }
        const size_t si = s_index4(jc, cg, c0 / 4, r, nc);
#pragma unroll
        for (int v = 0; v < 4; ++v) in.sp[v] = ld_stream4(s4 + si + (size_t)v * kTile);   // past L1
    };
    for (int c0 = 0; c0 < w; c0 += 16) {
        uint32_t g[2][8];
        tmem_ld8(lane_addr + (uint32_t)(cg * w + c0), g[0]);
        tmem_ld8(lane_addr + (uint32_t)(cg * w + c0 + 8), g[1]);
        UpdIn cur;
        if (k > 0) {
            load_in(c0, cur);
        } else {
#pragma unroll
            for (int h = 0; h < 2; ++h) cur.zh[h] = cur.zl[h] = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
            for (int v = 0; v < 4; ++v) cur.sp[v] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        tmem_wait_ld();
        const size_t si = s_index4(jc, cg, c0 / 4, r, nc);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t zhw[4] = {cur.zh[h].x, cur.zh[h].y, cur.zh[h].z, cur.zh[h].w};
            const uint32_t zlw[4] = {cur.zl[h].x, cur.zl[h].y, cur.zl[h].z, cur.zl[h].w};
            const float4 sa = cur.sp[2 * h], sb = cur.sp[2 * h + 1];
            const float spv[8] = {sa.x, sa.y, sa.z, sa.w, sb.x, sb.y, sb.z, sb.w};
            float sv[8];
            uint32_t nh[4], nl[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float2 zhf = unpack2s<BF>(zhw[e]), zlf = unpack2s<BF>(zlw[e]);
                const float2 z2 = make_float2(zhf.x + zlf.x, zhf.y + zlf.y);
                const float2 v = fma2(make_float2(__uint_as_float(g[h][2 * e]), __uint_as_float(g[h][2 * e + 1])),
                                      ginv2, z2);
                const float2 cl = make_float2(fminf(fmaxf(v.x, -tau), tau), fminf(fmaxf(v.y, -tau), tau));
                const float2 s2 = sub2(v, cl);
                const float2 zn = fma2(b2, sub2(s2, make_float2(spv[2 * e], spv[2 * e + 1])), s2);
                sv[2 * e] = s2.x;
                sv[2 * e + 1] = s2.y;
                nh[e] = pack2s<BF>(zn);
                nl[e] = pack2s<BF>(sub2(zn, unpack2s<BF>(nh[e])));
            }
            s4[si + (size_t)(2 * h) * kTile] = make_float4(sv[0], sv[1], sv[2], sv[3]);
            s4[si + (size_t)(2 * h + 1) * kTile] = make_float4(sv[4], sv[5], sv[6], sv[7]);
            if (want_z) {
                const uint32_t zoff = sw64_offset((uint32_t)r, (uint32_t)(jb + c0 + 8 * h), kTile / 8);
                *reinterpret_cast<uint4*>(z_hi + zoff) = make_uint4(nh[0], nh[1], nh[2], nh[3]);
                *reinterpret_cast<uint4*>(z_lo + zoff) = make_uint4(nl[0], nl[1], nl[2], nl[3]);
            }
        }
    }
}

// Wait for accumulator chunk `acc`, then (after the caller has read it) give
// it back to the MMA warp.
__device__ __forceinline__ void acc_wait(const TcsLaunch& L, MiscS* ms, uint32_t acc) {
    wait_s(ms, &ms->acc_full, acc & 1, L.err);
    fence_after_sync();
}
__device__ __forceinline__ void acc_release(MiscS* ms, uint32_t acc, int lane) {
    fence_before_sync();
    __syncwarp();
    if (lane == 0) mbar_arrive(&ms->acc_empty);
}
// The epilogue's global writes of an operand image are complete: let the copy warp read it.
__device__ __forceinline__ void signal_copy(uint64_t* bar, int lane, bool withhold = false) {
    fence_proxy_async_global();
    __syncwarp();
    if (lane == 0 && !withhold) mbar_arrive(bar);
}

// Warps 2 .. 17.
template <bool BF>
__device__ __forceinline__ void epi_role_s(const TcsLaunch& L, MiscS* ms, uint8_t* sm, uint32_t tbase, int warp,
                                           int lane) {
    const int ew = warp - 2, q = warp & 3, cg = ew >> 2;
    const int r = 32 * q + lane;                      // TMEM lane = tile row
    const int et = threadIdx.x - 64;                  // 0 .. kEpiThreads - 1
    const uint32_t lane_addr = tbase + ((uint32_t)(32 * q) << 16);
    uint8_t* scr = L.scratch + (size_t)blockIdx.x * kScrBytes;
    float* c_s = reinterpret_cast<float*>(sm + kOffC);
    uint32_t acc = 0;
    bool first_tile = true;
    for (;;) {
        const int tile = fetch_tile_s(L, ms);
        if (tile < 0) break;
        const TcsJob& J = ms->job;
        const GopShape& gs = J.gs;
        const int n = J.n, m16 = J.m16, K = J.iters;
        const int bsz = gs.b;
        if (cg == 0) ms->colmax[r] = 0u;
        for (int i = et; i < bsz * bsz; i += kEpiThreads) c_s[i] = J.dct[i];
        cta_sync_s();   // B
        const long long tile_row0 = J.row0 + ms->tile_in_job * kTile;
        uint8_t* p_hi = scr + kScrP;
        uint8_t* p_lo = p_hi + (size_t)p_slices(m16) * kTBytes;
        float4* y4 = reinterpret_cast<float4*>(scr + kScrY);
        const int nch2 = n / g2_width(n), w2 = g2_width(n) / kColGroups;
        if (K > 0) {
            // the tile's y, read once (coalesced) and stored as [m16 / 4][128 rows] float4,
            // zero beyond M and beyond the call's last block
            {
                const int m = gs.m;
                const long long rows_left = J.rows - tile_row0;
                float* yf = reinterpret_cast<float*>(y4);
                const float* src = J.y + tile_row0 * m;
                for (int q = et; q < kTile * m16; q += kEpiThreads) {
                    const int rr = q / m16, i = q % m16;
                    const float v = (i < m && rr < rows_left) ? src[(size_t)rr * m + i] : 0.f;
                    yf[((size_t)(i / 4) * kTile + rr) * 4 + (i & 3)] = v;
                }
                __threadfence_block();
                named_sync(kBarEpi, kEpiThreads);
            }
            const bool split0 = 0 >= J.split_from;
            // P = -y for GEMM2 of k = 0 (z = 0, so U = 0)
            for (int c = 0; c < g1_chunks(m16); ++c)
                epi_residual<BF>(J, p_hi, p_lo, lane_addr, c, cg, r, y4, false, split0);
            // (the test hook withholds one warp's arrival in CTA 0: the copy warp's
            // bounded wait then gives up and the CTA drains)
            signal_copy(&ms->p_ready, lane, L.drop_arrival && blockIdx.x == 0 && ew == 1 && first_tile);
            // lambda_b = lambda_rel ||A^T y_b||_inf from G = -A^T y
            float mx = 0.f;
            for (int jc = 0; jc < nch2; ++jc, ++acc) {
                acc_wait(L, ms, acc);
                mx = epi_gmax(lane_addr, w2, cg, mx);
                acc_release(ms, acc, lane);
            }
            atomicMax(&ms->colmax[r], __float_as_uint(mx * J.sg));
            named_sync(kBarEpi, kEpiThreads);
            const float tau = J.lambda_rel * __uint_as_float(ms->colmax[r]) * J.inv_l;
            for (int k = 0; k < K; ++k) {
                const bool want_z = k + 1 < K;
                if (k > 0) {
                    const bool split = k >= J.split_from;
                    for (int c = 0; c < g1_chunks(m16); ++c, ++acc) {
                        acc_wait(L, ms, acc);
                        epi_residual<BF>(J, p_hi, p_lo, lane_addr, c, cg, r, y4, true, split);
                        acc_release(ms, acc, lane);
                    }
                    signal_copy(&ms->p_ready, lane);
                }
                const float bk = L.beta[k];
                for (int jc = 0; jc < nch2; ++jc, ++acc) {
                    acc_wait(L, ms, acc);
                    epi_update<BF>(J, scr, lane_addr, jc, cg, r, k, tau, bk, want_z);
                    acc_release(ms, acc, lane);
                }
                if (want_z) signal_copy(&ms->z_ready, lane);
            }
        }
        // --- reconstruct: R = C^T S C per block, S = s^K; 1024 / n blocks at a time ---
        __threadfence_block();
        named_sync(kBarEpi, kEpiThreads);
        float* s_s = reinterpret_cast<float*>(sm);   // stage 0 is idle now
        float* t_s = s_s + 1024;
        const float4* s4 = reinterpret_cast<const float4*>(scr + kScrS);
        const int nc = g2_width(n), w = nc / kColGroups, gb = 1024 / n;
        const size_t frame_px = (size_t)gs.h * gs.w;
        for (int b0 = 0; b0 < kTile; b0 += gb) {
            for (int e = et; e < gb * n; e += kEpiThreads) {
                const int bl = e / n, j = e % n;
                float v = 0.f;
                if (K > 0) {
                    const int jc = j / nc, rem = j % nc, cgj = rem / w, cc = rem % w;
                    const float* f = reinterpret_cast<const float*>(s4 + s_index4(jc, cgj, cc / 4, b0 + bl, nc));
                    v = f[cc % 4];
                }
                s_s[e] = v;
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
        cta_sync_s();   // C
        first_tile = false;
    }
}

template <bool BF>
__global__ void __launch_bounds__(kThreads, kCtasPerSm) k_fista_tcs(const __grid_constant__ TcsLaunch L) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
    MiscS* ms = reinterpret_cast<MiscS*>(sm + kOffMisc);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        if (lane == 0) {
            for (int s = 0; s < kStages; ++s) {
                mbar_init(&ms->full[s], 1);
                mbar_init(&ms->empty[s], 1);
            }
            mbar_init(&ms->acc_full, 1);
            mbar_init(&ms->acc_empty, kEpiWarps);
            mbar_init(&ms->p_ready, kEpiWarps);
            mbar_init(&ms->z_ready, kEpiWarps);
            mbar_init(&ms->drain, 1);
            ms->abort = 0;
            fence_mbar_init();
        }
        __syncwarp();
        tmem_alloc(&ms->tmem_base, kChunk);
        tmem_relinquish();
    }
    cta_sync_s();
    const uint32_t tbase = ms->tmem_base;
    if (warp == 0)
        mma_role_s<BF>(L, ms, sm, tbase, lane);
    else if (warp == 1)
        copy_role<BF>(L, ms, sm, lane);
    else
        epi_role_s<BF>(L, ms, sm, tbase, warp, lane);
    cta_sync_s();
    if (warp == 0) tmem_dealloc(tbase, kChunk);
}

int m16_of_s(int m) { return (m + 15) / 16 * 16; }
int m32_of_s(int m) { return (m + 31) / 32 * 32; }

// The plan's operand images of A * 2^ea for this kernel, in four types each
// (fp16 hi, fp16 lo, bf16 hi, bf16 lo), rows i >= M zero, 64-byte-swizzled atoms
// of 8 rows x 32 columns:
//   GEMM1 image, m16 x n: atom (i / 8, j / 32) at ((j / 32) * m16 / 8 + i / 8) * 512,
//     so a K slice (32 columns j) of any run of rows is contiguous;
//   GEMM2 image, m32 x n: atom (i / 8, j / 32) at (((i / 32) * n / 32 + j / 32) * 4 +
//     (i % 32) / 8) * 512, so a K slice (32 rows i) of any run of 32-column atoms
//     is contiguous (read MN-major: j along the 64-byte rows).
__global__ void k_tcs_images(const float* __restrict__ a, uint8_t* __restrict__ img, int n, int m, int m16,
                             int m32, float scale) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m32 * n) return;
    const int row = idx / n, col = idx % n;
    const float v = row < m ? a[(size_t)row * n + col] * scale : 0.f;
    const __half hh = __float2half_rn(v);
    const __half hl = __float2half_rn(v - __half2float(hh));
    const __nv_bfloat16 bh = __float2bfloat16_rn(v);
    const __nv_bfloat16 bl = __float2bfloat16_rn(v - __bfloat162float(bh));
    const size_t img1 = (size_t)m16 * n * 2, img2 = (size_t)m32 * n * 2;
    if (row < m16) {
        const uint32_t off = sw64_offset((uint32_t)row, (uint32_t)col, (uint32_t)m16 / 8);
        *reinterpret_cast<__half*>(img + off) = hh;
        *reinterpret_cast<__half*>(img + img1 + off) = hl;
        *reinterpret_cast<__nv_bfloat16*>(img + 2 * img1 + off) = bh;
        *reinterpret_cast<__nv_bfloat16*>(img + 3 * img1 + off) = bl;
    }
    const uint32_t r8 = (uint32_t)row & 7, chunk = ((uint32_t)col & 31) >> 3;
    const size_t atom = ((size_t)(row / 32) * (n / 32) + col / 32) * 4 + (row % 32) / 8;
    const size_t off2 = 4 * img1 + atom * 512 + r8 * 64 + ((chunk ^ (r8 >> 1)) << 4) + ((col & 7) << 1);
    *reinterpret_cast<__half*>(img + off2) = hh;
    *reinterpret_cast<__half*>(img + img2 + off2) = hl;
    *reinterpret_cast<__nv_bfloat16*>(img + 2 * img2 + off2) = bh;
    *reinterpret_cast<__nv_bfloat16*>(img + 3 * img2 + off2) = bl;
}

}  // namespace

bool tcs_plan_supported(int n, int m) {
    return (n == 64 || n == 256 || n == kMaxNs) && m >= 1 && m16_of_s(m) <= kMaxM16s;
}
size_t tcs_operand_bytes(int n, int m) {
    return 4ull * (size_t)(m16_of_s(m) + m32_of_s(m)) * (size_t)n * 2;
}
size_t tcs_slot_bytes(int sm_count) {
    return (size_t)(kCtasPerSm * sm_count) * kScrBytes;
}

cudaError_t launch_tcs_images(const float* a, uint8_t* img, int n, int m, int ea, cudaStream_t s) {
    const int m16 = m16_of_s(m), m32 = m32_of_s(m);
    const int total = m32 * n;
    k_tcs_images<<<(total + 255) / 256, 256, 0, s>>>(a, img, n, m, m16, m32, ldexpf(1.f, ea));
    return cudaGetLastError();
}

bool tcs_supported(const cs_plan* plan) {
    return plan->a_tcs != nullptr && plan->ctx->tcs_scratch != nullptr && tcs_plan_supported(plan->n, plan->m);
}

static void fill_job_s(const DecodeArgs& d, int tile_begin, TcsJob* J) {
    const cs_plan* p = d.plan;
    const bool bf = d.precision == CS_BF16 || d.precision == CS_BF16X2;
    const int m16 = m16_of_s(p->m);
    const size_t img1 = (size_t)m16 * p->n * 2, img2 = (size_t)m32_of_s(p->m) * p->n * 2;
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
    J->y_vec = p->m % 4 == 0 && (reinterpret_cast<uintptr_t>(d.y) & 15) == 0;
    J->lambda_rel = d.lambda_rel;
    J->inv_l = (float)(1.0 / p->lipschitz);
    J->su = ldexpf(1.f, -p->tc_ea);
    J->sg = ldexpf(1.f, -(p->tc_ea + p->tc_ep));
    J->sp = ldexpf(1.f, p->tc_ep);
}

static long long job_rows_s(const DecodeArgs& d) {
    const long long total = (long long)d.gs.n_cs * d.gs.nblk;
    return (d.row_end < 0 ? total : d.row_end) - d.row_begin;
}

static double job_cost_s(const DecodeArgs& d) {
    const double m16 = (double)m16_of_s(d.plan->m), n = (double)d.plan->n;
    const double blocks = (double)job_rows_s(d);
    return blocks * (double)d.iters * (m16 > kChunk ? 2.0 * kChunk : m16) * n;
}

// One launch for up to kMaxJobsS jobs of one operand type (fp16 or bf16), any
// (N, M) this kernel supports; jobs heaviest first.
static cudaError_t launch_group_s(const DecodeArgs* const* jobs, int n_jobs, bool bf, cudaStream_t s,
                                  int max_ctas) {
    cs_ctx* ctx = jobs[0]->plan->ctx;
    if (!ctx->tcs_scratch) return cudaErrorInvalidValue;
    TcsLaunch L{};
    L.beta = jobs[0]->beta;
    L.err = ctx->err_dev;
    std::lock_guard<std::mutex> lock(ctx->launch_mu);
    int cslot = 0, sslot = 0;
    cudaError_t e = slot_take(&ctx->counter_ring, s, &cslot);
    if (e == cudaSuccess) e = slot_take(&ctx->tcs_ring, s, &sslot);
    if (e != cudaSuccess) return e;
    L.tile_counter = ctx->counters_dev + cslot;
    L.drop_arrival = ctx->debug_flags.exchange(0) & CS_DEBUG_DROP_ARRIVAL;
    L.scratch = ctx->tcs_scratch + (size_t)sslot * tcs_slot_bytes(ctx->sm_count);
    e = cudaMemsetAsync(L.tile_counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    int tiles = 0;
    for (int i = 0; i < n_jobs; ++i) {
        fill_job_s(*jobs[i], tiles, &L.jobs[i]);
        tiles += (int)((L.jobs[i].rows - L.jobs[i].row0 + kTile - 1) / kTile);
    }
    L.n_jobs = n_jobs;
    L.n_tiles = tiles;
    int grid = std::min(tiles, kCtasPerSm * ctx->sm_count);
    if (max_ctas > 0) grid = std::min(grid, max_ctas);
    const void* fn = bf ? (const void*)k_fista_tcs<true> : (const void*)k_fista_tcs<false>;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    if (bf)
        k_fista_tcs<true><<<grid, kThreads, kSmemBytes, s>>>(L);
    else
        k_fista_tcs<false><<<grid, kThreads, kSmemBytes, s>>>(L);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = slot_done(&ctx->counter_ring, cslot, s);
    if (e == cudaSuccess) e = slot_done(&ctx->tcs_ring, sslot, s);
    return e;
}

int tcs_ctas_per_sm() { return kCtasPerSm; }

cudaError_t launch_decode_tcs_batch(const DecodeArgs* jobs, int n_jobs, cudaStream_t s, int max_ctas) {
    std::vector<const DecodeArgs*> groups[2];
    for (int i = 0; i < n_jobs; ++i) {
        if (job_rows_s(jobs[i]) <= 0) continue;
        const bool bf = jobs[i].precision == CS_BF16 || jobs[i].precision == CS_BF16X2;
        groups[bf ? 1 : 0].push_back(&jobs[i]);
    }
    for (int bf = 0; bf < 2; ++bf) {
        std::vector<const DecodeArgs*>& g = groups[bf];
        std::stable_sort(g.begin(), g.end(), [](const DecodeArgs* a, const DecodeArgs* b) {
            return job_cost_s(*a) > job_cost_s(*b);
        });
        for (size_t i = 0; i < g.size(); i += kMaxJobsS) {
            const int nj = (int)std::min(g.size() - i, (size_t)kMaxJobsS);
            cudaError_t e = launch_group_s(g.data() + i, nj, bf == 1, s, max_ctas);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

cudaError_t launch_decode_tcs(const DecodeArgs& d, cudaStream_t s) { return launch_decode_tcs_batch(&d, 1, s); }

}  // namespace csvc

// ---------------------------------------------------------------------------
// The device work queue of the serving path.  One persistent launch of this
// kernel takes tiles of any admitted request (any N, M this kernel covers, fp16
// operands) as the host publishes them; CTAs that find nothing for
// kQueueIdleNs close the launch, and the host launches it again when work
// arrives.  Ring entries are published from a host callback on the request's
// stream once its inputs are on the device, so requests overlap on the SMs
// tile by tile whatever their size.
namespace csvc {

constexpr unsigned long long kQueueIdleNs = 20000000ull;   // 20 ms

struct TcsQueue {
    QShared* host = nullptr;           // host-mapped; host writes jobs and entries
    QShared* dev = nullptr;            // the same memory's device address
    unsigned int* done_dev = nullptr;  // device: tiles finished per job slot (cumulative)
    unsigned int done_total[kQJobs] = {};
    bool slot_used[kQJobs] = {};
    unsigned int next_seq = 1;
    unsigned long long next_pos = 0;   // next ring position handed out
    cudaStream_t stream = nullptr;     // the persistent launch
    cudaEvent_t running = nullptr;     // recorded after it: complete = not running
    bool launched = false;
};

namespace {
struct PublishArgs {
    QShared* q;
    unsigned long long p0;
    int n, job;
};
// Host callback (no CUDA calls): publish positions p0 .. p0 + n - 1, each entry
// made valid by its sequence number last.
void CUDART_CB publish_cb(void* a) {
    PublishArgs* pa = static_cast<PublishArgs*>(a);
    std::atomic_thread_fence(std::memory_order_acquire);
    for (int i = 0; i < pa->n; ++i) {
        QEntry& e = pa->q->ring[(pa->p0 + i) % kQRing];
        e.job = pa->job;
        e.tile = i;
        __atomic_store_n(&e.seq, pa->p0 + (unsigned long long)i + 1ull, __ATOMIC_RELEASE);
    }
    delete pa;
}
}  // namespace

cudaError_t tcsq_create(cs_ctx* ctx) {
    TcsQueue* q = new (std::nothrow) TcsQueue();
    if (!q) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaHostAlloc(&q->host, sizeof(QShared), cudaHostAllocMapped);
    if (e == cudaSuccess) {
        memset(q->host, 0, sizeof(QShared));
        e = cudaHostGetDevicePointer((void**)&q->dev, q->host, 0);
    }
    if (e == cudaSuccess) e = cudaMalloc(&q->done_dev, sizeof(unsigned int) * kQJobs);
    if (e == cudaSuccess) e = cudaMemset(q->done_dev, 0, sizeof(unsigned int) * kQJobs);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&q->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q->running, cudaEventDisableTiming);
    ctx->tcsq = q;
    return e;
}

void tcsq_destroy(cs_ctx* ctx) {
    TcsQueue* q = ctx->tcsq;
    if (!q) return;
    if (q->host) __atomic_store_n(&q->host->closing, 1, __ATOMIC_RELEASE);
    if (q->stream) {
        cudaStreamSynchronize(q->stream);
        cudaStreamDestroy(q->stream);
    }
    if (q->running) cudaEventDestroy(q->running);
    if (q->done_dev) cudaFree(q->done_dev);
    if (q->host) cudaFreeHost(q->host);
    delete q;
    ctx->tcsq = nullptr;
}

bool tcsq_accepts(const DecodeArgs& d) {
    return d.plan->ctx->tcsq && tcs_supported(d.plan) &&
           (d.precision == CS_FP32 || d.precision == CS_FP16);
}

// Launch the persistent kernel if it is not running and some position handed
// out has not been claimed yet.  Caller holds ctx->mu.
cudaError_t tcsq_kick(cs_ctx* ctx) {
    TcsQueue* q = ctx->tcsq;
    if (q->launched) {
        const cudaError_t st = cudaEventQuery(q->running);
        if (st == cudaErrorNotReady) return cudaSuccess;
        if (st != cudaSuccess) return st;
        q->launched = false;
    }
    const unsigned long long head = __atomic_load_n(&q->host->head, __ATOMIC_ACQUIRE);
    if (head >= q->next_pos) return cudaSuccess;
    __atomic_store_n(&q->host->closing, 0, __ATOMIC_RELEASE);
    TcsLaunch L{};
    L.beta = ctx->beta_dev;
    L.err = ctx->err_dev;
    L.q = q->dev;
    L.q_done = q->done_dev;
    L.q_idle_ns = kQueueIdleNs;
    std::lock_guard<std::mutex> lock(ctx->launch_mu);
    int sslot = 0;
    cudaError_t e = slot_take(&ctx->tcs_ring, q->stream, &sslot);
    if (e != cudaSuccess) return e;
    L.scratch = ctx->tcs_scratch + (size_t)sslot * tcs_slot_bytes(ctx->sm_count);
    e = cudaFuncSetAttribute((const void*)k_fista_tcs<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    k_fista_tcs<false><<<kCtasPerSm * ctx->sm_count, kThreads, kSmemBytes, q->stream>>>(L);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = slot_done(&ctx->tcs_ring, sslot, q->stream);
    if (e == cudaSuccess) e = cudaEventRecord(q->running, q->stream);
    if (e == cudaSuccess) q->launched = true;
    return e;
}

// Post one request's decode: a job slot and ring positions are taken now; the
// entries are published by a host callback on `s` once the work already on `s`
// (the request's copy-in) is done.  Caller holds ctx->mu.  Returns CS_EAGAIN
// when no job slot or ring room is free.
int tcsq_post(cs_ctx* ctx, const DecodeArgs& d, cudaStream_t s, int* slot, unsigned int* seq) {
    TcsQueue* q = ctx->tcsq;
    const long long total = (long long)d.gs.n_cs * d.gs.nblk;
    const int tiles = (int)((total + kTile - 1) / kTile);
    if (tiles <= 0) return fail(CS_EINVAL, "empty request");
    if (tiles > kQRing) return fail(CS_EINVAL, "request larger than the device work queue");
    int js = -1;
    for (int i = 0; i < kQJobs && js < 0; ++i)
        if (!q->slot_used[i]) js = i;
    if (js < 0) return fail(CS_EAGAIN, "no free queue job slot");
    const unsigned long long head = __atomic_load_n(&q->host->head, __ATOMIC_ACQUIRE);
    if (q->next_pos + (unsigned long long)tiles - head > (unsigned long long)kQRing)
        return fail(CS_EAGAIN, "device work queue full");
    QJob& qj = q->host->jobs[js];
    fill_job_s(d, 0, &qj.job);
    q->done_total[js] += (unsigned int)tiles;
    qj.done_target = q->done_total[js];
    qj.seq = q->next_seq++;
    if (q->next_seq == 0) q->next_seq = 1;
    PublishArgs* pa = new (std::nothrow) PublishArgs{q->host, q->next_pos, tiles, js};
    if (!pa) return fail(CS_ENOMEM, "host allocation failed");
    std::atomic_thread_fence(std::memory_order_release);
    cudaError_t e = cudaLaunchHostFunc(s, publish_cb, pa);
    if (e != cudaSuccess) {
        delete pa;
        q->done_total[js] -= (unsigned int)tiles;
        return cuda_fail(e, "queue publish");
    }
    q->slot_used[js] = true;
    q->next_pos += (unsigned long long)tiles;
    *slot = js;
    *seq = qj.seq;
    // the request is posted whatever happens now: a failed launch is retried (and
    // reported) by the next cs_poll
    if (tcsq_kick(ctx) != cudaSuccess) set_error("device work queue: launch failed, retried at the next poll");
    return CS_OK;
}

bool tcsq_done(cs_ctx* ctx, int slot, unsigned int seq) {
    return __atomic_load_n(&ctx->tcsq->host->done_seq[slot], __ATOMIC_ACQUIRE) == seq;
}

void tcsq_release(cs_ctx* ctx, int slot) { ctx->tcsq->slot_used[slot] = false; }

}  // namespace csvc
