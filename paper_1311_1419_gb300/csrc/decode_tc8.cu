// K6 + K7 for 32 x 32 blocks (N = 1024): persistent tcgen05 decode on clusters
// of 8 CTAs.
//
// The same FISTA recovery as the 16 x 16 kernel (Eq. 1 with an l1 regulariser
// in the DCT basis, fixed K, key add-back of Eq. 4), for blocks whose operator
// A = Phi Psi (M x 1024) and iterate state do not fit one SM.  A tile of 128
// blocks is decoded by a cluster of 8 CTAs; CTA q holds coefficients
// 128 q .. 128 q + 127 of every block (rows 4q .. 4q + 3 of the 32 x 32 DCT
// coefficient matrix) and the matching 128 columns of A.  Per iteration:
//
//   GEMM1 (partial)  U_q [128 x M16] = Z_q [128 x 128] . A_q^T   (K = this CTA's coefficients)
//   reduce-scatter   U = sum_q U_q: the measurement rows are split into 8 owner
//                    ranges of whole 8-row groups; every CTA bulk-copies its
//                    partial rows to their owners through distributed shared memory
//   residual         the owner forms P = U - y for its rows and bulk-copies them
//                    into every CTA's P operand (MN-major, so an owner's rows
//                    are one contiguous range)
//   GEMM2            G_q [128 x 128] = P [128 x M16] . A_q
//   gradient step, soft threshold and momentum on the CTA's 128 coefficients;
//   lambda_b needs the max over all 1024 and is exchanged once per tile.
//
// Per CTA: shared memory holds the A_q images (hi, lo), the P operand (hi, lo;
// its slots of other owners' rows double as the staging of outgoing partial
// U), the incoming partial U of this CTA's rows from its 7 peers, the 32 x 32
// DCT and barriers; tensor memory holds G, U, Z hi and Z lo in separate
// columns; each epilogue thread keeps its 32 momentum values in registers.
// The reconstruction all-gathers s^K through a global scratch between two
// cluster barriers, then each CTA rebuilds 16 of the tile's blocks.
// Roles and register split as in the 16 x 16 kernel: warp 0 issues the MMAs
// and the bulk copies, warps 4 .. 19 run the epilogue.  Every mbarrier wait is
// bounded (1 s); a wait that gives up sets the context's error word and every
// role drains through the same control flow.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "cluster_ptx.h"
#include "internal.h"
#include "tc_ptx.h"

namespace csvc {
namespace {

using namespace tc;

constexpr int kCl = 8;                      // CTAs per cluster
constexpr int kN = 1024, kBlk = 32;
constexpr int kW = kN / kCl;                // coefficients per CTA
constexpr int kMaxM16 = 128;
constexpr int kTile = 128;                  // blocks per tile = TMEM lanes
constexpr int kEpiWarps = 16, kEpiThreads = kEpiWarps * 32;
constexpr int kProdWarps = 4;
constexpr int kThreads = (kProdWarps + kEpiWarps) * 32;
constexpr int kLaunchRegs = 96, kProdRegs = 32, kEpiRegs = 112;
static_assert(kProdWarps * 32 * kProdRegs + kEpiThreads * kEpiRegs <= kThreads * kLaunchRegs,
              "register split exceeds the launch allocation");
constexpr int kPerThread = kW / 4;          // coefficients per epilogue thread
constexpr int kMaxOwnerRows = 16;           // at most 2 of the 16 row groups per owner
constexpr uint32_t kBarEpi = 1;
// shared memory
constexpr uint32_t kAImg = kMaxM16 * kW * 2;                // 32 KB per 16-bit image
constexpr uint32_t kPImg = kTile * kMaxM16 * 2;             // 32 KB
constexpr uint32_t kOffAHi = 0, kOffALo = kAImg;
constexpr uint32_t kOffPHi = 2 * kAImg, kOffPLo = kOffPHi + kPImg;
constexpr uint32_t kRecvSlot = kMaxOwnerRows * kTile * 4;   // [row][block] float
constexpr uint32_t kOffRecv = kOffPLo + kPImg;              // 7 slots
constexpr uint32_t kOffOwn = kOffRecv + (kCl - 1) * kRecvSlot;   // own partial of own rows, [row][block]
constexpr uint32_t kOffLam = kOffOwn + kRecvSlot;                 // [7][128] float
constexpr uint32_t kOffC = kOffLam + (kCl - 1) * kTile * 4;       // [32][32] float
constexpr uint32_t kOffRowTab = kOffC + kBlk * kBlk * 4;        // [128] staging offset of row m
constexpr uint32_t kOffMisc = kOffRowTab + kMaxM16 * 4;
constexpr uint32_t kSmemBytes = kOffMisc + 1024 + 1024;
// tensor memory columns
constexpr uint32_t kColG = 0, kColU = 128, kColZHi = 256, kColZLo = 320;
constexpr uint64_t kWaitNs = 1000000000ull;
constexpr uint64_t kDrainNs = 20000000ull;   // inbound copies land within microseconds

struct Misc8 {
    uint64_t bar_load, bar_u, bar_g, bar_stage, bar_urecv, bar_pown, bar_precv, bar_lam, bar_z0,
        bar_z1, bar_drain;
    uint32_t tmem_base;
    int abort;
    int load_failed;
    // parities of the phases the roles would have waited for next (the drain)
    uint32_t ph_urecv_end, ph_precv_end, ph_lam_end;
    uint32_t colmax[kTile];
};
static_assert(sizeof(Misc8) <= 1024, "barrier block");

}  // namespace

// One job of a launch: the blocks of one cs_decode_gop call with 32 x 32 blocks.
struct Tc8Job {
    const uint8_t* a_img;   // 8 slices x (fp16 hi, fp16 lo, bf16 hi, bf16 lo), m16 x 128 each
    const float* y;
    const uint8_t* keys;
    float* out_f32;
    uint8_t* out_u8;
    const float* dct;       // [32][32]
    GopShape gs;
    long long rows;
    int tile_begin;
    int m16;
    int iters;
    int split_from;
    float lambda_rel, inv_l;
    float su, sg, sp;
};

constexpr int kMaxJobs8 = 48;
struct Tc8Launch {
    const float* beta;
    int* err;
    float* scratch;         // [clusters][128][1024] float: s^K of a tile, all-gathered
    int drop_arrival;       // test hook: cluster 0's CTA 0 withholds one partial-U staging arrival
    int n_jobs;
    int n_tiles;
    Tc8Job jobs[kMaxJobs8];
};

namespace {

__device__ __forceinline__ bool wait_bar(Misc8* ms, uint64_t* bar, uint32_t parity, int* err) {
    if (*(volatile int*)&ms->abort) return false;
    if (mbar_wait(bar, parity, kWaitNs)) return true;
    *(volatile int*)&ms->abort = 1;
    atomicExch(err, 1);
    return false;
}
__device__ __forceinline__ void cta_sync() {
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
}

template <bool BF>
__device__ __forceinline__ void issue_gemm1(uint32_t tbase, uint32_t s_base, int m16, int ks0, int nks,
                                            bool split) {
    const uint32_t rg = (uint32_t)(m16 / 8);
    const uint64_t d_hi = desc_sw128(s_base + kOffAHi, 16, 1024);
    const uint64_t d_lo = desc_sw128(s_base + kOffALo, 16, 1024);
    const uint32_t id1 = idesc_f16(128, (uint32_t)m16, BF ? 1u : 0u, 0u, 0u);
#pragma unroll 1
    for (int j = 0; j < nks; ++j) {
        const uint32_t ks = (uint32_t)(ks0 + j);
        const uint32_t n0 = 16 * ks;
        const uint32_t b16 = ((n0 >> 6) * rg * 1024 + ((n0 & 63) >> 4) * 32) >> 4;
        const uint32_t zh = tbase + kColZHi + 8 * ks;
        const uint32_t zl = tbase + kColZLo + 8 * ks;
        mma_f16_tmem_a(tbase + kColU, zh, d_hi + b16, id1, ks != 0);
        if (split) {
            mma_f16_tmem_a(tbase + kColU, zl, d_hi + b16, id1, 1);
            mma_f16_tmem_a(tbase + kColU, zh, d_lo + b16, id1, 1);
        }
    }
}

template <bool BF>
__device__ __forceinline__ void issue_gemm2(uint32_t tbase, uint32_t s_base, int m16, bool split) {
    const uint32_t id2 = idesc_f16(128, kW, BF ? 1u : 0u, 1u, 1u);
#pragma unroll 1
    for (int ks = 0; ks < m16 / 16; ++ks) {
        const uint64_t dp_hi = desc_sw128(s_base + kOffPHi + 4096u * ks, 1024, 2048);
        const uint64_t dp_lo = desc_sw128(s_base + kOffPLo + 4096u * ks, 1024, 2048);
        const uint64_t da_hi = desc_sw128(s_base + kOffAHi + 2048u * ks, (uint32_t)(m16 / 8) * 1024, 1024);
        const uint64_t da_lo = desc_sw128(s_base + kOffALo + 2048u * ks, (uint32_t)(m16 / 8) * 1024, 1024);
        mma_f16(tbase + kColG, dp_hi, da_hi, id2, ks > 0);
        if (split) {
            mma_f16(tbase + kColG, dp_lo, da_hi, id2, 1);
            mma_f16(tbase + kColG, dp_hi, da_lo, id2, 1);
        }
    }
}

__device__ __forceinline__ int job_of8(const Tc8Launch& L, int tile) {
    int j = 0;
    while (j + 1 < L.n_jobs && L.jobs[j + 1].tile_begin <= tile) ++j;
    return j;
}

// Reconstruction shared by all roles: the epilogue writes s^K to the scratch,
// then (after a cluster barrier) rebuilds this CTA's 16 blocks of the tile.
// The other roles only meet the two cluster barriers.
template <bool EPI>
__device__ __forceinline__ void recon(const Tc8Launch& L, const Tc8Job& J, uint8_t* sm, int tile,
                                      uint32_t q, int et, const float2 (&sp)[kPerThread / 2], int blk,
                                      int cgrp) {
    float* scratch = L.scratch + (size_t)cluster_id() * kTile * kN;
    if (EPI) {
        // this thread's coefficients: slices 64 h + 16 cgrp .. + 15, as pairs in sp[]
        float* dst = scratch + (size_t)blk * kN + kW * q;
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int i = 0; i < 8; ++i)
                *reinterpret_cast<float2*>(dst + 64 * h + 16 * cgrp + 2 * i) = sp[8 * h + i];
    }
    cluster_sync();
    if (EPI) {
        const float* c_s = reinterpret_cast<const float*>(sm + kOffC);
        float* t_s = reinterpret_cast<float*>(sm + kOffRecv);      // [8 blocks][32][32]
        const GopShape& gs = J.gs;
        const size_t frame_px = (size_t)gs.h * gs.w;
        const long long tile_row0 = (long long)(tile - J.tile_begin) * kTile;
        for (int pass = 0; pass < 2; ++pass) {
            const int jb = et >> 5, kr = et & 31;                   // block of the pass, row
            const int tb = 16 * (int)q + 8 * pass + jb;             // block of the tile
            const bool act = et < 256;
            if (act) {
                // T[k][:] = S[k][:] C
                const float* srow = scratch + (size_t)tb * kN + kBlk * kr;
                float s_row[kBlk];
#pragma unroll
                for (int l = 0; l < kBlk; ++l) s_row[l] = srow[l];
                for (int jj = 0; jj < kBlk; ++jj) {
                    float acc = 0.f;
#pragma unroll
                    for (int l = 0; l < kBlk; ++l) acc = fmaf(s_row[l], c_s[l * kBlk + jj], acc);
                    t_s[(jb * kBlk + kr) * kBlk + jj] = acc;
                }
            }
            named_sync(kBarEpi, kEpiThreads);
            if (act) {
                // R[p][:] = sum_k C[k][p] T[k][:], p = kr
                const long long row = tile_row0 + tb;
                if (row < J.rows) {
                    const int c_idx = (int)(row / gs.nblk), bl = (int)(row % gs.nblk);
                    const int g_key = c_idx / (gs.g - 1);
                    const int bi = bl / gs.nbc, bj = bl % gs.nbc;
                    const int py = bi * kBlk + kr;
                    if (py < gs.h) {
                        float r[kBlk];
#pragma unroll
                        for (int x = 0; x < kBlk; ++x) r[x] = 0.f;
                        for (int k = 0; k < kBlk; ++k) {
                            const float cv = c_s[k * kBlk + kr];
                            const float* trow = t_s + (jb * kBlk + k) * kBlk;
#pragma unroll
                            for (int x = 0; x < kBlk; ++x) r[x] = fmaf(cv, trow[x], r[x]);
                        }
#pragma unroll
                        for (int x = 0; x < kBlk; ++x) {
                            const int px = bj * kBlk + x;
                            if (px >= gs.w) continue;
                            const size_t off = (size_t)py * gs.w + px;
                            const float v = (float)J.keys[(size_t)g_key * frame_px + off] + r[x];
                            if (J.out_f32) J.out_f32[(size_t)c_idx * frame_px + off] = v;
                            if (J.out_u8)
                                J.out_u8[(size_t)c_idx * frame_px + off] =
                                    (uint8_t)fminf(fmaxf(rintf(v), 0.f), 255.f);
                        }
                    }
                }
            }
            named_sync(kBarEpi, kEpiThreads);
        }
    }
    cluster_sync();   // the scratch and the T staging are free again
}

template <bool BF>
__device__ __forceinline__ void mma_role8(const Tc8Launch& L, Misc8* ms, uint8_t* sm, uint32_t tbase,
                                          uint32_t q, int lane) {
    const uint32_t s_base = smem_u32(sm);
    uint32_t ph_stage = 0, ph_urecv = 0, ph_pown = 0, ph_precv = 0, ph_z0 = 0, ph_z1 = 0, ph_load = 0;
    int cur_job = -1;
    bool ok = true;
    for (int tile = (int)cluster_id(); tile < L.n_tiles; tile += (int)n_clusters()) {
        const int jid = job_of8(L, tile);
        const Tc8Job& J = L.jobs[jid];
        int row0_q, rows_q;
        owner_rows((int)q, J.m16, &row0_q, &rows_q);
        if (jid != cur_job) {
            if (lane == 0) {
                const uint32_t img = (uint32_t)J.m16 * kW * 2;
                const uint8_t* slice = J.a_img + (size_t)q * 4 * img + (BF ? 2 * img : 0);
                mbar_arrive_expect_tx(&ms->bar_load, 2 * img);
                bulk_g2s(sm + kOffAHi, slice, img, &ms->bar_load);
                bulk_g2s(sm + kOffALo, slice + img, img, &ms->bar_load);
            }
            __syncwarp();
            const bool loaded = wait_bar(ms, &ms->bar_load, ph_load, L.err);
            if (!loaded) ms->load_failed = 1;
            ok = loaded && ok;
            ph_load ^= 1;
            cur_job = jid;
        }
        if (J.iters > 0 && ok && lane == 0) {
            // incoming data of iteration 0 and the tile's lambda exchange (armed only
            // while healthy: after a wait gave up, the open phases stay as they are
            // for the drain at the end)
            mbar_arrive_expect_tx(&ms->bar_lam, (kCl - 1) * kTile * 4);
            // a CTA that owns no measurement rows receives no partials: its barrier
            // is never armed (an arming of 0 bytes would complete at once, and two
            // such phases could pass before the epilogue looked)
            if (rows_q > 0) mbar_arrive_expect_tx(&ms->bar_urecv, (uint32_t)((kCl - 1) * rows_q * kTile * 4));
            const uint32_t pb = (uint32_t)((J.m16 - rows_q) * kTile * 2) * (0 >= J.split_from ? 2u : 1u);
            mbar_arrive_expect_tx(&ms->bar_precv, pb);
        }
        __syncwarp();
        cta_sync();   // B: Z = 0 in tensor memory
        if (J.iters > 0 && ok && lane == 0) {
            issue_gemm1<BF>(tbase, s_base, J.m16, 0, 8, 0 >= J.split_from);
            mma_commit(&ms->bar_u);
        }
        __syncwarp();
        for (int k = 0; k < J.iters; ++k) {
            const bool split = k >= J.split_from;
            // partial U of the other owners' rows is staged: send it
            ok = wait_bar(ms, &ms->bar_stage, ph_stage, L.err) && ok;
            ph_stage ^= 1;
            // (lane d - 1 serves peer q + d: the seven peers' copies go out together)
            if (ok && lane < kCl - 1) {
                const uint32_t p = (q + 1u + (uint32_t)lane) % kCl;
                int row0_p, rows_p;
                owner_rows((int)p, J.m16, &row0_p, &rows_p);
                if (rows_p > 0) {
                    const uint32_t half = (uint32_t)rows_p * kTile * 2;   // bytes of each staged half
                    const uint32_t dst = mapa(s_base + kOffRecv + (uint32_t)slot_of((int)q, (int)p) * kRecvSlot, p);
                    const uint32_t rbar = mapa(smem_u32(&ms->bar_urecv), p);
                    bulk_s2peer(dst, s_base + kOffPHi + (uint32_t)row0_p * 256u, half, rbar);
                    bulk_s2peer(dst + half, s_base + kOffPLo + (uint32_t)row0_p * 256u, half, rbar);
                }
            }
            __syncwarp();
            // this CTA's rows have all their partials: arm the next iteration's
            if (rows_q > 0) {
                if (wait_bar(ms, &ms->bar_urecv, ph_urecv, L.err))
                    ph_urecv ^= 1;
                else
                    ok = false;
                if (ok && k + 1 < J.iters && lane == 0)
                    mbar_arrive_expect_tx(&ms->bar_urecv, (uint32_t)((kCl - 1) * rows_q * kTile * 4));
            }
            __syncwarp();
            // this CTA's residual rows are written: broadcast them
            ok = wait_bar(ms, &ms->bar_pown, ph_pown, L.err) && ok;
            ph_pown ^= 1;
            if (ok && lane < kCl - 1 && rows_q > 0) {
                const uint32_t bytes = (uint32_t)rows_q * kTile * 2;
                const uint32_t p = (q + 1u + (uint32_t)lane) % kCl;
                const uint32_t rbar = mapa(smem_u32(&ms->bar_precv), p);
                const uint32_t hi = s_base + kOffPHi + (uint32_t)row0_q * 256u;
                bulk_s2peer(mapa(hi, p), hi, bytes, rbar);
                if (split) {
                    const uint32_t lo = s_base + kOffPLo + (uint32_t)row0_q * 256u;
                    bulk_s2peer(mapa(lo, p), lo, bytes, rbar);
                }
            }
            __syncwarp();
            if (wait_bar(ms, &ms->bar_precv, ph_precv, L.err))
                ph_precv ^= 1;
            else
                ok = false;
            if (ok && k + 1 < J.iters && lane == 0) {
                const uint32_t pb = (uint32_t)((J.m16 - rows_q) * kTile * 2) * (k + 1 >= J.split_from ? 2u : 1u);
                mbar_arrive_expect_tx(&ms->bar_precv, pb);
            }
            __syncwarp();
            fence_after_sync();
            if (ok && lane == 0) {
                issue_gemm2<BF>(tbase, s_base, J.m16, split);
                mma_commit(&ms->bar_g);
            }
            __syncwarp();
            if (k + 1 < J.iters) {
                const bool z_split = k + 1 >= J.split_from;
                ok = wait_bar(ms, &ms->bar_z0, ph_z0, L.err) && ok;
                ph_z0 ^= 1;
                fence_after_sync();
                if (ok && lane == 0) issue_gemm1<BF>(tbase, s_base, J.m16, 0, 4, z_split);
                __syncwarp();
                ok = wait_bar(ms, &ms->bar_z1, ph_z1, L.err) && ok;
                ph_z1 ^= 1;
                fence_after_sync();
                if (ok && lane == 0) {
                    issue_gemm1<BF>(tbase, s_base, J.m16, 4, 4, z_split);
                    mma_commit(&ms->bar_u);
                }
                __syncwarp();
            }
        }
        cta_sync();   // C: the epilogue has waited for the last G
        const float2 none[kPerThread / 2] = {};
        recon<false>(L, J, sm, tile, q, 0, none, 0, 0);
    }
    if (lane == 0) {
        mma_commit(&ms->bar_drain);
        mbar_wait(&ms->bar_drain, 0, kWaitNs);
        if (ms->load_failed) mbar_wait(&ms->bar_load, ph_load ^ 1, kWaitNs);
        ms->ph_urecv_end = ph_urecv;
        ms->ph_precv_end = ph_precv;
    }
    __syncwarp();
}

__device__ __forceinline__ void idle_role8(const Tc8Launch& L, uint8_t* sm, uint32_t q) {
    for (int tile = (int)cluster_id(); tile < L.n_tiles; tile += (int)n_clusters()) {
        const Tc8Job& J = L.jobs[job_of8(L, tile)];
        cta_sync();   // B
        cta_sync();   // C
        const float2 none[kPerThread / 2] = {};
        recon<false>(L, J, sm, tile, q, 0, none, 0, 0);
    }
}

template <bool BF>
__device__ __forceinline__ void epi_role8(const Tc8Launch& L, Misc8* ms, uint8_t* sm, uint32_t tbase,
                                          uint32_t q, int warp, int lane) {
    const uint32_t s_base = smem_u32(sm);
    const int ew = warp - kProdWarps, et = ew * 32 + lane;
    const int qq = warp & 3, cgrp = ew >> 2;                 // TMEM lane quarter = warp % 4
    const int blk = 32 * qq + lane;                          // TMEM lane = block of the tile
    const uint32_t lane_addr = tbase + ((uint32_t)(32 * qq) << 16);
    uint8_t* p_hi = sm + kOffPHi;
    uint8_t* p_lo = sm + kOffPLo;
    const float* recv = reinterpret_cast<const float*>(sm + kOffRecv);
    const float* lam_in = reinterpret_cast<const float*>(sm + kOffLam);
    uint32_t ph_u = 0, ph_g = 0, ph_urecv = 0, ph_lam = 0;
    float2 sp[kPerThread / 2];
    for (int tile = (int)cluster_id(); tile < L.n_tiles; tile += (int)n_clusters()) {
        const Tc8Job& J = L.jobs[job_of8(L, tile)];
        const long long row = (long long)(tile - J.tile_begin) * kTile + blk;
        const bool live = row < J.rows;
        const float* y_row = J.y + (live ? row : 0) * J.gs.m;
        int row0_q, rows_q;
        owner_rows((int)q, J.m16, &row0_q, &rows_q);
        const int per_q = rows_q / 4;                        // own rows of this thread: 0, 2 or 4
        const float2 ginv2 = make_float2(-J.sg * J.inv_l, -J.sg * J.inv_l);
#pragma unroll
        for (int i = 0; i < kPerThread / 2; ++i) sp[i] = make_float2(0.f, 0.f);
        float tau = 0.f;
        {   // Z = 0
            uint32_t zr[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) zr[i] = 0u;
            tmem_st16(lane_addr + kColZHi + 16 * cgrp, zr);
            tmem_st16(lane_addr + kColZLo + 16 * cgrp, zr);
            if (cgrp == 0) ms->colmax[blk] = 0u;
            tmem_wait_st();
        }
        if (et < J.m16) {
            // where row m of the partial U is staged: the own rows in kOffOwn, a
            // peer's in the P slots of its rows (first half hi, the rest lo)
            const int p = owner_of(et, J.m16);
            int row0_p, rows_p;
            owner_rows(p, J.m16, &row0_p, &rows_p);
            const int r = et - row0_p, half = rows_p / 2;
            reinterpret_cast<uint32_t*>(sm + kOffRowTab)[et] =
                (uint32_t)p == q ? kOffOwn + r * 512
                : r < half       ? kOffPHi + row0_p * 256 + r * 512
                                 : kOffPLo + row0_p * 256 + (r - half) * 512;
        }
        cta_sync();   // B
        for (int k = 0; k < J.iters; ++k) {
            const float bk = L.beta[k];
            const bool p_split = k >= J.split_from;
            // this thread's y of the own rows, requested before the waits
            float yv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int m = row0_q + per_q * cgrp + i;
                yv[i] = (i < per_q && live && m < J.gs.m) ? __ldg(y_row + m) : 0.f;
            }
            // --- partial U: keep the own rows, stage the others' for their owners ---
            const bool ok_u = wait_bar(ms, &ms->bar_u, ph_u, L.err);
            ph_u ^= 1;
            fence_after_sync();
            {
                // this thread's quarter of the measurement rows, m = mq cgrp .. mq cgrp + mq - 1,
                // to their owners' staging ([row][block] floats; the own rows to kOffOwn; a
                // peer's rows, first half in P hi's slots of its rows, the rest in P lo's)
                const int mq = J.m16 / 4;
                uint32_t u[32];
                tmem_ld32(lane_addr + kColU + (uint32_t)(mq * cgrp), u);
                tmem_wait_ld();
                if (ok_u) {
                    const uint32_t* tab = reinterpret_cast<const uint32_t*>(sm + kOffRowTab);
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        if (j >= mq) break;
                        *reinterpret_cast<uint32_t*>(sm + tab[mq * cgrp + j] + blk * 4) = u[j];
                    }
                }
            }
            fence_proxy_async_smem();
            fence_before_sync();
            __syncwarp();
            // (the test hook withholds one warp's first arrival in cluster 0's CTA 0:
            // the MMA warp's bounded wait gives up, its peers' waits for its data run
            // out in turn, and every CTA drains)
            const bool withhold = L.drop_arrival && blockIdx.x == 0 && ew == 1 && k == 0 &&
                                  tile == (int)cluster_id();
            if (lane == 0 && !withhold) mbar_arrive(&ms->bar_stage);
            // --- residual rows of this CTA: P = (U su - y) sp ---
            if (rows_q > 0 && wait_bar(ms, &ms->bar_urecv, ph_urecv, L.err)) ph_urecv ^= 1;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (i >= per_q) break;
                const int r = per_q * cgrp + i;
                float u = reinterpret_cast<const float*>(sm + kOffOwn)[r * kTile + blk];
#pragma unroll
                for (int s = 0; s < kCl - 1; ++s) u += recv[(s * kMaxOwnerRows + r) * kTile + blk];
                const float pv = (u * J.su - yv[i]) * J.sp;
                const uint16_t h = pack1<BF>(pv);
                const uint32_t off = p_off((uint32_t)blk, (uint32_t)(row0_q + r));
                *reinterpret_cast<uint16_t*>(p_hi + off) = h;
                if (p_split) *reinterpret_cast<uint16_t*>(p_lo + off) = pack1<BF>(pv - unpack1<BF>(h));
            }
            fence_proxy_async_smem();
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&ms->bar_pown);

            // --- gradient step, soft threshold, momentum ---
            const bool ok_g = wait_bar(ms, &ms->bar_g, ph_g, L.err);
            ph_g ^= 1;
            fence_after_sync();
            if (k == 0) {
                // lambda_b = lambda_rel ||A^T y_b||_inf over all 1024 coefficients;
                // at k = 0, G = -A^T y
                float mx = 0.f;
#pragma unroll
                for (int ch = 0; ch < kPerThread / 8; ++ch) {
                    uint32_t g[8];
                    tmem_ld8(lane_addr + kColG + 64 * (ch >> 1) + 16 * cgrp + 8 * (ch & 1), g);
                    tmem_wait_ld();
#pragma unroll
                    for (int i = 0; i < 8; ++i) mx = fmaxf(mx, fabsf(__uint_as_float(g[i])));
                }
                atomicMax(&ms->colmax[blk], __float_as_uint(mx * J.sg));
                named_sync(kBarEpi, kEpiThreads);
                if (cgrp == 0) {
                    const uint32_t v = ms->colmax[blk];
                    for (int d = 1; d < kCl; ++d) {
                        const uint32_t p = (q + (uint32_t)d) % kCl;
                        const uint32_t dst = s_base + kOffLam +
                                             (uint32_t)(slot_of((int)q, (int)p) * kTile + blk) * 4u;
                        st_async_u32(mapa(dst, p), v, mapa(smem_u32(&ms->bar_lam), p));
                    }
                }
                if (wait_bar(ms, &ms->bar_lam, ph_lam, L.err)) ph_lam ^= 1;
                float lmax = __uint_as_float(ms->colmax[blk]);
#pragma unroll
                for (int s = 0; s < kCl - 1; ++s) lmax = fmaxf(lmax, lam_in[s * kTile + blk]);
                tau = J.lambda_rel * lmax * J.inv_l;
            }
            const bool want_z = k + 1 < J.iters;
            const float2 b2 = make_float2(bk, bk);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
#pragma unroll
                for (int ch = 0; ch < 2; ++ch) {
                    const int o = 64 * h + 16 * cgrp + 8 * ch;        // first coefficient
                    uint32_t g[8], zh[4], zl[4];
                    tmem_ld8(lane_addr + kColG + o, g);
                    tmem_ld4(lane_addr + kColZHi + o / 2, zh);
                    tmem_ld4(lane_addr + kColZLo + o / 2, zl);
                    tmem_wait_ld();
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int si = 8 * h + 4 * ch + e;
                        const float2 zhf = unpack2<BF>(zh[e]), zlf = unpack2<BF>(zl[e]);
                        const float2 z2 = make_float2(zhf.x + zlf.x, zhf.y + zlf.y);
                        const float2 v = fma2(u2f2(g[2 * e], g[2 * e + 1]), ginv2, z2);
                        const float2 cl = make_float2(fminf(fmaxf(v.x, -tau), tau),
                                                      fminf(fmaxf(v.y, -tau), tau));
                        const float2 sv = sub2(v, cl);
                        const float2 zn = fma2(b2, sub2(sv, sp[si]), sv);
                        sp[si] = sv;
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
        cta_sync();   // C
        recon<true>(L, J, sm, tile, q, et, sp, blk, cgrp);
    }
    if (et == 0) ms->ph_lam_end = ph_lam;
}

template <bool BF>
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(kThreads, 1)
    k_fista_tc8(const __grid_constant__ Tc8Launch L) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
    Misc8* ms = reinterpret_cast<Misc8*>(sm + kOffMisc);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t q = cluster_rank();
    if (warp == 0) {
        if (lane == 0) {
            mbar_init(&ms->bar_load, 1);
            mbar_init(&ms->bar_u, 1);
            mbar_init(&ms->bar_g, 1);
            mbar_init(&ms->bar_stage, kEpiWarps);
            mbar_init(&ms->bar_urecv, 1);
            mbar_init(&ms->bar_pown, kEpiWarps);
            mbar_init(&ms->bar_precv, 1);
            mbar_init(&ms->bar_lam, 1);
            mbar_init(&ms->bar_z0, kEpiWarps);
            mbar_init(&ms->bar_z1, kEpiWarps);
            mbar_init(&ms->bar_drain, 1);
            ms->abort = 0;
            ms->load_failed = 0;
            fence_mbar_init();
        }
        __syncwarp();
        tmem_alloc(&ms->tmem_base, 512);
        tmem_relinquish();
    }
    float* c_s = reinterpret_cast<float*>(sm + kOffC);
    for (int i = threadIdx.x; i < kBlk * kBlk; i += kThreads) c_s[i] = L.jobs[0].dct[i];
    cta_sync();
    cluster_sync();   // every CTA's barriers exist before any peer signals them
    const uint32_t tbase = ms->tmem_base;
    if (warp < kProdWarps) {
        regs_dec<kProdRegs>();
        if (warp == 0)
            mma_role8<BF>(L, ms, sm, tbase, q, lane);
        else
            idle_role8(L, sm, q);
    } else {
        regs_inc<kEpiRegs>();
        epi_role8<BF>(L, ms, sm, tbase, q, warp, lane);
    }
    cta_sync();
    cluster_sync();   // every CTA has left its tile loop: no copy is issued from here on
    if (ms->abort) {
        // after a wait gave up, a peer's copy or store issued before that peer
        // stopped may still be landing here: wait (bounded) for this CTA's open
        // inbound phases before any CTA of the cluster leaves
        if (warp == 0 && lane == 0) {
            mbar_wait(&ms->bar_urecv, ms->ph_urecv_end, kDrainNs);
            mbar_wait(&ms->bar_precv, ms->ph_precv_end, kDrainNs);
            mbar_wait(&ms->bar_lam, ms->ph_lam_end, kDrainNs);
        }
        __syncthreads();
    }
    cluster_sync();   // no CTA leaves while a peer may still write its shared memory
    if (warp == 0) tmem_dealloc(tbase, 512);
}

int m16_of8(int m) { return (m + 15) / 16 * 16; }

// The operand images of A * 2^ea for the 8 column slices of 128 coefficients:
// slice q holds fp16 hi, fp16 lo, bf16 hi, bf16 lo of A[:, 128 q .. 128 q + 127],
// each m16 rows x 128, rows >= M zero, 128-byte swizzled atoms of 8 rows x 64
// columns (atom (col/64, row/8) at ((col/64) * m16/8 + row/8) * 1024).
__global__ void k_tc8_images(const float* __restrict__ a, uint8_t* __restrict__ img, int m, int m16,
                             float scale) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m16 * kN) return;
    const int row = idx / kN, col = idx % kN;
    const int slice = col / kW, cl = col % kW;
    const float v = row < m ? a[(size_t)row * kN + col] * scale : 0.f;
    const size_t img_bytes = (size_t)m16 * kW * 2;
    uint8_t* base = img + (size_t)slice * 4 * img_bytes +
                    sw128_offset((uint32_t)row, (uint32_t)cl, (uint32_t)m16 / 8);
    const __half hh = __float2half_rn(v);
    const __half hl = __float2half_rn(v - __half2float(hh));
    const __nv_bfloat16 bh = __float2bfloat16_rn(v);
    const __nv_bfloat16 bl = __float2bfloat16_rn(v - __bfloat162float(bh));
    *reinterpret_cast<__half*>(base) = hh;
    *reinterpret_cast<__half*>(base + img_bytes) = hl;
    *reinterpret_cast<__nv_bfloat16*>(base + 2 * img_bytes) = bh;
    *reinterpret_cast<__nv_bfloat16*>(base + 3 * img_bytes) = bl;
}

}  // namespace

cudaError_t launch_tc8_images(const float* a, uint8_t* img, int m, int ea, cudaStream_t s) {
    const int m16 = m16_of8(m);
    const int total = m16 * kN;
    k_tc8_images<<<(total + 255) / 256, 256, 0, s>>>(a, img, m, m16, ldexpf(1.f, ea));
    return cudaGetLastError();
}

static size_t tc8_slot_floats(int sm_count) { return (size_t)(sm_count / kCl + 1) * kTile * kN; }

size_t tc8_slot_bytes(int sm_count) {
    return tc8_slot_floats(sm_count) * sizeof(float);
}

static void fill_job8(const DecodeArgs& d, int tile_begin, Tc8Job* J) {
    const cs_plan* p = d.plan;
    J->a_img = p->a_tc;
    J->y = d.y;
    J->keys = d.key;
    J->out_f32 = d.out_f32;
    J->out_u8 = d.out_u8;
    J->dct = p->dct;
    J->gs = d.gs;
    // this launch recovers blocks [0, rows) of the call (a tail may go to the streaming kernel)
    J->rows = d.row_end < 0 ? (long long)d.gs.n_cs * d.gs.nblk : d.row_end;
    J->tile_begin = tile_begin;
    J->m16 = m16_of8(p->m);
    J->iters = d.iters;
    const bool mixed = d.precision == CS_BF16 || d.precision == CS_FP16;
    J->split_from = mixed ? (d.iters > d.tail_iters ? d.iters - d.tail_iters : 0) : 0;
    J->lambda_rel = d.lambda_rel;
    J->inv_l = (float)(1.0 / p->lipschitz);
    J->su = ldexpf(1.f, -p->tc_ea);
    J->sg = ldexpf(1.f, -(p->tc_ea + p->tc_ep));
    J->sp = ldexpf(1.f, p->tc_ep);
}

// Clusters of the kernel that fit the device at once (each tile's 8 CTAs wait
// on one another, so only co-resident clusters may run).
static cudaError_t co_resident_clusters(bool bf, int* clusters) {
    const void* fn = bf ? (const void*)k_fista_tc8<true> : (const void*)k_fista_tc8<false>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kCl, 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = kSmemBytes;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = kCl;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(clusters, fn, &cfg);
}

// One cluster launch for up to kMaxJobs8 jobs of one operand type.
static cudaError_t launch_group8(const DecodeArgs* const* jobs, int n_jobs, bool bf, cudaStream_t s) {
    cs_ctx* ctx = jobs[0]->plan->ctx;
    if (!ctx->tc8_scratch) return cudaErrorInvalidValue;
    Tc8Launch L{};
    L.beta = jobs[0]->beta;
    L.err = ctx->err_dev;
    std::lock_guard<std::mutex> lock(ctx->launch_mu);
    int slot = 0;
    cudaError_t e = slot_take(&ctx->tc8_ring, s, &slot);
    if (e != cudaSuccess) return e;
    L.scratch = ctx->tc8_scratch + (size_t)slot * tc8_slot_floats(ctx->sm_count);
    L.drop_arrival = ctx->debug_flags.exchange(0) & CS_DEBUG_DROP_ARRIVAL;
    int tiles = 0;
    for (int i = 0; i < n_jobs; ++i) {
        fill_job8(*jobs[i], tiles, &L.jobs[i]);
        tiles += (int)((L.jobs[i].rows + kTile - 1) / kTile);
    }
    L.n_jobs = n_jobs;
    L.n_tiles = tiles;
    const void* fn = bf ? (const void*)k_fista_tc8<true> : (const void*)k_fista_tc8<false>;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    // the epilogue's setmaxnreg.inc draws on the registers the CTA was launched with
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    if (fa.numRegs < kLaunchRegs || fa.maxThreadsPerBlock < kThreads) return cudaErrorInvalidConfiguration;
    // as many clusters as are co-resident, and no more than the scratch holds
    int max_clusters = 0;
    e = co_resident_clusters(bf, &max_clusters);
    if (e != cudaSuccess) return e;
    if (max_clusters < 1) return cudaErrorInvalidConfiguration;
    int clusters = std::min(max_clusters, ctx->sm_count / kCl + 1);
    clusters = std::min(clusters, tiles);
    if (bf)
        k_fista_tc8<true><<<clusters * kCl, kThreads, kSmemBytes, s>>>(L);
    else
        k_fista_tc8<false><<<clusters * kCl, kThreads, kSmemBytes, s>>>(L);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return slot_done(&ctx->tc8_ring, slot, s);
}

int tc8_clusters(bool bf) {
    int c = 0;
    return co_resident_clusters(bf, &c) == cudaSuccess ? c : 0;
}

static double job_cost8(const DecodeArgs& d) {
    return (double)((long long)d.gs.n_cs * d.gs.nblk) * (double)d.iters * (double)m16_of8(d.plan->m);
}

// The SMs that whole clusters leave idle (GPCs whose SM count is not a multiple
// of 8) take a tail of each large job on the streaming kernel, two CTAs each.
// A tile there lasts about kTcsTileRatio times a cluster's tile, so the tail is
// r rounds of 2 x idle tiles with r (2 x idle) + clusters x r x kTcsTileRatio <=
// the job's tiles, or, when not one whole round fits, a partial round of the
// tiles beyond clusters x kTcsTileRatio: both kernels then finish at about the
// same time.  The split depends on the job alone, so a job decodes to the same
// bits in any batch.
constexpr int kTcsTileRatio = 13;

// (a job's blocks end at row_end when it is set: a range handed over by another kernel)
static long long job_end8(const DecodeArgs& d) {
    return d.row_end < 0 ? (long long)d.gs.n_cs * d.gs.nblk : d.row_end;
}

static long long tail_rows(const DecodeArgs& d, int clusters, int idle_ctas) {
    if (idle_ctas <= 0 || !tcs_supported(d.plan)) return 0;
    const long long total = job_end8(d);
    const long long tiles = (total + kTile - 1) / kTile;
    const long long one_round = (long long)clusters * kTcsTileRatio;
    const long long rounds = tiles / (one_round + idle_ctas);
    const long long tail_tiles =
        rounds > 0 ? rounds * idle_ctas : std::min<long long>(idle_ctas, tiles - one_round);
    if (tail_tiles <= 0) return 0;
    return total - (tiles - tail_tiles) * kTile;
}

cudaError_t launch_decode_tc8_batch(const DecodeArgs* jobs, int n_jobs, cudaStream_t s) {
    std::vector<DecodeArgs> head[2], tail[2];
    for (int i = 0; i < n_jobs; ++i) {
        if ((long long)jobs[i].gs.n_cs * jobs[i].gs.nblk == 0) continue;
        const bool bf = jobs[i].precision == CS_BF16 || jobs[i].precision == CS_BF16X2;
        head[bf ? 1 : 0].push_back(jobs[i]);
    }
    cs_ctx* ctx = n_jobs > 0 ? jobs[0].plan->ctx : nullptr;
    for (int bf = 0; bf < 2; ++bf) {
        if (head[bf].empty()) continue;
        int clusters = 0;
        cudaError_t e = co_resident_clusters(bf == 1, &clusters);
        if (e != cudaSuccess) return e;
        const int idle_ctas = tcs_ctas_per_sm() * (ctx->sm_count - clusters * kCl);
        for (DecodeArgs& d : head[bf]) {
            const long long t = tail_rows(d, clusters, idle_ctas);
            if (t <= 0) continue;
            const long long total = job_end8(d);
            DecodeArgs dt = d;
            dt.row_begin = total - t;
            dt.row_end = total;
            d.row_end = total - t;
            tail[bf].push_back(dt);
        }
        std::vector<const DecodeArgs*> g;
        for (DecodeArgs& d : head[bf]) g.push_back(&d);
        std::stable_sort(g.begin(), g.end(), [](const DecodeArgs* a, const DecodeArgs* b) {
            return job_cost8(*a) > job_cost8(*b);
        });
        // with tails: the clusters on the context's highest-priority stream, so that
        // the dispatcher places them before the tails' CTAs, and the tails beside
        // them; both forked from s and joined back on it
        cudaStream_t hs = s, fs = nullptr;
        cudaEvent_t fork = nullptr, join_h = nullptr, join_t = nullptr;
        if (!tail[bf].empty()) {
            hs = fork_stream(ctx, s, kForkTc8Head);
            fs = fork_stream(ctx, s, kForkTc8Tail);
            e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join_h, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join_t, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventRecord(fork, s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(hs, fork, 0);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(fs, fork, 0);
        }
        for (size_t i = 0; e == cudaSuccess && i < g.size(); i += kMaxJobs8) {
            const int n = (int)std::min(g.size() - i, (size_t)kMaxJobs8);
            e = launch_group8(g.data() + i, n, bf == 1, hs);
        }
        if (fork) {
            if (e == cudaSuccess)
                e = launch_decode_tcs_batch(tail[bf].data(), (int)tail[bf].size(), fs, idle_ctas);
            if (e == cudaSuccess) e = cudaEventRecord(join_h, hs);
            if (e == cudaSuccess) e = cudaEventRecord(join_t, fs);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, join_h, 0);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, join_t, 0);
            cudaEventDestroy(fork);
            if (join_h) cudaEventDestroy(join_h);
            if (join_t) cudaEventDestroy(join_t);
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace csvc
