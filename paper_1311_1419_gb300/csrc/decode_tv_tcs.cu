// TV recovery on the tensor cores for the shapes whose state does not fit on one
// SM (8 x 8 blocks, 16 x 16 blocks with M > 128, 32 x 32 blocks; M <= 512): the
// same iteration as the plain TV kernel (decode_tv.cu) and the on-chip one
// (decode_tc.cu), Eq. 1 with the total variation, with both Phi products of an
// iteration on tcgen05 and the state in a per-CTA global scratch.
//
//   GEMM1  U [128 x M16] = R [128 x N] . Phi^T     (Phi r per block)
//   GEMM2  G [128 x N]   = P [128 x M16] . Phi     (Phi^T P, P = mu (Phi r - y) - lam)
//
// The operands stream as in the streaming FISTA kernel (decode_tcs.cu): a copy warp
// feeds a three-slot ring of 32-wide K slices (64-byte-swizzled; the tile operand R
// or P from the scratch, the Phi slice from the plan's two images of Phi, which stay
// in L2), one thread issues three MMAs per K step (hi.hi + lo.hi + hi.lo), and the
// accumulator is double-buffered in tensor memory (two 256-column chunks).
// The iterate r and q = nu + beta w (two planes) live in the scratch, double-
// buffered, as [pixel / 4][128 blocks] float4 (a warp's 32 blocks read 512
// contiguous bytes).  The w-step is fused into the r step: from r_k and q_{k-1},
//   d = D r_k,  nu_k = q_{k-1} - beta d,  w_k = shrink(d - nu_k / beta, 1 / beta),
//   q_k = nu_k + beta w_k,  t = beta d - q_k,  r_{k+1} = r_k - alpha (D^T t + G),
// so each GEMM2 chunk's pixels are updated in one pass that reads r_k and q_{k-1}
// (with one row of neighbours on each side) and writes r_{k+1}, q_k and the next
// GEMM1's operand image of r_{k+1} (fp16 hi / lo).  The multiplier step lam -= mu
// (Phi r' - y) is deferred to the next GEMM1 as in the on-chip kernel: P_k = 2 mu
// (U_k - y) - lam_{k-1}, lam_k = lam_{k-1} - mu (U_k - y), P_0 = -mu y.  Every
// mbarrier wait is bounded and reports through the context's error word.
#include <cuda_fp16.h>
#include <math.h>

#include <algorithm>
#include <mutex>

#include "internal.h"
#include "tc_ptx.h"

namespace csvc {
namespace {

using namespace tc;

constexpr int kTile = 128;                  // blocks per tile = TMEM lanes
constexpr int kEpiWarps = 16;               // 4 TMEM lane quarters x 4 column groups
constexpr int kColGroups = kEpiWarps / 4;
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kThreads = 64 + kEpiThreads;  // warp 0 MMAs, warp 1 copies, warps 2 .. 17 epilogue
constexpr int kChunk = 256;                 // accumulator columns per chunk
constexpr int kSliceK = 32;                 // K per ring slot: one 64-byte swizzle atom
constexpr uint32_t kTBytes = kTile * 64;    // one K slice of the tile operand (8 KB)
constexpr uint32_t kBBytes = kChunk * 64;   // one K slice of up to 256 rows of Phi (16 KB)
constexpr int kStages = 3;
constexpr uint32_t kStageBytes = 2 * (kTBytes + kBBytes);   // hi and lo of both: 48 KB
constexpr uint32_t kOffMisc = kStages * kStageBytes;
constexpr uint32_t kSmemBytes = kOffMisc + 1024 + 1024;
constexpr uint64_t kWaitNs = 1000000000ull;
constexpr uint32_t kBarEpi = 1;
constexpr int kMaxNv = 1024, kMaxM16v = 512;

// Per-CTA scratch (bytes), for N = n and M16 = m16.
struct ScrLayout {
    size_t r_img, p_img, y4, lam4, r[2], q[2], total;
};
__host__ __device__ inline ScrLayout scr_layout(int n, int m16) {
    ScrLayout s;
    size_t o = 0;
    s.r_img = o;  o += (size_t)n * kTile * 4;                 // R hi then lo
    const size_t ps = (size_t)((m16 + kSliceK - 1) / kSliceK) * kTBytes;
    s.p_img = o;  o += 2 * ps;                                // P hi then lo
    s.y4 = o;     o += (size_t)m16 * kTile * 4;               // [m16 / 4][128] float4
    s.lam4 = o;   o += (size_t)m16 * kTile * 4;
    for (int i = 0; i < 2; ++i) { s.r[i] = o; o += (size_t)n * kTile * 4; }
    for (int i = 0; i < 2; ++i) { s.q[i] = o; o += 2 * (size_t)n * kTile * 4; }
    s.total = (o + 4095) / 4096 * 4096;
    return s;
}

}  // namespace

struct TvsJob {
    const uint8_t* a1_img;  // GEMM1 image of Phi 2^e: hi then lo, m16 x n x 2 bytes each
    const uint8_t* a2_img;  // GEMM2 image: hi then lo, m32 x n x 2 bytes each
    const float* y;
    const uint8_t* keys;
    float* out_f32;
    uint8_t* out_u8;
    GopShape gs;
    long long rows;
    int n, m16, iters;
    float su, sg, sp;       // U = acc su, G = acc sg, P operand = P sp
    float beta, mu, alpha;
};
struct TvsLaunch {
    int* err;
    int* tile_counter;
    uint8_t* scratch;       // gridDim.x areas of scr_layout(n, m16).total bytes
    size_t scr_stride;
    int n_tiles;
    int drop_arrival;       // test hook: CTA 0 withholds one warp's first P-ready arrival
    TvsJob job;
};

namespace {

struct MiscV {
    uint64_t full[kStages], empty[kStages];
    uint64_t acc_full[2], acc_empty[2];
    uint64_t p_ready, z_ready, drain;
    uint32_t tmem_base;
    int abort;
    int next_tile;
};
static_assert(sizeof(MiscV) <= 1024, "barrier block");

__device__ __forceinline__ bool wait_v(MiscV* ms, uint64_t* bar, uint32_t parity, int* err) {
    if (*(volatile int*)&ms->abort) return false;
    if (mbar_wait(bar, parity, kWaitNs)) return true;
    *(volatile int*)&ms->abort = 1;
    atomicExch(err, 1);
    return false;
}
__device__ __forceinline__ int fetch_tile_v(const TvsLaunch& L, MiscV* ms) {
    if (threadIdx.x == 0) {
        const int t = atomicAdd(L.tile_counter, 1);
        ms->next_tile = t < L.n_tiles ? t : -1;
    }
    __syncthreads();
    return ms->next_tile;
}
__device__ __forceinline__ void cta_sync_v() {
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
}
__device__ __forceinline__ uint32_t pack2h(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ float2 unpack2h(uint32_t v) {
    __half2 h = *reinterpret_cast<__half2*>(&v);
    return __half22float2(h);
}
__device__ __forceinline__ float shrink_v(float v, float t) { return v - fminf(fmaxf(v, -t), t); }

// Chunk geometry (as the streaming FISTA kernel): GEMM1 U in one chunk of m16
// columns or two of about m16 / 2; GEMM2 G in n / min(n, 256) chunks.
__device__ __forceinline__ int g1_chunks_v(int m16) { return m16 > kChunk ? 2 : 1; }
__device__ __forceinline__ int g1_width_v(int m16, int c) {
    if (m16 <= kChunk) return m16;
    const int w0 = (m16 / 2 + 15) / 16 * 16;
    return c == 0 ? w0 : m16 - w0;
}
__device__ __forceinline__ int g1_base_v(int m16, int c) { return c == 0 ? 0 : g1_width_v(m16, 0); }
__device__ __forceinline__ int g2_width_v(int n) { return n < kChunk ? n : kChunk; }
__device__ __forceinline__ int p_slices_v(int m16) { return (m16 + kSliceK - 1) / kSliceK; }

// Passes of a tile with K iterations: 0 = GEMM2 of k = 0, then GEMM1 (odd) and
// GEMM2 (even) of k = (pass + 1) / 2.
__device__ __forceinline__ bool pass_g2(int pass) { return (pass & 1) == 0; }

// Warp 1: streams the operands of every pass into the stage ring.
__device__ __forceinline__ void copy_role_v(const TvsLaunch& L, MiscV* ms, uint8_t* sm, int lane) {
    const TvsJob& J = L.job;
    const int n = J.n, m16 = J.m16;
    const ScrLayout sl = scr_layout(n, m16);
    uint8_t* scr = L.scratch + (size_t)blockIdx.x * L.scr_stride;
    const size_t img1 = (size_t)m16 * n * 2, img2 = (size_t)((m16 + 31) / 32 * 32) * n * 2;
    const uint8_t* r_hi = scr + sl.r_img;
    const uint8_t* r_lo = r_hi + (size_t)n * 256;
    const uint8_t* p_hi = scr + sl.p_img;
    const uint8_t* p_lo = p_hi + (size_t)p_slices_v(m16) * kTBytes;
    uint32_t st = 0, pc = 0, zc = 0;
    uint32_t last_par = 0, issued = 0;   // per stage, one bit each
    bool ok = true;
    for (;;) {
        const int tile = fetch_tile_v(L, ms);
        if (tile < 0) break;
        cta_sync_v();   // B
        for (int pass = 0; pass < 2 * J.iters - 1; ++pass) {
            const bool g2 = pass_g2(pass);
            if (g2) {
                ok = wait_v(ms, &ms->p_ready, pc & 1, L.err) && ok;
                ++pc;
            } else {
                ok = wait_v(ms, &ms->z_ready, zc & 1, L.err) && ok;
                ++zc;
            }
            const int nch = g2 ? n / g2_width_v(n) : g1_chunks_v(m16);
            const int nst = g2 ? p_slices_v(m16) : n / kSliceK;
            for (int c = 0; c < nch; ++c) {
                for (int ks = 0; ks < nst; ++ks) {
                    const uint32_t s = st % kStages, par = (st / kStages) & 1;
                    ok = wait_v(ms, &ms->empty[s], par ^ 1, L.err) && ok;
                    if (ok && lane == 0) {
                        uint8_t* stg = sm + s * kStageBytes;
                        const uint32_t bbytes = g2 ? (uint32_t)g2_width_v(n) * 64u : (uint32_t)g1_width_v(m16, c) * 64u;
                        mbar_arrive_expect_tx(&ms->full[s], 2u * (kTBytes + bbytes));
                        for (int h = 0; h < 2; ++h) {
                            uint8_t* t_dst = stg + h * kTBytes;
                            uint8_t* b_dst = stg + 2 * kTBytes + h * kBBytes;
                            if (g2) {
                                const uint8_t* aimg = J.a2_img + (h ? img2 : 0);
                                bulk_g2s(t_dst, (h ? p_lo : p_hi) + (size_t)ks * kTBytes, kTBytes, &ms->full[s]);
                                bulk_g2s(b_dst, aimg + ((size_t)ks * (n / 32) + (size_t)c * (g2_width_v(n) / 32)) * 2048,
                                         bbytes, &ms->full[s]);
                            } else {
                                const uint8_t* aimg = J.a1_img + (h ? img1 : 0);
                                bulk_g2s(t_dst, (h ? r_lo : r_hi) + (size_t)ks * kTBytes, kTBytes, &ms->full[s]);
                                bulk_g2s(b_dst, aimg + ((size_t)ks * (m16 / 8) + g1_base_v(m16, c) / 8) * 512, bbytes,
                                         &ms->full[s]);
                            }
                        }
                        last_par = (last_par & ~(1u << s)) | (par << s);
                        issued |= 1u << s;
                    }
                    __syncwarp();
                    ++st;
                }
            }
        }
        cta_sync_v();   // C
    }
    if (lane == 0) {
        // copies whose consumer gave up may still be in flight (bounded)
        for (int s = 0; s < kStages; ++s)
            if ((issued >> s) & 1u) mbar_wait(&ms->full[s], (last_par >> s) & 1u, kWaitNs);
    }
    __syncwarp();
}

// Warp 0: issues every MMA (lane 0), chunk by chunk into the two accumulators.
__device__ __forceinline__ void mma_role_v(const TvsLaunch& L, MiscV* ms, uint8_t* sm, uint32_t tbase, int lane) {
    const TvsJob& J = L.job;
    const int n = J.n, m16 = J.m16;
    const uint32_t s_base = smem_u32(sm);
    uint32_t st = 0, acc = 0;
    bool ok = true;
    for (;;) {
        const int tile = fetch_tile_v(L, ms);
        if (tile < 0) break;
        cta_sync_v();   // B
        for (int pass = 0; pass < 2 * J.iters - 1; ++pass) {
            const bool g2 = pass_g2(pass);
            const int nch = g2 ? n / g2_width_v(n) : g1_chunks_v(m16);
            const int nst = g2 ? p_slices_v(m16) : n / kSliceK;
            for (int c = 0; c < nch; ++c) {
                const uint32_t a = acc & 1;
                ok = wait_v(ms, &ms->acc_empty[a], ((acc >> 1) & 1) ^ 1, L.err) && ok;
                fence_after_sync();
                const uint32_t d = tbase + a * kChunk;
                const int width = g2 ? g2_width_v(n) : g1_width_v(m16, c);
                const uint32_t id = idesc_f16(128, (uint32_t)width, 0u, 0u, g2 ? 1u : 0u);
#pragma unroll 1
                for (int ks = 0; ks < nst; ++ks) {
                    const uint32_t s = st % kStages, par = (st / kStages) & 1;
                    ok = wait_v(ms, &ms->full[s], par, L.err) && ok;
                    fence_after_sync();
                    if (ok && lane == 0) {
                        const uint32_t stg = s_base + s * kStageBytes;
                        const uint64_t t_hi = desc_sw64(stg, 16, 512);
                        const uint64_t t_lo = desc_sw64(stg + kTBytes, 16, 512);
                        const uint64_t b_hi = g2 ? desc_sw64(stg + 2 * kTBytes, 2048, 512)
                                                 : desc_sw64(stg + 2 * kTBytes, 16, 512);
                        const uint64_t b_lo = g2 ? desc_sw64(stg + 2 * kTBytes + kBBytes, 2048, 512)
                                                 : desc_sw64(stg + 2 * kTBytes + kBBytes, 16, 512);
                        const int nk = g2 ? min(2, m16 / 16 - 2 * ks) : 2;
                        for (int kk = 0; kk < nk; ++kk) {
                            const uint32_t to = (uint32_t)kk * 2u;
                            const uint32_t bo = g2 ? (uint32_t)kk * 64u : (uint32_t)kk * 2u;
                            const uint32_t accum = (ks > 0 || kk > 0) ? 1u : 0u;
                            mma_f16(d, t_hi + to, b_hi + bo, id, accum);
                            mma_f16(d, t_lo + to, b_hi + bo, id, 1u);
                            mma_f16(d, t_hi + to, b_lo + bo, id, 1u);
                        }
                        mma_commit(&ms->empty[s]);
                    }
                    __syncwarp();
                    ++st;
                }
                if (ok && lane == 0) mma_commit(&ms->acc_full[a]);
                __syncwarp();
                ++acc;
            }
        }
        cta_sync_v();   // C
    }
    if (lane == 0) {
        mma_commit(&ms->drain);
        mbar_wait(&ms->drain, 0, kWaitNs);
    }
    __syncwarp();
}

__device__ __forceinline__ void acc_wait_v(const TvsLaunch& L, MiscV* ms, uint32_t acc) {
    wait_v(ms, &ms->acc_full[acc & 1], (acc >> 1) & 1, L.err);
    fence_after_sync();
}
__device__ __forceinline__ void acc_release_v(MiscV* ms, uint32_t acc, int lane) {
    fence_before_sync();
    __syncwarp();
    if (lane == 0) mbar_arrive(&ms->acc_empty[acc & 1]);
}
// The epilogue's global writes of an operand image are complete: let the copy warp read it.
__device__ __forceinline__ void signal_copy_v(uint64_t* bar, int lane, bool withhold = false) {
    fence_proxy_async_global();
    __syncwarp();
    if (lane == 0 && !withhold) mbar_arrive(bar);
}

// P for measurements i0 .. i0 + w4 - 1 of block blk (U from accumulator columns
// starting at ucol, none at k = 0): rho = U su - y, P = mu rho - lam at k = 0 (lam =
// 0, U = 0), else 2 mu rho - lam_{k-1}, lam_k = lam_{k-1} - mu rho; P sp as fp16
// hi / lo into the P image.
__device__ __forceinline__ void residual_v(const TvsJob& J, uint8_t* __restrict__ p_hi, uint8_t* __restrict__ p_lo,
                                           const float4* __restrict__ y4, float4* __restrict__ lam4, uint32_t ucol,
                                           int i0, int w4, int blk, int k, bool live) {
    const float mu = J.mu, cmu = k == 0 ? mu : 2.f * mu;
    const bool use_u = k > 0, read_lam = live && k > 1, write_lam = live && k > 0 && k + 1 < J.iters;
    for (int cc = 0; cc < w4; cc += 4) {
        const int i = i0 + cc;
        uint32_t u[4] = {0u, 0u, 0u, 0u};
        if (use_u) tmem_ld4(ucol + (uint32_t)cc, u);
        const size_t vi = (size_t)(i / 4) * kTile + blk;
        const float4 yv = live ? y4[vi] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 lv = read_lam ? lam4[vi] : make_float4(0.f, 0.f, 0.f, 0.f);
        if (use_u) tmem_wait_ld();
        const float yy[4] = {yv.x, yv.y, yv.z, yv.w};
        float l[4] = {lv.x, lv.y, lv.z, lv.w}, p[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float rho = __uint_as_float(u[e]) * J.su - yy[e];
            p[e] = live ? (cmu * rho - l[e]) * J.sp : 0.f;
            l[e] -= mu * rho;
        }
        if (write_lam) lam4[vi] = make_float4(l[0], l[1], l[2], l[3]);
        const uint32_t h0 = pack2h(p[0], p[1]), h1 = pack2h(p[2], p[3]);
        const float2 d0 = unpack2h(h0), d1 = unpack2h(h1);
        const uint32_t off = sw64_offset((uint32_t)blk, (uint32_t)i, kTile / 8);
        *reinterpret_cast<uint2*>(p_hi + off) = make_uint2(h0, h1);
        *reinterpret_cast<uint2*>(p_lo + off) = make_uint2(pack2h(p[0] - d0.x, p[1] - d0.y), pack2h(p[2] - d1.x, p[3] - d1.y));
    }
}

// One row of four pixels (p, 4 c4 .. 4 c4 + 3) of the r step with the fused w-step:
// r[0..3] the row's r_k and r[4] its right neighbour's, rd the row below, qh / qv
// the row's q_{k-1}, tu the t_v of the pixels above (0 on a block's first row), g
// the accumulator's G; th_carry carries t_h from the pixel on the left.  Writes
// q_k (qhn, qvn), r_{k+1} (rnew) and the row's t_v (the next row's tu).
__device__ __forceinline__ void tv_row4(const float r[5], const float rd[4], const float qh[4], const float qv[4],
                                        const float tu[4], const uint32_t g[4], int p, int c4, int b, float beta,
                                        float ib, float alpha, float sg, float& th_carry, float qhn[4],
                                        float qvn[4], float rnew[4], float tv[4]) {
    float tl = th_carry;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int pc = 4 * c4 + e;
        const float dh = pc < b - 1 ? r[e + 1] - r[e] : 0.f;
        const float nh = qh[e] - beta * dh;
        qhn[e] = nh + beta * shrink_v(dh - nh * ib, ib);
        const float th = pc < b - 1 ? beta * dh - qhn[e] : 0.f;
        const float dv = p < b - 1 ? rd[e] - r[e] : 0.f;
        const float nv = qv[e] - beta * dv;
        qvn[e] = nv + beta * shrink_v(dv - nv * ib, ib);
        tv[e] = p < b - 1 ? beta * dv - qvn[e] : 0.f;
        const float dt = (pc > 0 ? tl : 0.f) - th + tu[e] - tv[e];
        rnew[e] = r[e] - alpha * fmaf(__uint_as_float(g[e]), sg, dt);
        tl = th;
    }
    th_carry = tl;
}

// The row's results: q_k and r_{k+1} into (qn, rn) at float4 index vi (a live lane
// only), r_{k+1} as fp16 hi / lo into the R image.
__device__ __forceinline__ void tv_store4(float4* __restrict__ rn, float4* __restrict__ qn,
                                          uint8_t* __restrict__ r_hi, uint8_t* __restrict__ r_lo, size_t vi,
                                          size_t plane4, int blk, int j, bool live, const float qhn[4],
                                          const float qvn[4], const float rnew[4]) {
    if (live) {
        qn[vi] = make_float4(qhn[0], qhn[1], qhn[2], qhn[3]);
        qn[vi + plane4] = make_float4(qvn[0], qvn[1], qvn[2], qvn[3]);
        rn[vi] = make_float4(rnew[0], rnew[1], rnew[2], rnew[3]);
    }
    const uint32_t h0 = pack2h(rnew[0], rnew[1]), h1 = pack2h(rnew[2], rnew[3]);
    const float2 d0 = unpack2h(h0), d1 = unpack2h(h1);
    const uint32_t off = sw64_offset((uint32_t)blk, (uint32_t)j, kTile / 8);
    *reinterpret_cast<uint2*>(r_hi + off) = make_uint2(h0, h1);
    *reinterpret_cast<uint2*>(r_lo + off) =
        make_uint2(pack2h(rnew[0] - d0.x, rnew[1] - d0.y), pack2h(rnew[2] - d1.x, rnew[3] - d1.y));
}

// The r step (with the fused w-step) for pixel rows p0 .. p0 + nrows - 1 (nrows
// even) of block blk: r_k, q_{k-1} from (rc, qc), r_{k+1}, q_k into (rn, qn) and the
// R image; G from accumulator columns gcol + (pixel - pix0).  k = 0 (first): r = q =
// 0.  Rows go in pairs, so that one wait covers both rows' loads and the second row
// takes its neighbours above (r, q_v and t_v) from the first.  A lane with no block
// (live false) moves no state and writes zeros into the R image.
__device__ __forceinline__ void r_step_v(const TvsJob& J, const float4* __restrict__ rc,
                                         const float4* __restrict__ qc, float4* __restrict__ rn,
                                         float4* __restrict__ qn, uint8_t* __restrict__ r_hi,
                                         uint8_t* __restrict__ r_lo, uint32_t gcol, int pix0, int p0, int nrows,
                                         int blk, bool first, bool live) {
    const int n = J.n, b = J.gs.b, nq = b / 4;
    const float beta = J.beta, ib = 1.f / beta, alpha = J.alpha, sg = J.sg;
    const float* rcf = reinterpret_cast<const float*>(rc);
    const size_t row4 = (size_t)nq * kTile, plane4 = (size_t)(n / 4) * kTile;
    const bool ld = !first && live;
    for (int p = p0; p < p0 + nrows; p += 2) {
        float thc0 = 0.f, thc1 = 0.f;
        for (int c4 = 0; c4 < nq; ++c4) {
            const int j = p * b + 4 * c4;
            const size_t vi = (size_t)(j / 4) * kTile + blk;
            uint32_t g0[4], g1[4];
            tmem_ld4(gcol + (uint32_t)(j - pix0), g0);
            tmem_ld4(gcol + (uint32_t)(j + b - pix0), g1);
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            float4 Ru = z, R0 = z, R1 = z, Rd = z, Qu = z, Qh0 = z, Qv0 = z, Qh1 = z, Qv1 = z;
            float rr0 = 0.f, rr1 = 0.f;
            if (ld) {
                R0 = rc[vi];
                R1 = rc[vi + row4];
                Ru = p > 0 ? rc[vi - row4] : R0;
                Rd = p + 2 < b ? rc[vi + 2 * row4] : R1;
                if (c4 + 1 < nq) {
                    rr0 = rcf[(vi + kTile) * 4];
                    rr1 = rcf[(vi + row4 + kTile) * 4];
                }
                Qh0 = qc[vi];
                Qv0 = qc[vi + plane4];
                Qh1 = qc[vi + row4];
                Qv1 = qc[vi + plane4 + row4];
                if (p > 0) Qu = qc[vi + plane4 - row4];
            }
            tmem_wait_ld();
            const float r0[5] = {R0.x, R0.y, R0.z, R0.w, rr0}, r1[5] = {R1.x, R1.y, R1.z, R1.w, rr1};
            const float ru[4] = {Ru.x, Ru.y, Ru.z, Ru.w}, rd[4] = {Rd.x, Rd.y, Rd.z, Rd.w};
            const float qu[4] = {Qu.x, Qu.y, Qu.z, Qu.w};
            const float qh0[4] = {Qh0.x, Qh0.y, Qh0.z, Qh0.w}, qv0[4] = {Qv0.x, Qv0.y, Qv0.z, Qv0.w};
            const float qh1[4] = {Qh1.x, Qh1.y, Qh1.z, Qh1.w}, qv1[4] = {Qv1.x, Qv1.y, Qv1.z, Qv1.w};
            float tu[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {   // t_v of the pixels above row p, from their r_k and q_{k-1}
                tu[e] = 0.f;
                if (p > 0) {
                    const float du = r0[e] - ru[e];
                    const float nu = qu[e] - beta * du;
                    tu[e] = beta * du - (nu + beta * shrink_v(du - nu * ib, ib));
                }
            }
            float qhn[4], qvn[4], rnew[4], tv[4];
            tv_row4(r0, r1, qh0, qv0, tu, g0, p, c4, b, beta, ib, alpha, sg, thc0, qhn, qvn, rnew, tv);
            if (!live) rnew[0] = rnew[1] = rnew[2] = rnew[3] = 0.f;
            tv_store4(rn, qn, r_hi, r_lo, vi, plane4, blk, j, live, qhn, qvn, rnew);
            float tv1[4];
            tv_row4(r1, rd, qh1, qv1, tv, g1, p + 1, c4, b, beta, ib, alpha, sg, thc1, qhn, qvn, rnew, tv1);
            if (!live) rnew[0] = rnew[1] = rnew[2] = rnew[3] = 0.f;
            tv_store4(rn, qn, r_hi, r_lo, vi + row4, plane4, blk, j + b, live, qhn, qvn, rnew);
        }
    }
}

// Warps 2 .. 17.
__device__ __forceinline__ void epi_role_v(const TvsLaunch& L, MiscV* ms, uint32_t tbase, int warp, int lane) {
    const TvsJob& J = L.job;
    const GopShape& gs = J.gs;
    const int ew = warp - 2, q = warp & 3, cg = ew >> 2;
    const int blk = 32 * q + lane;                    // TMEM lane = block of the tile
    const int et = threadIdx.x - 64;
    const uint32_t lane_addr = tbase + ((uint32_t)(32 * q) << 16);
    const int n = J.n, m16 = J.m16, K = J.iters, b = gs.b;
    const ScrLayout sl = scr_layout(n, m16);
    uint8_t* scr = L.scratch + (size_t)blockIdx.x * L.scr_stride;
    uint8_t* r_hi = scr + sl.r_img;
    uint8_t* r_lo = r_hi + (size_t)n * 256;
    uint8_t* p_hi = scr + sl.p_img;
    uint8_t* p_lo = p_hi + (size_t)p_slices_v(m16) * kTBytes;
    float4* y4 = reinterpret_cast<float4*>(scr + sl.y4);
    float4* lam4 = reinterpret_cast<float4*>(scr + sl.lam4);
    const int nc = g2_width_v(n), nch2 = n / nc, pw = nc / kColGroups;   // pixels per column group and chunk
    uint32_t acc = 0;
    bool first_tile = true;
    for (;;) {
        const int tile = fetch_tile_v(L, ms);
        if (tile < 0) break;
        cta_sync_v();   // B
        const long long tile_row0 = (long long)tile * kTile;
        const long long rows_left = J.rows - tile_row0;
        const bool live = blk < rows_left;   // the last tile's lanes beyond its blocks move no state
        if (K > 0) {
            {   // the tile's y, read once (coalesced), [m16 / 4][128] float4, zero beyond M and the tile's blocks
                float* yf = reinterpret_cast<float*>(y4);
                const float* src = J.y + tile_row0 * gs.m;
                for (int e = et; e < kTile * m16; e += kEpiThreads) {
                    const int rr = e / m16, i = e % m16;
                    const float v = (i < gs.m && rr < rows_left) ? src[(size_t)rr * gs.m + i] : 0.f;
                    yf[((size_t)(i / 4) * kTile + rr) * 4 + (i & 3)] = v;
                }
                __threadfence_block();
                named_sync(kBarEpi, kEpiThreads);
            }
            for (int c = 0; c < g1_chunks_v(m16); ++c) {   // P_0 = -mu y
                const int w4 = g1_width_v(m16, c) / kColGroups;
                residual_v(J, p_hi, p_lo, y4, lam4, 0u, g1_base_v(m16, c) + cg * w4, w4, blk, 0, live);
            }
            // (the test hook withholds one warp's first arrival in CTA 0)
            signal_copy_v(&ms->p_ready, lane, L.drop_arrival && blockIdx.x == 0 && ew == 1 && first_tile);
            for (int k = 0; k < K; ++k) {
                if (k > 0) {
                    for (int c = 0; c < g1_chunks_v(m16); ++c, ++acc) {
                        acc_wait_v(L, ms, acc);
                        const int w4 = g1_width_v(m16, c) / kColGroups;
                        residual_v(J, p_hi, p_lo, y4, lam4, lane_addr + (acc & 1) * kChunk + (uint32_t)(cg * w4),
                                   g1_base_v(m16, c) + cg * w4, w4, blk, k, live);
                        acc_release_v(ms, acc, lane);
                    }
                    signal_copy_v(&ms->p_ready, lane);
                }
                const bool odd = k & 1;   // (selects: a runtime index would put the layout in local memory)
                const float4* rc = reinterpret_cast<const float4*>(scr + (odd ? sl.r[1] : sl.r[0]));
                const float4* qc = reinterpret_cast<const float4*>(scr + (odd ? sl.q[1] : sl.q[0]));
                float4* rn = reinterpret_cast<float4*>(scr + (odd ? sl.r[0] : sl.r[1]));
                float4* qn = reinterpret_cast<float4*>(scr + (odd ? sl.q[0] : sl.q[1]));
                for (int jc = 0; jc < nch2; ++jc, ++acc) {
                    acc_wait_v(L, ms, acc);
                    const int pix0 = jc * nc + cg * pw;
                    r_step_v(J, rc, qc, rn, qn, r_hi, r_lo, lane_addr + (acc & 1) * kChunk + (uint32_t)(cg * pw),
                             pix0, pix0 / b, pw / b, blk, k == 0, live);
                    acc_release_v(ms, acc, lane);
                }
                if (k + 1 < K) signal_copy_v(&ms->z_ready, lane);
                // the next iteration reads neighbours the other threads have just written
                __threadfence_block();
                named_sync(kBarEpi, kEpiThreads);
            }
        }
        // r^K plus the key (Eq. 4), crop; the thread's pixels of every chunk
        const long long row = tile_row0 + blk;
        const float4* rK = reinterpret_cast<const float4*>(scr + ((K & 1) ? sl.r[1] : sl.r[0]));
        if (live) {
            const int c_idx = (int)(row / gs.nblk), bl = (int)(row % gs.nblk);
            const int g_key = c_idx / (gs.g - 1);
            const int bi = bl / gs.nbc, bj = bl % gs.nbc;
            const size_t frame_px = (size_t)gs.h * gs.w;
            for (int jc = 0; jc < nch2; ++jc) {
                for (int j = jc * nc + cg * pw; j < jc * nc + (cg + 1) * pw; j += 4) {
                    const float4 v4 = K > 0 ? rK[(size_t)(j / 4) * kTile + blk] : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int py = bi * b + (j + e) / b, px = bj * b + (j + e) % b;
                        if (py >= gs.h || px >= gs.w) continue;
                        const size_t off = (size_t)py * gs.w + px;
                        const float x = (float)J.keys[(size_t)g_key * frame_px + off] + vv[e];
                        if (J.out_f32) J.out_f32[(size_t)c_idx * frame_px + off] = x;
                        if (J.out_u8) J.out_u8[(size_t)c_idx * frame_px + off] = (uint8_t)fminf(fmaxf(rintf(x), 0.f), 255.f);
                    }
                }
            }
        }
        first_tile = false;
        cta_sync_v();   // C
    }
}

__global__ void __maxnreg__(96) k_tv_tcs(const __grid_constant__ TvsLaunch L) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
    MiscV* ms = reinterpret_cast<MiscV*>(sm + kOffMisc);
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
            mbar_init(&ms->p_ready, kEpiWarps);
            mbar_init(&ms->z_ready, kEpiWarps);
            mbar_init(&ms->drain, 1);
            ms->abort = 0;
            fence_mbar_init();
        }
        __syncwarp();
        tmem_alloc(&ms->tmem_base, 2 * kChunk);
        tmem_relinquish();
    }
    cta_sync_v();
    const uint32_t tbase = ms->tmem_base;
    if (warp == 0)
        mma_role_v(L, ms, sm, tbase, lane);
    else if (warp == 1)
        copy_role_v(L, ms, sm, lane);
    else
        epi_role_v(L, ms, tbase, warp, lane);
    cta_sync_v();
    if (warp == 0) tmem_dealloc(tbase, 2 * kChunk);
}

int m16_of_v(int m) { return (m + 15) / 16 * 16; }

}  // namespace

size_t tv_tcs_slot_bytes(int sm_count) { return (size_t)sm_count * scr_layout(kMaxNv, kMaxM16v).total; }

bool tv_tcs_supported(const cs_plan* plan) {
    return plan->phi_tcs != nullptr && tcs_plan_supported(plan->n, plan->m);
}

cudaError_t launch_decode_tv_tcs(const cs_plan* plan, const GopShape& gs, int iters, float beta, float mu,
                                 float alpha, const uint8_t* key, const float* y, float* out_f32,
                                 uint8_t* out_u8, cudaStream_t s) {
    cs_ctx* ctx = plan->ctx;
    {
        // the per-CTA state areas, allocated on first use (within the scratch budget)
        std::lock_guard<std::mutex> lock(ctx->mu);
        if (!ctx->tv_scratch) {
            const size_t bytes = tv_tcs_slot_bytes(ctx->sm_count);
            if (bytes > scratch_room_of(ctx)) return cudaErrorMemoryAllocation;
            cudaError_t e = cudaMalloc(&ctx->tv_scratch, bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();   // clear it: the caller may fall back to the plain kernel
                ctx->tv_scratch = nullptr;
                return cudaErrorMemoryAllocation;
            }
            e = slot_ring_init(&ctx->tv_ring, 1);
            if (e != cudaSuccess) return e;
            ctx->scratch_bytes += bytes;
        }
    }
    TvsLaunch L{};
    L.err = ctx->err_dev;
    TvsJob& J = L.job;
    const int m16 = m16_of_v(plan->m);
    const size_t img1 = (size_t)m16 * plan->n * 2;
    J.a1_img = plan->phi_tcs;                       // fp16 hi, then fp16 lo
    J.a2_img = plan->phi_tcs + 4 * img1;
    J.y = y;
    J.keys = key;
    J.out_f32 = out_f32;
    J.out_u8 = out_u8;
    J.gs = gs;
    J.rows = (long long)gs.n_cs * gs.nblk;
    J.n = plan->n;
    J.m16 = m16;
    J.iters = iters;
    // P = 2 mu (U - y) - lam in fp16: FISTA's residual scale, halved once more and
    // again for every doubling of mu above 1
    const int ep = plan->tc_ep - 1 - (mu > 1.f ? (int)ceil(log2((double)mu)) : 0);
    J.su = ldexpf(1.f, -plan->tc_ephi);
    J.sg = ldexpf(1.f, -(plan->tc_ephi + ep));
    J.sp = ldexpf(1.f, ep);
    J.beta = beta;
    J.mu = mu;
    J.alpha = alpha;
    L.n_tiles = (int)((J.rows + kTile - 1) / kTile);
    const int grid = L.n_tiles < ctx->sm_count ? L.n_tiles : ctx->sm_count;
    L.scr_stride = scr_layout(J.n, m16).total;
    cudaError_t e = cudaFuncSetAttribute((const void*)k_tv_tcs, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(ctx->launch_mu);
    int cslot = 0, sslot = 0;
    e = slot_take(&ctx->counter_ring, s, &cslot);
    if (e == cudaSuccess) e = slot_take(&ctx->tv_ring, s, &sslot);
    if (e != cudaSuccess) return e;
    L.tile_counter = ctx->counters_dev + cslot;
    L.scratch = ctx->tv_scratch;
    L.drop_arrival = ctx->debug_flags.exchange(0) & CS_DEBUG_DROP_ARRIVAL;
    e = cudaMemsetAsync(L.tile_counter, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        k_tv_tcs<<<grid, kThreads, kSmemBytes, s>>>(L);
        e = cudaGetLastError();
    }
    const cudaError_t e1 = slot_done(&ctx->counter_ring, cslot, s);
    const cudaError_t e2 = slot_done(&ctx->tv_ring, sslot, s);
    return e != cudaSuccess ? e : e1 != cudaSuccess ? e1 : e2;
}

}  // namespace csvc
