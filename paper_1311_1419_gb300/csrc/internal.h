// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/csvc.h"

namespace csvc {

// Maximum FISTA iteration count accepted by a call (size of the momentum table).
constexpr int kMaxIters = 1 << 17;
constexpr int kMaxN = 4096;
constexpr int kTileCounters = 256;   // per-launch tile counters of the persistent decode
constexpr int kScratchSlots = 16;    // per-launch scratch areas of the 32 x 32 cluster decode
constexpr int kTcsSlotsMax = 8;      // per-launch iterate scratch areas of the streaming decode

void set_error(const std::string& msg);
int fail(int status, const std::string& msg);
int cuda_fail(cudaError_t err, const char* what);

#define CS_CUDA_TRY(expr)                                         \
    do {                                                          \
        cudaError_t _e = (expr);                                  \
        if (_e != cudaSuccess) return ::csvc::cuda_fail(_e, #expr); \
    } while (0)

struct Ticket;
struct Pool;
struct TcsQueue;

// A ring of per-launch device resources (tile counters, scratch areas).  A
// launch takes the next slot; its stream first waits for the completion event
// of the slot's previous holder, and the event is recorded again after the
// launch.  So two launches never hold one slot at the same time, whatever the
// number of streams.  Inside a stream capture the wait and the record become
// external event nodes of the graph, so that replays order themselves the same
// way against eager launches and other replays.  The caller holds the
// context's launch_mu from slot_take to slot_done, so the holders of a slot
// record its event in the order in which they took it.
struct SlotRing {
    std::vector<cudaEvent_t> ev;
    uint64_t next = 0;
};
cudaError_t slot_ring_init(SlotRing* r, int n);
void slot_ring_destroy(SlotRing* r);
cudaError_t slot_take(SlotRing* r, cudaStream_t s, int* slot);
cudaError_t slot_done(SlotRing* r, int slot, cudaStream_t s);

}  // namespace csvc

struct cs_ctx {
    int device = 0;
    int sm_count = 0;
    size_t hbm_budget = 0;
    float* beta_dev = nullptr;          // FISTA momentum (t_k - 1)/t_{k+1}, k = 1..kMaxIters
    int* err_dev = nullptr;             // set to 1 by a kernel whose bounded wait gave up
    int* counters_dev = nullptr;        // csvc::kTileCounters tile counters (counter_ring)
    // s^K all-gather of the 32 x 32 cluster decode: csvc::kScratchSlots
    // per-launch areas (tc8_ring)
    float* tc8_scratch = nullptr;
    // iterates of the streaming tensor-core decode: tcs_slots per-launch areas
    // of (CTAs per SM x sm_count) per-CTA scratches (tcs_ring)
    uint8_t* tcs_scratch = nullptr;
    int tcs_slots = 0;
    // state of the streaming TV decode (allocated on its first use): one per-launch
    // area of sm_count per-CTA scratches (tv_ring)
    uint8_t* tv_scratch = nullptr;
    size_t scratch_bytes = 0;           // tc8_scratch + tcs_scratch + tv_scratch
    std::mutex launch_mu;               // held from slot_take to slot_done
    csvc::SlotRing counter_ring, tc8_ring, tcs_ring, tv_ring;
    // device staging of cs_codec_host (grown on demand), one holder at a time
    std::mutex stage_mu;
    uint8_t* stage = nullptr;
    size_t stage_bytes = 0;
    csvc::SlotRing stage_ring;
    std::atomic<int> debug_flags{0};        // CS_DEBUG_*, consumed by the next launch
    // autotuned decode shape per (N, M): engine, plain-kernel threads and blocks per CTA
    std::mutex tune_mu;
    std::map<std::pair<int, int>, std::array<int, 3>> tuned;
    // serving state
    std::mutex mu;
    csvc::Pool* pool = nullptr;         // device pool carved from the HBM budget, on first use
    csvc::TcsQueue* tcsq = nullptr;     // device work queue of the streaming decode (serving)
    bool serving_queue = true;          // cs_submit posts to the device work queue where it can
    int max_slots = 64;
    std::vector<csvc::Ticket*> live;
    uint64_t next_ticket = 1;
    std::vector<cudaStream_t> streams;
    // extra persistent launches of one batched decode: csvc::kForkStreams fork
    // streams per origin, set 0 for callers' own streams, set 1 + i for serving
    // stream i (so that serving requests never queue behind one another's forks)
    std::vector<cudaStream_t> fork_streams;
    int next_stream = 0;
};

struct cs_plan {
    cs_ctx* ctx = nullptr;
    int n = 0, m = 0, b = 0;
    uint64_t seed = 0;
    double lipschitz = 0.0;   // L = 1.0001 * lambda_max(Phi Phi^T)
    float* phi = nullptr;     // [M][N] float32
    float* a = nullptr;       // [M][N] float32, A = Phi Psi
    float* dct = nullptr;     // [B][B] float32, C[k][j]
    // tensor-core operands: shared-memory images of A * 2^tc_ea (fp16 hi, fp16
    // lo, bf16 hi, bf16 lo); NULL when the shape has no tensor-core kernel
    uint8_t* a_tc = nullptr;
    int tc_ea = 0;            // log2 scale of A in the 16-bit operands
    // fp16 hi / lo (then bf16 hi / lo) images of Phi * 2^tc_ephi in the on-chip
    // kernels' layout (16 x 16 blocks, M <= 128): the tensor-core encode's and TV
    // decode's operand; NULL otherwise
    uint8_t* phi_tc = nullptr;
    int tc_ephi = 0;
    // fp16 hi / lo images of Phi * 2^tc_ephi in 64-column K chunks for the
    // tensor-core encode of every other shape (N = 64, 256, 1024, M <= 256); NULL
    // otherwise
    uint8_t* phi_tcg = nullptr;
    int tc_ep = 0;            // log2 scale of the residual operand P
    // images of A * 2^tc_ea (same four types, m16 x N, 128-byte-swizzled atoms)
    // for the streaming tensor-core decode; NULL when it does not take the shape
    uint8_t* a_tcs = nullptr;
    // the same images of Phi * 2^tc_ephi: the streaming TV decode's B operands
    uint8_t* phi_tcs = nullptr;
};

namespace csvc {

// plan construction kernels (phi.cu)
cudaError_t launch_phi(float* phi, int n, int m, uint64_t seed, cudaStream_t s);
cudaError_t launch_form_a(const float* phi, float* a, float* dct, int n, int m, int b,
                          cudaStream_t s);
cudaError_t launch_lambda_max(const float* phi, int n, int m, double* gram_scratch,
                              double* result_dev, cudaStream_t s);

// encode (encode.cu)
struct GopShape {
    int h, w, g, n_gops, b, n, m;
    int nbr, nbc, nblk;   // block rows, block cols, blocks per frame
    int n_cs;             // CS frames in the call = n_gops * (g - 1)
};
cudaError_t launch_encode(const cs_plan* plan, const GopShape& gs, const uint8_t* frames,
                          float* y, cudaStream_t s);
// the tensor-core encode (encode_tcg.cu): every block size, M <= 256, one or
// several plans of the same N per launch
bool encode_tcg_plan_supported(int n, int m);
bool encode_tcg_supported(const cs_plan* plan);   // the plan has Phi images for it
size_t encode_tcg_image_bytes(int n, int m);
cudaError_t launch_phi_images_g(const float* phi, uint8_t* img, int n, int m, int e, cudaStream_t s);
cudaError_t launch_encode_tcg(const cs_plan* plan, const GopShape& gs, const uint8_t* frames, float* y,
                              cudaStream_t s);
cudaError_t launch_encode_tcg_multi(const cs_plan* const* plans, float* const* ys, int n_plans,
                                    const GopShape& gs, const uint8_t* frames, cudaStream_t s);

// decode (decode_plain.cu, decode_tc.cu)
struct DecodeArgs {
    const cs_plan* plan;
    GopShape gs;
    const uint8_t* key;
    const float* y;
    float* out_f32;
    uint8_t* out_u8;
    int iters;
    int tail_iters;
    float lambda_rel;
    int precision;
    const float* beta;
    int plain_threads;        // threads per CTA of the plain kernel; 0 = default rule
    int plain_blocks;         // measured blocks per CTA of the plain kernel; 0 = 1
    // measured blocks [row_begin, row_end) of the call this launch recovers (row_end
    // < 0: to the last); the cluster kernel hands a tail range to the streaming one
    long long row_begin = 0;
    long long row_end = -1;
};
cudaError_t launch_decode_plain(const DecodeArgs& d, cudaStream_t s);
bool plain_threads_valid(int threads, int n);
bool plain_shape_valid(int threads, int blocks_per_cta, int n, int m);
int plain_threads_default(int n);
// the plain kernel's launch shape for an (N, M) the autotuner has not timed
void plain_default_shape(int n, int m, int* threads, int* blocks_per_cta);
bool tc_supported(const cs_plan* plan, int precision);
cudaError_t launch_decode_tc(const DecodeArgs& d, cudaStream_t s);
cudaError_t launch_decode_tc_batch(const DecodeArgs* jobs, int n_jobs, cudaStream_t s);
// TV recovery on the tensor cores: 16 x 16 blocks with M <= 128, state in a slot
// of the streaming decode's scratch (decode_tc.cu)
bool tv_tc_supported(const cs_plan* plan);
cudaError_t launch_decode_tv_tc(const cs_plan* plan, const GopShape& gs, int iters, float beta, float mu,
                                float alpha, const uint8_t* key, const float* y, float* out_f32,
                                uint8_t* out_u8, cudaStream_t s);
// TV recovery on the tensor cores with streamed operands: N = 64, 256, 1024 with
// M <= 512, state in the context's TV scratch (decode_tv_tcs.cu); on a budget that
// has no room for that scratch the launch returns cudaErrorMemoryAllocation
bool tv_tcs_supported(const cs_plan* plan);
size_t tv_tcs_slot_bytes(int sm_count);
cudaError_t launch_decode_tv_tcs(const cs_plan* plan, const GopShape& gs, int iters, float beta, float mu,
                                 float alpha, const uint8_t* key, const float* y, float* out_f32,
                                 uint8_t* out_u8, cudaStream_t s);
// room left for decode scratch under the context's HBM budget (caller holds ctx->mu)
size_t scratch_room_of(const cs_ctx* ctx);
// 32 x 32 blocks (N = 1024): clusters of 8 CTAs (decode_tc8.cu)
cudaError_t launch_decode_tc8_batch(const DecodeArgs* jobs, int n_jobs, cudaStream_t s);
int tc8_clusters(bool bf);   // clusters of the cluster kernel co-resident on the device (0: none)
cudaError_t launch_tc8_images(const float* a, uint8_t* img, int m, int ea, cudaStream_t s);
size_t tc8_slot_bytes(int sm_count);   // one per-launch area of the cluster decode
// any N in {64, 256, 1024}, M <= 512, iterates in global memory (decode_tcs.cu)
bool tcs_plan_supported(int n, int m);
size_t tcs_operand_bytes(int n, int m);
size_t tcs_slot_bytes(int sm_count);   // one per-launch area of the streaming decode
cudaError_t launch_tcs_images(const float* a, uint8_t* img, int n, int m, int ea, cudaStream_t s);
bool tcs_supported(const cs_plan* plan);
cudaError_t launch_decode_tcs(const DecodeArgs& d, cudaStream_t s);
// max_ctas > 0 caps the launch's grid (the SMs the cluster kernel leaves idle)
cudaError_t launch_decode_tcs_batch(const DecodeArgs* jobs, int n_jobs, cudaStream_t s,
                                    int max_ctas = 0);
int tcs_ctas_per_sm();
// N in {256, 1024}, M <= 128: A streamed, GEMM1 per 128-coefficient chunk from tensor
// memory, s^{k-1} and s^{k-2} in a slot of the streaming decode's scratch (decode_tcz.cu)
bool tcz_plan_supported(int n, int m);
bool tcz_supported(const cs_plan* plan);
cudaError_t launch_decode_tcz(const DecodeArgs& d, cudaStream_t s);
cudaError_t launch_decode_tcz_batch(const DecodeArgs* jobs, int n_jobs, cudaStream_t s);
// fork streams of a context: 0 .. 2 the on-chip kernel's extra groups, 3 the batched
// streaming launch, 4 the streaming tail of cluster-kernel jobs, 5 (the device's
// highest stream priority) the cluster kernel when it has tails beside it
constexpr int kForkTcGroups = 3, kForkTcs = 3, kForkTc8Tail = 4, kForkTc8Head = 5, kForkStreams = 6;
// The fork stream `which` of the set that belongs to origin stream s.
cudaStream_t fork_stream(const cs_ctx* ctx, cudaStream_t s, int which);

// the device work queue of the serving path (decode_tcs.cu); callers hold ctx->mu
cudaError_t tcsq_create(cs_ctx* ctx);
void tcsq_destroy(cs_ctx* ctx);
bool tcsq_accepts(const DecodeArgs& d);
cudaError_t tcsq_kick(cs_ctx* ctx);
int tcsq_post(cs_ctx* ctx, const DecodeArgs& d, cudaStream_t s, int* slot, unsigned int* seq);
bool tcsq_done(cs_ctx* ctx, int slot, unsigned int seq);
void tcsq_release(cs_ctx* ctx, int slot);

// serving (serving.cu)
void serving_destroy(cs_ctx* ctx);
size_t serving_pool_bytes(const cs_ctx* ctx);   // 0 until the first cs_submit

// metrics (metrics.cu)
cudaError_t launch_psnr(const uint8_t* ref, const float* test, int n_frames, int h, int w,
                        double* out, cudaStream_t s);

// tensor-core operand preparation (decode_tc.cu)
bool tc_plan_supported(int n, int m);
size_t tc_operand_bytes(int n, int m);
cudaError_t launch_tc_ranges(const float* a, const float* phi, int n, int m, float* out,
                             cudaStream_t s);
cudaError_t launch_tc_images(const float* a, uint8_t* img, int n, int m, int ea, cudaStream_t s);

}  // namespace csvc
