/*
 * csvc.h -- C ABI of the GB300 (sm_103a) library for the hot path of the
 * multiple-residual compressive-sensing (CS) surveillance video codec of
 * Yu, Qiao, Luo and Yang, "Increasing compression ratio of low complexity
 * compressive sensing video encoder with application-aware configurable
 * mechanism" (arXiv 1311.1419).
 *
 * A video is split into GOPs of G frames: one key frame followed by G-1 CS
 * frames (Sec. 3, Sec. 3.1).  Every CS frame subtracts the SAME key frame of
 * its GOP (the multiple-residual scheme, Sec. 3.2), and each residual is
 * measured block by block with one Gaussian random matrix Phi (M x N,
 * N = B*B pixels per block): y_b = Phi r_b (Sec. 3.1, Sec. 4).  The decoder
 * recovers every residual block by solving Eq. (1), read here as
 * min_s 1/2 ||A s - y||^2 + lambda ||s||_1 with A = Phi Psi and Psi the
 * orthonormal 2-D DCT of the block, by a fixed number of FISTA iterations,
 * then adds it back to the key frame (Eq. 4).  Key frames are passed raw.
 *
 * Conventions for every call:
 *  - Pointers named *_dev are device pointers on the context's GPU (for
 *    example from torch.empty(..., device="cuda").data_ptr()); pointers named
 *    *_host are host memory.  The caller owns all frame, measurement and
 *    output buffers; the library owns contexts, plans and their device memory.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *    that take a stream only enqueue work on it and return; the caller
 *    synchronises.  Calls without a stream return after their work is done.
 *  - Frames are uint8 [F][H][W], row-major, no row padding.  Measurements are
 *    float32 [n_cs][nblk][M]: CS frame, then block in raster order over the
 *    zero-padded grid of ceil(H/B) x ceil(W/B) blocks, then measurement row.
 *    Inside a block, pixel (p, q) is vector entry p*B + q.
 *  - Every call returns a cs_status: 0 on success, a negative CS_E* code
 *    otherwise; no exception or abort crosses the ABI.  On error nothing has
 *    been enqueued unless the code is CS_ECUDA (see cs_last_error()).
 */
#ifndef CSVC_H
#define CSVC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;                     /* cudaStream_t == struct CUstream_st* */
typedef struct CUstream_st* cs_stream_t;

typedef struct cs_ctx cs_ctx;
typedef struct cs_plan cs_plan;

/* status codes */
#define CS_OK 0
#define CS_EINVAL (-1)     /* bad argument: shape, size, null pointer, plan mismatch */
#define CS_ENOMEM (-2)     /* device allocation failed or HBM budget exceeded */
#define CS_EAGAIN (-3)     /* serving admission refused for now: retry later */
#define CS_ETIMEDOUT (-4)  /* a bounded device-side wait gave up */
#define CS_ECUDA (-5)      /* a CUDA runtime call or kernel launch failed */
#define CS_ENOTFOUND (-6)  /* unknown serving ticket */
#define CS_ENODEV (-7)     /* no usable sm_103 device */

/* arithmetic of the recovery (cs_params.precision) */
#define CS_FP32 0          /* FP32-grade products: FP32 SIMT, or FP16 hi+lo split on tensor cores */
#define CS_BF16 1          /* BF16 A and iterate, FP32 accumulate, FP32-grade tail iterations */
#define CS_BF16X2 2        /* split-BF16 A (hi+lo), BF16 iterate, FP32-grade tail iterations */
#define CS_FP16 3          /* FP16 A and iterate (scaled), FP32-grade tail iterations */

/* decode kernel (cs_params.engine) */
#define CS_ENGINE_AUTO 0   /* the autotuned engine of the (N, M) (cs_autotune), else CS_ENGINE_TC
                            * if the shape allows it, else CS_ENGINE_TC_STREAM, else plain */
#define CS_ENGINE_PLAIN 1  /* one CTA per block, FP32 SIMT: the plain baseline */
#define CS_ENGINE_TC 2     /* persistent tcgen05 kernel with the iterates on chip: N = 256 or
                            * 1024 with M <= 128; CS_EINVAL for any other shape */
#define CS_ENGINE_TC_STREAM 3  /* persistent tcgen05 kernel with A streamed from L2 and the
                                * iterates in global memory: N = 64, 256 or 1024 with
                                * M <= 512; CS_EINVAL for any other shape */
#define CS_ENGINE_TC_CHUNK 4   /* persistent tcgen05 kernel with A streamed from L2, GEMM1 in
                                * 128-coefficient chunks from tensor memory and only the last
                                * two iterates s in global memory: N = 256 or 1024 with
                                * M <= 128; CS_EINVAL for any other shape */

/* Codec parameters of one encode/decode call (Sec. 3.1: "GOP size and
 * measurement matrix size" are the encoder's configuration). */
typedef struct cs_params {
    int32_t height, width;    /* frame size in pixels, >= 1 */
    int32_t gop;              /* G: frames per GOP including the key frame, >= 2 */
    int32_t n_gops;           /* consecutive GOPs handled by one call; 0 means 1 */
    int32_t block;            /* B: block side; B*B must equal the plan's N */
    int32_t m;                /* M: measurements per block; must equal the plan's M */
    int32_t iters;            /* K: FISTA iterations (fixed count, no early stop), >= 0 */
    int32_t fp32_tail_iters;  /* last iterations run FP32-grade when precision != CS_FP32 */
    float lambda_rel;         /* lambda_b = lambda_rel * ||A^T y_b||_inf, >= 0 (0.01 default) */
    int32_t precision;        /* CS_FP32, CS_BF16, CS_BF16X2 or CS_FP16 */
    int32_t engine;           /* CS_ENGINE_* */
} cs_params;

/* ---- context ------------------------------------------------------------
 * cs_ctx_create: bind a context to CUDA device `device` (must be sm_103).
 * hbm_budget_bytes caps the device memory of serving and of the decode
 * kernels' scratch (0 = no cap): the scratch rings (allocated with the first
 * plan whose shape needs them) take at most half of the budget and what the
 * serving pool leaves; a ring that does not fit is not allocated, and shapes
 * that would use it decode on another kernel.  The serving pool (allocated at
 * the first cs_submit) gets the budget less the scratch allocated by then (1 GiB
 * with no budget).  *out receives the context; destroy it with cs_ctx_destroy
 * after every plan made from it has been destroyed. */
int cs_ctx_create(cs_ctx** out, int device, size_t hbm_budget_bytes);
int cs_ctx_destroy(cs_ctx* ctx);
/* cs_ctx_status: synchronise the context's device, then report CS_ETIMEDOUT
 * (and clear the condition) if a kernel of this context gave up one of its
 * bounded device-side waits since the last call: its outputs are incomplete.
 * Otherwise CS_OK.  The context stays usable either way. */
int cs_ctx_status(cs_ctx* ctx);
/* cs_ctx_set_debug: test hooks for the failure path, consumed by the next
 * launch of the context's tensor-core decodes (CS_ENGINE_TC with N = 256 or
 * 1024, CS_ENGINE_TC_STREAM, CS_ENGINE_TC_CHUNK, or either tensor-core TV
 * kernel of cs_decode_gop_tv).  CS_DEBUG_DROP_ARRIVAL makes one
 * warp of that launch withhold one barrier arrival, so that a device-side wait
 * runs out (after 1 s): the launch then drains, its outputs are incomplete and
 * cs_ctx_status reports CS_ETIMEDOUT; the context stays usable.  No GPU fault
 * is involved. */
#define CS_DEBUG_DROP_ARRIVAL 1
int cs_ctx_set_debug(cs_ctx* ctx, int32_t flags);

/* ---- plans: Phi, A = Phi Psi and the FISTA step --------------------------
 * cs_make_phi: build the plan for blocks of N = B*B pixels and M measurements
 * (1 <= M <= N <= 4096, N a perfect square) under `seed`, entirely on the
 * device.  Phi (Sec. 3.1, Sec. 4: a Gaussian random matrix) has entries
 * N(0, 1/M): pair q of row-major entries (2q, 2q+1) is Box-Muller of the
 * Philox4x64-10 block with counter (q, (N << 16) | M, 0, 0) and key (seed, 0),
 * u1 = ((x0 >> 11) + 1) 2^-53, u2 = (x1 >> 11) 2^-53, each entry divided by
 * sqrt(M) in double and rounded to float; the result is bit-identical on
 * every device.  The plan also holds A = Phi Psi (float32 [M][N], formed in
 * FP64), the tensor-core operand copies of A, the DCT matrix and
 * L = 1.0001 * lambda_max(Phi Phi^T) from 1000 FP64 power iterations.
 * Returns after the plan is complete.  A plan is immutable: any number of
 * streams may use it at once. */
int cs_make_phi(cs_ctx* ctx, int32_t n, int32_t m, uint64_t seed, cs_plan** out);
int cs_plan_destroy(cs_plan* plan);
/* Borrowed device pointers (valid until cs_plan_destroy): Phi and A, float32
 * [M][N] row-major.  *lipschitz receives L. */
int cs_plan_phi(const cs_plan* plan, const float** phi_dev);
int cs_plan_a(const cs_plan* plan, const float** a_dev);
int cs_plan_lipschitz(const cs_plan* plan, double* lipschitz);

/* ---- encode (Sec. 3.1) ----------------------------------------------------
 * frames_dev: uint8 [n_gops*G][H][W]; frame t of the call is a key frame when
 * t % G == 0.  y_dev: float32 [n_gops*(G-1)][nblk][M] with
 * nblk = ceil(H/B) * ceil(W/B).  For CS frame t the residual is
 * int(F_t) - int(F_key), key = floor(t/G)*G, zero outside the frame, and
 * y_b = Phi r_b with FP32-grade products (exact residuals, FP32 accumulation). */
int cs_encode_gop(cs_plan* plan, const cs_params* params, const uint8_t* frames_dev,
                  float* y_dev, cs_stream_t stream);
/* cs_encode_batch: cs_encode_gop for n_plans plans (any M, one block size)
 * over the same clip: params[i] must all describe the same clip (height,
 * width, gop, n_gops, block), y_dev[i] is plan i's output.  The plans the
 * tensor-core encode takes share one launch (several when their M add up to
 * more than one launch holds), which reads the clip once.  Each y is FP32-grade
 * like cs_encode_gop's and equal to it up to FP32 rounding (the hi and lo
 * products of a plan may be summed in another order when the launch is
 * crowded); the same call always gives the same bytes.  Host arrays, device
 * buffers; CS_EINVAL when the calls differ in their clip. */
int cs_encode_batch(cs_ctx* ctx, int32_t n_plans, cs_plan* const* plans, const cs_params* params,
                    const uint8_t* frames_dev, float* const* y_dev, cs_stream_t stream);

/* ---- decode (Sec. 3.2, Eqs. 1-4) ------------------------------------------
 * key_dev: uint8 [n_gops][H][W] (the key frame of each GOP); y_dev as written
 * by cs_encode_gop.  Per block: lambda_b = lambda_rel ||A^T y_b||_inf,
 * s^0 = z^1 = 0, t_1 = 1, K iterations of
 *   s^k = soft(z^k - A^T(A z^k - y_b)/L, lambda_b/L),
 *   z^{k+1} = s^k + ((t_k - 1)/t_{k+1})(s^k - s^{k-1}),
 * then F'_t = F_key + Psi s^K cropped to H x W.  frames_f32_dev: float32
 * [n_gops*(G-1)][H][W] or NULL; frames_u8_dev: uint8, same shape, clamp of
 * round-half-even, or NULL (at least one must be non-NULL).
 * CS_ENGINE_TC_CHUNK: a call of 32 x 32 blocks with more 128-block tiles than the
 * device has SMs, whose last round would hold at most four rounds of the
 * CS_ENGINE_TC kernel's co-resident clusters, has its first (tiles mod SMs)
 * tiles decoded by that kernel and the rest by the chunked one, one after the
 * other on the stream; the split depends on the call and the device only. */
int cs_decode_gop(cs_plan* plan, const cs_params* params, const uint8_t* key_dev,
                  const float* y_dev, float* frames_f32_dev, uint8_t* frames_u8_dev,
                  cs_stream_t stream);

/* ---- batched decode ---------------------------------------------------------
 * cs_decode_batch: decode n_jobs GOP calls (cs_decode_gop semantics, job i =
 * plans[i], params[i], key_dev[i], y_dev[i], frames_f32_dev[i] and
 * frames_u8_dev[i]; the two output arrays may be NULL, or hold NULL entries)
 * as one persistent tensor-core launch per kernel and operand type: plans of
 * different N and M and calls of different frame size, GOP size, iteration
 * count and precision share the SMs, each CTA taking the next 128-block tile.
 * All plans belong to ctx.  Jobs no tensor-core kernel covers (or that ask for
 * CS_ENGINE_PLAIN) run on the plain kernel on the same stream.  Results are
 * identical to decoding each job alone.  Host arrays, device buffers. */
int cs_decode_batch(cs_ctx* ctx, int32_t n_jobs, cs_plan* const* plans, const cs_params* params,
                    const uint8_t* const* key_dev, const float* const* y_dev,
                    float* const* frames_f32_dev, uint8_t* const* frames_u8_dev,
                    cs_stream_t stream);

/* cs_decode_gop_tv: the same call as cs_decode_gop with the paper's own
 * regulariser: every residual block r is recovered by total-variation
 * minimisation, Eq. 1 with Phi(x) = ||D r||_1 (the TVAL3 decoder of Sec. 4),
 * min ||D r||_1 s.t. Phi r = y, D the forward differences along the block's
 * rows and columns (zero at its last column / row), by the augmented
 * Lagrangian / alternating-direction scheme: per iteration one shrinkage step
 * of the splitting variable w = D r, one gradient step of length
 * 1 / (8 beta + mu L) for r (L = the plan's Lipschitz constant) and one update
 * of each multiplier; params->iters iterations from zero.  beta and mu are the
 * penalties of the splitting and of the measurement constraint (0.125 and 1
 * suit 8-bit residuals).  FP32-grade results; params->precision must be
 * CS_FP32 and lambda_rel is not used.  Engines (both tensor-core kernels put
 * the two Phi products of an iteration on tcgen05, three fp16 MMAs per K step):
 * - CS_ENGINE_TC: the on-chip kernel (Phi resident in shared memory, the
 *   multiplier state in the context's streaming-decode scratch); 16 x 16
 *   blocks with M <= 128 only, CS_EINVAL for any other shape;
 * - CS_ENGINE_TC_STREAM: the streaming kernel (Phi streamed from L2, the
 *   iterate and multipliers in a per-SM state area of about 4.3 MB that the
 *   context allocates on first use, within its scratch budget); N = 64, 256 or
 *   1024 with M <= 512, CS_EINVAL for any other shape, CS_ENOMEM when the
 *   state area cannot be had;
 * - CS_ENGINE_AUTO: the on-chip kernel where it applies, else the streaming
 *   one, else (or when the state area cannot be had) the plain kernel;
 * - CS_ENGINE_PLAIN: the plain per-block FP32 kernel.
 * Buffers and errors as cs_decode_gop; CS_EINVAL for beta or mu <= 0. */
int cs_decode_gop_tv(cs_plan* plan, const cs_params* params, float beta, float mu,
                     const uint8_t* key_dev, const float* y_dev, float* frames_f32_dev,
                     uint8_t* frames_u8_dev, cs_stream_t stream);

/* cs_autotune: pick the decode's launch shape for the plan's (N, M) by timing
 * the candidates on the device: the on-chip tensor-core kernel where the
 * shape has one (16 x 16 and 32 x 32 blocks, M <= 128), the streaming
 * tensor-core kernel where it has one (8 x 8, 16 x 16 and 32 x 32 blocks,
 * M <= 512), the chunked one where it has one (16 x 16 and 32 x 32 blocks,
 * M <= 128), and the plain FP32 kernel at 64,
 * 128, 256, 512 and 1024 threads per CTA with 1, 2, 4, 8 or 16 (up to 512
 * threads) measured blocks per CTA (the blocks of a CTA share each load of A;
 * shapes whose shared memory exceeds 200 KB are skipped; after its default shape
 * the plain sweep stops when that is more than 4x slower than a tensor-core
 * kernel of the shape).  Each runs a synthetic call (random
 * measurements, zero key, two tiles of 128 blocks per SM up to 40 M pixels,
 * 16 iterations, FP32: the throughput of a call that fills the GPU); the
 * fastest is recorded in ctx for this (N, M) and used from then on by
 * decodes whose engine is CS_ENGINE_AUTO (an explicit engine still wins; mixed
 * precision takes the recorded engine when it is a tensor-core kernel, else the
 * default order, which always gives it a tensor-core kernel).  Synchronises the
 * device: call it before serving or before capturing decodes into a CUDA
 * graph.  Outputs (each may be NULL): the chosen engine (CS_ENGINE_TC,
 * CS_ENGINE_TC_STREAM, CS_ENGINE_TC_CHUNK or CS_ENGINE_PLAIN), the plain kernel's threads and
 * blocks per CTA (0 for the tensor-core kernels) and the measured time per
 * block per iteration in ns.
 * The paper has no counterpart (its decoder is a MATLAB solver). */
int cs_autotune(cs_ctx* ctx, cs_plan* plan, int32_t* engine, int32_t* plain_threads,
                int32_t* plain_blocks_per_cta, float* ns_per_block_iter);

/* ---- quality and compression accounting (Sec. 4, Table I) ----------------
 * cs_psnr: per-frame PSNR 10 log10(255^2 / MSE) of test_dev (float32
 * [n][H][W]) against ref_dev (uint8 [n][H][W]), FP64 reductions on the device;
 * psnr_dev: double [n]; +inf where the frames are identical. */
int cs_psnr(const uint8_t* ref_dev, const float* test_dev, int32_t n_frames,
            int32_t height, int32_t width, double* psnr_dev, cs_stream_t stream);
/* Total CR of a GOP of 1 key + (G-1) CS frames, G / (1/cr_key + (G-1)/cr_cs):
 * the closed form behind Table I.  Returns NaN for G < 1 or non-positive CRs. */
double cs_total_cr(int32_t gop, double cr_key, double cr_cs);
/* CR of one GOP with a raw key frame: G*H*W / (H*W + (G-1)*nblk*M). */
double cs_raw_key_cr(int32_t gop, int32_t height, int32_t width, int32_t block, int32_t m);

/* ---- serving --------------------------------------------------------------
 * cs_submit: enqueue the decode of one request (cs_decode_gop semantics,
 * uint8 output) from HOST buffers: key_host uint8 [n_gops][H][W], y_host float32
 * [n_cs][nblk][M], frames_u8_host uint8 [n_cs][H][W] (the output).  Use pinned
 * memory for overlap; the buffers must stay valid until cs_poll reports done.
 * Admission takes one of the context's slots (64) and carves the request's
 * device working set (key + y + output) out of a device pool of
 * hbm_budget_bytes (1 GiB if the context was created with 0), first fit; when
 * either is exhausted the call returns CS_EAGAIN and enqueues nothing (a
 * request larger than the whole pool returns CS_ENOMEM).  Admitted requests
 * run on the context's streams and overlap on the device.  *ticket identifies
 * the request.
 * With the device work queue (the default, see cs_ctx_set_serving), a request
 * the streaming tensor-core decode covers (N = 64, 256 or 1024 with M <= 512;
 * CS_FP32 or CS_FP16; engine CS_ENGINE_AUTO or CS_ENGINE_TC_STREAM; the
 * context's decode scratch allocated, see cs_ctx_create) is not launched on its
 * own: once its inputs are on the device its tiles join a queue in device-
 * visible memory, which one persistent launch of that kernel drains, so tiles
 * of every request in flight share the SMs as they arrive (continuous
 * batching).  The launch ends itself after 20 ms without work and is started
 * again by the next cs_submit or cs_poll.  Its results are bit for bit those of
 * cs_decode_gop with CS_ENGINE_TC_STREAM.  Any other request runs as its own
 * decode launch on the context's streams.
 * cs_poll: non-blocking; *done = 1 once the output is in frames_u8_host, then
 * *latency_ms is the submit-to-completion time, the request's device memory
 * and slot are released and the ticket is retired.  Call it often: it also
 * restarts the queue's launch when work is waiting.  A request whose decode
 * gave up a bounded device wait still completes; cs_ctx_status reports it. */
int cs_submit(cs_ctx* ctx, cs_plan* plan, const cs_params* params, const uint8_t* key_host,
              const float* y_host, uint8_t* frames_u8_host, uint64_t* ticket);
int cs_poll(cs_ctx* ctx, uint64_t ticket, int32_t* done, float* latency_ms);
/* cs_ctx_set_serving: how cs_submit runs requests from now on: CS_SERVING_QUEUE
 * (the device work queue where it applies; the default) or CS_SERVING_LAUNCH
 * (one decode launch per request, on the kernel cs_decode_gop would pick).
 * The paper has no counterpart (its decoder is offline). */
#define CS_SERVING_LAUNCH 0
#define CS_SERVING_QUEUE 1
int cs_ctx_set_serving(cs_ctx* ctx, int32_t mode);

/* ---- the whole codec of a clip, host memory in and out ------------------------
 * cs_codec_host: encode a clip and decode it again under n_plans plans, from
 * and to HOST memory (Sec. 3: key + CS frames per GOP; Sec. 3.1: every CS
 * frame's residual measured per block; Sec. 3.2, Eqs. 1-4: every residual block
 * recovered and added back to its key; Sec. 4: PSNR of the decoded frames).
 * clip_host: uint8 [n_gops*G][H][W]; every params[i] must give the same H, W,
 * G and n_gops, and its block and M must match plans[i].  The clip is copied to
 * the device once; each plan measures it as cs_encode_gop does; all plans'
 * measurements are decoded in one cs_decode_batch call (results identical to
 * cs_decode_gop); each decoded CS frame is scored against the original with
 * cs_psnr.  Outputs per plan i: frames_u8_host[i], uint8 [n_gops*(G-1)][H][W]
 * (the decoded CS frames in clip order, keys left out), and psnr_host[i],
 * double [n_gops*(G-1)].  Device staging belongs to the context: one buffer
 * that grows with the largest call so far (a cudaMalloc, after the previous
 * call using it has finished); calls on different streams take turns on it.
 * Enqueues on `stream` and returns; the host buffers must stay valid until the
 * stream has passed the call (pinned memory makes the copies asynchronous).
 * Errors as the calls it makes; CS_EINVAL for mismatched shapes. */
int cs_codec_host(cs_ctx* ctx, int32_t n_plans, cs_plan* const* plans, const cs_params* params,
                  const uint8_t* clip_host, uint8_t* const* frames_u8_host,
                  double* const* psnr_host, cs_stream_t stream);

/* ---- allocation-free Lipschitz estimate -------------------------------------
 * The paper has no counterpart to this call; it is a service for callers that
 * must not allocate device memory: a serving process whose HBM was reserved
 * in full at start-up, or a latency-critical loop that cannot take the
 * device-wide synchronisation cudaMalloc/cudaFree may cause.
 * cs_lambda_max_noalloc computes lambda_max(Phi Phi^T) of phi_dev (float32
 * [M][N], for example cs_plan_phi's pointer) by the same FP64 Gram matrix and
 * 1000 power iterations cs_make_phi uses, and writes it to lambda_max_dev (one
 * device double; the plan's L is 1.0001 times this value).  It calls no
 * cudaMalloc, cudaFree or allocating library routine: the M x M Gram matrix
 * lives in a 512 KB array inside the library, which every GPU that loads the
 * library holds until the process exits.  Limits: 1 <= M <= min(N, 256),
 * N <= 4096; larger sizes return CS_EINVAL and enqueue nothing.  The first call
 * on each device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.
 * Every call shares the one array, so calls whose work overlaps on the GPU
 * race and must be serialised by the caller.  Enqueues on `stream` and
 * returns. */
int cs_lambda_max_noalloc(const float* phi_dev, int32_t n, int32_t m, double* lambda_max_dev,
                          cs_stream_t stream);

/* ---- errors --------------------------------------------------------------- */
const char* cs_strerror(int status);
/* Detail of the last failure on the calling thread (empty if none). */
const char* cs_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CSVC_H */
