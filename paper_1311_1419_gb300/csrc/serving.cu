// Serving: GOP decode requests from many cameras, admitted as device slots and
// memory free up, run concurrently on the context's streams.
//
// Each request brings host buffers (key frames, measurements, decoded output).
// Admission carves its device working set (key, y and output) out of a pool
// sized by the context's HBM budget, first fit; a request that finds no free
// slot or no room is refused with CS_EAGAIN and retried by the caller.  An
// admitted request is enqueued on the next of the context's streams as
// copy-in, decode, copy-out; the persistent decode kernel takes as many SMs as
// its tiles need, so requests on different streams overlap on the device
// (continuous batching: nothing waits for a batch to fill or to drain).  A
// host callback stamps the completion time; cs_poll reports submit-to-done
// latency and returns the request's memory to the pool.
#include <algorithm>
#include <chrono>
#include <map>
#include <new>

#include "internal.h"

namespace csvc {

namespace {
constexpr size_t kDefaultPool = 1ull << 30;   // 1 GiB when the context has no budget
constexpr size_t kAlign = 256;

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}
size_t round_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
}  // namespace

struct Ticket {
    uint64_t id = 0;
    size_t offset = 0, bytes = 0;
    double submit_ms = 0.0;
    std::atomic<double> done_ms{-1.0};   // stamped by a host callback after the copy-out
    cudaEvent_t done_event = nullptr;
    // posted to the device work queue: the copy-out is enqueued once the job's
    // last tile reports
    bool queued = false, copy_issued = false;
    int qslot = -1;
    unsigned int qseq = 0;
    cudaStream_t stream = nullptr;
    const uint8_t* out_dev = nullptr;
    uint8_t* out_host = nullptr;
    size_t out_b = 0;
};

struct Pool {
    uint8_t* base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_blocks;   // offset -> size

    bool alloc(size_t bytes, size_t* off) {
        for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes;
            const size_t next = it->first + bytes;
            free_blocks.erase(it);
            if (rest) free_blocks[next] = rest;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        auto it = free_blocks.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_blocks.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_blocks.erase(nx);
        }
        if (it != free_blocks.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_blocks.erase(it);
            }
        }
    }
};

namespace {
void CUDART_CB mark_done(void* p) { static_cast<Ticket*>(p)->done_ms.store(now_ms()); }
}  // namespace

size_t serving_pool_bytes(const cs_ctx* ctx) { return ctx->pool ? ctx->pool->size : 0; }

void serving_destroy(cs_ctx* ctx) {
    for (Ticket* t : ctx->live) {
        if (t->done_event) cudaEventDestroy(t->done_event);
        delete t;
    }
    ctx->live.clear();
    if (ctx->pool) {
        cudaFree(ctx->pool->base);
        delete ctx->pool;
        ctx->pool = nullptr;
    }
}

int decode_enqueue(cs_plan* plan, const cs_params* params, const uint8_t* key, const float* y,
                   float* out_f32, uint8_t* out_u8, cudaStream_t stream);
int prepare_decode_args(cs_plan* plan, const cs_params* params, const uint8_t* key, const float* y,
                        float* out_f32, uint8_t* out_u8, DecodeArgs* d, int* engine);
int make_shape(const cs_plan* plan, const cs_params* p, GopShape* gs);

}  // namespace csvc

using namespace csvc;

extern "C" int cs_submit(cs_ctx* ctx, cs_plan* plan, const cs_params* params,
                         const uint8_t* key_host, const float* y_host, uint8_t* frames_u8_host,
                         uint64_t* ticket) {
    if (!ctx || !plan || !params || !ticket || !key_host || !y_host || !frames_u8_host)
        return fail(CS_EINVAL, "null argument");
    if (plan->ctx != ctx) return fail(CS_EINVAL, "plan belongs to another context");
    GopShape gs;
    int st = make_shape(plan, params, &gs);
    if (st) return st;
    const size_t key_b = (size_t)gs.n_gops * gs.h * gs.w;
    const size_t y_b = (size_t)gs.n_cs * gs.nblk * gs.m * sizeof(float);
    const size_t out_b = (size_t)gs.n_cs * gs.h * gs.w;
    const size_t bytes = round_up(key_b) + round_up(y_b) + round_up(out_b);
    std::lock_guard<std::mutex> lock(ctx->mu);
    CS_CUDA_TRY(cudaSetDevice(ctx->device));
    if (!ctx->pool) {
        Pool* p = new (std::nothrow) Pool();
        if (!p) return fail(CS_ENOMEM, "host allocation failed");
        // the budget less the decode kernels' scratch already allocated
        const size_t avail = ctx->hbm_budget > ctx->scratch_bytes ? ctx->hbm_budget - ctx->scratch_bytes : 0;
        p->size = ctx->hbm_budget ? avail / kAlign * kAlign : kDefaultPool;
        if (p->size == 0) {
            delete p;
            return fail(CS_ENOMEM, "the HBM budget is taken by decode scratch");
        }
        cudaError_t e = cudaMalloc(&p->base, p->size);
        if (e != cudaSuccess) {
            delete p;
            return cuda_fail(e, "serving pool");
        }
        p->free_blocks[0] = p->size;
        ctx->pool = p;
    }
    if (bytes > ctx->pool->size) return fail(CS_ENOMEM, "request larger than the HBM budget");
    if ((int)ctx->live.size() >= ctx->max_slots) return fail(CS_EAGAIN, "no free serving slot");
    size_t off = 0;
    if (!ctx->pool->alloc(bytes, &off)) return fail(CS_EAGAIN, "HBM budget exhausted");
    Ticket* t = new (std::nothrow) Ticket();
    if (!t) {
        ctx->pool->release(off, bytes);
        return fail(CS_ENOMEM, "host allocation failed");
    }
    uint8_t* key_dev = ctx->pool->base + off;
    float* y_dev = reinterpret_cast<float*>(key_dev + round_up(key_b));
    uint8_t* out_dev = reinterpret_cast<uint8_t*>(y_dev) + round_up(y_b);
    cudaStream_t s = ctx->streams[ctx->next_stream++ % ctx->streams.size()];
    t->id = ctx->next_ticket++;
    t->offset = off;
    t->bytes = bytes;
    t->submit_ms = now_ms();
    // the device work queue takes the request when the streaming kernel covers it
    DecodeArgs qd;
    int qeng = 0;
    bool queue = ctx->serving_queue &&
                 prepare_decode_args(plan, params, key_dev, y_dev, nullptr, out_dev, &qd, &qeng) == CS_OK &&
                 (params->engine == CS_ENGINE_AUTO || params->engine == CS_ENGINE_TC_STREAM) &&
                 tcsq_accepts(qd);
    cudaError_t e = cudaEventCreateWithFlags(&t->done_event, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemcpyAsync(key_dev, key_host, key_b, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(y_dev, y_host, y_b, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        st = cuda_fail(e, "cs_submit copy-in");
    } else if (queue) {
        st = tcsq_post(ctx, qd, s, &t->qslot, &t->qseq);
        t->queued = st == CS_OK;
        t->stream = s;
        t->out_dev = out_dev;
        t->out_host = frames_u8_host;
        t->out_b = out_b;
    } else {
        st = decode_enqueue(plan, params, key_dev, y_dev, nullptr, out_dev, s);
    }
    if (st == CS_OK && !queue) {
        e = cudaMemcpyAsync(frames_u8_host, out_dev, out_b, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaLaunchHostFunc(s, mark_done, t);
        if (e == cudaSuccess) e = cudaEventRecord(t->done_event, s);
        if (e != cudaSuccess) st = cuda_fail(e, "cs_submit copy-out");
    }
    if (st != CS_OK) {
        // whatever was enqueued still runs; wait for it before releasing its memory
        cudaStreamSynchronize(s);
        if (t->done_event) cudaEventDestroy(t->done_event);
        ctx->pool->release(off, bytes);
        delete t;
        return st;
    }
    ctx->live.push_back(t);
    *ticket = t->id;
    return CS_OK;
}

extern "C" int cs_poll(cs_ctx* ctx, uint64_t ticket, int32_t* done, float* latency_ms) {
    if (!ctx || !done) return fail(CS_EINVAL, "null argument");
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (ctx->tcsq) {
        // a launch of the queue kernel that closed while work was posted: relaunch
        const cudaError_t ke = tcsq_kick(ctx);
        if (ke != cudaSuccess) return cuda_fail(ke, "cs_poll: queue launch");
    }
    for (size_t i = 0; i < ctx->live.size(); ++i) {
        Ticket* t = ctx->live[i];
        if (t->id != ticket) continue;
        if (t->queued && !t->copy_issued) {
            if (!tcsq_done(ctx, t->qslot, t->qseq)) {
                *done = 0;
                return CS_OK;
            }
            // decoded: copy the frames out, then stamp the time
            tcsq_release(ctx, t->qslot);
            t->copy_issued = true;
            cudaError_t ce = cudaMemcpyAsync(t->out_host, t->out_dev, t->out_b, cudaMemcpyDeviceToHost, t->stream);
            if (ce == cudaSuccess) ce = cudaLaunchHostFunc(t->stream, mark_done, t);
            if (ce == cudaSuccess) ce = cudaEventRecord(t->done_event, t->stream);
            if (ce != cudaSuccess) return cuda_fail(ce, "cs_poll copy-out");
            *done = 0;
            return CS_OK;
        }
        cudaError_t e = cudaEventQuery(t->done_event);
        if (e != cudaSuccess && e != cudaErrorNotReady) {
            // the request failed on the device: report it once and retire the ticket
            const int st = cuda_fail(e, "cs_poll");
            ctx->pool->release(t->offset, t->bytes);
            cudaEventDestroy(t->done_event);
            delete t;
            ctx->live.erase(ctx->live.begin() + i);
            return st;
        }
        if (e == cudaErrorNotReady || t->done_ms.load() < 0.0) {
            *done = 0;
            return CS_OK;
        }
        *done = 1;
        if (latency_ms) *latency_ms = (float)(t->done_ms.load() - t->submit_ms);
        ctx->pool->release(t->offset, t->bytes);
        cudaEventDestroy(t->done_event);
        delete t;
        ctx->live.erase(ctx->live.begin() + i);
        return CS_OK;
    }
    return fail(CS_ENOTFOUND, "unknown or retired ticket");
}
