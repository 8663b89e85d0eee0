// cs_lambda_max_noalloc: lambda_max(Phi Phi^T) without any device allocation.
//
// Some callers cannot call cudaMalloc: a serving process whose device memory
// was all reserved at start-up and must stay inside that reservation, or a
// latency-critical loop that cannot afford the implicit device-wide
// synchronisation cudaMalloc/cudaFree may trigger.  cs_make_phi allocates a
// Gram-matrix scratch buffer for its power iteration; this entry point runs
// the same two kernels with that scratch in a file-scope device array instead.
//
// The array holds the M x M FP64 Gram matrix for M <= kNoAllocMaxM (256), i.e.
// 512 KB, and every GPU that loads this library keeps it until the process
// exits.  All calls share it: the Gram kernel writes every entry the power
// iteration reads, so nothing needs clearing between calls, but calls whose
// work overlaps on the GPU (different streams, or different host threads)
// race on it and must be serialised by the caller.
#include <mutex>

#include "internal.h"

namespace csvc {
namespace {

constexpr int kNoAllocMaxM = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_gram_scratch[kNoAllocMaxM * kNoAllocMaxM];

std::mutex g_scratch_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of g_gram_scratch in the current device's context.  In host
// code the symbol itself is only a host-side stand-in, so the address is looked
// up once per device with that device current.
int scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cs_lambda_max_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(CS_ENODEV, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_gram_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cs_lambda_max_noalloc: cudaGetSymbolAddress");
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return CS_OK;
}

}  // namespace
}  // namespace csvc

using namespace csvc;

extern "C" int cs_lambda_max_noalloc(const float* phi_dev, int32_t n, int32_t m,
                                     double* lambda_max_dev, cs_stream_t stream) {
    if (!phi_dev || !lambda_max_dev) return fail(CS_EINVAL, "null pointer");
    if (n < 1 || n > kMaxN) return fail(CS_EINVAL, "N must be in [1, 4096]");
    if (m < 1 || m > n) return fail(CS_EINVAL, "need 1 <= M <= N");
    if (m > kNoAllocMaxM)
        return fail(CS_EINVAL,
                    "M exceeds 256, the size of the built-in scratch of cs_lambda_max_noalloc");
    double* scratch = nullptr;
    int st = scratch_address(&scratch);
    if (st != CS_OK) return st;
    cudaError_t e = launch_lambda_max(phi_dev, n, m, scratch, lambda_max_dev, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cs_lambda_max_noalloc launch");
    return CS_OK;
}
