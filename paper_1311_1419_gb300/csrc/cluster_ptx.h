// Cluster helpers of the 32 x 32 tensor-core decodes: cluster indices, the
// distributed-shared-memory address map, cluster barriers, copies and stores
// into a peer CTA's shared memory, 16-bit packing, and the layout rules the
// two cluster kernels share (which CTA owns which measurement rows, where
// element (block, row) of the MN-major P operand lives).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace csvc {
namespace tc {

constexpr int kCl8 = 8;   // CTAs per cluster of the 32 x 32 decodes

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_id() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t n_clusters() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa(uint32_t saddr, uint32_t rank) {
    uint32_t d;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(saddr), "r"(rank));
    return d;
}
// Every thread of every CTA of the cluster; global and shared writes before it
// are visible to every thread of the cluster after it.
__device__ __forceinline__ void cluster_sync() {
    asm volatile(
        "fence.acq_rel.gpu;\n\t"
        "barrier.cluster.arrive.release.aligned;\n\t"
        "barrier.cluster.wait.acquire.aligned;\n\t"
        "fence.acq_rel.gpu;" ::: "memory");
}
__device__ __forceinline__ void st_async_u32(uint32_t raddr, uint32_t v, uint32_t rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(
                     raddr),
                 "r"(v), "r"(rbar)
                 : "memory");
}
// Bulk copy of this CTA's shared memory into a peer's (addresses from mapa),
// completion counted in bytes on the peer's barrier.
__device__ __forceinline__ void bulk_s2peer(uint32_t rdst, uint32_t src, uint32_t bytes, uint32_t rbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            rdst),
        "r"(src), "r"(bytes), "r"(rbar)
        : "memory");
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
template <bool BF>
__device__ __forceinline__ uint16_t pack1(float v) {
    if constexpr (BF) {
        __nv_bfloat16 h = __float2bfloat16_rn(v);
        return *reinterpret_cast<uint16_t*>(&h);
    } else {
        __half h = __float2half_rn(v);
        return *reinterpret_cast<uint16_t*>(&h);
    }
}
template <bool BF>
__device__ __forceinline__ float unpack1(uint16_t v) {
    if constexpr (BF) {
        return __bfloat162float(*reinterpret_cast<__nv_bfloat16*>(&v));
    } else {
        return __half2float(*reinterpret_cast<__half*>(&v));
    }
}
__device__ __forceinline__ float2 u2f2(uint32_t a, uint32_t b) {
    return make_float2(__uint_as_float(a), __uint_as_float(b));
}


// Owner of measurement rows: the m16 / 8 row groups are dealt to the 8 CTAs,
// the first (groups % 8) CTAs taking one more.
__device__ __forceinline__ void owner_rows(int p, int m16, int* row0, int* rows) {
    const int groups = m16 / 8, base = groups / kCl8, extra = groups % kCl8;
    const int ng = base + (p < extra ? 1 : 0);
    const int g0 = p * base + (p < extra ? p : extra);
    *row0 = 8 * g0;
    *rows = 8 * ng;
}
// Owner of measurement row m (inverse of owner_rows).
__device__ __forceinline__ int owner_of(int m, int m16) {
    const int groups = m16 / 8, base = groups / kCl8, extra = groups % kCl8;
    const int g = m >> 3, big = extra * (base + 1);
    return g < big ? g / (base + 1) : extra + (g - big) / base;
}
// Slot of sender s in receiver r's incoming buffers (s != r): 0 .. 6.
__device__ __forceinline__ int slot_of(int s, int r) { return (s - r + kCl8 - 1) % kCl8; }

// Byte offset of P[b][m] in the MN-major operand: 8-row groups 2 KB apart, two
// 64-block atoms of 1 KB in each, 128-byte swizzle inside the atom.
__device__ __forceinline__ uint32_t p_off(uint32_t b, uint32_t m) {
    return (m >> 3) * 2048u + (b >> 6) * 1024u + (m & 7u) * 128u + ((((b & 63u) >> 3) ^ (m & 7u)) << 4) +
           ((b & 7u) << 1);
}


}  // namespace tc
}  // namespace csvc
