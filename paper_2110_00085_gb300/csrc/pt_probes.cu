// pt_probes.cu -- memory-rate probes (include/pt_probes.h): each kernel runs
// one access pattern of the recycled passes alone, so that a pass's achieved
// rate has a measured denominator on the device it runs on.
//   gather  : random 4-byte loads (the extinction gathers of shadow rays and
//             flights; an 8 MB grid stays in L2)
//   red f64 : FP64 reductions resolved in L2 (the gradient's adds), at
//             random distinct addresses, 32 consecutive doubles per warp,
//             or one address per warp
//   red f32 : the same with FP32 terms (for comparison)
//   copy    : 16-byte streaming copy (the stored records come from HBM)
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/pathrecycle.h"
#include "../../include/pt_probes.h"
#include "pt_kernels.cuh"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kUnroll = 8;   // independent accesses in flight per thread

// per-thread index sequence: x <- a x + c (mod 2^32); the high bits index
__device__ __forceinline__ uint32_t lcg(uint32_t x) { return x * 1664525u + 1013904223u; }
__device__ __forceinline__ uint32_t mix(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) k_probe(void* __restrict__ buf, int shift, uint32_t mask,
                                                         int64_t iters, float* __restrict__ sink) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t warp = tid >> 5;
    const uint32_t lane = threadIdx.x & 31u;
    // random kinds index with the sequence's high bits (shift = 32 - log2 n);
    // the warp-shared kinds draw one sequence per warp
    uint32_t x = mix(KIND == PT_PROBE_RED_F64_WARP || KIND == PT_PROBE_RED_F64_SAME ? warp : tid);
    float acc = 0.0f;
    for (int64_t it = 0; it < iters; it += kUnroll) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            x = lcg(x);
            const uint32_t r = (x >> shift) & mask;
            if (KIND == PT_PROBE_GATHER_F32) {
                acc += __ldg(static_cast<const float*>(buf) + r);
            } else if (KIND == PT_PROBE_RED_F64) {
                atomicAdd(static_cast<double*>(buf) + r, 1.0);
            } else if (KIND == PT_PROBE_RED_F64_WARP) {
                atomicAdd(static_cast<double*>(buf) + ((r & ~31u) | lane), 1.0);
            } else if (KIND == PT_PROBE_RED_F64_SAME) {
                atomicAdd(static_cast<double*>(buf) + r, 1.0);
            } else if (KIND == PT_PROBE_RED_F32) {
                atomicAdd(static_cast<float*>(buf) + r, 1.0f);
            }
        }
    }
    if (KIND == PT_PROBE_GATHER_F32) sink[tid] = acc;
}

// shared-memory atomics (the accumulation a block could do before its
// FP64 reductions leave the SM): a table of 16 KB per block
template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) k_probe_shared(float* __restrict__ out, int64_t iters) {
    constexpr int kSlots = KIND == PT_PROBE_SHARED_F64 ? 2048 : 4096;
    __shared__ __align__(16) unsigned char tab_raw[16384];
    float* tf = reinterpret_cast<float*>(tab_raw);
    uint32_t* tu = reinterpret_cast<uint32_t*>(tab_raw);
    double* td = reinterpret_cast<double*>(tab_raw);
    for (int i = threadIdx.x; i < 4096; i += blockDim.x) tu[i] = 0u;
    __syncthreads();
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    // RUN4: the four lanes of a group draw the same sequence
    uint32_t x = mix(KIND == PT_PROBE_SHARED_F32_RUN4 ? (tid >> 2) : tid);
    for (int64_t it = 0; it < iters; it += kUnroll) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            x = lcg(x);
            const uint32_t r = (x >> 20) & (uint32_t)(kSlots - 1);
            if (KIND == PT_PROBE_SHARED_F32 || KIND == PT_PROBE_SHARED_F32_RUN4)
                atomicAdd(tf + r, 1.0f);
            else if (KIND == PT_PROBE_SHARED_U32)
                atomicAdd(tu + r, 1u);
            else
                atomicAdd(td + r, 1.0);
        }
    }
    __syncthreads();
    out[tid] = tf[threadIdx.x];
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_copy(float4* __restrict__ dst,
                                                              const float4* __restrict__ src, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __ldcs(src + i);
}

}  // namespace

extern "C" int pt_probe(int kind, void* buf, int64_t n, const void* src, int64_t iters, int blocks, float* sink,
                        void* stream) {
    if (kind < 0 || kind >= PT_PROBE_KINDS) return pt::fail(PT_E_INVALID, "pt_probe: unknown kind %d", kind);
    if (!buf || n < 1) return pt::fail(PT_E_INVALID, "pt_probe: null buffer or empty size");
    if (blocks < 1 || blocks > (1 << 20)) return pt::fail(PT_E_INVALID, "pt_probe: blocks must be in 1..2^20");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (kind >= PT_PROBE_SHARED_F32) {
        if (n < (int64_t)blocks * kProbeThreads)
            return pt::fail(PT_E_INVALID, "pt_probe: shared probes need blocks * 256 output floats");
        if (iters < 1 || iters > (1 << 24)) return pt::fail(PT_E_INVALID, "pt_probe: iters must be in 1..2^24");
        const int64_t it = (iters + kUnroll - 1) / kUnroll * kUnroll;
        float* o = static_cast<float*>(buf);
        switch (kind) {
            case PT_PROBE_SHARED_F32: k_probe_shared<PT_PROBE_SHARED_F32><<<blocks, kProbeThreads, 0, st>>>(o, it); break;
            case PT_PROBE_SHARED_F32_RUN4:
                k_probe_shared<PT_PROBE_SHARED_F32_RUN4><<<blocks, kProbeThreads, 0, st>>>(o, it);
                break;
            case PT_PROBE_SHARED_U32: k_probe_shared<PT_PROBE_SHARED_U32><<<blocks, kProbeThreads, 0, st>>>(o, it); break;
            default: k_probe_shared<PT_PROBE_SHARED_F64><<<blocks, kProbeThreads, 0, st>>>(o, it); break;
        }
    } else if (kind == PT_PROBE_COPY) {
        if (!src) return pt::fail(PT_E_INVALID, "pt_probe: copy needs a source");
        k_probe_copy<<<blocks, kProbeThreads, 0, st>>>(static_cast<float4*>(buf), static_cast<const float4*>(src),
                                                       n);
    } else {
        if (n < 32 || n > ((int64_t)1 << 31) || (n & (n - 1)))
            return pt::fail(PT_E_INVALID, "pt_probe: n must be a power of two in 32..2^31");
        if (iters < 1 || iters > (1 << 24)) return pt::fail(PT_E_INVALID, "pt_probe: iters must be in 1..2^24");
        if (kind == PT_PROBE_GATHER_F32 && !sink) return pt::fail(PT_E_INVALID, "pt_probe: gather needs a sink");
        int lg = 0;
        while (((int64_t)1 << lg) < n) ++lg;
        const int shift = 32 - lg;
        const uint32_t mask = (uint32_t)(n - 1);
        const int64_t it = (iters + kUnroll - 1) / kUnroll * kUnroll;
        switch (kind) {
            case PT_PROBE_GATHER_F32:
                k_probe<PT_PROBE_GATHER_F32><<<blocks, kProbeThreads, 0, st>>>(buf, shift, mask, it, sink);
                break;
            case PT_PROBE_RED_F64:
                k_probe<PT_PROBE_RED_F64><<<blocks, kProbeThreads, 0, st>>>(buf, shift, mask, it, nullptr);
                break;
            case PT_PROBE_RED_F64_WARP:
                k_probe<PT_PROBE_RED_F64_WARP><<<blocks, kProbeThreads, 0, st>>>(buf, shift, mask, it, nullptr);
                break;
            case PT_PROBE_RED_F64_SAME:
                k_probe<PT_PROBE_RED_F64_SAME><<<blocks, kProbeThreads, 0, st>>>(buf, shift, mask, it, nullptr);
                break;
            default:
                k_probe<PT_PROBE_RED_F32><<<blocks, kProbeThreads, 0, st>>>(buf, shift, mask, it, nullptr);
                break;
        }
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return pt::fail(PT_E_CUDA, "pt_probe launch: %s", cudaGetErrorString(e));
    return PT_OK;
}
