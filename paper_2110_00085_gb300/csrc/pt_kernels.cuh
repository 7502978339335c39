// pt_kernels.cuh -- kernel launch interfaces shared between the kernel
// translation units and the C-ABI translation unit.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "pt_device.cuh"

namespace pt {

// unsorted vertex records written by the sampling kernel: slot k of path i
// at k * stride + i; cnt[i] = number of collisions B of path i
struct StoreBuf {
    uint4* rec_a;
    float4* rec_b;
    uint8_t* cnt;
    uint64_t stride;
};

// sorted layout: paths grouped by B (bucket), slot-major inside a bucket;
// record (slot k, rank j) of bucket b at rec_off[b] + k * count[b] + j
struct Buckets {
    uint64_t count[kBuckets];
    uint64_t path_off[kBuckets + 1];
    uint64_t rec_off[kBuckets + 1];
    uint64_t cache_off[kBuckets + 1];   // floats, (event, camera)-major
};

struct SortedPaths {
    const uint4* rec_a;
    const float4* rec_b;
    const Buckets* buckets;   // device
    uint64_t n_max;           // upper bound of stored paths (launch size)
    float inv_norm;
};

void launch_sample(const DevScene& S, const float* beta, uint64_t first, uint64_t n, float inv_norm, uint64_t seed,
                   uint32_t epoch, double* images, double* tallies, uint64_t* fps, const StoreBuf* store,
                   cudaStream_t st);

void launch_sort(const StoreBuf& in, uint64_t n, int n_buckets, uint32_t* blk_hist, Buckets* buckets, int n_cams,
                 uint4* out_a, float4* out_b, cudaStream_t st);

void launch_reweight(const DevScene& S, const SortedPaths& P, const float* beta_t, const float* beta_ref,
                     const float* dbeta, double* images, float* cache, cudaStream_t st);

void launch_grad(const DevScene& S, const SortedPaths& P, const float* beta_t, const float* beta_ref,
                 const float* dbeta, const double* dldi, double* grad, const float* cache, cudaStream_t st);

void launch_delta(const float* a, const float* b, float* out, int64_t n, cudaStream_t st);

// host side (pt_api.cu): record an error message for pt_last_error() and
// return `code`; validate a scene description and derive its constants
// (hc: n_cams cameras, tans: 2 * n_cams half-field tangents x, y)
int fail(int code, const char* fmt, ...);
int describe_scene(const pt_scene_desc* d, DevScene& S, DevCam* hc, double* tans);

}  // namespace pt
