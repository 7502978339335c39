// pt_kernels.cuh -- kernel launch interfaces shared between the kernel
// translation units and the C-ABI translation unit.
#pragma once
#include <nvtx3/nvToolsExt.h>
#include <cstdint>
#include <cuda_runtime.h>

#include "pt_device.cuh"

namespace pt {

// NVTX range over one library call (the pass names profilers show); header
// only, and a no-op unless a tool is attached
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

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
    uint64_t n_events;                  // collision vertices of the stored paths
};

// Collision vertices ("events") of the stored paths, binned by the Morton
// code of their voxel and, with spare bits, of their position inside it:
// neighbouring events share a warp, so their shadow rays to a camera start
// together and run side by side.
struct Events {
    uint4* a;          // {x, y, z bits, packed voxel}
    float4* b;         // {incoming direction, W: path weight before the vertex}
    uint32_t* of_rec;  // event slot of each sorted record (slots >= 1)
    float* val;        // per-event scalar (gradient: sum over cameras of a)
    uint32_t* hist;    // per bin
    uint32_t* cursor;  // per bin: exclusive offsets, then fill positions
    uint32_t* partial; // block sums of the scan
    uint32_t n_bins;
    int bin_bits;      // Morton bits per axis (<= 8: at most 2^24 bins)
    int bin_shift;     // voxel coordinates >> bin_shift give the bin coordinates
    int bin_sub;       // sub-voxel bits per axis appended to the voxel coordinates
    uint64_t cap;      // event capacity
};

struct SortedPaths {
    const uint4* rec_a;
    const float4* rec_b;
    const Buckets* buckets;   // device
    uint64_t n_max;           // upper bound of stored paths (launch size)
    float inv_norm;
};

// ------------------------------------------ stored-path access helpers --
struct PathRef {
    int B;
    uint64_t base;    // record (slot 0)
    uint64_t stride;  // records between slots
};

__device__ __forceinline__ bool locate(const uint64_t* po, const uint64_t* ro, const uint64_t* cnt, int max_orders,
                                       uint64_t j, PathRef& r) {
    for (int b = 1; b <= max_orders; ++b) {
        if (j >= po[b] && j < po[b + 1]) {
            const uint64_t pos = j - po[b];
            r.B = b;
            r.stride = cnt[b];
            r.base = ro[b] + pos;
            return true;
        }
    }
    return false;
}

__device__ __forceinline__ float3 xyz(uint4 a) {
    return make_float3(__uint_as_float(a.x), __uint_as_float(a.y), __uint_as_float(a.z));
}

struct SharedBk {
    uint64_t po[kBuckets + 1], ro[kBuckets + 1], cnt[kBuckets];
};

__device__ __forceinline__ void load_shared(const DevScene& S, const SortedPaths& P, DevCam* cams, SharedBk& sb) {
    for (int c = threadIdx.x; c < S.n_cams; c += blockDim.x) cams[c] = S.cams[c];
    for (int k = threadIdx.x; k <= kBuckets; k += blockDim.x) {
        sb.po[k] = P.buckets->path_off[k];
        sb.ro[k] = P.buckets->rec_off[k];
        if (k < kBuckets) sb.cnt[k] = P.buckets->count[k];
    }
    __syncthreads();
}

void launch_sample(const DevScene& S, const float* beta, uint64_t first, uint64_t n, float inv_norm, uint64_t seed,
                   uint32_t epoch, double* images, double* tallies, uint64_t* fps, const StoreBuf* store,
                   cudaStream_t st);

// counting sort of the stored paths by collision count and, inside a
// count, by the Morton code of the first collision's voxel (kPathBins bins):
// keys, counts and bucket offsets (readable from `buckets` when the stream
// reaches this point), then the scatter of the records into bucket-
// contiguous order.  Scratch: sort_scratch_words(n) 32-bit words.
constexpr uint32_t kPathBins = 4096;
constexpr uint32_t kSortBins = kBuckets * kPathBins;
struct SortScratch {
    uint32_t* keys;      // n
    uint32_t* hist;      // kSortBins
    uint32_t* cursor;    // kSortBins
    uint32_t* partial;   // 3 x 4096 (scan)
    uint32_t* n_zero;    // 1: paths without a collision
};
uint64_t sort_scratch_words(uint64_t n);
SortScratch sort_scratch(uint32_t* base, uint64_t n);
void launch_sort_count(const StoreBuf& in, uint64_t n, int n_buckets, int key_shift, const SortScratch& w,
                       Buckets* buckets, cudaStream_t st);
void launch_sort_scatter(const StoreBuf& in, uint64_t n, const SortScratch& w, Buckets* buckets, uint4* out_a,
                         float4* out_b, cudaStream_t st, const uint32_t* abort = nullptr);
// exclusive scan of n <= 2^24 counts (in -> out); partial: 3 x 4096 words
void launch_scan(const uint32_t* in, uint32_t* out, uint32_t* partial, uint32_t n, cudaStream_t st);
// device-side fit check of a store that does not synchronise: an invalid
// extinction grid (*bad != 0) or more records / events than the kept
// buffers hold empties the bucket table, sets *abort and the error bit
// kErrStore; else *abort = 0
void launch_store_guard(Buckets* buckets, uint64_t rec_cap, uint64_t ev_cap, const uint32_t* bad, uint32_t* abort,
                        int* err, cudaStream_t st);

void launch_events(const DevScene& S, const SortedPaths& P, const Events& E, cudaStream_t st);

void launch_reweight(const DevScene& S, const SortedPaths& P, const Events& E, const float* beta_t,
                     const float* beta_ref, const float* dbeta, double* images, float* cache, cudaStream_t st);

void launch_grad(const DevScene& S, const SortedPaths& P, const Events& E, const float* beta_t,
                 const float* beta_ref, const float* dbeta, const double* dldi, double* grad, const float* cache,
                 cudaStream_t st);

void launch_delta(const float* a, const float* b, float* out, int64_t n, cudaStream_t st);

// ------------------------------------------------------------ batches --
// One scene of a batch: its constants, stored paths, events and the device
// buffers bound for the current step.
struct BatchScene {
    DevScene S;
    SortedPaths P;
    Events E;
    const float* beta_t;
    const float* beta_ref;
    float* dbeta;
    double* images;
    const double* dldi;
    double* grad;
    float* cache;
    int64_t V;
};

// Work-queue state of a batch (device): per pass, tile offsets per scene
// and the item counter.
struct BatchQueue {
    uint32_t* off;       // kBatchPasses x (n + 1)
    uint32_t* counter;   // kBatchPasses
};
constexpr int kBatchPasses = 6;   // delta, path weights, event forward, event grad, path grad, (spare)

// Grouped launches: one ordinary grid per pass over the tiles of up to
// kGroupMax scenes, laid out from host-known upper bounds (stored paths,
// event capacity, voxels).  The table travels as a kernel parameter, so a
// block's scene (found from blockIdx) and every field of it are uniform
// constant-bank reads, as in the single-scene kernels.
constexpr int kGroupMax = 64;
constexpr int kGroupPasses = 5;   // delta, path weights, event forward, event grad, path grad
struct GroupTable {
    int n;
    uint32_t off[kGroupPasses][kGroupMax + 1];   // first block of each scene, per pass
    BatchScene sc[kGroupMax];
};
static_assert(sizeof(GroupTable) <= 32000, "a group table must fit the kernel parameter space");
// tiles of one scene for each pass (upper bounds)
void group_tiles(const BatchScene& s, uint32_t tiles[kGroupPasses]);
void launch_group_reweight(const GroupTable& t, bool cache, int reg_cap, cudaStream_t st);
void launch_group_grad(const GroupTable& t, int reg_cap, cudaStream_t st);

// persistent launches over all scenes: reweight = delta + path weights +
// event forward; grad = event grad + path grad.  blocks = resident blocks;
// reg_cap 1 selects the kernels compiled for 10 resident blocks per SM.
void launch_batch_reweight(const BatchScene* scenes, int n, const BatchQueue& q, bool cache, int reg_cap, int blocks,
                           cudaStream_t st);
void launch_batch_grad(const BatchScene* scenes, int n, const BatchQueue& q, int reg_cap, int blocks,
                       cudaStream_t st);
int batch_blocks_per_sm(int reg_cap);   // occupancy of the slowest-filling pass

// gradient without a contribution cache: per path, re-traces the shadow rays
void launch_grad_reference(const DevScene& S, const SortedPaths& P, const float* beta_t, const float* beta_ref,
                           const float* dbeta, const double* dldi, double* grad, cudaStream_t st);

// host side (pt_api.cu): record an error message for pt_last_error() and
// return `code`; validate a scene description and derive its constants
// (hc: n_cams cameras, tans: 2 * n_cams half-field tangents x, y)
int fail(int code, const char* fmt, ...);
int device_sms();                               // SMs of the current device (cached per device)
const DevCam* scene_cams(const pt_scene* sc);   // device camera table of a scene
const float* scene_omega(const pt_scene* sc);   // device pixel solid angles of a scene
int describe_scene(const pt_scene_desc* d, DevScene& S, DevCam* hc, double* tans);

}  // namespace pt
