// pt_batch.cu -- many scenes of uneven size in one launch per pass, two
// schedules over the same tiles (128 paths, 128 events or 1024 voxels; the
// tile bodies are the single-scene ones, pt_event_ops.cuh):
//   persistent: a device table holds one descriptor per scene (constants,
//     stored paths, events, the buffers bound for the step); a small kernel
//     turns each scene's device-side counts into tile offsets; resident
//     blocks then pull (scene, tile) items from an atomic counter until the
//     queue is empty, keeping the descriptor and camera table of their
//     current scene in shared memory.  No block waits on another: the queue
//     is a plain fetch-and-add.
//   grouped: one block per tile of every scene, the descriptors passed as a
//     kernel parameter; a block finds its scene from blockIdx, so the
//     descriptor's fields are uniform constant-bank reads and need no
//     registers of their own, and the hardware block scheduler balances the
//     load.  Tiles past a scene's actual count exit at once.
#include "pt_event_ops.cuh"

namespace pt {

namespace {

constexpr int kTileThreads = 128;
constexpr int kVoxPerThread = 8;
enum Pass : int { kPassDelta = 0, kPassWeights = 1, kPassForward = 2, kPassGrad = 3, kPassPathGrad = 4 };

__global__ void k_batch_tiles(const BatchScene* __restrict__ sc, int n, uint32_t* __restrict__ off) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    uint32_t acc[kBatchPasses] = {0, 0, 0, 0, 0, 0};
    for (int p = 0; p < kBatchPasses; ++p) off[p * (n + 1)] = 0;
    for (int s = 0; s < n; ++s) {
        const uint64_t ev = sc[s].P.buckets->n_events;
        const uint64_t paths = sc[s].P.buckets->path_off[kBuckets];
        const uint64_t vox = (uint64_t)sc[s].V;
        const uint32_t t_ev = (uint32_t)((ev + kTileThreads - 1) / kTileThreads);
        const uint32_t t_path = (uint32_t)((paths + kTileThreads - 1) / kTileThreads);
        const uint32_t t_vox = (uint32_t)((vox + kTileThreads * kVoxPerThread - 1) / (kTileThreads * kVoxPerThread));
        const uint32_t t[kBatchPasses] = {t_vox, t_path, t_ev, t_ev, t_path, 0};
        for (int p = 0; p < kBatchPasses; ++p) {
            acc[p] += t[p];
            off[p * (n + 1) + s + 1] = acc[p];
        }
    }
}

// scene holding item t: off[s] <= t < off[s + 1]
__device__ __forceinline__ int scene_of(const uint32_t* off, int n, uint32_t t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// MINB: minimum resident blocks per SM the compiler must allow (1: its own
// register allocation; larger values cap registers per thread, trading a few
// spills for more resident warps -- an autotuning knob)
template <int PASS, bool CACHE, int MINB>
__global__ void __launch_bounds__(kTileThreads, MINB) k_batch(const BatchScene* __restrict__ sc, int n,
                                                        const uint32_t* __restrict__ off_all,
                                                        uint32_t* __restrict__ counter) {
    __shared__ BatchScene B;
    __shared__ DevCam cams[kMaxCams];
    __shared__ SharedBk sb;
    __shared__ uint32_t s_item;
    const uint32_t* off = off_all + PASS * (n + 1);
    const uint32_t total = off[n];
    int cur = -1;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter + PASS, 1u);
        __syncthreads();
        const uint32_t t = s_item;
        if (t >= total) break;
        const int s = scene_of(off, n, t);
        if (s != cur) {
            if (threadIdx.x == 0) B = sc[s];
            __syncthreads();
            for (int c = threadIdx.x; c < B.S.n_cams; c += blockDim.x) cams[c] = B.S.cams[c];
            load_buckets(B.P, sb);
            __syncthreads();
            cur = s;
        }
        const uint64_t base = (uint64_t)(t - off[s]) * kTileThreads;
        if (PASS == kPassDelta) {
            const uint64_t v0 = base * kVoxPerThread;
            for (int k = 0; k < kVoxPerThread; ++k) {
                const uint64_t v = v0 + (uint64_t)k * kTileThreads + threadIdx.x;
                if (v < (uint64_t)B.V) B.dbeta[v] = B.beta_t[v] - B.beta_ref[v];
            }
        } else if (PASS == kPassWeights) {
            path_weights_one(B.S, B.P, B.E, sb, base + threadIdx.x, B.beta_t, B.beta_ref, B.dbeta);
        } else if (PASS == kPassForward) {
            event_forward_one<CACHE>(B.S, cams, B.E, B.P.inv_norm, B.P.buckets->n_events, base + threadIdx.x,
                                     B.beta_t, B.beta_ref, B.images, B.cache);
        } else if (PASS == kPassGrad) {
            event_grad_warp(B.S, cams, B.E, B.P.buckets->n_events, base + threadIdx.x, B.beta_t, B.dldi, B.grad,
                            B.cache);
        } else if (PASS == kPassPathGrad) {
            path_grad_one(B.S, B.P, B.E, sb, base + threadIdx.x, B.beta_t, B.grad);
        }
        __syncthreads();
    }
}

// scene of block b in a grouped launch: off[s] <= b < off[s + 1]
__device__ __forceinline__ int group_scene(const uint32_t* off, int n, uint32_t b) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int PASS, bool CACHE, int MINB>
__global__ void __launch_bounds__(kTileThreads, MINB) k_group(const __grid_constant__ GroupTable T) {
    __shared__ DevCam cams[kMaxCams];
    __shared__ SharedBk sb;
    const int s = group_scene(T.off[PASS], T.n, blockIdx.x);
    const BatchScene& B = T.sc[s];
    const uint64_t base = (uint64_t)(blockIdx.x - T.off[PASS][s]) * kTileThreads;
    if (PASS == kPassDelta) {
        const uint64_t v0 = base * kVoxPerThread;
        for (int k = 0; k < kVoxPerThread; ++k) {
            const uint64_t v = v0 + (uint64_t)k * kTileThreads + threadIdx.x;
            if (v < (uint64_t)B.V) B.dbeta[v] = B.beta_t[v] - B.beta_ref[v];
        }
    } else if (PASS == kPassWeights || PASS == kPassPathGrad) {
        if (base >= B.P.n_max) return;
        load_buckets(B.P, sb);
        __syncthreads();
        if (PASS == kPassWeights)
            path_weights_one(B.S, B.P, B.E, sb, base + threadIdx.x, B.beta_t, B.beta_ref, B.dbeta);
        else
            path_grad_one(B.S, B.P, B.E, sb, base + threadIdx.x, B.beta_t, B.grad);
    } else {
        const uint32_t n_events = B.P.buckets->n_events;
        if (base >= n_events) return;   // tiles past the actual events (capacity layout)
        load_cams(B.S, cams);
        if (PASS == kPassForward)
            event_forward_one<CACHE>(B.S, cams, B.E, B.P.inv_norm, n_events, base + threadIdx.x, B.beta_t,
                                     B.beta_ref, B.images, B.cache);
        else
            event_grad_warp(B.S, cams, B.E, n_events, base + threadIdx.x, B.beta_t, B.dldi, B.grad, B.cache);
    }
}

// reg_cap 1: per pass, the resident blocks of 128 threads per SM that the
// single-scene kernel of the pass reaches with the compiler's allocation
// (path weights 56 registers -> 9, event forward 48 -> 10, event gradient
// 54 -> 9); the delta and path-gradient passes are left alone
template <int PASS>
constexpr int cap_blocks() {
    return PASS == kPassWeights ? 9 : PASS == kPassForward ? 16 : PASS == kPassGrad ? 9 : 1;
}

template <int PASS, bool CACHE>
void run_group(const GroupTable& t, int reg_cap, cudaStream_t st) {
    const unsigned g = t.off[PASS][t.n];
    if (g == 0) return;
    if (reg_cap)
        k_group<PASS, CACHE, cap_blocks<PASS>()><<<g, kTileThreads, 0, st>>>(t);
    else
        k_group<PASS, CACHE, 1><<<g, kTileThreads, 0, st>>>(t);
}

template <int PASS, bool CACHE>
void run(const BatchScene* scenes, int n, const BatchQueue& q, int reg_cap, int blocks, cudaStream_t st) {
    if (reg_cap)
        k_batch<PASS, CACHE, cap_blocks<PASS>()><<<blocks, kTileThreads, 0, st>>>(scenes, n, q.off, q.counter);
    else
        k_batch<PASS, CACHE, 1><<<blocks, kTileThreads, 0, st>>>(scenes, n, q.off, q.counter);
}

template <int PASS, bool CACHE, int MINB>
int occ() {
    int a = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_batch<PASS, CACHE, MINB>, kTileThreads, 0);
    return a;
}

template <bool CAP>
int occupancy() {
    const int v[5] = {occ<kPassForward, true, CAP ? cap_blocks<kPassForward>() : 1>(),
                      occ<kPassForward, false, CAP ? cap_blocks<kPassForward>() : 1>(),
                      occ<kPassGrad, false, CAP ? cap_blocks<kPassGrad>() : 1>(),
                      occ<kPassWeights, false, CAP ? cap_blocks<kPassWeights>() : 1>(),
                      occ<kPassPathGrad, false, CAP ? cap_blocks<kPassPathGrad>() : 1>()};
    int m = v[0];
    for (int x : v) m = (x > 0 && x < m) ? x : m;
    return m > 0 ? m : 1;
}

}  // namespace

int batch_blocks_per_sm(int reg_cap) { return reg_cap ? occupancy<true>() : occupancy<false>(); }

void group_tiles(const BatchScene& s, uint32_t tiles[kGroupPasses]) {
    const uint64_t paths = (s.P.n_max + kTileThreads - 1) / kTileThreads;
    const uint64_t ev = (s.E.cap + kTileThreads - 1) / kTileThreads;
    const uint64_t vox = ((uint64_t)s.V + kTileThreads * kVoxPerThread - 1) / (kTileThreads * kVoxPerThread);
    tiles[kPassDelta] = (uint32_t)vox;
    tiles[kPassWeights] = (uint32_t)paths;
    tiles[kPassForward] = (uint32_t)ev;
    tiles[kPassGrad] = (uint32_t)ev;
    tiles[kPassPathGrad] = (uint32_t)paths;
}

void launch_group_reweight(const GroupTable& t, bool cache, int reg_cap, cudaStream_t st) {
    run_group<kPassDelta, false>(t, reg_cap, st);
    run_group<kPassWeights, false>(t, reg_cap, st);
    if (cache)
        run_group<kPassForward, true>(t, reg_cap, st);
    else
        run_group<kPassForward, false>(t, reg_cap, st);
}

void launch_group_grad(const GroupTable& t, int reg_cap, cudaStream_t st) {
    run_group<kPassGrad, false>(t, reg_cap, st);
    run_group<kPassPathGrad, false>(t, reg_cap, st);
}

void launch_batch_reweight(const BatchScene* scenes, int n, const BatchQueue& q, bool cache, int reg_cap, int blocks,
                           cudaStream_t st) {
    cudaMemsetAsync(q.counter, 0, sizeof(uint32_t) * kBatchPasses, st);
    k_batch_tiles<<<1, 32, 0, st>>>(scenes, n, q.off);
    run<kPassDelta, false>(scenes, n, q, reg_cap, blocks, st);
    run<kPassWeights, false>(scenes, n, q, reg_cap, blocks, st);
    if (cache)
        run<kPassForward, true>(scenes, n, q, reg_cap, blocks, st);
    else
        run<kPassForward, false>(scenes, n, q, reg_cap, blocks, st);
}

void launch_batch_grad(const BatchScene* scenes, int n, const BatchQueue& q, int reg_cap, int blocks,
                       cudaStream_t st) {
    cudaMemsetAsync(q.counter, 0, sizeof(uint32_t) * kBatchPasses, st);
    k_batch_tiles<<<1, 32, 0, st>>>(scenes, n, q.off);
    run<kPassGrad, false>(scenes, n, q, reg_cap, blocks, st);
    run<kPassPathGrad, false>(scenes, n, q, reg_cap, blocks, st);
}

}  // namespace pt
