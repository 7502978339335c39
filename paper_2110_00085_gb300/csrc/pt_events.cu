// pt_events.cu -- the recycled passes over stored paths, split by what each
// step depends on (Sec. 5.2 estimator, Sec. 4.4 path score).
//
// A stored path's weight before each of its collisions depends on its
// earlier vertices (the correction factor of Eq. 20 multiplies along the
// path), but a collision's local estimates toward the cameras depend only
// on that weight, the collision point and the current extinction.  So:
//   per path  : flights and vertex ratios -> the weight W_e before event e;
//               for the gradient, suffix sums S_e over the events' A_e,
//               flight scatters -S_e l and scattering-vertex terms;
//   per event : shadow rays toward every camera (transmittance, pixel add,
//               optional cache) and, for the gradient, shadow-ray scatters
//               -a l and local-estimate vertex terms, A_e = sum_d a.
// Paths are fixed for N_r steps, so events are binned once per store by the
// Morton code of their voxel (the paper's path sorting applied to collision
// points): the 32 events of a warp lie close together -- events of one voxel
// on adjacent lanes -- so their shadow rays to one camera start together, run
// nearly parallel through the same voxels (shared cache lines) and end at
// nearly the same box exit.
#include "pt_event_ops.cuh"

namespace pt {

namespace {


__global__ void __launch_bounds__(128) k_ev_hist(DevScene S, SortedPaths P, Events E) {
    const int max_orders = S.max_orders;
    __shared__ SharedBk sb;
    for (int k = threadIdx.x; k <= kBuckets; k += blockDim.x) {
        sb.po[k] = P.buckets->path_off[k];
        sb.ro[k] = P.buckets->rec_off[k];
        if (k < kBuckets) sb.cnt[k] = P.buckets->count[k];
    }
    __syncthreads();
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    PathRef pr;
    if (!locate(sb.po, sb.ro, sb.cnt, max_orders, j, pr)) return;
    for (int e = 1; e <= pr.B; ++e)
        atomicAdd(E.hist + event_bin(S, E, P.rec_a[pr.base + (uint64_t)e * pr.stride]), 1u);
}

__global__ void __launch_bounds__(128) k_ev_scatter(DevScene S, SortedPaths P, Events E) {
    const int max_orders = S.max_orders;
    __shared__ SharedBk sb;
    for (int k = threadIdx.x; k <= kBuckets; k += blockDim.x) {
        sb.po[k] = P.buckets->path_off[k];
        sb.ro[k] = P.buckets->rec_off[k];
        if (k < kBuckets) sb.cnt[k] = P.buckets->count[k];
    }
    __syncthreads();
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    PathRef pr;
    if (!locate(sb.po, sb.ro, sb.cnt, max_orders, j, pr)) return;
    for (int e = 1; e <= pr.B; ++e) {
        const uint64_t rec = pr.base + (uint64_t)e * pr.stride;
        const uint4 a = P.rec_a[rec];
        const float4 b = P.rec_b[rec];
        const uint32_t pos = atomicAdd(E.cursor + event_bin(S, E, a), 1u);
        E.a[pos] = make_uint4(a.x, a.y, a.z, a.w & kVoxMask);
        E.b[pos] = make_float4(b.x, b.y, b.z, 0.0f);
        E.of_rec[rec] = pos;
    }
}

// exclusive scan of n counts (in -> out), three levels of at most 4096
constexpr int kScanItems = 4096;
__global__ void __launch_bounds__(1024) k_scan_blocks(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                      uint32_t* __restrict__ partial, uint32_t n) {
    __shared__ uint32_t s[1024];
    const uint32_t base = blockIdx.x * kScanItems + threadIdx.x * 4;
    uint32_t v[4], t = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = base + k < n ? in[base + k] : 0u;
        t += v[k];
    }
    s[threadIdx.x] = t;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const uint32_t x = threadIdx.x >= (unsigned)off ? s[threadIdx.x - off] : 0u;
        __syncthreads();
        s[threadIdx.x] += x;
        __syncthreads();
    }
    uint32_t run = s[threadIdx.x] - t;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 1023) partial[blockIdx.x] = s[1023];
}
__global__ void __launch_bounds__(1024) k_scan_add(uint32_t* __restrict__ out, const uint32_t* __restrict__ offs,
                                                   uint32_t n) {
    const uint32_t base = blockIdx.x * kScanItems + threadIdx.x * 4;
    const uint32_t o = offs[blockIdx.x];
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (base + k < n) out[base + k] += o;
}

// ------------------------------------------------ single-scene kernels --
__global__ void __launch_bounds__(128) k_path_weights(DevScene S, SortedPaths P, Events E,
                                                      const float* __restrict__ beta_t,
                                                      const float* __restrict__ beta_ref,
                                                      const float* __restrict__ dbeta) {
    __shared__ SharedBk sb;
    load_buckets(P, sb);
    __syncthreads();
    path_weights_one(S, P, E, sb, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, beta_t, beta_ref, dbeta);
}

__global__ void __launch_bounds__(128) k_path_grad(DevScene S, SortedPaths P, Events E,
                                                   const float* __restrict__ beta_t, double* __restrict__ grad) {
    __shared__ SharedBk sb;
    load_buckets(P, sb);
    __syncthreads();
    path_grad_one(S, P, E, sb, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, beta_t, grad);
}

template <bool CACHE>
// 16 resident blocks per SM (32 registers, a few spilled bytes): the extra warps
// hide the beta gathers' latency (97.9 -> 94.9 ms at 2^24 paths, 15 cameras)
__global__ void __launch_bounds__(128, 16) k_event_forward(DevScene S, SortedPaths P, Events E,
                                                       const float* __restrict__ beta_t,
                                                       const float* __restrict__ beta_ref,
                                                       double* __restrict__ images, float* __restrict__ cache) {
    __shared__ DevCam cams[kMaxCams];
    load_cams(S, cams);
    event_forward_one<CACHE>(S, cams, E, P.inv_norm, P.buckets->n_events,
                             (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, beta_t, beta_ref, images, cache);
}

__global__ void __launch_bounds__(128) k_event_grad(DevScene S, SortedPaths P, Events E,
                                                    const float* __restrict__ beta_t,
                                                    const double* __restrict__ dldi, double* __restrict__ grad,
                                                    const float* __restrict__ cache) {
    __shared__ DevCam cams[kMaxCams];
    load_cams(S, cams);
    event_grad_warp(S, cams, E, P.buckets->n_events, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, beta_t, dldi,
                    grad, cache);
}


unsigned blocks(uint64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

void launch_scan(const uint32_t* in, uint32_t* out, uint32_t* partial, uint32_t n, cudaStream_t st) {
    if (n == 0) return;
    const uint32_t nb = (n + kScanItems - 1) / kScanItems;   // <= 4096 for n <= 2^24
    k_scan_blocks<<<nb, 1024, 0, st>>>(in, out, partial, n);
    k_scan_blocks<<<1, 1024, 0, st>>>(partial, partial + kScanItems, partial + 2 * kScanItems, nb);
    k_scan_add<<<nb, 1024, 0, st>>>(out, partial + kScanItems, n);
}

void launch_events(const DevScene& S, const SortedPaths& P, const Events& E, cudaStream_t st) {
    const unsigned g = blocks(P.n_max, 128);
    if (g == 0) return;
    cudaMemsetAsync(E.hist, 0, sizeof(uint32_t) * E.n_bins, st);
    k_ev_hist<<<g, 128, 0, st>>>(S, P, E);
    launch_scan(E.hist, E.cursor, E.partial, E.n_bins, st);
    k_ev_scatter<<<g, 128, 0, st>>>(S, P, E);
}

void launch_reweight(const DevScene& S, const SortedPaths& P, const Events& E, const float* beta_t,
                     const float* beta_ref, const float* dbeta, double* images, float* cache, cudaStream_t st) {
    const unsigned gp = blocks(P.n_max, 128);
    const unsigned ge = blocks(E.cap, 128);
    if (gp == 0 || ge == 0) return;
    k_path_weights<<<gp, 128, 0, st>>>(S, P, E, beta_t, beta_ref, dbeta);
    if (cache)
        k_event_forward<true><<<ge, 128, 0, st>>>(S, P, E, beta_t, beta_ref, images, cache);
    else
        k_event_forward<false><<<ge, 128, 0, st>>>(S, P, E, beta_t, beta_ref, images, nullptr);
}

void launch_grad(const DevScene& S, const SortedPaths& P, const Events& E, const float* beta_t,
                 const float* beta_ref, const float* dbeta, const double* dldi, double* grad, const float* cache,
                 cudaStream_t st) {
    if (!cache) {
        launch_grad_reference(S, P, beta_t, beta_ref, dbeta, dldi, grad, st);
        return;
    }
    const unsigned gp = blocks(P.n_max, 128);
    const unsigned ge = blocks(E.cap, 128);
    if (gp == 0 || ge == 0) return;
    k_event_grad<<<ge, 128, 0, st>>>(S, P, E, beta_t, dldi, grad, cache);
    k_path_grad<<<gp, 128, 0, st>>>(S, P, E, beta_t, grad);
}

}  // namespace pt
