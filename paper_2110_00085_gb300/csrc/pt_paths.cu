// pt_paths.cu -- stored light paths: the path sort (Sec. 5.3), the recycled
// forward pass and the gradient pass over sorted paths (Sec. 5.2, Sec. 4.4).
//
// Sort: stable counting sort of paths by their number of collisions B
// (histogram per block -> per-bucket scan over blocks -> scatter), so that
// the 32 lanes of a warp always hold paths of equal size (the paper's path
// sorting, which lets every lane run the same number of events).
//
// Recycled forward (Eq. forward_simualtion_recycling): for each stored event
// b the contribution under the current extinction M_t, times the correction
// factor mu(x|M_t)/mu(x|M_ref) of its sub-path, which factorises into
//   exp(-sum_v (beta_t - beta_ref)_v l_v) per flight   (transmittances)
//   albedo_ref(x_k) f_s,t(x_k, mu_k) / f_s,ref(x_k, mu_k) per vertex k < b
// over the plain (albedo-product) weight.  Gradient (Eq.
// gradient_simualtion_recycling with the PSF of Sec. 4.4): per event and
// camera a = dL/dI[pixel] * contribution; the shadow ray scatters -a * l_v,
// the vertex adds a * h(x_b, mu_bd); per flight k the suffix sum
// S_k = sum_{b >= k} A_b scatters -S_k * l_v and vertex k adds
// h(x_k, mu_k) * S_{k+1}, with h = albedo_c f^c / f_s.
#include "pt_kernels.cuh"

namespace pt {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;

// ------------------------------------------------------------ sort ------
__device__ __forceinline__ void warp_bucket_counts(uint32_t b, uint32_t (*wc)[kBuckets], uint32_t& rank) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t peers = __match_any_sync(0xffffffffu, b);
    rank = __popc(peers & ((1u << lane) - 1u));
    if (lane == __ffs(peers) - 1 && b < (uint32_t)kBuckets) wc[warp][b] = __popc(peers);
}

__global__ void __launch_bounds__(kSortThreads) k_sort_count(const uint8_t* __restrict__ cnt, uint64_t n,
                                                             uint32_t* __restrict__ blk_hist, uint32_t nblk) {
    __shared__ uint32_t wc[kSortWarps][kBuckets];
    for (int k = threadIdx.x; k < kSortWarps * kBuckets; k += blockDim.x) (&wc[0][0])[k] = 0;
    __syncthreads();
    const uint64_t i = (uint64_t)blockIdx.x * kSortThreads + threadIdx.x;
    const uint32_t b = i < n ? (uint32_t)cnt[i] : 0xffu;
    uint32_t rank;
    warp_bucket_counts(b, wc, rank);
    __syncthreads();
    if (threadIdx.x < kBuckets) {
        uint32_t s = 0;
        for (int w = 0; w < kSortWarps; ++w) s += wc[w][threadIdx.x];
        blk_hist[(uint64_t)threadIdx.x * nblk + blockIdx.x] = s;
    }
}

// exclusive scan of one bucket's per-block counts (in place); count -> Buckets
__global__ void __launch_bounds__(1024) k_sort_scan(uint32_t* __restrict__ blk_hist, uint32_t nblk,
                                                    Buckets* __restrict__ bk) {
    __shared__ uint64_t part[1024];
    uint32_t* h = blk_hist + (uint64_t)blockIdx.x * nblk;
    const uint32_t chunk = (nblk + 1023) / 1024;
    const uint32_t a = threadIdx.x * chunk, e = min(a + chunk, nblk);
    uint64_t s = 0;
    for (uint32_t j = a; j < e; ++j) s += h[j];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const uint64_t v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint64_t run = part[threadIdx.x] - s;   // exclusive prefix of this chunk
    for (uint32_t j = a; j < e; ++j) {
        const uint32_t v = h[j];
        h[j] = (uint32_t)run;
        run += v;
    }
    if (threadIdx.x == 1023) bk->count[blockIdx.x] = part[1023];
}

__global__ void k_bucket_offsets(Buckets* bk, int n_buckets) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    uint64_t p = 0, r = 0, ev = 0;
    for (int b = 0; b < kBuckets; ++b) {
        const uint64_t n = (b >= 1 && b < n_buckets) ? bk->count[b] : 0;   // B = 0 paths are not stored
        if (b >= n_buckets) bk->count[b] = 0;
        bk->path_off[b] = p;
        bk->rec_off[b] = r;
        p += n;
        r += n * (uint64_t)(b + 1);
        ev += n * (uint64_t)b;
    }
    bk->path_off[kBuckets] = p;
    bk->rec_off[kBuckets] = r;
    bk->n_events = ev;
}

__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(StoreBuf in, uint64_t n, const uint32_t* __restrict__ blk_off,
                                                               uint32_t nblk, const Buckets* __restrict__ bk,
                                                               uint4* __restrict__ out_a, float4* __restrict__ out_b,
                                                               const uint32_t* __restrict__ abort) {
    if (abort && *abort) return;   // block-uniform: the store did not fit (nothing is written)
    __shared__ uint32_t wc[kSortWarps][kBuckets];
    __shared__ uint32_t wp[kSortWarps][kBuckets];
    for (int k = threadIdx.x; k < kSortWarps * kBuckets; k += blockDim.x) (&wc[0][0])[k] = 0;
    __syncthreads();
    const uint64_t i = (uint64_t)blockIdx.x * kSortThreads + threadIdx.x;
    const uint32_t b = i < n ? (uint32_t)in.cnt[i] : 0xffu;
    uint32_t rank;
    warp_bucket_counts(b, wc, rank);
    __syncthreads();
    if (threadIdx.x < kBuckets) {
        uint32_t run = 0;
        for (int w = 0; w < kSortWarps; ++w) {
            wp[w][threadIdx.x] = run;
            run += wc[w][threadIdx.x];
        }
    }
    __syncthreads();
    if (i >= n || b == 0 || b >= (uint32_t)kBuckets) return;
    const uint64_t pos = (uint64_t)blk_off[(uint64_t)b * nblk + blockIdx.x] + wp[threadIdx.x >> 5][b] + rank;
    const uint64_t cb = bk->count[b], ro = bk->rec_off[b];
    for (uint32_t k = 0; k <= b; ++k) {
        const uint64_t src = (uint64_t)k * in.stride + i;
        const uint64_t dst = ro + (uint64_t)k * cb + pos;
        out_a[dst] = in.rec_a[src];
        out_b[dst] = in.rec_b[src];
    }
}

// gradient without a contribution cache (reference form): per path,
// phase 1 re-traces every shadow ray for its transmittance, scatters it at
// once and adds the local-estimate vertex term; phase 2 walks the stored
// flights backwards with the suffix sums S_k.
__global__ void __launch_bounds__(128) k_grad(DevScene S, SortedPaths P, const float* __restrict__ beta_t,
                                              const float* __restrict__ beta_ref, const float* __restrict__ dbeta,
                                              const double* __restrict__ dldi, double* __restrict__ grad) {
    __shared__ DevCam cams[kMaxCams];
    __shared__ SharedBk sb;
    load_shared(S, P, cams, sb);
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    PathRef pr;
    if (!locate(sb.po, sb.ro, sb.cnt, S.max_orders, j, pr)) return;
    float Aev[kMaxOrders + 1];
    uint4 a0 = P.rec_a[pr.base];
    float3 xp = xyz(a0);
    uint32_t pvp = a0.w & kVoxMask;
    float w = S.w0;
    float4 bin = P.rec_b[pr.base + pr.stride];
    // ---- phase 1: events (shadow rays and local-estimate vertex terms) ----
    for (int e = 1; e <= pr.B; ++e) {
        const uint4 ra = P.rec_a[pr.base + (uint64_t)e * pr.stride];
        const float3 om = make_float3(bin.x, bin.y, bin.z);
        const float3 x = xyz(ra);
        const uint32_t pv = ra.w & kVoxMask;
        if (!vox_ok(S, pv) || !vox_ok(S, pvp)) {
            atomicOr(S.err, kErrRecord);
            return;
        }
        const int v = lin_vox(S, pv);
        const float bct = __ldg(beta_t + v), bcr = __ldg(beta_ref + v);
        const float btr = bcr + S.beta_air;
        const float W = w * expf(-delta_depth(S, dbeta, xp, om, pvp, bin.w));
        float A = 0.0f;
        for (int c = 0; c < S.n_cams; ++c) {
            const Proj q = project(cams[c], x);
            if (q.pix < 0) continue;
            const int gp = cams[c].off + q.pix;
            const float mu = dot3(om, q.dir);
            const float T = expf(-optical_depth_to_exit(S, beta_t, x, q.dir, pv, nullptr));
            const float ev = local_contrib(W, fs_medium(S, bct, mu), btr, T, q.r2, __ldg(S.omega + gp), P.inv_norm);
            if (ev == 0.0f) continue;
            const float a = (float)__ldg(dldi + gp) * ev;
            if (a == 0.0f) continue;
            A += a;
            scatter_ray(S, grad, x, q.dir, pv, __int_as_float(0x7f800000), a);
            red_add(grad + v, a * score_vertex(S, bct, mu));
        }
        Aev[e] = A;
        if (e < pr.B) {
            const float4 bnext = P.rec_b[pr.base + (uint64_t)(e + 1) * pr.stride];
            const float mu = om.x * bnext.x + om.y * bnext.y + om.z * bnext.z;
            const float fsr = fs_medium(S, bcr, mu);
            if (fsr == 0.0f) {
                w = 0.0f;
            } else {
                const float albr = (S.alb_c * bcr + S.alb_a * S.beta_air) / btr;
                w = W * (albr * (fs_medium(S, bct, mu) / fsr));
                if (e >= S.rr_start) w *= S.inv_q;
            }
            bin = bnext;
        }
        xp = x;
        pvp = pv;
    }
    // ---- phase 2: flights and scattering vertices, suffix sums ----
    float Ssum = 0.0f;
    for (int e = pr.B; e >= 1; --e) {
        const uint4 ra = P.rec_a[pr.base + (uint64_t)e * pr.stride];
        const float4 be = P.rec_b[pr.base + (uint64_t)e * pr.stride];
        if (e < pr.B && Ssum != 0.0f) {
            // vertex e: angle between the flight into it and the flight out
            const float4 bn = P.rec_b[pr.base + (uint64_t)(e + 1) * pr.stride];
            const float mu = be.x * bn.x + be.y * bn.y + be.z * bn.z;
            const int v = lin_vox(S, ra.w & kVoxMask);
            red_add(grad + v, Ssum * score_vertex(S, __ldg(beta_t + v), mu));
        }
        Ssum += Aev[e];
        if (Ssum != 0.0f) {
            const uint4 rp = P.rec_a[pr.base + (uint64_t)(e - 1) * pr.stride];
            scatter_ray(S, grad, xyz(rp), make_float3(be.x, be.y, be.z), rp.w & kVoxMask, be.w, Ssum);
        }
    }
}

__global__ void k_delta(const float* __restrict__ a, const float* __restrict__ b, float* __restrict__ out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i] - b[i];
}

unsigned blocks_for(uint64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

void launch_sort_count(const StoreBuf& in, uint64_t n, int n_buckets, uint32_t* blk_hist, Buckets* buckets,
                       cudaStream_t st) {
    const uint32_t nblk = blocks_for(n, kSortThreads);
    k_sort_count<<<nblk, kSortThreads, 0, st>>>(in.cnt, n, blk_hist, nblk);
    k_sort_scan<<<kBuckets, 1024, 0, st>>>(blk_hist, nblk, buckets);
    k_bucket_offsets<<<1, 32, 0, st>>>(buckets, n_buckets);
}

void launch_sort_scatter(const StoreBuf& in, uint64_t n, const uint32_t* blk_hist, Buckets* buckets, uint4* out_a,
                         float4* out_b, cudaStream_t st, const uint32_t* abort) {
    const uint32_t nblk = blocks_for(n, kSortThreads);
    k_sort_scatter<<<nblk, kSortThreads, 0, st>>>(in, n, blk_hist, nblk, buckets, out_a, out_b, abort);
}

namespace {
__global__ void k_store_guard(Buckets* bk, uint64_t rec_cap, uint64_t ev_cap, const uint32_t* bad, uint32_t* abort,
                              int* err) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const bool fail = *bad != 0u || bk->rec_off[kBuckets] > rec_cap || bk->n_events > ev_cap;
    *abort = fail ? 1u : 0u;
    if (!fail) return;
    for (int b = 0; b < kBuckets; ++b) bk->count[b] = 0;
    for (int b = 0; b <= kBuckets; ++b) {
        bk->path_off[b] = 0;
        bk->rec_off[b] = 0;
    }
    bk->n_events = 0;
    atomicOr(err, kErrStore);
}
}  // namespace

void launch_store_guard(Buckets* buckets, uint64_t rec_cap, uint64_t ev_cap, const uint32_t* bad, uint32_t* abort,
                        int* err, cudaStream_t st) {
    k_store_guard<<<1, 32, 0, st>>>(buckets, rec_cap, ev_cap, bad, abort, err);
}

uint64_t sort_blocks(uint64_t n) { return blocks_for(n, kSortThreads); }

void launch_grad_reference(const DevScene& S, const SortedPaths& P, const float* beta_t, const float* beta_ref,
                           const float* dbeta, const double* dldi, double* grad, cudaStream_t st) {
    const unsigned g = blocks_for(P.n_max, 128);
    if (g == 0) return;
    k_grad<<<g, 128, 0, st>>>(S, P, beta_t, beta_ref, dbeta, dldi, grad);
}

void launch_delta(const float* a, const float* b, float* out, int64_t n, cudaStream_t st) {
    const int bs = 256;
    unsigned g = (unsigned)std::min<int64_t>((n + bs - 1) / bs, (int64_t)device_sms() * 16);
    if (g == 0) return;
    k_delta<<<g, bs, 0, st>>>(a, b, out, n);
}

}  // namespace pt
