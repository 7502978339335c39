// pt_paths.cu -- stored light paths: the path sort (Sec. 5.3), the recycled
// forward pass and the gradient pass over sorted paths (Sec. 5.2, Sec. 4.4).
//
// Sort: counting sort of paths by their number of collisions B (the paper's
// path sorting: the 32 lanes of a warp hold paths of equal size, so every
// lane runs the same number of events) and, inside a size, by the Morton
// code of the voxel of the first collision (4096 bins of the grid), so that
// a warp's paths also start their walks close together: key histogram ->
// scan -> scatter.
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
#include "pt_event_ops.cuh"

namespace pt {

namespace {

constexpr int kSortThreads = 256;
constexpr uint32_t kNoKey = 0xffffffffu;

// ------------------------------------------------------------ sort ------
// key of path i: its size B (1 .. n_buckets - 1) times kPathBins plus the
// Morton code of its first collision's voxel >> key_shift; kNoKey for a path
// that is not stored (B = 0)
__global__ void __launch_bounds__(kSortThreads) k_sort_keys(StoreBuf in, uint64_t n, int n_buckets, int key_shift,
                                                            uint32_t* __restrict__ keys, uint32_t* __restrict__ hist,
                                                            uint32_t* __restrict__ n_zero) {
    const uint64_t i = (uint64_t)blockIdx.x * kSortThreads + threadIdx.x;
    const uint32_t b = i < n ? (uint32_t)in.cnt[i] : 0xffu;
    // paths without a collision are counted (bucket 0 of the table) but not stored
    const unsigned zeros = __ballot_sync(0xffffffffu, b == 0u);
    if ((threadIdx.x & 31) == 0 && zeros) atomicAdd(n_zero, (uint32_t)__popc(zeros));
    if (i >= n) return;
    uint32_t key = kNoKey;
    if (b >= 1 && b < (uint32_t)n_buckets) {
        const uint32_t pv = in.rec_a[in.stride + i].w & kVoxMask;
        const uint32_t m = (spread3(pv & 511u) | (spread3((pv >> 9) & 511u) << 1) | (spread3((pv >> 18) & 511u) << 2))
                           >> key_shift;
        key = b * kPathBins + min(m, kPathBins - 1u);
        atomicAdd(hist + key, 1u);
    }
    keys[i] = key;
}

// bucket table from the scanned key bins: bucket b's paths are the bins
// [b kPathBins, (b + 1) kPathBins), in order
__global__ void k_bucket_offsets(const uint32_t* __restrict__ hist, const uint32_t* __restrict__ cursor,
                                 const uint32_t* __restrict__ n_zero, Buckets* bk, int n_buckets) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const uint32_t last = kSortBins - 1;
    const uint64_t total = (uint64_t)cursor[last] + hist[last];
    uint64_t p = 0, r = 0, ev = 0;
    for (int b = 0; b < kBuckets; ++b) {
        const uint64_t hi = b + 1 < kBuckets ? cursor[(b + 1) * kPathBins] : total;
        const uint64_t n = (b >= 1 && b < n_buckets) ? hi - cursor[b * kPathBins] : 0;   // B = 0 paths are not stored
        bk->count[b] = b == 0 ? *n_zero : n;
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

__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(StoreBuf in, uint64_t n, const uint32_t* __restrict__ keys,
                                                               uint32_t* __restrict__ cursor,
                                                               const Buckets* __restrict__ bk,
                                                               uint4* __restrict__ out_a, float4* __restrict__ out_b,
                                                               const uint32_t* __restrict__ abort) {
    if (abort && *abort) return;   // the store did not fit (nothing is written)
    const uint64_t i = (uint64_t)blockIdx.x * kSortThreads + threadIdx.x;
    if (i >= n) return;
    const uint32_t key = keys[i];
    if (key == kNoKey) return;
    const uint32_t b = key / kPathBins;
    const uint64_t pos = (uint64_t)atomicAdd(cursor + key, 1u) - bk->path_off[b];
    const uint64_t cb = bk->count[b], ro = bk->rec_off[b];
    if (pos >= cb) return;   // (cannot happen: the key was counted)
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

SortScratch sort_scratch(uint32_t* base, uint64_t n) {
    SortScratch s;
    s.keys = base;
    s.hist = base + n;
    s.cursor = s.hist + kSortBins;
    s.partial = s.cursor + kSortBins;
    s.n_zero = s.partial + 3 * 4096;
    return s;
}

uint64_t sort_scratch_words(uint64_t n) { return n + 2ull * kSortBins + 3ull * 4096 + 1; }

void launch_sort_count(const StoreBuf& in, uint64_t n, int n_buckets, int key_shift, const SortScratch& w,
                       Buckets* buckets, cudaStream_t st) {
    cudaMemsetAsync(w.hist, 0, sizeof(uint32_t) * kSortBins, st);
    cudaMemsetAsync(w.n_zero, 0, sizeof(uint32_t), st);
    const unsigned g = blocks_for(n, kSortThreads);
    if (g) k_sort_keys<<<g, kSortThreads, 0, st>>>(in, n, n_buckets, key_shift, w.keys, w.hist, w.n_zero);
    launch_scan(w.hist, w.cursor, w.partial, kSortBins, st);
    k_bucket_offsets<<<1, 32, 0, st>>>(w.hist, w.cursor, w.n_zero, buckets, n_buckets);
}

void launch_sort_scatter(const StoreBuf& in, uint64_t n, const SortScratch& w, Buckets* buckets, uint4* out_a,
                         float4* out_b, cudaStream_t st, const uint32_t* abort) {
    const unsigned g = blocks_for(n, kSortThreads);
    if (g) k_sort_scatter<<<g, kSortThreads, 0, st>>>(in, n, w.keys, w.cursor, buckets, out_a, out_b, abort);
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
