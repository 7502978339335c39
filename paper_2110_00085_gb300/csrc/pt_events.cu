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
#include "pt_kernels.cuh"

namespace pt {

namespace {

// ---------------------------------------------------------- binning ----
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
    // bits of v (< 2^10) moved to positions 3i
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}
__device__ __forceinline__ uint32_t event_bin(uint32_t pv, int bits, int shift) {
    const uint32_t m = (1u << bits) - 1u;
    const uint32_t bx = (pv & 511u) >> shift, by = ((pv >> 9) & 511u) >> shift, bz = ((pv >> 18) & 511u) >> shift;
    return spread3(bx & m) | (spread3(by & m) << 1) | (spread3(bz & m) << 2);
}

__global__ void __launch_bounds__(128) k_ev_hist(SortedPaths P, Events E, int max_orders) {
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
        const uint32_t pv = P.rec_a[pr.base + (uint64_t)e * pr.stride].w & kVoxMask;
        atomicAdd(E.hist + event_bin(pv, E.bin_bits, E.bin_shift), 1u);
    }
}

__global__ void __launch_bounds__(128) k_ev_scatter(SortedPaths P, Events E, int max_orders) {
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
        const uint32_t pos = atomicAdd(E.cursor + event_bin(a.w & kVoxMask, E.bin_bits, E.bin_shift), 1u);
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

// ----------------------------------------------------- per-path pieces --
// W_e for every event: w0 times, per earlier flight, exp(-sum dbeta l) and,
// per earlier vertex, albedo_ref f_s,t / f_s,ref (and 1/q after roulette)
__global__ void __launch_bounds__(128) k_path_weights(DevScene S, SortedPaths P, Events E,
                                                      const float* __restrict__ beta_t,
                                                      const float* __restrict__ beta_ref,
                                                      const float* __restrict__ dbeta) {
    __shared__ SharedBk sb;
    for (int k = threadIdx.x; k <= kBuckets; k += blockDim.x) {
        sb.po[k] = P.buckets->path_off[k];
        sb.ro[k] = P.buckets->rec_off[k];
        if (k < kBuckets) sb.cnt[k] = P.buckets->count[k];
    }
    __syncthreads();
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    PathRef pr;
    if (!locate(sb.po, sb.ro, sb.cnt, S.max_orders, j, pr)) return;
    const uint4 a0 = P.rec_a[pr.base];
    float3 xp = xyz(a0);
    uint32_t pvp = a0.w & kVoxMask;
    float w = S.w0;
    float4 bin = P.rec_b[pr.base + pr.stride];
    for (int e = 1; e <= pr.B; ++e) {
        const uint64_t rec = pr.base + (uint64_t)e * pr.stride;
        const uint4 ra = P.rec_a[rec];
        const uint32_t pv = ra.w & kVoxMask;
        const uint32_t pos = E.of_rec[rec];
        if (!vox_ok(S, pv) || !vox_ok(S, pvp) || pos >= E.cap) {
            atomicOr(S.err, kErrRecord);
            return;
        }
        const float3 om = make_float3(bin.x, bin.y, bin.z);
        const float W = w * expf(-delta_depth(S, dbeta, xp, om, pvp, bin.w));
        reinterpret_cast<float*>(E.b + pos)[3] = W;
        if (e < pr.B) {
            const int v = lin_vox(S, pv);
            const float bct = __ldg(beta_t + v), bcr = __ldg(beta_ref + v);
            const float btr = bcr + S.beta_air;
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
        xp = xyz(ra);
        pvp = pv;
    }
}

// gradient, per path: suffix sums S_e of the events' A_e, scattering-vertex
// terms h(x_e, mu_e) S_{e+1}, flight scatters -S_e l along flight e
__global__ void __launch_bounds__(128) k_path_grad(DevScene S, SortedPaths P, Events E,
                                                   const float* __restrict__ beta_t, double* __restrict__ grad) {
    __shared__ SharedBk sb;
    for (int k = threadIdx.x; k <= kBuckets; k += blockDim.x) {
        sb.po[k] = P.buckets->path_off[k];
        sb.ro[k] = P.buckets->rec_off[k];
        if (k < kBuckets) sb.cnt[k] = P.buckets->count[k];
    }
    __syncthreads();
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    PathRef pr;
    if (!locate(sb.po, sb.ro, sb.cnt, S.max_orders, j, pr)) return;
    float Ssum = 0.0f;
    for (int e = pr.B; e >= 1; --e) {
        const uint64_t rec = pr.base + (uint64_t)e * pr.stride;
        const uint4 ra = P.rec_a[rec];
        const float4 be = P.rec_b[rec];
        const uint32_t pos = E.of_rec[rec];
        const uint4 rp = P.rec_a[rec - pr.stride];
        if (!vox_ok(S, ra.w & kVoxMask) || !vox_ok(S, rp.w & kVoxMask) || pos >= E.cap) {
            atomicOr(S.err, kErrRecord);
            return;
        }
        if (e < pr.B && Ssum != 0.0f) {
            const float4 bn = P.rec_b[rec + pr.stride];
            const float mu = be.x * bn.x + be.y * bn.y + be.z * bn.z;
            const int v = lin_vox(S, ra.w & kVoxMask);
            red_add(grad + v, Ssum * score_vertex(S, __ldg(beta_t + v), mu));
        }
        Ssum += E.val[pos];
        if (Ssum != 0.0f)
            scatter_ray(S, grad, xyz(rp), make_float3(be.x, be.y, be.z), rp.w & kVoxMask, be.w, Ssum);
    }
}

// ---------------------------------------------------- per-event pieces --
__device__ __forceinline__ void load_cams(const DevScene& S, DevCam* cams) {
    for (int c = threadIdx.x; c < S.n_cams; c += blockDim.x) cams[c] = S.cams[c];
    __syncthreads();
}

// recycled forward: local estimates of every event toward every camera
template <bool CACHE>
__global__ void __launch_bounds__(128) k_event_forward(DevScene S, SortedPaths P, Events E,
                                                       const float* __restrict__ beta_t,
                                                       const float* __restrict__ beta_ref,
                                                       double* __restrict__ images, float* __restrict__ cache) {
    __shared__ DevCam cams[kMaxCams];
    load_cams(S, cams);
    const uint64_t pos = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= P.buckets->n_events) return;
    const uint4 a = E.a[pos];
    const float4 b = E.b[pos];
    const uint32_t pv = a.w;
    if (!vox_ok(S, pv)) {
        atomicOr(S.err, kErrRecord);
        return;
    }
    const float3 x = xyz(a), om = make_float3(b.x, b.y, b.z);
    const float W = b.w;
    const int v = lin_vox(S, pv);
    const float bct = __ldg(beta_t + v), btr = __ldg(beta_ref + v) + S.beta_air;
    for (int c = 0; c < S.n_cams; ++c) {
        const Proj q = project(cams[c], x);
        float ev = 0.0f;
        if (q.pix >= 0) {
            const float T = expf(-optical_depth_to_exit(S, beta_t, x, q.dir, pv, nullptr));
            const int gp = cams[c].off + q.pix;
            ev = local_contrib(W, fs_medium(S, bct, dot3(om, q.dir)), btr, T, q.r2, __ldg(S.omega + gp), P.inv_norm);
            red_add(images + gp, ev);
        }
        if (CACHE) cache[(uint64_t)c * E.cap + pos] = ev;
    }
}

// gradient, per event: shadow-ray scatters -a l, local-estimate vertex
// terms a h(x_b, mu_bd), and A_e = sum_d a for the per-path suffix sums.
// The warp takes the cameras one at a time and walks its 32 shadow rays in
// step.  Lanes holding events of one voxel are adjacent and their rays stay
// together, so at each step the -a l terms of adjacent lanes in the same
// voxel are summed (a segmented shuffle scan over runs of equal voxel ids,
// 8 lanes deep) and one FP64 red per run (per 8 lanes of a longer run)
// leaves the warp.
__device__ __forceinline__ void red_runs(double* __restrict__ grad, int idx, float val, int lane) {
    const unsigned full = 0xffffffffu;
    const int prev = __shfl_up_sync(full, idx, 1);
    const unsigned heads = __ballot_sync(full, lane == 0 || prev != idx);
    if (heads == full) {                       // no lane shares its voxel
        if (idx >= 0 && val != 0.0f) red_add(grad + idx, val);
        return;
    }
    const int start = 31 - __clz(heads & ((2u << lane) - 1u));   // first lane of my run
    const int chunk = start + ((lane - start) & ~7);               // first lane of my 8-lane chunk
    float s = val;
#pragma unroll
    for (int d = 1; d < 8; d <<= 1) {
        const float o = __shfl_up_sync(full, s, d);
        if (lane - d >= chunk) s += o;
    }
    // the last lane of a run or of a chunk holds the chunk's sum
    const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u) || ((lane - start) & 7) == 7;
    if (tail && idx >= 0 && s != 0.0f) red_add(grad + idx, s);
}

__global__ void __launch_bounds__(128) k_event_grad(DevScene S, SortedPaths P, Events E,
                                                    const float* __restrict__ beta_t,
                                                    const double* __restrict__ dldi, double* __restrict__ grad,
                                                    const float* __restrict__ cache) {
    __shared__ DevCam cams[kMaxCams];
    load_cams(S, cams);
    const int lane = threadIdx.x & 31;
    const uint64_t pos = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool ok = pos < P.buckets->n_events;
    float3 x = make_float3(0.f, 0.f, 0.f), om = x;
    uint32_t pv = 0;
    int v = 0;
    float bct = 0.0f;
    if (ok) {
        const uint4 a4 = E.a[pos];
        const float4 b4 = E.b[pos];
        pv = a4.w;
        if (!vox_ok(S, pv)) {
            atomicOr(S.err, kErrRecord);
            ok = false;
        } else {
            x = xyz(a4);
            om = make_float3(b4.x, b4.y, b4.z);
            v = lin_vox(S, pv);
            bct = __ldg(beta_t + v);
        }
    }
    const unsigned full = 0xffffffffu;
    float A = 0.0f, hv = 0.0f;
    for (int c = 0; c < S.n_cams; ++c) {
        float a = 0.0f;
        float3 dir = x;
        if (ok) {
            const float ev = cache[(uint64_t)c * E.cap + pos];
            if (ev != 0.0f) {
                const Proj q = project(cams[c], x);
                if (q.pix >= 0) {
                    a = (float)__ldg(dldi + cams[c].off + q.pix) * ev;
                    dir = q.dir;
                    A += a;
                    if (a != 0.0f) hv += a * score_vertex(S, bct, dot3(om, q.dir));
                }
            }
        }
        bool live = a != 0.0f;
        if (!__any_sync(full, live)) continue;
        Dda r;
        r.init(S, x, dir, pv, __int_as_float(0x7f800000));
        while (__any_sync(full, live)) {
            int idx = -1 - lane;   // never equal across lanes
            float val = 0.0f;
            if (live) {
                const float tn = r.next();
                idx = r.idx;
                val = -a * r.seg(tn);
                live = r.step(S, tn);
            }
            red_runs(grad, idx, val, lane);
        }
    }
    if (ok) {
        if (hv != 0.0f) red_add(grad + v, hv);
        E.val[pos] = A;
    }
}

unsigned blocks(uint64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

void launch_events(const DevScene& S, const SortedPaths& P, const Events& E, cudaStream_t st) {
    const unsigned g = blocks(P.n_max, 128);
    if (g == 0) return;
    cudaMemsetAsync(E.hist, 0, sizeof(uint32_t) * E.n_bins, st);
    k_ev_hist<<<g, 128, 0, st>>>(P, E, S.max_orders);
    const uint32_t nb = (E.n_bins + kScanItems - 1) / kScanItems;   // <= 4096 for 2^24 bins
    k_scan_blocks<<<nb, 1024, 0, st>>>(E.hist, E.cursor, E.partial, E.n_bins);
    k_scan_blocks<<<1, 1024, 0, st>>>(E.partial, E.partial + kScanItems, E.partial + 2 * kScanItems, nb);
    k_scan_add<<<nb, 1024, 0, st>>>(E.cursor, E.partial + kScanItems, E.n_bins);
    k_ev_scatter<<<g, 128, 0, st>>>(P, E, S.max_orders);
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
