// pt_event_ops.cuh -- per-path and per-event bodies of the recycled passes
// (Sec. 5.2 estimator, Sec. 4.4 path score), shared by the single-scene
// kernels (pt_events.cu) and the batched persistent kernels (pt_batch.cu).
#pragma once
#include "pt_kernels.cuh"

namespace pt {

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
// sub-voxel cell (0 .. 2^sub - 1) of coordinate c in voxel i along one axis
__device__ __forceinline__ uint32_t sub_cell(float c, float o, float inv_vox, uint32_t i, int sub) {
    const int q = (int)floorf((c - o) * inv_vox * (float)(1 << sub)) - (int)(i << sub);
    return (uint32_t)min(max(q, 0), (1 << sub) - 1);
}
// Bin of an event: Morton code of its voxel coordinates (>> shift), with
// `sub` bits of its position inside the voxel appended per axis, so that
// events of one voxel are ordered by where they lie in it.  Only the order
// of events depends on the bin; their voxel is the record's.
__device__ __forceinline__ uint32_t event_bin(const DevScene& S, const Events& E, uint4 a) {
    const uint32_t pv = a.w & kVoxMask;
    const uint32_t m = (1u << E.bin_bits) - 1u;
    const uint32_t ix = pv & 511u, iy = (pv >> 9) & 511u, iz = (pv >> 18) & 511u;
    uint32_t bx = ix >> E.bin_shift, by = iy >> E.bin_shift, bz = iz >> E.bin_shift;
    if (E.bin_sub) {
        const int s = E.bin_sub;
        bx = (bx << s) | sub_cell(__uint_as_float(a.x), S.ox, S.inv_vox, ix, s);
        by = (by << s) | sub_cell(__uint_as_float(a.y), S.oy, S.inv_vox, iy, s);
        bz = (bz << s) | sub_cell(__uint_as_float(a.z), S.oz, S.inv_vox, iz, s);
    }
    return spread3(bx & m) | (spread3(by & m) << 1) | (spread3(bz & m) << 2);
}

// ----------------------------------------------------- per-path pieces --
// W_e for every event: w0 times, per earlier flight, exp(-sum dbeta l) and,
// per earlier vertex, albedo_ref f_s,t / f_s,ref (and 1/q after roulette)
__device__ __forceinline__ void path_weights_one(const DevScene& S, const SortedPaths& P, const Events& E,
                                                 const SharedBk& sb, uint64_t j, const float* __restrict__ beta_t,
                                                 const float* __restrict__ beta_ref,
                                                 const float* __restrict__ dbeta) {
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
__device__ __forceinline__ void path_grad_one(const DevScene& S, const SortedPaths& P, const Events& E,
                                              const SharedBk& sb, uint64_t j, const float* __restrict__ beta_t,
                                              double* __restrict__ grad) {
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
// camera table into shared memory (blocks of the kernels below)
__device__ __forceinline__ void load_cams(const DevScene& S, DevCam* cams) {
    for (int c = threadIdx.x; c < S.n_cams; c += blockDim.x) cams[c] = S.cams[c];
    __syncthreads();
}

// recycled forward: local estimates of every event toward every camera
template <bool CACHE>
__device__ __forceinline__ void event_forward_one(const DevScene& S, const DevCam* cams, const Events& E,
                                                  float inv_norm, uint64_t n_events, uint64_t pos,
                                                  const float* __restrict__ beta_t,
                                                  const float* __restrict__ beta_ref, double* __restrict__ images,
                                                  float* __restrict__ cache) {
    if (pos >= n_events) return;
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
            ev = local_contrib(W, fs_medium(S, bct, dot3(om, q.dir)), btr, T, q.r2, __ldg(S.omega + gp), inv_norm);
            red_add(images + gp, ev);
        }
        if (CACHE) cache[(uint64_t)c * E.cap + pos] = ev;
    }
}

// gradient, per event: shadow-ray scatters -a l, local-estimate vertex
// terms a h(x_b, mu_bd), and A_e = sum_d a for the per-path suffix sums.
// The warp takes the cameras one at a time and walks its 32 shadow rays in
// step, ordered across the direction to the camera (lateral_order), so that
// lanes whose rays run side by side are adjacent.  At each step the -a l
// terms of adjacent lanes in the same voxel are summed (a segmented shuffle
// scan over runs of equal voxel ids, kRunChunk lanes deep) and one FP64 red
// per run (per kRunChunk lanes of a longer run) leaves the warp.
constexpr int kRunChunk = 8;    // lanes summed per red at most (a power of two; 16 measured no faster)
__device__ __forceinline__ void red_runs(double* __restrict__ grad, int idx, float val, int lane) {
    const unsigned full = 0xffffffffu;
    const int prev = __shfl_up_sync(full, idx, 1);
    const unsigned heads = __ballot_sync(full, lane == 0 || prev != idx);
    if (heads == full) {                       // no lane shares its voxel
        if (idx >= 0 && val != 0.0f) red_add(grad + idx, val);
        return;
    }
    const int start = 31 - __clz(heads & ((2u << lane) - 1u));   // first lane of my run
    const int chunk = start + ((lane - start) & ~(kRunChunk - 1));  // first lane of my chunk
    float s = val;
#pragma unroll
    for (int d = 1; d < kRunChunk; d <<= 1) {
        const float o = __shfl_up_sync(full, s, d);
        if (lane - d >= chunk) s += o;
    }
    // the last lane of a run or of a chunk holds the chunk's sum
    const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u) || ((lane - start) & (kRunChunk - 1)) == kRunChunk - 1;
    if (tail && idx >= 0 && s != 0.0f) red_add(grad + idx, s);
}

// 8-bit value with its bits moved to the even positions
__device__ __forceinline__ uint32_t spread2(uint32_t v) {
    v &= 0xffu;
    v = (v | (v << 4)) & 0x0f0fu;
    v = (v | (v << 2)) & 0x3333u;
    v = (v | (v << 1)) & 0x5555u;
    return v;
}

// Lane that should march the ray of this step's lane order: the warp's rays
// to one camera are ordered by a 2D Morton code of where their events lie
// across the direction to the camera (relative to the first live lane's
// event, in 1/32 voxel, +-4 voxels), so that lanes whose rays run side by
// side are adjacent and the run merge of red_runs finds their shared
// voxels.  Lanes without a ray go last.  A bitonic sort of the 32 keys
// (lane number in the low bits: all keys distinct) gives the permutation.
__device__ __forceinline__ int lateral_order(const DevScene& S, float3 x, float3 dir, bool live, int lane) {
    const unsigned full = 0xffffffffu;
    const int ld = __ffs(__ballot_sync(full, live)) - 1;
    const float3 d0 = make_float3(__shfl_sync(full, dir.x, ld), __shfl_sync(full, dir.y, ld),
                                  __shfl_sync(full, dir.z, ld));
    const float3 rel = make_float3(x.x - __shfl_sync(full, x.x, ld), x.y - __shfl_sync(full, x.y, ld),
                                   x.z - __shfl_sync(full, x.z, ld));
    // an orthonormal pair across d0 (Duff et al., JCGT 2017)
    const float sg = copysignf(1.0f, d0.z);
    const float ia = -1.0f / (sg + d0.z);
    const float bb = d0.x * d0.y * ia;
    const float3 e1 = make_float3(1.0f + sg * d0.x * d0.x * ia, sg * bb, -sg * d0.x);
    const float3 e2 = make_float3(bb, sg + d0.y * d0.y * ia, -d0.y);
    const float k = 32.0f * S.inv_vox;
    const int qu = min(max((int)floorf(dot3(rel, e1) * k) + 128, 0), 255);
    const int qv = min(max((int)floorf(dot3(rel, e2) * k) + 128, 0), 255);
    uint32_t key = live ? (((spread2((uint32_t)qu) | (spread2((uint32_t)qv) << 1)) << 5) | (uint32_t)lane)
                        : ((1u << 21) | (uint32_t)lane);
#pragma unroll
    for (int k2 = 2; k2 <= 32; k2 <<= 1) {
#pragma unroll
        for (int j = k2 >> 1; j > 0; j >>= 1) {
            const uint32_t o = __shfl_xor_sync(full, key, j);
            const bool keep_min = ((lane & j) == 0) == ((lane & k2) == 0);
            key = keep_min ? min(key, o) : max(key, o);
        }
    }
    return (int)(key & 31u);
}

// Warp-synchronous: every lane of the warp calls it (lanes past the last
// event pass pos >= n_events).
__device__ __forceinline__ void event_grad_warp(const DevScene& S, const DevCam* cams, const Events& E,
                                                uint64_t n_events, uint64_t pos, const float* __restrict__ beta_t,
                                                const double* __restrict__ dldi, double* __restrict__ grad,
                                                const float* __restrict__ cache) {
    const int lane = threadIdx.x & 31;
    bool ok = pos < n_events;
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
        // march the rays in this camera's lateral order (A and the vertex
        // terms above stay with the event's own lane)
        const int src = lateral_order(S, x, dir, live, lane);
        const float3 xs = make_float3(__shfl_sync(full, x.x, src), __shfl_sync(full, x.y, src),
                                      __shfl_sync(full, x.z, src));
        const float3 ds = make_float3(__shfl_sync(full, dir.x, src), __shfl_sync(full, dir.y, src),
                                      __shfl_sync(full, dir.z, src));
        const uint32_t pvs = __shfl_sync(full, pv, src);
        const float as = __shfl_sync(full, a, src);
        live = __shfl_sync(full, (int)live, src) != 0;
        Dda r;
        r.init(S, xs, ds, pvs, __int_as_float(0x7f800000));
        while (__any_sync(full, live)) {
            int idx = -1 - lane;   // never equal across lanes
            float val = 0.0f;
            if (live) {
                const float tn = r.next();
                idx = r.idx;
                val = -as * r.seg(tn);
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

__device__ __forceinline__ void load_buckets(const SortedPaths& P, SharedBk& sb) {
    for (int k = threadIdx.x; k <= kBuckets; k += blockDim.x) {
        sb.po[k] = P.buckets->path_off[k];
        sb.ro[k] = P.buckets->rec_off[k];
        if (k < kBuckets) sb.cnt[k] = P.buckets->count[k];
    }
}

}  // namespace pt
