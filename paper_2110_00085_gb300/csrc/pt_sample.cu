// pt_sample.cu -- the path-sampling megakernel: one thread traces one light
// path from the sun through the extinction grid (Sec. 3.4), adds a local
// estimate toward every camera at every collision (Sec. 3.4.3, Eq. Qd) and,
// when storing, writes the path's vertex records for recycling (Sec. 5).
//
// Per path: sun-rectangle start point and box entry; distance sampling by
// accumulating beta * l along the 3D-DDA until tau ~ Exp(1) is reached
// (Sec. 3.4.1); at each collision the shadow ray to each camera (3D-DDA,
// transmittance under the same grid), an FP64 red into the pixel, then
// termination (order limit, Russian roulette after rr_start), particle-type
// choice with probability albedo_j beta_j / beta_s and direction sampling
// from that type's phase function (Sec. 3.4.2).
#include "pt_kernels.cuh"

namespace pt {

namespace {

template <bool STORE, bool IMG, bool TALLY, bool FP>
__device__ __forceinline__ void trace_one(const DevScene& S, const DevCam* cams, const float* __restrict__ beta,
                                          uint64_t i, uint64_t first, float inv_norm, uint64_t seed, uint32_t epoch,
                                          double* __restrict__ images, uint64_t* __restrict__ fps,
                                          const StoreBuf& st, float* tal) {
    const uint64_t pid = first + i;
    Rng rng;
    rng.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    rng.pid_lo = (uint32_t)pid;
    rng.pid_hi = (uint32_t)(pid >> 32);
    rng.epoch = epoch;
    rng.scene = S.scene_id;

    uint64_t h = kFnvBasis;

    // --- source: uniform point on the sun rectangle, ray along the sun ---
    float4 u = rng.draw(0, 0);
    const float a = fmaf(u.x, S.alen, S.amin);
    const float b = fmaf(u.y, S.blen, S.bmin);
    const float3 sd = make_float3(S.sx, S.sy, S.sz);
    float3 p = make_float3(a * S.e1[0] + b * S.e2[0] + S.hmin * S.sx, a * S.e1[1] + b * S.e2[1] + S.hmin * S.sy,
                           a * S.e1[2] + b * S.e2[2] + S.hmin * S.sz);
    // slab test against the box
    float t0 = 0.0f, t1 = __int_as_float(0x7f800000);
    bool hit = true;
    {
        const float lo[3] = {S.ox, S.oy, S.oz};
        const float hi[3] = {fmaf((float)S.nx, S.vox, S.ox), fmaf((float)S.ny, S.vox, S.oy),
                             fmaf((float)S.nz, S.vox, S.oz)};
        const float pp[3] = {p.x, p.y, p.z};
        const float dd[3] = {sd.x, sd.y, sd.z};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (dd[k] == 0.0f) {
                if (pp[k] < lo[k] || pp[k] > hi[k]) hit = false;
            } else {
                float ua = (lo[k] - pp[k]) / dd[k], ub = (hi[k] - pp[k]) / dd[k];
                if (ua > ub) { const float tt = ua; ua = ub; ub = tt; }
                t0 = fmaxf(t0, ua);
                t1 = fminf(t1, ub);
            }
        }
        if (!(t1 > t0)) hit = false;
    }
    if (!hit) {
        if (TALLY) tal[PT_T_MISSED] += S.w0;
        if (FP) *fps = fnv_word(fnv_word(h, 0u), kEndMiss);
        if (STORE) st.cnt[i] = 0;
        return;
    }
    {
        float3 x = make_float3(fmaf(t0, sd.x, p.x), fmaf(t0, sd.y, p.y), fmaf(t0, sd.z, p.z));
        int vx = min(max((int)floorf((x.x - S.ox) * S.inv_vox), 0), S.nx - 1);
        int vy = min(max((int)floorf((x.y - S.oy) * S.inv_vox), 0), S.ny - 1);
        int vz = min(max((int)floorf((x.z - S.oz) * S.inv_vox), 0), S.nz - 1);
        int v = vx + S.nx * (vy + S.ny * vz);
        uint32_t pv = pack_vox(vx, vy, vz);
        float3 om = sd;
        float w = S.w0;
        float tau = -logf(u.z);
        if (TALLY) { tal[PT_T_INJECTED] += S.w0; tal[PT_T_ENTERED] += 1.0f; }
        if (STORE) {
            st.rec_a[i] = rec_a(x, pv, kKindEntry);
            st.rec_b[i] = make_float4(sd.x, sd.y, sd.z, 0.0f);
        }
        int B = 0;
        uint32_t end = kEndNone;
        for (int k = 1;; ++k) {
            // ---- distance sampling (regular tracking through the grid) ----
            Dda r;
            r.init(S, x, om, pv, __int_as_float(0x7f800000));
            float tcol = -1.0f;
            int ncross = 0;
            // remaining optical depth kept as tau + comp (compensated: the
            // rounding of every product and difference is carried in comp, so
            // the collision point stays accurate where beta is small)
            float comp = 0.0f;
            for (;;) {
                const float tn = r.next();
                const float l = r.seg(tn);
                const float bt = __ldg(beta + r.idx) + S.beta_air;
                ++ncross;
                // __fmul_rn/__fsub_rn are never contracted into FMAs, which
                // keeps the error terms exact
                const float prod = __fmul_rn(bt, l);
                if (bt > 0.0f && tau + comp <= prod) {
                    tcol = fminf(r.t + (tau + comp) / bt, fminf(tn, r.tend));
                    break;
                }
                const float perr = fmaf(bt, l, -prod);
                const float nt = __fsub_rn(tau, prod);
                comp += __fsub_rn(__fsub_rn(tau, nt), prod) - perr;
                tau = nt;
                if (!r.step(S, tn)) break;
            }
            if (TALLY) tal[PT_T_SEG_CROSS] += (float)ncross;
            if (tcol < 0.0f) {
                end = kEndEscape;
                if (TALLY) tal[PT_T_ESCAPED] += w;
                break;
            }
            v = r.idx;
            pv = r.coords(pv, om);
            x = make_float3(fmaf(tcol, om.x, x.x), fmaf(tcol, om.y, x.y), fmaf(tcol, om.z, x.z));
            B = k;
            if (STORE) {
                st.rec_a[(uint64_t)k * st.stride + i] = rec_a(x, pv, kKindScatter);
                st.rec_b[(uint64_t)k * st.stride + i] = make_float4(om.x, om.y, om.z, tcol);
            }
            const float bc = __ldg(beta + v);
            const float bt = bc + S.beta_air;
            const float bs = S.alb_c * bc + S.alb_a * S.beta_air;
            if (FP) h = fnv_word(h, (uint32_t)v);
            if (TALLY) tal[PT_T_COLLISIONS] += 1.0f;
            // ---- local estimation toward every camera ----
            for (int c = 0; c < S.n_cams; ++c) {
                const Proj pr = project(cams[c], x);
                if (FP) h = fnv_word(h, (uint32_t)pr.pix);
                if (!IMG || pr.pix < 0) continue;
                int nc = 0;
                const float T = expf(-optical_depth_to_exit(S, beta, x, pr.dir, pv, TALLY ? &nc : nullptr));
                const float mu = dot3(om, pr.dir);
                const int gp = cams[c].off + pr.pix;
                const float ev = local_contrib(w, fs_medium(S, bc, mu), bt, T, pr.r2, __ldg(S.omega + gp), inv_norm);
                red_add(images + gp, ev);
                if (TALLY) { tal[PT_T_IN_VIEW] += 1.0f; tal[PT_T_SHADOW_CROSS] += (float)nc; }
            }
            // ---- collision: absorption, termination, new direction ----
            const float alb = bs / bt;
            if (TALLY) tal[PT_T_ABSORBED] += w * (1.0f - alb);
            w *= alb;
            u = rng.draw((uint32_t)k, 0);
            if (k == S.max_orders) {
                end = kEndTrunc;
                if (TALLY) tal[PT_T_TRUNCATED] += w;
                if (FP) h = fnv_word(h, 2u);
                break;
            }
            if (k >= S.rr_start) {
                if (u.x <= S.rr_q) {
                    if (TALLY) tal[PT_T_RR_GAIN] += w * (S.inv_q - 1.0f);
                    w *= S.inv_q;
                } else {
                    end = kEndRR;
                    if (TALLY) tal[PT_T_RR_KILLED] += w;
                    if (FP) h = fnv_word(h, 2u);
                    break;
                }
            }
            const bool cloud = u.y * bs <= S.alb_c * bc;
            if (FP) h = fnv_word(h, cloud ? 0u : 1u);
            const Polar pc = cloud ? sample_hg(S, u.z) : sample_rayleigh(u.z);
            om = rotate_dir(om, pc, u.w);
            tau = -logf(rng.draw((uint32_t)k, 1).x);
        }
        if (FP) *fps = fnv_word(fnv_word(h, (uint32_t)B), end);
        if (STORE) {
            st.cnt[i] = (uint8_t)B;
            if (B > 0) {
                uint4 ra = st.rec_a[(uint64_t)B * st.stride + i];
                ra.w |= end << 30;
                st.rec_a[(uint64_t)B * st.stride + i] = ra;
            }
        }
    }
}

template <bool STORE, bool IMG, bool DIAG>
__global__ void __launch_bounds__(128) k_sample(DevScene S, const float* __restrict__ beta, uint64_t first, uint64_t n,
                                                float inv_norm, uint64_t seed, uint32_t epoch,
                                                double* __restrict__ images, double* __restrict__ tallies,
                                                uint64_t* __restrict__ fps, StoreBuf st) {
    __shared__ DevCam cams[kMaxCams];
    __shared__ float stal[PT_TALLY_COUNT];
    for (int c = threadIdx.x; c < S.n_cams; c += blockDim.x) cams[c] = S.cams[c];
    constexpr bool TALLY = DIAG, FP = DIAG;
    if (TALLY && threadIdx.x < PT_TALLY_COUNT) stal[threadIdx.x] = 0.0f;
    __syncthreads();
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float tal[PT_TALLY_COUNT];
#pragma unroll
    for (int k = 0; k < PT_TALLY_COUNT; ++k) tal[k] = 0.0f;
    uint64_t fp = 0;
    if (i < n) trace_one<STORE, IMG, TALLY, FP>(S, cams, beta, i, first, inv_norm, seed, epoch, images, &fp, st, tal);
    if (FP && fps && i < n) fps[i] = fp;
    if (TALLY && tallies) {
        // block reduction in shared memory, one FP64 add per tally per block
#pragma unroll
        for (int k = 0; k < PT_TALLY_COUNT; ++k)
            if (tal[k] != 0.0f) atomicAdd(&stal[k], tal[k]);
        __syncthreads();
        if (threadIdx.x < PT_TALLY_COUNT) atomicAdd(tallies + threadIdx.x, (double)stal[threadIdx.x]);
    }
}

template <bool STORE, bool IMG, bool DIAG>
void launch_t(const DevScene& S, const float* beta, uint64_t first, uint64_t n, float inv_norm, uint64_t seed,
              uint32_t epoch, double* images, double* tallies, uint64_t* fps, const StoreBuf& st, cudaStream_t s) {
    const int bs = 128;
    const uint64_t grid = (n + bs - 1) / bs;
    k_sample<STORE, IMG, DIAG><<<(unsigned)grid, bs, 0, s>>>(S, beta, first, n, inv_norm, seed, epoch, images,
                                                           tallies, fps, st);
}

template <bool STORE>
void launch_s(const DevScene& S, const float* beta, uint64_t first, uint64_t n, float inv_norm, uint64_t seed,
              uint32_t epoch, double* images, double* tallies, uint64_t* fps, const StoreBuf& sb, cudaStream_t st) {
    const bool I = images != nullptr, D = tallies != nullptr || fps != nullptr;
    if (I && D) launch_t<STORE, true, true>(S, beta, first, n, inv_norm, seed, epoch, images, tallies, fps, sb, st);
    else if (I) launch_t<STORE, true, false>(S, beta, first, n, inv_norm, seed, epoch, images, tallies, fps, sb, st);
    else if (D) launch_t<STORE, false, true>(S, beta, first, n, inv_norm, seed, epoch, images, tallies, fps, sb, st);
    else launch_t<STORE, false, false>(S, beta, first, n, inv_norm, seed, epoch, images, tallies, fps, sb, st);
}

}  // namespace

void launch_sample(const DevScene& S, const float* beta, uint64_t first, uint64_t n, float inv_norm, uint64_t seed,
                   uint32_t epoch, double* images, double* tallies, uint64_t* fps, const StoreBuf* store,
                   cudaStream_t st) {
    StoreBuf sb{};
    if (store) {
        sb = *store;
        launch_s<true>(S, beta, first, n, inv_norm, seed, epoch, images, tallies, fps, sb, st);
    } else {
        launch_s<false>(S, beta, first, n, inv_norm, seed, epoch, images, tallies, fps, sb, st);
    }
}

}  // namespace pt
