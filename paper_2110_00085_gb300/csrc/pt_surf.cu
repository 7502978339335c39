// pt_surf.cu -- reflectometry (Sec. 6): light paths among surfaces in a
// closed box, with one sphere whose Phong BRDF (Eq. phong) is recovered.
//
// Paths start on a square Lambertian emitter in the ceiling, make a local
// estimate toward the camera at every surface hit (the surface counterpart
// of Eq. Qd: BRDF f_r / pi times the cosine at the hit instead of the phase
// function) and continue in a cosine-weighted direction about the normal.
// The path pdf does not depend on the BRDF parameters (kappa, gamma), so a
// stored path is re-evaluated under new parameters by its Phong factors
// alone (Eq. 19 with mu independent of the parameters): the store keeps,
// per camera event, everything that does not depend on (kappa, gamma) and,
// per path, the lobe cosines of its Phong vertices; reweighting and the
// gradient in (kappa, gamma) are then a map and a reduction over events.
#include <algorithm>
#include <cstdio>
#include <new>

#include "pt_kernels.cuh"

namespace pt {

namespace {

constexpr float kSurfEps = 1e-4f;     // hits closer than this along a ray are ignored (the start surface)
constexpr float kNoPhong = -2.0f;     // lobe cosine of an event vertex that is not on the Phong sphere

struct SurfDev {
    DevCam cam;
    const float* omega;    // pixel solid angles of the camera
    const float4* sph;     // centre, radius
    int n_sph, phong, max_orders, rr_start;
    float lx0, lx1, ly0, ly1;
    float w0;              // emitted power (pi radiance area)
    float rr_q, inv_q;
};

struct SurfStore {
    uint4* ev;             // {base bits, lobe cosine bits (or kNoPhong), pixel, path | phong count << 28},
                           // sorted by pixel
    uint4* raw;            // the same records in the order the tracer wrote them
    uint32_t* bins;        // per pixel: event count [0, n_pix), then the scatter cursor [n_pix, 2 n_pix)
    uint32_t n_pix;
    uint32_t* count;       // events written
    float* pc;             // lobe cosines of the Phong continuations, [slot * n + path]
    uint64_t n, cap;
};

__device__ __forceinline__ float3 cosine_dir(float3 n, float u1, float u2) {
    // orthonormal basis of Duff et al. (JCGT 2017) about n
    const float sign = copysignf(1.0f, n.z);
    const float a = -1.0f / (sign + n.z);
    const float b = n.x * n.y * a;
    const float3 b1 = make_float3(1.0f + sign * n.x * n.x * a, sign * b, -sign * n.x);
    const float3 b2 = make_float3(b, sign + n.y * n.y * a, -n.y);
    const float rr = sqrtf(u1), ct = sqrtf(fmaxf(0.0f, 1.0f - u1));
    float sp, cp;
    sincospif(2.0f * u2, &sp, &cp);
    return make_float3(rr * cp * b1.x + rr * sp * b2.x + ct * n.x, rr * cp * b1.y + rr * sp * b2.y + ct * n.y,
                       rr * cp * b1.z + rr * sp * b2.z + ct * n.z);
}

// nearest surface along p + t d: sphere i >= 0 or wall -1..-6 (x-, x+, y-,
// y+, z-, z+), the distance and the normal facing the ray; -100: none
__device__ int surf_hit(const SurfDev& S, float3 p, float3 d, float& t_out, float3& nrm) {
    float best = __int_as_float(0x7f800000);
    int id = -100;
    for (int i = 0; i < S.n_sph; ++i) {
        const float4 c = __ldg(S.sph + i);
        const float ox = p.x - c.x, oy = p.y - c.y, oz = p.z - c.z;
        const float b = ox * d.x + oy * d.y + oz * d.z;
        const float cc = ox * ox + oy * oy + oz * oz - c.w * c.w;
        const float disc = b * b - cc;
        if (disc < 0.0f || b >= 0.0f) continue;           // no sphere ahead (rays start outside spheres)
        const float t = cc / (sqrtf(disc) - b);             // near root, without cancellation
        if (t > kSurfEps && t < best) { best = t; id = i; }
    }
    const float pa[3] = {p.x, p.y, p.z}, da[3] = {d.x, d.y, d.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (da[a] == 0.0f) continue;
        const float t = ((da[a] > 0.0f ? 1.0f : 0.0f) - pa[a]) / da[a];
        if (t > kSurfEps && t < best) { best = t; id = -(2 * a + (da[a] > 0.0f ? 2 : 1)); }
    }
    if (id == -100) return id;
    t_out = best;
    if (id >= 0) {
        // normalised by the distance, not the radius: a hit point off the
        // sphere by rounding still gives a unit normal, so the next direction
        // stays unit (otherwise the error grows along chains of sphere hits)
        const float4 c = __ldg(S.sph + id);
        const float qx = p.x + best * d.x - c.x, qy = p.y + best * d.y - c.y, qz = p.z + best * d.z - c.z;
        const float iq = 1.0f / sqrtf(qx * qx + qy * qy + qz * qz);
        nrm = make_float3(qx * iq, qy * iq, qz * iq);
    } else {
        const int a = (-id - 1) / 2;
        const float s = ((-id - 1) % 2) ? -1.0f : 1.0f;
        nrm = make_float3(a == 0 ? s : 0.0f, a == 1 ? s : 0.0f, a == 2 ? s : 0.0f);
    }
    return id;
}

__device__ bool surf_visible(const SurfDev& S, float3 x, float3 w, float r) {
    for (int i = 0; i < S.n_sph; ++i) {
        const float4 c = __ldg(S.sph + i);
        const float ox = x.x - c.x, oy = x.y - c.y, oz = x.z - c.z;
        const float b = ox * w.x + oy * w.y + oz * w.z;
        const float cc = ox * ox + oy * oy + oz * oz - c.w * c.w;
        const float disc = b * b - cc;
        if (disc < 0.0f || b >= 0.0f) continue;
        const float t = cc / (sqrtf(disc) - b);
        if (t > kSurfEps && t < r) return false;
    }
    return true;
}

__global__ void __launch_bounds__(128) k_surf_store(SurfDev S, SurfStore P, uint64_t first, float inv_norm, Rng rng,
                                                    double* __restrict__ tallies, uint64_t* __restrict__ fps) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const uint64_t pid = first + i;
    rng.pid_lo = (uint32_t)pid;
    rng.pid_hi = (uint32_t)(pid >> 32);
    uint64_t h = kFnvBasis;
    float4 u = rng.draw(0, 0);
    float3 x = make_float3(fmaf(u.x, S.lx1 - S.lx0, S.lx0), fmaf(u.y, S.ly1 - S.ly0, S.ly0), 1.0f);
    float3 nrm = make_float3(0.0f, 0.0f, -1.0f);
    float3 d = cosine_dir(nrm, u.z, u.w);
    float w = S.w0;
    int m = 0;                          // Phong continuations so far
    float hits = 0.0f, in_view = 0.0f;
    uint32_t end = 0;
    for (int k = 1;; ++k) {
        float t;
        const int id = surf_hit(S, x, d, t, nrm);
        if (id == -100) {
            end = 1;
            break;
        }
        x = make_float3(fmaf(t, d.x, x.x), fmaf(t, d.y, x.y), fmaf(t, d.z, x.z));
        hits += 1.0f;
        h = fnv_word(h, (uint32_t)(id + 100));
        const bool phong = id == S.phong;
        const float dn = d.x * nrm.x + d.y * nrm.y + d.z * nrm.z;
        const float3 mir = make_float3(d.x - 2.0f * dn * nrm.x, d.y - 2.0f * dn * nrm.y, d.z - 2.0f * dn * nrm.z);
        int32_t pixv = -1;
        const Proj q = project(S.cam, x);
        if (q.pix >= 0) {
            const float cn = nrm.x * q.dir.x + nrm.y * q.dir.y + nrm.z * q.dir.z;
            if (cn > 0.0f && surf_visible(S, x, q.dir, sqrtf(q.r2))) {
                pixv = q.pix;
                in_view += 1.0f;
                const float base = w * (0.318309886183790672f * cn) / (q.r2 * __ldg(S.omega + q.pix)) * inv_norm;
                const float cm = phong ? mir.x * q.dir.x + mir.y * q.dir.y + mir.z * q.dir.z : kNoPhong;
                const uint32_t pos = atomicAdd(P.count, 1u);
                if (pos < P.cap)
                    P.raw[pos] = make_uint4(__float_as_uint(base), __float_as_uint(cm), (uint32_t)q.pix,
                                           (uint32_t)i | ((uint32_t)m << 28));
            }
        }
        h = fnv_word(h, (uint32_t)pixv);
        u = rng.draw((uint32_t)k, 0);
        if (k == S.max_orders) {
            end = 2;
            break;
        }
        if (k >= S.rr_start) {
            if (u.x <= S.rr_q) {
                w *= S.inv_q;
            } else {
                end = 3;
                break;
            }
        }
        d = cosine_dir(nrm, u.y, u.z);
        if (phong && m < 15) {
            P.pc[(uint64_t)m * P.n + i] = mir.x * d.x + mir.y * d.y + mir.z * d.z;
            ++m;
        }
    }
    h = fnv_word(h, end);
    if (fps) fps[i] = h;
    if (tallies) {
        // counts only: the weights depend on (kappa, gamma), which the store does not know
        atomicAdd(tallies + PT_T_COLLISIONS, (double)hits);
        atomicAdd(tallies + PT_T_IN_VIEW, (double)in_view);
        atomicAdd(tallies + PT_T_INJECTED, (double)S.w0);
    }
}

__device__ __forceinline__ float phong_f(float kappa, float gamma, float c) {
    return 1.0f - kappa + kappa * powf(fmaxf(c, 0.0f), gamma);
}

// Counting sort of the events by pixel, once per store: histogram, one-block
// exclusive scan, scatter.  (The pixel is in range by construction; the clamp
// keeps every index inside the bins.)
__device__ __forceinline__ uint32_t ev_pixel(const SurfStore& P, const uint4& r) { return min(r.z, P.n_pix - 1u); }

__global__ void k_surf_hist(SurfStore P) {
    const uint32_t n_ev = min(*P.count, (uint32_t)P.cap);
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n_ev; e += gridDim.x * blockDim.x)
        atomicAdd(P.bins + ev_pixel(P, P.raw[e]), 1u);
}

__global__ void __launch_bounds__(1024) k_surf_scan(SurfStore P) {
    __shared__ uint32_t part[1024];
    const uint32_t n = P.n_pix, per = (n + 1023u) / 1024u;
    const uint32_t lo = min(threadIdx.x * per, n), hi = min(lo + per, n);
    uint32_t s = 0;
    for (uint32_t k = lo; k < hi; ++k) s += P.bins[k];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {
        const uint32_t v = threadIdx.x >= (unsigned)d ? part[threadIdx.x - d] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
    for (uint32_t k = lo; k < hi; ++k) {
        const uint32_t c = P.bins[k];
        P.bins[n + k] = run;
        run += c;
    }
}

__global__ void k_surf_scatter(SurfStore P) {
    const uint32_t n_ev = min(*P.count, (uint32_t)P.cap);
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n_ev; e += gridDim.x * blockDim.x) {
        const uint4 r = P.raw[e];
        P.ev[atomicAdd(P.bins + P.n_pix + ev_pixel(P, r), 1u)] = r;
    }
}

// (kappa, gamma) come from the arguments, or from device memory when theta is
// given (the optimiser's parameters, read without a host round trip).  A warp
// takes 32 consecutive events (sorted by pixel), sums the contributions of
// each run of equal pixels in FP64 (a segmented shuffle scan) and sends one
// red per run.
__global__ void k_surf_reweight(SurfStore P, float kappa, float gamma, const float* __restrict__ theta,
                                double* __restrict__ images, float* __restrict__ cache) {
    if (theta) {
        kappa = theta[0];
        gamma = theta[1];
    }
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint64_t n_ev = min(*P.count, (uint32_t)P.cap);
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t c = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c * 32 < n_ev; c += warps) {
        const uint64_t e = c * 32 + lane;
        int key = -1 - lane;   // never equal across lanes
        double sum = 0.0;
        if (e < n_ev) {
            const uint4 r = P.ev[e];
            const uint32_t i = r.w & 0x0fffffffu, m = r.w >> 28;
            float f = __uint_as_float(r.x);
            for (uint32_t k = 0; k < m; ++k) f *= phong_f(kappa, gamma, P.pc[(uint64_t)k * P.n + i]);
            const float cm = __uint_as_float(r.y);
            if (cm > -1.5f) f *= phong_f(kappa, gamma, cm);
            cache[e] = f;
            key = (int)ev_pixel(P, r);
            sum = (double)f;
        }
        const int prev = __shfl_up_sync(full, key, 1);
        const unsigned heads = __ballot_sync(full, lane == 0 || prev != key);
        const int start = 31 - __clz(heads & ((2u << lane) - 1u));
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const double o = __shfl_up_sync(full, sum, d);
            if (lane - d >= start) sum += o;
        }
        const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
        if (tail && key >= 0 && sum != 0.0) atomicAdd(images + key, sum);
    }
}

// d log f_r / d (kappa, gamma) at lobe cosine c
__device__ __forceinline__ float2 phong_dlog(float kappa, float gamma, float c) {
    const float cg = c > 0.0f ? powf(c, gamma) : 0.0f;
    const float f = 1.0f - kappa + kappa * cg;
    return make_float2((cg - 1.0f) / f, c > 0.0f ? kappa * cg * logf(c) / f : 0.0f);
}

__global__ void __launch_bounds__(256) k_surf_grad(SurfStore P, float kappa, float gamma,
                                                   const float* __restrict__ theta,
                                                   const double* __restrict__ dldi, const float* __restrict__ cache,
                                                   double* __restrict__ grad) {
    if (theta) {
        kappa = theta[0];
        gamma = theta[1];
    }
    const uint32_t n_ev = min(*P.count, (uint32_t)P.cap);
    double g0 = 0.0, g1 = 0.0;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n_ev; e += gridDim.x * blockDim.x) {
        const uint4 r = P.ev[e];
        const uint32_t i = r.w & 0x0fffffffu, m = r.w >> 28;
        float2 dl = make_float2(0.0f, 0.0f);
        for (uint32_t k = 0; k < m; ++k) {
            const float2 q = phong_dlog(kappa, gamma, P.pc[(uint64_t)k * P.n + i]);
            dl.x += q.x;
            dl.y += q.y;
        }
        const float cm = __uint_as_float(r.y);
        if (cm > -1.5f) {
            const float2 q = phong_dlog(kappa, gamma, cm);
            dl.x += q.x;
            dl.y += q.y;
        }
        const double a = dldi[r.z] * (double)cache[e];
        g0 += a * (double)dl.x;
        g1 += a * (double)dl.y;
    }
    // both sums go to the same two addresses: reduce over the block first, so
    // that one FP64 atomic per block and parameter reaches memory
    for (int o = 16; o > 0; o >>= 1) {
        g0 += __shfl_xor_sync(0xffffffffu, g0, o);
        g1 += __shfl_xor_sync(0xffffffffu, g1, o);
    }
    __shared__ double part[2][8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        part[0][warp] = g0;
        part[1][warp] = g1;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        g0 = lane < nw ? part[0][lane] : 0.0;
        g1 = lane < nw ? part[1][lane] : 0.0;
        for (int o = 4; o > 0; o >>= 1) {
            g0 += __shfl_xor_sync(0xffffffffu, g0, o);
            g1 += __shfl_xor_sync(0xffffffffu, g1, o);
        }
        if (lane == 0) {
            if (g0 != 0.0) atomicAdd(grad, g0);
            if (g1 != 0.0) atomicAdd(grad + 1, g1);
        }
    }
}

// Adam on u = (kappa, gamma / scale) (one step size suits both), then the
// projection onto 0 <= kappa <= 1, gamma >= 0 of Eq. phong; the step number
// lives in device memory (t = ++*step), so the whole update, including the
// step size lr / (1 + (t - 1) / decay) (decay = 0: constant), can be
// captured in a graph.  trace[2 (t-1) ..] receives (kappa, gamma) after step t.
__global__ void k_surf_adam(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                            const double* __restrict__ g, int32_t* __restrict__ step, float lr, float decay,
                            float scale, float b1, float b2, float eps, float* __restrict__ trace,
                            int32_t trace_cap) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int32_t t = ++(*step);
    if (decay > 0.0f) lr = (float)((double)lr / (1.0 + (double)(t - 1) / (double)decay));
    const float inv_bc1 = (float)(1.0 / (1.0 - pow((double)b1, (double)t)));
    const float inv_bc2 = (float)(1.0 / (1.0 - pow((double)b2, (double)t)));
    const float gu[2] = {__double2float_rn(g[0]), __double2float_rn(g[1] * (double)scale)};
    float u[2] = {theta[0], theta[1] / scale};
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const float mj = fmaf(b1, m[j], (1.0f - b1) * gu[j]);
        const float vj = fmaf(b2, v[j], (1.0f - b2) * gu[j] * gu[j]);
        m[j] = mj;
        v[j] = vj;
        u[j] = fmaxf(u[j] - lr * (mj * inv_bc1) / (sqrtf(vj * inv_bc2) + eps), 0.0f);
    }
    theta[0] = fminf(u[0], 1.0f);
    theta[1] = u[1] * scale;
    if (trace && t <= trace_cap) {
        trace[2 * (t - 1)] = theta[0];
        trace[2 * (t - 1) + 1] = theta[1];
    }
}

}  // namespace
}  // namespace pt

using namespace pt;

struct pt_surf {
    pt_scene* cams = nullptr;      // the camera (a one-voxel scene: frame, projection, pixel solid angles)
    float4* d_sph = nullptr;
    SurfDev dev{};
    int64_t n_pixels = 0;
};

struct pt_surf_paths {
    const pt_surf* scene = nullptr;
    SurfStore st{};
    uint64_t n_cap = 0;
    float* cache = nullptr;
    bool cache_valid = false;
};

namespace {
unsigned surf_grid(uint64_t n) { return (unsigned)std::min<uint64_t>((n + 255) / 256, (uint64_t)device_sms() * 16); }

void free_store(pt_surf_paths* p) {
    cudaFree(p->st.ev); cudaFree(p->st.raw); cudaFree(p->st.bins); cudaFree(p->st.pc); cudaFree(p->st.count);
    cudaFree(p->cache);
    p->st = SurfStore{};
    p->cache = nullptr;
    p->n_cap = 0;
}

int surf_status(const char* what) {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PT_OK : fail(PT_E_CUDA, "%s launch: %s", what, cudaGetErrorString(e));
}
}  // namespace

extern "C" {

int surf_scene_create(const pt_surf_desc* d, pt_surf** out) {
    if (!d || !out || (!d->spheres && d->n_spheres > 0)) return fail(PT_E_INVALID, "surf_scene_create: null argument");
    *out = nullptr;
    if (d->n_spheres < 0 || d->n_spheres > 1024 || d->phong >= d->n_spheres || d->max_orders < 1 ||
        d->max_orders > PT_MAX_ORDERS || !(d->rr_q > 0.0f && d->rr_q <= 1.0f) || !(d->radiance >= 0.0f) ||
        !(d->light[0] < d->light[1] && d->light[2] < d->light[3]))
        return fail(PT_E_INVALID, "surf_scene_create: bad scene description");
    for (int i = 0; i < d->n_spheres; ++i)
        if (!(d->spheres[4 * i + 3] > 0.0f)) return fail(PT_E_INVALID, "surf_scene_create: sphere %d radius", i);
    // the camera through the volume scene's camera model: a one-voxel unit box
    pt_scene_desc vd{};
    vd.nx = vd.ny = vd.nz = 1;
    vd.voxel = 1.0f;
    vd.albedo_cloud = 1.0f;
    vd.albedo_air = 1.0f;
    vd.sun_dir[2] = -1.0f;
    vd.sun_irradiance = 1.0f;
    vd.n_cams = 1;
    vd.cams = &d->camera;
    vd.max_orders = d->max_orders;
    vd.rr_start = d->rr_start;
    vd.rr_q = d->rr_q;
    pt_surf* s = new (std::nothrow) pt_surf();
    if (!s) return fail(PT_E_OOM, "host allocation");
    if (int rc = pt_scene_create(&vd, &s->cams)) {
        delete s;
        return rc;
    }
    if (d->n_spheres > 0) {
        if (cudaMalloc(&s->d_sph, sizeof(float4) * d->n_spheres) != cudaSuccess ||
            cudaMemcpy(s->d_sph, d->spheres, sizeof(float4) * d->n_spheres, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            pt_scene_free(s->cams);
            cudaFree(s->d_sph);
            delete s;
            return fail(PT_E_OOM, "surf_scene_create: sphere table");
        }
    }
    SurfDev& S = s->dev;
    if (cudaMemcpy(&S.cam, scene_cams(s->cams), sizeof(DevCam), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        pt_scene_free(s->cams);
        cudaFree(s->d_sph);
        delete s;
        return fail(PT_E_CUDA, "surf_scene_create: camera");
    }
    S.omega = scene_omega(s->cams);
    S.sph = s->d_sph;
    S.n_sph = d->n_spheres;
    S.phong = d->phong;
    S.max_orders = d->max_orders;
    S.rr_start = d->rr_start;
    S.lx0 = d->light[0]; S.lx1 = d->light[1]; S.ly0 = d->light[2]; S.ly1 = d->light[3];
    S.w0 = (float)(3.14159265358979323846 * (double)d->radiance * ((double)d->light[1] - d->light[0]) *
                   ((double)d->light[3] - d->light[2]));
    S.rr_q = d->rr_q;
    S.inv_q = 1.0f / d->rr_q;
    s->n_pixels = pt_scene_pixels(s->cams);
    *out = s;
    return PT_OK;
}

int surf_scene_free(pt_surf* s) {
    if (!s) return PT_OK;
    cudaDeviceSynchronize();
    pt_scene_free(s->cams);
    cudaFree(s->d_sph);
    delete s;
    return PT_OK;
}

int64_t surf_scene_pixels(const pt_surf* s) { return s ? s->n_pixels : 0; }

int surf_store(const pt_surf* s, uint64_t first, uint64_t n, double n_norm, uint64_t seed, uint32_t epoch,
               pt_surf_paths** pp, double* tallies, uint64_t* fps, uint32_t flags, void* stream) {
    NvtxRange nvtx_range("surf_store");
    if (!s || !pp) return fail(PT_E_INVALID, "surf_store: null scene or handle slot");
    if (n == 0 || n >= (1ull << 28)) return fail(PT_E_INVALID, "surf_store: n_paths must be in 1..2^28-1");
    if (!(n_norm > 0.0)) return fail(PT_E_INVALID, "surf_store: n_norm must be > 0");
    cudaStream_t st = (cudaStream_t)stream;
    pt_surf_paths* p = *pp;
    const bool created = !p;
    if (!p) {
        p = new (std::nothrow) pt_surf_paths();
        if (!p) return fail(PT_E_OOM, "host allocation");
    } else if (p->scene != s) {
        return fail(PT_E_INVALID, "surf_store: handle belongs to another scene");
    }
    p->scene = s;
    if (p->n_cap < n) {
        if (!created) cudaStreamSynchronize(st);
        free_store(p);
        const uint64_t cap = n * (uint64_t)s->dev.max_orders;
        if (cudaMalloc(&p->st.ev, sizeof(uint4) * cap) != cudaSuccess ||
            cudaMalloc(&p->st.raw, sizeof(uint4) * cap) != cudaSuccess ||
            cudaMalloc(&p->st.bins, sizeof(uint32_t) * 2 * (uint64_t)s->n_pixels) != cudaSuccess ||
            cudaMalloc(&p->st.pc, sizeof(float) * n * 15) != cudaSuccess ||
            cudaMalloc(&p->st.count, sizeof(uint32_t)) != cudaSuccess ||
            cudaMalloc(&p->cache, sizeof(float) * cap) != cudaSuccess) {
            cudaGetLastError();
            free_store(p);
            if (created) delete p;
            return fail(PT_E_OOM, "surf_store: no device memory for %llu paths", (unsigned long long)n);
        }
        p->n_cap = n;
        p->st.cap = cap;
        p->st.n_pix = (uint32_t)s->n_pixels;
    }
    *pp = p;
    p->st.n = n;
    p->cache_valid = false;
    const bool sort = (flags & PT_SORT) != 0;
    cudaMemsetAsync(p->st.count, 0, sizeof(uint32_t), st);
    if (sort) cudaMemsetAsync(p->st.bins, 0, sizeof(uint32_t) * p->st.n_pix, st);
    // the tracer writes the kept buffer directly unless a sort follows
    SurfStore w = p->st;
    if (!sort) w.raw = w.ev;
    Rng rng{};
    rng.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    rng.epoch = epoch;
    rng.scene = 0;
    k_surf_store<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(s->dev, w, first, (float)(1.0 / n_norm), rng,
                                                             tallies, fps);
    if (sort) {
        k_surf_hist<<<surf_grid(p->st.cap), 256, 0, st>>>(p->st);
        k_surf_scan<<<1, 1024, 0, st>>>(p->st);
        k_surf_scatter<<<surf_grid(p->st.cap), 256, 0, st>>>(p->st);
    }
    return surf_status("surf_store");
}

int surf_reweight(pt_surf_paths* p, double kappa, double gamma, double* images, uint32_t flags, void* stream) {
    NvtxRange nvtx_range("surf_reweight");
    if (!p || !p->scene || !images) return fail(PT_E_INVALID, "surf_reweight: null argument");
    if (!(kappa >= 0.0 && kappa <= 1.0 && gamma >= 0.0)) return fail(PT_E_INVALID, "surf_reweight: kappa in [0,1], gamma >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    if (!(flags & PT_ACCUMULATE)) cudaMemsetAsync(images, 0, sizeof(double) * p->scene->n_pixels, st);
    k_surf_reweight<<<surf_grid(p->st.cap), 256, 0, st>>>(p->st, (float)kappa, (float)gamma, nullptr, images,
                                                          p->cache);
    p->cache_valid = true;
    return surf_status("surf_reweight");
}

int surf_reweight_dev(pt_surf_paths* p, const float* theta, double* images, uint32_t flags, void* stream) {
    NvtxRange nvtx_range("surf_reweight_dev");
    if (!p || !p->scene || !theta || !images) return fail(PT_E_INVALID, "surf_reweight_dev: null argument");
    cudaStream_t st = (cudaStream_t)stream;
    if (!(flags & PT_ACCUMULATE)) cudaMemsetAsync(images, 0, sizeof(double) * p->scene->n_pixels, st);
    k_surf_reweight<<<surf_grid(p->st.cap), 256, 0, st>>>(p->st, 0.0f, 0.0f, theta, images, p->cache);
    p->cache_valid = true;
    return surf_status("surf_reweight_dev");
}

int surf_grad(pt_surf_paths* p, double kappa, double gamma, const double* dldi, double* grad, uint32_t flags,
              void* stream) {
    NvtxRange nvtx_range("surf_grad");
    if (!p || !p->scene || !dldi || !grad) return fail(PT_E_INVALID, "surf_grad: null argument");
    if (!p->cache_valid) return fail(PT_E_INVALID, "surf_grad: needs a preceding surf_reweight");
    cudaStream_t st = (cudaStream_t)stream;
    if (!(flags & PT_ACCUMULATE)) cudaMemsetAsync(grad, 0, 2 * sizeof(double), st);
    k_surf_grad<<<surf_grid(p->st.cap), 256, 0, st>>>(p->st, (float)kappa, (float)gamma, nullptr, dldi, p->cache,
                                                      grad);
    return surf_status("surf_grad");
}

int surf_grad_dev(pt_surf_paths* p, const float* theta, const double* dldi, double* grad, uint32_t flags,
                  void* stream) {
    NvtxRange nvtx_range("surf_grad_dev");
    if (!p || !p->scene || !theta || !dldi || !grad) return fail(PT_E_INVALID, "surf_grad_dev: null argument");
    if (!p->cache_valid) return fail(PT_E_INVALID, "surf_grad_dev: needs a preceding surf_reweight");
    cudaStream_t st = (cudaStream_t)stream;
    if (!(flags & PT_ACCUMULATE)) cudaMemsetAsync(grad, 0, 2 * sizeof(double), st);
    k_surf_grad<<<surf_grid(p->st.cap), 256, 0, st>>>(p->st, 0.0f, 0.0f, theta, dldi, p->cache, grad);
    return surf_status("surf_grad_dev");
}

int surf_adam_step(float* theta, float* m, float* v, const double* grad, int32_t* step, float lr, float lr_decay,
                   float gamma_scale, float b1, float b2, float eps, float* trace, int32_t trace_cap, void* stream) {
    if (!theta || !m || !v || !grad || !step) return fail(PT_E_INVALID, "surf_adam_step: null argument");
    if (!(gamma_scale > 0.0f) || !(lr >= 0.0f) || !(lr_decay >= 0.0f) || trace_cap < 0)
        return fail(PT_E_INVALID, "surf_adam_step: gamma_scale > 0, lr >= 0, lr_decay >= 0, trace_cap >= 0");
    k_surf_adam<<<1, 32, 0, (cudaStream_t)stream>>>(theta, m, v, grad, step, lr, lr_decay, gamma_scale, b1, b2, eps,
                                                    trace, trace ? trace_cap : 0);
    return surf_status("surf_adam_step");
}

int surf_paths_events(const pt_surf_paths* p, uint64_t* n_events) {
    if (!p || !n_events) return fail(PT_E_INVALID, "surf_paths_events: null argument");
    uint32_t c = 0;
    if (cudaMemcpy(&c, p->st.count, sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
        return surf_status("surf_paths_events");
    *n_events = c;
    return c <= p->st.cap ? PT_OK : fail(PT_E_INVALID, "surf_paths_events: event capacity exceeded");
}

int surf_paths_free(pt_surf_paths* p) {
    if (!p) return PT_OK;
    cudaDeviceSynchronize();
    free_store(p);
    delete p;
    return PT_OK;
}

}  // extern "C"
