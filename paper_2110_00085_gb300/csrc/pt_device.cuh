// pt_device.cuh -- device building blocks shared by the kernels of
// libpathrecycle: scene constants, Philox4x32-10, phase functions and their
// samplers, the orthonormal basis, the camera projection, the voxel
// traversal (3D-DDA) and the FP32 -> FP64 widening used for accumulation.
//
// Method: Czerninski & Schechner, arXiv 2110.00085, Sec. 3.4 (path tracing
// with distance and direction sampling, local estimation), Sec. 4.4 (path
// score function), Sec. 5 (path recycling and sorting).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/pathrecycle.h"

namespace pt {

constexpr float kPi = 3.14159265358979323846f;
constexpr int kMaxCams = PT_MAX_CAMS;
constexpr int kMaxOrders = PT_MAX_ORDERS;
constexpr int kBuckets = PT_MAX_ORDERS + 1;

// vertex record kinds (bits 28..29 of the voxel word) and path ends (30..31)
constexpr uint32_t kVoxMask = 0x0fffffffu;
constexpr uint32_t kKindEntry = 0u << 28;
constexpr uint32_t kKindScatter = 1u << 28;
enum : uint32_t { kEndNone = 0, kEndEscape = 1, kEndTrunc = 2, kEndRR = 3, kEndMiss = 4 };

// device-side error bits (pt_check)
enum : int { kErrIndex = 1, kErrIter = 2, kErrRecord = 4 };

struct DevCam {
    float C[3], F[3], R[3], U[3];
    float inv_tx, inv_ty;   // 1 / tan(half field of view)
    float half_w, half_h;   // W/2, H/2
    int W, H;
    int off;                // first pixel of this camera in the image array
    int pad;
};

struct DevScene {
    int nx, ny, nz, n_cams;
    int max_orders, rr_start;
    uint32_t scene_id;
    int V;
    float vox, inv_vox;
    float ox, oy, oz;
    float beta_air, alb_c, alb_a, hg_g;
    float hg_k;             // (1 - g^2) / (4 pi)
    float hg_1pg2, hg_m2g;  // 1 + g^2, -2 g
    float sx, sy, sz;       // sun propagation direction
    float e1[3], e2[3];     // sun-rectangle axes
    float amin, alen, bmin, blen, hmin;
    float w0;               // sun irradiance * rectangle area
    float rr_q, inv_q;
    int64_t n_pixels;
    const DevCam* cams;
    const float* omega;     // pixel solid angles, images layout
    int* err;
};

// --------------------------------------------------------------- Philox --
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// uniform in (0, 1]: exact in FP32 (24 bits)
__device__ __forceinline__ float u01(uint32_t w) {
    return __uint2float_rn((w >> 8) + 1u) * 5.9604644775390625e-8f;
}

struct Rng {
    uint2 key;
    uint32_t pid_lo, pid_hi, epoch, scene;
    __device__ __forceinline__ float4 draw(uint32_t event, uint32_t tag) const {
        const uint4 c = make_uint4(pid_lo, pid_hi, (event & 0xffu) | ((tag & 0xffu) << 8) | ((epoch & 0xffffu) << 16),
                                   scene);
        const uint4 w = philox4x32_10(c, key);
        return make_float4(u01(w.x), u01(w.y), u01(w.z), u01(w.w));
    }
};

// -------------------------------------------------------------- FNV-1a --
__device__ __forceinline__ uint64_t fnv_word(uint64_t h, uint32_t w) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        h ^= (uint64_t)((w >> (8 * i)) & 0xffu);
        h *= 0x100000001b3ull;
    }
    return h;
}
constexpr uint64_t kFnvBasis = 0xcbf29ce484222325ull;

// ------------------------------------------------- FP32 -> FP64 widening --
// Exact widening with integer operations only (no FP64 pipe, which is
// narrow on GB300).  Subnormal floats flush to zero; inf/nan keep class.
__device__ __forceinline__ double widen(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = (b >> 23) & 0xffu;
    const uint64_t sign = (uint64_t)(b & 0x80000000u) << 32;
    uint64_t out;
    if (e == 0u) {
        out = sign;
    } else if (e == 0xffu) {
        out = sign | (0x7ffull << 52) | ((uint64_t)(b & 0x7fffffu) << 29);
    } else {
        out = sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)(b & 0x7fffffu) << 29);
    }
    return __longlong_as_double((long long)out);
}

__device__ __forceinline__ void red_add(double* p, float v) { atomicAdd(p, widen(v)); }

// ------------------------------------------------------ phase functions --
// Henyey-Greenstein (cloud) and Rayleigh (air), normalised on the sphere.
__device__ __forceinline__ float phase_hg(const DevScene& S, float mu) {
    const float den = fmaf(S.hg_m2g, mu, S.hg_1pg2);
    return S.hg_k / (den * sqrtf(den));
}
__device__ __forceinline__ float phase_rayleigh(float mu) {
    return 0.0596831036594607509f * fmaf(mu, mu, 1.0f);  // 3 / (16 pi)
}
// scattering function f_s = albedo_c beta_c f^c + albedo_a beta_a f^a
// (Eq. fs_scattering): the local-estimate and vertex factor of an event.
__device__ __forceinline__ float fs_medium(const DevScene& S, float bc, float mu) {
    return S.alb_c * bc * phase_hg(S, mu) + S.alb_a * S.beta_air * phase_rayleigh(mu);
}
// its cloud part divided by it: the vertex term of the path score (Eq. fs_deriv)
__device__ __forceinline__ float score_vertex(const DevScene& S, float bc, float mu) {
    return S.alb_c * phase_hg(S, mu) / fs_medium(S, bc, mu);
}

// A sampled polar angle is returned as (mu, 1 - mu): near forward
// scattering 1 - mu carries the angle, and computing it directly keeps its
// relative precision (the strongly peaked HG phase function amplifies
// direction errors in later local estimates).
struct Polar {
    float mu, omu;
};

// HG inverse CDF: with t = (1 - g^2) / (1 - g + 2 g u), mu = (1 + g^2 - t^2)/(2g),
// and equivalently 1 - mu = (1 - g)(1 - u)(t + 1 - g) / (1 - g + 2 g u).
__device__ __forceinline__ Polar sample_hg(const DevScene& S, float u) {
    const float g = S.hg_g;
    Polar p;
    if (fabsf(g) < 1e-3f) {
        p.omu = 2.0f * (1.0f - u);
        p.mu = fmaf(2.0f, u, -1.0f);
        return p;
    }
    const float den = 1.0f - g + 2.0f * g * u;
    const float t = (1.0f - g * g) / den;
    p.omu = fminf(2.0f, fmaxf(0.0f, (1.0f - g) * (1.0f - u) * (t + 1.0f - g) / den));
    p.mu = 1.0f - p.omu;
    return p;
}
// Rayleigh inverse CDF (Cardano on (mu^3 + 3 mu + 4)/8 = u)
__device__ __forceinline__ Polar sample_rayleigh(float u) {
    const float q = fmaf(4.0f, u, -2.0f);
    const float w = cbrtf(q + sqrtf(fmaf(q, q, 1.0f)));
    Polar p;
    p.mu = fminf(1.0f, fmaxf(-1.0f, w - 1.0f / w));
    p.omu = 1.0f - p.mu;
    return p;
}

// new direction at polar angle (mu, 1 - mu) and azimuth 2 pi u_phi about d,
// in the orthonormal basis of Duff et al. (JCGT 2017)
__device__ __forceinline__ float3 rotate_dir(float3 d, Polar pc, float u_phi) {
    const float mu = pc.mu;
    const float sign = copysignf(1.0f, d.z);
    const float a = -1.0f / (sign + d.z);
    const float b = d.x * d.y * a;
    const float3 b1 = make_float3(1.0f + sign * d.x * d.x * a, sign * b, -sign * d.x);
    const float3 b2 = make_float3(b, sign + d.y * d.y * a, -d.y);
    const float st = sqrtf(fmaxf(0.0f, pc.omu * (2.0f - pc.omu)));
    float sp, cp;
    sincospif(2.0f * u_phi, &sp, &cp);
    return make_float3(st * cp * b1.x + st * sp * b2.x + mu * d.x,
                       st * cp * b1.y + st * sp * b2.y + mu * d.y,
                       st * cp * b1.z + st * sp * b2.z + mu * d.z);
}

__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// ---------------------------------------------------------------- camera --
// pixel index inside camera k (row-major, row 0 at top), -1 when the point
// is behind the camera or outside the image; also the vector to the camera.
struct Proj {
    int pix;       // -1: not in view
    float r2;
    float3 dir;    // unit, from the point toward the camera
};
__device__ __forceinline__ Proj project(const DevCam& k, float3 x) {
    Proj p;
    p.pix = -1;
    const float qx = x.x - k.C[0], qy = x.y - k.C[1], qz = x.z - k.C[2];
    const float z = qx * k.F[0] + qy * k.F[1] + qz * k.F[2];
    if (!(z > 0.0f)) return p;
    const float sxn = (qx * k.R[0] + qy * k.R[1] + qz * k.R[2]) / z * k.inv_tx;
    const float syn = (qx * k.U[0] + qy * k.U[1] + qz * k.U[2]) / z * k.inv_ty;
    const float fc = floorf((sxn + 1.0f) * k.half_w);
    const float fr = floorf((1.0f - syn) * k.half_h);
    if (!(fc >= 0.0f && fc < (float)k.W && fr >= 0.0f && fr < (float)k.H)) return p;
    p.pix = (int)fr * k.W + (int)fc;
    p.r2 = qx * qx + qy * qy + qz * qz;
    const float r = sqrtf(p.r2);   // correctly rounded: the phase function is steep
    p.dir = make_float3(-qx / r, -qy / r, -qz / r);
    return p;
}

// contribution of one local estimate (one event, one camera): path weight,
// scattering function over the extinction that drew the collision, shadow
// transmittance, 1/r^2 and the pixel response 1/Omega -- one fixed order of
// operations shared by the plain and the recycled passes.
__device__ __forceinline__ float local_contrib(float w, float fs, float beta_draw, float T, float r2, float omega,
                                               float inv_norm) {
    return ((w * (fs / beta_draw)) * T) / (r2 * omega) * inv_norm;
}

// ------------------------------------------------------------------ DDA --
// Traversal of the voxels cut by p + t d, t in [0, tmax] (clipped to the
// box), starting in voxel (ix, iy, iz) that contains p.  Face crossings are
// recomputed from the face index each step (no accumulated error); ties
// step x before y before z; zero-length crossings are visited with length 0.
struct Dda {
    float px, py, pz;
    float ivx, ivy, ivz;   // 1/d per axis
    float kx, ky, kz;      // index of the next face per axis
    float tnx, tny, tnz;   // t of that face
    float gx, gy, gz;      // step (+1 / -1)
    int dx, dy, dz;        // linear-index step
    int idx;
    float t, tend;
    int iter, max_iter;

    __device__ __forceinline__ void init(const DevScene& S, float3 p, float3 d, int ix, int iy, int iz, float tmax) {
        px = p.x; py = p.y; pz = p.z;
        idx = ix + S.nx * (iy + S.ny * iz);
        t = 0.0f;
        tend = tmax;
        iter = 0;
        max_iter = S.nx + S.ny + S.nz + 4;
        const float INF = __int_as_float(0x7f800000);
        // x
        if (d.x != 0.0f) {
            ivx = 1.0f / d.x;
            gx = d.x > 0.0f ? 1.0f : -1.0f;
            kx = (float)(d.x > 0.0f ? ix + 1 : ix);
            dx = d.x > 0.0f ? 1 : -1;
            tnx = (fmaf(kx, S.vox, S.ox) - px) * ivx;
            const float te = (fmaf(d.x > 0.0f ? (float)S.nx : 0.0f, S.vox, S.ox) - px) * ivx;
            tend = fminf(tend, te);
        } else {
            ivx = 0.0f; gx = 0.0f; kx = 0.0f; dx = 0; tnx = INF;
        }
        if (d.y != 0.0f) {
            ivy = 1.0f / d.y;
            gy = d.y > 0.0f ? 1.0f : -1.0f;
            ky = (float)(d.y > 0.0f ? iy + 1 : iy);
            dy = d.y > 0.0f ? S.nx : -S.nx;
            tny = (fmaf(ky, S.vox, S.oy) - py) * ivy;
            const float te = (fmaf(d.y > 0.0f ? (float)S.ny : 0.0f, S.vox, S.oy) - py) * ivy;
            tend = fminf(tend, te);
        } else {
            ivy = 0.0f; gy = 0.0f; ky = 0.0f; dy = 0; tny = INF;
        }
        if (d.z != 0.0f) {
            ivz = 1.0f / d.z;
            gz = d.z > 0.0f ? 1.0f : -1.0f;
            kz = (float)(d.z > 0.0f ? iz + 1 : iz);
            dz = d.z > 0.0f ? S.nx * S.ny : -S.nx * S.ny;
            tnz = (fmaf(kz, S.vox, S.oz) - pz) * ivz;
            const float te = (fmaf(d.z > 0.0f ? (float)S.nz : 0.0f, S.vox, S.oz) - pz) * ivz;
            tend = fminf(tend, te);
        } else {
            ivz = 0.0f; gz = 0.0f; kz = 0.0f; dz = 0; tnz = INF;
        }
    }

    // t of the next face crossing
    __device__ __forceinline__ float next() const { return fminf(tnx, fminf(tny, tnz)); }

    // length of the current voxel's crossing, given next() == tn
    __device__ __forceinline__ float seg(float tn) const { return fmaxf(fminf(tn, tend) - t, 0.0f); }

    // move into the next voxel; false when the ray ended or an invariant broke
    __device__ __forceinline__ bool step(const DevScene& S, float tn) {
        if (tn >= tend) return false;
        if (tnx <= tny && tnx <= tnz) {
            kx += gx;
            idx += dx;
            tnx = (fmaf(kx, S.vox, S.ox) - px) * ivx;
        } else if (tny <= tnz) {
            ky += gy;
            idx += dy;
            tny = (fmaf(ky, S.vox, S.oy) - py) * ivy;
        } else {
            kz += gz;
            idx += dz;
            tnz = (fmaf(kz, S.vox, S.oz) - pz) * ivz;
        }
        t = fmaxf(t, tn);
        if ((unsigned)idx >= (unsigned)S.V) {
            atomicOr(S.err, kErrIndex);
            return false;
        }
        if (++iter > max_iter) {
            atomicOr(S.err, kErrIter);
            return false;
        }
        return true;
    }
};

__device__ __forceinline__ void voxel_coords(const DevScene& S, int v, int& ix, int& iy, int& iz) {
    ix = v % S.nx;
    const int r = v / S.nx;
    iy = r % S.ny;
    iz = r / S.ny;
}

// optical depth of the grid `beta` (+ air) from p along d to the box exit
__device__ __forceinline__ float optical_depth_to_exit(const DevScene& S, const float* __restrict__ beta, float3 p,
                                                       float3 d, int v, int* crossings) {
    int ix, iy, iz;
    voxel_coords(S, v, ix, iy, iz);
    Dda r;
    r.init(S, p, d, ix, iy, iz, __int_as_float(0x7f800000));
    float tau = 0.0f;
    int n = 0;
    for (;;) {
        const float tn = r.next();
        tau = fmaf(__ldg(beta + r.idx) + S.beta_air, r.seg(tn), tau);
        ++n;
        if (!r.step(S, tn)) break;
    }
    if (crossings) *crossings += n;
    return tau;
}

// scatter -s * l_v into grad over the voxels of the ray p + t d, t <= tmax
__device__ __forceinline__ void scatter_ray(const DevScene& S, double* __restrict__ grad, float3 p, float3 d, int v,
                                            float tmax, float s) {
    int ix, iy, iz;
    voxel_coords(S, v, ix, iy, iz);
    Dda r;
    r.init(S, p, d, ix, iy, iz, tmax);
    for (;;) {
        const float tn = r.next();
        const float l = r.seg(tn);
        if (l > 0.0f) red_add(grad + r.idx, -s * l);
        if (!r.step(S, tn)) break;
    }
}

// sum of dbeta * l over the segment p + t d, t <= tmax (stored flight)
__device__ __forceinline__ float delta_depth(const DevScene& S, const float* __restrict__ dbeta, float3 p, float3 d,
                                             int v, float tmax) {
    int ix, iy, iz;
    voxel_coords(S, v, ix, iy, iz);
    Dda r;
    r.init(S, p, d, ix, iy, iz, tmax);
    float acc = 0.0f;
    for (;;) {
        const float tn = r.next();
        acc = fmaf(__ldg(dbeta + r.idx), r.seg(tn), acc);
        if (!r.step(S, tn)) break;
    }
    return acc;
}

// -------------------------------------------------------- path records --
// Vertex record, two 16-byte streams:
//   A = {x, y, z (float bits), voxel | kind << 28 | end << 30}
//   B = {incoming direction x, y, z, length of the flight into the vertex}
// Vertex 0 is the box entry (incoming = sun direction, length 0).
__device__ __forceinline__ uint4 rec_a(float3 x, int v, uint32_t kind) {
    return make_uint4(__float_as_uint(x.x), __float_as_uint(x.y), __float_as_uint(x.z), ((uint32_t)v & kVoxMask) | kind);
}

}  // namespace pt
