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
constexpr uint32_t kKindEntry = 0u << 28;
constexpr uint32_t kKindScatter = 1u << 28;
enum : uint32_t { kEndNone = 0, kEndEscape = 1, kEndTrunc = 2, kEndRR = 3, kEndMiss = 4 };

// device-side error bits (pt_check)
enum : int { kErrIndex = 1, kErrIter = 2, kErrRecord = 4, kErrStore = 8 };

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

// ------------------------------------------------------- FP64 accumulation --
// FP32 terms are converted exactly to FP64 and added with one red each: the
// only FP64 steps.  (The conversion uses the FP64 conversion unit; at well
// under one conversion per voxel crossing it is far from that unit's rate.)
__device__ __forceinline__ void red_add(double* p, float v) { atomicAdd(p, (double)v); }

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
    const float inv_r = 1.0f / sqrtf(p.r2);   // correctly rounded: the phase function is steep
    p.dir = make_float3(-qx * inv_r, -qy * inv_r, -qz * inv_r);
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

// ---------------------------------------------------------- voxel ids --
// Vertices carry packed voxel coordinates, ix | iy << 9 | iz << 18 (grids of
// at most 512 voxels per axis); gathers use the linear x-fastest index.
constexpr uint32_t kVoxMask = 0x07ffffffu;
constexpr int kAxisMax = 512;

__device__ __forceinline__ uint32_t pack_vox(int ix, int iy, int iz) {
    return (uint32_t)ix | ((uint32_t)iy << 9) | ((uint32_t)iz << 18);
}
__device__ __forceinline__ int lin_vox(const DevScene& S, uint32_t pv) {
    return (int)(pv & 511u) + S.nx * ((int)((pv >> 9) & 511u) + S.ny * (int)((pv >> 18) & 511u));
}
__device__ __forceinline__ bool vox_ok(const DevScene& S, uint32_t pv) {
    return (int)(pv & 511u) < S.nx && (int)((pv >> 9) & 511u) < S.ny && (int)((pv >> 18) & 511u) < S.nz;
}

// ------------------------------------------------------------------ DDA --
// Traversal of the voxels cut by p + t d, t in [0, tmax] (clipped to the
// box), starting in the voxel (ix, iy, iz) that contains p.  Per axis the
// k-th face crossed after the start lies at t = t0 + k D (t0 the first face,
// D = voxel / |d| the spacing), one rounding from its exact value; the
// three candidates are recomputed every step without branches.  Ties step x
// before y before z; zero-length crossings are visited with length 0.  The
// box exit bounds the walk (the exit face has the same formula), and an
// index check with a step budget records an error instead of running off.
struct Dda {
    float tnx, tny, tnz;   // t of the next face per axis
    float kx, ky, kz;      // faces crossed so far per axis
    float Dx, Dy, Dz;      // face spacing per axis
    float Ax, Ay, Az;      // t of the first face per axis
    int sx, sy, sz;        // linear-index step per axis
    int idx;
    float t, tend;
    int budget;

    __device__ __forceinline__ void axis(float pc, float dc, int ic, int n, float o, float vox, int stride, float& tn,
                                         float& k, float& D, float& A, int& si) {
        const float INF = __int_as_float(0x7f800000);
        k = 0.0f;
        if (dc != 0.0f) {
            const float inv = 1.0f / dc;
            D = vox * fabsf(inv);
            const bool up = dc > 0.0f;
            A = (fmaf((float)(up ? ic + 1 : ic), vox, o) - pc) * inv;
            si = up ? stride : -stride;
            tn = A;
            tend = fminf(tend, fmaf((float)(up ? n - 1 - ic : ic), D, A));   // exit face
        } else {
            D = 0.0f;
            A = INF;
            si = 0;
            tn = INF;
        }
    }

    __device__ __forceinline__ void init(const DevScene& S, float3 p, float3 d, int ix, int iy, int iz, float tmax) {
        idx = ix + S.nx * (iy + S.ny * iz);
        t = 0.0f;
        tend = tmax;
        budget = S.nx + S.ny + S.nz + 4;
        axis(p.x, d.x, ix, S.nx, S.ox, S.vox, 1, tnx, kx, Dx, Ax, sx);
        axis(p.y, d.y, iy, S.ny, S.oy, S.vox, S.nx, tny, ky, Dy, Ay, sy);
        axis(p.z, d.z, iz, S.nz, S.oz, S.vox, S.nx * S.ny, tnz, kz, Dz, Az, sz);
    }
    __device__ __forceinline__ void init(const DevScene& S, float3 p, float3 d, uint32_t pv, float tmax) {
        init(S, p, d, (int)(pv & 511u), (int)((pv >> 9) & 511u), (int)((pv >> 18) & 511u), tmax);
    }

    // t of the next face crossing
    __device__ __forceinline__ float next() const { return fminf(tnx, fminf(tny, tnz)); }

    // length of the current voxel's crossing, given next() == tn
    __device__ __forceinline__ float seg(float tn) const { return fmaxf(fminf(tn, tend) - t, 0.0f); }

    // move into the next voxel; false when the ray ended or an invariant broke
    __device__ __forceinline__ bool step(const DevScene& S, float tn) {
        if (tn >= tend) return false;
        const bool mx = tnx == tn;
        const bool my = !mx && tny == tn;
        const bool mz = !mx && !my;
        kx = mx ? kx + 1.0f : kx;
        ky = my ? ky + 1.0f : ky;
        kz = mz ? kz + 1.0f : kz;
        idx += mx ? sx : (my ? sy : sz);
        tnx = fmaf(kx, Dx, Ax);
        tny = fmaf(ky, Dy, Ay);
        tnz = fmaf(kz, Dz, Az);
        t = fmaxf(t, tn);
        if ((unsigned)idx >= (unsigned)S.V || --budget < 0) {
            atomicOr(S.err, (unsigned)idx >= (unsigned)S.V ? kErrIndex : kErrIter);
            return false;
        }
        return true;
    }

    // packed coordinates of the current voxel, given the start voxel and d
    __device__ __forceinline__ uint32_t coords(uint32_t pv0, float3 d) const {
        const int cx = (int)(pv0 & 511u) + (d.x > 0.0f ? (int)kx : -(int)kx);
        const int cy = (int)((pv0 >> 9) & 511u) + (d.y > 0.0f ? (int)ky : -(int)ky);
        const int cz = (int)((pv0 >> 18) & 511u) + (d.z > 0.0f ? (int)kz : -(int)kz);
        return pack_vox(cx, cy, cz);
    }
};

// optical depth of the grid `beta` (+ air) from p along d to the box exit
__device__ __forceinline__ float optical_depth_to_exit(const DevScene& S, const float* __restrict__ beta, float3 p,
                                                       float3 d, uint32_t pv, int* crossings) {
    Dda r;
    r.init(S, p, d, pv, __int_as_float(0x7f800000));
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
__device__ __forceinline__ void scatter_ray(const DevScene& S, double* __restrict__ grad, float3 p, float3 d,
                                            uint32_t pv, float tmax, float s) {
    Dda r;
    r.init(S, p, d, pv, tmax);
    for (;;) {
        const float tn = r.next();
        const float l = r.seg(tn);
        if (l > 0.0f) red_add(grad + r.idx, -s * l);
        if (!r.step(S, tn)) break;
    }
}

// sum of dbeta * l over the segment p + t d, t <= tmax (stored flight)
__device__ __forceinline__ float delta_depth(const DevScene& S, const float* __restrict__ dbeta, float3 p, float3 d,
                                             uint32_t pv, float tmax) {
    Dda r;
    r.init(S, p, d, pv, tmax);
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
//   A = {x, y, z (float bits), packed voxel | kind << 28 | end << 30}
//   B = {incoming direction x, y, z, length of the flight into the vertex}
// Vertex 0 is the box entry (incoming = sun direction, length 0).
__device__ __forceinline__ uint4 rec_a(float3 x, uint32_t pv, uint32_t kind) {
    return make_uint4(__float_as_uint(x.x), __float_as_uint(x.y), __float_as_uint(x.z), (pv & kVoxMask) | kind);
}

}  // namespace pt
