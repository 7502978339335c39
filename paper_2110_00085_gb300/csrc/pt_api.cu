// pt_api.cu -- the C ABI of libpathrecycle (declared in include/pathrecycle.h):
// argument checks, handle lifetime, device buffers, and the small
// element-wise kernels (pixel solid angles, grid difference, loss residual,
// Adam).  Every call launches on the caller's stream; errors are returned,
// never raised, and described by pt_last_error().
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "pt_kernels.cuh"

using namespace pt;

// ------------------------------------------------------------ errors -----
namespace {
thread_local char g_err[512] = "";
}  // namespace

int pt::fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

namespace {

#define PT_CUDA(call)                                                                                \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) return fail(PT_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_));      \
    } while (0)

int launch_status(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(PT_E_CUDA, "%s launch: %s", what, cudaGetErrorString(e));
    return PT_OK;
}

cudaStream_t S_(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// ------------------------------------------------ small kernels ---------
// exact solid angle of each pixel (float64 arithmetic): signed corner sums of
// F(x, y) = atan(x y / sqrt(1 + x^2 + y^2)) on the unit-distance image plane
__global__ void k_pixel_omega(const DevCam* cams, int n_cams, const double* tans, float* omega, int64_t npix) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= npix) return;
    int c = 0;
    while (c + 1 < n_cams && g >= cams[c + 1].off) ++c;
    const DevCam& k = cams[c];
    const int64_t p = g - k.off;
    const int col = (int)(p % k.W), row = (int)(p / k.W);
    const double tx = tans[2 * c], ty = tans[2 * c + 1];
    const double xa = tx * (-1.0 + 2.0 * col / (double)k.W), xb = tx * (-1.0 + 2.0 * (col + 1) / (double)k.W);
    const double ya = ty * (1.0 - 2.0 * (row + 1) / (double)k.H), yb = ty * (1.0 - 2.0 * row / (double)k.H);
    auto F = [](double x, double y) { return atan(x * y / sqrt(1.0 + x * x + y * y)); };
    omega[g] = (float)(F(xb, yb) - F(xa, yb) - F(xb, ya) + F(xa, ya));
}

// photo-hull: a voxel stays unless some camera sees its centre on a clear
// pixel (radiance <= thr); cameras that do not see the centre have no say
__global__ void k_space_carve(DevScene S, const double* __restrict__ images, double thr,
                              uint8_t* __restrict__ mask) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < S.V; v += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(v % S.nx), iy = (int)((v / S.nx) % S.ny), iz = (int)(v / ((int64_t)S.nx * S.ny));
        const float3 x = make_float3(fmaf((float)ix + 0.5f, S.vox, S.ox), fmaf((float)iy + 0.5f, S.vox, S.oy),
                                     fmaf((float)iz + 0.5f, S.vox, S.oz));
        uint8_t keep = 1;
        for (int c = 0; c < S.n_cams && keep; ++c) {
            const Proj q = project(S.cams[c], x);
            if (q.pix >= 0 && images[S.cams[c].off + q.pix] <= thr) keep = 0;
        }
        mask[v] = keep;
    }
}

__global__ void k_resid(const double* __restrict__ img, const double* __restrict__ gt, int64_t n,
                        double* __restrict__ r, double* __restrict__ loss) {
    __shared__ double part[256];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double d = img[i] - gt[i];
        r[i] = d;
        s += d * d;
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss) atomicAdd(loss, 0.5 * part[0]);
}

// voxels with mask[i] == 0 (mask non-null) keep beta, m and v
__global__ void k_adam(float* __restrict__ beta, float* __restrict__ m, float* __restrict__ v,
                       const double* __restrict__ g, const uint8_t* __restrict__ mask, int64_t n, float lr, float b1,
                       float b2, float eps, float inv_bc1, float inv_bc2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (mask && !mask[i]) continue;
        const float gi = __double2float_rn(g[i]);
        const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        const float step = lr * (mi * inv_bc1) / (sqrtf(vi * inv_bc2) + eps);
        beta[i] = fmaxf(beta[i] - step, 0.0f);
    }
}

// voxels of an extinction grid that are NaN, infinite or negative
__global__ void k_check_beta(const float* __restrict__ beta, int64_t n, uint32_t* __restrict__ bad) {
    uint32_t c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float b = beta[i];
        if (!(b >= 0.0f) || isinf(b)) ++c;
    }
    if (c) atomicAdd(bad, c);
}

// step counter on the device: t = ++(*step); bias corrections 1/(1 - b^t)
__global__ void k_adam_count(int32_t* step, float b1, float b2, float* inv_bc) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int32_t t = ++(*step);
    inv_bc[0] = (float)(1.0 / (1.0 - pow((double)b1, (double)t)));
    inv_bc[1] = (float)(1.0 / (1.0 - pow((double)b2, (double)t)));
}

__global__ void k_adam_dev(float* __restrict__ beta, float* __restrict__ m, float* __restrict__ v,
                           const double* __restrict__ g, const uint8_t* __restrict__ mask, int64_t n, float lr,
                           float b1, float b2, float eps, const float* __restrict__ inv_bc) {
    const float inv_bc1 = inv_bc[0], inv_bc2 = inv_bc[1];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (mask && !mask[i]) continue;
        const float gi = __double2float_rn(g[i]);
        const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        const float step = lr * (mi * inv_bc1) / (sqrtf(vi * inv_bc2) + eps);
        beta[i] = fmaxf(beta[i] - step, 0.0f);
    }
}

unsigned grid_for(int64_t n, int bs, int per_sm = 32) {
    int64_t g = (n + bs - 1) / bs;
    const int64_t cap = (int64_t)device_sms() * per_sm;
    if (g > cap) g = cap;
    return (unsigned)(g < 1 ? 1 : g);
}

// ---------------------------------------------------- host geometry -----
void cross(const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
bool normalize(double* a) {
    const double n = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    if (!(n > 0.0) || !std::isfinite(n)) return false;
    a[0] /= n; a[1] /= n; a[2] /= n;
    return true;
}
}  // namespace

// ------------------------------------------------------------ handles ----
struct pt_scene {
    DevScene ds;
    DevCam* d_cams = nullptr;
    float* d_omega = nullptr;
    int* d_err = nullptr;
    int64_t n_pixels = 0;
};

int pt::device_sms() {
    static std::atomic<int> sms[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    int v = sms[dev].load(std::memory_order_relaxed);
    if (v <= 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
            cudaGetLastError();
            v = 1;
        }
        sms[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

const DevCam* pt::scene_cams(const pt_scene* sc) { return sc->d_cams; }
const float* pt::scene_omega(const pt_scene* sc) { return sc->d_omega; }

struct pt_paths {
    const pt_scene* scene = nullptr;
    uint64_t n = 0;            // paths of the latest store
    uint64_t rec_cap = 0;      // sorted records (and record-to-event map entries) the buffers hold
    int slots = 0;             // max_orders + 1
    float inv_norm = 1.0f;
    int64_t V = 0;
    float* beta_ref = nullptr;
    float* dbeta = nullptr;
    uint4* sa = nullptr;       // sorted records (stream A)
    float4* sb = nullptr;      // sorted records (stream B)
    Buckets* bk = nullptr;
    uint32_t* bad = nullptr;   // invalid extinction voxels found by the store's check
    uint32_t* abort_flag = nullptr;   // PT_ASYNC: the latest store did not fit (device)
    Events ev{};               // ev.cap = events the buffers hold
    float* cache = nullptr;
    uint64_t cache_cap = 0;    // floats
    uint64_t bytes = 0;
    bool cache_valid = false;
    uint64_t cache_token = 0;          // token of the reweight the cache holds (0: none)
    const float* cache_beta = nullptr; // that reweight's extinction grid
};

namespace {
// tokens of cache-writing reweights, unique over all handles of the process
uint64_t next_cache_token() {
    static std::atomic<uint64_t> counter{0};
    return ++counter;
}

void set_cache(pt_paths* p, bool valid, const float* beta_t) {
    p->cache_valid = valid;
    p->cache_token = valid ? next_cache_token() : 0;
    p->cache_beta = valid ? beta_t : nullptr;
}

// Stream-ordered pool of this library for the transient buffers of
// paths_store (one per device, created on first use).  It keeps the memory
// it has mapped (release threshold: unlimited), so repeated stores reuse it
// instead of mapping gigabytes again; no other allocator is affected.
cudaMemPool_t store_pool() {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        pools[dev] = pool;
    }
    return pools[dev];
}

void free_paths_buffers(pt_paths* p) {
    cudaFree(p->beta_ref); cudaFree(p->dbeta); cudaFree(p->sa); cudaFree(p->sb); cudaFree(p->bk); cudaFree(p->cache);
    cudaFree(p->bad);
    cudaFree(p->abort_flag);
    p->bad = nullptr;
    p->abort_flag = nullptr;
    cudaFree(p->ev.a); cudaFree(p->ev.b); cudaFree(p->ev.of_rec); cudaFree(p->ev.val); cudaFree(p->ev.hist);
    cudaFree(p->ev.cursor); cudaFree(p->ev.partial);
    p->beta_ref = p->dbeta = nullptr; p->sa = nullptr; p->sb = nullptr;
    p->bk = nullptr; p->cache = nullptr; p->cache_cap = 0; p->rec_cap = 0; p->bytes = 0;
    p->ev = Events{};
}

// Morton bits per axis for per-voxel event bins
int event_bin_bits(const DevScene& S) {
    const int m = std::max(std::max(S.nx, S.ny), S.nz);
    int b = 1;
    while ((1 << b) < m) ++b;
    return b;
}

template <class T>
int dev_alloc(T** p, uint64_t count, uint64_t* bytes, const char* what) {
    const size_t b = (size_t)count * sizeof(T);
    cudaError_t e = cudaMalloc((void**)p, b ? b : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(PT_E_OOM, "cudaMalloc(%s, %zu bytes): %s", what, b, cudaGetErrorString(e));
    }
    if (bytes) *bytes += b;
    return PT_OK;
}

SortedPaths sorted_view(const pt_paths* p) {
    SortedPaths s;
    s.rec_a = p->sa;
    s.rec_b = p->sb;
    s.buckets = p->bk;
    s.n_max = p->n;
    s.inv_norm = p->inv_norm;
    return s;
}
}  // namespace

extern "C" {

const char* pt_last_error(void) { return g_err; }
const char* pt_version(void) { return "pathrecycle 0.1 (sm_103a)"; }

}  // extern "C"

// Validates a scene description and derives its device constants on the host
// (camera frames, solid-angle inputs, sun rectangle).  Shared by every entry
// point that takes a pt_scene_desc.
int pt::describe_scene(const pt_scene_desc* d, DevScene& S, DevCam* hc, double* tans) {
    if (!d) return fail(PT_E_INVALID, "scene description: null");
    if (d->nx < 1 || d->ny < 1 || d->nz < 1) return fail(PT_E_INVALID, "grid dims must be >= 1");
    if (d->nx > kAxisMax || d->ny > kAxisMax || d->nz > kAxisMax)
        return fail(PT_E_INVALID, "grid dims must be <= %d per axis", kAxisMax);
    const int64_t V = (int64_t)d->nx * d->ny * d->nz;
    if (V >= (int64_t)1 << 28) return fail(PT_E_INVALID, "grid has %lld voxels; limit 2^28", (long long)V);
    if (!(d->voxel > 0.0f) || !std::isfinite(d->voxel)) return fail(PT_E_INVALID, "voxel size must be > 0");
    if (d->n_cams < 1 || d->n_cams > PT_MAX_CAMS || !d->cams)
        return fail(PT_E_INVALID, "n_cams must be in 1..%d with a camera array", PT_MAX_CAMS);
    if (d->max_orders < 1 || d->max_orders > PT_MAX_ORDERS)
        return fail(PT_E_INVALID, "max_orders must be in 1..%d", PT_MAX_ORDERS);
    if (!(d->rr_q > 0.0f && d->rr_q <= 1.0f)) return fail(PT_E_INVALID, "rr_q must be in (0, 1]");
    if (!(d->beta_air >= 0.0f) || !(d->albedo_cloud >= 0.0f && d->albedo_cloud <= 1.0f) ||
        !(d->albedo_air >= 0.0f && d->albedo_air <= 1.0f) || !(d->hg_g > -1.0f && d->hg_g < 1.0f))
        return fail(PT_E_INVALID, "medium parameters out of range");
    double s[3] = {d->sun_dir[0], d->sun_dir[1], d->sun_dir[2]};
    if (!normalize(s)) return fail(PT_E_INVALID, "sun_dir must be a nonzero vector");

    memset(&S, 0, sizeof(S));
    S.nx = d->nx; S.ny = d->ny; S.nz = d->nz; S.n_cams = d->n_cams; S.V = (int)V;
    S.max_orders = d->max_orders; S.rr_start = d->rr_start; S.scene_id = d->scene_id;
    S.vox = d->voxel; S.inv_vox = (float)(1.0 / (double)d->voxel);
    S.ox = d->origin[0]; S.oy = d->origin[1]; S.oz = d->origin[2];
    S.beta_air = d->beta_air; S.alb_c = d->albedo_cloud; S.alb_a = d->albedo_air; S.hg_g = d->hg_g;
    const double g = d->hg_g;
    S.hg_k = (float)((1.0 - g * g) / (4.0 * M_PI));
    S.hg_1pg2 = (float)(1.0 + g * g);
    S.hg_m2g = (float)(-2.0 * g);
    S.sx = (float)s[0]; S.sy = (float)s[1]; S.sz = (float)s[2];
    S.rr_q = d->rr_q; S.inv_q = (float)(1.0 / (double)d->rr_q);
    // sun rectangle: basis of Duff et al. around s, projections of the corners
    {
        const double sign = std::copysign(1.0, s[2]);
        const double a = -1.0 / (sign + s[2]);
        const double b = s[0] * s[1] * a;
        const double e1[3] = {1.0 + sign * s[0] * s[0] * a, sign * b, -sign * s[0]};
        const double e2[3] = {b, sign + s[1] * s[1] * a, -s[1]};
        double amin = INFINITY, amax = -INFINITY, bmin = INFINITY, bmax = -INFINITY, hmin = INFINITY;
        const double L[3] = {d->nx * (double)d->voxel, d->ny * (double)d->voxel, d->nz * (double)d->voxel};
        for (int c = 0; c < 8; ++c) {
            double p[3];
            for (int k = 0; k < 3; ++k) p[k] = d->origin[k] + ((c >> k) & 1) * L[k];
            const double pa = p[0] * e1[0] + p[1] * e1[1] + p[2] * e1[2];
            const double pb = p[0] * e2[0] + p[1] * e2[1] + p[2] * e2[2];
            const double ph = p[0] * s[0] + p[1] * s[1] + p[2] * s[2];
            amin = std::fmin(amin, pa); amax = std::fmax(amax, pa);
            bmin = std::fmin(bmin, pb); bmax = std::fmax(bmax, pb);
            hmin = std::fmin(hmin, ph);
        }
        for (int k = 0; k < 3; ++k) { S.e1[k] = (float)e1[k]; S.e2[k] = (float)e2[k]; }
        S.amin = (float)amin; S.alen = (float)(amax - amin);
        S.bmin = (float)bmin; S.blen = (float)(bmax - bmin);
        S.hmin = (float)(hmin - 1.0);
        S.w0 = (float)((double)d->sun_irradiance * (amax - amin) * (bmax - bmin));
    }
    // cameras
    int64_t off = 0;
    for (int c = 0; c < d->n_cams; ++c) {
        const pt_camera& k = d->cams[c];
        if (k.width < 1 || k.height < 1 || !(k.fov_y > 0.0f && k.fov_y < 3.1f))
            return fail(PT_E_INVALID, "camera %d: bad size or field of view", c);
        double F[3] = {(double)k.look_at[0] - k.pos[0], (double)k.look_at[1] - k.pos[1], (double)k.look_at[2] - k.pos[2]};
        double up[3] = {k.up[0], k.up[1], k.up[2]};
        double R[3], U[3];
        if (!normalize(F)) return fail(PT_E_INVALID, "camera %d: look_at == pos", c);
        cross(F, up, R);
        if (!normalize(R)) return fail(PT_E_INVALID, "camera %d: up parallel to view", c);
        cross(R, F, U);
        DevCam& h = hc[c];
        memset(&h, 0, sizeof(h));
        for (int i = 0; i < 3; ++i) {
            h.C[i] = k.pos[i]; h.F[i] = (float)F[i]; h.R[i] = (float)R[i]; h.U[i] = (float)U[i];
        }
        const double ty = std::tan(0.5 * (double)k.fov_y);
        const double tx = ty * (double)k.width / (double)k.height;
        tans[2 * c] = tx; tans[2 * c + 1] = ty;
        h.inv_tx = (float)(1.0 / tx); h.inv_ty = (float)(1.0 / ty);
        h.half_w = 0.5f * (float)k.width; h.half_h = 0.5f * (float)k.height;
        h.W = k.width; h.H = k.height; h.off = (int)off;
        off += (int64_t)k.width * k.height;
    }
    if (off >= ((int64_t)1 << 31)) return fail(PT_E_INVALID, "too many pixels");
    S.n_pixels = off;
    S.cams = nullptr;
    S.omega = nullptr;
    S.err = nullptr;
    return PT_OK;
}

extern "C" {

int pt_scene_create(const pt_scene_desc* d, pt_scene** out) {
    if (!d || !out) return fail(PT_E_INVALID, "pt_scene_create: null argument");
    *out = nullptr;
    pt_scene* sc = new (std::nothrow) pt_scene();
    if (!sc) return fail(PT_E_OOM, "host allocation");
    DevScene& S = sc->ds;
    DevCam hc[PT_MAX_CAMS];
    double tans[2 * PT_MAX_CAMS];
    if (int rc = describe_scene(d, S, hc, tans)) {
        delete sc;
        return rc;
    }
    const int64_t off = S.n_pixels;
    sc->n_pixels = off;
    double* d_tans = nullptr;
    int rc = PT_OK;
    if ((rc = dev_alloc(&sc->d_cams, (uint64_t)d->n_cams, nullptr, "cameras")) ||
        (rc = dev_alloc(&sc->d_omega, (uint64_t)off, nullptr, "pixel solid angles")) ||
        (rc = dev_alloc(&sc->d_err, 1, nullptr, "error word")) ||
        (rc = dev_alloc(&d_tans, (uint64_t)(2 * d->n_cams), nullptr, "tans"))) {
        cudaFree(sc->d_cams); cudaFree(sc->d_omega); cudaFree(sc->d_err); cudaFree(d_tans);
        delete sc;
        return rc;
    }
    cudaError_t e = cudaMemcpy(sc->d_cams, hc, sizeof(DevCam) * d->n_cams, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_tans, tans, sizeof(double) * 2 * d->n_cams, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(sc->d_err, 0, sizeof(int));
    if (e == cudaSuccess) {
        k_pixel_omega<<<(unsigned)((off + 255) / 256), 256>>>(sc->d_cams, d->n_cams, d_tans, sc->d_omega, off);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(d_tans);
    if (e != cudaSuccess) {
        cudaFree(sc->d_cams); cudaFree(sc->d_omega); cudaFree(sc->d_err);
        delete sc;
        return fail(PT_E_CUDA, "pt_scene_create: %s", cudaGetErrorString(e));
    }
    S.cams = sc->d_cams;
    S.omega = sc->d_omega;
    S.err = sc->d_err;
    *out = sc;
    return PT_OK;
}

int pt_scene_free(pt_scene* sc) {
    if (!sc) return PT_OK;
    cudaFree(sc->d_cams);
    cudaFree(sc->d_omega);
    cudaFree(sc->d_err);
    delete sc;
    return PT_OK;
}

int64_t pt_scene_pixels(const pt_scene* sc) { return sc ? sc->n_pixels : -1; }

int render_forward(const pt_scene* sc, const float* beta, uint64_t first, uint64_t n, double n_norm, uint64_t seed,
                   uint32_t epoch, double* images, uint32_t flags, double* tallies, uint64_t* fps, void* stream) {
    NvtxRange nvtx_range("render_forward");
    if (!sc || !beta || !images) return fail(PT_E_INVALID, "render_forward: null scene, grid or images");
    if (!(n_norm > 0.0)) return fail(PT_E_INVALID, "render_forward: n_norm must be > 0");
    if (n >= ((uint64_t)1 << 40)) return fail(PT_E_INVALID, "render_forward: n_paths too large");
    cudaStream_t st = S_(stream);
    if (!(flags & PT_ACCUMULATE)) PT_CUDA(cudaMemsetAsync(images, 0, sizeof(double) * sc->n_pixels, st));
    if (n == 0) return PT_OK;
    launch_sample(sc->ds, beta, first, n, (float)(1.0 / n_norm), seed, epoch, images, tallies, fps, nullptr, st);
    return launch_status("render_forward");
}

int paths_store(const pt_scene* sc, const float* beta, uint64_t first, uint64_t n, double n_norm, uint64_t seed,
                uint32_t epoch, pt_paths** pp, double* images_ref, uint32_t flags, double* tallies, uint64_t* fps,
                void* stream) {
    NvtxRange nvtx_range("paths_store");
    if (!sc || !beta || !pp) return fail(PT_E_INVALID, "paths_store: null scene, grid or handle slot");
    if (!(n_norm > 0.0)) return fail(PT_E_INVALID, "paths_store: n_norm must be > 0");
    if (n == 0 || n >= ((uint64_t)1 << 32)) return fail(PT_E_INVALID, "paths_store: n_paths must be in 1..2^32-1");
    cudaStream_t st = S_(stream);
    pt_paths* p = *pp;
    bool created = false;
    if (!p) {
        p = new (std::nothrow) pt_paths();
        if (!p) return fail(PT_E_OOM, "host allocation");
        created = true;
    } else if (p->scene != sc) {
        return fail(PT_E_INVALID, "paths_store: handle belongs to another scene");
    }
    p->scene = sc;
    const int slots = sc->ds.max_orders + 1;
    int rc;
    if (!p->beta_ref || p->V != sc->ds.V || p->slots != slots) {
        // buffers of fixed size: grids, bucket table, event bins
        if (!created) PT_CUDA(cudaStreamSynchronize(st));
        free_paths_buffers(p);
        uint64_t by = 0;
        p->V = sc->ds.V;
        Events& E = p->ev;
        E.bin_bits = event_bin_bits(sc->ds);
        E.bin_shift = 0;
        while (E.bin_bits > 8) {   // keep the two-level bin scan within 2^24 bins
            --E.bin_bits;
            ++E.bin_shift;
        }
        // spare bin bits order the events inside their voxel (up to 2 per axis):
        // lanes of a warp then hold nearby events, whose shadow rays keep together
        E.bin_sub = std::min(2, 8 - E.bin_bits);
        E.bin_bits += E.bin_sub;
        E.n_bins = 1u << (3 * E.bin_bits);
        if ((rc = dev_alloc(&p->beta_ref, (uint64_t)p->V, &by, "beta_ref")) ||
            (rc = dev_alloc(&p->dbeta, (uint64_t)p->V, &by, "dbeta")) ||
            (rc = dev_alloc(&p->bk, 1, &by, "buckets")) ||
            (rc = dev_alloc(&p->bad, 1, &by, "extinction check")) ||
            (rc = dev_alloc(&p->abort_flag, 1, &by, "store fit flag")) ||
            (rc = dev_alloc(&E.hist, E.n_bins, &by, "event bins")) ||
            (rc = dev_alloc(&E.cursor, E.n_bins, &by, "event bin cursors")) ||
            (rc = dev_alloc(&E.partial, 3 * 4096, &by, "scan partials"))) {
            free_paths_buffers(p);
            if (created) delete p;
            return rc;
        }
        p->slots = slots;
        p->bytes = by;
    }
    p->n = n;
    p->inv_norm = (float)(1.0 / n_norm);
    set_cache(p, false, nullptr);
    *pp = p;
    // PT_ASYNC on a sized handle: the checks run on the device (see the header)
    const bool async = (flags & PT_ASYNC) && p->sa && p->ev.a && p->rec_cap > 0 && p->ev.cap > 0;

    // no path kernel runs on an extinction grid with NaN, infinite or negative
    // voxels: count them first (one synchronisation; the store has another)
    if (async) {
        PT_CUDA(cudaMemsetAsync(p->bad, 0, sizeof(uint32_t), st));
        k_check_beta<<<grid_for(p->V, 256), 256, 0, st>>>(beta, p->V, p->bad);
        if ((rc = launch_status("paths_store check"))) return rc;
    } else {
        uint32_t bad = 0;
        PT_CUDA(cudaMemsetAsync(p->bad, 0, sizeof(uint32_t), st));
        k_check_beta<<<grid_for(p->V, 256), 256, 0, st>>>(beta, p->V, p->bad);
        if ((rc = launch_status("paths_store check"))) return rc;
        PT_CUDA(cudaMemcpyAsync(&bad, p->bad, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        PT_CUDA(cudaStreamSynchronize(st));
        if (bad) {
            p->n = 0;
            return fail(PT_E_INVALID, "paths_store: beta has %u voxels that are NaN, infinite or negative", bad);
        }
    }

    // The sampled records (slot-major, every path's maximum slots) live only
    // until the sort: stream-ordered allocations, returned to the pool after
    // the scatter.  The kept arrays are sized from the actual record and
    // event counts, read once the counting sort has run.
    StoreBuf sbuf{nullptr, nullptr, nullptr, n};
    uint32_t* sortw = nullptr;
    cudaMemPool_t pool = store_pool();
    auto tmp = [&](void** q, uint64_t bytes, const char* what) -> int {
        const cudaError_t e = pool ? cudaMallocFromPoolAsync(q, bytes ? bytes : 16, pool, st)
                                   : cudaMallocAsync(q, bytes ? bytes : 16, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(PT_E_OOM, "paths_store: no device memory for %s (%llu bytes)", what,
                        (unsigned long long)bytes);
        }
        return PT_OK;
    };
    auto release = [&]() {
        for (void* q : {(void*)sbuf.rec_a, (void*)sbuf.rec_b, (void*)sbuf.cnt, (void*)sortw})
            if (q) cudaFreeAsync(q, st);
    };
    if ((rc = tmp((void**)&sbuf.rec_a, sizeof(uint4) * n * slots, "sampled records A")) ||
        (rc = tmp((void**)&sbuf.rec_b, sizeof(float4) * n * slots, "sampled records B")) ||
        (rc = tmp((void**)&sbuf.cnt, sizeof(uint8_t) * n, "collision counts")) ||
        (rc = tmp((void**)&sortw, sizeof(uint32_t) * sort_scratch_words(n), "path sort keys and bins"))) {
        release();
        return rc;
    }
    PT_CUDA(cudaMemcpyAsync(p->beta_ref, beta, sizeof(float) * p->V, cudaMemcpyDeviceToDevice, st));
    if (images_ref && !(flags & PT_ACCUMULATE)) PT_CUDA(cudaMemsetAsync(images_ref, 0, sizeof(double) * sc->n_pixels, st));
    // without images_ref the kernel traces flights only (no shadow rays)
    launch_sample(sc->ds, beta, first, n, p->inv_norm, seed, epoch, images_ref, tallies, fps, &sbuf, st);
    if ((rc = launch_status("paths_store"))) { release(); return rc; }
    // Morton bins of the first collision: the grid's Morton code reduced to 12 bits
    const SortScratch sw = sort_scratch(sortw, n);
    const int key_shift = std::max(0, 3 * event_bin_bits(sc->ds) - 12);
    launch_sort_count(sbuf, n, slots, key_shift, sw, p->bk, st);
    if ((rc = launch_status("paths_store sort"))) { release(); return rc; }
    if (async) {
        launch_store_guard(p->bk, p->rec_cap, p->ev.cap, p->bad, p->abort_flag, sc->d_err, st);
        launch_sort_scatter(sbuf, n, sw, p->bk, p->sa, p->sb, st, p->abort_flag);
        release();
        if ((rc = launch_status("paths_store sort"))) return rc;
        launch_events(sc->ds, sorted_view(p), p->ev, st);
        return launch_status("paths_store events");
    }
    Buckets hb;
    if (cudaMemcpyAsync(&hb, p->bk, sizeof(Buckets), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        release();
        return launch_status("paths_store counts");
    }
    const uint64_t n_rec = hb.rec_off[kBuckets], n_ev = hb.n_events;
    // grow the kept arrays (1/8 headroom, so that later stores of a similar
    // path set reuse them); a grown handle must be bound again in a batch
    auto grow = [](uint64_t need) { return need + need / 8 + 1024; };
    if (p->rec_cap < n_rec || !p->sa) {
        cudaFree(p->sa); cudaFree(p->sb); cudaFree(p->ev.of_rec);
        p->sa = nullptr; p->sb = nullptr; p->ev.of_rec = nullptr;
        p->bytes -= p->rec_cap * (sizeof(uint4) + sizeof(float4) + sizeof(uint32_t));
        p->rec_cap = 0;
        const uint64_t c = grow(n_rec);
        if ((rc = dev_alloc(&p->sa, c, &p->bytes, "sorted records A")) ||
            (rc = dev_alloc(&p->sb, c, &p->bytes, "sorted records B")) ||
            (rc = dev_alloc(&p->ev.of_rec, c, &p->bytes, "record-to-event map"))) {
            release();
            return rc;
        }
        p->rec_cap = c;
    }
    if (p->ev.cap < n_ev || !p->ev.a) {
        Events& E = p->ev;
        cudaFree(E.a); cudaFree(E.b); cudaFree(E.val);
        E.a = nullptr; E.b = nullptr; E.val = nullptr;
        p->bytes -= E.cap * (sizeof(uint4) + sizeof(float4) + sizeof(float));
        E.cap = 0;
        const uint64_t c = grow(n_ev);
        if ((rc = dev_alloc(&E.a, c, &p->bytes, "events A")) || (rc = dev_alloc(&E.b, c, &p->bytes, "events B")) ||
            (rc = dev_alloc(&E.val, c, &p->bytes, "event values"))) {
            release();
            return rc;
        }
        E.cap = c;
    }
    launch_sort_scatter(sbuf, n, sw, p->bk, p->sa, p->sb, st);
    release();
    if ((rc = launch_status("paths_store sort"))) return rc;
    launch_events(sc->ds, sorted_view(p), p->ev, st);
    return launch_status("paths_store events");
}

int paths_reweight(pt_paths* p, const float* beta_t, double* images, uint32_t flags, void* stream) {
    NvtxRange nvtx_range("paths_reweight");
    if (!p || !p->scene || !beta_t || !images) return fail(PT_E_INVALID, "paths_reweight: null argument");
    if (p->n == 0) return fail(PT_E_INVALID, "paths_reweight: handle holds no paths");
    cudaStream_t st = S_(stream);
    const pt_scene* sc = p->scene;
    float* cache = nullptr;
    if (flags & PT_CACHE) {
        const uint64_t need = p->ev.cap * (uint64_t)sc->ds.n_cams;
        if (p->cache_cap < need) {
            PT_CUDA(cudaStreamSynchronize(st));
            cudaFree(p->cache);
            p->cache = nullptr;
            p->bytes -= p->cache_cap * sizeof(float);
            p->cache_cap = 0;
            if (int rc = dev_alloc(&p->cache, need, &p->bytes, "contribution cache")) return rc;
            p->cache_cap = need;
        }
        cache = p->cache;
    }
    if (!(flags & PT_ACCUMULATE)) PT_CUDA(cudaMemsetAsync(images, 0, sizeof(double) * sc->n_pixels, st));
    launch_delta(beta_t, p->beta_ref, p->dbeta, p->V, st);
    launch_reweight(sc->ds, sorted_view(p), p->ev, beta_t, p->beta_ref, p->dbeta, images, cache, st);
    set_cache(p, (flags & PT_CACHE) != 0, beta_t);
    return launch_status("paths_reweight");
}

int render_grad(pt_paths* p, const float* beta_t, const double* dldi, double* grad, uint32_t flags, void* stream) {
    NvtxRange nvtx_range("render_grad");
    if (!p || !p->scene || !beta_t || !dldi || !grad) return fail(PT_E_INVALID, "render_grad: null argument");
    if (p->n == 0) return fail(PT_E_INVALID, "render_grad: handle holds no paths");
    if ((flags & PT_CACHE) && !p->cache_valid)
        return fail(PT_E_INVALID, "render_grad: PT_CACHE without a preceding paths_reweight(PT_CACHE)");
    if ((flags & PT_CACHE) && p->cache_beta != beta_t)
        return fail(PT_E_INVALID, "render_grad: PT_CACHE with another extinction grid than the cached reweight's");
    cudaStream_t st = S_(stream);
    const pt_scene* sc = p->scene;
    if (!(flags & PT_ACCUMULATE)) PT_CUDA(cudaMemsetAsync(grad, 0, sizeof(double) * p->V, st));
    if (!(flags & PT_CACHE)) launch_delta(beta_t, p->beta_ref, p->dbeta, p->V, st);
    launch_grad(sc->ds, sorted_view(p), p->ev, beta_t, p->beta_ref, p->dbeta, dldi, grad,
                (flags & PT_CACHE) ? p->cache : nullptr, st);
    return launch_status("render_grad");
}

uint64_t paths_cache_token(const pt_paths* p) { return p && p->cache_valid ? p->cache_token : 0; }

int paths_drop_cache(pt_paths* p) {
    if (!p) return PT_OK;
    if (p->cache) {
        const cudaError_t e = cudaFree(p->cache);
        if (e != cudaSuccess) return fail(PT_E_CUDA, "paths_drop_cache: %s", cudaGetErrorString(e));
    }
    p->cache = nullptr;
    p->bytes -= p->cache_cap * sizeof(float);
    p->cache_cap = 0;
    set_cache(p, false, nullptr);
    return PT_OK;
}

int paths_free(pt_paths* p) {
    if (!p) return PT_OK;
    cudaDeviceSynchronize();
    free_paths_buffers(p);
    delete p;
    return PT_OK;
}

int paths_info(const pt_paths* p, pt_paths_info* out, void* stream) {
    if (!p || !out) return fail(PT_E_INVALID, "paths_info: null argument");
    memset(out, 0, sizeof(*out));
    out->n_paths = p->n;
    out->bytes_device = p->bytes;
    if (!p->bk || p->n == 0) return PT_OK;
    Buckets h;
    PT_CUDA(cudaMemcpyAsync(&h, p->bk, sizeof(h), cudaMemcpyDeviceToHost, S_(stream)));
    PT_CUDA(cudaStreamSynchronize(S_(stream)));
    for (int b = 0; b < kBuckets; ++b) out->bucket[b] = h.count[b];
    out->n_stored = h.path_off[kBuckets];
    out->n_records = h.rec_off[kBuckets];
    return PT_OK;
}

int adam_step(float* beta, float* m, float* v, const double* grad, const uint8_t* mask, int64_t n, int32_t t,
              float lr, float b1, float b2, float eps, void* stream) {
    if (!beta || !m || !v || !grad || n < 0 || t < 1) return fail(PT_E_INVALID, "adam_step: bad argument");
    if (n == 0) return PT_OK;
    const double bc1 = 1.0 - std::pow((double)b1, (double)t);
    const double bc2 = 1.0 - std::pow((double)b2, (double)t);
    k_adam<<<grid_for(n, 256), 256, 0, S_(stream)>>>(beta, m, v, grad, mask, n, lr, b1, b2, eps,
                                                      (float)(1.0 / bc1), (float)(1.0 / bc2));
    return launch_status("adam_step");
}

int adam_step_counted(float* beta, float* m, float* v, const double* grad, const uint8_t* mask, int64_t n,
                      int32_t* step, float* scratch, float lr, float b1, float b2, float eps, void* stream) {
    if (!beta || !m || !v || !grad || !step || !scratch || n < 0)
        return fail(PT_E_INVALID, "adam_step_counted: bad argument");
    cudaStream_t st = S_(stream);
    k_adam_count<<<1, 32, 0, st>>>(step, b1, b2, scratch);
    if (n > 0) k_adam_dev<<<grid_for(n, 256), 256, 0, st>>>(beta, m, v, grad, mask, n, lr, b1, b2, eps, scratch);
    return launch_status("adam_step_counted");
}

int loss_residual(const double* images, const double* gt, int64_t n, double* dldi, double* loss, void* stream) {
    if (!images || !gt || !dldi || n < 0) return fail(PT_E_INVALID, "loss_residual: bad argument");
    cudaStream_t st = S_(stream);
    if (loss) PT_CUDA(cudaMemsetAsync(loss, 0, sizeof(double), st));
    if (n == 0) return PT_OK;
    k_resid<<<grid_for(n, 256, 4), 256, 0, st>>>(images, gt, n, dldi, loss);
    return launch_status("loss_residual");
}

int space_carve(const pt_scene* sc, const double* images, double threshold, uint8_t* mask, void* stream) {
    NvtxRange nvtx_range("space_carve");
    if (!sc || !images || !mask) return fail(PT_E_INVALID, "space_carve: null argument");
    cudaStream_t st = S_(stream);
    k_space_carve<<<grid_for(sc->ds.V, 256), 256, 0, st>>>(sc->ds, images, threshold, mask);
    return launch_status("space_carve");
}

// ------------------------------------------------------------ batches --
}  // extern "C"

struct pt_batch {
    std::vector<pt_paths*> paths;
    std::vector<BatchScene> host;
    BatchScene* dev = nullptr;
    BatchQueue q{};
    int blocks = 0;    // resident blocks in all (persistent schedule)
    int reg_cap = 0;
    bool grouped = false;            // one block per tile, hardware-scheduled
    bool sequence = false;           // the single-scene launches, scene by scene
    std::vector<GroupTable> groups;  // grouped schedule: kGroupMax scenes per launch
    bool bound = false;
};

namespace {
int sm_count() { return device_sms(); }

int ensure_cache(pt_paths* p, cudaStream_t st) {
    const uint64_t need = p->ev.cap * (uint64_t)p->scene->ds.n_cams;
    if (p->cache_cap >= need) return PT_OK;
    PT_CUDA(cudaStreamSynchronize(st));
    cudaFree(p->cache);
    p->cache = nullptr;
    p->bytes -= p->cache_cap * sizeof(float);
    p->cache_cap = 0;
    if (int rc = dev_alloc(&p->cache, need, &p->bytes, "contribution cache")) return rc;
    p->cache_cap = need;
    return PT_OK;
}
}  // namespace

extern "C" {

int batch_create(pt_paths* const* paths, int n, pt_batch** out) {
    if (!paths || !out || n < 1) return fail(PT_E_INVALID, "batch_create: need 1 or more stored-path handles");
    *out = nullptr;
    for (int s = 0; s < n; ++s)
        if (!paths[s] || !paths[s]->scene || paths[s]->n == 0)
            return fail(PT_E_INVALID, "batch_create: handle %d holds no stored paths", s);
    pt_batch* b = new (std::nothrow) pt_batch();
    if (!b) return fail(PT_E_OOM, "host allocation");
    b->paths.assign(paths, paths + n);
    b->host.resize(n);
    int rc;
    if ((rc = dev_alloc(&b->dev, (uint64_t)n, nullptr, "batch table")) ||
        (rc = dev_alloc(&b->q.off, (uint64_t)kBatchPasses * (n + 1), nullptr, "batch tiles")) ||
        (rc = dev_alloc(&b->q.counter, (uint64_t)kBatchPasses, nullptr, "batch counters"))) {
        cudaFree(b->dev); cudaFree(b->q.off); cudaFree(b->q.counter);
        delete b;
        return rc;
    }
    b->blocks = sm_count() * batch_blocks_per_sm(0);
    *out = b;
    return PT_OK;
}

int batch_launch_limits(pt_batch* b, int reg_cap, int* max_blocks_per_sm) {
    if (!b || !max_blocks_per_sm || (reg_cap != 0 && reg_cap != 1))
        return fail(PT_E_INVALID, "batch_launch_limits: bad argument");
    *max_blocks_per_sm = batch_blocks_per_sm(reg_cap);
    return PT_OK;
}

int batch_set_launch(pt_batch* b, int reg_cap, int blocks_per_sm) {
    if (!b || blocks_per_sm < -1 || (reg_cap != 0 && reg_cap != 1))
        return fail(PT_E_INVALID, "batch_set_launch: bad argument");
    b->reg_cap = reg_cap;
    b->grouped = blocks_per_sm == 0;
    b->sequence = blocks_per_sm == -1;
    if (blocks_per_sm > 0) b->blocks = sm_count() * std::min(blocks_per_sm, batch_blocks_per_sm(reg_cap));
    return PT_OK;
}

int batch_bind(pt_batch* b, const float* const* beta_t, double* const* images, const double* const* dldi,
               double* const* grad, void* stream) {
    if (!b || !beta_t || !images || !dldi || !grad) return fail(PT_E_INVALID, "batch_bind: null argument");
    cudaStream_t st = S_(stream);
    const int n = (int)b->paths.size();
    for (int s = 0; s < n; ++s) {
        pt_paths* p = b->paths[s];
        if (!beta_t[s] || !images[s] || !dldi[s] || !grad[s])
            return fail(PT_E_INVALID, "batch_bind: null buffer for scene %d", s);
        if (int rc = ensure_cache(p, st)) return rc;
        BatchScene& B = b->host[s];
        B.S = p->scene->ds;
        B.P = sorted_view(p);
        B.E = p->ev;
        B.beta_t = beta_t[s];
        B.beta_ref = p->beta_ref;
        B.dbeta = p->dbeta;
        B.images = images[s];
        B.dldi = dldi[s];
        B.grad = grad[s];
        B.cache = p->cache;
        B.V = p->V;
    }
    // grouped schedule: kernel-parameter tables of up to kGroupMax scenes,
    // blocks laid out from the scenes' upper bounds
    b->groups.assign((size_t)((n + kGroupMax - 1) / kGroupMax), GroupTable{});
    for (int s = 0; s < n; ++s) {
        GroupTable& t = b->groups[(size_t)(s / kGroupMax)];
        const int k = t.n++;
        t.sc[k] = b->host[s];
        uint32_t tiles[kGroupPasses];
        group_tiles(b->host[s], tiles);
        for (int p = 0; p < kGroupPasses; ++p) {
            const uint64_t end = (uint64_t)t.off[p][k] + tiles[p];
            if (end > 0x7fffffffull) return fail(PT_E_INVALID, "batch_bind: too many tiles in one group");
            t.off[p][k + 1] = (uint32_t)end;
        }
    }
    PT_CUDA(cudaMemcpyAsync(b->dev, b->host.data(), sizeof(BatchScene) * n, cudaMemcpyHostToDevice, st));
    PT_CUDA(cudaStreamSynchronize(st));
    b->bound = true;
    return PT_OK;
}

int batch_reweight(pt_batch* b, uint32_t flags, void* stream) {
    NvtxRange nvtx_range("batch_reweight");
    if (!b || !b->bound) return fail(PT_E_INVALID, "batch_reweight: batch not bound");
    cudaStream_t st = S_(stream);
    const int n = (int)b->paths.size();
    if (!(flags & PT_ACCUMULATE))
        for (int s = 0; s < n; ++s)
            PT_CUDA(cudaMemsetAsync(b->host[s].images, 0, sizeof(double) * b->paths[s]->scene->n_pixels, st));
    if (b->sequence) {
        for (int s = 0; s < n; ++s) {
            const BatchScene& B = b->host[s];
            launch_delta(B.beta_t, B.beta_ref, B.dbeta, B.V, st);
            launch_reweight(B.S, B.P, B.E, B.beta_t, B.beta_ref, B.dbeta, B.images,
                            (flags & PT_CACHE) ? B.cache : nullptr, st);
        }
    } else if (b->grouped)
        for (const GroupTable& t : b->groups) launch_group_reweight(t, (flags & PT_CACHE) != 0, b->reg_cap, st);
    else
        launch_batch_reweight(b->dev, n, b->q, (flags & PT_CACHE) != 0, b->reg_cap, b->blocks, st);
    for (int s = 0; s < n; ++s) set_cache(b->paths[s], (flags & PT_CACHE) != 0, b->host[s].beta_t);
    return launch_status("batch_reweight");
}

int batch_grad(pt_batch* b, uint32_t flags, void* stream) {
    NvtxRange nvtx_range("batch_grad");
    if (!b || !b->bound) return fail(PT_E_INVALID, "batch_grad: batch not bound");
    if (!(flags & PT_CACHE)) return fail(PT_E_INVALID, "batch_grad: the batched gradient reads the cache (PT_CACHE)");
    const int n = (int)b->paths.size();
    for (int s = 0; s < n; ++s)
        if (!b->paths[s]->cache_valid)
            return fail(PT_E_INVALID, "batch_grad: scene %d has no cache from batch_reweight(PT_CACHE)", s);
    cudaStream_t st = S_(stream);
    if (!(flags & PT_ACCUMULATE))
        for (int s = 0; s < n; ++s)
            PT_CUDA(cudaMemsetAsync(b->host[s].grad, 0, sizeof(double) * b->paths[s]->V, st));
    if (b->sequence) {
        for (int s = 0; s < n; ++s) {
            const BatchScene& B = b->host[s];
            launch_grad(B.S, B.P, B.E, B.beta_t, B.beta_ref, B.dbeta, B.dldi, B.grad, B.cache, st);
        }
    } else if (b->grouped)
        for (const GroupTable& t : b->groups) launch_group_grad(t, b->reg_cap, st);
    else
        launch_batch_grad(b->dev, n, b->q, b->reg_cap, b->blocks, st);
    return launch_status("batch_grad");
}

int batch_free(pt_batch* b) {
    if (!b) return PT_OK;
    cudaDeviceSynchronize();
    cudaFree(b->dev);
    cudaFree(b->q.off);
    cudaFree(b->q.counter);
    delete b;
    return PT_OK;
}

int pt_check(const pt_scene* sc, void* stream) {
    if (!sc) return fail(PT_E_INVALID, "pt_check: null scene");
    int h = 0;
    PT_CUDA(cudaMemcpyAsync(&h, sc->d_err, sizeof(int), cudaMemcpyDeviceToHost, S_(stream)));
    PT_CUDA(cudaStreamSynchronize(S_(stream)));
    if (h) {
        PT_CUDA(cudaMemsetAsync(sc->d_err, 0, sizeof(int), S_(stream)));
        PT_CUDA(cudaStreamSynchronize(S_(stream)));
        return fail(PT_E_DEVICE_ASSERT,
                    "kernel invariant violated (bits 0x%x: 1 index, 2 traversal length, 4 record, 8 a PT_ASYNC store "
                    "did not fit its buffers or had an invalid extinction grid)",
                    h);
    }
    return PT_OK;
}

int pt_inject_error(pt_scene* sc, int bits, void* stream) {
    if (!sc) return fail(PT_E_INVALID, "pt_inject_error: null scene");
    if (bits <= 0 || bits > 15) return fail(PT_E_INVALID, "pt_inject_error: bits must be in 1..15");
    int h = 0;
    PT_CUDA(cudaMemcpyAsync(&h, sc->d_err, sizeof(int), cudaMemcpyDeviceToHost, S_(stream)));
    PT_CUDA(cudaStreamSynchronize(S_(stream)));
    h |= bits;
    PT_CUDA(cudaMemcpyAsync(sc->d_err, &h, sizeof(int), cudaMemcpyHostToDevice, S_(stream)));
    PT_CUDA(cudaStreamSynchronize(S_(stream)));
    return PT_OK;
}

}  // extern "C"
