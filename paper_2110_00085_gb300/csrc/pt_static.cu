// pt_static.cu -- render_forward_static: forward path tracing for callers
// that cannot allocate device memory.
//
// render_forward needs a pt_scene, whose creation allocates the camera
// table, the per-pixel solid angles and an error word on the device.  Some
// callers cannot do that: a host application whose allocator owns all device
// memory, or code that runs where allocation is forbidden after start-up.
// This entry point derives the same tables on every call into one
// file-scope device array and then runs the unchanged sampling kernel.  It
// calls no cudaMalloc, cudaFree or allocating library routine.
//
//   - limits: at most kStaticCams cameras and kStaticPixels pixels in total
//     (about 1 MiB of device memory, held by every GPU that loads the
//     library until the process exits);
//   - the first call on a device looks up the array's device address with
//     cudaGetSymbolAddress (once per device, with that device current); make
//     that first call before any stream capture;
//   - every call rewrites the tables and clears the error word; calls that
//     overlap on the GPU share the array and race;
//   - kernel-side invariant checks are recorded in the array and are not
//     reported by this entry point.
#include <algorithm>
#include <mutex>

#include "pt_kernels.cuh"

namespace pt {
namespace {

constexpr int kStaticCams = 16;
constexpr int64_t kStaticPixels = (int64_t)1 << 18;
constexpr size_t kOffErr = 2048;
constexpr size_t kOffOmega = 4096;
constexpr size_t kStaticBytes = kOffOmega + sizeof(float) * (size_t)kStaticPixels;
static_assert(sizeof(DevCam) * kStaticCams <= kOffErr, "camera table overflows its slot");

// scratch: [cameras | error word | pixel solid angles]
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

struct CamPack {
    DevCam cam[kStaticCams];
    double tans[2 * kStaticCams];
    int n_cams;
};

// camera table, cleared error word and the pixel solid angles (float64
// corner sums of atan(x y / sqrt(1 + x^2 + y^2)) on the unit image plane)
__global__ void k_static_setup(CamPack pack, unsigned char* scratch, int64_t npix) {
    DevCam* cams = reinterpret_cast<DevCam*>(scratch);
    int* err = reinterpret_cast<int*>(scratch + kOffErr);
    float* omega = reinterpret_cast<float*>(scratch + kOffOmega);
    const int64_t g0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g0 < pack.n_cams) cams[g0] = pack.cam[g0];
    if (g0 == 0) *err = 0;
    for (int64_t g = g0; g < npix; g += (int64_t)gridDim.x * blockDim.x) {
        int c = 0;
        while (c + 1 < pack.n_cams && g >= pack.cam[c + 1].off) ++c;
        const DevCam& k = pack.cam[c];
        const int64_t p = g - k.off;
        const int col = (int)(p % k.W), row = (int)(p / k.W);
        const double tx = pack.tans[2 * c], ty = pack.tans[2 * c + 1];
        const double xa = tx * (-1.0 + 2.0 * col / (double)k.W), xb = tx * (-1.0 + 2.0 * (col + 1) / (double)k.W);
        const double ya = ty * (1.0 - 2.0 * (row + 1) / (double)k.H), yb = ty * (1.0 - 2.0 * row / (double)k.H);
        auto F = [](double x, double y) { return atan(x * y / sqrt(1.0 + x * x + y * y)); };
        omega[g] = (float)(F(xb, yb) - F(xa, yb) - F(xb, ya) + F(xa, ya));
    }
}

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};

// device address of the scratch array on the current device (looked up once)
int scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(PT_E_CUDA, "render_forward_static: cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(PT_E_INVALID, "render_forward_static: device %d unsupported", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            return fail(PT_E_CUDA, "render_forward_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_addr[dev];
    return PT_OK;
}

}  // namespace
}  // namespace pt

using namespace pt;

extern "C" int render_forward_static(const pt_scene_desc* desc, const float* beta, uint64_t first, uint64_t n,
                                     double n_norm, uint64_t seed, uint32_t epoch, double* images, uint32_t flags,
                                     void* stream) {
    if (!desc || !beta || !images) return fail(PT_E_INVALID, "render_forward_static: null description, grid or images");
    if (!(n_norm > 0.0)) return fail(PT_E_INVALID, "render_forward_static: n_norm must be > 0");
    if (n >= ((uint64_t)1 << 40)) return fail(PT_E_INVALID, "render_forward_static: n_paths too large");
    if (desc->n_cams > kStaticCams)
        return fail(PT_E_INVALID, "render_forward_static: %d cameras; this entry point holds at most %d",
                    desc->n_cams, kStaticCams);
    DevScene S;
    DevCam hc[PT_MAX_CAMS];
    double tans[2 * PT_MAX_CAMS];
    if (int rc = describe_scene(desc, S, hc, tans)) return rc;
    if (S.n_pixels > kStaticPixels)
        return fail(PT_E_INVALID, "render_forward_static: %lld pixels; this entry point holds at most %lld",
                    (long long)S.n_pixels, (long long)kStaticPixels);
    unsigned char* scr = nullptr;
    if (int rc = scratch_address(&scr)) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    CamPack pack;
    for (int c = 0; c < desc->n_cams; ++c) {
        pack.cam[c] = hc[c];
        pack.tans[2 * c] = tans[2 * c];
        pack.tans[2 * c + 1] = tans[2 * c + 1];
    }
    pack.n_cams = desc->n_cams;
    if (!(flags & PT_ACCUMULATE)) {
        cudaError_t e = cudaMemsetAsync(images, 0, sizeof(double) * (size_t)S.n_pixels, st);
        if (e != cudaSuccess) return fail(PT_E_CUDA, "render_forward_static: memset: %s", cudaGetErrorString(e));
    }
    const unsigned blocks = (unsigned)std::min<int64_t>((S.n_pixels + 255) / 256, (int64_t)device_sms() * 8);
    k_static_setup<<<blocks, 256, 0, st>>>(pack, scr, S.n_pixels);
    S.cams = reinterpret_cast<const DevCam*>(scr);
    S.err = reinterpret_cast<int*>(scr + kOffErr);
    S.omega = reinterpret_cast<const float*>(scr + kOffOmega);
    if (n > 0) launch_sample(S, beta, first, n, (float)(1.0 / n_norm), seed, epoch, images, nullptr, nullptr, nullptr, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(PT_E_CUDA, "render_forward_static launch: %s", cudaGetErrorString(e));
    return PT_OK;
}
