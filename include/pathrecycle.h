/*
 * pathrecycle.h -- C ABI of libpathrecycle.so: Monte-Carlo scattering
 * tomography with path recycling on one GB300 (sm_103a).
 *
 * Method: Czerninski & Schechner, "Accelerating Inverse Rendering By Using
 * a GPU and Reuse of Light Paths" (arXiv 2110.00085).
 *   - forward model: path tracing through a voxel grid of extinction with a
 *     directional sun, free-path (distance) sampling, particle-type and
 *     direction sampling, and local estimation toward every camera pixel
 *     (Sec. 3.4, Eq. Qd; scene of Sec. 6.1);
 *   - loss and gradient: L = 1/2 ||F - I_gt||^2 (Eq. appearance_loss), its
 *     gradient through the path score function (Eqs. loss_gradient,
 *     gradient_simualtion; PSF of scattering tomography, Sec. 4.4);
 *   - path recycling: stored paths reweighted by f(x|M_t)/mu(x|M_ref)
 *     (Sec. 5.2, Eqs. forward_simualtion_recycling, correction factor,
 *     gradient_simualtion_recycling) and sorted by path size (Sec. 5.3).
 *
 * Conventions shared by every call
 *   - Units: km and 1/km.  Grids are float32, x fastest (index
 *     x + nx*(y + ny*z)), at most 512 voxels per axis.
 *   - Images are float64, camera after camera, each row-major W x H with
 *     row 0 at the top; pixel values are radiance averaged over the pixel's
 *     solid angle, for unit sun irradiance times sun_irradiance.
 *   - All device pointers are CUDA device memory of the current device and
 *     are owned by the caller unless stated otherwise; `stream` is a
 *     cudaStream_t (NULL = legacy default stream).  Every call is
 *     asynchronous on `stream` except where stated.
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11) with key = seed
 *     and counter (path id lo, path id hi, event | tag << 8 | epoch << 16,
 *     scene id); uniforms u = ((w >> 8) + 1) * 2^-24 in (0, 1].
 *   - Return value: PT_OK or a PT_E_* code; the message of the latest
 *     failure on the calling thread is pt_last_error().  No call aborts the
 *     process.  Kernel-side invariant violations are recorded in the handle
 *     and reported by pt_check().
 */
#ifndef PATHRECYCLE_H
#define PATHRECYCLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PT_OK 0
#define PT_E_INVALID 1        /* bad argument or handle                     */
#define PT_E_OOM 2            /* device allocation failed                   */
#define PT_E_CUDA 3           /* a CUDA runtime call failed                 */
#define PT_E_TIMEOUT 4        /* a bounded device-side wait gave up         */
#define PT_E_DEVICE_ASSERT 5  /* a kernel detected a violated invariant     */

#define PT_MAX_CAMS 64
#define PT_MAX_ORDERS 15

/* flags */
#define PT_ACCUMULATE 1u      /* add into the outputs instead of zeroing them */
#define PT_CACHE 2u           /* paths_reweight: keep per-(event, camera)
                                 contributions in the handle; render_grad: use
                                 them instead of re-tracing shadow rays (the
                                 caller guarantees beta_t is unchanged)        */
#define PT_SORT 4u            /* surf_store: counting-sort the events by pixel,
                                 so that each re-evaluation merges same-pixel
                                 terms before its FP64 adds (pays off when the
                                 paths are re-evaluated more than once)       */
#define PT_ASYNC 8u           /* paths_store: do not synchronise the stream;
                                 see paths_store                             */

/* tallies: float64[PT_TALLY_COUNT], same meaning as the CPU oracle's */
enum {
    PT_T_INJECTED = 0, PT_T_MISSED, PT_T_ESCAPED, PT_T_ABSORBED, PT_T_TRUNCATED,
    PT_T_RR_KILLED, PT_T_RR_GAIN, PT_T_COLLISIONS, PT_T_ENTERED, PT_T_SEG_CROSS,
    PT_T_SHADOW_CROSS, PT_T_IN_VIEW, PT_TALLY_COUNT
};

/* Perspective pinhole camera.  The image plane sits at unit distance along
 * normalize(look_at - pos); right = normalize(forward x up), image-up =
 * right x forward; fov_y is the full vertical field of view (radians);
 * pixels are square.  Pixel response (a reading of the pixel response W_d of
 * Sec. 3.3 for a perspective pixel): 1 / (exact solid angle of the pixel). */
typedef struct {
    float pos[3];
    float look_at[3];
    float up[3];
    float fov_y;
    int32_t width, height;
} pt_camera;

/* Scene of scattering tomography (Sec. 4.4, Sec. 6.1): cloud droplets with
 * unknown extinction (passed per call), albedo_cloud and a Henyey-Greenstein
 * phase function of asymmetry hg_g; air with known uniform extinction
 * beta_air, albedo_air and a Rayleigh phase function; a sun with parallel
 * rays travelling along the unit vector sun_dir with irradiance
 * sun_irradiance.  Paths stop after max_orders collisions (<= PT_MAX_ORDERS)
 * and after collision k >= rr_start survive Russian roulette with
 * probability rr_q (weight / rr_q). */
typedef struct {
    int32_t nx, ny, nz;
    float voxel;                 /* km, cubic voxels                  */
    float origin[3];             /* km, corner of voxel (0,0,0)       */
    float beta_air, albedo_cloud, albedo_air, hg_g;
    float sun_dir[3];
    float sun_irradiance;
    int32_t n_cams;              /* 1 .. PT_MAX_CAMS                  */
    const pt_camera* cams;       /* host array, copied by pt_scene_create */
    int32_t max_orders, rr_start;
    float rr_q;                  /* (0, 1]                            */
    uint32_t scene_id;           /* Philox counter word 3             */
} pt_scene_desc;

typedef struct pt_scene pt_scene;   /* device-resident scene constants      */
typedef struct pt_paths pt_paths;   /* stored, size-sorted light paths      */

typedef struct {
    uint64_t n_paths;        /* paths sampled by the latest paths_store      */
    uint64_t n_stored;       /* of which stored (at least one collision)     */
    uint64_t n_records;      /* stored vertices (sum of B+1)                 */
    uint64_t bucket[PT_MAX_ORDERS + 1];   /* paths per path size B           */
    uint64_t bytes_device;   /* device memory held by the handle            */
} pt_paths_info;

/* Create a scene on the current device: copies the cameras, computes every
 * pixel's solid angle (float64 arithmetic, stored float32) and the sun's
 * sampling rectangle.  Synchronous.  Owner: the caller frees it with
 * pt_scene_free after every handle that uses it. */
int pt_scene_create(const pt_scene_desc* desc, pt_scene** out);
int pt_scene_free(pt_scene* scene);
int64_t pt_scene_pixels(const pt_scene* scene);

/*
 * render_forward -- plain path tracing (Alg. 1 forward step; estimator of
 * Eq. forward_simualtion with local estimation, Eq. Qd).
 * Traces paths first_path .. first_path+n_paths-1 under beta_cloud (device,
 * nx*ny*nz) and adds sum(contributions) / n_norm into images (device,
 * pt_scene_pixels doubles; zeroed first unless PT_ACCUMULATE).
 * tallies (device, PT_TALLY_COUNT doubles, accumulated) and fingerprints
 * (device, n_paths uint64: FNV-1a of each path's discrete decisions) may be
 * NULL.
 */
int render_forward(const pt_scene* scene, const float* beta_cloud,
                   uint64_t first_path, uint64_t n_paths, double n_norm,
                   uint64_t seed, uint32_t epoch, double* images, uint32_t flags,
                   double* tallies, uint64_t* fingerprints, void* stream);

/*
 * paths_store -- sample, sort and store light paths (Alg. 2, the resample
 * branch: sample under M_t, sort by path size, set M_ref <- M_t).
 * Traces the same paths as render_forward would and keeps every path with at
 * least one collision, counting-sorted by its number of collisions B and,
 * among paths of one size, by the Morton code of its first collision's voxel
 * (4096 bins; the order inside a bin is not fixed), as compact vertex
 * records.  The handle keeps a copy
 * of beta_cloud as M_ref.  *paths == NULL creates a handle (owned by the
 * caller, freed with paths_free); an existing handle of the same scene is
 * reused.  images_ref (nullable) receives the plain estimate under M_ref (as
 * render_forward).
 * Memory: the sampled records (every path's maximum number of slots) live
 * only until the sort, in a stream-ordered pool of this library that keeps
 * its memory for later stores; the kept records, events and the
 * contribution cache are sized from the actual record and event counts
 * (1/8 headroom), which paths_store reads after its counting sort: the call
 * synchronises the stream once, and growing a buffer synchronises again.
 * Before tracing, beta_cloud is checked (one more synchronisation): a grid
 * with NaN, infinite or negative voxels returns PT_E_INVALID, traces
 * nothing and leaves the handle without paths.
 * n_paths < 2^32 per handle; larger path sets are stored as several handles
 * over ranges of path ids (first_path) sharing n_norm.
 * PT_ASYNC (on a handle that an earlier store of this scene has sized):
 * nothing synchronises and nothing is allocated but the transient records
 * (stream-ordered).  The extinction check and the fit of the new path set
 * in the handle's buffers are made on the device instead: an invalid grid,
 * or more records or events than the buffers hold, leaves the handle
 * holding no paths (later passes add nothing) and sets bit 8 of the
 * scene's error word, which pt_check reports as PT_E_DEVICE_ASSERT.
 * Callers that use it check pt_check (a store of a similar path set after a
 * synchronous one fits: the buffers keep 1/8 headroom).  On a handle not
 * yet sized, PT_ASYNC is ignored.
 */
int paths_store(const pt_scene* scene, const float* beta_cloud,
                uint64_t first_path, uint64_t n_paths, double n_norm,
                uint64_t seed, uint32_t epoch, pt_paths** paths,
                double* images_ref, uint32_t flags, double* tallies,
                uint64_t* fingerprints, void* stream);

/*
 * paths_reweight -- recycled forward model F(M_t | M_ref) (Eqs.
 * forward_simualtion_recycling and correction factor): every event of every
 * stored path contributes f(x|M_t)/mu(x|M_ref), i.e. its contribution under
 * beta_t times the ratio of path pdfs under beta_t and the stored M_ref.
 * beta_t: device grid; images as in render_forward, divided by the n_norm of
 * the store.  With PT_CACHE the per-(event, camera) contributions are kept
 * in the handle for render_grad.
 */
int paths_reweight(pt_paths* paths, const float* beta_t, double* images,
                   uint32_t flags, void* stream);

/*
 * render_grad -- gradient of the loss with respect to the cloud extinction
 * (Eq. loss_gradient with the recycled estimator of Eq.
 * gradient_simualtion_recycling and the path score function of Sec. 4.4):
 * grad[v] += sum over events and cameras of dL_dI[pixel] * contribution *
 * score_v.  dL_dI: device, images layout (e.g. F - I_gt); grad: device,
 * nx*ny*nz doubles, zeroed first unless PT_ACCUMULATE.  With PT_CACHE the
 * contributions come from the latest paths_reweight (which must have been
 * called with PT_CACHE and the same beta_t, unchanged since): a call whose
 * beta_t is another buffer than that reweight's, or that no
 * paths_reweight(PT_CACHE) preceded since the latest store, is refused
 * with PT_E_INVALID before anything is launched.  (The library cannot see
 * a grid changed in place; paths_cache_token tells callers which reweight
 * the cache holds.)
 */
int render_grad(pt_paths* paths, const float* beta_t, const double* dL_dI,
                double* grad, uint32_t flags, void* stream);

/*
 * paths_cache_token -- which paths_reweight(PT_CACHE) the handle's
 * contribution cache holds: a number that changes with every such call on
 * any handle, or 0 when the cache is invalid (no such call since the latest
 * store).  A caller that keeps the token of its reweight can tell whether a
 * later render_grad(PT_CACHE) would read that reweight's contributions
 * (differentiation through several forward passes before one backward).
 * Host only; never fails (0 for a null handle).
 */
uint64_t paths_cache_token(const pt_paths* paths);

int paths_free(pt_paths* paths);

/*
 * paths_drop_cache -- frees the handle's contribution cache (4 bytes per
 * event and camera, the largest buffer of a stored path set) and
 * invalidates it; the next paths_reweight(PT_CACHE) allocates it again.
 * For path sets stored as several handles whose caches do not fit side by
 * side: reweight every handle without the cache for the images, then per
 * handle reweight with the cache, take its gradient and drop the cache.
 * Synchronises the device (cudaFree); never fails on a null handle.
 */
int paths_drop_cache(pt_paths* paths);
/* Synchronises the stream; fills counts of the latest store. */
int paths_info(const pt_paths* paths, pt_paths_info* out, void* stream);

/*
 * adam_step -- Adam (Kingma & Ba; moment decays b1, b2, step lr, epsilon
 * eps, step number t >= 1) on the cloud extinction with the projection
 * beta >= 0 (Sec. 6: a modified Adam; the modification is not given, the
 * projection keeps extinction physical).  beta, m, v: device float32[n];
 * grad: device float64[n]; mask (nullable): device uint8[n], voxels with 0
 * keep beta, m and v (the optimisation restricted to the photo-hull of
 * space_carve, the initialisation of Sec. 6).
 */
int adam_step(float* beta, float* m, float* v, const double* grad, const uint8_t* mask,
              int64_t n, int32_t t, float lr, float b1, float b2, float eps, void* stream);

/*
 * adam_step_counted -- adam_step with the step number kept on the device:
 * *step (device int32, start at 0) is incremented, then used for the bias
 * corrections (written to scratch, device float[2]).  One captured CUDA
 * graph can so replay every step.
 */
int adam_step_counted(float* beta, float* m, float* v, const double* grad, const uint8_t* mask,
                      int64_t n, int32_t* step, float* scratch, float lr, float b1, float b2,
                      float eps, void* stream);

/*
 * loss_residual -- dL_dI = images - gt and *loss = 1/2 sum (images - gt)^2
 * (Eq. appearance_loss).  All device float64; loss is one double, written
 * (not accumulated).
 */
int loss_residual(const double* images, const double* gt, int64_t n,
                  double* dL_dI, double* loss, void* stream);

/*
 * space_carve -- photo-hull of a cloud from its images (space carving,
 * Kutulakos & Seitz 2000), the initialisation of the reconstructions of
 * Sec. 6.  images: device float64, camera-major as render_forward's.
 * mask: device, V bytes (x fastest), 1 = voxel kept.  A voxel is kept
 * unless some camera sees its centre on a clear pixel (radiance <=
 * threshold); a camera that does not see the centre has no say.  The
 * centre and its projection are computed in float32.
 */
int space_carve(const pt_scene* scene, const double* images, double threshold,
                uint8_t* mask, void* stream);

/*
 * Reflectometry (Sec. 6): light paths among surfaces (the surface rendering
 * equation of Sec. 3) in the closed unit box [0,1]^3 -- diffuse walls, a
 * square Lambertian emitter of the given radiance in the ceiling z = 1,
 * diffuse spheres and one sphere (index phong) with the Phong BRDF
 * f_r = 1 - kappa + kappa (r . w')^gamma (Eq. phong) taken as f_r / pi,
 * r the mirror of the incoming direction, the cosine clamped at 0.  Paths
 * start on the emitter (cosine-weighted), make a local estimate toward the
 * camera at every hit (BRDF times the cosine at the hit, the visibility of
 * the camera, 1/r^2 and the pixel response 1/Omega) and continue in a
 * cosine-weighted direction; roulette and the order limit as for volumes.
 * The path pdf does not depend on (kappa, gamma): stored paths are
 * re-evaluated under new parameters exactly (Eq. 19).
 *   surf_scene_create : copies the spheres (host float[n_spheres * 4]:
 *                  centre, radius) and the camera.  Synchronous.
 *   surf_store   : traces paths first .. first+n-1 (n < 2^28), seed, epoch
 *                  (Philox counter as render_forward, scene id 0), keeping
 *                  per camera event the parameter-free factors and per
 *                  path the lobe cosines of its Phong vertices; tallies
 *                  (nullable, accumulated): injected, hits (collisions),
 *                  camera events (in_view); fingerprints (nullable, n):
 *                  per path, FNV-1a of (surface, pixel or -1) per hit and
 *                  the end.  flags: PT_SORT orders the kept events by pixel
 *                  (a counting sort after tracing); results are the same
 *                  either way up to the order of the FP64 additions.
 *   surf_reweight: images (device float64[W*H], zeroed unless
 *                  PT_ACCUMULATE) of the stored paths under (kappa, gamma)
 *                  divided by n_norm; keeps each event's contribution.
 *   surf_grad    : grad (device float64[2], zeroed unless PT_ACCUMULATE)
 *                  += d loss / d (kappa, gamma) for dL_dI (device float64
 *                  [W*H]), from the contributions of the latest
 *                  surf_reweight, which must have used the same (kappa,
 *                  gamma).
 *   surf_reweight_dev, surf_grad_dev: the same with (kappa, gamma) read
 *                  from device memory (theta: float[2]), so that an
 *                  optimisation loop needs no host round trip and can be
 *                  captured in a graph.
 *   surf_adam_step: one Adam step (Sec. 6's modified Adam: moments b1, b2;
 *                  bias corrections from the step number) on
 *                  u = (kappa, gamma / gamma_scale) with gradient
 *                  (grad[0], grad[1] * gamma_scale), step size
 *                  lr / (1 + (t - 1) / lr_decay) at step t (lr_decay = 0:
 *                  constant lr), then the projection onto
 *                  0 <= kappa <= 1, gamma >= 0 of Eq. phong.  theta
 *                  (device float[2], in/out), m, v (device float[2], the
 *                  moments of u), grad (device float64[2]), step (device
 *                  int32, incremented; bias corrections use the new value).
 *                  trace (nullable device float[2 * trace_cap]) receives
 *                  (kappa, gamma) after step t at 2 (t-1) while
 *                  t <= trace_cap.  One thread; asynchronous.
 */
typedef struct {
    int32_t n_spheres;
    const float* spheres;        /* host, n_spheres x 4: centre, radius  */
    int32_t phong;               /* index of the Phong sphere, -1 none   */
    float light[4];              /* emitter on z = 1: x0, x1, y0, y1     */
    float radiance;
    pt_camera camera;
    int32_t max_orders, rr_start;
    float rr_q;
} pt_surf_desc;

typedef struct pt_surf pt_surf;
typedef struct pt_surf_paths pt_surf_paths;
int surf_scene_create(const pt_surf_desc* desc, pt_surf** out);
int surf_scene_free(pt_surf* scene);
int64_t surf_scene_pixels(const pt_surf* scene);
int surf_store(const pt_surf* scene, uint64_t first_path, uint64_t n_paths, double n_norm, uint64_t seed,
               uint32_t epoch, pt_surf_paths** paths, double* tallies, uint64_t* fingerprints, uint32_t flags,
               void* stream);
int surf_reweight(pt_surf_paths* paths, double kappa, double gamma, double* images, uint32_t flags,
                  void* stream);
int surf_grad(pt_surf_paths* paths, double kappa, double gamma, const double* dL_dI, double* grad,
              uint32_t flags, void* stream);
int surf_reweight_dev(pt_surf_paths* paths, const float* theta, double* images, uint32_t flags, void* stream);
int surf_grad_dev(pt_surf_paths* paths, const float* theta, const double* dL_dI, double* grad, uint32_t flags,
                  void* stream);
int surf_adam_step(float* theta, float* m, float* v, const double* grad, int32_t* step, float lr,
                   float lr_decay, float gamma_scale, float b1, float b2, float eps, float* trace,
                   int32_t trace_cap, void* stream);
int surf_paths_events(const pt_surf_paths* paths, uint64_t* n_events);   /* synchronous */
int surf_paths_free(pt_surf_paths* paths);

/*
 * Batches: many scenes (each with its own grid size, cameras and stored
 * paths) run each pass in one persistent launch.  Resident blocks pull
 * (scene, tile) work items from a device counter (tiles of 128 paths, 128
 * events or 1024 voxels), so scenes of uneven size share the GPU without a
 * launch per scene.  The passes are those of paths_reweight(PT_CACHE) and
 * render_grad(PT_CACHE), with the same results per scene.
 *   batch_create : groups stored-path handles (owned by the caller, which
 *                  must outlive the batch); sizes the persistent grid from
 *                  the occupancy of the batched kernels.
 *   batch_bind   : host arrays of n device pointers per scene: beta_t
 *                  (grid), images (output), dL_dI (images layout), grad
 *                  (grid, FP64).  Allocates missing contribution caches
 *                  (synchronises).  Bind again after a paths_store that grew
 *                  a handle.
 *   batch_reweight, batch_grad : as paths_reweight / render_grad for every
 *                  scene (outputs zeroed unless PT_ACCUMULATE); batch_grad
 *                  requires PT_CACHE and a preceding batch_reweight(PT_CACHE).
 *                  No allocation or synchronisation: capturable in a CUDA
 *                  graph once bound.
 *   batch_set_launch : launch shape (autotuning knobs).  reg_cap 0 runs the
 *                  kernels with the compiler's register allocation, 1 the
 *                  ones compiled for 10 resident blocks of 128 threads per
 *                  SM for the event forward pass and 9 for the path-weight
 *                  and event-gradient passes (as the single-scene kernels
 *                  reach; a few registers spilled).  blocks_per_sm >= 1
 *                  selects the persistent schedule with that many resident
 *                  blocks per SM (clamped to the variant's occupancy);
 *                  blocks_per_sm = 0 the grouped schedule: one block per
 *                  tile of every scene (tiles laid out from the stored path
 *                  count and event capacity), scene descriptors passed as a
 *                  kernel parameter, up to 64 scenes per launch;
 *                  blocks_per_sm = -1 the per-scene sequence: the launches
 *                  of paths_reweight / render_grad, scene after scene (best
 *                  when every scene fills the GPU on its own).  Results
 *                  do not depend on the shape except for the order of the
 *                  FP64 additions (and, across reg_cap variants, FP32
 *                  rounding of single contributions).  Default: persistent,
 *                  reg_cap 0, the occupancy limit.
 *   batch_launch_limits : the occupancy limit (resident blocks per SM) of
 *                  variant reg_cap.
 */
typedef struct pt_batch pt_batch;
int batch_create(pt_paths* const* paths, int n, pt_batch** out);
int batch_bind(pt_batch* batch, const float* const* beta_t, double* const* images,
               const double* const* dL_dI, double* const* grad, void* stream);
int batch_reweight(pt_batch* batch, uint32_t flags, void* stream);
int batch_grad(pt_batch* batch, uint32_t flags, void* stream);
int batch_set_launch(pt_batch* batch, int reg_cap, int blocks_per_sm);
int batch_launch_limits(pt_batch* batch, int reg_cap, int* max_blocks_per_sm);
int batch_free(pt_batch* batch);

/*
 * render_forward_static -- render_forward for callers that cannot allocate
 * device memory (the paper has no counterpart; this is a deployment
 * variant).  A host application whose allocator owns all device memory, or
 * code running where allocation is not allowed after start-up, cannot
 * create a pt_scene.  This call takes the scene description directly and
 * keeps the tables a pt_scene would hold (camera frames, pixel solid angles,
 * an error word) in one file-scope device array of about 1 MiB that every
 * GPU loading the library holds until the process exits.  It calls no
 * cudaMalloc, cudaFree or allocating library routine.
 * Limits: at most 16 cameras and 2^18 pixels in total; larger scenes return
 * PT_E_INVALID with a message naming the limit.  Arguments and output are as
 * for render_forward (desc is read on the host; cams is a host array).
 * The first call on a device looks up the array's address (once per device,
 * with that device current); make that call before any stream capture.
 * Every call overwrites the array and clears its error word, so calls that
 * overlap on the GPU race; kernel-side invariant checks are not reported.
 */
int render_forward_static(const pt_scene_desc* desc, const float* beta_cloud,
                          uint64_t first_path, uint64_t n_paths, double n_norm,
                          uint64_t seed, uint32_t epoch, double* images,
                          uint32_t flags, void* stream);

/* Synchronises the stream and reports (then clears) kernel-side invariant
 * violations recorded in the scene: PT_E_DEVICE_ASSERT, the text naming the
 * bits (1 voxel index out of range, 2 traversal longer than the grid allows,
 * 4 stored record with an invalid voxel, 8 a paths_store(PT_ASYNC) whose path
 * set did not fit the handle's buffers or whose extinction grid was
 * invalid). */
int pt_check(const pt_scene* scene, void* stream);

/* Test hook for the reporting path: ORs `bits` (1..15, the bits above) into
 * the scene's device error word on the stream, as a kernel that detected the
 * violation would, without running any kernel. */
int pt_inject_error(pt_scene* scene, int bits, void* stream);

const char* pt_last_error(void);
const char* pt_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PATHRECYCLE_H */
