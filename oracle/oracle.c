/*
 * oracle.c -- plain, slow, FP64 CPU reference for Monte-Carlo scattering
 * tomography with path recycling (Czerninski & Schechner, "Accelerating
 * Inverse Rendering By Using a GPU and Reuse of Light Paths", arXiv
 * 2110.00085).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path links, loads or
 * calls this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg do.  It shares no code, header, table or
 * constant with the CUDA implementation: the random-number generator,
 * voxel traversal, phase functions, camera model and estimators below are
 * written from their published definitions.
 *
 * What it computes, in the paper's order and notation:
 *   - forward path tracing through a voxel extinction grid with a
 *     directional sun (Sec. 3.4; sun with parallel rays, Sec. 6.1):
 *     distance sampling by inverting the transmittance (Sec. 3.4.1),
 *     particle-type choice then direction sampling (Sec. 3.4.2);
 *   - local estimation toward every camera pixel (Sec. 3.4.3, Eq. Qd);
 *   - the path-recycling estimator F(M_t | M_ref), i.e. f(x|M_t) over
 *     mu(x|M_ref) for paths sampled under M_ref (Sec. 5.2, Eqs. 19-21);
 *     with M_t = M_ref it is the plain estimator of Eq. (forward_simulation);
 *   - the loss gradient sum_d (F_d - I_d) dF_d/dbeta_v with the path score
 *     function of scattering tomography (Sec. 4.4 and Appendix C, the
 *     equation closing Sec. C.1), evaluated term by term per event;
 *   - reflectometry (Sec. 6): light paths among surfaces (the surface
 *     rendering equation of Sec. 3) with one Phong sphere (Eq. phong),
 *     local estimates at every hit, and the gradient in (kappa, gamma).
 *
 * Readings where the paper is silent or inconsistent are marked READING.
 * Parity status: every function here is pinned by the CPU test suite
 * (closed forms, invariants, quadrature, finite differences, brute force).
 * The two-type medium (cloud + air) is pinned by the first- and
 * second-order radiance of a homogeneous slab and by the law of the first
 * scattering angle; images beyond second order have no closed form and are
 * pinned through energy balance, unbiasedness and the FD identity.
 *
 * Floating point: all path arithmetic is double.  Build with
 * -ffp-contract=off so results do not depend on the host's FMA contraction.
 *
 * Planted mistakes (OR_PLANT_* macros) exist only so that the CPU tests can
 * show their pins reject a plausible error; oracle.build() never defines
 * them, and the tests compile them into separate copies of this file.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846
#define OR_MAXV 64        /* vertices kept per path (max_orders + 1) */

/* tallies (doubles) */
enum {
    T_INJECTED = 0,   /* w0 of paths that entered the box               */
    T_MISSED,         /* w0 of paths that missed the box                */
    T_ESCAPED,        /* weight leaving the box                         */
    T_ABSORBED,       /* w (1 - albedo) at every collision              */
    T_TRUNCATED,      /* weight after the last allowed order            */
    T_RR_KILLED,      /* weight of paths ended by Russian roulette      */
    T_RR_GAIN,        /* weight added by the 1/q survival boost         */
    T_COLLISIONS,     /* number of collisions                           */
    T_ENTERED,        /* number of paths that entered the box           */
    T_SEG_CROSS,      /* voxel intervals crossed by sampled flights     */
    T_SHADOW_CROSS,   /* voxel intervals crossed by in-view shadow rays */
    T_IN_VIEW,        /* local estimates that landed in a pixel         */
    T_COUNT
};

/* event types of a path end */
enum { END_NONE = 0, END_ESCAPE = 1, END_TRUNC = 2, END_RR = 3, END_MISS = 4 };

/* ------------------------------------------------------------------------ */
/* scene description (filled from Python through ctypes)                   */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t nx, ny, nz, n_cams;
    int32_t max_orders, rr_start;
    uint32_t epoch, scene_id;
    uint64_t seed;
    double voxel;                /* km, cubic voxels                        */
    double origin[3];
    double beta_air, albedo_cloud, albedo_air, hg_g;
    double sun[3];               /* unit propagation direction              */
    double sun_irradiance;
    double rr_q;
    const double* cams;          /* n_cams x 12: pos, look_at, up, fov_y, W, H */
} or_scene;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of the      */
/* multiply-xor bijection with Weyl-sequence key schedule.                  */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0; k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* uniform on (0, 1]: the top 24 bits plus one, times 2^-24 */
static double u01(uint32_t x) { return (double)((x >> 8) + 1u) * (1.0 / 16777216.0); }

/* Draw the 4 words of (path, event, tag).  Counter layout:
 * (path lo, path hi, event | tag << 8 | epoch << 16, scene id); key = seed. */
static void draw(const or_scene* s, uint64_t path, uint32_t event, uint32_t tag, double u[4])
{
    uint32_t ctr[4], key[2], w[4];
    ctr[0] = (uint32_t)path;
    ctr[1] = (uint32_t)(path >> 32);
    ctr[2] = (event & 0xffu) | ((tag & 0xffu) << 8) | ((s->epoch & 0xffffu) << 16);
    ctr[3] = s->scene_id;
    key[0] = (uint32_t)s->seed;
    key[1] = (uint32_t)(s->seed >> 32);
    or_philox4x32_10(ctr, key, w);
    for (int i = 0; i < 4; ++i) u[i] = u01(w[i]);
}

/* ---- float32 error budget by perturbation (test infrastructure only) ----
 * The images' budget for float32 implementations is measured, not bounded:
 * each path is sampled again with every computed vertex moved by its
 * float32 roundoff scale in a random direction (Monte Carlo arithmetic,
 * Parker 1997), and the change of each event's contribution is recorded.
 * The directions come from splitmix64 (Steele, Lea and Flood, OOPSLA 2014),
 * independent of the method's Philox streams. */
static uint64_t splitmix64(uint64_t x)
{
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

/* unit vector, uniform on the sphere, for (path, vertex, draw) */
static void pert_dir(uint64_t pid, int k, int r, double e[3])
{
    uint64_t h = splitmix64(pid ^ splitmix64(((uint64_t)(uint32_t)k << 32) | (uint32_t)r));
    double a = (double)(h >> 40) / 16777216.0, b = (double)(splitmix64(h) >> 40) / 16777216.0;
    double z = 2.0 * a - 1.0, q = sqrt(fmax(0.0, 1.0 - z * z)), ph = 2.0 * OR_PI * b;
    e[0] = q * cos(ph); e[1] = q * sin(ph); e[2] = z;
}

#define OR_PERT_DRAWS 4     /* perturbed re-samplings per path */
#define OR_PERT_SAFETY 4.0  /* budget = safety * max over draws of |change| */
#define OR_PERT_ULPS 2.0    /* roundoffs per computed quantity */
#define OR_U32 (1.0 / 16777216.0)   /* float32 unit roundoff, 2^-24 */

/* FNV-1a, 64 bit, over the little-endian bytes of 32-bit words */
static uint64_t fnv_word(uint64_t h, uint32_t w)
{
    for (int i = 0; i < 4; ++i) {
        h ^= (uint64_t)((w >> (8 * i)) & 0xffu);
        h *= 0x100000001b3ull;
    }
    return h;
}
uint64_t or_fnv1a_words(const uint32_t* w, int n)
{
    uint64_t h = 0xcbf29ce484222325ull;
    for (int i = 0; i < n; ++i) h = fnv_word(h, w[i]);
    return h;
}

/* ------------------------------------------------------------------------ */
/* small vector helpers                                                      */
/* ------------------------------------------------------------------------ */
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static void normalize3(double a[3])
{
    double n = sqrt(dot3(a, a));
    a[0] /= n; a[1] /= n; a[2] /= n;
}

/* Orthonormal basis around unit n (Duff et al., JCGT 6(1), 2017). */
void or_onb(const double n[3], double b1[3], double b2[3])
{
    double sign = copysign(1.0, n[2]);
    double a = -1.0 / (sign + n[2]);
    double b = n[0] * n[1] * a;
    b1[0] = 1.0 + sign * n[0] * n[0] * a; b1[1] = sign * b; b1[2] = -sign * n[0];
    b2[0] = b; b2[1] = sign + n[1] * n[1] * a; b2[2] = -n[1];
}

/* ------------------------------------------------------------------------ */
/* phase functions (Sec. 3.1.4): HG for cloud, Rayleigh for air.  Both are  */
/* normalised over the sphere (Eq. phase_conservation); mu = cos(theta)     */
/* between incoming and outgoing propagation directions.                    */
/* ------------------------------------------------------------------------ */
double or_phase_hg(double g, double mu)
{
    double den = 1.0 + g * g - 2.0 * g * mu;
    return (1.0 - g * g) / (4.0 * OR_PI * den * sqrt(den));
}
double or_phase_rayleigh(double mu) { return 3.0 * (1.0 + mu * mu) / (16.0 * OR_PI); }

/* inverse CDF of HG in mu (cdf increasing from mu=-1 at u->0 to mu=1 at u=1) */
double or_sample_hg(double g, double u)
{
    if (fabs(g) < 1e-3) return 2.0 * u - 1.0;
    double t = (1.0 - g * g) / (1.0 - g + 2.0 * g * u);
    double mu = (1.0 + g * g - t * t) / (2.0 * g);
    if (mu > 1.0) mu = 1.0;
    if (mu < -1.0) mu = -1.0;
    return mu;
}
/* inverse CDF of Rayleigh: cdf(mu) = (mu^3 + 3 mu + 4)/8, solved by Cardano */
double or_sample_rayleigh(double u)
{
    double q = 4.0 * u - 2.0;
    double w = cbrt(q + sqrt(q * q + 1.0));
    double mu = w - 1.0 / w;
    if (mu > 1.0) mu = 1.0;
    if (mu < -1.0) mu = -1.0;
    return mu;
}

/* rotate unit d by polar cosine mu and azimuth phi about itself */
void or_rotate(const double d[3], double mu, double phi, double out[3])
{
    double b1[3], b2[3];
    or_onb(d, b1, b2);
    double st = sqrt(fmax(0.0, 1.0 - mu * mu));
    double c = cos(phi), s = sin(phi);
    for (int i = 0; i < 3; ++i) out[i] = st * c * b1[i] + st * s * b2[i] + mu * d[i];
}

/* ------------------------------------------------------------------------ */
/* grid geometry: a segment p + t d, t in [0, tmax], is cut by the voxel    */
/* faces into intervals; each interval lies in exactly one voxel, which is  */
/* the voxel containing its midpoint.  This is the set {l_{b,v}} of Sec.    */
/* 4.4 (Fig. inverse_notations) computed by brute force: every face         */
/* crossing is listed and the list sorted.                                  */
/* ------------------------------------------------------------------------ */
typedef struct { int64_t v; double t0, t1; int a0, a1; } ivl;
typedef struct { double t; int axis; } tcut;   /* a face crossing and its axis (-1: segment end) */

static int cmp_cut(const void* a, const void* b)
{
    double x = ((const tcut*)a)->t, y = ((const tcut*)b)->t;
    return (x < y) ? -1 : (x > y) ? 1 : 0;
}

/* clip [0, tmax] to the box; returns 0 when the segment misses it.  The
 * axes of the box faces that bound the clipped range go to *aa, *ab (-1 when
 * the range ends at the segment's own ends). */
static int clip_box_axes(const or_scene* s, const double p[3], const double d[3], double tmax, double* ta,
                         double* tb, int* aa, int* ab)
{
    const int n[3] = {s->nx, s->ny, s->nz};
    double t0 = 0.0, t1 = tmax;
    int a0 = -1, a1 = -1;
    for (int a = 0; a < 3; ++a) {
        double lo = s->origin[a], hi = s->origin[a] + n[a] * s->voxel;
        if (d[a] == 0.0) {
            if (p[a] < lo || p[a] > hi) return 0;
            continue;
        }
        double u0 = (lo - p[a]) / d[a], u1 = (hi - p[a]) / d[a];
        if (u0 > u1) { double tmp = u0; u0 = u1; u1 = tmp; }
        if (u0 > t0) { t0 = u0; a0 = a; }
        if (u1 < t1) { t1 = u1; a1 = a; }
    }
    if (!(t1 > t0)) return 0;
    *ta = t0; *tb = t1;
    if (aa) *aa = a0;
    if (ab) *ab = a1;
    return 1;
}
static int clip_box(const or_scene* s, const double p[3], const double d[3], double tmax, double* ta, double* tb)
{
    return clip_box_axes(s, p, d, tmax, ta, tb, NULL, NULL);
}

/* list the voxel intervals of p + t d on [0, tmax]; out must hold nx+ny+nz+4 */
static int intervals(const or_scene* s, const double p[3], const double d[3], double tmax, ivl* out, tcut* tbuf)
{
    const int n[3] = {s->nx, s->ny, s->nz};
    double ta, tb;
    int aa, ab;
    if (!clip_box_axes(s, p, d, tmax, &ta, &tb, &aa, &ab)) return 0;
    int m = 0;
    tbuf[m].t = ta; tbuf[m++].axis = aa;
    tbuf[m].t = tb; tbuf[m++].axis = ab;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) continue;
        double c0 = (p[a] + ta * d[a] - s->origin[a]) / s->voxel;
        double c1 = (p[a] + tb * d[a] - s->origin[a]) / s->voxel;
        double lo = fmin(c0, c1), hi = fmax(c0, c1);
        long k0 = (long)ceil(lo), k1 = (long)floor(hi);
        if (k0 < 1) k0 = 1;
        if (k1 > n[a] - 1) k1 = n[a] - 1;
        for (long k = k0; k <= k1; ++k) {
            double t = (s->origin[a] + (double)k * s->voxel - p[a]) / d[a];
            if (t > ta && t < tb) { tbuf[m].t = t; tbuf[m++].axis = a; }
        }
    }
    qsort(tbuf, (size_t)m, sizeof(tcut), cmp_cut);
    int cnt = 0;
    for (int i = 0; i + 1 < m; ++i) {
        double t0 = tbuf[i].t, t1 = tbuf[i + 1].t;
        if (!(t1 > t0)) continue;
        double tm = 0.5 * (t0 + t1);
        int64_t idx[3];
        for (int a = 0; a < 3; ++a) {
            double c = floor((p[a] + tm * d[a] - s->origin[a]) / s->voxel);
            if (c < 0) c = 0;
            if (c > n[a] - 1) c = n[a] - 1;
            idx[a] = (int64_t)c;
        }
        out[cnt].v = idx[0] + (int64_t)s->nx * (idx[1] + (int64_t)s->ny * idx[2]);
        out[cnt].t0 = t0;
        out[cnt].t1 = t1;
        out[cnt].a0 = tbuf[i].axis;
        out[cnt].a1 = tbuf[i + 1].axis;
        ++cnt;
    }
    return cnt;
}

static int max_intervals(const or_scene* s) { return s->nx + s->ny + s->nz + 8; }

static double beta_tot(const or_scene* s, const float* bc, int64_t v) { return (double)bc[v] + s->beta_air; }

/* sum of beta * length over the intervals (optical depth) */
static double optical_depth(const or_scene* s, const float* bc, const ivl* iv, int n)
{
    double tau = 0.0;
    for (int i = 0; i < n; ++i) tau += beta_tot(s, bc, iv[i].v) * (iv[i].t1 - iv[i].t0);
    return tau;
}

/* exported: transmittance exp(-tau) between p and p + tmax d (d unit) */
double or_transmittance(const or_scene* s, const float* bc, const double p[3], const double d[3], double tmax)
{
    ivl* iv = (ivl*)malloc(sizeof(ivl) * (size_t)max_intervals(s));
    tcut* tb = (tcut*)malloc(sizeof(tcut) * (size_t)max_intervals(s));
    int n = intervals(s, p, d, tmax, iv, tb);
    double tau = optical_depth(s, bc, iv, n);
    free(iv); free(tb);
    return exp(-tau);
}

/* exported: voxel intervals, for the geometry pins */
int or_intervals(const or_scene* s, const double p[3], const double d[3], double tmax,
                 int64_t* vox, double* len, int cap)
{
    ivl* iv = (ivl*)malloc(sizeof(ivl) * (size_t)max_intervals(s));
    tcut* tb = (tcut*)malloc(sizeof(tcut) * (size_t)max_intervals(s));
    int n = intervals(s, p, d, tmax, iv, tb);
    if (n > cap) n = cap;
    for (int i = 0; i < n; ++i) { vox[i] = iv[i].v; len[i] = iv[i].t1 - iv[i].t0; }
    free(iv); free(tb);
    return n;
}

/* ------------------------------------------------------------------------ */
/* cameras: pinhole, image plane at unit distance along the forward axis.   */
/* READING (pixel response W_d is not given for a perspective pixel): a     */
/* point whose projection falls in pixel d has W_d = 1 / Omega_d, Omega_d    */
/* being the pixel's exact solid angle, so the pixel value is the radiance  */
/* averaged over its solid angle; pixel (col,row) = floor of the scaled     */
/* image-plane coordinates, row 0 at the top, edges go to the higher index. */
/* ------------------------------------------------------------------------ */
typedef struct {
    double C[3], F[3], R[3], U[3];
    double tx, ty;
    int W, H;
    int64_t off;   /* offset of the camera's first pixel in the image array */
} ocam;

static void setup_cams(const or_scene* s, ocam* cams)
{
    int64_t off = 0;
    for (int c = 0; c < s->n_cams; ++c) {
        const double* q = s->cams + 12 * c;
        ocam* k = &cams[c];
        for (int i = 0; i < 3; ++i) { k->C[i] = q[i]; k->F[i] = q[3 + i] - q[i]; }
        normalize3(k->F);
        cross3(k->F, q + 6, k->R);
        normalize3(k->R);
        cross3(k->R, k->F, k->U);
        k->W = (int)q[10];
        k->H = (int)q[11];
        k->ty = tan(0.5 * q[9]);
        k->tx = k->ty * (double)k->W / (double)k->H;
        k->off = off;
        off += (int64_t)k->W * k->H;
    }
}

/* solid angle of [0,x] x [0,y] on the plane at unit distance (signed) */
static double rect_sa(double x, double y) { return atan(x * y / sqrt(1.0 + x * x + y * y)); }

double or_pixel_solid_angle(double tx, double ty, int W, int H, int col, int row)
{
    double xa = tx * (-1.0 + 2.0 * col / (double)W), xb = tx * (-1.0 + 2.0 * (col + 1) / (double)W);
    double ya = ty * (1.0 - 2.0 * (row + 1) / (double)H), yb = ty * (1.0 - 2.0 * row / (double)H);
    return rect_sa(xb, yb) - rect_sa(xa, yb) - rect_sa(xb, ya) + rect_sa(xa, ya);
}

/* pixel of point x in camera k, -1 if behind or outside the image */
static int64_t project(const ocam* k, const double x[3], int* col_out, int* row_out)
{
    double q[3] = {x[0] - k->C[0], x[1] - k->C[1], x[2] - k->C[2]};
    double z = dot3(q, k->F);
    if (!(z > 0.0)) return -1;
    double sx = dot3(q, k->R) / (z * k->tx);
    double sy = dot3(q, k->U) / (z * k->ty);
    double fc = floor((sx + 1.0) * 0.5 * k->W);
    double fr = floor((1.0 - sy) * 0.5 * k->H);
    if (fc < 0 || fc >= k->W || fr < 0 || fr >= k->H) return -1;
    *col_out = (int)fc;
    *row_out = (int)fr;
    return (int64_t)fr * k->W + (int64_t)fc;
}

/* ------------------------------------------------------------------------ */
/* medium (Sec. 4.4): beta = beta_c + beta_a, scattering function            */
/* f_s = beta_s^c f^c + beta_s^a f^a = albedo_c beta_c f^c + albedo_a        */
/* beta_a f^a (Eq. fs_scattering), albedo = beta_s / beta (Eq. eff_sinscat) */
/* ------------------------------------------------------------------------ */
static double fs_medium(const or_scene* s, double bc, double mu)
{
#ifdef OR_PLANT_AIR_BY_EXTINCTION
    /* planted mistake (tests only): the air term weighted by its extinction */
    return s->albedo_cloud * bc * or_phase_hg(s->hg_g, mu) + s->beta_air * or_phase_rayleigh(mu);
#endif
    return s->albedo_cloud * bc * or_phase_hg(s->hg_g, mu) + s->albedo_air * s->beta_air * or_phase_rayleigh(mu);
}
static double beta_s(const or_scene* s, double bc) { return s->albedo_cloud * bc + s->albedo_air * s->beta_air; }

/* ------------------------------------------------------------------------ */
/* sun source.  READING (the derivation uses an isotropic point light, the  */
/* experiments a sun with parallel rays): start points are uniform on the   */
/* rectangle normal to the sun direction that bounds the projected box;     */
/* the first ray runs along the sun direction; the emitted-radiance over    */
/* start-pdf factor is F0 * A (A = rectangle area); rays that miss the box  */
/* count in N and contribute nothing.                                       */
/* ------------------------------------------------------------------------ */
typedef struct {
    double e1[3], e2[3];
    double amin, amax, bmin, bmax, hmin;
    double area;
} osun;

static void setup_sun(const or_scene* s, osun* o)
{
    or_onb(s->sun, o->e1, o->e2);
    double L[3] = {s->nx * s->voxel, s->ny * s->voxel, s->nz * s->voxel};
    o->amin = o->bmin = o->hmin = INFINITY;
    o->amax = o->bmax = -INFINITY;
    for (int c = 0; c < 8; ++c) {
        double p[3];
        for (int a = 0; a < 3; ++a) p[a] = s->origin[a] + ((c >> a) & 1) * L[a];
        double pa = dot3(p, o->e1), pb = dot3(p, o->e2), ph = dot3(p, s->sun);
        o->amin = fmin(o->amin, pa); o->amax = fmax(o->amax, pa);
        o->bmin = fmin(o->bmin, pb); o->bmax = fmax(o->bmax, pb);
        o->hmin = fmin(o->hmin, ph);
    }
    o->hmin -= 1.0;
    o->area = (o->amax - o->amin) * (o->bmax - o->bmin);
}

/* ------------------------------------------------------------------------ */
/* one sampled path (Sec. 3.4): vertices x_0 (box entry) .. x_B (last       */
/* collision), outgoing directions om_k, flight lengths l_k into x_k,       */
/* collision voxels v_k.                                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int B, end, entered;
    double x[OR_MAXV][3];
    double om[OR_MAXV][3];
    double l[OR_MAXV];
    int64_t v[OR_MAXV];
    int type[OR_MAXV];       /* particle type chosen at x_k: 0 cloud, 1 air, 2 none */
} opath;

typedef struct {
    const or_scene* s;
    osun sun;
    ocam* cams;
    ivl* iv;
    tcut* tb;
    ivl* iv2;
    tcut* tb2;
    int64_t* touch;   /* budget only: voxels written by grad_add, when set */
    int64_t ntouch, tcap;
} octx;

/* grad[v] += t, recording v in the touched list when one is attached */
static void grad_add(octx* c, double* grad, int64_t v, double t)
{
    grad[v] += t;
    if (c->touch && c->ntouch < c->tcap) c->touch[c->ntouch++] = v;
}

/*
 * Sample path `pid` under extinction bc (Secs. 3.4.1-3.4.2).
 *  - distance: tau ~ Exp(1), the flight ends where the optical depth from
 *    the previous vertex reaches tau (collision), or at the box exit (escape);
 *    a collision needs beta > 0 in its voxel;
 *  - READING (Sec. 3.4.2 picks the type by extinction, while Appendix B
 *    needs the direction pdf to be f_p, which weights types by their
 *    scattering coefficient): the type is picked with probability
 *    albedo_j beta_j / beta_s, which makes the direction pdf exactly f_p;
 *  - READING (termination; the paper ends only on escape): after the local
 *    estimates at collision k, the path stops if k == max_orders, and for
 *    k >= rr_start it survives with constant probability q, its weight
 *    divided by q.  A constant q does not depend on the medium and cancels
 *    in the recycling ratio.
 * Tallies follow the physical weight for the energy-balance check.
 */
static void sample_path(octx* c, const float* bc, uint64_t pid, opath* P, double* tal, int pert)
{
    const or_scene* s = c->s;
    double u[4];
    double w0 = s->sun_irradiance * c->sun.area;
    draw(s, pid, 0, 0, u);
    double a = c->sun.amin + u[0] * (c->sun.amax - c->sun.amin);
    double b = c->sun.bmin + u[1] * (c->sun.bmax - c->sun.bmin);
    double p[3];
    for (int i = 0; i < 3; ++i) p[i] = a * c->sun.e1[i] + b * c->sun.e2[i] + c->sun.hmin * s->sun[i];
    double ta, tbx;
    P->B = 0;
    P->end = END_NONE;
    if (!clip_box(s, p, s->sun, INFINITY, &ta, &tbx)) {
        P->entered = 0;
        P->end = END_MISS;
        if (tal) tal[T_MISSED] += w0;
        return;
    }
    P->entered = 1;
    if (tal) { tal[T_INJECTED] += w0; tal[T_ENTERED] += 1.0; }
    for (int i = 0; i < 3; ++i) { P->x[0][i] = p[i] + ta * s->sun[i]; P->om[0][i] = s->sun[i]; }
    P->v[0] = -1;
    P->l[0] = 0.0;
    P->type[0] = 2;
    /* perturbed re-sampling only (error budget, pert > 0): every computed
     * point moves by a float32 roundoff of the coordinate scale, a collision
     * point also by the roundoff of the optical depth accumulated to it
     * divided by beta there (large where beta is small): u (tau + 1) for the
     * sampled depth, u times the sum of the partial depths of the running
     * sum (the recursive-summation bound), and for every face the flight
     * crossed, its crossing time's roundoff u t_f times the jump of beta at
     * that face */
    double Lsc = 0.0;
    for (int a = 0; a < 3; ++a) {
        const int na = a == 0 ? s->nx : a == 1 ? s->ny : s->nz;
        Lsc = fmax(Lsc, fabs(s->origin[a]) + na * s->voxel);
    }
    if (pert) {
        double e[3];
        pert_dir(pid, 0, pert, e);
        for (int i = 0; i < 3; ++i) P->x[0][i] += OR_PERT_ULPS * OR_U32 * Lsc * e[i];
    }
    double w = w0;
    double tau = -log(u[2]);
    for (int k = 1;; ++k) {
        /* distance sampling from x_{k-1} along om_{k-1} */
        int n = intervals(s, P->x[k - 1], P->om[k - 1], INFINITY, c->iv, c->tb);
        double acc = 0.0;
        int hit = 0;
        double tcol = 0.0;
        int64_t vcol = -1;
        /* budget only: sum of t_f |beta jump| over the faces before the
         * collision (start included), and the sum of the partial optical
         * depths (a float32 running sum rounds relative to each partial sum) */
        double jumps = 0.0, bprev = 0.0, partials = 0.0;
        for (int i = 0; i < n; ++i) {
            double bt = beta_tot(s, bc, c->iv[i].v);
            double len = c->iv[i].t1 - c->iv[i].t0;
            jumps += fabs(bt - bprev) * c->iv[i].t0;
            bprev = bt;
            if (tal) tal[T_SEG_CROSS] += 1.0;
            if (bt > 0.0 && tau - acc <= bt * len) {
                tcol = c->iv[i].t0 + (tau - acc) / bt;
                vcol = c->iv[i].v;
                hit = 1;
                break;
            }
            acc += bt * len;
            partials += acc;
        }
        if (!hit) {
            P->end = END_ESCAPE;
            if (tal) tal[T_ESCAPED] += w;
            return;
        }
        for (int i = 0; i < 3; ++i) P->x[k][i] = P->x[k - 1][i] + tcol * P->om[k - 1][i];
        P->l[k] = tcol;
        P->v[k] = vcol;
        P->type[k] = 2;
        P->B = k;
        if (pert) {
            double e[3];
            pert_dir(pid, k, pert, e);
            double m = OR_PERT_ULPS * OR_U32 * (Lsc + (tau + 1.0 + partials + jumps) / beta_tot(s, bc, vcol));
            for (int i = 0; i < 3; ++i) P->x[k][i] += m * e[i];
        }
        double bcv = (double)bc[vcol];
        double alb = beta_s(s, bcv) / beta_tot(s, bc, vcol);
        if (tal) { tal[T_COLLISIONS] += 1.0; tal[T_ABSORBED] += w * (1.0 - alb); }
        w *= alb;
        draw(s, pid, (uint32_t)k, 0, u);
        if (k == s->max_orders) {
            P->end = END_TRUNC;
            if (tal) tal[T_TRUNCATED] += w;
            return;
        }
        if (k >= s->rr_start) {
            if (u[0] <= s->rr_q) {
                if (tal) tal[T_RR_GAIN] += w * (1.0 / s->rr_q - 1.0);
                w /= s->rr_q;
            } else {
                P->end = END_RR;
                if (tal) tal[T_RR_KILLED] += w;
                return;
            }
        }
        /* particle type, then direction from that type's phase function */
        double bsc = s->albedo_cloud * bcv;
        int cloud = (u[1] * beta_s(s, bcv) <= bsc);
#ifdef OR_PLANT_TYPE_BY_EXTINCTION
        /* planted mistake (tests only): type chosen by extinction */
        cloud = (u[1] * beta_tot(s, bc, vcol) <= bcv);
#endif
        P->type[k] = cloud ? 0 : 1;
        double mu = cloud ? or_sample_hg(s->hg_g, u[2]) : or_sample_rayleigh(u[2]);
        or_rotate(P->om[k - 1], mu, 2.0 * OR_PI * u[3], P->om[k]);
        draw(s, pid, (uint32_t)k, 1, u);
        tau = -log(u[0]);
        if (k + 1 >= OR_MAXV) { P->end = END_TRUNC; return; }
    }
}

/*
 * Evaluate the sampled path under extinction bt (paths drawn under br):
 * every event b = 1..B is a local estimate toward each camera (Eq. Qd);
 * its estimate of f(x|M_t)/mu(x|M_ref) (Eq. forward_simualtion_recycling)
 * is written out factor by factor:
 *   F0 A                                  source radiance / start pdf
 *   prod_{k<=b} T_t(seg k)/T_ref(seg k)   flights x_{k-1} -> x_k; the
 *                                         beta(x_k) factor of the distance pdf
 *                                         is kept with the vertex below
 *   prod_{k<b} f_s,t(x_k, mu_k) / (beta_ref(x_k) f_p,ref(x_k, mu_k))
 *                                         scattering vs. collision and
 *                                         direction pdfs (Eqs. gk_scatter,
 *                                         final_mu)
 *   f_s,t(x_b, mu_bd) / beta_ref(x_b)     local estimate (P_le of Sec. 3.4.3)
 *   T_t(x_b -> C_d) / |x_b - C_d|^2       shadow ray and G
 *   1 / Omega_d                           pixel response
 *   q^-(number of roulette survivals)     termination pdf
 * READING (Eq. Qd's indices are garbled): event b uses the albedo-like
 * factors of vertices 1..b, the phase function at x_b for the angle between
 * om_{b-1} and the direction to the camera, and the transmittance from x_b
 * to the camera.
 * READING (the correction factor of Eq. 20 is written for a whole path):
 * each event is its own sub-path, so its ratio covers vertices 0..b.
 *
 * With dldi != NULL the loss gradient is accumulated: for each event,
 * a = dL/dI[pixel] * contribution, times the path score function of
 * Sec. 4.4 written for the sub-path ending at the camera:
 *   -sum_{k=1..b} l_{k,v}  - l_{(b->d),v}
 *   + sum_{k=1..b-1} [x_k in v] h(x_k, mu_k) + [x_b in v] h(x_b, mu_bd),
 *   h = albedo_c f^c(mu) / f_s,t(mu)   (Eq. fs_deriv).
 * READING (the paper's sums run over vertex 0, the source, which has no
 * scattering term, and over the segment after the last vertex): vertex
 * terms cover the scattering vertices of the sub-path only, segment terms
 * its sampled flights plus the shadow ray; the escape flight is in no
 * sub-path.  Events with zero contribution are skipped (their score may be
 * infinite where beta_c = 0 and there is no air).
 */
/* float32 error budget of an interval's length (budget only, not part of
 * the method): a float32 traversal computes each crossing time t with an
 * error of a few units of roundoff of t itself, and the face it crosses
 * sits at a float32 coordinate X, off by up to u |X|, which moves the
 * crossing time by u |X| / |d_a| (large for a ray nearly parallel to the
 * face, where the face's coordinate is large against the distance to it) */
static double face_roundoff(const double p[3], const double d[3], double t, int a)
{
    if (a < 0 || d[a] == 0.0) return 0.0;
    return 2.0 * OR_U32 * fabs(p[a] + t * d[a]) / fabs(d[a]);
}

static double time_roundoff(const ivl* iv, const double p[3], const double d[3])
{
    return 4.0 * OR_U32 * (fabs(iv->t0) + fabs(iv->t1)) + face_roundoff(p, d, iv->t0, iv->a0) +
           face_roundoff(p, d, iv->t1, iv->a1);
}

/* the same for an optical depth: sum_i x_i (t1 - t0) with x_i the total
 * extinction under ba (minus that under bb when given); each face trades the
 * jump of x there over its crossing time's roundoff, and the float32 running
 * sum adds u times the sum of its partial sums */
static double depth_roundoff(const or_scene* s, const float* ba, const float* bb, const ivl* iv, int n,
                             const double p[3], const double d[3])
{
    double prev = 0.0, own = 0.0, acc = 0.0, partials = 0.0;
    for (int i = 0; i < n; ++i) {
        double x = beta_tot(s, ba, iv[i].v) - (bb ? beta_tot(s, bb, iv[i].v) : 0.0);
        own += fabs(x - prev) * (4.0 * OR_U32 * fabs(iv[i].t0) + face_roundoff(p, d, iv[i].t0, iv[i].a0));
        prev = x;
        acc += x * (iv[i].t1 - iv[i].t0);
        partials += fabs(acc);
    }
    if (n > 0) own += fabs(prev) * (4.0 * OR_U32 * fabs(iv[n - 1].t1) + face_roundoff(p, d, iv[n - 1].t1, iv[n - 1].a1));
    /* the running sum itself rounds relative to each partial sum */
    return own + OR_U32 * partials;
}

static void eval_path(octx* c, const float* br, const float* bt, const opath* P,
                      double inv_norm, double* img, double* icond, int64_t* egp, double* eval,
                      const double* dldi, double* grad, double* gabs, double* gcond, double* tal, uint64_t* fp)
{
    const or_scene* s = c->s;
    /* fingerprint words: per event (voxel, pixel per camera, particle type),
     * then the event count and the end type */
    uint64_t h = 0xcbf29ce484222325ull;
    if (!P->entered) {
        h = fnv_word(h, 0u);
        h = fnv_word(h, (uint32_t)P->end);
        if (fp) *fp = h;
        return;
    }
    double w0 = s->sun_irradiance * c->sun.area;
    double log_tr = 0.0;       /* sum over flights of tau_ref - tau_t */
    double vert = 1.0;         /* product of the vertex ratios k < b  */
    double tr_cond = 0.0;      /* error budget of log_tr (float32 vertices) */
    for (int b = 1; b <= P->B; ++b) {
        int n = intervals(s, P->x[b - 1], P->om[b - 1], P->l[b], c->iv, c->tb);
        log_tr += optical_depth(s, br, c->iv, n) - optical_depth(s, bt, c->iv, n);
        if (icond && br != bt)
            tr_cond += depth_roundoff(s, br, bt, c->iv, n, P->x[b - 1], P->om[b - 1]);
        if (b >= 2) {
            int64_t vk = P->v[b - 1];
            double mu = dot3(P->om[b - 2], P->om[b - 1]);
            double bref = (double)br[vk];
            double fs_ref = fs_medium(s, bref, mu);
            if (fs_ref == 0.0) {
                vert = 0.0;       /* zero weight under M_ref from here on */
            } else {
                double fp_ref = fs_ref / beta_s(s, bref);
#ifdef OR_PLANT_DIRECTION_PDF_BY_EXTINCTION
                /* planted mistake (tests only): the direction pdf normalised
                 * by the extinction, which drops the vertex's albedo */
                fp_ref = fs_ref / beta_tot(s, br, vk);
#endif
                vert *= fs_medium(s, (double)bt[vk], mu) / (beta_tot(s, br, vk) * fp_ref);
            }
        }
        int nrr = b - s->rr_start;
        if (nrr < 0) nrr = 0;
        double base = w0 * exp(log_tr) * vert * pow(s->rr_q, -(double)nrr);
        int64_t vb = P->v[b];
        h = fnv_word(h, (uint32_t)vb);
        for (int d = 0; d < s->n_cams; ++d) {
            const ocam* k = &c->cams[d];
            int col, row;
            int64_t pix = project(k, P->x[b], &col, &row);
            h = fnv_word(h, (uint32_t)(int32_t)pix);
            if (egp) { egp[(b - 1) * s->n_cams + d] = pix < 0 ? -1 : k->off + pix; eval[(b - 1) * s->n_cams + d] = 0.0; }
            if (pix < 0) continue;
            double to[3] = {k->C[0] - P->x[b][0], k->C[1] - P->x[b][1], k->C[2] - P->x[b][2]};
            double r2 = dot3(to, to);
            double r = sqrt(r2);
            double dir[3] = {to[0] / r, to[1] / r, to[2] / r};
            double mu = dot3(P->om[b - 1], dir);
            int ns = intervals(s, P->x[b], dir, r, c->iv2, c->tb2);
            double T = exp(-optical_depth(s, bt, c->iv2, ns));
            double om = or_pixel_solid_angle(k->tx, k->ty, k->W, k->H, col, row);
            double ev = base * fs_medium(s, (double)bt[vb], mu) / beta_tot(s, br, vb) * T / r2 / om;
            if (tal) { tal[T_IN_VIEW] += 1.0; tal[T_SHADOW_CROSS] += (double)ns; }
            int64_t gp = k->off + pix;
            if (img) img[gp] += ev * inv_norm;
            if (eval) eval[(b - 1) * s->n_cams + d] = ev * inv_norm;
            /* the shadow ray's and the flights' own float32 crossing times;
             * the vertices' roundoff is measured by perturbation (or_render) */
            if (icond) icond[gp] += fabs(ev * inv_norm) * (depth_roundoff(s, bt, NULL, c->iv2, ns, P->x[b], dir) + tr_cond);
            if (!dldi || ev == 0.0) continue;
            double A = dldi[gp] * ev * inv_norm;
            /* flights 1..b */
            for (int j = 1; j <= b; ++j) {
                int nj = intervals(s, P->x[j - 1], P->om[j - 1], P->l[j], c->iv, c->tb);
                for (int i = 0; i < nj; ++i) {
                    double t = A * (c->iv[i].t1 - c->iv[i].t0);
                    grad_add(c, grad, c->iv[i].v, -t);
                    if (gabs) gabs[c->iv[i].v] += fabs(t);
                    if (gcond) gcond[c->iv[i].v] += fabs(A) * time_roundoff(&c->iv[i], P->x[j - 1], P->om[j - 1]);
                }
            }
            /* shadow ray x_b -> camera */
            for (int i = 0; i < ns; ++i) {
                double t = A * (c->iv2[i].t1 - c->iv2[i].t0);
                grad_add(c, grad, c->iv2[i].v, -t);
                if (gabs) gabs[c->iv2[i].v] += fabs(t);
                if (gcond) gcond[c->iv2[i].v] += fabs(A) * time_roundoff(&c->iv2[i], P->x[b], dir);
            }
            /* scattering vertices 1..b-1 (angle between sampled directions) */
            for (int j = 1; j < b; ++j) {
                int64_t vj = P->v[j];
                double muj = dot3(P->om[j - 1], P->om[j]);
                double t = A * s->albedo_cloud * or_phase_hg(s->hg_g, muj) / fs_medium(s, (double)bt[vj], muj);
                grad_add(c, grad, vj, t);
                if (gabs) gabs[vj] += fabs(t);
            }
            /* vertex b toward the camera */
            {
                double t = A * s->albedo_cloud * or_phase_hg(s->hg_g, mu) / fs_medium(s, (double)bt[vb], mu);
                grad_add(c, grad, vb, t);
                if (gabs) gabs[vb] += fabs(t);
            }
        }
        h = fnv_word(h, (uint32_t)P->type[b]);
    }
    h = fnv_word(h, (uint32_t)P->B);
    h = fnv_word(h, (uint32_t)P->end);
    if (fp) *fp = h;
}

static int64_t total_pixels(const or_scene* s)
{
    int64_t n = 0;
    for (int c = 0; c < s->n_cams; ++c) n += (int64_t)s->cams[12 * c + 10] * (int64_t)s->cams[12 * c + 11];
    return n;
}

/*
 * Paths first_path .. first_path+n_paths-1, sampled under beta_ref and
 * evaluated under beta_t (pass the same grid for plain path tracing).
 * images (sum of camera W*H, camera-major, row-major) receive the event
 * contributions divided by n_norm; grad/gabs (V doubles) receive the loss
 * gradient and the sum of the absolute values of its terms when dldi is
 * given.  All outputs are accumulated into; tallies (T_COUNT doubles) and
 * fingerprints (n_paths) are optional.  threads > 1 splits paths over
 * OpenMP threads with private buffers (summation order then differs).
 */
int or_render(const or_scene* s, const float* beta_ref, const float* beta_t,
              uint64_t first_path, uint64_t n_paths, double n_norm,
              double* images, double* icond, const double* dldi, double* grad, double* gabs,
              double* gcond, double* tallies, uint64_t* fingerprints, int threads)
{
    if (s->max_orders + 1 >= OR_MAXV || s->max_orders < 1) return -1;
    int64_t npix = total_pixels(s);
    int64_t nvox = (int64_t)s->nx * s->ny * s->nz;
    double inv_norm = 1.0 / n_norm;
    if (threads < 1) threads = 1;
#ifndef _OPENMP
    threads = 1;
#endif
    int err = 0;
#ifdef _OPENMP
#pragma omp parallel num_threads(threads)
#endif
    {
        int tid = 0, nt = 1;
#ifdef _OPENMP
        tid = omp_get_thread_num();
        nt = omp_get_num_threads();
#endif
        octx c;
        c.s = s;
        c.touch = NULL;
        c.ntouch = c.tcap = 0;
        setup_sun(s, &c.sun);
        c.cams = (ocam*)malloc(sizeof(ocam) * (size_t)(s->n_cams > 0 ? s->n_cams : 1));
        setup_cams(s, c.cams);
        int mi = max_intervals(s);
        c.iv = (ivl*)malloc(sizeof(ivl) * (size_t)mi);
        c.tb = (tcut*)malloc(sizeof(tcut) * (size_t)mi);
        c.iv2 = (ivl*)malloc(sizeof(ivl) * (size_t)mi);
        c.tb2 = (tcut*)malloc(sizeof(tcut) * (size_t)mi);
        opath* P = (opath*)malloc(sizeof(opath));
        double* img = images;
        double* ic = icond;
        double* g = grad;
        double* ga = gabs;
        double* gc = gcond;
        double tal[T_COUNT];
        memset(tal, 0, sizeof(tal));
        if (nt > 1) {
            img = images ? (double*)calloc((size_t)npix, sizeof(double)) : NULL;
            ic = icond ? (double*)calloc((size_t)npix, sizeof(double)) : NULL;
            g = grad ? (double*)calloc((size_t)nvox, sizeof(double)) : NULL;
            ga = gabs ? (double*)calloc((size_t)nvox, sizeof(double)) : NULL;
            gc = gcond ? (double*)calloc((size_t)nvox, sizeof(double)) : NULL;
        }
        /* per-event contributions (events b = 1..max_orders, camera d) of
         * the path and of its perturbed re-samplings, for the image budget */
        const int nev = s->max_orders * s->n_cams;
        int64_t* egp0 = NULL; int64_t* egp1 = NULL;
        double* ev0 = NULL; double* ev1 = NULL; double* dm = NULL;
        if (ic) {
            dm = (double*)malloc(sizeof(double) * (size_t)(nev > 0 ? nev : 1));
            egp0 = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nev > 0 ? nev : 1));
            egp1 = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nev > 0 ? nev : 1));
            ev0 = (double*)malloc(sizeof(double) * (size_t)(nev > 0 ? nev : 1));
            ev1 = (double*)malloc(sizeof(double) * (size_t)(nev > 0 ? nev : 1));
        }
        /* the path's own gradient terms, unperturbed and perturbed, with the
         * voxels each evaluation wrote, for the gradient budget */
        const int want_g = gc != NULL && dldi != NULL && g != NULL;
        double* gp0 = NULL; double* gp1 = NULL; double* gmax = NULL;
        int64_t* mark = NULL; int64_t* t0 = NULL; int64_t* t1 = NULL; int64_t* un = NULL;
        const int64_t tcap = (int64_t)s->max_orders * s->n_cams *
                             ((int64_t)(s->max_orders + 2) * mi + s->max_orders + 1);
        if (want_g) {
            gp0 = (double*)calloc((size_t)nvox, sizeof(double));
            gp1 = (double*)calloc((size_t)nvox, sizeof(double));
            gmax = (double*)calloc((size_t)nvox, sizeof(double));
            mark = (int64_t*)calloc((size_t)nvox, sizeof(int64_t));
            un = (int64_t*)malloc(sizeof(int64_t) * (size_t)(tcap > 0 ? tcap : 1) * (OR_PERT_DRAWS + 1));
            t0 = (int64_t*)malloc(sizeof(int64_t) * (size_t)(tcap > 0 ? tcap : 1));
            t1 = (int64_t*)malloc(sizeof(int64_t) * (size_t)(tcap > 0 ? tcap : 1));
        }
        int64_t stamp = 0;
        int overflow = 0;
        for (uint64_t i = (uint64_t)tid; i < n_paths; i += (uint64_t)nt) {
            uint64_t pid = first_path + i;
            if (ic) for (int j = 0; j < nev; ++j) { egp0[j] = -1; ev0[j] = 0.0; }
            sample_path(&c, beta_ref, pid, P, tal, 0);
            eval_path(&c, beta_ref, beta_t, P, inv_norm, img, ic, egp0, ev0, dldi, g, ga, gc, tal,
                      fingerprints ? &fingerprints[i] : NULL);
            if (!ic && !want_g) continue;
            int64_t n0 = 0;
            if (want_g) {
                c.touch = t0; c.ntouch = 0; c.tcap = tcap;
                eval_path(&c, beta_ref, beta_t, P, inv_norm, NULL, NULL, NULL, NULL, dldi, gp0, NULL, NULL, NULL,
                          NULL);
                n0 = c.ntouch;
                c.touch = NULL;
                if (n0 >= tcap) overflow = 1;
            }
            /* an event that stays on its pixel adds the largest change of its
             * contribution over the draws; one that moves (a near-tie of a
             * discrete decision) adds its whole contribution on both pixels;
             * a voxel adds the largest change of the path's gradient terms */
            const double k = OR_PERT_SAFETY;
            int64_t nun = 0;
            ++stamp;
            if (ic) for (int j = 0; j < nev; ++j) dm[j] = 0.0;
            for (int r = 1; r <= OR_PERT_DRAWS; ++r) {
                if (ic) for (int j = 0; j < nev; ++j) { egp1[j] = -1; ev1[j] = 0.0; }
                sample_path(&c, beta_ref, pid, P, NULL, r);
                if (want_g) { c.touch = t1; c.ntouch = 0; c.tcap = tcap; }
                eval_path(&c, beta_ref, beta_t, P, inv_norm, NULL, NULL, ic ? egp1 : NULL, ic ? ev1 : NULL,
                          want_g ? dldi : NULL, want_g ? gp1 : NULL, NULL, NULL, NULL, NULL);
                const int64_t n1 = want_g ? c.ntouch : 0;
                c.touch = NULL;
                if (ic) {
                    for (int j = 0; j < nev; ++j) {
                        if (egp0[j] == egp1[j]) {
                            dm[j] = fmax(dm[j], fabs(ev1[j] - ev0[j]));
                        } else {
                            if (egp0[j] >= 0) ic[egp0[j]] += k * fabs(ev0[j]) / OR_PERT_DRAWS;
                            if (egp1[j] >= 0) ic[egp1[j]] += k * fabs(ev1[j]) / OR_PERT_DRAWS;
                        }
                    }
                }
                if (want_g) {
                    if (n1 >= tcap) overflow = 1;
                    for (int64_t j = 0; j < n0 + n1; ++j) {
                        int64_t v = j < n0 ? t0[j] : t1[j - n0];
                        if (mark[v] != stamp) { mark[v] = stamp; un[nun++] = v; }
                        gmax[v] = fmax(gmax[v], fabs(gp1[v] - gp0[v]));
                    }
                    for (int64_t j = 0; j < n1; ++j) gp1[t1[j]] = 0.0;
                }
            }
            if (ic)
                for (int j = 0; j < nev; ++j)
                    if (egp0[j] >= 0) ic[egp0[j]] += k * dm[j];
            if (want_g) {
                for (int64_t j = 0; j < nun; ++j) { gc[un[j]] += k * gmax[un[j]]; gmax[un[j]] = 0.0; }
                for (int64_t j = 0; j < n0; ++j) gp0[t0[j]] = 0.0;
            }
        }
        free(egp0); free(egp1); free(ev0); free(ev1); free(dm);
        free(gp0); free(gp1); free(gmax); free(mark); free(t0); free(t1); free(un);
#ifdef _OPENMP
#pragma omp critical
#endif
        {
            if (nt > 1) {
                if (img) for (int64_t j = 0; j < npix; ++j) images[j] += img[j];
                if (ic) for (int64_t j = 0; j < npix; ++j) icond[j] += ic[j];
                if (g) for (int64_t j = 0; j < nvox; ++j) grad[j] += g[j];
                if (ga) for (int64_t j = 0; j < nvox; ++j) gabs[j] += ga[j];
                if (gc) for (int64_t j = 0; j < nvox; ++j) gcond[j] += gc[j];
            }
            if (tallies) for (int j = 0; j < T_COUNT; ++j) tallies[j] += tal[j];
            if (overflow) err = -2;
        }
        if (nt > 1) { free(img); free(ic); free(g); free(ga); free(gc); }
        free(P); free(c.iv); free(c.tb); free(c.iv2); free(c.tb2); free(c.cams);
    }
    return err;
}

/*
 * Space carving (Kutulakos & Seitz, IJCV 2000), the initialisation of the
 * reconstructions of Sec. 6: the photo-hull of the cloud from its images.
 * READING (the paper names the method only): a voxel stays in the hull
 * unless some camera sees its centre on a clear pixel (radiance at or below
 * threshold); a camera whose image does not contain the centre, or that has
 * it behind, has no say.  images: camera-major, as render_forward's.
 * mask: V bytes, 1 = in the hull.
 */
void or_space_carve(const or_scene* s, const double* images, double threshold, uint8_t* mask)
{
    ocam* cams = (ocam*)malloc(sizeof(ocam) * (size_t)(s->n_cams > 0 ? s->n_cams : 1));
    setup_cams(s, cams);
    for (int iz = 0; iz < s->nz; ++iz)
        for (int iy = 0; iy < s->ny; ++iy)
            for (int ix = 0; ix < s->nx; ++ix) {
                const double x[3] = {s->origin[0] + (ix + 0.5) * s->voxel, s->origin[1] + (iy + 0.5) * s->voxel,
                                     s->origin[2] + (iz + 0.5) * s->voxel};
                uint8_t keep = 1;
                for (int d = 0; d < s->n_cams && keep; ++d) {
                    int col, row;
                    const int64_t pix = project(&cams[d], x, &col, &row);
                    if (pix >= 0 && images[cams[d].off + pix] <= threshold) keep = 0;
                }
                mask[ix + (int64_t)s->nx * (iy + (int64_t)s->ny * iz)] = keep;
            }
    free(cams);
}

/* continuous image coordinates (column, row; pixel (c, r) covers [c, c+1) x
 * [r, r+1)) of point x in camera cam; returns 0 when x is behind it */
int or_pixel_coords(const or_scene* s, int cam, const double x[3], double out[2])
{
    ocam* cams = (ocam*)malloc(sizeof(ocam) * (size_t)(s->n_cams > 0 ? s->n_cams : 1));
    setup_cams(s, cams);
    const ocam* k = &cams[cam];
    const double q[3] = {x[0] - k->C[0], x[1] - k->C[1], x[2] - k->C[2]};
    const double z = dot3(q, k->F);
    int ok = z > 0.0;
    if (ok) {
        out[0] = (dot3(q, k->R) / (z * k->tx) + 1.0) * 0.5 * k->W;
        out[1] = (1.0 - dot3(q, k->U) / (z * k->ty)) * 0.5 * k->H;
    }
    free(cams);
    return ok;
}

/* Vertices of one path, for inspection: returns B; x (3*(B+1)), om, v, l */
int or_path(const or_scene* s, const float* beta, uint64_t pid, double* x, double* om, int64_t* v, double* l, int* end)
{
    octx c;
    c.s = s;
    c.touch = NULL;
    c.ntouch = c.tcap = 0;
    setup_sun(s, &c.sun);
    int mi = max_intervals(s);
    c.cams = NULL;
    c.iv = (ivl*)malloc(sizeof(ivl) * (size_t)mi);
    c.tb = (tcut*)malloc(sizeof(tcut) * (size_t)mi);
    opath* P = (opath*)malloc(sizeof(opath));
    sample_path(&c, beta, pid, P, NULL, 0);
    int B = P->entered ? P->B : -1;
    for (int k = 0; k <= P->B && P->entered; ++k) {
        for (int i = 0; i < 3; ++i) { x[3 * k + i] = P->x[k][i]; om[3 * k + i] = P->om[k][i]; }
        v[k] = P->v[k];
        l[k] = P->l[k];
    }
    *end = P->end;
    free(P); free(c.iv); free(c.tb);
    return B;
}

/* sun rectangle (for the host-side checks): e1, e2, amin, amax, bmin, bmax, hmin, area */
void or_sun_rect(const or_scene* s, double* out)
{
    osun o;
    setup_sun(s, &o);
    for (int i = 0; i < 3; ++i) { out[i] = o.e1[i]; out[3 + i] = o.e2[i]; }
    out[6] = o.amin; out[7] = o.amax; out[8] = o.bmin; out[9] = o.bmax; out[10] = o.hmin; out[11] = o.area;
}

/*
 * Deterministic single-scattering image by quadrature (a pin for first-order
 * Monte-Carlo): per pixel, sub x sub stratified rays through the pixel,
 * weighted by their solid angle; along each ray the in-scattered radiance
 * beta_s f_p F0 T_sun(x) T_view(x) (first-order term of the integrated RTE,
 * Sec. 3.2) is integrated with `steps` midpoint steps per voxel interval.
 */
void or_single_scatter_quad(const or_scene* s, const float* bc, int sub, int steps, double* images)
{
    int mi = max_intervals(s);
    ocam* cams = (ocam*)malloc(sizeof(ocam) * (size_t)s->n_cams);
    setup_cams(s, cams);
    double ms[3] = {-s->sun[0], -s->sun[1], -s->sun[2]};
    for (int cidx = 0; cidx < s->n_cams; ++cidx) {
        const ocam* k = &cams[cidx];
        int64_t npx = (int64_t)k->W * k->H;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic)
#endif
        for (int64_t pix = 0; pix < npx; ++pix) {
            ivl* iv = (ivl*)malloc(sizeof(ivl) * (size_t)mi);
            tcut* tb = (tcut*)malloc(sizeof(tcut) * (size_t)mi);
            ivl* iv2 = (ivl*)malloc(sizeof(ivl) * (size_t)mi);
            tcut* tb2 = (tcut*)malloc(sizeof(tcut) * (size_t)mi);
            int col = (int)(pix % k->W), row = (int)(pix / k->W);
            double num = 0.0, den = 0.0;
            for (int i = 0; i < sub; ++i) {
                for (int j = 0; j < sub; ++j) {
                    double sx = -1.0 + 2.0 * (col + (i + 0.5) / sub) / k->W;
                    double sy = 1.0 - 2.0 * (row + (j + 0.5) / sub) / k->H;
                    double x = sx * k->tx, y = sy * k->ty;
                    double wgt = 1.0 / pow(1.0 + x * x + y * y, 1.5);
                    double d[3];
                    for (int a = 0; a < 3; ++a) d[a] = k->F[a] + x * k->R[a] + y * k->U[a];
                    normalize3(d);
                    double mu = -dot3(s->sun, d);   /* sun direction vs. toward-camera direction */
                    int n = intervals(s, k->C, d, INFINITY, iv, tb);
                    double Tv = 1.0, L = 0.0;
                    for (int q = 0; q < n; ++q) {
                        double bcv = (double)bc[iv[q].v];
                        double bt = bcv + s->beta_air;
                        double fsv = fs_medium(s, bcv, mu);
                        double h = (iv[q].t1 - iv[q].t0) / steps;
                        for (int m = 0; m < steps; ++m) {
                            double t = iv[q].t0 + (m + 0.5) * h;
                            double p[3];
                            for (int a = 0; a < 3; ++a) p[a] = k->C[a] + t * d[a];
                            int n2 = intervals(s, p, ms, INFINITY, iv2, tb2);
                            double Ts = exp(-optical_depth(s, bc, iv2, n2));
                            double Tw = Tv * exp(-bt * (m + 0.5) * h);
                            L += fsv * s->sun_irradiance * Ts * Tw * h;
                        }
                        Tv *= exp(-bt * (iv[q].t1 - iv[q].t0));
                    }
                    num += wgt * L;
                    den += wgt;
                }
            }
            images[k->off + pix] = num / den;
            free(iv); free(tb); free(iv2); free(tb2);
        }
    }
    free(cams);
}

/* exported geometry of a camera (C, F, R, U, tx, ty), for the host checks */
void or_camera_frame(const or_scene* s, int cam, double* out)
{
    ocam* cams = (ocam*)malloc(sizeof(ocam) * (size_t)s->n_cams);
    setup_cams(s, cams);
    const ocam* k = &cams[cam];
    for (int i = 0; i < 3; ++i) { out[i] = k->C[i]; out[3 + i] = k->F[i]; out[6 + i] = k->R[i]; out[9 + i] = k->U[i]; }
    out[12] = k->tx; out[13] = k->ty;
    free(cams);
}

int or_tally_count(void) { return T_COUNT; }

/* ======================================================================== */
/* Reflectometry (Sec. 6): surfaces (the surface rendering equation of      */
/* Sec. 3) in a closed box -- diffuse walls, a square Lambertian emitter in */
/* the ceiling, diffuse spheres and one sphere with the Phong BRDF          */
/* f_r = 1 - kappa + kappa (r . w')^gamma (Eq. phong).                      */
/* READINGS (the paper gives the experiment, not its scene or sampler):     */
/* - the BRDF is f_r / pi, so a diffuse surface (f_r = 1) reflects all the  */
/*   light (no absorption); the lobe's cosine is taken between the mirror   */
/*   direction r of the incoming propagation direction and the outgoing    */
/*   one, clamped at 0;                                                      */
/* - paths start on the emitter (uniform point, cosine-weighted direction   */
/*   into the box, weight = emitted power) and make a local estimate toward */
/*   the camera at every surface hit (as the volumetric method), with       */
/*   cosine-weighted directions about the normal: the path pdf does not     */
/*   depend on (kappa, gamma), so the recycled estimate is the plain one    */
/*   evaluated under the new parameters (Eq. 19 with mu independent of M);  */
/* - roulette and the order limit as for volumes.                           */
/* ======================================================================== */
typedef struct {
    int32_t n_spheres, phong, max_orders, rr_start;
    uint32_t epoch, pad;
    uint64_t seed;
    double rr_q;
    double light[4];          /* emitter on the ceiling z = 1: x0, x1, y0, y1 */
    double radiance;          /* emitted radiance */
    const double* spheres;    /* n_spheres x 4: centre, radius */
    double cam[12];           /* pos, look_at, up, fov_y, W, H */
} or_surf;

#define SURF_EPS 1e-4

static void surf_draw(const or_surf* s, uint64_t path, uint32_t event, uint32_t tag, double u[4])
{
    uint32_t ctr[4], key[2], w[4];
    ctr[0] = (uint32_t)path;
    ctr[1] = (uint32_t)(path >> 32);
    ctr[2] = (event & 0xffu) | ((tag & 0xffu) << 8) | ((s->epoch & 0xffffu) << 16);
    ctr[3] = 0u;
    key[0] = (uint32_t)s->seed;
    key[1] = (uint32_t)(s->seed >> 32);
    or_philox4x32_10(ctr, key, w);
    for (int i = 0; i < 4; ++i) u[i] = u01(w[i]);
}

/* Phong factor f_r(c) for the lobe cosine c (clamped at 0) and its log
 * derivatives in kappa and gamma */
static double phong_f(double kappa, double gamma, double c) { return 1.0 - kappa + kappa * pow(fmax(c, 0.0), gamma); }
static void phong_dlog(double kappa, double gamma, double c, double out[2])
{
    const double f = phong_f(kappa, gamma, c);
    const double cg = c > 0.0 ? pow(c, gamma) : 0.0;
    out[0] = (cg - 1.0) / f;
    out[1] = c > 0.0 ? kappa * cg * log(c) / f : 0.0;
}

/* nearest surface along p + t d (d unit, p inside the box): returns the
 * surface id (spheres 0..n-1, walls -1..-6 for x-, x+, y-, y+, z-, z+) and
 * fills t and the normal facing the ray; no surface (numerically) -> -100 */
static int surf_hit_p(const or_surf* s, const double p[3], const double d[3], double* t_out, double n[3],
                      double disc_pert)
{
    double best = INFINITY;
    int id = -100;
    for (int i = 0; i < s->n_spheres; ++i) {
        const double* c = s->spheres + 4 * i;
        const double oc[3] = {p[0] - c[0], p[1] - c[1], p[2] - c[2]};
        const double b = dot3(oc, d), cc = dot3(oc, oc) - c[3] * c[3];
        const double disc = b * b - cc + disc_pert * (b * b + fabs(cc));
        if (disc < 0.0) continue;
        const double t = -b - sqrt(disc);
        if (t > SURF_EPS && t < best) { best = t; id = i; }
    }
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) continue;
        const double t = ((d[a] > 0.0 ? 1.0 : 0.0) - p[a]) / d[a];
        if (t > SURF_EPS && t < best) { best = t; id = -(2 * a + (d[a] > 0.0 ? 2 : 1)); }
    }
    if (id == -100) return id;
    *t_out = best;
    if (id >= 0) {
        /* unit normal from the centre to the hit point: divided by the distance
           itself, not the radius, so that a hit point off the sphere by
           rounding gives a unit normal (with the radius, the error of a
           non-unit normal grows along chains of sphere hits) */
        const double* c = s->spheres + 4 * id;
        double q[3];
        for (int k = 0; k < 3; ++k) q[k] = p[k] + best * d[k] - c[k];
        const double ql = sqrt(dot3(q, q));
        for (int k = 0; k < 3; ++k) n[k] = q[k] / ql;
    } else {
        const int a = (-id - 1) / 2;
        for (int k = 0; k < 3; ++k) n[k] = 0.0;
        n[a] = (-id - 1) % 2 ? -1.0 : 1.0;     /* x+ wall faces -x, x- wall faces +x */
    }
    return id;
}

static int surf_hit(const or_surf* s, const double p[3], const double d[3], double* t_out, double n[3])
{
    return surf_hit_p(s, p, d, t_out, n, 0.0);
}

/* is the segment x -> x + r w free of spheres? */
static int surf_visible(const or_surf* s, const double x[3], const double w[3], double r)
{
    for (int i = 0; i < s->n_spheres; ++i) {
        const double* c = s->spheres + 4 * i;
        const double oc[3] = {x[0] - c[0], x[1] - c[1], x[2] - c[2]};
        const double b = dot3(oc, w), cc = dot3(oc, oc) - c[3] * c[3];
        const double disc = b * b - cc;
        if (disc < 0.0) continue;
        const double t = -b - sqrt(disc);
        if (t > SURF_EPS && t < r) return 0;
    }
    return 1;
}


/* a random unit vector at right angles to n (for the perturbed re-samplings) */
static void tangent_dir(uint64_t pid, int k, int r, const double n[3], double e[3])
{
    pert_dir(pid, k, r, e);
    const double en = dot3(e, n);
    for (int a = 0; a < 3; ++a) e[a] -= en * n[a];
    const double m = sqrt(dot3(e, e));
    if (m > 0.0)
        for (int a = 0; a < 3; ++a) e[a] /= m;
}

/* one path (identical draws to the CUDA path); pert > 0: perturbed
 * re-sampling r = pert for the float32 budget -- every direction moves by
 * OR_PERT_ULPS roundoffs, every hit point by as many roundoffs of its
 * coordinates along its surface, and every sphere's discriminant by as many
 * roundoffs of its two terms (it is their difference, nearly 0 for a ray
 * that grazes the sphere, where the hit moves far); events: epix / eval per hit (1 camera),
 * the path's gradient terms in gpath[2] */
static uint64_t surf_path(const or_surf* s, const ocam* cam, double kappa, double gamma, uint64_t pid, int pert,
                          double inv_norm, double* images, const double* dldi, double* grad, double* gabs,
                          double* tal, int32_t* epix, double* eval, double gpath[2])
{
    uint64_t h = 0xcbf29ce484222325ull;
    double u[4];
    const double area = (s->light[1] - s->light[0]) * (s->light[3] - s->light[2]);
    const double w0 = OR_PI * s->radiance * area;
    surf_draw(s, pid, 0, 0, u);
    double x[3] = {s->light[0] + u[0] * (s->light[1] - s->light[0]),
                   s->light[2] + u[1] * (s->light[3] - s->light[2]), 1.0};
    double nrm[3] = {0.0, 0.0, -1.0};
    double b1[3], b2[3], d[3];
    {
        const double rr = sqrt(u[2]), ph = 2.0 * OR_PI * u[3], ct = sqrt(fmax(0.0, 1.0 - u[2]));
        or_onb(nrm, b1, b2);
        for (int k = 0; k < 3; ++k) d[k] = rr * cos(ph) * b1[k] + rr * sin(ph) * b2[k] + ct * nrm[k];
    }
    double w = w0;               /* parameter-free part of the weight */
    double dlog_path[2] = {0.0, 0.0};
    double fpath = 1.0;          /* Phong factors of the path so far */
    if (gpath) gpath[0] = gpath[1] = 0.0;
    if (tal) tal[T_INJECTED] += w0;
    int end = END_NONE;
    for (int k = 1;; ++k) {
        if (pert) {                                  /* direction roundoff */
            double e[3];
            pert_dir(pid, 2 * k, pert, e);
            for (int a = 0; a < 3; ++a) d[a] += OR_PERT_ULPS * OR_U32 * e[a];
            normalize3(d);
        }
        double t, dp = 0.0;
        if (pert) {                                  /* discriminant roundoff */
            double e[3];
            pert_dir(pid, 2 * k + 64, pert, e);
            dp = OR_PERT_ULPS * OR_U32 * e[0];
        }
        const int id = surf_hit_p(s, x, d, &t, nrm, dp);
        if (id == -100) {
            end = END_ESCAPE;
            if (tal) tal[T_ESCAPED] += w * fpath;
            break;
        }
        for (int a = 0; a < 3; ++a) x[a] += t * d[a];
        if (pert) {                                  /* hit-point roundoff, along the surface */
            double e[3];
            tangent_dir(pid, 2 * k + 1, pert, nrm, e);
            const double m = OR_PERT_ULPS * OR_U32 * (1.0 + sqrt(dot3(x, x)));
            for (int a = 0; a < 3; ++a) x[a] += m * e[a];
        }
        if (tal) tal[T_COLLISIONS] += 1.0;
        h = fnv_word(h, (uint32_t)(id + 100));
        const int phong = id == s->phong;
        /* mirror direction of the incoming propagation direction */
        const double dn = dot3(d, nrm);
        const double mir[3] = {d[0] - 2.0 * dn * nrm[0], d[1] - 2.0 * dn * nrm[1], d[2] - 2.0 * dn * nrm[2]};
        /* local estimate toward the camera */
        int32_t pixv = -1;
        {
            const double to[3] = {cam->C[0] - x[0], cam->C[1] - x[1], cam->C[2] - x[2]};
            const double r2 = dot3(to, to), r = sqrt(r2);
            const double wc[3] = {to[0] / r, to[1] / r, to[2] / r};
            const double cn = dot3(nrm, wc);
            int col, row;
            const int64_t pix = cn > 0.0 ? project(cam, x, &col, &row) : -1;
            if (pix >= 0 && surf_visible(s, x, wc, r)) {
                pixv = (int32_t)pix;
                const double cm = dot3(mir, wc);
                const double fe = phong ? phong_f(kappa, gamma, cm) : 1.0;
                const double om = or_pixel_solid_angle(cam->tx, cam->ty, cam->W, cam->H, col, row);
                const double ev = w * fpath * fe / OR_PI * cn / r2 / om;
                if (tal) tal[T_IN_VIEW] += 1.0;
                if (images) images[pix] += ev * inv_norm;
                if (eval) { epix[k - 1] = pixv; eval[k - 1] = ev * inv_norm; }
                if (dldi && ev != 0.0) {
                    double dl[2] = {dlog_path[0], dlog_path[1]};
                    if (phong) {
                        double e2[2];
                        phong_dlog(kappa, gamma, cm, e2);
                        dl[0] += e2[0];
                        dl[1] += e2[1];
                    }
                    const double A = dldi[pix] * ev * inv_norm;
                    for (int j = 0; j < 2; ++j) {
                        if (grad) grad[j] += A * dl[j];
                        if (gabs) gabs[j] += fabs(A * dl[j]);
                        if (gpath) gpath[j] += A * dl[j];
                    }
                }
            }
        }
        h = fnv_word(h, (uint32_t)pixv);
        surf_draw(s, pid, (uint32_t)k, 0, u);
        if (k == s->max_orders) {
            end = END_TRUNC;
            if (tal) tal[T_TRUNCATED] += w * fpath;
            break;
        }
        if (k >= s->rr_start) {
            if (u[0] <= s->rr_q) {
                if (tal) tal[T_RR_GAIN] += w * fpath * (1.0 / s->rr_q - 1.0);
                w /= s->rr_q;
            } else {
                end = END_RR;
                if (tal) tal[T_RR_KILLED] += w * fpath;
                break;
            }
        }
        /* cosine-weighted direction about the normal */
        {
            const double rr = sqrt(u[1]), ph = 2.0 * OR_PI * u[2], ct = sqrt(fmax(0.0, 1.0 - u[1]));
            or_onb(nrm, b1, b2);
            for (int a = 0; a < 3; ++a) d[a] = rr * cos(ph) * b1[a] + rr * sin(ph) * b2[a] + ct * nrm[a];
        }
        if (phong) {
            const double c = dot3(mir, d);
            const double f = phong_f(kappa, gamma, c);
            if (tal) tal[T_ABSORBED] += w * fpath * (1.0 - f);
            fpath *= f;
            double e2[2];
            phong_dlog(kappa, gamma, c, e2);
            dlog_path[0] += e2[0];
            dlog_path[1] += e2[1];
        }
    }
    h = fnv_word(h, (uint32_t)end);
    return h;
}

/*
 * Paths first .. first+n-1 (sampling independent of the BRDF parameters),
 * evaluated under (kappa, gamma): images (W*H, row-major) += contributions /
 * n_norm; with dldi, grad[2] += d loss / d (kappa, gamma) and gabs[2] the sum
 * of the absolute values of its terms; tallies as or_render's; fingerprints
 * (nullable): per path, FNV-1a of (surface id, pixel or -1) per hit and the
 * end.  icond (nullable, W*H) and gcond (nullable, 2, with dldi): float32
 * budgets measured by perturbed re-sampling as or_render's (test
 * infrastructure).
 */
int or_surf_render(const or_surf* s, double kappa, double gamma, uint64_t first, uint64_t n, double n_norm,
                   double* images, const double* dldi, double* grad, double* gabs, double* tal, uint64_t* fp,
                   double* icond, double* gcond)
{
    or_scene tmp;
    memset(&tmp, 0, sizeof(tmp));
    tmp.n_cams = 1;
    tmp.cams = s->cam;
    ocam cam;
    setup_cams(&tmp, &cam);
    const double inv_norm = 1.0 / n_norm;
    const int K = s->max_orders > 0 ? s->max_orders : 1;
    int32_t e0p[OR_MAXV], e1p[OR_MAXV];
    double e0v[OR_MAXV], e1v[OR_MAXV], dm[OR_MAXV], g0[2], g1[2];
    for (uint64_t i = 0; i < n; ++i) {
        const uint64_t pid = first + i;
        const int want = icond || (gcond && dldi);
        for (int j = 0; j < K; ++j) { e0p[j] = -1; e0v[j] = 0.0; dm[j] = 0.0; }
        const uint64_t h = surf_path(s, &cam, kappa, gamma, pid, 0, inv_norm, images, dldi, grad, gabs, tal,
                                     want ? e0p : NULL, want ? e0v : NULL, want ? g0 : NULL);
        if (fp) fp[i] = h;
        if (!want) continue;
        double gm[2] = {0.0, 0.0};
        for (int r = 1; r <= OR_PERT_DRAWS; ++r) {
            for (int j = 0; j < K; ++j) { e1p[j] = -1; e1v[j] = 0.0; }
            surf_path(s, &cam, kappa, gamma, pid, r, inv_norm, NULL, dldi, NULL, NULL, NULL, e1p, e1v, g1);
            for (int j = 0; j < K; ++j) {
                if (e0p[j] == e1p[j]) {
                    dm[j] = fmax(dm[j], fabs(e1v[j] - e0v[j]));
                } else if (icond) {
                    if (e0p[j] >= 0) icond[e0p[j]] += OR_PERT_SAFETY * fabs(e0v[j]) / OR_PERT_DRAWS;
                    if (e1p[j] >= 0) icond[e1p[j]] += OR_PERT_SAFETY * fabs(e1v[j]) / OR_PERT_DRAWS;
                }
            }
            if (dldi)
                for (int j = 0; j < 2; ++j) gm[j] = fmax(gm[j], fabs(g1[j] - g0[j]));
        }
        if (icond)
            for (int j = 0; j < K; ++j)
                if (e0p[j] >= 0) icond[e0p[j]] += OR_PERT_SAFETY * dm[j];
        if (gcond && dldi)
            for (int j = 0; j < 2; ++j) gcond[j] += OR_PERT_SAFETY * gm[j];
    }
    return 0;
}
