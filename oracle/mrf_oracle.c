/*
 * FP64 CPU oracle for the hybrid mesh + radiance-field light-transport loop of
 * "Dynamic Mesh-Aware Radiance Fields" (Qiao, Gao et al., ICCV 2023).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * definition that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg load it; the renderer
 * never calls it and shares no code, header or table with it.
 *
 * Everything is computed in double precision, step by step in the order of the
 * paper's Algorithm 1 (Sec. 3.1 "Hybrid Rendering Algorithm"):
 *   per pixel: T = 1, L = 0; for each segment j: cast the ray (Eq. 3, the ray
 *   casting function t(p, w)), march the radiance field along the segment
 *   (Eqs. 10-11: T' = T exp(-int sigma), L += int T(t) sigma m r dt), cast
 *   shadow rays toward the lights, sample the BSDF at the hit and update
 *   L (Eq. 12) and T (Eq. 13, T = T' f |cos| / P), then test termination
 *   (leaves the scene, throughput below tau, bounce limit).
 *
 * Readings of passages the paper leaves open (the CUDA path takes the same ones):
 *  - quadrature: midpoint rule; either a fixed number of samples per segment,
 *    or a fixed step dt whose last interval is clipped at the segment end;
 *    alpha_i = 1 - exp(-sigma_i delta_i), L += T_i alpha_i r_i, T *= exp(-sigma_i delta_i).
 *  - shadow mask m(p_t) = 1 in the march; shadow rays are cast at diffuse hits
 *    toward point lights and uniformly drawn points of triangle area lights
 *    (next-event estimation), visibility from any mesh and transmittance
 *    exp(-int sigma) from the same field march; area lights emit from their
 *    front side and are seen by shadow rays only.
 *  - BSDFs: perfect mirror (T *= rho); smooth dielectric with the exact
 *    unpolarised Fresnel term choosing reflection or Snell refraction (T kept);
 *    Lambertian with cosine-weighted sampling (T *= albedo).
 *  - the emitted-light term of Eq. 12 uses the attenuated throughput T'; all
 *    meshes have L_e = 0 so the term vanishes.
 *  - random numbers: Philox4x64-10 (Salmon et al., SC'11), counter
 *    (ray, spp, segment, 0), key (seed, 0); uniforms from the top 24 bits.
 *
 * Ambiguity flags mark pixels whose path contains a discrete decision within a
 * small margin of its threshold (a hit point within margin_dist world units of
 * a triangle edge, a t tie, a Fresnel draw next to F, ...); FP32 and FP64 may
 * legitimately decide those differently.
 */
#define _DEFAULT_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_NO_HIT 0xFFFFFFFFu

enum { ORC_FIELD_CONST = 0, ORC_FIELD_GAUSS = 1, ORC_FIELD_HASH = 2 };
enum { ORC_MIRROR = 0, ORC_GLASS = 1, ORC_DIFFUSE = 2 };
enum { ORC_LIGHT_POINT = 0, ORC_LIGHT_AREA = 1 };
enum {
    ORC_FLAG_EDGE = 1,      /* near-edge candidate or t tie in a closest-hit cast */
    ORC_FLAG_SHADOW = 2,    /* near-edge candidate in a shadow any-hit test */
    ORC_FLAG_FRESNEL = 4,   /* Fresnel draw, TIR boundary or grazing incidence */
    ORC_FLAG_TAU = 8,       /* throughput next to the termination threshold */
    ORC_FLAG_BASIS = 16,    /* normal z next to the sign switch of the tangent frame */
    ORC_FLAG_TMIN = 32      /* candidate distance next to t_min */
};

/* Scene description.  Mirrored field by field by oracle/__init__.py. */
typedef struct {
    float cam_pos[3], cam_look[3], cam_up[3];
    float vfov_deg;
    uint32_t width, height;
    const float *ray_o, *ray_d;
    uint32_t n_rays;

    int32_t field_kind;
    float aabb_min[3], aabb_max[3];
    float const_sigma, const_rgb[3];
    uint32_t n_blobs;
    const float *blob_c, *blob_r, *blob_peak, *blob_e;
    uint32_t n_levels, log2_T, n_feat;
    const uint32_t *level_res;
    const uint16_t *table;
    uint32_t mlp_width;
    const float *w1, *b1, *w2, *b2, *w3, *b3;
    uint32_t n_support;
    const float *sup_c, *sup_r;

    uint32_t n_verts;
    const float *verts;
    uint32_t n_tris;
    const uint32_t *tris, *tri_mat;
    uint32_t n_mats;
    const int32_t *mat_kind;
    const float *mat_rgb, *mat_ior;
    uint32_t n_lights;
    const float *light_pos, *light_I;

    uint32_t max_bounces, spp;
    uint64_t seed;
    uint32_t steps_per_segment;
    float dt, tau, tmin;

    double margin_dist, margin_t, margin_fresnel;
    const float *field_pose;   /* 3x4 local-to-world [R | t] of the field (rigid), NULL = identity */
    /* several pinhole views in one batch: view k has camera view_cam[10k..10k+9]
     * (pos, look_at, up, vfov) and size view_size[2k], view_size[2k+1]; rays are
     * numbered view by view, row-major within a view */
    uint32_t n_views;
    const float *view_cam;
    const uint32_t *view_size;
    /* light kinds (NULL = every light is a point light).  An area light l is the
     * triangle (light_pos[l], light_v1[l], light_v2[l]) emitting radiance
     * light_I[l] from its front side (normal (v1 - v0) x (v2 - v0)), sampled
     * light_samples[l] times per diffuse hit */
    const int32_t *light_kind;
    const float *light_v1, *light_v2;
    const uint32_t *light_samples;
    /* learned shadow transmittance (shadow_net.c), or NULL: shadow rays from
     * points inside the field box take T from it instead of the march */
    const struct orc_snet *shadow_net;
    /* shadow mask of Sec. 3.1 on the field's samples: when non-zero, a sample's
     * radiance is scaled by prod over lights of (1 - light_mask[l]) for every
     * light whose shadow ray from the sample is blocked by a mesh */
    int32_t shadow_mask;
    const float *light_mask;
    /* view-dependent radiance (the network layout of Instant-NGP): when
     * non-zero the hash field's density network is 32 -> 64 (w1, b1) -> 16
     * (wd2: 16 x 64, bd2), sigma from its output 0, and a colour network takes
     * those 16 outputs and the 16 spherical harmonics of the view direction
     * (in the field's frame): 32 -> 64 (wc1, bc1) -> 64 (wc2, bc2) -> 3
     * (wc3: 3 x 64, bc3), rgb = softplus; w2, b2, w3, b3 are unused */
    int32_t view_dep;
    const float *wd2, *bd2, *wc1, *bc1, *wc2, *bc2, *wc3, *bc3;
    /* base relative margin of the throughput-threshold flag (0: 2e-6): a path
     * is flagged when |max T - tau| <= (margin_tau + depth uncertainty) * tau
     * at a termination test */
    double margin_tau;
} orc_scene;

/* First-order bounds on how far the FP32 path of the CUDA library may lie from
 * this FP64 path.  They decide nothing in the path itself: they only widen the
 * margins of the ambiguity flags as FP32 errors accumulate along a path.
 *   lat : lateral offset of the current ray's line (world units);
 *   dir : angle between the FP32 and FP64 directions (radians);
 *   unc : uncertainty of the path's optical depth, i.e. of ln T, from the FP32
 *         positions of the field samples (see march()). */
typedef struct {
    double lat, dir, unc;
} orc_err;
#define ORC_ERR_POS 2.4e-7   /* FP32 rounding of a point or distance below 2 (two ulps of 1.x) */
#define ORC_ERR_DIR 4e-7     /* FP32 rounding of a unit direction from a camera basis, reflection or refraction */

/* relative margin of the throughput-threshold flag at one termination test */
static double tau_margin(const orc_scene *sc, const orc_err *e) {
    return (sc->margin_tau > 0 ? sc->margin_tau : 2e-6) + (e ? e->unc : 0.0);
}

/* Support of the hash field at p (the value s of orc_support) and its
 * sensitivity to a position error: |grad s| = 2 |p - c| / r^2 = 2 sqrt(1 - s) / r
 * for the sphere that attains the maximum. */
static double support_slope(const orc_scene *sc, const double p[3], double *s_out) {
    double s = 0.0, slope = 0.0;
    for (uint32_t k = 0; k < sc->n_support; ++k) {
        double d2 = 0.0;
        for (int a = 0; a < 3; ++a) { double q = p[a] - sc->sup_c[3 * k + a]; d2 += q * q; }
        double r = sc->sup_r[k], v = 1.0 - d2 / (r * r);
        if (v > s) { s = v; slope = 2.0 * sqrt(d2) / (r * r); }
    }
    *s_out = s;
    return slope;
}

void orc_sh16(const double w[3], double Y[16]);

double orc_snet_forward(const struct orc_snet *n, const double p[3], const double w[3]);

/* per-thread counters: segments, shadow rays, nominal samples, samples with
 * non-zero support, surface hits, paths */
enum { C_SEG = 0, C_SHADOW, C_NOMINAL, C_SUPPORTED, C_HITS, C_PATHS, C_END_MISS, C_END_TAU, C_END_CAP, C_N };

/* ---------------------------------------------------------------- vectors */
typedef struct { double x, y, z; } v3;
static inline v3 mk(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static inline v3 fv(const float *p) { return mk(p[0], p[1], p[2]); }
static inline v3 fv3(const double *p) { return mk(p[0], p[1], p[2]); }
static inline v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static inline v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static inline v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static inline double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static inline v3 cross(v3 a, v3 b) { return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
static inline v3 unit(v3 a) { return scl(a, 1.0 / sqrt(dot(a, a))); }
static inline double comp(v3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }

/* ------------------------------------------------------------ binary16 */
/* IEEE 754 binary16 -> double, from the format definition: 1 sign bit,
 * 5 exponent bits (bias 15), 10 fraction bits; exponent 0 = subnormal. */
double orc_half_to_double(uint16_t h) {
    int sign = (h >> 15) & 1, e = (h >> 10) & 31, f = h & 1023;
    double v;
    if (e == 0) v = ldexp((double)f, -24);
    else if (e == 31) v = f ? NAN : INFINITY;
    else v = ldexp(1024.0 + f, e - 25);
    return sign ? -v : v;
}

/* ------------------------------------------------------------ Philox4x64-10 */
/* Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
 * (SC'11): ten rounds of two 64x64->128 multiplies with a Weyl key schedule. */
static inline void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
    unsigned __int128 p = (unsigned __int128)a * b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}
void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3], k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(0xD2E7470EE14C6C93ull, c0, &hi0, &lo0);
        mulhilo64(0xCA5A826395121157ull, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B97F4A7C15ull;
        k1 += 0xBB67AE8584CAA73Bull;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}
static inline double u24(uint64_t x) { return (double)(x >> 40) * (1.0 / 16777216.0); }

/* three uniforms for the surface event at the end of segment `seg` */
static void draw3(const orc_scene *sc, uint64_t ray, uint64_t s, uint64_t seg, double u[3]) {
    uint64_t ctr[4] = {ray, s, seg, 0}, key[2] = {sc->seed, 0}, out[4];
    orc_philox4x64(ctr, key, out);
    u[0] = u24(out[0]); u[1] = u24(out[1]); u[2] = u24(out[2]);
}

/* two uniforms for shadow sample q of the surface event ending segment `seg`
 * (counter word 3 = 1 + q, so they never meet the surface-event draw) */
static void draw_shadow(const orc_scene *sc, uint64_t ray, uint64_t s, uint64_t seg, uint64_t q, double u[2]) {
    uint64_t ctr[4] = {ray, s, seg, 1 + q}, key[2] = {sc->seed, 0}, out[4];
    orc_philox4x64(ctr, key, out);
    u[0] = u24(out[0]); u[1] = u24(out[1]);
}

/* ---------------------------------------------------------------- camera */
/* Pinhole camera (Algorithm 1: p_0 and w_0 from the pixel and the camera
 * centre): the ray leaves the camera centre through the pixel centre.
 * Pixel index = y * width + x, row y = 0 at the top of the image. */
static void pinhole(const float *cpos, const float *clook, const float *cup, double vfov, uint32_t W, uint32_t H,
                    uint32_t pix, double o[3], double d[3]) {
    v3 pos = fv(cpos), f = unit(sub(fv(clook), pos));
    v3 r = unit(cross(f, fv(cup))), u = cross(r, f);
    double th = tan(0.5 * vfov * M_PI / 180.0), aspect = (double)W / H;
    uint32_t px = pix % W, py = pix / W;
    double sx = (2.0 * (px + 0.5) / W - 1.0) * th * aspect;
    double sy = (1.0 - 2.0 * (py + 0.5) / H) * th;
    v3 dir = unit(add(f, add(scl(r, sx), scl(u, sy))));
    o[0] = pos.x; o[1] = pos.y; o[2] = pos.z;
    d[0] = dir.x; d[1] = dir.y; d[2] = dir.z;
}

void orc_camera_ray(const orc_scene *sc, uint32_t pix, double o[3], double d[3]) {
    if (sc->n_rays) {
        for (int i = 0; i < 3; ++i) { o[i] = sc->ray_o[3 * pix + i]; d[i] = sc->ray_d[3 * pix + i]; }
        v3 dd = unit(mk(d[0], d[1], d[2]));
        d[0] = dd.x; d[1] = dd.y; d[2] = dd.z;
        return;
    }
    if (sc->n_views) {
        uint32_t k = 0, off = 0;
        while (k + 1 < sc->n_views && pix >= off + sc->view_size[2 * k] * sc->view_size[2 * k + 1]) {
            off += sc->view_size[2 * k] * sc->view_size[2 * k + 1];
            ++k;
        }
        const float *c = sc->view_cam + 10 * k;
        pinhole(c, c + 3, c + 6, c[9], sc->view_size[2 * k], sc->view_size[2 * k + 1], pix - off, o, d);
        return;
    }
    pinhole(sc->cam_pos, sc->cam_look, sc->cam_up, sc->vfov_deg, sc->width, sc->height, pix, o, d);
}

/* ---------------------------------------------------------------- field */
/* Multiresolution hash encoding (the Instant-NGP field the paper renders,
 * Sec. 3.3): per level l the point is scaled to the level grid, the 8 corners
 * of its cell are looked up (dense row-major index when the level grid fits the
 * table, else the spatial hash x*1 ^ y*2654435761 ^ z*805459861 mod T), and
 * the features are trilinearly interpolated; levels are concatenated. */
void orc_hash_encode(const orc_scene *sc, const double p[3], double *feat) {
    const uint64_t T = 1ull << sc->log2_T;
    const uint32_t F = sc->n_feat;
    for (uint32_t l = 0; l < sc->n_levels; ++l) {
        const uint32_t N = sc->level_res[l];
        const int dense = (uint64_t)(N + 1) * (N + 1) * (N + 1) <= T;
        int64_t c[3];
        double w[3];
        for (int a = 0; a < 3; ++a) {
            double u = (p[a] - sc->aabb_min[a]) / ((double)sc->aabb_max[a] - sc->aabb_min[a]) * N;
            double fl = floor(u);
            if (fl < 0) fl = 0;
            if (fl > N - 1) fl = N - 1;
            c[a] = (int64_t)fl;
            w[a] = u - fl;
        }
        for (uint32_t f = 0; f < F; ++f) feat[l * F + f] = 0.0;
        for (int k = 0; k < 8; ++k) {
            uint32_t x = (uint32_t)(c[0] + (k & 1)), y = (uint32_t)(c[1] + ((k >> 1) & 1)),
                     z = (uint32_t)(c[2] + ((k >> 2) & 1));
            double wt = ((k & 1) ? w[0] : 1.0 - w[0]) * (((k >> 1) & 1) ? w[1] : 1.0 - w[1]) *
                        (((k >> 2) & 1) ? w[2] : 1.0 - w[2]);
            uint64_t idx;
            if (dense) idx = x + (uint64_t)(N + 1) * (y + (uint64_t)(N + 1) * z);
            else idx = (uint32_t)(x * 1u ^ y * 2654435761u ^ z * 805459861u) & (uint32_t)(T - 1);
            const uint16_t *e = sc->table + ((uint64_t)l * T + idx) * F;
            for (uint32_t f = 0; f < F; ++f) feat[l * F + f] += wt * orc_half_to_double(e[f]);
        }
    }
}

/* The tiny MLP: h1 = ReLU(W1 f + b1), h2 = ReLU(W2 h1 + b2), o = W3 h2 + b3. */
void orc_mlp(const orc_scene *sc, const double *feat, double out[4]) {
    const uint32_t W = sc->mlp_width, D = sc->n_levels * sc->n_feat;
    double h1[256], h2[256];
    for (uint32_t j = 0; j < W; ++j) {
        double a = sc->b1[j];
        for (uint32_t i = 0; i < D; ++i) a += (double)sc->w1[j * D + i] * feat[i];
        h1[j] = a > 0 ? a : 0;
    }
    for (uint32_t j = 0; j < W; ++j) {
        double a = sc->b2[j];
        for (uint32_t i = 0; i < W; ++i) a += (double)sc->w2[j * W + i] * h1[i];
        h2[j] = a > 0 ? a : 0;
    }
    for (uint32_t j = 0; j < 4; ++j) {
        double a = sc->b3[j];
        for (uint32_t i = 0; i < W; ++i) a += (double)sc->w3[j * W + i] * h2[i];
        out[j] = a;
    }
}

/* Compact density support of the hash field: max over spheres of
 * (1 - |p - c|^2 / r^2), clamped at 0. */
double orc_support(const orc_scene *sc, const double p[3]) {
    double s = 0.0;
    for (uint32_t k = 0; k < sc->n_support; ++k) {
        double d2 = 0.0;
        for (int a = 0; a < 3; ++a) { double q = p[a] - sc->sup_c[3 * k + a]; d2 += q * q; }
        double r = sc->sup_r[k], v = 1.0 - d2 / (r * r);
        if (v > s) s = v;
    }
    return s;
}

static int inside_box(const orc_scene *sc, const double p[3]) {
    for (int a = 0; a < 3; ++a)
        if (p[a] < sc->aabb_min[a] || p[a] > sc->aabb_max[a]) return 0;
    return 1;
}

/* Density sigma(p) and linear-HDR radiance r(p) (Eq. 7 and the HDR radiance of
 * Sec. 3.1).  Returns 1 when the sample needed a network evaluation (non-zero
 * support), for the sample counters. */
/* View-dependent hash field: density network, then the colour network of
 * the density outputs and SH16 of the unit view direction d (field frame). */
void orc_mlp_view(const orc_scene *sc, const double *feat, const double d[3], double *sigma_logit, double rgb[3]) {
    const uint32_t W = sc->mlp_width, D = sc->n_levels * sc->n_feat;
    double h1[256], dn[16], x[32], c1[256], c2[256];
    for (uint32_t j = 0; j < W; ++j) {
        double a = sc->b1[j];
        for (uint32_t i = 0; i < D; ++i) a += (double)sc->w1[j * D + i] * feat[i];
        h1[j] = a > 0 ? a : 0;
    }
    for (uint32_t j = 0; j < 16; ++j) {
        double a = sc->bd2[j];
        for (uint32_t i = 0; i < W; ++i) a += (double)sc->wd2[j * W + i] * h1[i];
        dn[j] = a;
    }
    *sigma_logit = dn[0];
    double n = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double u[3] = {d[0] / n, d[1] / n, d[2] / n};
    for (int j = 0; j < 16; ++j) x[j] = dn[j];
    orc_sh16(u, x + 16);
    for (uint32_t j = 0; j < W; ++j) {
        double a = sc->bc1[j];
        for (int i = 0; i < 32; ++i) a += (double)sc->wc1[j * 32 + i] * x[i];
        c1[j] = a > 0 ? a : 0;
    }
    for (uint32_t j = 0; j < W; ++j) {
        double a = sc->bc2[j];
        for (uint32_t i = 0; i < W; ++i) a += (double)sc->wc2[j * W + i] * c1[i];
        c2[j] = a > 0 ? a : 0;
    }
    for (int c = 0; c < 3; ++c) {
        double a = sc->bc3[c];
        for (uint32_t i = 0; i < W; ++i) a += (double)sc->wc3[c * W + i] * c2[i];
        rgb[c] = log1p(exp(a));   /* softplus */
    }
}

static int field_eval_dir(const orc_scene *sc, const double p[3], const double d[3], double *sigma, double rgb[3]);

int orc_field_eval(const orc_scene *sc, const double p[3], double *sigma, double rgb[3]) {
    const double d[3] = {0.0, 0.0, 1.0};
    return field_eval_dir(sc, p, d, sigma, rgb);
}

/* Field at p seen along d (d only matters for view-dependent radiance). */
int orc_field_eval_dir(const orc_scene *sc, const double p[3], const double d[3], double *sigma, double rgb[3]) {
    return field_eval_dir(sc, p, d, sigma, rgb);
}

static int field_eval_dir(const orc_scene *sc, const double p[3], const double d[3], double *sigma, double rgb[3]) {
    *sigma = 0.0; rgb[0] = rgb[1] = rgb[2] = 0.0;
    if (!inside_box(sc, p)) return 0;
    if (sc->field_kind == ORC_FIELD_CONST) {
        *sigma = sc->const_sigma;
        for (int c = 0; c < 3; ++c) rgb[c] = sc->const_rgb[c];
        return 1;
    }
    if (sc->field_kind == ORC_FIELD_GAUSS) {
        /* sigma = sum_k sigma_k, radiance = emission weighted by sigma_k */
        double s = 0.0, se[3] = {0, 0, 0};
        for (uint32_t k = 0; k < sc->n_blobs; ++k) {
            double d2 = 0.0;
            for (int a = 0; a < 3; ++a) { double q = p[a] - sc->blob_c[3 * k + a]; d2 += q * q; }
            double r = sc->blob_r[k], sk = sc->blob_peak[k] * exp(-d2 / (2.0 * r * r));
            s += sk;
            for (int c = 0; c < 3; ++c) se[c] += sk * sc->blob_e[3 * k + c];
        }
        *sigma = s;
        if (s > 0) for (int c = 0; c < 3; ++c) rgb[c] = se[c] / s;
        return 1;
    }
    double sup = orc_support(sc, p);
    if (sup <= 0.0) return 0;   /* sigma = 0 * exp(...) exactly */
    double feat[64], o[4];
    orc_hash_encode(sc, p, feat);
    if (sc->view_dep) {
        double logit;
        orc_mlp_view(sc, feat, d, &logit, rgb);
        *sigma = sup * exp(logit < 15.0 ? logit : 15.0);
        return 1;
    }
    orc_mlp(sc, feat, o);
    *sigma = sup * exp(o[0] < 15.0 ? o[0] : 15.0);
    for (int c = 0; c < 3; ++c) rgb[c] = log1p(exp(o[1 + c]));   /* softplus */
    return 1;
}

/* ------------------------------------------------------- segment bounds */
/* Parameter interval of the ray inside the field box (slab test). */
int orc_box_interval(const orc_scene *sc, const double o[3], const double d[3], double *t0, double *t1) {
    double lo = -INFINITY, hi = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (o[a] < sc->aabb_min[a] || o[a] > sc->aabb_max[a]) return 0;
            continue;
        }
        double ta = (sc->aabb_min[a] - o[a]) / d[a], tb = (sc->aabb_max[a] - o[a]) / d[a];
        if (ta > tb) { double q = ta; ta = tb; tb = q; }
        if (ta > lo) lo = ta;
        if (tb < hi) hi = tb;
    }
    *t0 = lo; *t1 = hi;
    return hi > lo;
}

/* A field that moves as a rigid body (Sec. 3.2: the simulator's homogeneous
 * transform t of a NeRF object; queries use t^-1 p).  With the pose [R | t]
 * (local to world), a world ray (o, d) is the local ray (R^T (o - t), R^T d);
 * R is orthonormal, so ray parameters and lengths are unchanged. */
static void to_field_frame(const orc_scene *sc, const double o[3], const double d[3], double lo[3], double ld[3]) {
    if (!sc->field_pose) {
        for (int a = 0; a < 3; ++a) { lo[a] = o[a]; ld[a] = d[a]; }
        return;
    }
    const float *M = sc->field_pose;
    double q[3] = {o[0] - M[3], o[1] - M[7], o[2] - M[11]};
    for (int a = 0; a < 3; ++a) {
        lo[a] = M[0 + a] * q[0] + M[4 + a] * q[1] + M[8 + a] * q[2];
        ld[a] = M[0 + a] * d[0] + M[4 + a] * d[1] + M[8 + a] * d[2];
    }
}

/* ---------------------------------------------------------------- march */
/* Quadrature of Eqs. 10-11 over [a, b] of the ray, with the shadow mask m = 1:
 *   alpha_i = 1 - exp(-sigma_i delta_i); L += T alpha_i r_i; T *= exp(-sigma_i delta_i).
 * T is the RGB path throughput (it carries T(p_j) into the segment).  Returns
 * 1 if the path ended inside the march because max(T) fell below tau. */
static double shadow_mask(const orc_scene *sc, const double pw[3], uint32_t *flags, double dp);

static int march(const orc_scene *sc, const double ow[3], const double dw[3], double a, double b, double T[3],
                 double L[3], uint64_t *cnt, uint32_t *flags, orc_err *e) {
    double o[3], d[3];
    to_field_frame(sc, ow, dw, o, d);
    double tb0, tb1;
    if (!orc_box_interval(sc, o, d, &tb0, &tb1)) return 0;
    double t0 = a > tb0 ? a : tb0, t1 = b < tb1 ? b : tb1;
    if (!(t1 > t0)) return 0;
    uint64_t n;
    double h;
    if (sc->steps_per_segment) { n = sc->steps_per_segment; h = (t1 - t0) / n; }
    else { h = sc->dt; n = (uint64_t)ceil((t1 - t0) / h); }
    for (uint64_t i = 0; i < n; ++i) {
        double lo = t0 + i * h, hi = sc->steps_per_segment ? t0 + (i + 1) * h : lo + h;
        if (!sc->steps_per_segment && hi > t1) hi = t1;
        double tm = 0.5 * (lo + hi), delta = hi - lo;
        if (delta <= 0) continue;
        double p[3] = {o[0] + tm * d[0], o[1] + tm * d[1], o[2] + tm * d[2]}, sigma, rgb[3];
        cnt[C_NOMINAL]++;
        cnt[C_SUPPORTED] += field_eval_dir(sc, p, d, &sigma, rgb);
        if (e && sigma > 0.0) {
            /* uncertainty of sigma * delta in FP32: rounding, and for the hash
             * field the support's response to the sample's position error,
             * |ds| <= 2 |dp| / r_min, times the density before the support */
            double du = 1e-6 * sigma * delta;
            if (sc->field_kind == ORC_FIELD_HASH && sc->n_support) {
                double sup, slope = support_slope(sc, p, &sup), dp = ORC_ERR_POS + e->lat + tm * e->dir;
                if (sup > 0.0) du += sigma / sup * delta * slope * dp;
            }
            e->unc += du;
        }
        double att = exp(-sigma * delta), alpha = -expm1(-sigma * delta), m = 1.0;
        if (sc->shadow_mask && sigma > 0.0) {
            /* the sample in world space: the pose keeps ray parameters */
            double pw[3] = {ow[0] + tm * dw[0], ow[1] + tm * dw[1], ow[2] + tm * dw[2]};
            m = shadow_mask(sc, pw, flags, e ? ORC_ERR_POS + e->lat + tm * e->dir : 0.0);
        }
        for (int c = 0; c < 3; ++c) { L[c] += T[c] * alpha * m * rgb[c]; T[c] *= att; }
        if (sc->tau > 0) {
            double m = T[0] > T[1] ? T[0] : T[1];
            if (T[2] > m) m = T[2];
            if (fabs(m - sc->tau) <= tau_margin(sc, e) * sc->tau) *flags |= ORC_FLAG_TAU;
            if (m < sc->tau) return 1;
        }
    }
    return 0;
}

/* Field transmittance exp(-int sigma) over [a, b] by the same quadrature. */
double orc_transmittance(const orc_scene *sc, const double ow[3], const double dw[3], double a, double b,
                         uint64_t *cnt) {
    double o[3], d[3];
    to_field_frame(sc, ow, dw, o, d);
    double tb0, tb1;
    uint64_t dummy[C_N] = {0};
    if (!cnt) cnt = dummy;
    if (!orc_box_interval(sc, o, d, &tb0, &tb1)) return 1.0;
    double t0 = a > tb0 ? a : tb0, t1 = b < tb1 ? b : tb1;
    if (!(t1 > t0)) return 1.0;
    uint64_t n;
    double h, tau = 0.0;
    if (sc->steps_per_segment) { n = sc->steps_per_segment; h = (t1 - t0) / n; }
    else { h = sc->dt; n = (uint64_t)ceil((t1 - t0) / h); }
    for (uint64_t i = 0; i < n; ++i) {
        double lo = t0 + i * h, hi = sc->steps_per_segment ? t0 + (i + 1) * h : lo + h;
        if (!sc->steps_per_segment && hi > t1) hi = t1;
        double tm = 0.5 * (lo + hi), delta = hi - lo;
        if (delta <= 0) continue;
        double p[3] = {o[0] + tm * d[0], o[1] + tm * d[1], o[2] + tm * d[2]}, sigma, rgb[3];
        cnt[C_NOMINAL]++;
        cnt[C_SUPPORTED] += orc_field_eval(sc, p, &sigma, rgb);
        tau += sigma * delta;
    }
    return exp(-tau);
}

/* Public wrapper of the march for tests (no threshold). */
void orc_march(const orc_scene *sc, const double o[3], const double d[3], double a, double b, double T[3],
               double L[3]) {
    uint64_t cnt[C_N] = {0};
    uint32_t fl = 0;
    march(sc, o, d, a, b, T, L, cnt, &fl, NULL);
}

/* ---------------------------------------------------------- ray casting */
/* Moller-Trumbore ray/triangle test in FP64 with edge-inclusive barycentrics.
 * Returns 1 on a hit with t > tmin; always reports t, b1, b2 when det != 0. */
int orc_intersect_tri(const double o[3], const double d[3], const double v0[3], const double v1[3],
                      const double v2[3], double tmin, double *t, double *b1, double *b2) {
    v3 O = mk(o[0], o[1], o[2]), D = mk(d[0], d[1], d[2]);
    v3 V0 = mk(v0[0], v0[1], v0[2]);
    v3 e1 = sub(mk(v1[0], v1[1], v1[2]), V0), e2 = sub(mk(v2[0], v2[1], v2[2]), V0);
    v3 pv = cross(D, e2);
    double det = dot(e1, pv);
    if (det == 0.0) { *t = INFINITY; *b1 = *b2 = -1; return 0; }
    double inv = 1.0 / det;
    v3 tv = sub(O, V0);
    double u = dot(tv, pv) * inv;
    v3 qv = cross(tv, e1);
    double v = dot(D, qv) * inv;
    *t = dot(e2, qv) * inv;
    *b1 = u; *b2 = v;
    return u >= 0.0 && v >= 0.0 && u + v <= 1.0 && *t > tmin;
}

static void tri_verts(const orc_scene *sc, uint32_t i, double v0[3], double v1[3], double v2[3]) {
    const uint32_t *t = sc->tris + 3 * i;
    for (int a = 0; a < 3; ++a) {
        v0[a] = sc->verts[3 * t[0] + a];
        v1[a] = sc->verts[3 * t[1] + a];
        v2[a] = sc->verts[3 * t[2] + a];
    }
}

/* Signed distance (world units) from the ray's hit point on the triangle's
 * plane to the nearest edge line: barycentric b_i times the altitude from
 * vertex i.  Negative outside the triangle. */
static double edge_distance(const double v0[3], const double v1[3], const double v2[3], double b1, double b2) {
    v3 a = fv3(v0), b = fv3(v1), c = fv3(v2);
    double area2 = sqrt(dot(cross(sub(b, a), sub(c, a)), cross(sub(b, a), sub(c, a))));
    double l0 = sqrt(dot(sub(c, b), sub(c, b))), l1 = sqrt(dot(sub(c, a), sub(c, a))),
           l2 = sqrt(dot(sub(b, a), sub(b, a)));
    double d0 = (1.0 - b1 - b2) * area2 / l0, d1 = b1 * area2 / l1, d2 = b2 * area2 / l2;
    double m = d0 < d1 ? d0 : d1;
    return d2 < m ? d2 : m;
}

/* Closest hit by brute force over every triangle (the ray-casting function of
 * Eq. 3), skipping the triangle the ray leaves.  Ties within 1e-12 relative go
 * to the lower id.  Sets ORC_FLAG_EDGE / ORC_FLAG_TMIN when a triangle whose
 * hit/miss decision lies within the margins could change the answer. */
/* Edge margin of a candidate hit at parameter t of a ray whose FP32 error
 * bounds are e (NULL: none): the base margin plus the in-plane error of the
 * hit point, (lat + t dir) / |cos| at the triangle (|cos| clamped at 0.01). */
static double edge_margin(const orc_scene *sc, const orc_err *e, const double d[3], const double v0[3],
                          const double v1[3], const double v2[3], double t) {
    if (!e) return sc->margin_dist;
    v3 n = unit(cross(sub(fv3(v1), fv3(v0)), sub(fv3(v2), fv3(v0))));
    double c = fabs(d[0] * n.x + d[1] * n.y + d[2] * n.z);
    if (c < 0.01) c = 0.01;
    return sc->margin_dist + (e->lat + (t > 0.0 ? t : 0.0) * e->dir) / c;
}

static uint32_t closest_hit_e(const orc_scene *sc, const double o[3], const double d[3], uint32_t skip,
                              double *t_out, uint32_t *flags, const orc_err *e);

uint32_t orc_closest_hit(const orc_scene *sc, const double o[3], const double d[3], uint32_t skip, double *t_out,
                         uint32_t *flags) {
    return closest_hit_e(sc, o, d, skip, t_out, flags, NULL);
}

static uint32_t closest_hit_e(const orc_scene *sc, const double o[3], const double d[3], uint32_t skip,
                              double *t_out, uint32_t *flags, const orc_err *e) {
    double best = INFINITY, second = INFINITY, edge_t = INFINITY, tmin_t = INFINITY;
    uint32_t best_id = ORC_NO_HIT;
    for (uint32_t i = 0; i < sc->n_tris; ++i) {
        if (i == skip) continue;
        double v0[3], v1[3], v2[3], t, b1, b2;
        tri_verts(sc, i, v0, v1, v2);
        int hit = orc_intersect_tri(o, d, v0, v1, v2, sc->tmin, &t, &b1, &b2);
        if (!isfinite(t)) continue;
        const double md = edge_margin(sc, e, d, v0, v1, v2, t);
        double ed = edge_distance(v0, v1, v2, b1, b2);
        if (fabs(ed) <= md && t > sc->tmin && t < edge_t) edge_t = t;
        if (ed >= -md && fabs(t - sc->tmin) <= md && t < tmin_t) tmin_t = t;
        if (!hit) continue;
        if (t < best || (fabs(t - best) <= 1e-12 * best && i < best_id)) {
            if (best_id != ORC_NO_HIT) second = best < second ? best : second;
            best = t; best_id = i;
        } else if (t < second) second = t;
    }
    if (flags) {
        double lim = isfinite(best) ? best * (1.0 + sc->margin_t) : INFINITY;
        if (isfinite(edge_t) && edge_t <= lim) *flags |= ORC_FLAG_EDGE;
        if (isfinite(second) && second <= lim) *flags |= ORC_FLAG_EDGE;
        if (isfinite(tmin_t) && tmin_t <= lim) *flags |= ORC_FLAG_TMIN;
    }
    *t_out = best;
    return best_id;
}

/* Any mesh between the shadow-ray origin and the light, t in (tmin, dist).
 * The decision is flagged as ambiguous only when it rests on near-edge or
 * near-endpoint candidates: one triangle hit well inside its edges and well
 * inside (tmin, dist) settles "blocked" whatever the others do. */
static int occluded(const orc_scene *sc, const double o[3], const double d[3], uint32_t skip, double dist,
                    uint32_t *flags, const orc_err *e) {
    int blocked = 0, robust = 0, doubtful = 0;
    for (uint32_t i = 0; i < sc->n_tris; ++i) {
        if (i == skip) continue;
        double v0[3], v1[3], v2[3], t, b1, b2;
        tri_verts(sc, i, v0, v1, v2);
        int hit = orc_intersect_tri(o, d, v0, v1, v2, sc->tmin, &t, &b1, &b2);
        if (!isfinite(t)) continue;
        const double md = edge_margin(sc, e, d, v0, v1, v2, t);
        int near = 0;
        if (t > sc->tmin && t < dist * (1.0 + sc->margin_t)) {
            if (fabs(edge_distance(v0, v1, v2, b1, b2)) <= md) near = 1;
            if (hit && fabs(t - dist) <= sc->margin_t * dist) near = 1;
        }
        doubtful |= near;
        if (hit && t < dist) {
            blocked = 1;
            if (!near) robust = 1;
        }
    }
    if (doubtful && !robust) *flags |= ORC_FLAG_SHADOW;
    return blocked;
}

/* Shadow mask m(p_t) of Sec. 3.1 ("Shadow rays" and Algorithm 1, step 3): a
 * ray from the field sample toward each light (a point light's position, an
 * area light's centroid); each light that a mesh blocks multiplies m by
 * 1 - r_src, its mask strength.  Unblocked: m = 1. */
/* dp: bound on the FP32 position error of the sample (0: none) */
static double shadow_mask(const orc_scene *sc, const double pw[3], uint32_t *flags, double dp) {
    double m = 1.0;
    for (uint32_t l = 0; l < sc->n_lights; ++l) {
        double r = sc->light_mask ? sc->light_mask[l] : 0.0;
        if (r == 0.0) continue;
        v3 y = fv(sc->light_pos + 3 * l);
        if (sc->light_kind && sc->light_kind[l] == ORC_LIGHT_AREA)
            y = scl(add(add(y, fv(sc->light_v1 + 3 * l)), fv(sc->light_v2 + 3 * l)), 1.0 / 3.0);
        double w[3] = {y.x - pw[0], y.y - pw[1], y.z - pw[2]};
        double D = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
        if (!(D > 0)) continue;
        for (int a = 0; a < 3; ++a) w[a] /= D;
        const orc_err Es = {dp, ORC_ERR_DIR + dp / D, 0.0};
        if (occluded(sc, pw, w, ORC_NO_HIT, D, flags, &Es)) m *= 1.0 - r;
    }
    return m;
}

/* ---------------------------------------------------------------- BSDFs */
void orc_reflect(const double d[3], const double n[3], double out[3]) {
    double k = 2.0 * (d[0] * n[0] + d[1] * n[1] + d[2] * n[2]);
    for (int a = 0; a < 3; ++a) out[a] = d[a] - k * n[a];
}

/* Unpolarised Fresnel reflectance of a smooth dielectric interface from the
 * Fresnel equations: F = (r_s^2 + r_p^2) / 2; total internal reflection -> 1. */
double orc_fresnel(double cos_i, double eta_i, double eta_t) {
    double s2t = (eta_i / eta_t) * (eta_i / eta_t) * (1.0 - cos_i * cos_i);
    if (s2t >= 1.0) return 1.0;
    double cos_t = sqrt(1.0 - s2t);
    double rs = (eta_i * cos_i - eta_t * cos_t) / (eta_i * cos_i + eta_t * cos_t);
    double rp = (eta_t * cos_i - eta_i * cos_t) / (eta_t * cos_i + eta_i * cos_t);
    return 0.5 * (rs * rs + rp * rp);
}

/* Snell refraction of unit d through the interface with unit normal n facing
 * the incident side (d.n < 0), eta = eta_i / eta_t.  Returns 0 on TIR. */
int orc_refract(const double d[3], const double n[3], double eta, double out[3]) {
    double cos_i = -(d[0] * n[0] + d[1] * n[1] + d[2] * n[2]);
    double s2t = eta * eta * (1.0 - cos_i * cos_i);
    if (s2t >= 1.0) return 0;
    double cos_t = sqrt(1.0 - s2t);
    for (int a = 0; a < 3; ++a) out[a] = eta * d[a] + (eta * cos_i - cos_t) * n[a];
    return 1;
}

/* Cosine-weighted hemisphere direction around unit n from (u1, u2), in the
 * tangent frame of Duff et al., "Building an Orthonormal Basis, Revisited"
 * (JCGT 2017). */
void orc_sample_cosine(const double n[3], double u1, double u2, double out[3]) {
    double sgn = copysign(1.0, n[2]);
    double a = -1.0 / (sgn + n[2]), b = n[0] * n[1] * a;
    double t1[3] = {1.0 + sgn * n[0] * n[0] * a, sgn * b, -sgn * n[0]};
    double t2[3] = {b, sgn + n[1] * n[1] * a, -n[1]};
    double r = sqrt(u1), phi = 2.0 * M_PI * u2;
    double x = r * cos(phi), y = r * sin(phi), z = sqrt(1.0 - u1 > 0 ? 1.0 - u1 : 0.0);
    for (int k = 0; k < 3; ++k) out[k] = x * t1[k] + y * t2[k] + z * n[k];
}

static inline double maxc(const double T[3]) {
    double m = T[0] > T[1] ? T[0] : T[1];
    return T[2] > m ? T[2] : m;
}

/* Field transmittance of a shadow ray from p along w over (0, D): the
 * network's value when one is given and p lies in the field box (in the
 * field's frame), else the march of Eq. 10. */
static double shadow_transmittance(const orc_scene *sc, const double p[3], const double w[3], double D,
                                   uint64_t *cnt) {
    if (sc->shadow_net) {
        double pl[3], wl[3];
        to_field_frame(sc, p, w, pl, wl);
        int inside = 1;
        for (int a = 0; a < 3; ++a) inside &= pl[a] >= sc->aabb_min[a] && pl[a] <= sc->aabb_max[a];
        if (inside) return orc_snet_forward(sc->shadow_net, p, w);
    }
    return orc_transmittance(sc, p, w, 0.0, D, cnt);
}

/* Next-event estimate of one area light (a triangle of the pruned emissive
 * mesh, Sec. 3.1 "Estimating light sources"): N points y_s drawn uniformly on
 * the triangle (square-root barycentric warp of Shirley and Turk), each a
 * shadow ray; the estimator of the light's reflected radiance is
 *   (albedo / pi) Le A / N  sum_s V_s T_s cos_x cos_y / |y_s - p|^2,
 * with cos_x at the surface normal facing the ray, cos_y at the light's front
 * normal, V the mesh visibility and T the field transmittance of Eq. 10. */
static void area_light_nee(const orc_scene *sc, uint32_t l, uint32_t ray, uint32_t s, uint32_t j, uint32_t *q,
                           const double p[3], const double nf[3], uint32_t hit, const float *rgb, const double T[3],
                           double L[3], uint32_t *flags, uint64_t *cnt, double e_hit) {
    v3 a = fv(sc->light_pos + 3 * l), b = fv(sc->light_v1 + 3 * l), c = fv(sc->light_v2 + 3 * l);
    v3 cr = cross(sub(b, a), sub(c, a));
    double A = 0.5 * sqrt(dot(cr, cr));
    v3 nl = unit(cr);
    uint32_t N = sc->light_samples ? sc->light_samples[l] : 1;
    if (N == 0) N = 1;
    for (uint32_t k = 0; k < N; ++k, ++*q) {
        double u[2];
        draw_shadow(sc, ray, s, j, *q, u);
        double su = sqrt(u[0]), b0 = 1.0 - su, b1 = u[1] * su, b2 = 1.0 - b0 - b1;
        v3 y = add(add(scl(a, b0), scl(b, b1)), scl(c, b2));
        double w[3] = {y.x - p[0], y.y - p[1], y.z - p[2]};
        double D2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2], D = sqrt(D2);
        for (int e = 0; e < 3; ++e) w[e] /= D;
        double cosx = nf[0] * w[0] + nf[1] * w[1] + nf[2] * w[2];
        double cosy = -(nl.x * w[0] + nl.y * w[1] + nl.z * w[2]);
        if (cosx <= 0.0 || cosy <= 0.0) continue;
        cnt[C_SHADOW]++;
        const orc_err Es = {e_hit, ORC_ERR_DIR + e_hit / D, 0.0};
        if (occluded(sc, p, w, hit, D, flags, &Es)) continue;
        double Tf = shadow_transmittance(sc, p, w, D, cnt);
        for (int e = 0; e < 3; ++e)
            L[e] += T[e] * (rgb[e] / M_PI) * sc->light_I[3 * l + e] * A / N * cosx * cosy / D2 * Tf;
    }
}

/* ---------------------------------------------------------- one path */
/* Algorithm 1 for one (ray, spp) pair. */
/* *first_flag receives the segment j during which the path raised its first
 * flag on a decision that can change its course (a closest hit, a Fresnel
 * draw, the tangent frame, the throughput threshold; 0: none): the hit
 * records of the segments before it rest on decisions clear of every margin.
 * Shadow-ray flags change radiance only and do not count here. */
static void trace_path(const orc_scene *sc, uint32_t ray, uint32_t s, double L[3], double *alpha0,
                       uint32_t *segs_out, uint32_t *tri_rec, double *t_rec, uint32_t *path_flags,
                       uint32_t *first_flag, uint64_t *cnt) {
    uint32_t pf = 0, *flags = &pf;
    *first_flag = 0;
#define NOTE_FLAGS(j) do { if ((pf & ~(uint32_t)ORC_FLAG_SHADOW) && !*first_flag) *first_flag = (j); } while (0)
    double o[3], d[3];
    orc_camera_ray(sc, ray, o, d);
    double T[3] = {1, 1, 1};
    L[0] = L[1] = L[2] = 0.0;
    *alpha0 = 0.0;
    uint32_t prev = ORC_NO_HIT, segs = 0;
    /* FP32 error bounds of the camera ray: an exact origin, a direction built
     * from the FP32 camera basis */
    orc_err E = {ORC_ERR_POS, ORC_ERR_DIR, 0.0};
    cnt[C_PATHS]++;
    for (uint32_t j = 1; j <= sc->max_bounces; ++j) {
        double th;
        uint32_t hit = closest_hit_e(sc, o, d, prev, &th, flags, &E);
        double Tprev = T[0];
        int stop = march(sc, o, d, 0.0, th, T, L, cnt, flags, &E);
        if (j == 1) *alpha0 = Tprev > 0 ? 1.0 - T[0] / Tprev : 0.0;
        segs = j;
        cnt[C_SEG]++;
        if (tri_rec) { tri_rec[j - 1] = hit; t_rec[j - 1] = th; }
        NOTE_FLAGS(j);
        if (stop) { cnt[C_END_TAU]++; break; }
        if (hit == ORC_NO_HIT) { cnt[C_END_MISS]++; break; }
        cnt[C_HITS]++;
        double p[3] = {o[0] + th * d[0], o[1] + th * d[1], o[2] + th * d[2]};
        double v0[3], v1[3], v2[3];
        tri_verts(sc, hit, v0, v1, v2);
        v3 ng = unit(cross(sub(fv3(v1), fv3(v0)), sub(fv3(v2), fv3(v0))));
        double n[3] = {ng.x, ng.y, ng.z};
        double dn = d[0] * n[0] + d[1] * n[1] + d[2] * n[2];
        double nf[3] = {dn > 0 ? -n[0] : n[0], dn > 0 ? -n[1] : n[1], dn > 0 ? -n[2] : n[2]};
        /* error of the hit point within the surface, and of the ray line at it */
        const double cos_h = fabs(dn) > 0.01 ? fabs(dn) : 0.01;
        const double e_line = E.lat + th * E.dir, e_hit = e_line / cos_h + ORC_ERR_POS;
        uint32_t m = sc->tri_mat[hit];
        int kind = sc->mat_kind[m];
        const float *rgb = sc->mat_rgb + 3 * m;
        double u[3];
        draw3(sc, ray, s, j, u);
        double nd[3];
        /* Eq. 12: L += T' L_e(p_{j+1}); every mesh has L_e = 0 here. */
        if (kind == ORC_MIRROR) {
            orc_reflect(d, n, nd);
            for (int c = 0; c < 3; ++c) T[c] *= rgb[c];
            /* a mirror keeps a ray bundle's width and its angular spread */
            E.lat = e_line + ORC_ERR_POS;
            E.dir += ORC_ERR_DIR;
        } else if (kind == ORC_GLASS) {
            double ior = sc->mat_ior[m], cos_i = fabs(dn);
            int entering = dn < 0;
            double ei = entering ? 1.0 : ior, et = entering ? ior : 1.0;
            double F = orc_fresnel(cos_i, ei, et);
            double s2t = (ei / et) * (ei / et) * (1.0 - cos_i * cos_i);
            if (fabs(u[0] - F) <= sc->margin_fresnel || fabs(s2t - 1.0) <= 1e-9 || cos_i <= 1e-7)
                *flags |= ORC_FLAG_FRESNEL;
            if (u[0] < F) {
                orc_reflect(d, n, nd);
                E.lat = e_line + ORC_ERR_POS;
                E.dir += ORC_ERR_DIR;
            } else {
                orc_refract(d, nf, ei / et, nd);
                /* Snell: angles scale by eta cos_i / cos_t, bundle widths by cos_t / cos_i */
                double ct = sqrt(1.0 - (s2t < 1.0 ? s2t : 1.0)), ci = cos_h;
                if (ct < 0.01) ct = 0.01;
                E.lat = e_line * ct / ci + ORC_ERR_POS;
                E.dir = E.dir * (ei / et) * ci / ct + ORC_ERR_DIR;
            }
        } else {
            /* next-event estimation toward each light (the shadow rays of
             * Sec. 3.1, "Shadow rays" and Algorithm 1) */
            uint32_t q = 0;   /* shadow-sample index over all area lights of this hit */
            for (uint32_t l = 0; l < sc->n_lights; ++l) {
                if (sc->light_kind && sc->light_kind[l] == ORC_LIGHT_AREA) {
                    area_light_nee(sc, l, ray, s, j, &q, p, nf, hit, rgb, T, L, flags, cnt, e_hit);
                    continue;
                }
                double w[3], D2 = 0.0;
                for (int a = 0; a < 3; ++a) { w[a] = sc->light_pos[3 * l + a] - p[a]; D2 += w[a] * w[a]; }
                double D = sqrt(D2);
                for (int a = 0; a < 3; ++a) w[a] /= D;
                double cosl = nf[0] * w[0] + nf[1] * w[1] + nf[2] * w[2];
                if (cosl <= 0.0) continue;
                cnt[C_SHADOW]++;
                /* the shadow ray starts at the hit point and aims at the light */
                const orc_err Es = {e_hit, ORC_ERR_DIR + e_hit / D, 0.0};
                if (occluded(sc, p, w, hit, D, flags, &Es)) continue;
                double Tf = shadow_transmittance(sc, p, w, D, cnt);
                for (int c = 0; c < 3; ++c)
                    L[c] += T[c] * (rgb[c] / M_PI) * cosl * sc->light_I[3 * l + c] / D2 * Tf;
            }
            if (nf[2] != 0.0 && fabs(nf[2]) <= 1e-6) *flags |= ORC_FLAG_BASIS;
            orc_sample_cosine(nf, u[1], u[2], nd);
            for (int c = 0; c < 3; ++c) T[c] *= rgb[c];
            /* the sampled direction depends on the normal only; the new ray
             * starts at the hit point */
            E.lat = e_hit;
            E.dir = ORC_ERR_DIR;
        }
        v3 ndu = unit(mk(nd[0], nd[1], nd[2]));
        o[0] = p[0]; o[1] = p[1]; o[2] = p[2];
        d[0] = ndu.x; d[1] = ndu.y; d[2] = ndu.z;
        prev = hit;
        if (sc->tau > 0) {
            double mt = maxc(T);
            if (fabs(mt - sc->tau) <= tau_margin(sc, &E) * sc->tau) *flags |= ORC_FLAG_TAU;
            NOTE_FLAGS(j);
            if (mt < sc->tau) { cnt[C_END_TAU]++; break; }
        }
        NOTE_FLAGS(j);
        if (j == sc->max_bounces) cnt[C_END_CAP]++;   /* the loop ends after this surface event */
    }
#undef NOTE_FLAGS
    *segs_out = segs;
    *path_flags |= pf;
}

/* Render the given rays (pixel indices, or explicit-ray indices).
 *   out_rgba[4*i]   : mean over spp of L (linear HDR), alpha = mean camera-segment opacity
 *   out_segments    : [n_ids * spp] segments per path (nullable)
 *   out_tri, out_t  : [n_ids * spp * max_bounces] hit triangle / distance per segment (nullable)
 *   out_flags       : [n_ids] OR of ambiguity flags over spp (nullable)
 *   out_first_flag  : [n_ids * spp] segment of each path's first ambiguity flag, 0 = none (nullable)
 *   out_counts      : [C_N] totals (nullable) */
int orc_render_ex(const orc_scene *sc, const uint32_t *ids, uint32_t n_ids, double *out_rgba, uint32_t *out_segments,
                  uint32_t *out_tri, double *out_t, uint32_t *out_flags, uint64_t *out_counts, int n_threads,
                  uint32_t *out_first_flag) {
    uint64_t tot[C_N] = {0};
#ifdef _OPENMP
    if (n_threads <= 0) n_threads = omp_get_max_threads();
#endif
    const uint32_t B = sc->max_bounces, S = sc->spp;
#pragma omp parallel num_threads(n_threads)
    {
        uint64_t cnt[C_N] = {0};
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < (int64_t)n_ids; ++i) {
            double acc[4] = {0, 0, 0, 0};
            uint32_t fl = 0;
            for (uint32_t s = 0; s < S; ++s) {
                double L[3], a0;
                uint32_t segs;
                uint64_t k = (uint64_t)i * S + s;
                uint32_t *tr = out_tri ? out_tri + k * B : NULL;
                double *tt = out_t ? out_t + k * B : NULL;
                if (tr) for (uint32_t j = 0; j < B; ++j) { tr[j] = ORC_NO_HIT; tt[j] = INFINITY; }
                uint32_t first;
                trace_path(sc, ids[i], s, L, &a0, &segs, tr, tt, &fl, &first, cnt);
                if (out_first_flag) out_first_flag[k] = first;
                for (int c = 0; c < 3; ++c) acc[c] += L[c];
                acc[3] += a0;
                if (out_segments) out_segments[k] = segs;
            }
            for (int c = 0; c < 4; ++c) out_rgba[4 * i + c] = acc[c] / S;
            if (out_flags) out_flags[i] = fl;
        }
#pragma omp critical
        for (int c = 0; c < C_N; ++c) tot[c] += cnt[c];
    }
    if (out_counts) for (int c = 0; c < C_N; ++c) out_counts[c] = tot[c];
    return 0;
}

int orc_render(const orc_scene *sc, const uint32_t *ids, uint32_t n_ids, double *out_rgba, uint32_t *out_segments,
               uint32_t *out_tri, double *out_t, uint32_t *out_flags, uint64_t *out_counts, int n_threads) {
    return orc_render_ex(sc, ids, n_ids, out_rgba, out_segments, out_tri, out_t, out_flags, out_counts, n_threads,
                         NULL);
}

/* Training pairs of the shadow-transmittance surrogate: pair i is a point p
 * uniform in the field box (uniforms u0..u2 of Philox4x64-10 with counter
 * (i, 0, 0, 0) and key (seed, 0x736861646F77), mapped through the field pose),
 * light l = floor(u3 n_lights) (clamped), a point y on it (the point light's
 * position, or for an area light the barycentrics (1 - sqrt(a), b sqrt(a),
 * rest) from the first two uniforms of counter (i, 1, 0, 0)), the direction
 * w = (y - p)/|y - p|, D = |y - p| and the label exp(-int_0^D sigma), the
 * transmittance the shadow ray of Sec. 3.1 marches.  out: n x 8 values
 * (p, w, D, label). */
void orc_shadow_pairs(const orc_scene *sc, uint64_t seed, uint64_t first, uint32_t n, double *out) {
    const uint64_t key[2] = {seed, 0x736861646F77ull};
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < (int64_t)n; ++k) {
        const uint64_t i = first + (uint64_t)k;
        uint64_t c0[4] = {i, 0, 0, 0}, r0[4], c1[4] = {i, 1, 0, 0}, r1[4];
        orc_philox4x64(c0, key, r0);
        orc_philox4x64(c1, key, r1);
        double pl[3], p[3];
        for (int a = 0; a < 3; ++a) pl[a] = sc->aabb_min[a] + u24(r0[a]) * ((double)sc->aabb_max[a] - sc->aabb_min[a]);
        if (sc->field_pose) {
            const float *M = sc->field_pose;
            for (int a = 0; a < 3; ++a) p[a] = M[4 * a] * pl[0] + M[4 * a + 1] * pl[1] + M[4 * a + 2] * pl[2] + M[4 * a + 3];
        } else {
            for (int a = 0; a < 3; ++a) p[a] = pl[a];
        }
        uint32_t l = (uint32_t)(u24(r0[3]) * sc->n_lights);
        if (l >= sc->n_lights) l = sc->n_lights - 1;
        v3 y;
        if (sc->light_kind && sc->light_kind[l] == ORC_LIGHT_AREA) {
            v3 a = fv(sc->light_pos + 3 * l), b = fv(sc->light_v1 + 3 * l), c = fv(sc->light_v2 + 3 * l);
            double su = sqrt(u24(r1[0])), b0 = 1.0 - su, b1 = u24(r1[1]) * su, b2 = 1.0 - b0 - b1;
            y = add(add(scl(a, b0), scl(b, b1)), scl(c, b2));
        } else {
            y = fv(sc->light_pos + 3 * l);
        }
        double w[3] = {y.x - p[0], y.y - p[1], y.z - p[2]};
        double D = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
        for (int a = 0; a < 3; ++a) w[a] /= D;
        uint64_t cnt[C_N] = {0};
        double T = orc_transmittance(sc, p, w, 0.0, D, cnt);
        double *o = out + 8 * (uint64_t)k;
        o[0] = p[0]; o[1] = p[1]; o[2] = p[2];
        o[3] = w[0]; o[4] = w[1]; o[5] = w[2];
        o[6] = D; o[7] = T;
    }
}

/* Tone map psi (Eq. 14 of the paper: linear radiance to sRGB for display,
 * applied after the path ends): scale by the exposure, clamp to [0, 1], then
 * the sRGB transfer function of IEC 61966-2-1. */
double orc_tonemap(double L, double exposure) {
    double c = L * exposure;
    if (c < 0.0) c = 0.0;
    if (c > 1.0) c = 1.0;
    return c <= 0.0031308 ? 12.92 * c : 1.055 * pow(c, 1.0 / 2.4) - 0.055;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
