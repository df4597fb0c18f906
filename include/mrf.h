/*
 * mrf.h - C ABI of the mesh-aware radiance-field renderer (GB300, sm_103a).
 *
 * The library renders the hybrid light-transport loop of "Dynamic Mesh-Aware
 * Radiance Fields" (Qiao, Gao et al., ICCV 2023), Sec. 3.1 "Hybrid Rendering
 * Algorithm" and its Algorithm 1: for every pixel a path alternates between
 * marching a radiance field along a straight segment (Eqs. 10-11) and a
 * surface event at a triangle mesh (Eqs. 12-13), with shadow rays toward the
 * lights whose transmittance comes from the same field march.
 *
 * Conventions shared by every entry point:
 *  - Every function returns an mrf_status; no C++ exception crosses the ABI.
 *    On failure a human-readable message is kept per thread: mrf_last_error().
 *  - Array arguments may live in host or device memory unless stated; the
 *    library finds out with cudaPointerGetAttributes.  Inputs of the create /
 *    build / set calls are copied into library-owned device memory, so the
 *    caller may free them as soon as the call returns.
 *  - Handles belong to the context (and its CUDA device) that made them; they
 *    are not thread-safe.  Destroy functions accept NULL.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Device work is enqueued on it and the call returns without
 *    waiting, except where noted (host output buffers, statistics).
 *  - Asynchronous device faults surface as MRF_ERR_CUDA from the next call.
 *    A kernel that gives up after its iteration budget sets the context's
 *    status word; a render call reports it as MRF_ERR_TIMEOUT without blocking
 *    the host (each call ends by copying the word to pinned host memory on its
 *    stream, and the next call reads that copy once it has landed), so the
 *    report may come one call late.  mrf_sync_status waits and reports at once.
 */
#ifndef MRF_H
#define MRF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum mrf_status {
    MRF_OK = 0,
    MRF_ERR_INVALID_ARG = 1,  /* bad pointer, size, enum value or mismatched handle */
    MRF_ERR_CUDA = 2,         /* a CUDA runtime call failed (message holds its text) */
    MRF_ERR_OOM = 3,          /* device allocation failed */
    MRF_ERR_TIMEOUT = 4,      /* a kernel gave up after its iteration budget */
    MRF_ERR_NOT_READY = 5,    /* handle not initialised */
    MRF_ERR_UNSUPPORTED = 6   /* feature not available on this device or build */
} mrf_status;

typedef struct mrf_context mrf_context;
typedef struct mrf_field mrf_field;
typedef struct mrf_shadow_net mrf_shadow_net;
typedef struct mrf_bvh mrf_bvh;

/* ---------------------------------------------------------------- context */
/* Binds the calling thread to CUDA device `device` and creates a context that
 * owns materials, lights, statistics counters and scratch memory.
 * MRF_ERR_INVALID_ARG if `out` is NULL or the device does not exist;
 * MRF_ERR_UNSUPPORTED if the device is not compute capability 10.3. */
mrf_status mrf_context_create(int device, mrf_context **out);
void mrf_context_destroy(mrf_context *ctx);
/* Thread-local text of the last failure (never NULL, "" if none). */
const char *mrf_last_error(void);
/* Library version as "major.minor.patch". */
const char *mrf_version(void);
/* The library's error channel (the paper has no counterpart).  Waits for all
 * work on the context's device (cudaDeviceSynchronize), then reads and clears
 * the context's status word.  MRF_ERR_CUDA for an asynchronous
 * CUDA error, MRF_ERR_TIMEOUT if a kernel gave up since the last report (its
 * bits in *status_word, nullable), else MRF_OK. */
mrf_status mrf_sync_status(mrf_context *ctx, uint32_t *status_word);

/* ------------------------------------------------------------------ field */
/* The radiance field: density sigma(p) and linear-HDR radiance r(p) on the
 * axis-aligned box [aabb_min, aabb_max] (sigma = 0 outside), the field of
 * Eq. 7 / Eq. 9 of the paper, trained there with HDR images (Sec. 3.1,
 * "Unifying color space").  Three kinds:
 *   CONST    : sigma = const_sigma, r = const_rgb.
 *   GAUSS    : sigma = sum_k peak_k exp(-|p - c_k|^2 / (2 radius_k^2)),
 *              r = sum_k sigma_k emission_k / sigma (emission-weighted mix).
 *   HASHGRID : the Instant-NGP field the paper renders (Sec. 3.3): a
 *              multiresolution hash encoding (n_levels levels, 2^log2_table_size
 *              entries of n_features FP16 values per level, per-level grid
 *              resolution level_res[l]; dense row-major indexing when
 *              (N_l + 1)^3 fits the table, else the spatial hash
 *              x ^ y*2654435761 ^ z*805459861 mod T; trilinear interpolation),
 *              feeding an MLP in -> width -> width -> 4 with ReLU hidden layers:
 *              sigma = support(p) * exp(min(o0, 15)), r = softplus(o1..3).
 *              support(p) = max_k max(0, 1 - |p - s_k|^2 / rs_k^2) over the
 *              support spheres gives the density its compact support.
 *              occ_bits is a conservative occupancy bitfield (occ_res^3 bits,
 *              cell x + R*(y + R*z), word i>>5 bit i&31) covering the support;
 *              the renderer skips samples in empty cells.  mrf_field_create
 *              checks the cover (every cell a support sphere reaches is set);
 *              when it holds, the wavefront sample walk tests the support
 *              only, otherwise it also tests every sample's cell.
 * Layouts: blob_center (n_blobs x 3), blob_emission (n_blobs x 3), table
 * [level][entry][feature] as IEEE binary16 bits, w1 (width x in) row-major,
 * w2 (width x width), w3 (4 x width), in = n_levels * n_features (<= 64),
 * width = 64.  `precision` selects the MLP arithmetic of the tensor-core
 * engine (MRF_PREC_FP16 / BF16 operands with FP32 accumulation); FP32 runs the
 * whole network in FP32 on the CUDA cores. */
enum { MRF_FIELD_CONST = 0, MRF_FIELD_GAUSS = 1, MRF_FIELD_HASHGRID = 2 };
enum { MRF_PREC_FP32 = 0, MRF_PREC_FP16 = 1, MRF_PREC_BF16 = 2 };

typedef struct mrf_field_desc {
    int32_t kind;
    float aabb_min[3], aabb_max[3];
    /* CONST */
    float const_sigma, const_rgb[3];
    /* GAUSS */
    uint32_t n_blobs;
    const float *blob_center, *blob_radius, *blob_peak, *blob_emission;
    /* HASHGRID */
    uint32_t n_levels, log2_table_size, n_features;
    const uint32_t *level_res;
    const uint16_t *table;
    uint32_t mlp_width;
    const float *w1, *b1, *w2, *b2, *w3, *b3;
    uint32_t n_support;
    const float *support_center, *support_radius;
    uint32_t occ_res;              /* 0 = no occupancy grid (every sample evaluated) */
    const uint32_t *occ_bits;
    int32_t precision;
    /* Rigid pose of the field: 3x4 row-major local-to-world [R | t] (NULL =
     * identity).  The paper moves NeRF objects with the simulator's transform
     * and queries them at t^-1 p (Sec. 3.2); the box, hash grid, occupancy and
     * support above are given in the field's local frame.  R must be a rotation
     * (orthonormal within 1e-4), else MRF_ERR_INVALID_ARG. */
    const float *pose;
    /* View-dependent radiance (the network layout of Instant-NGP, which the
     * paper renders with, Sec. 3.3): when non-zero, layer 1 (w1, b1) feeds a
     * density head wd2 (16 x 64), bd2 whose output 0 gives sigma, and a colour
     * network takes the 16 head outputs and the 16 real spherical harmonics of
     * the unit view direction in the field's frame (bands 0..3):
     * 32 -> 64 (wc1: 64 x 32, bc1) -> 64 (wc2, bc2) -> 3 (wc3: 3 x 64, bc3),
     * r = softplus.  w2, b2, w3, b3 may then be NULL; n_levels * n_features
     * must be 32.  FP32 runs on the CUDA cores (both engines); FP16/BF16 on the
     * tensor cores in the wavefront engine (five chained MMAs per tile).
     * mrf_field_query evaluates them for the view direction +z. */
    int32_t view_dependent;
    const float *wd2, *bd2, *wc1, *bc1, *wc2, *bc2, *wc3, *bc3;
} mrf_field_desc;

/* Copies the description into device memory.  MRF_ERR_INVALID_ARG for an
 * unknown kind, an empty box, n_levels * n_features > 64, mlp_width != 64,
 * occ_res not a multiple of 8 or > 1024, or a NULL array the kind needs. */
mrf_status mrf_field_create(mrf_context *ctx, const mrf_field_desc *desc, mrf_field **out);
void mrf_field_destroy(mrf_field *field);
/* Changes the MLP precision of an existing HASHGRID field. */
mrf_status mrf_field_set_precision(mrf_field *field, int32_t precision);

/* Evaluates sigma and r at n points (n x 3, FP32, in the field's local frame)
 * into out (n x 4: sigma, r, g, b)
 * in the field's precision: FP32 on the CUDA cores, or for FP16/BF16 hash
 * fields the tensor-core kernel the wavefront engine uses.  points and out must
 * be device pointers.  For tests of the field alone (Eq. 7 / hash encoding / MLP). */
mrf_status mrf_field_query(mrf_context *ctx, const mrf_field *field, const float *points, uint32_t n, float *out,
                           void *stream);

/* -------------------------------------------------------------------- BVH */
/* Builds a bounding-volume hierarchy over a triangle mesh for the ray-casting
 * function t(p, w) of Eq. 3 (the paper does not name its acceleration
 * structure; this one is a binned-SAH binary BVH built on the host, 64-byte
 * nodes holding both children's boxes, leaves of at most 4 triangles).  The
 * traversals walk a four-child copy of it (128-byte nodes holding a node's
 * grandchildren), which build, refit and rebuild rewrite on the GPU; the
 * statistics count the four-child nodes visited.
 * verts: n_verts x 3 FP32; tris: n_tris x 3 vertex indices; mat_id: n_tris
 * material indices into the table of mrf_materials_set.  Triangle ids reported
 * by the renderer are indices into `tris`.  n_tris may be 0 (no meshes).
 * MRF_ERR_INVALID_ARG for an index >= n_verts or a NULL array with n > 0. */
mrf_status mrf_bvh_build(mrf_context *ctx, const float *verts, uint32_t n_verts, const uint32_t *tris,
                         const uint32_t *mat_id, uint32_t n_tris, mrf_bvh **out);
/* Refits the BVH boxes to moved vertices (same topology; the dynamic meshes of
 * Sec. 3.2 change their vertices every simulation step).  verts: n_verts x 3,
 * n_verts must equal the build's (else MRF_ERR_INVALID_ARG).  Runs on `stream`
 * (the boxes, then the four-child copy). */
mrf_status mrf_bvh_refit(mrf_bvh *bvh, const float *verts, uint32_t n_verts, void *stream);
/* Rebuild of the hierarchy on the GPU for new vertex positions (same
 * triangles, n_verts as at build; host or device array): a linear BVH over the
 * 30-bit Morton order of the triangle centroids (Karras, HPG 2012), one
 * triangle per leaf, enqueued on `stream` without host synchronisation (the
 * first call allocates room for n - 1 nodes and the sort buffers and waits).
 * For deforming meshes whose refitted boxes have grown loose: casts give the
 * same closest hits as with the original tree. */
mrf_status mrf_bvh_rebuild(mrf_bvh *bvh, const float *verts, uint32_t n_verts, void *stream);
void mrf_bvh_destroy(mrf_bvh *bvh);

/* Closest hit of n rays (origins, dirs: n x 3 FP32 device arrays; dirs need
 * not be unit) against the mesh: out_t (FP32, +inf on a miss) and out_tri
 * (0xFFFFFFFF on a miss), skipping triangle skip[i] if skip is non-NULL, with
 * t > tmin.  Same traversal as the renderer. */
mrf_status mrf_cast(mrf_context *ctx, const mrf_bvh *bvh, const float *origins, const float *dirs,
                    const uint32_t *skip, uint32_t n, float tmin, float *out_t, uint32_t *out_tri, void *stream);

/* -------------------------------------------------------- materials/lights */
/* BSDFs of the paper's Sec. 3.3: reflective (perfect mirror, T *= rgb),
 * refractive (smooth dielectric of index `ior`, exact unpolarised Fresnel
 * choice between reflection and Snell refraction, T unchanged) and Lambertian
 * (cosine-weighted sampling, T *= rgb albedo). */
enum { MRF_MAT_MIRROR = 0, MRF_MAT_GLASS = 1, MRF_MAT_DIFFUSE = 2 };
typedef struct mrf_material {
    int32_t kind;
    float rgb[3];
    float ior;
} mrf_material;
/* Lights for the shadow rays of Sec. 3.1 ("Shadow rays"), cast at diffuse hits.
 *
 * POINT: position `pos`, RGB intensity I in `intensity`.  A diffuse hit at
 * distance D receives (albedo / pi) cos I / D^2 times the mesh visibility and
 * the field transmittance exp(-int sigma) along the shadow ray (Eq. 10).
 *
 * AREA: the triangle (pos, v1, v2) of an estimated emitter mesh (Sec. 3.1,
 * "Estimating light sources": the faces left after pruning the emission
 * texture), emitting RGB radiance Le (`intensity`) from its front side, whose
 * normal is (v1 - pos) x (v2 - pos).  Each diffuse hit casts `samples` shadow
 * rays (1..64) to points drawn uniformly on the triangle and adds
 *   (albedo / pi) Le A / samples * sum_s V_s T_s cos_x cos_y / D_s^2,
 * with A the triangle's area and cos_y the cosine at the emitter.  The points
 * come from Philox4x64-10 with counter (ray, spp, segment, 1 + q), key
 * (seed, 0), where q counts the area-light samples of the hit in light order;
 * uniforms are the top 24 bits of words 0 and 1, and the point has
 * barycentrics (1 - sqrt(u0), u1 sqrt(u0), rest) (Shirley and Turk's warp).
 * Emitters are seen only by shadow rays: camera and bounce rays pass through
 * them (the field already holds the scene's appearance).
 *
 * One diffuse hit casts at most 64 shadow rays in all (point lights count
 * one each) on the wavefront engine. */
enum { MRF_LIGHT_POINT = 0, MRF_LIGHT_AREA = 1 };
typedef struct mrf_light {
    int32_t kind;
    float pos[3];          /* POINT: position; AREA: vertex v0 */
    float intensity[3];    /* POINT: intensity I; AREA: radiance Le of the front side */
    float v1[3], v2[3];    /* AREA only */
    uint32_t samples;      /* AREA only: shadow rays per diffuse hit */
    float mask_strength;   /* r_src of the field-sample shadow mask, in [0, 1] (see mrf_render_opts) */
} mrf_light;
/* Replace the context's material / light tables (host or device arrays, n <= 65535). */
mrf_status mrf_materials_set(mrf_context *ctx, const mrf_material *mats, uint32_t n);
mrf_status mrf_lights_set(mrf_context *ctx, const mrf_light *lights, uint32_t n);

/* ----------------------------------------------------------------- render */
/* Pinhole camera: ray from `pos` through the centre of pixel (x, y), row 0 at
 * the top; vfov_deg is the full vertical field of view. */
typedef struct mrf_camera {
    float pos[3], look_at[3], up[3];
    float vfov_deg;
    uint32_t width, height;
} mrf_camera;

/* The primary rays: a camera (count = width * height, ray index = y * width + x),
 * several cameras rendered as one batch, or explicit FP32 origins / directions
 * (count x 3, host or device).
 *
 * Several views (n_cameras > 1): `camera` points to n_cameras host records and
 * the rays are numbered view by view, each view row-major, so view k starts at
 * ray sum_{j<k} width_j * height_j and out_hdr holds the images one after the
 * other.  The views may differ in size, position and field of view; all of
 * them go through one launch sequence.  Alg. 1 renders every pixel
 * independently, so batching views changes nothing but the ray index, which is
 * also the index the random numbers are drawn with.  n_cameras 0 or 1 means
 * one camera; at most 65,536 views.  mrf_render only: mrf_render_static takes
 * one camera or explicit rays. */
typedef struct mrf_rays {
    const mrf_camera *camera;
    const float *origins, *dirs;
    uint32_t count;
    uint32_t spp;                  /* paths per ray (>= 1) */
    uint32_t n_cameras;            /* records behind `camera` (0 = 1) */
} mrf_rays;

/* MEGAKERNEL: one thread runs a whole path (FP32 field only).  WAVEFRONT: one
 * launch sequence per segment over all live paths, with every field sample of
 * the segment evaluated in one flat pass (tensor cores for FP16/BF16 hash
 * fields).  AUTO picks WAVEFRONT for FP16/BF16 hash fields, else MEGAKERNEL. */
enum { MRF_ENGINE_AUTO = 0, MRF_ENGINE_MEGAKERNEL = 1, MRF_ENGINE_WAVEFRONT = 2 };
/* kernel kinds of the per-kernel timing in mrf_render_opts.kernel_ms */
enum {
    MRF_KERNEL_MEGAKERNEL = 0, MRF_KERNEL_CAST_GEN = 1, MRF_KERNEL_FIELD = 2, MRF_KERNEL_SHADE = 3,
    MRF_KERNEL_FINALIZE = 4, MRF_KERNEL_GEN = 5, MRF_KERNEL_COMPOSITE = 6, MRF_KERNEL_SHADOW_NET = 7,
    MRF_KERNEL_SHADOW_VIS = 8, MRF_KERNEL_OVERFLOW = 9, MRF_KERNEL_MASK = 10, MRF_KERNEL_TAIL = 11,
    MRF_KERNEL_COUNT = 12
};

typedef struct mrf_render_opts {
    uint64_t seed;                 /* Philox4x64-10 key word 0 */
    uint32_t steps_per_segment;    /* > 0: that many midpoint samples per segment */
    float dt;                      /* steps_per_segment == 0: fixed step, last interval clipped */
    float tau;                     /* end a path when max(T) < tau (0 = never) */
    float tmin;                    /* smallest accepted ray-triangle distance */
    int32_t engine;                /* MRF_ENGINE_* */
    /* optional per-path records, device pointers or NULL:
     * rec_segments[count * spp], rec_tri / rec_t[count * spp * max_bounces] */
    uint32_t *rec_segments;
    uint32_t *rec_tri;
    float *rec_t;
    /* optional host arrays of MRF_KERNEL_COUNT entries: summed CUDA-event
     * duration (ms) and launch count of each kernel kind; when set, the call
     * records events around every launch on `stream` and waits for them */
    float *kernel_ms;
    uint32_t *kernel_launches;
    /* learned shadow transmittance (see mrf_shadow_net_create), or NULL: shadow
     * rays leaving a point inside the field box take T from the network instead
     * of marching the field; the rest are marched */
    const mrf_shadow_net *shadow_net;
    /* shadow mask m(p_t) of Sec. 3.1 on the field's samples (0 = off): a ray
     * from every field sample with sigma > 0 toward each light with
     * mask_strength r > 0 (a point light's position, an area light's centroid);
     * each light a mesh blocks scales the sample's radiance by 1 - r, so
     * L += T alpha m r(p).  The density and throughput are unchanged. */
    int32_t shadow_mask;
} mrf_render_opts;

typedef struct mrf_stats {
    uint64_t paths, segments, surface_hits, shadow_rays;
    uint64_t samples_nominal;      /* quadrature samples on all marched segments */
    uint64_t samples_evaluated;    /* samples in occupied cells (field network run) */
    uint64_t shadow_samples_evaluated;
    uint64_t fp64_retests;         /* near-edge triangle tests redone in FP64 */
    uint64_t status;               /* device status word (0 = ok); bits: 1 BVH traversal stack overflow,
                                      2 a segment of more than 2^24 samples, 4 a tensor-core wait gave
                                      up, 8 the self-test wait gave up, 0x100 a bad index (bounds-checked
                                      build) */
    uint64_t shadow_net_evals;     /* shadow rays answered by the shadow network */
    uint64_t ended_miss, ended_tau, ended_cap;   /* paths that left the scene, fell below tau, hit the bounce cap */
    uint64_t bvh_nodes;            /* four-child BVH nodes visited (closest-hit, shadow and mask rays) */
    uint64_t bvh_tri_tests;        /* ray-triangle tests made by those traversals */
    uint64_t bvh_worst_nodes;      /* nodes visited by the longest closest-hit traversal */
    uint64_t bvh_worst_path;       /* the path (ray * spp + sample) that made it */
} mrf_stats;

/* Renders every path of `rays` (Algorithm 1) with at most max_bounces
 * segments per path (the camera segment counts as the first), writing
 * out_hdr[4 * i + c] = mean over spp of the linear-HDR radiance L (c < 3) and
 * the camera segment's field opacity (c = 3).  out_hdr is count x 4 FP32; if
 * it is host memory the call copies the image back and waits.  If `stats` is
 * non-NULL the call waits and fills it.  MRF_ERR_INVALID_ARG for NULL
 * handles, count == 0, spp == 0, max_bounces == 0 or > 64, or records with a
 * host pointer. */
mrf_status mrf_render(mrf_context *ctx, const mrf_field *field, const mrf_bvh *bvh, const mrf_rays *rays,
                      uint32_t max_bounces, const mrf_render_opts *opts, float *out_hdr, void *stream,
                      mrf_stats *stats);

/* Tone map psi of the paper (Eq. 14, applied after the path ends): per pixel
 * and colour channel out = sRGB(clamp(exposure * L, 0, 1)), the transfer
 * function of IEC 61966-2-1; alpha is copied.  in and out are n x 4 FP32
 * device arrays (they may alias). */
mrf_status mrf_tonemap(mrf_context *ctx, const float *in, uint32_t n, float exposure, float *out, void *stream);

/* Allocation-free variant of mrf_render.  The paper has no counterpart: this
 * entry point exists for embedders that cannot call cudaMalloc while they
 * render, such as hosts whose device memory belongs to another allocator's
 * pool, or real-time loops that cannot afford the device-wide synchronisation
 * an allocation may cause.  It runs the wavefront engine out of a file-scope
 * device arena of 64 MiB that every GPU loading the library holds until the
 * process exits, and it allocates no device or pinned memory itself.
 *  - Limits: rays->count * rays->spp <= 131072 paths, at most 8 shadow rays per
 *    hit (K), and the per-path state, about (172 + 48 max(K, 1)) bytes a path,
 *    must leave the arena room for at least one 128-sample tile: at K = 8 that
 *    allows about 120,000 paths, at K <= 7 the full 131072.  Larger requests
 *    return MRF_ERR_INVALID_ARG naming the limit (use mrf_render).
 *  - Samples that do not fit the arena's sample buffer are left for the next
 *    generation round (mrf_tuning.rounds); with enough rounds the image is
 *    mrf_render's bit for bit.  Jobs still pending after the last round are
 *    marched in place on the CUDA cores in FP32, so at FP16/BF16 their pixels
 *    differ from mrf_render's by up to the reduced-precision error.
 *  - out_hdr, explicit rays and records must be device memory; per-kernel
 *    timing (kernel_ms, kernel_launches) is rejected.
 *  - The arena's device address is resolved (cudaGetSymbolAddress) once per
 *    context, by mrf_context_create with the context's device current.
 *  - Without `stats` the call does not block the host: a kernel that gave up
 *    is reported by a later call or by mrf_sync_status.
 *  - All calls share the arena, which keeps the last call's contents; the
 *    engine clears its counters at the start of every call.  Calls that overlap
 *    on the GPU (for example on two streams) race on the arena.
 * Arguments, outputs and statistics otherwise as mrf_render. */
mrf_status mrf_render_static(mrf_context *ctx, const mrf_field *field, const mrf_bvh *bvh, const mrf_rays *rays,
                             uint32_t max_bounces, const mrf_render_opts *opts, float *out_hdr, void *stream,
                             mrf_stats *stats);

/* ------------------------------------------------------------------ tuning
 * Launch shapes and queue sizes of the wavefront engine, kept per context
 * and used by every later render call of the context.  The paper names no
 * such parameters; results do not depend on them (only speed and memory). */
typedef struct mrf_tuning {
    uint32_t field_groups;       /* 128-sample tiles in flight per CTA of the tensor-core field kernel:
                                    8 (one CTA per SM, all TMEM) or 4 (two CTAs per SM), the layers' A
                                    operands in shared memory; or 5 (one CTA per SM) with every A operand
                                    in tensor memory (view-dependent fields then use 8); default 8 */
    uint32_t samples_per_path;   /* sample-buffer capacity per path (plus 4 Mi samples); 16..4096, default 96 */
    uint32_t rounds;             /* sample-generation rounds per segment, 1..16, default 1: the paths whose
                                    samples did not fit the buffer go to the next round; those left after
                                    the last round are marched in place on the CUDA cores in FP32 */
    uint32_t tail_paths;         /* persistent tail, 0..2^20, default 0 (off): once at most this many paths
                                    are live at the start of a segment (from the second on), one persistent
                                    kernel finishes all of them, a warp per path, instead of the per-segment
                                    launches; its field samples run on the CUDA cores with the FP32 weights
                                    (for an FP32 field the image is the same bit for bit) */
} mrf_tuning;
mrf_status mrf_tuning_get(const mrf_context *ctx, mrf_tuning *out);
mrf_status mrf_tuning_set(mrf_context *ctx, const mrf_tuning *t);
/* Autotuner: renders the given request (arguments as mrf_render, device
 * out_hdr) with every candidate, field_groups in {8, 4} x samples_per_path in
 * {48, 96, 192} x rounds in {1, 8}, times `reps` frames of each with CUDA
 * events on `stream` after one warm-up frame, keeps the fastest in the
 * context and returns it in `best` (nullable); `ms` (nullable) receives the
 * mean frame time of the twelve candidates in that order. */
mrf_status mrf_autotune(mrf_context *ctx, const mrf_field *field, const mrf_bvh *bvh, const mrf_rays *rays,
                        uint32_t max_bounces, const mrf_render_opts *opts, float *out_hdr, void *stream, uint32_t reps,
                        mrf_tuning *best, float *ms);

/* --------------------------------------------------------- captured frames
 * One render call captured once into a CUDA graph and replayed: every launch
 * of a frame (Algorithm 1 over all paths) goes to the GPU as one graph, with
 * no per-launch host work.  For sequences whose camera and outputs stay put
 * while the scene's contents change (a BVH refit per frame for deforming
 * meshes, new ray origins in the same arrays, a shadow network in training).
 *  - The graph keeps the device addresses seen at capture: out_hdr, explicit
 *    ray arrays, records, and the field's, BVH's and shadow network's memory.
 *    Their contents are read at every replay.
 *  - Camera records, materials and lights are copied at capture; later
 *    mrf_materials_set / mrf_lights_set calls do not change the frame.
 *  - The frame owns its scratch memory and statistics.  Replays of one frame
 *    must not overlap on the GPU.
 *  - MRF_ERR_INVALID_ARG for a host out_hdr, host explicit rays or per-kernel
 *    timing; other arguments as mrf_render.
 * mrf_frame_stats waits for `stream` and returns the last replay's
 * statistics. */
typedef struct mrf_frame mrf_frame;
mrf_status mrf_frame_capture(mrf_context *ctx, const mrf_field *field, const mrf_bvh *bvh, const mrf_rays *rays,
                             uint32_t max_bounces, const mrf_render_opts *opts, float *out_hdr, mrf_frame **out);
mrf_status mrf_frame_replay(mrf_frame *frame, void *stream);
mrf_status mrf_frame_stats(mrf_frame *frame, void *stream, mrf_stats *stats);
void mrf_frame_destroy(mrf_frame *frame);

/* ------------------------------------------ learned shadow transmittance
 * A small network stands in for the field march of a shadow ray (Sec. 3.1,
 * "Shadow rays": the transmittance exp(-int sigma) from a shading point toward
 * a light).  It is trained on the GPU by this library's own kernels on pairs
 * whose targets come from the plain FP32 march, which stays the fallback and
 * the reference the network's error is measured against.
 *  - Input: the point in the field's local frame, scaled to [0,1]^3 by the
 *    field box and clamped, encoded by a hash grid of 8 levels of 2 FP32
 *    features (resolution level_res[l]; 2^log2_table entries per level; dense
 *    index x + (N+1)(y + (N+1) z) when (N+1)^3 fits, else the spatial hash
 *    x ^ 2654435761 y ^ 805459861 z modulo the table size), followed by the
 *    16 real spherical harmonics of bands 0..3 of the unit direction to the
 *    light (in the local frame).
 *  - Network: 32 -> 64 ReLU -> 64 ReLU -> 64 ReLU -> 1, T = sigmoid(z).
 *  - Loss: mean squared error against the marched transmittance; Adam
 *    (Kingma and Ba) with bias correction over every parameter.
 *  - Parameters, one flat FP32 vector of mrf_shadow_net_param_count() values:
 *    the table (level-major, entry-major, 2 features), W1 (64 x 32 row-major),
 *    b1 (64), W2 (64 x 64), b2, W3 (64 x 64), b3, W4 (64), b4 (1).
 * The network answers shadow rays from points inside the field box; rays from
 * other points keep the march.  Handles are not thread-safe. */
typedef struct mrf_shadow_net_desc {
    uint32_t log2_table;       /* 10..22 */
    uint32_t level_res[8];     /* 2..4096 each */
    const float *params;       /* initial parameters (host or device), NULL = seeded default */
    uint64_t seed;             /* default initialisation: table U(-1e-4, 1e-4), Xavier-uniform W, zero b */
    float lr, beta1, beta2, eps;  /* Adam */
    int32_t precision;         /* weights used when rendering: MRF_PREC_FP32 or MRF_PREC_BF16 (the table stays FP32) */
    float lr_decay;            /* step t (from 1) uses lr * lr_decay^(t-1); 0 means 1 (constant) */
} mrf_shadow_net_desc;

/* The network belongs to `field`'s frame and box (copied at creation). */
mrf_status mrf_shadow_net_create(mrf_context *ctx, const mrf_field *field, const mrf_shadow_net_desc *desc,
                                 mrf_shadow_net **out);
void mrf_shadow_net_destroy(mrf_shadow_net *net);
uint64_t mrf_shadow_net_param_count(const mrf_shadow_net *net);
/* Copy the FP32 parameters out / in (host or device arrays); setting them
 * clears Adam's moments and step count. */
mrf_status mrf_shadow_net_get_params(const mrf_shadow_net *net, float *out, void *stream);
mrf_status mrf_shadow_net_set_params(mrf_shadow_net *net, const float *in, void *stream);

/* Training pairs first..first+n-1 for the context's lights, written to the
 * device array out (n x 8 FP32: point p, unit direction w, distance D, label).
 * Pair i: Philox4x64-10 with key (seed, 0x736861646F77); counter (i, 0, 0, 0)
 * gives the point uniformly in the field box (top 24 bits of words 0..2,
 * mapped through the field pose) and the light floor(u3 n_lights); for an
 * area light, counter (i, 1, 0, 0) gives the point on the triangle as in the
 * renderer.  The label is exp(-int_0^D sigma) by the FP32 march of the
 * renderer (step rule from opts: steps_per_segment or dt).  Needs >= 1 light. */
mrf_status mrf_shadow_pairs(mrf_context *ctx, const mrf_field *field, const mrf_render_opts *opts, uint64_t seed,
                            uint64_t first, uint32_t n, float *out, void *stream);

/* Loss and gradient of the network over the n pairs (device, n x 8), in FP32:
 * grad (device, mrf_shadow_net_param_count() values) and loss (device, 1
 * value) are overwritten.  The parameters are not changed. */
mrf_status mrf_shadow_net_grad(mrf_shadow_net *net, const float *pairs, uint32_t n, float *grad, float *loss,
                               void *stream);

/* `steps` Adam steps on batches of `batch` consecutive pairs of the device
 * array pairs (n_pairs x 8, taken cyclically from where the last call
 * stopped); loss (device, `steps` values, nullable) receives each batch's loss
 * before its update. */
mrf_status mrf_shadow_net_train(mrf_shadow_net *net, const float *pairs, uint64_t n_pairs, uint32_t batch,
                                uint32_t steps, float *loss, void *stream);

/* Checkpoint of a network in training: parameters, Adam's moments and step
 * count, the training-pair cursor and the optimiser settings, to a binary
 * file (a header then three arrays of mrf_shadow_net_param_count() FP32
 * values); loading requires the same table size and level resolutions and
 * resumes training where the saved network stopped.  Both wait for the
 * device. */
mrf_status mrf_shadow_net_save(const mrf_shadow_net *net, const char *path);
mrf_status mrf_shadow_net_load(mrf_shadow_net *net, const char *path);

/* Network transmittance for the n pairs (device, n x 8; p and w are read) into
 * the device array out (n values), with the rendering weights. */
mrf_status mrf_shadow_net_eval(mrf_shadow_net *net, const float *pairs, uint32_t n, float *out, void *stream);

/* ----------------------------------------------------------- diagnostics
 * The paper has no counterpart.  mrf_l2_read_bandwidth measures the L2 read
 * bandwidth the field kernel's table gathers are compared with: it fills
 * `bytes` of the context's scratch memory (a multiple of 16 in [1 MiB,
 * 256 MiB]; allocated or grown if needed), reads it once to make it resident,
 * then times `reps` (1..1000) passes of 16-byte loads that bypass L1 with
 * CUDA events on `stream`, waits, and stores bytes * reps / time in GB/s in
 * *gbs.  A buffer larger than the L2 measures DRAM instead. */
mrf_status mrf_l2_read_bandwidth(mrf_context *ctx, uint64_t bytes, uint32_t reps, void *stream, double *gbs);

/* ------------------------------------------------------------ self tests
 * Failure paths exercised without faulting the GPU.  Every wait of the
 * library's kernels (mbarrier waits on tensor-core work) is bounded; a wait
 * that gives up sets a bit of the context's status word and its kernel
 * returns, and the next call reports MRF_ERR_TIMEOUT.
 * mrf_selftest_timeout runs one such wait on a barrier that nothing arrives
 * at, with a budget of `cycles` SM cycles (at most 2^32).  With `wait` it
 * waits for the device, returns MRF_ERR_TIMEOUT and clears the status word;
 * without, it returns MRF_OK at once and the give-up is reported like any
 * other: by the next render call or mrf_sync_status.  The context stays usable.
 * mrf_debug_fail_allocations makes the library's next n device allocations
 * fail as if the device were out of memory (MRF_ERR_OOM); 0 turns it off. */
mrf_status mrf_selftest_timeout(mrf_context *ctx, uint64_t cycles, int32_t wait);
void mrf_debug_fail_allocations(uint32_t n);

#ifdef __cplusplus
}
#endif
#endif /* MRF_H */
