// Internal structures shared by the host side of the C ABI and the kernels.
// Everything a kernel reads is reached through plain device pointers held in
// these structs, which are passed by value as kernel parameters.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "mrf.h"

namespace mrf {

constexpr uint32_t kNoHit = 0xFFFFFFFFu;
constexpr int kMaxLevels = 32;
constexpr int kMlpWidth = 64;
constexpr int kMaxIn = 64;
constexpr int kMaxBounces = 64;
constexpr int kWideStackSize = 96;   // traversal stack of the wide BVH (up to three pushes per step)

// Packed FP32 MLP weights (floats):  W1T[in][64] | b1[64] | W2[64][64] | b2[64] | W3T[64][4] | b3[4]
__host__ __device__ constexpr int mlp_floats(int n_in) { return n_in * 64 + 64 + 64 * 64 + 64 + 64 * 4 + 4; }
// View-dependent heads appended after it (floats): WdT[64][16] bd[16] | Wc1T[32][64] bc1[64] |
// Wc2[64][64] bc2[64] | Wc3T[64][4] bc3[4]
constexpr int kViewFloats = 64 * 16 + 16 + 32 * 64 + 64 + 64 * 64 + 64 + 64 * 4 + 4;

struct FieldDev {
    int kind;
    float lo[3], hi[3], ext_inv[3];
    float const_sigma, const_rgb[3];
    // GAUSS: blob_a = (cx, cy, cz, 1 / (2 r^2)), blob_b = (peak, e_r, e_g, e_b)
    int n_blobs;
    const float4 *blob_a, *blob_b;
    // HASHGRID
    int n_levels;
    uint32_t log2T;
    uint32_t res[kMaxLevels];
    uint32_t dense_mask;        // bit l set: level l indexed densely
    const uint32_t *table;      // [level][entry] binary16 pairs (feature 0 low half)
    int n_in;
    const float *mlp;           // packed FP32, see mlp_floats (+ kViewFloats when view_dep)
    int view_dep;               // view-dependent radiance (colour network of the view direction)
    // FP32 biases for the tensor-core kernels, read from the kernel-parameter
    // constant bank (uniform across the warp: no shared-memory loads).  Plain
    // network: b1[64] b2[64] b3[4]; view-dependent: b1[64] bd[16] bc1[64]
    // bc2[64] bc3[3] 0.
    float bias_c[212];
    const void *mlp_lp;         // [FP16 | BF16] copies of W1, W2, W3 (W3 padded to 16 rows) in the
                                // tensor-core operand layout, 64 * n_in * 2 + 10240 bytes each
    int n_support;
    const float4 *support;      // (cx, cy, cz, 1 / r^2)
    int occ_res;
    const uint32_t *occ;
    float occ_scale[3];         // occ_res / extent
    // coarse occupancy: one bit per 8^3 block of fine cells (bit set if any is occupied)
    int occ_coarse_res;         // occ_res / 8
    const uint32_t *occ_coarse;
    float occ_coarse_scale[3];  // occ_coarse_res / extent
    float occ_cell[3], occ_coarse_cell[3];  // cell widths (extent / resolution)
    // 1 when every occupancy cell a support sphere reaches is marked (checked on
    // the host at creation): a sample with positive support then always lies in
    // an occupied cell, and walks that test the support may skip the grid.
    int occ_covers_support;
    int precision;
    // rigid pose: world-to-local [R^T | -R^T t] applied to every marched ray
    int has_pose;
    float to_local[12];
    unsigned *status;           // the context's status word (bounds-checked builds report here)
};

// BVH node: 4 x float4 = both children's boxes + (left, right, left_count, right_count).
// count > 0: leaf child whose triangles are [index, index + count) of `tris`.
struct BvhDev {
    const float4 *nodes;
    const float4 *wide;         // four-child copy (8 float4 per node), what the traversals walk
    const float4 *tris;         // 3 x float4 per triangle: (v0, id) (v1, material) (v2, 0)
    int n_nodes;
    int n_tris;
    unsigned *status;           // the context's status word (bounds-checked builds report here)
};

// Bounds-checked builds (-DMRF_BOUNDS_CHECK, libmrf_checked.so) test every
// table, node and triangle index before the access; a bad index sets `bit` in
// the status word and is replaced by 0, so the access stays in bounds and the
// next call reports MRF_ERR_TIMEOUT-class status.  Release builds compile the
// check away.
constexpr unsigned kStatusBadIndex = 0x100u;
#ifdef __CUDACC__
__device__ __forceinline__ uint32_t checked_index(uint32_t i, uint64_t n, unsigned *status) {
#ifdef MRF_BOUNDS_CHECK
    if ((uint64_t)i >= n) {
        if (status) atomicOr(status, kStatusBadIndex);
        return 0u;
    }
#else
    (void)n;
    (void)status;
#endif
    return i;
}
#endif

struct MaterialDev {
    int kind;
    float rgb[3];
    float ior;
};

// A light: point (pos, I) or triangle emitter (v0 = pos, v1, v2, radiance I,
// unit front normal n, area A, `samples` shadow rays per hit whose random
// numbers use counters 1 + q0 .. q0 + samples).
struct LightDev {
    float pos[3];
    float I[3];
    float v1[3], v2[3];
    float n[3];
    float area;
    int kind;
    uint32_t samples;
    uint32_t q0;
    uint32_t slot0;     // index of the light's first shadow ray among the hit's rays
    float mask;         // r_src of the field-sample shadow mask
    float target[3];    // point the shadow-mask rays aim at (position or centroid)
};

// FP32 weights the CUDA-core field kernels stage in shared memory
inline __host__ __device__ int field_mlp_floats(const FieldDev &F) {
    return mlp_floats(F.n_in) + (F.view_dep ? kViewFloats : 0);
}

// device statistics counters (unsigned long long), in this order
enum StatIndex {
    ST_PATHS = 0, ST_SEGMENTS, ST_HITS, ST_SHADOW, ST_NOMINAL, ST_EVALUATED, ST_SHADOW_EVALUATED, ST_FP64,
    ST_STATUS, ST_NET, ST_END_MISS, ST_END_TAU, ST_END_CAP, ST_NODES, ST_TRIS, ST_WORST, ST_COUNT
};

// Shadow-transmittance network (shadow_net.cu): 8-level hash grid of the point
// + 16 spherical harmonics of the direction -> 64 -> 64 -> 64 -> 1, sigmoid.
constexpr int kSnetLevels = 8;
constexpr int kSnetIn = 32;
constexpr int kSnetW = 64;
// MLP part of the flat parameter vector: W1[64][32] b1 W2[64][64] b2 W3[64][64] b3 W4[64] b4
constexpr int kSnetMlp = kSnetW * kSnetIn + kSnetW + 2 * (kSnetW * kSnetW + kSnetW) + kSnetW + 1;
constexpr int kSnetOffB1 = kSnetW * kSnetIn, kSnetOffW2 = kSnetOffB1 + kSnetW, kSnetOffB2 = kSnetOffW2 + kSnetW * kSnetW,
              kSnetOffW3 = kSnetOffB2 + kSnetW, kSnetOffB3 = kSnetOffW3 + kSnetW * kSnetW,
              kSnetOffW4 = kSnetOffB3 + kSnetW, kSnetOffB4 = kSnetOffW4 + kSnetW;

struct ShadowNetDev {
    uint32_t log2T;
    uint32_t res[kSnetLevels];
    uint32_t dense_mask;
    float lo[3], hi[3], ext_inv[3];     // field box, local frame
    int has_pose;
    float to_local[12];                 // world-to-local [R^T | -R^T t]
    const float *table;                 // FP32, [level][entry][2]
    const float *mlp;                   // rendering copy of the MLP part (BF16-rounded for BF16)
    const uint8_t *lp;                  // BF16 weights in the tensor-core operand layout (BF16 networks), or NULL
};

// One pinhole view of a multi-view batch: orthonormal basis in FP32 (built in
// FP64 on the host) and the index of its first ray.
struct ViewDev {
    float pos[3], f[3], r[3], u[3];
    float tan_half, aspect;
    uint32_t W, H, offset, pad;
};

struct RenderParams {
    FieldDev F;
    BvhDev B;
    const MaterialDev *mats;
    int n_mats;
    const LightDev *lights;
    int n_lights;
    int n_shadow;                // shadow rays per diffuse hit (point lights 1, area lights `samples`)
    int use_camera;
    float cam_pos[3], cam_f[3], cam_r[3], cam_u[3];
    float tan_half, aspect;
    uint32_t W, H;
    const ViewDev *views;        // multi-view batch (device), n_views > 1; else NULL
    uint32_t n_views;
    const float *ray_o, *ray_d;
    uint32_t count, spp, max_bounces;
    uint64_t seed;
    uint32_t steps;
    float dt, tau, tmin;
    float *out;
    uint32_t *rec_seg, *rec_tri;
    float *rec_t;
    unsigned long long *stats;   // nullable statistics counters
    unsigned *status;            // context status word: bits set when a kernel gave up
    int shadow_mask;             // field samples blocked from a light emit (1 - r_src) r
    int tc_groups;               // tuning: tile groups per CTA of the tensor-core field kernel (4 or 8)
    uint32_t cap_per_path;       // tuning: sample-buffer capacity per path
    int max_rounds;              // tuning: sample-generation rounds per segment
    uint32_t tail_paths;         // tuning: live paths at which the persistent tail takes over (0: never)
    int has_snet;                // shadow rays from inside the field box use the network
    ShadowNetDev snet;
};

// Optional per-launch CUDA-event timing of the renderer's kernels (host side).
struct KernelTimer {
    static constexpr int kMax = 4096;   // launches of one call (16 segments x 16 rounds fit)
    cudaEvent_t ev[2 * kMax];
    int kind[kMax];
    int n = 0;
    bool ok = true;
    void begin(int k, cudaStream_t s) {
        if (n >= kMax) { ok = false; return; }
        kind[n] = k;
        cudaEventRecord(ev[2 * n], s);
    }
    void end(cudaStream_t s) {
        if (n >= kMax) return;
        cudaEventRecord(ev[2 * n + 1], s);
        ++n;
    }
};
inline void timer_begin(KernelTimer *t, int kind, cudaStream_t s) { if (t) t->begin(kind, s); }
inline void timer_end(KernelTimer *t, cudaStream_t s) { if (t) t->end(s); }

// launchers (render_mega.cu)
cudaError_t launch_render_megakernel(const RenderParams &P, cudaStream_t s, KernelTimer *timer = nullptr);
// Field kernels: point i is pts[stride * i .. + 2].  With stride 4 the fourth
// float is the quadrature interval delta of the sample and out[i].x is its
// optical depth sigma * delta (FP32 product); with stride 3, out[i].x is sigma.
// out[i].yzw is the radiance.
cudaError_t launch_field_simt(const FieldDev &F, const float *pts, int stride, const uint32_t *n_dev, uint32_t n_host,
                              float4 *out, int grid, cudaStream_t s, const float4 *dirs = nullptr);
// field_tc.cu
cudaError_t launch_field_tc(const FieldDev &F, bool bf16, const float *pts, int stride, const uint32_t *n_dev,
                            uint32_t n_host, float4 *out, unsigned *status, int grid, cudaStream_t s, int groups = 8);
int field_tc_blocks_per_sm(int groups = 8);
cudaError_t launch_field_tc_view(const FieldDev &F, bool bf16, const float *pts, int stride, const float4 *dirs,
                                 const uint32_t *n_dev, uint32_t n_host, float4 *out, unsigned *status, int grid,
                                 cudaStream_t s, int groups = 8);
cudaError_t launch_cast(const BvhDev &B, const float *o, const float *d, const uint32_t *skip, uint32_t n, float tmin,
                        float *out_t, uint32_t *out_tri, unsigned long long *stats, cudaStream_t s);
cudaError_t launch_tonemap(const float4 *in, uint32_t n, float exposure, float4 *out, cudaStream_t s);
cudaError_t launch_selftest_timeout(long long cycles, unsigned *status, cudaStream_t s);
// the L2 read-bandwidth kernels: fill and warm the buffer, then `reps` passes of reads
cudaError_t launch_l2_fill(void *buf, size_t bytes, float *sink, cudaStream_t s);
cudaError_t launch_l2_read(const void *buf, size_t bytes, int reps, float *sink, cudaStream_t s);
// shadow_net.cu
size_t snet_train_smem();
cudaError_t launch_snet_pairs(const RenderParams &P, uint64_t seed, uint64_t first, uint32_t n, float *out,
                              cudaStream_t s);
cudaError_t launch_snet_grad(const ShadowNetDev &N, const float *params, unsigned long long *gacc, const float *pairs,
                             uint64_t n_pairs, uint64_t b0, uint32_t B, float *loss, cudaStream_t s);
cudaError_t launch_snet_adam(float *p, float *m, float *v, unsigned long long *g, uint64_t n, float lr, float b1,
                             float b2, float eps, double c1, double c2, cudaStream_t s);
cudaError_t launch_snet_grad_out(unsigned long long *g, float *out, uint64_t n, cudaStream_t s);
cudaError_t launch_snet_refresh(const float *mlp, float *out, bool bf16, cudaStream_t s);
cudaError_t launch_snet_eval(const ShadowNetDev &N, const float *pairs, uint32_t n, float *out, cudaStream_t s);
size_t snet_lp_bytes();
cudaError_t launch_snet_pack_lp(const float *mlp, uint8_t *lp, cudaStream_t s);
cudaError_t launch_snet_tc(const ShadowNetDev &N, const uint8_t *lp, const float *mlp, const uint32_t *queue,
                           const float4 *hp, const float4 *sdir, int K, const float *pairs, const uint32_t *n_dev,
                           uint32_t n_host, float *out, unsigned *status, unsigned long long *stats, cudaStream_t s);
// bvh_lbvh.cu
size_t bvh_rebuild_scratch_words(uint32_t n);
cudaError_t launch_bvh_rebuild(float4 *nodes, int *parent, int *counters, float4 *tris, uint32_t *order,
                               const uint32_t *tri_idx, const uint32_t *mat, const float *verts, uint32_t n,
                               uint32_t *scratch, cudaStream_t s);
// bvh_refit.cu
cudaError_t launch_bvh_refit(float4 *nodes, int n_nodes, float4 *tris, int n_tris, const uint32_t *tri_order,
                             const uint32_t *tri_idx, const float *verts, const int *parent, int *counters,
                             const int *leaf_parent_of_tri, cudaStream_t s);
// the wide copy of the BVH that traversals walk (8 float4 per binary node), from the binary nodes
cudaError_t launch_bvh_widen(const float4 *nodes, int n_nodes, float4 *wide, cudaStream_t s);

}  // namespace mrf
