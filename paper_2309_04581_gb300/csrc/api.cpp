// The C ABI of include/mrf.h: argument checks, device memory ownership and
// kernel dispatch.  No C++ exception crosses the boundary.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "common.h"

namespace mrf {
void bvh_build_host(const float *verts, const uint32_t *tris, uint32_t n_tris, std::vector<float> &nodes,
                    std::vector<uint32_t> &order, std::vector<int> &parent);
cudaError_t launch_render_wavefront(const RenderParams &P, void *scratch, size_t scratch_bytes, cudaStream_t s,
                                    KernelTimer *timer);
size_t wavefront_scratch_bytes(const RenderParams &P);
bool wavefront_available();
cudaError_t static_arena(void **ptr, size_t *bytes);
uint32_t static_arena_paths_that_fit(int n_shadow);
cudaError_t launch_render_wavefront_arena(const RenderParams &P, void *arena, size_t arena_bytes, cudaStream_t s);
uint32_t static_arena_max_paths();
int static_arena_max_lights();
}  // namespace mrf

using namespace mrf;

static thread_local std::string g_err;

static mrf_status fail(mrf_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

static mrf_status cuda_fail(cudaError_t e, const char *what) {
    cudaGetLastError();  // clear a sticky-free error so later calls start clean
    return fail(e == cudaErrorMemoryAllocation ? MRF_ERR_OOM : MRF_ERR_CUDA, "%s: %s (%s)", what,
                cudaGetErrorString(e), cudaGetErrorName(e));
}

#define CUDA_TRY(expr, what)                         \
    do {                                             \
        cudaError_t e_ = (expr);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

struct mrf_context {
    int device = 0;
    MaterialDev *mats = nullptr;
    int n_mats = 0;
    LightDev *lights = nullptr;
    int n_lights = 0;
    int n_shadow = 0;   // shadow rays per diffuse hit over all lights
    unsigned long long *stats = nullptr;
    unsigned *status = nullptr;  // device status word: non-zero after a kernel gave up
    unsigned *status_host = nullptr;   // pinned copy of the status word, written at the end of render calls
    cudaEvent_t status_ev = nullptr;   // completes when that copy has landed
    bool status_pending = false;       // a copy was enqueued and not read yet
    void *arena = nullptr;             // device address of the allocation-free render arena
    size_t arena_bytes = 0;
    cudaError_t arena_err = cudaSuccess;
    KernelTimer *timer = nullptr;
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    mrf_tuning tuning{8, 96, 1, 0};
};

struct mrf_field {
    mrf_context *ctx = nullptr;
    FieldDev dev{};
    std::vector<void *> allocs;
};

struct mrf_bvh {
    mrf_context *ctx = nullptr;
    BvhDev dev{};
    float4 *nodes = nullptr, *tris = nullptr;
    float4 *wide = nullptr;              // four-child copy the traversals walk (8 float4 per node)
    uint32_t *order = nullptr, *tri_idx = nullptr;
    float *verts = nullptr;
    int *parent = nullptr, *counters = nullptr;
    uint32_t *mat = nullptr;             // material per original triangle (for rebuilds)
    uint32_t *rebuild_scratch = nullptr; // sort buffers of the GPU rebuild, allocated at the first one
    uint32_t n_verts = 0, n_tris = 0;
    int n_nodes = 0, node_cap = 0;
};

struct mrf_shadow_net {
    mrf_context *ctx = nullptr;
    ShadowNetDev dev{};
    float *params = nullptr, *m = nullptr, *v = nullptr, *mlp_inf = nullptr;
    unsigned long long *grad = nullptr;   // gradient sums in 64-bit fixed point (order-independent)
    uint8_t *lp = nullptr;   // BF16 tensor-core weights (BF16 networks)
    uint64_t n_params = 0;
    uint32_t t = 0;          // Adam steps taken
    uint64_t cursor = 0;     // next training pair
    float lr = 1e-2f, b1 = 0.9f, b2 = 0.99f, eps = 1e-15f, decay = 1.f;
    int precision = MRF_PREC_FP32;
};

static bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static std::atomic<uint32_t> g_fail_allocs{0};   // allocations still to fail (mrf_debug_fail_allocations)

template <class T>
static mrf_status dev_alloc(T **p, size_t n, const char *what) {
    *p = nullptr;
    if (n == 0) return MRF_OK;
    for (uint32_t k = g_fail_allocs.load(); k > 0;)
        if (g_fail_allocs.compare_exchange_weak(k, k - 1))
            return fail(MRF_ERR_OOM, "%s: injected allocation failure", what);
    cudaError_t e = cudaMalloc((void **)p, n * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(e, what);
    }
    return MRF_OK;
}

// IEEE binary16 from FP32, round to nearest even (overflow to infinity)
static uint16_t f32_to_f16(float f) {
    uint32_t x;
    std::memcpy(&x, &f, 4);
    const uint32_t sign = (x >> 16) & 0x8000u, e32 = (x >> 23) & 0xFFu, mant = x & 0x7FFFFFu;
    if (e32 == 0xFFu) return (uint16_t)(sign | 0x7C00u | (mant ? 0x200u : 0u));
    const int exp = (int)e32 - 127 + 15;
    if (exp >= 31) return (uint16_t)(sign | 0x7C00u);
    if (exp <= 0) {
        if (exp < -10) return (uint16_t)sign;
        const uint32_t m = mant | 0x800000u, shift = (uint32_t)(14 - exp);
        uint32_t h = m >> shift;
        const uint32_t rem = m & ((1u << shift) - 1u), half = 1u << (shift - 1u);
        if (rem > half || (rem == half && (h & 1u))) ++h;
        return (uint16_t)(sign | h);
    }
    uint32_t h = sign | ((uint32_t)exp << 10) | (mant >> 13);
    const uint32_t rem = mant & 0x1FFFu;
    if (rem > 0x1000u || (rem == 0x1000u && (h & 1u))) ++h;
    return (uint16_t)h;
}

// bfloat16 from FP32, round to nearest even
static uint16_t f32_to_bf16(float f) {
    uint32_t x;
    std::memcpy(&x, &f, 4);
    if ((x & 0x7F800000u) == 0x7F800000u) return (uint16_t)((x >> 16) | ((x & 0xFFFFu) ? 0x40u : 0u));
    x += 0x7FFFu + ((x >> 16) & 1u);
    return (uint16_t)(x >> 16);
}

// byte offset of element (row r, column k) of a K-major operand with K columns
// in the tensor-core layout without swizzle (8 x 16-byte core matrices)
static size_t umma_offset(int r, int k, int K) {
    return (size_t)(r / 8) * (K / 8) * 128 + (size_t)(k / 8) * 128 + (size_t)(r % 8) * 16 + (size_t)(k % 8) * 2;
}

// copy n elements from host or device memory into host vector
template <class T>
static mrf_status fetch(std::vector<T> &dst, const T *src, size_t n) {
    dst.resize(n);
    if (n == 0) return MRF_OK;
    CUDA_TRY(cudaMemcpy(dst.data(), src, n * sizeof(T), cudaMemcpyDefault), "copy input");
    return MRF_OK;
}

// Entry points keep the C linkage of their declarations in mrf.h.
const char *mrf_last_error(void) { return g_err.c_str(); }
const char *mrf_version(void) { return "0.1.0"; }

mrf_status mrf_context_create(int device, mrf_context **out) {
    if (!out) return fail(MRF_ERR_INVALID_ARG, "mrf_context_create: out is NULL");
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return cuda_fail(e, "mrf_context_create: cudaGetDeviceCount");
    if (device < 0 || device >= n) return fail(MRF_ERR_INVALID_ARG, "mrf_context_create: no device %d", device);
    CUDA_TRY(cudaSetDevice(device), "mrf_context_create: cudaSetDevice");
    cudaDeviceProp prop;
    CUDA_TRY(cudaGetDeviceProperties(&prop, device), "mrf_context_create: cudaGetDeviceProperties");
    if (!(prop.major == 10 && prop.minor == 3))
        return fail(MRF_ERR_UNSUPPORTED, "mrf_context_create: device %d is sm_%d%d, the library is built for sm_103a",
                    device, prop.major, prop.minor);
    mrf_context *c = new (std::nothrow) mrf_context();
    if (!c) return fail(MRF_ERR_OOM, "mrf_context_create: host allocation");
    c->device = device;
    mrf_status st = dev_alloc(&c->stats, ST_COUNT, "mrf_context_create: stats");
    if (st != MRF_OK) {
        delete c;
        return st;
    }
    if ((st = dev_alloc(&c->status, 1, "mrf_context_create: status")) != MRF_OK) {
        cudaFree(c->stats);
        delete c;
        return st;
    }
    cudaMemset(c->stats, 0, sizeof(unsigned long long) * ST_COUNT);
    cudaMemset(c->status, 0, sizeof(unsigned));
    cudaError_t e2 = cudaHostAlloc((void **)&c->status_host, sizeof(unsigned), cudaHostAllocDefault);
    if (e2 == cudaSuccess) e2 = cudaEventCreateWithFlags(&c->status_ev, cudaEventDisableTiming);
    if (e2 != cudaSuccess) {
        mrf_context_destroy(c);
        return cuda_fail(e2, "mrf_context_create: status mirror");
    }
    *c->status_host = 0;
    // the allocation-free entry point's arena: its device address is resolved
    // here, once per context, with the context's device current
    c->arena_err = static_arena(&c->arena, &c->arena_bytes);
    if (c->arena_err != cudaSuccess) cudaGetLastError();
    *out = c;
    return MRF_OK;
}

void mrf_context_destroy(mrf_context *c) {
    if (!c) return;
    cudaFree(c->mats);
    cudaFree(c->lights);
    cudaFree(c->stats);
    cudaFree(c->status);
    cudaFree(c->scratch);
    if (c->status_host) cudaFreeHost(c->status_host);
    if (c->status_ev) cudaEventDestroy(c->status_ev);
    if (c->timer) {
        for (auto &e : c->timer->ev) cudaEventDestroy(e);
        delete c->timer;
    }
    delete c;
}

// ------------------------------------------------------------------ field
static void field_free(mrf_field *f) {
    for (void *p : f->allocs) cudaFree(p);
    f->allocs.clear();
}

template <class T>
static mrf_status upload(mrf_field *f, const T *src, size_t n, const T **dst, const char *what) {
    *dst = nullptr;
    if (n == 0) return MRF_OK;
    if (!src) return fail(MRF_ERR_INVALID_ARG, "mrf_field_create: %s is NULL", what);
    T *d = nullptr;
    mrf_status st = dev_alloc(&d, n, what);
    if (st != MRF_OK) return st;
    f->allocs.push_back(d);
    CUDA_TRY(cudaMemcpy(d, src, n * sizeof(T), cudaMemcpyDefault), what);
    *dst = d;
    return MRF_OK;
}

// True when every occupancy cell that a support sphere can reach is marked, so
// that no sample with positive support is ever rejected by the occupancy test.
// The sphere is grown by 1e-5 relative and by 1e-5 of the box, and cells are
// tested as closed boxes: this absorbs the FP32 rounding of the walk's support
// test and of its cell index (a few ulps of the coordinates).
static bool occupancy_covers_support(const std::vector<uint32_t> &bits, uint32_t R, const double lo[3],
                                     const double ext[3], const std::vector<float> &sc, const std::vector<float> &sr) {
    const double m = 1e-5 * std::max(ext[0], std::max(ext[1], ext[2]));
    for (size_t k = 0; k < sr.size(); ++k) {
        const double r = (double)sr[k] * (1.0 + 1e-5) + m;
        const double c[3] = {sc[3 * k], sc[3 * k + 1], sc[3 * k + 2]};
        int a[3], b[3];
        for (int q = 0; q < 3; ++q) {
            const double cell = ext[q] / R;
            a[q] = std::max(0, (int)std::floor((c[q] - r - lo[q]) / cell) - 1);
            b[q] = std::min((int)R - 1, (int)std::floor((c[q] + r - lo[q]) / cell) + 1);
        }
        for (int z = a[2]; z <= b[2]; ++z)
            for (int y = a[1]; y <= b[1]; ++y)
                for (int x = a[0]; x <= b[0]; ++x) {
                    const int ii[3] = {x, y, z};
                    double d2 = 0.0;
                    for (int q = 0; q < 3; ++q) {
                        const double cell = ext[q] / R, e0 = lo[q] + ii[q] * cell, e1 = e0 + cell;
                        const double g = std::max(0.0, std::max(e0 - c[q], c[q] - e1));
                        d2 += g * g;
                    }
                    const size_t i = (size_t)x + (size_t)R * ((size_t)y + (size_t)R * (size_t)z);
                    if (d2 <= r * r && !((bits[i >> 5] >> (i & 31)) & 1u)) return false;
                }
    }
    return true;
}

static mrf_status field_create_impl(mrf_context *ctx, const mrf_field_desc *D, mrf_field *f) {
    FieldDev &F = f->dev;
    F.kind = D->kind;
    F.status = ctx->status;
    for (int k = 0; k < 3; ++k) {
        if (!(D->aabb_max[k] > D->aabb_min[k])) return fail(MRF_ERR_INVALID_ARG, "mrf_field_create: empty box");
        F.lo[k] = D->aabb_min[k];
        F.hi[k] = D->aabb_max[k];
        F.ext_inv[k] = (float)(1.0 / ((double)D->aabb_max[k] - (double)D->aabb_min[k]));
    }
    F.precision = D->precision;
    if (D->precision < MRF_PREC_FP32 || D->precision > MRF_PREC_BF16)
        return fail(MRF_ERR_INVALID_ARG, "mrf_field_create: unknown precision %d", D->precision);
    F.has_pose = 0;
    if (D->pose) {
        std::vector<float> M;
        mrf_status st0;
        if ((st0 = fetch(M, D->pose, 12))) return st0;
        // R must be orthonormal: R^T R = I within 1e-4
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double dotab = 0.0;
                for (int k = 0; k < 3; ++k) dotab += (double)M[4 * k + a] * M[4 * k + b];
                if (std::fabs(dotab - (a == b ? 1.0 : 0.0)) > 1e-4)
                    return fail(MRF_ERR_INVALID_ARG, "mrf_field_create: pose rotation is not orthonormal");
            }
        // world-to-local: [R^T | -R^T t]
        for (int a = 0; a < 3; ++a) {
            double tt = 0.0;
            for (int k = 0; k < 3; ++k) {
                F.to_local[4 * a + k] = M[4 * k + a];
                tt += (double)M[4 * k + a] * M[4 * k + 3];
            }
            F.to_local[4 * a + 3] = (float)-tt;
        }
        F.has_pose = 1;
    }
    if (D->kind == MRF_FIELD_CONST) {
        F.const_sigma = D->const_sigma;
        for (int k = 0; k < 3; ++k) F.const_rgb[k] = D->const_rgb[k];
        return MRF_OK;
    }
    if (D->kind == MRF_FIELD_GAUSS) {
        const uint32_t K = D->n_blobs;
        if (K > 0 && (!D->blob_center || !D->blob_radius || !D->blob_peak || !D->blob_emission))
            return fail(MRF_ERR_INVALID_ARG, "mrf_field_create: GAUSS arrays missing");
        std::vector<float> c, r, pk, em;
        mrf_status st;
        if ((st = fetch(c, D->blob_center, 3 * (size_t)K)) || (st = fetch(r, D->blob_radius, K)) ||
            (st = fetch(pk, D->blob_peak, K)) || (st = fetch(em, D->blob_emission, 3 * (size_t)K)))
            return st;
        std::vector<float4> a(K), b(K);
        for (uint32_t k = 0; k < K; ++k) {
            a[k] = make_float4(c[3 * k], c[3 * k + 1], c[3 * k + 2], (float)(1.0 / (2.0 * r[k] * (double)r[k])));
            b[k] = make_float4(pk[k], em[3 * k], em[3 * k + 1], em[3 * k + 2]);
        }
        F.n_blobs = (int)K;
        if ((st = upload(f, a.data(), K, &F.blob_a, "blob params")) || (st = upload(f, b.data(), K, &F.blob_b, "blob params")))
            return st;
        return MRF_OK;
    }
    if (D->kind != MRF_FIELD_HASHGRID) return fail(MRF_ERR_INVALID_ARG, "mrf_field_create: unknown kind %d", D->kind);
    if (D->n_levels == 0 || D->n_levels > (uint32_t)kMaxLevels)
        return fail(MRF_ERR_INVALID_ARG, "mrf_field_create: n_levels %u out of range", D->n_levels);
    if (D->n_features != 2) return fail(MRF_ERR_UNSUPPORTED, "mrf_field_create: only 2 features per level are supported");
    if (D->n_levels * D->n_features > (uint32_t)kMaxIn || (D->n_levels * D->n_features) % 16 != 0)
        return fail(MRF_ERR_INVALID_ARG, "mrf_field_create: n_levels * n_features must be a multiple of 16 and <= 64");
    if (D->mlp_width != (uint32_t)kMlpWidth) return fail(MRF_ERR_INVALID_ARG, "mrf_field_create: mlp_width must be 64");
    if (D->log2_table_size < 4 || D->log2_table_size > 24)
        return fail(MRF_ERR_INVALID_ARG, "mrf_field_create: log2_table_size out of range");
    if (!D->level_res || !D->table || !D->w1 || !D->b1 || !D->w2 || !D->b2 || !D->w3 || !D->b3)
        return fail(MRF_ERR_INVALID_ARG, "mrf_field_create: HASHGRID arrays missing");
    const uint32_t L = D->n_levels, T = 1u << D->log2_table_size, n_in = L * D->n_features;
    std::vector<uint32_t> res;
    mrf_status st;
    if ((st = fetch(res, D->level_res, L))) return st;
    F.n_levels = (int)L;
    F.log2T = D->log2_table_size;
    F.dense_mask = 0;
    for (uint32_t l = 0; l < L; ++l) {
        if (res[l] < 1 || res[l] > (1u << 20)) return fail(MRF_ERR_INVALID_ARG, "mrf_field_create: bad level resolution");
        F.res[l] = res[l];
        const uint64_t n1 = (uint64_t)res[l] + 1;
        if (n1 * n1 * n1 <= T) F.dense_mask |= 1u << l;
    }
    if ((st = upload(f, reinterpret_cast<const uint32_t *>(D->table), (size_t)L * T, &F.table, "hash table")))
        return st;
    // pack the MLP: W1T[in][64], b1, W2[64][64], b2, W3T[64][4], b3 (+ the view-dependent heads)
    const bool vd = D->view_dependent != 0;
    if (vd && n_in != 32) return fail(MRF_ERR_INVALID_ARG, "mrf_field_create: view-dependent fields need 32 inputs");
    std::vector<float> w1, b1, w2(64 * 64, 0.f), b2(64, 0.f), w3(4 * 64, 0.f), b3(4, 0.f);
    if ((st = fetch(w1, D->w1, 64 * (size_t)n_in)) || (st = fetch(b1, D->b1, 64))) return st;
    if (!vd || D->w2) {
        if (!D->w2 || !D->b2 || !D->w3 || !D->b3) return fail(MRF_ERR_INVALID_ARG, "mrf_field_create: MLP arrays missing");
        if ((st = fetch(w2, D->w2, 64 * 64)) || (st = fetch(b2, D->b2, 64)) || (st = fetch(w3, D->w3, 4 * 64)) ||
            (st = fetch(b3, D->b3, 4)))
            return st;
    }
    std::vector<float> pk(mlp_floats((int)n_in) + (vd ? kViewFloats : 0));
    float *W1T = pk.data(), *B1 = W1T + n_in * 64, *W2 = B1 + 64, *B2 = W2 + 4096, *W3T = B2 + 64, *B3 = W3T + 256;
    for (uint32_t j = 0; j < 64; ++j)
        for (uint32_t i = 0; i < n_in; ++i) W1T[i * 64 + j] = w1[j * n_in + i];
    std::memcpy(B1, b1.data(), 64 * 4);
    std::memcpy(W2, w2.data(), 4096 * 4);
    std::memcpy(B2, b2.data(), 64 * 4);
    for (int j = 0; j < 64; ++j)
        for (int o = 0; o < 4; ++o) W3T[j * 4 + o] = w3[o * 64 + j];
    std::memcpy(B3, b3.data(), 4 * 4);
    std::vector<float> wd2, bd2, wc1, bc1, wc2, bc2, wc3, bc3;
    if (vd) {
        if (!D->wd2 || !D->bd2 || !D->wc1 || !D->bc1 || !D->wc2 || !D->bc2 || !D->wc3 || !D->bc3)
            return fail(MRF_ERR_INVALID_ARG, "mrf_field_create: view-dependent heads missing");
        if ((st = fetch(wd2, D->wd2, 16 * 64)) || (st = fetch(bd2, D->bd2, 16)) || (st = fetch(wc1, D->wc1, 64 * 32)) ||
            (st = fetch(bc1, D->bc1, 64)) || (st = fetch(wc2, D->wc2, 64 * 64)) || (st = fetch(bc2, D->bc2, 64)) ||
            (st = fetch(wc3, D->wc3, 3 * 64)) || (st = fetch(bc3, D->bc3, 3)))
            return st;
        float *WdT = pk.data() + mlp_floats((int)n_in), *BD = WdT + 64 * 16, *Wc1T = BD + 16, *BC1 = Wc1T + 32 * 64,
              *WC2 = BC1 + 64, *BC2 = WC2 + 64 * 64, *Wc3T = BC2 + 64, *BC3 = Wc3T + 256;
        for (int j = 0; j < 64; ++j)
            for (int o = 0; o < 16; ++o) WdT[j * 16 + o] = wd2[o * 64 + j];
        std::memcpy(BD, bd2.data(), 16 * 4);
        for (int j = 0; j < 64; ++j)
            for (int i = 0; i < 32; ++i) Wc1T[i * 64 + j] = wc1[j * 32 + i];
        std::memcpy(BC1, bc1.data(), 64 * 4);
        std::memcpy(WC2, wc2.data(), 4096 * 4);
        std::memcpy(BC2, bc2.data(), 64 * 4);
        for (int j = 0; j < 64; ++j)
            for (int o = 0; o < 3; ++o) Wc3T[j * 4 + o] = wc3[o * 64 + j];
        for (int o = 0; o < 3; ++o) BC3[o] = bc3[o];
        F.view_dep = 1;
        std::memcpy(F.bias_c, b1.data(), 64 * 4);
        std::memcpy(F.bias_c + 64, bd2.data(), 16 * 4);
        std::memcpy(F.bias_c + 80, bc1.data(), 64 * 4);
        std::memcpy(F.bias_c + 144, bc2.data(), 64 * 4);
        for (int o = 0; o < 3; ++o) F.bias_c[208 + o] = bc3[o];
    } else {
        std::memcpy(F.bias_c, b1.data(), 64 * 4);
        std::memcpy(F.bias_c + 64, b2.data(), 64 * 4);
        std::memcpy(F.bias_c + 128, b3.data(), 4 * 4);
    }
    F.n_in = (int)n_in;
    if ((st = upload(f, pk.data(), pk.size(), &F.mlp, "mlp weights"))) return st;
    // FP16 and BF16 copies of W1 (64 x in), W2 (64 x 64), W3 (padded to 16 x 64) in the
    // tensor-core operand layout
    // (view-dependent fields: W1 (64 x 32) at 0, Wd (16 x 64) at 4096, Wc1 (64 x 32) at 6144,
    // Wc2 (64 x 64) at 10240, Wc3 (padded to 16 x 64) at 18432; 20480 bytes per precision)
    {
        const size_t w1b = 64 * (size_t)n_in * 2, per = vd ? 20480 : w1b + 10240;
        std::vector<uint8_t> lp(2 * per, 0);
        for (int prec = 0; prec < 2; ++prec) {
            uint8_t *base = lp.data() + prec * per;
            auto put = [&](size_t off, float v) {
                const uint16_t h = prec == 0 ? f32_to_f16(v) : f32_to_bf16(v);
                std::memcpy(base + off, &h, 2);
            };
            for (int j = 0; j < 64; ++j)
                for (int i = 0; i < (int)n_in; ++i) put(umma_offset(j, i, (int)n_in), w1[j * n_in + i]);
            if (vd) {
                for (int j = 0; j < 16; ++j)
                    for (int i = 0; i < 64; ++i) put(4096 + umma_offset(j, i, 64), wd2[j * 64 + i]);
                for (int j = 0; j < 64; ++j)
                    for (int i = 0; i < 32; ++i) put(6144 + umma_offset(j, i, 32), wc1[j * 32 + i]);
                for (int j = 0; j < 64; ++j)
                    for (int i = 0; i < 64; ++i) put(10240 + umma_offset(j, i, 64), wc2[j * 64 + i]);
                for (int j = 0; j < 3; ++j)
                    for (int i = 0; i < 64; ++i) put(18432 + umma_offset(j, i, 64), wc3[j * 64 + i]);
                continue;
            }
            for (int j = 0; j < 64; ++j)
                for (int i = 0; i < 64; ++i) put(w1b + umma_offset(j, i, 64), w2[j * 64 + i]);
            for (int j = 0; j < 4; ++j)
                for (int i = 0; i < 64; ++i) put(w1b + 8192 + umma_offset(j, i, 64), w3[j * 64 + i]);
        }
        const uint8_t *d = nullptr;
        if ((st = upload(f, lp.data(), lp.size(), &d, "mlp weights (fp16/bf16)"))) return st;
        F.mlp_lp = d;
    }
    // support spheres
    const uint32_t S = D->n_support;
    std::vector<float> sc, sr;
    if (S > 0) {
        if (!D->support_center || !D->support_radius)
            return fail(MRF_ERR_INVALID_ARG, "mrf_field_create: support arrays missing");
        if ((st = fetch(sc, D->support_center, 3 * (size_t)S)) || (st = fetch(sr, D->support_radius, S))) return st;
        std::vector<float4> sp(S);
        for (uint32_t k = 0; k < S; ++k)
            sp[k] = make_float4(sc[3 * k], sc[3 * k + 1], sc[3 * k + 2], (float)(1.0 / ((double)sr[k] * sr[k])));
        F.n_support = (int)S;
        if ((st = upload(f, sp.data(), S, &F.support, "support spheres"))) return st;
    }
    // occupancy
    if (D->occ_res) {
        const uint32_t R = D->occ_res;
        if (R % 8 != 0 || R > 1024 || !D->occ_bits)
            return fail(MRF_ERR_INVALID_ARG, "mrf_field_create: occ_res must be a multiple of 8 <= 1024 with occ_bits");
        const size_t words = (size_t)R * R * R / 32;
        if ((st = upload(f, D->occ_bits, words, &F.occ, "occupancy"))) return st;
        F.occ_res = (int)R;
        for (int k = 0; k < 3; ++k)
            F.occ_scale[k] = (float)((double)R / ((double)D->aabb_max[k] - (double)D->aabb_min[k]));
        // coarse level for empty-space skipping: OR over 8^3 blocks
        std::vector<uint32_t> fine;
        if ((st = fetch(fine, D->occ_bits, words))) return st;
        const uint32_t Rc = R / 8;
        std::vector<uint32_t> coarse(((size_t)Rc * Rc * Rc + 31) / 32, 0u);
        for (uint32_t z = 0; z < R; ++z)
            for (uint32_t y = 0; y < R; ++y)
                for (uint32_t x = 0; x < R; ++x) {
                    const size_t i = x + (size_t)R * (y + (size_t)R * z);
                    if ((fine[i >> 5] >> (i & 31)) & 1u) {
                        const size_t c = x / 8 + (size_t)Rc * (y / 8 + (size_t)Rc * (z / 8));
                        coarse[c >> 5] |= 1u << (c & 31);
                    }
                }
        if ((st = upload(f, coarse.data(), coarse.size(), &F.occ_coarse, "coarse occupancy"))) return st;
        F.occ_coarse_res = (int)Rc;
        double lo[3], ext[3];
        for (int k = 0; k < 3; ++k) {
            lo[k] = D->aabb_min[k];
            ext[k] = (double)D->aabb_max[k] - (double)D->aabb_min[k];
            F.occ_coarse_scale[k] = (float)((double)Rc / ext[k]);
            F.occ_cell[k] = (float)(ext[k] / (double)R);
            F.occ_coarse_cell[k] = (float)(ext[k] / (double)Rc);
        }
        F.occ_covers_support = S > 0 && occupancy_covers_support(fine, R, lo, ext, sc, sr) ? 1 : 0;
    }
    (void)ctx;
    return MRF_OK;
}

mrf_status mrf_field_create(mrf_context *ctx, const mrf_field_desc *desc, mrf_field **out) {
    if (!ctx || !desc || !out) return fail(MRF_ERR_INVALID_ARG, "mrf_field_create: NULL argument");
    *out = nullptr;
    CUDA_TRY(cudaSetDevice(ctx->device), "mrf_field_create: cudaSetDevice");
    mrf_field *f = new (std::nothrow) mrf_field();
    if (!f) return fail(MRF_ERR_OOM, "mrf_field_create: host allocation");
    f->ctx = ctx;
    mrf_status st = field_create_impl(ctx, desc, f);
    if (st != MRF_OK) {
        field_free(f);
        delete f;
        return st;
    }
    *out = f;
    return MRF_OK;
}

void mrf_field_destroy(mrf_field *f) {
    if (!f) return;
    field_free(f);
    delete f;
}

mrf_status mrf_field_set_precision(mrf_field *f, int32_t precision) {
    if (!f) return fail(MRF_ERR_INVALID_ARG, "mrf_field_set_precision: NULL field");
    if (precision < MRF_PREC_FP32 || precision > MRF_PREC_BF16)
        return fail(MRF_ERR_INVALID_ARG, "mrf_field_set_precision: unknown precision %d", precision);
    f->dev.precision = precision;
    return MRF_OK;
}

mrf_status mrf_field_query(mrf_context *ctx, const mrf_field *field, const float *points, uint32_t n, float *out,
                           void *stream) {
    if (!ctx || !field || (!points && n) || (!out && n)) return fail(MRF_ERR_INVALID_ARG, "mrf_field_query: NULL argument");
    if (n == 0) return MRF_OK;
    if (!is_device_ptr(points) || !is_device_ptr(out))
        return fail(MRF_ERR_INVALID_ARG, "mrf_field_query: points and out must be device memory");
    const FieldDev &F = field->dev;
    const cudaStream_t s = (cudaStream_t)stream;
    if (F.kind == MRF_FIELD_HASHGRID && F.precision != MRF_PREC_FP32 && F.view_dep) {
        const int grid = (int)std::min<uint32_t>((n + 127) / 128, 152u * (uint32_t)field_tc_blocks_per_sm());
        CUDA_TRY(launch_field_tc_view(F, F.precision == MRF_PREC_BF16, points, 3, nullptr, nullptr, n,
                                      reinterpret_cast<float4 *>(out), ctx->status, grid, s),
                 "mrf_field_query: tensor-core launch");
    } else if (F.kind == MRF_FIELD_HASHGRID && F.precision != MRF_PREC_FP32) {
        const int grid = (int)std::min<uint32_t>((n + 127) / 128, 152u * (uint32_t)field_tc_blocks_per_sm());
        CUDA_TRY(launch_field_tc(F, F.precision == MRF_PREC_BF16, points, 3, nullptr, n, reinterpret_cast<float4 *>(out),
                                 ctx->status, grid, s),
                 "mrf_field_query: launch");
    } else {
        CUDA_TRY(launch_field_simt(F, points, 3, nullptr, n, reinterpret_cast<float4 *>(out), (int)((n + 127) / 128), s),
                 "mrf_field_query: launch");
    }
    return MRF_OK;
}

// -------------------------------------------------------------------- BVH
mrf_status mrf_bvh_build(mrf_context *ctx, const float *verts, uint32_t n_verts, const uint32_t *tris,
                         const uint32_t *mat_id, uint32_t n_tris, mrf_bvh **out) {
    if (!ctx || !out) return fail(MRF_ERR_INVALID_ARG, "mrf_bvh_build: NULL argument");
    *out = nullptr;
    if (n_tris > 0 && (!verts || !tris || !mat_id || n_verts == 0))
        return fail(MRF_ERR_INVALID_ARG, "mrf_bvh_build: NULL array with n_tris > 0");
    if (n_tris > (1u << 28)) return fail(MRF_ERR_INVALID_ARG, "mrf_bvh_build: too many triangles");
    CUDA_TRY(cudaSetDevice(ctx->device), "mrf_bvh_build: cudaSetDevice");
    std::vector<float> hv;
    std::vector<uint32_t> ht, hm;
    mrf_status st;
    if ((st = fetch(hv, verts, 3 * (size_t)n_verts)) || (st = fetch(ht, tris, 3 * (size_t)n_tris)) ||
        (st = fetch(hm, mat_id, n_tris)))
        return st;
    for (size_t i = 0; i < ht.size(); ++i)
        if (ht[i] >= n_verts) return fail(MRF_ERR_INVALID_ARG, "mrf_bvh_build: vertex index %u >= n_verts", ht[i]);
    for (size_t i = 0; i < hv.size(); ++i)
        if (!std::isfinite(hv[i])) return fail(MRF_ERR_INVALID_ARG, "mrf_bvh_build: non-finite vertex coordinate");
    std::vector<float> nodes;
    std::vector<uint32_t> order;
    std::vector<int> parent;
    bvh_build_host(hv.data(), ht.data(), n_tris, nodes, order, parent);
    std::vector<float4> tv(3 * (size_t)n_tris);
    for (uint32_t s = 0; s < n_tris; ++s) {
        const uint32_t t = order[s];
        for (int v = 0; v < 3; ++v) {
            const float *p = &hv[3 * (size_t)ht[3 * (size_t)t + v]];
            float w = 0.f;
            if (v == 0) std::memcpy(&w, &t, 4);
            if (v == 1) std::memcpy(&w, &hm[t], 4);
            tv[3 * (size_t)s + v] = make_float4(p[0], p[1], p[2], w);
        }
    }
    mrf_bvh *b = new (std::nothrow) mrf_bvh();
    if (!b) return fail(MRF_ERR_OOM, "mrf_bvh_build: host allocation");
    b->ctx = ctx;
    b->n_verts = n_verts;
    b->n_tris = n_tris;
    b->n_nodes = (int)parent.size();
    auto cleanup = [&](mrf_status s2) {
        mrf_bvh_destroy(b);
        return s2;
    };
    if ((st = dev_alloc(&b->nodes, 4 * (size_t)b->n_nodes, "bvh nodes")) ||
        (st = dev_alloc(&b->wide, 8 * (size_t)b->n_nodes, "bvh wide nodes")) || (st = dev_alloc(&b->tris, tv.size(), "bvh tris")) ||
        (st = dev_alloc(&b->order, n_tris, "bvh order")) || (st = dev_alloc(&b->tri_idx, 3 * (size_t)n_tris, "bvh indices")) ||
        (st = dev_alloc(&b->verts, 3 * (size_t)n_verts, "bvh verts")) || (st = dev_alloc(&b->parent, (size_t)b->n_nodes, "bvh parents")) ||
        (st = dev_alloc(&b->counters, (size_t)b->n_nodes, "bvh counters")) ||
        (st = dev_alloc(&b->mat, n_tris, "bvh materials")))
        return cleanup(st);
    b->node_cap = b->n_nodes;
    cudaError_t e = cudaSuccess;
    if (b->n_nodes) {
        e = cudaMemcpy(b->nodes, nodes.data(), nodes.size() * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(b->parent, parent.data(), parent.size() * 4, cudaMemcpyHostToDevice);
    }
    if (n_tris && e == cudaSuccess) {
        e = cudaMemcpy(b->tris, tv.data(), tv.size() * sizeof(float4), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(b->order, order.data(), order.size() * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(b->tri_idx, ht.data(), ht.size() * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(b->verts, hv.data(), hv.size() * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(b->mat, hm.data(), hm.size() * 4, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "mrf_bvh_build: upload"));
    // the wide copy, finished before the call returns (renders may run on any stream)
    if ((e = launch_bvh_widen(b->nodes, b->n_nodes, b->wide, 0)) == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "mrf_bvh_build: wide nodes"));
    b->dev.nodes = b->nodes;
    b->dev.wide = b->wide;
    b->dev.tris = b->tris;
    b->dev.n_nodes = b->n_nodes;
    b->dev.n_tris = (int)n_tris;
    b->dev.status = ctx->status;
    *out = b;
    return MRF_OK;
}

mrf_status mrf_bvh_rebuild(mrf_bvh *b, const float *verts, uint32_t n_verts, void *stream) {
    if (!b || (!verts && n_verts)) return fail(MRF_ERR_INVALID_ARG, "mrf_bvh_rebuild: NULL argument");
    if (n_verts != b->n_verts)
        return fail(MRF_ERR_INVALID_ARG, "mrf_bvh_rebuild: %u vertices, the BVH was built with %u", n_verts, b->n_verts);
    if (b->n_tris == 0) return MRF_OK;
    CUDA_TRY(cudaSetDevice(b->ctx->device), "mrf_bvh_rebuild: cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    const int need = b->n_tris > 1 ? (int)b->n_tris - 1 : 1;
    if (b->node_cap < need || !b->rebuild_scratch) {
        // first rebuild: room for n - 1 internal nodes and the sort buffers
        CUDA_TRY(cudaStreamSynchronize(s), "mrf_bvh_rebuild: synchronize");
        float4 *nodes = nullptr, *wide = nullptr;
        int *parent = nullptr, *counters = nullptr;
        uint32_t *scr = nullptr;
        mrf_status st;
        if ((st = dev_alloc(&nodes, 4 * (size_t)need, "bvh nodes")) || (st = dev_alloc(&wide, 8 * (size_t)need, "bvh wide nodes")) ||
            (st = dev_alloc(&parent, (size_t)need, "bvh parents")) || (st = dev_alloc(&counters, (size_t)need, "bvh counters")) ||
            (st = dev_alloc(&scr, bvh_rebuild_scratch_words(b->n_tris), "bvh rebuild scratch"))) {
            cudaFree(nodes);
            cudaFree(wide);
            cudaFree(parent);
            cudaFree(counters);
            cudaFree(scr);
            return st;
        }
        cudaFree(b->nodes);
        cudaFree(b->wide);
        cudaFree(b->parent);
        cudaFree(b->counters);
        cudaFree(b->rebuild_scratch);
        b->nodes = nodes;
        b->wide = wide;
        b->parent = parent;
        b->counters = counters;
        b->rebuild_scratch = scr;
        b->node_cap = need;
        b->dev.nodes = b->nodes;
        b->dev.wide = b->wide;
    }
    CUDA_TRY(cudaMemcpyAsync(b->verts, verts, 3 * sizeof(float) * (size_t)n_verts, cudaMemcpyDefault, s),
             "mrf_bvh_rebuild: vertex upload");
    CUDA_TRY(launch_bvh_rebuild(b->nodes, b->parent, b->counters, b->tris, b->order, b->tri_idx, b->mat, b->verts,
                                b->n_tris, b->rebuild_scratch, s),
             "mrf_bvh_rebuild");
    CUDA_TRY(launch_bvh_widen(b->nodes, need, b->wide, s), "mrf_bvh_rebuild: wide nodes");
    b->n_nodes = need;
    b->dev.n_nodes = need;
    if (!is_device_ptr(verts)) CUDA_TRY(cudaStreamSynchronize(s), "mrf_bvh_rebuild: synchronize");
    return MRF_OK;
}

mrf_status mrf_bvh_refit(mrf_bvh *b, const float *verts, uint32_t n_verts, void *stream) {
    if (!b || (!verts && n_verts)) return fail(MRF_ERR_INVALID_ARG, "mrf_bvh_refit: NULL argument");
    if (n_verts != b->n_verts)
        return fail(MRF_ERR_INVALID_ARG, "mrf_bvh_refit: %u vertices, the BVH was built with %u", n_verts, b->n_verts);
    if (b->n_tris == 0) return MRF_OK;
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(b->verts, verts, 3 * sizeof(float) * (size_t)n_verts, cudaMemcpyDefault, s),
             "mrf_bvh_refit: vertex upload");
    CUDA_TRY(launch_bvh_refit(b->nodes, b->n_nodes, b->tris, (int)b->n_tris, b->order, b->tri_idx, b->verts, b->parent,
                              b->counters, nullptr, s),
             "mrf_bvh_refit: launch");
    CUDA_TRY(launch_bvh_widen(b->nodes, b->n_nodes, b->wide, s), "mrf_bvh_refit: wide nodes");
    return MRF_OK;
}

void mrf_bvh_destroy(mrf_bvh *b) {
    if (!b) return;
    cudaFree(b->nodes);
    cudaFree(b->wide);
    cudaFree(b->tris);
    cudaFree(b->order);
    cudaFree(b->tri_idx);
    cudaFree(b->verts);
    cudaFree(b->parent);
    cudaFree(b->counters);
    cudaFree(b->mat);
    cudaFree(b->rebuild_scratch);
    delete b;
}

mrf_status mrf_cast(mrf_context *ctx, const mrf_bvh *bvh, const float *origins, const float *dirs,
                    const uint32_t *skip, uint32_t n, float tmin, float *out_t, uint32_t *out_tri, void *stream) {
    if (!ctx || !bvh) return fail(MRF_ERR_INVALID_ARG, "mrf_cast: NULL handle");
    if (n == 0) return MRF_OK;
    if (!is_device_ptr(origins) || !is_device_ptr(dirs) || !is_device_ptr(out_t) || !is_device_ptr(out_tri) ||
        (skip && !is_device_ptr(skip)))
        return fail(MRF_ERR_INVALID_ARG, "mrf_cast: arrays must be device memory");
    CUDA_TRY(launch_cast(bvh->dev, origins, dirs, skip, n, tmin, out_t, out_tri, nullptr, (cudaStream_t)stream),
             "mrf_cast: launch");
    return MRF_OK;
}

// -------------------------------------------------------- materials/lights
mrf_status mrf_materials_set(mrf_context *ctx, const mrf_material *mats, uint32_t n) {
    if (!ctx || (!mats && n)) return fail(MRF_ERR_INVALID_ARG, "mrf_materials_set: NULL argument");
    if (n > 65535) return fail(MRF_ERR_INVALID_ARG, "mrf_materials_set: too many materials");
    std::vector<mrf_material> h;
    mrf_status st;
    if ((st = fetch(h, mats, n))) return st;
    std::vector<MaterialDev> d(n);
    for (uint32_t i = 0; i < n; ++i) {
        if (h[i].kind < MRF_MAT_MIRROR || h[i].kind > MRF_MAT_DIFFUSE)
            return fail(MRF_ERR_INVALID_ARG, "mrf_materials_set: unknown kind %d", h[i].kind);
        if (h[i].kind == MRF_MAT_GLASS && !(h[i].ior > 0.f))
            return fail(MRF_ERR_INVALID_ARG, "mrf_materials_set: glass needs ior > 0");
        d[i].kind = h[i].kind;
        for (int k = 0; k < 3; ++k) d[i].rgb[k] = h[i].rgb[k];
        d[i].ior = h[i].ior;
    }
    CUDA_TRY(cudaSetDevice(ctx->device), "mrf_materials_set: cudaSetDevice");
    cudaFree(ctx->mats);
    ctx->mats = nullptr;
    ctx->n_mats = 0;
    if (n) {
        if ((st = dev_alloc(&ctx->mats, n, "materials"))) return st;
        CUDA_TRY(cudaMemcpy(ctx->mats, d.data(), n * sizeof(MaterialDev), cudaMemcpyHostToDevice), "materials upload");
    }
    ctx->n_mats = (int)n;
    return MRF_OK;
}

mrf_status mrf_lights_set(mrf_context *ctx, const mrf_light *lights, uint32_t n) {
    if (!ctx || (!lights && n)) return fail(MRF_ERR_INVALID_ARG, "mrf_lights_set: NULL argument");
    if (n > 65535) return fail(MRF_ERR_INVALID_ARG, "mrf_lights_set: too many lights");
    std::vector<mrf_light> h;
    mrf_status st;
    if ((st = fetch(h, lights, n))) return st;
    std::vector<LightDev> d(n);
    uint32_t q = 0, slots = 0;
    for (uint32_t i = 0; i < n; ++i) {
        LightDev &L = d[i];
        std::memset(&L, 0, sizeof(L));
        for (int k = 0; k < 3; ++k) {
            L.pos[k] = h[i].pos[k];
            L.I[k] = h[i].intensity[k];
        }
        L.kind = h[i].kind;
        L.slot0 = slots;
        if (!(h[i].mask_strength >= 0.f && h[i].mask_strength <= 1.f))
            return fail(MRF_ERR_INVALID_ARG, "mrf_lights_set: light %u: mask_strength must be in [0, 1]", i);
        L.mask = h[i].mask_strength;
        for (int k = 0; k < 3; ++k) L.target[k] = h[i].pos[k];
        if (h[i].kind == MRF_LIGHT_POINT) {
            L.samples = 1;
        } else if (h[i].kind == MRF_LIGHT_AREA) {
            if (h[i].samples < 1 || h[i].samples > 64)
                return fail(MRF_ERR_INVALID_ARG, "mrf_lights_set: light %u: samples must be 1..64", i);
            double e1[3], e2[3], c[3];
            for (int k = 0; k < 3; ++k) {
                L.v1[k] = h[i].v1[k];
                L.v2[k] = h[i].v2[k];
                e1[k] = (double)h[i].v1[k] - h[i].pos[k];
                e2[k] = (double)h[i].v2[k] - h[i].pos[k];
            }
            c[0] = e1[1] * e2[2] - e1[2] * e2[1];
            c[1] = e1[2] * e2[0] - e1[0] * e2[2];
            c[2] = e1[0] * e2[1] - e1[1] * e2[0];
            const double len = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
            if (!(len > 0)) return fail(MRF_ERR_INVALID_ARG, "mrf_lights_set: light %u: degenerate triangle", i);
            for (int k = 0; k < 3; ++k) L.n[k] = (float)(c[k] / len);
            for (int k = 0; k < 3; ++k)
                L.target[k] = (float)(((double)h[i].pos[k] + h[i].v1[k] + h[i].v2[k]) / 3.0);
            L.area = (float)(0.5 * len);
            L.samples = h[i].samples;
            L.q0 = q;
            q += L.samples;
        } else {
            return fail(MRF_ERR_INVALID_ARG, "mrf_lights_set: light %u: unknown kind %d", i, h[i].kind);
        }
        slots += L.samples;
    }
    CUDA_TRY(cudaSetDevice(ctx->device), "mrf_lights_set: cudaSetDevice");
    cudaFree(ctx->lights);
    ctx->lights = nullptr;
    ctx->n_lights = 0;
    ctx->n_shadow = 0;
    if (n) {
        if ((st = dev_alloc(&ctx->lights, n, "lights"))) return st;
        CUDA_TRY(cudaMemcpy(ctx->lights, d.data(), n * sizeof(LightDev), cudaMemcpyHostToDevice), "lights upload");
    }
    ctx->n_lights = (int)n;
    ctx->n_shadow = (int)slots;
    return MRF_OK;
}

// ----------------------------------------------------------------- render
static mrf_status ensure_scratch(mrf_context *ctx, size_t bytes) {
    if (bytes <= ctx->scratch_bytes) return MRF_OK;
    cudaFree(ctx->scratch);
    ctx->scratch = nullptr;
    ctx->scratch_bytes = 0;
    size_t want = bytes + bytes / 4;
    cudaError_t e = cudaMalloc(&ctx->scratch, want);
    if (e != cudaSuccess) return cuda_fail(e, "render scratch");
    ctx->scratch_bytes = want;
    return MRF_OK;
}

// Pinhole basis of one camera, built in FP64 and rounded once to FP32.
// Returns NULL, or what is wrong with the camera.
static const char *camera_view(const mrf_camera &c, ViewDev &v) {
    if (c.width == 0 || c.height == 0 || !(c.vfov_deg > 0.f && c.vfov_deg < 180.f)) return "bad camera";
    double f[3], up[3], r[3], u[3];
    for (int k = 0; k < 3; ++k) {
        f[k] = (double)c.look_at[k] - c.pos[k];
        up[k] = c.up[k];
    }
    const double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    if (!(fl > 0)) return "camera looks at itself";
    for (double &x : f) x /= fl;
    r[0] = f[1] * up[2] - f[2] * up[1];
    r[1] = f[2] * up[0] - f[0] * up[2];
    r[2] = f[0] * up[1] - f[1] * up[0];
    const double rl = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (!(rl > 0)) return "camera up is parallel to the view direction";
    for (double &x : r) x /= rl;
    u[0] = r[1] * f[2] - r[2] * f[1];
    u[1] = r[2] * f[0] - r[0] * f[2];
    u[2] = r[0] * f[1] - r[1] * f[0];
    for (int k = 0; k < 3; ++k) {
        v.pos[k] = c.pos[k];
        v.f[k] = (float)f[k];
        v.r[k] = (float)r[k];
        v.u[k] = (float)u[k];
    }
    v.tan_half = (float)std::tan(0.5 * (double)c.vfov_deg * M_PI / 180.0);
    v.aspect = (float)((double)c.width / (double)c.height);
    v.W = c.width;
    v.H = c.height;
    v.offset = 0;
    v.pad = 0;
    return nullptr;
}

// A validated render request: kernel parameters, engine and scratch layout.
struct RenderPlan {
    RenderParams P{};
    int engine = MRF_ENGINE_MEGAKERNEL;
    uint32_t count = 0, n_views = 0;
    bool host_rays = false, host_out = false;
    size_t out_off = 0, wf_off = 0, scratch_need = 0;
    std::vector<ViewDev> views;
};

// Checks the arguments of a render call and fills the plan; no device work
// besides pointer queries.
static mrf_status plan_render(mrf_context *ctx, const mrf_field *field, const mrf_bvh *bvh, const mrf_rays *rays,
                              uint32_t max_bounces, const mrf_render_opts *opts, float *out_hdr, RenderPlan &R) {
    if (!ctx || !field || !bvh || !rays || !opts || !out_hdr)
        return fail(MRF_ERR_INVALID_ARG, "mrf_render: NULL argument");
    if (field->ctx != ctx || bvh->ctx != ctx) return fail(MRF_ERR_INVALID_ARG, "mrf_render: handle of another context");
    if (max_bounces == 0 || max_bounces > (uint32_t)kMaxBounces)
        return fail(MRF_ERR_INVALID_ARG, "mrf_render: max_bounces must be in [1, %d]", kMaxBounces);
    if (rays->spp == 0) return fail(MRF_ERR_INVALID_ARG, "mrf_render: spp must be >= 1");
    if (opts->steps_per_segment == 0 && !(opts->dt > 0.f))
        return fail(MRF_ERR_INVALID_ARG, "mrf_render: need steps_per_segment > 0 or dt > 0");
    if (!(opts->tau >= 0.f) || !(opts->tmin >= 0.f)) return fail(MRF_ERR_INVALID_ARG, "mrf_render: negative tau or tmin");
    if (bvh->n_tris && ctx->n_mats == 0) return fail(MRF_ERR_NOT_READY, "mrf_render: no materials set");
    if (opts->engine < MRF_ENGINE_AUTO || opts->engine > MRF_ENGINE_WAVEFRONT)
        return fail(MRF_ERR_INVALID_ARG, "mrf_render: unknown engine %d", opts->engine);
    if (opts->engine == MRF_ENGINE_WAVEFRONT && !wavefront_available())
        return fail(MRF_ERR_UNSUPPORTED, "mrf_render: wavefront engine not built");
    RenderParams &P = R.P;
    P.F = field->dev;
    P.B = bvh->dev;
    P.mats = ctx->mats;
    P.n_mats = ctx->n_mats;
    P.lights = ctx->lights;
    P.n_lights = ctx->n_lights;
    P.n_shadow = ctx->n_shadow;
    uint32_t count;
    size_t scratch_need = 0;
    R.host_rays = !rays->camera && !is_device_ptr(rays->origins);
    const uint32_t n_views = rays->camera && rays->n_cameras > 1 ? rays->n_cameras : 0;
    if (n_views) {
        // several views: a table in device scratch, searched by ray index
        if (n_views > 65536u) return fail(MRF_ERR_INVALID_ARG, "mrf_render: more than 65536 cameras");
        if (is_device_ptr(rays->camera)) return fail(MRF_ERR_INVALID_ARG, "mrf_render: camera records must be host memory");
        R.views.resize(n_views);
        uint64_t total = 0;
        for (uint32_t k = 0; k < n_views; ++k) {
            if (const char *why = camera_view(rays->camera[k], R.views[k]))
                return fail(MRF_ERR_INVALID_ARG, "mrf_render: camera %u: %s", k, why);
            R.views[k].offset = (uint32_t)std::min<uint64_t>(total, 0xFFFFFFFFull);
            total += (uint64_t)R.views[k].W * R.views[k].H;
        }
        if (total > 0xFFFFFFFFull / 4) return fail(MRF_ERR_INVALID_ARG, "mrf_render: views too large");
        count = (uint32_t)total;
        scratch_need = sizeof(ViewDev) * (size_t)n_views;
    } else if (rays->camera) {
        const mrf_camera &c = *rays->camera;
        ViewDev v;
        if (const char *why = camera_view(c, v)) return fail(MRF_ERR_INVALID_ARG, "mrf_render: %s", why);
        const uint64_t cnt = (uint64_t)c.width * c.height;
        if (cnt > 0xFFFFFFFFull / 4) return fail(MRF_ERR_INVALID_ARG, "mrf_render: image too large");
        count = (uint32_t)cnt;
        P.use_camera = 1;
        for (int k = 0; k < 3; ++k) {
            P.cam_pos[k] = v.pos[k];
            P.cam_f[k] = v.f[k];
            P.cam_r[k] = v.r[k];
            P.cam_u[k] = v.u[k];
        }
        P.tan_half = v.tan_half;
        P.aspect = v.aspect;
        P.W = v.W;
        P.H = v.H;
    } else {
        if (!rays->origins || !rays->dirs || rays->count == 0)
            return fail(MRF_ERR_INVALID_ARG, "mrf_render: explicit rays need origins, dirs and count > 0");
        count = rays->count;
        if (R.host_rays) scratch_need += 2 * 3 * sizeof(float) * (size_t)count;
        else {
            P.ray_o = rays->origins;
            P.ray_d = rays->dirs;
        }
    }
    R.n_views = n_views;
    if ((uint64_t)count * rays->spp > 0xFFFFFFFFull) return fail(MRF_ERR_INVALID_ARG, "mrf_render: too many paths");
    R.host_out = !is_device_ptr(out_hdr);
    R.out_off = (scratch_need + 255) & ~(size_t)255;
    if (R.host_out) scratch_need = R.out_off + 4 * sizeof(float) * (size_t)count;
    if ((opts->rec_segments && !is_device_ptr(opts->rec_segments)) || (opts->rec_tri && !is_device_ptr(opts->rec_tri)) ||
        (opts->rec_t && !is_device_ptr(opts->rec_t)) || (!opts->rec_tri != !opts->rec_t))
        return fail(MRF_ERR_INVALID_ARG, "mrf_render: records must be device pointers (rec_tri and rec_t together)");
    P.count = count;
    P.spp = rays->spp;
    P.max_bounces = max_bounces;
    P.seed = opts->seed;
    P.steps = opts->steps_per_segment;
    P.dt = opts->dt;
    P.tau = opts->tau;
    P.tmin = opts->tmin;
    P.rec_seg = opts->rec_segments;
    P.rec_tri = opts->rec_tri;
    P.rec_t = opts->rec_t;
    P.shadow_mask = opts->shadow_mask ? 1 : 0;
    P.tc_groups = (int)ctx->tuning.field_groups;
    P.cap_per_path = ctx->tuning.samples_per_path;
    P.max_rounds = (int)ctx->tuning.rounds;
    P.tail_paths = ctx->tuning.tail_paths;
    if (opts->shadow_net) {
        if (opts->shadow_net->ctx != ctx) return fail(MRF_ERR_INVALID_ARG, "shadow_net belongs to another context");
        P.has_snet = 1;
        P.snet = opts->shadow_net->dev;
    }
    // AUTO: tensor-core field evaluation needs the wavefront engine's flat sample
    // tiles; FP32 runs the megakernel
    const bool lowp = field->dev.kind == MRF_FIELD_HASHGRID && field->dev.precision != MRF_PREC_FP32;
    R.engine = opts->engine == MRF_ENGINE_AUTO ? (lowp ? MRF_ENGINE_WAVEFRONT : MRF_ENGINE_MEGAKERNEL) : opts->engine;
    if (R.engine == MRF_ENGINE_MEGAKERNEL && lowp)
        return fail(MRF_ERR_UNSUPPORTED, "mrf_render: FP16/BF16 fields run on the wavefront engine");
    if (R.engine == MRF_ENGINE_WAVEFRONT && ctx->n_shadow > 64)
        return fail(MRF_ERR_UNSUPPORTED, "mrf_render: the wavefront engine takes at most 64 shadow rays per hit");
    if (R.engine == MRF_ENGINE_WAVEFRONT) {
        R.wf_off = (scratch_need + 255) & ~(size_t)255;
        scratch_need = R.wf_off + wavefront_scratch_bytes(P);
    }
    R.count = count;
    R.scratch_need = scratch_need;
    P.status = ctx->status;
    return MRF_OK;
}

// Device pointers of the plan inside the context's scratch (which must hold
// R.scratch_need bytes).
static void place_render(mrf_context *ctx, RenderPlan &R, float *out_hdr) {
    char *scr = (char *)ctx->scratch;
    if (R.n_views) {
        R.P.views = (const ViewDev *)scr;
        R.P.n_views = R.n_views;
    }
    if (R.host_rays) {
        R.P.ray_o = (float *)scr;
        R.P.ray_d = (float *)scr + 3 * (size_t)R.count;
    }
    R.P.out = R.host_out ? (float *)(scr + R.out_off) : out_hdr;
}

// Every launch of the planned render on stream s.
static mrf_status launch_render(mrf_context *ctx, const RenderPlan &R, cudaStream_t s, KernelTimer *timer) {
    char *scr = (char *)ctx->scratch;
    if (R.engine == MRF_ENGINE_WAVEFRONT) {
        CUDA_TRY(launch_render_wavefront(R.P, scr + R.wf_off, R.scratch_need - R.wf_off, s, timer),
                 "mrf_render: wavefront launch");
    } else {
        CUDA_TRY(launch_render_megakernel(R.P, s, timer), "mrf_render: launch");
    }
    return MRF_OK;
}

static void stats_from(const unsigned long long *h, unsigned st_word, mrf_stats *stats) {
    stats->paths = h[ST_PATHS];
    stats->segments = h[ST_SEGMENTS];
    stats->surface_hits = h[ST_HITS];
    stats->shadow_rays = h[ST_SHADOW];
    stats->samples_nominal = h[ST_NOMINAL];
    stats->samples_evaluated = h[ST_EVALUATED];
    stats->shadow_samples_evaluated = h[ST_SHADOW_EVALUATED];
    stats->fp64_retests = h[ST_FP64];
    stats->shadow_net_evals = h[ST_NET];
    stats->ended_miss = h[ST_END_MISS];
    stats->ended_tau = h[ST_END_TAU];
    stats->ended_cap = h[ST_END_CAP];
    stats->bvh_nodes = h[ST_NODES];
    stats->bvh_tri_tests = h[ST_TRIS];
    stats->bvh_worst_nodes = h[ST_WORST] >> 32;
    stats->bvh_worst_path = h[ST_WORST] & 0xffffffffull;
    stats->status = st_word;
}

// Status of kernels that gave up, reported without blocking the host: every
// render call ends by copying the device status word to the context's pinned
// mirror on its stream (post_status); the next call reads the mirror if that
// copy has landed (poll_status) and otherwise goes on, so the report may come
// one call later.  mrf_sync_status waits for the device and reads the word.
static bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

static mrf_status poll_status(mrf_context *ctx, cudaStream_t s, const char *who) {
    if (!ctx->status_pending || capturing(s)) return MRF_OK;
    const cudaError_t q = cudaEventQuery(ctx->status_ev);
    if (q == cudaErrorNotReady) {
        if (cudaPeekAtLastError() == cudaErrorNotReady) cudaGetLastError();
        return MRF_OK;
    }
    if (q != cudaSuccess) return cuda_fail(q, who);
    ctx->status_pending = false;
    const unsigned w = *ctx->status_host;
    if (w) {
        *ctx->status_host = 0;
        CUDA_TRY(cudaMemsetAsync(ctx->status, 0, sizeof(unsigned), s), who);
        return fail(MRF_ERR_TIMEOUT, "%s: an earlier kernel gave up (status 0x%x)", who, w);
    }
    return MRF_OK;
}

static mrf_status post_status(mrf_context *ctx, cudaStream_t s, const char *who) {
    if (capturing(s)) return MRF_OK;
    CUDA_TRY(cudaMemcpyAsync(ctx->status_host, ctx->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s), who);
    CUDA_TRY(cudaEventRecord(ctx->status_ev, s), who);
    ctx->status_pending = true;
    return MRF_OK;
}

// After a call that waited for its stream: the status word as of that point.
static mrf_status read_status_after_sync(mrf_context *ctx, cudaStream_t s, unsigned &w, const char *who) {
    CUDA_TRY(cudaMemcpyAsync(ctx->status_host, ctx->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s), who);
    CUDA_TRY(cudaStreamSynchronize(s), who);
    w = *ctx->status_host;
    ctx->status_pending = false;
    if (w) {
        *ctx->status_host = 0;
        CUDA_TRY(cudaMemsetAsync(ctx->status, 0, sizeof(unsigned), s), who);
    }
    return MRF_OK;
}

mrf_status mrf_sync_status(mrf_context *ctx, uint32_t *status_word) {
    if (status_word) *status_word = 0;
    if (!ctx) return fail(MRF_ERR_INVALID_ARG, "mrf_sync_status: NULL context");
    CUDA_TRY(cudaSetDevice(ctx->device), "mrf_sync_status: cudaSetDevice");
    CUDA_TRY(cudaDeviceSynchronize(), "mrf_sync_status: asynchronous error");
    unsigned w = 0;
    CUDA_TRY(cudaMemcpy(&w, ctx->status, sizeof(unsigned), cudaMemcpyDeviceToHost), "mrf_sync_status: status read");
    ctx->status_pending = false;
    *ctx->status_host = 0;
    if (status_word) *status_word = w;
    if (w) {
        CUDA_TRY(cudaMemset(ctx->status, 0, sizeof(unsigned)), "mrf_sync_status: status clear");
        return fail(MRF_ERR_TIMEOUT, "mrf_sync_status: a kernel gave up (status 0x%x)", w);
    }
    return MRF_OK;
}

mrf_status mrf_render(mrf_context *ctx, const mrf_field *field, const mrf_bvh *bvh, const mrf_rays *rays,
                      uint32_t max_bounces, const mrf_render_opts *opts, float *out_hdr, void *stream,
                      mrf_stats *stats) {
    RenderPlan R;
    mrf_status st = plan_render(ctx, field, bvh, rays, max_bounces, opts, out_hdr, R);
    if (st) return st;
    CUDA_TRY(cudaSetDevice(ctx->device), "mrf_render: cudaSetDevice");
    {
        cudaError_t pending = cudaGetLastError();
        if (pending != cudaSuccess) return cuda_fail(pending, "mrf_render: earlier asynchronous error");
    }
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = poll_status(ctx, s, "mrf_render"))) return st;
    if (R.scratch_need && (st = ensure_scratch(ctx, R.scratch_need))) return st;
    place_render(ctx, R, out_hdr);
    if (R.n_views)
        CUDA_TRY(cudaMemcpyAsync((void *)R.P.views, R.views.data(), sizeof(ViewDev) * (size_t)R.n_views,
                                 cudaMemcpyHostToDevice, s),
                 "mrf_render: camera table upload");
    if (R.host_rays) {
        CUDA_TRY(cudaMemcpyAsync((void *)R.P.ray_o, rays->origins, 3 * sizeof(float) * (size_t)R.count,
                                 cudaMemcpyDefault, s), "ray upload");
        CUDA_TRY(cudaMemcpyAsync((void *)R.P.ray_d, rays->dirs, 3 * sizeof(float) * (size_t)R.count, cudaMemcpyDefault,
                                 s), "ray upload");
    }
    if (stats) {
        CUDA_TRY(cudaMemsetAsync(ctx->stats, 0, sizeof(unsigned long long) * ST_COUNT, s), "stats reset");
        R.P.stats = ctx->stats;
    }
    KernelTimer *timer = nullptr;
    if (opts->kernel_ms) {
        if (!ctx->timer) {
            ctx->timer = new (std::nothrow) KernelTimer();
            if (!ctx->timer) return fail(MRF_ERR_OOM, "mrf_render: timer allocation");
            for (auto &e : ctx->timer->ev) CUDA_TRY(cudaEventCreate(&e), "mrf_render: event create");
        }
        timer = ctx->timer;
        timer->n = 0;
        timer->ok = true;
    }
    if ((st = launch_render(ctx, R, s, timer))) return st;
    if (timer) {
        CUDA_TRY(cudaStreamSynchronize(s), "mrf_render: synchronize");
        if (!timer->ok)
            return fail(MRF_ERR_UNSUPPORTED, "mrf_render: kernel timing holds at most %d launches per call",
                        KernelTimer::kMax);
        for (int k = 0; k < MRF_KERNEL_COUNT; ++k) {
            opts->kernel_ms[k] = 0.f;
            if (opts->kernel_launches) opts->kernel_launches[k] = 0;
        }
        for (int i = 0; i < timer->n; ++i) {
            float ms = 0.f;
            CUDA_TRY(cudaEventElapsedTime(&ms, timer->ev[2 * i], timer->ev[2 * i + 1]), "mrf_render: event time");
            opts->kernel_ms[timer->kind[i]] += ms;
            if (opts->kernel_launches) opts->kernel_launches[timer->kind[i]] += 1;
        }
    }
    if (R.host_out) {
        CUDA_TRY(cudaMemcpyAsync(out_hdr, R.P.out, 4 * sizeof(float) * (size_t)R.count, cudaMemcpyDeviceToHost, s),
                 "mrf_render: image download");
    }
    if (stats) {
        unsigned long long h[ST_COUNT];
        CUDA_TRY(cudaMemcpyAsync(h, ctx->stats, sizeof(h), cudaMemcpyDeviceToHost, s), "stats download");
        unsigned st_word = 0;
        if ((st = read_status_after_sync(ctx, s, st_word, "mrf_render: status read"))) return st;
        stats_from(h, st_word, stats);
        if (st_word) return fail(MRF_ERR_TIMEOUT, "mrf_render: a kernel gave up (status 0x%x)", st_word);
        return MRF_OK;
    }
    if ((st = post_status(ctx, s, "mrf_render: status copy"))) return st;
    if (R.host_out) CUDA_TRY(cudaStreamSynchronize(s), "mrf_render: synchronize");
    return MRF_OK;
}

// ------------------------------------------------------------------ tuning
mrf_status mrf_tuning_get(const mrf_context *ctx, mrf_tuning *out) {
    if (!ctx || !out) return fail(MRF_ERR_INVALID_ARG, "mrf_tuning_get: NULL argument");
    *out = ctx->tuning;
    return MRF_OK;
}

mrf_status mrf_tuning_set(mrf_context *ctx, const mrf_tuning *t) {
    if (!ctx || !t) return fail(MRF_ERR_INVALID_ARG, "mrf_tuning_set: NULL argument");
    if ((t->field_groups != 4 && t->field_groups != 5 && t->field_groups != 8) || t->samples_per_path < 16 ||
        t->samples_per_path > 4096 || t->rounds < 1 || t->rounds > 16 || t->tail_paths > (1u << 20))
        return fail(MRF_ERR_INVALID_ARG, "mrf_tuning_set: field_groups 4, 5 or 8, samples_per_path 16..4096, "
                                         "rounds 1..16, tail_paths 0..2^20");
    ctx->tuning = *t;
    return MRF_OK;
}

mrf_status mrf_autotune(mrf_context *ctx, const mrf_field *field, const mrf_bvh *bvh, const mrf_rays *rays,
                        uint32_t max_bounces, const mrf_render_opts *opts, float *out_hdr, void *stream, uint32_t reps,
                        mrf_tuning *best, float *ms) {
    if (!ctx || !opts || reps == 0) return fail(MRF_ERR_INVALID_ARG, "mrf_autotune: NULL argument or reps 0");
    if (opts->kernel_ms || opts->kernel_launches)
        return fail(MRF_ERR_INVALID_ARG, "mrf_autotune: per-kernel timing is not allowed here");
    if (!is_device_ptr(out_hdr)) return fail(MRF_ERR_INVALID_ARG, "mrf_autotune: out_hdr must be device memory");
    CUDA_TRY(cudaSetDevice(ctx->device), "mrf_autotune: cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    const mrf_tuning keep = ctx->tuning;
    const uint32_t groups[2] = {8, 4}, caps[3] = {48, 96, 192}, rounds[2] = {1, 8};
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0), "mrf_autotune: event");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(cudaGetLastError(), "mrf_autotune: event");
    }
    float best_ms = INFINITY;
    mrf_tuning win = keep;
    mrf_status st = MRF_OK;
    int c = 0;
    for (uint32_t g : groups) {
        for (uint32_t cap : caps)
        for (uint32_t rr : rounds) {
            ctx->tuning = mrf_tuning{g, cap, rr, keep.tail_paths};
            float t = INFINITY;
            if ((st = mrf_render(ctx, field, bvh, rays, max_bounces, opts, out_hdr, stream, nullptr))) break;
            cudaEventRecord(e0, s);
            for (uint32_t r = 0; r < reps && !st; ++r)
                st = mrf_render(ctx, field, bvh, rays, max_bounces, opts, out_hdr, stream, nullptr);
            if (st) break;
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
                st = cuda_fail(cudaGetLastError(), "mrf_autotune: timing");
                break;
            }
            t /= (float)reps;
            if (ms) ms[c] = t;
            ++c;
            if (t < best_ms) {
                best_ms = t;
                win = ctx->tuning;
            }
        }
        if (st) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->tuning = st ? keep : win;
    if (best && !st) *best = win;
    return st;
}

// ------------------------------------------------------------ captured frames
struct mrf_frame {
    mrf_context *parent = nullptr;
    mrf_context own;             // private scratch, statistics, status, materials and lights
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

void mrf_frame_destroy(mrf_frame *f) {
    if (!f) return;
    cudaSetDevice(f->own.device);
    if (f->exec) cudaGraphExecDestroy(f->exec);
    if (f->graph) cudaGraphDestroy(f->graph);
    cudaFree(f->own.scratch);
    cudaFree(f->own.stats);
    cudaFree(f->own.status);
    cudaFree(f->own.mats);
    cudaFree(f->own.lights);
    delete f;
}

mrf_status mrf_frame_capture(mrf_context *ctx, const mrf_field *field, const mrf_bvh *bvh, const mrf_rays *rays,
                             uint32_t max_bounces, const mrf_render_opts *opts, float *out_hdr, mrf_frame **out) {
    if (!out) return fail(MRF_ERR_INVALID_ARG, "mrf_frame_capture: NULL argument");
    *out = nullptr;
    RenderPlan R;
    mrf_status st = plan_render(ctx, field, bvh, rays, max_bounces, opts, out_hdr, R);
    if (st) return st;
    if (R.host_out || R.host_rays || opts->kernel_ms || opts->kernel_launches)
        return fail(MRF_ERR_INVALID_ARG, "mrf_frame_capture: outputs and rays must be device memory, no kernel timing");
    CUDA_TRY(cudaSetDevice(ctx->device), "mrf_frame_capture: cudaSetDevice");
    auto *f = new (std::nothrow) mrf_frame();
    if (!f) return fail(MRF_ERR_OOM, "mrf_frame_capture");
    f->parent = ctx;
    mrf_context &fc = f->own;
    fc.device = ctx->device;
    fc.n_mats = ctx->n_mats;
    fc.n_lights = ctx->n_lights;
    fc.n_shadow = ctx->n_shadow;
    fc.tuning = ctx->tuning;
    auto bail = [&](mrf_status e) {
        mrf_frame_destroy(f);
        return e;
    };
    if ((st = dev_alloc(&fc.stats, ST_COUNT, "frame statistics")) || (st = dev_alloc(&fc.status, 1, "frame status")) ||
        (st = dev_alloc(&fc.mats, (size_t)fc.n_mats, "frame materials")) ||
        (st = dev_alloc(&fc.lights, (size_t)fc.n_lights, "frame lights")))
        return bail(st);
    if (cudaMemset(fc.status, 0, sizeof(unsigned)) != cudaSuccess ||
        (fc.n_mats && cudaMemcpy(fc.mats, ctx->mats, sizeof(MaterialDev) * fc.n_mats, cudaMemcpyDeviceToDevice)) ||
        (fc.n_lights && cudaMemcpy(fc.lights, ctx->lights, sizeof(LightDev) * fc.n_lights, cudaMemcpyDeviceToDevice)))
        return bail(cuda_fail(cudaGetLastError(), "mrf_frame_capture: copies"));
    if (R.scratch_need && (st = ensure_scratch(&fc, R.scratch_need))) return bail(st);
    place_render(&fc, R, out_hdr);
    R.P.mats = fc.mats;
    R.P.lights = fc.lights;
    R.P.status = fc.status;
    R.P.stats = fc.stats;
    if (R.n_views && cudaMemcpy((void *)R.P.views, R.views.data(), sizeof(ViewDev) * (size_t)R.n_views,
                                cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "mrf_frame_capture: camera table"));
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "mrf_frame_capture: stream"));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        e = cudaMemsetAsync(fc.stats, 0, sizeof(unsigned long long) * ST_COUNT, cs);
        mrf_status ls = e == cudaSuccess ? launch_render(&fc, R, cs, nullptr) : MRF_ERR_CUDA;
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (ls != MRF_OK || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaStreamDestroy(cs);
            return bail(ls != MRF_OK ? ls : cuda_fail(e2, "mrf_frame_capture: capture"));
        }
        f->graph = g;
        e = cudaGraphInstantiate(&f->exec, g, 0);
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return bail(cuda_fail(e, "mrf_frame_capture: graph"));
    *out = f;
    return MRF_OK;
}

mrf_status mrf_frame_replay(mrf_frame *f, void *stream) {
    if (!f) return fail(MRF_ERR_INVALID_ARG, "mrf_frame_replay: NULL frame");
    CUDA_TRY(cudaSetDevice(f->own.device), "mrf_frame_replay: cudaSetDevice");
    CUDA_TRY(cudaGraphLaunch(f->exec, (cudaStream_t)stream), "mrf_frame_replay");
    return MRF_OK;
}

mrf_status mrf_frame_stats(mrf_frame *f, void *stream, mrf_stats *stats) {
    if (!f || !stats) return fail(MRF_ERR_INVALID_ARG, "mrf_frame_stats: NULL argument");
    CUDA_TRY(cudaSetDevice(f->own.device), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long h[ST_COUNT];
    unsigned st_word = 0;
    CUDA_TRY(cudaMemcpyAsync(h, f->own.stats, sizeof(h), cudaMemcpyDeviceToHost, s), "mrf_frame_stats");
    CUDA_TRY(cudaMemcpyAsync(&st_word, f->own.status, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "mrf_frame_stats");
    CUDA_TRY(cudaStreamSynchronize(s), "mrf_frame_stats: synchronize");
    stats_from(h, st_word, stats);
    if (st_word) {
        cudaMemset(f->own.status, 0, sizeof(unsigned));
        return fail(MRF_ERR_TIMEOUT, "mrf_frame: a kernel gave up (status 0x%x)", st_word);
    }
    return MRF_OK;
}

// Allocation-free render: the wavefront engine on the library's static device
// arena (render_wavefront.cu), whose device address the context resolved when
// it was created.  Nothing here allocates device or pinned memory, and nothing
// blocks the host unless statistics are asked for.
mrf_status mrf_render_static(mrf_context *ctx, const mrf_field *field, const mrf_bvh *bvh, const mrf_rays *rays,
                             uint32_t max_bounces, const mrf_render_opts *opts, float *out_hdr, void *stream,
                             mrf_stats *stats) {
    if (!ctx || !field || !bvh || !rays || !opts || !out_hdr)
        return fail(MRF_ERR_INVALID_ARG, "mrf_render_static: NULL argument");
    if (field->ctx != ctx || bvh->ctx != ctx)
        return fail(MRF_ERR_INVALID_ARG, "mrf_render_static: handle of another context");
    if (max_bounces == 0 || max_bounces > (uint32_t)kMaxBounces)
        return fail(MRF_ERR_INVALID_ARG, "mrf_render_static: max_bounces must be in [1, %d]", kMaxBounces);
    if (rays->spp == 0) return fail(MRF_ERR_INVALID_ARG, "mrf_render_static: spp must be >= 1");
    if (opts->steps_per_segment == 0 && !(opts->dt > 0.f))
        return fail(MRF_ERR_INVALID_ARG, "mrf_render_static: need steps_per_segment > 0 or dt > 0");
    if (!(opts->tau >= 0.f) || !(opts->tmin >= 0.f))
        return fail(MRF_ERR_INVALID_ARG, "mrf_render_static: negative tau or tmin");
    if (opts->kernel_ms || opts->kernel_launches)
        return fail(MRF_ERR_INVALID_ARG, "mrf_render_static: per-kernel timing is not available here");
    if (bvh->n_tris && ctx->n_mats == 0) return fail(MRF_ERR_NOT_READY, "mrf_render_static: no materials set");
    if (ctx->n_shadow > static_arena_max_lights())
        return fail(MRF_ERR_INVALID_ARG, "mrf_render_static: %d shadow rays per hit exceed the arena limit of %d",
                    ctx->n_shadow, static_arena_max_lights());
    CUDA_TRY(cudaSetDevice(ctx->device), "mrf_render_static: cudaSetDevice");
    if (!is_device_ptr(out_hdr)) return fail(MRF_ERR_INVALID_ARG, "mrf_render_static: out_hdr must be device memory");
    if ((opts->rec_segments && !is_device_ptr(opts->rec_segments)) || (opts->rec_tri && !is_device_ptr(opts->rec_tri)) ||
        (opts->rec_t && !is_device_ptr(opts->rec_t)) || (!opts->rec_tri != !opts->rec_t))
        return fail(MRF_ERR_INVALID_ARG, "mrf_render_static: records must be device pointers (rec_tri and rec_t together)");
    {
        cudaError_t pending = cudaGetLastError();
        if (pending != cudaSuccess) return cuda_fail(pending, "mrf_render_static: earlier asynchronous error");
    }
    cudaStream_t s = (cudaStream_t)stream;
    RenderParams P{};
    P.F = field->dev;
    P.B = bvh->dev;
    P.mats = ctx->mats;
    P.n_mats = ctx->n_mats;
    P.lights = ctx->lights;
    P.n_lights = ctx->n_lights;
    P.n_shadow = ctx->n_shadow;
    uint32_t count;
    if (rays->camera && rays->n_cameras > 1)
        return fail(MRF_ERR_UNSUPPORTED, "mrf_render_static: one camera or explicit rays; several views go to mrf_render");
    if (field && field->dev.view_dep)
        return fail(MRF_ERR_UNSUPPORTED, "mrf_render_static: view-dependent fields go to mrf_render");
    if (rays->camera) {
        const mrf_camera &c = *rays->camera;
        if (c.width == 0 || c.height == 0 || !(c.vfov_deg > 0.f && c.vfov_deg < 180.f))
            return fail(MRF_ERR_INVALID_ARG, "mrf_render_static: bad camera");
        const uint64_t cnt = (uint64_t)c.width * c.height;
        if (cnt > 0xFFFFFFFFull / 4) return fail(MRF_ERR_INVALID_ARG, "mrf_render_static: image too large");
        count = (uint32_t)cnt;
        double f[3], up[3], r[3], u[3];
        for (int k = 0; k < 3; ++k) {
            f[k] = (double)c.look_at[k] - c.pos[k];
            up[k] = c.up[k];
        }
        const double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
        if (!(fl > 0)) return fail(MRF_ERR_INVALID_ARG, "mrf_render_static: camera looks at itself");
        for (double &x : f) x /= fl;
        r[0] = f[1] * up[2] - f[2] * up[1];
        r[1] = f[2] * up[0] - f[0] * up[2];
        r[2] = f[0] * up[1] - f[1] * up[0];
        const double rl = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        if (!(rl > 0)) return fail(MRF_ERR_INVALID_ARG, "mrf_render_static: camera up is parallel to the view direction");
        for (double &x : r) x /= rl;
        u[0] = r[1] * f[2] - r[2] * f[1];
        u[1] = r[2] * f[0] - r[0] * f[2];
        u[2] = r[0] * f[1] - r[1] * f[0];
        P.use_camera = 1;
        for (int k = 0; k < 3; ++k) {
            P.cam_pos[k] = c.pos[k];
            P.cam_f[k] = (float)f[k];
            P.cam_r[k] = (float)r[k];
            P.cam_u[k] = (float)u[k];
        }
        P.tan_half = (float)std::tan(0.5 * (double)c.vfov_deg * M_PI / 180.0);
        P.aspect = (float)((double)c.width / (double)c.height);
        P.W = c.width;
        P.H = c.height;
    } else {
        if (!rays->origins || !rays->dirs || rays->count == 0)
            return fail(MRF_ERR_INVALID_ARG, "mrf_render_static: explicit rays need origins, dirs and count > 0");
        if (!is_device_ptr(rays->origins) || !is_device_ptr(rays->dirs))
            return fail(MRF_ERR_INVALID_ARG, "mrf_render_static: explicit rays must be device memory");
        count = rays->count;
        P.ray_o = rays->origins;
        P.ray_d = rays->dirs;
    }
    const uint64_t paths = (uint64_t)count * rays->spp;
    if (paths > static_arena_max_paths())
        return fail(MRF_ERR_INVALID_ARG,
                    "mrf_render_static: %llu paths (rays x spp) exceed the static arena limit of %u; use mrf_render",
                    (unsigned long long)paths, static_arena_max_paths());
    const uint32_t fit = static_arena_paths_that_fit(ctx->n_shadow);
    if (paths > fit)
        return fail(MRF_ERR_INVALID_ARG,
                    "mrf_render_static: %llu paths with %d shadow rays per hit do not fit the static arena "
                    "(at most %u paths at that light count); use mrf_render",
                    (unsigned long long)paths, ctx->n_shadow, fit);
    P.count = count;
    P.spp = rays->spp;
    P.max_bounces = max_bounces;
    P.seed = opts->seed;
    P.steps = opts->steps_per_segment;
    P.dt = opts->dt;
    P.tau = opts->tau;
    P.tmin = opts->tmin;
    P.rec_seg = opts->rec_segments;
    P.rec_tri = opts->rec_tri;
    P.rec_t = opts->rec_t;
    P.tc_groups = (int)ctx->tuning.field_groups;
    P.max_rounds = (int)ctx->tuning.rounds;
    P.tail_paths = ctx->tuning.tail_paths;
    P.shadow_mask = opts->shadow_mask ? 1 : 0;
    if (opts->shadow_net) {
        if (opts->shadow_net->ctx != ctx) return fail(MRF_ERR_INVALID_ARG, "shadow_net belongs to another context");
        P.has_snet = 1;
        P.snet = opts->shadow_net->dev;
    }
    P.out = out_hdr;
    P.status = ctx->status;
    if (ctx->arena_err != cudaSuccess || !ctx->arena)
        return cuda_fail(ctx->arena_err != cudaSuccess ? ctx->arena_err : cudaErrorInvalidSymbol,
                         "mrf_render_static: arena address (cudaGetSymbolAddress at context creation)");
    mrf_status pst = poll_status(ctx, s, "mrf_render_static");
    if (pst) return pst;
    if (stats) {
        CUDA_TRY(cudaMemsetAsync(ctx->stats, 0, sizeof(unsigned long long) * ST_COUNT, s), "stats reset");
        P.stats = ctx->stats;
    }
    CUDA_TRY(launch_render_wavefront_arena(P, ctx->arena, ctx->arena_bytes, s), "mrf_render_static: launch");
    if (stats) {
        unsigned long long h[ST_COUNT];
        CUDA_TRY(cudaMemcpyAsync(h, ctx->stats, sizeof(h), cudaMemcpyDeviceToHost, s), "stats download");
        unsigned st_word = 0;
        if ((pst = read_status_after_sync(ctx, s, st_word, "mrf_render_static: status read"))) return pst;
        stats_from(h, st_word, stats);
        if (st_word) return fail(MRF_ERR_TIMEOUT, "mrf_render_static: a kernel gave up (status 0x%x)", st_word);
        return MRF_OK;
    }
    return post_status(ctx, s, "mrf_render_static: status copy");
}

mrf_status mrf_tonemap(mrf_context *ctx, const float *in, uint32_t n, float exposure, float *out, void *stream) {
    if (!ctx || (n && (!in || !out))) return fail(MRF_ERR_INVALID_ARG, "mrf_tonemap: NULL argument");
    if (!(exposure >= 0.f)) return fail(MRF_ERR_INVALID_ARG, "mrf_tonemap: exposure must be >= 0");
    if (n == 0) return MRF_OK;
    if (!is_device_ptr(in) || !is_device_ptr(out))
        return fail(MRF_ERR_INVALID_ARG, "mrf_tonemap: in and out must be device memory");
    CUDA_TRY(launch_tonemap(reinterpret_cast<const float4 *>(in), n, exposure, reinterpret_cast<float4 *>(out),
                            (cudaStream_t)stream),
             "mrf_tonemap: launch");
    return MRF_OK;
}


// ------------------------------------------------------ shadow network
namespace {
uint64_t snet_params(uint32_t log2T) {
    return ((uint64_t)kSnetLevels << log2T) * 2 + kSnetMlp;
}

uint64_t splitmix_next(uint64_t &x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// uniform in [-a, a) from the top 24 bits of a SplitMix64 stream
float splitmix_uniform(uint64_t &x, float a) {
    return (float)(((double)(splitmix_next(x) >> 40) * (1.0 / 16777216.0) * 2.0 - 1.0) * a);
}

mrf_status snet_refresh(mrf_shadow_net *n, cudaStream_t s) {
    CUDA_TRY(launch_snet_refresh(n->params + (n->n_params - kSnetMlp), n->mlp_inf, n->precision == MRF_PREC_BF16, s),
             "shadow net: refresh");
    if (n->lp) CUDA_TRY(launch_snet_pack_lp(n->params + (n->n_params - kSnetMlp), n->lp, s), "shadow net: pack");
    return MRF_OK;
}
}  // namespace

mrf_status mrf_shadow_net_create(mrf_context *ctx, const mrf_field *field, const mrf_shadow_net_desc *desc,
                                 mrf_shadow_net **out) {
    if (!ctx || !field || !desc || !out) return fail(MRF_ERR_INVALID_ARG, "mrf_shadow_net_create: NULL argument");
    *out = nullptr;
    if (desc->log2_table < 10 || desc->log2_table > 22)
        return fail(MRF_ERR_INVALID_ARG, "mrf_shadow_net_create: log2_table must be 10..22");
    for (int l = 0; l < kSnetLevels; ++l)
        if (desc->level_res[l] < 2 || desc->level_res[l] > 4096)
            return fail(MRF_ERR_INVALID_ARG, "mrf_shadow_net_create: level_res must be 2..4096");
    if (desc->precision != MRF_PREC_FP32 && desc->precision != MRF_PREC_BF16)
        return fail(MRF_ERR_INVALID_ARG, "mrf_shadow_net_create: precision must be FP32 or BF16");
    if (!(desc->lr > 0.f) || !(desc->beta1 >= 0.f && desc->beta1 < 1.f) || !(desc->beta2 >= 0.f && desc->beta2 < 1.f) ||
        !(desc->eps >= 0.f))
        return fail(MRF_ERR_INVALID_ARG, "mrf_shadow_net_create: bad Adam parameters");
    CUDA_TRY(cudaSetDevice(ctx->device), "mrf_shadow_net_create: cudaSetDevice");
    auto *n = new (std::nothrow) mrf_shadow_net();
    if (!n) return fail(MRF_ERR_OOM, "mrf_shadow_net_create");
    n->ctx = ctx;
    n->lr = desc->lr;
    n->b1 = desc->beta1;
    n->b2 = desc->beta2;
    n->eps = desc->eps;
    n->decay = desc->lr_decay > 0.f ? desc->lr_decay : 1.f;
    if (!(n->decay <= 1.f)) {
        delete n;
        return fail(MRF_ERR_INVALID_ARG, "mrf_shadow_net_create: lr_decay must be in (0, 1]");
    }
    n->precision = desc->precision;
    n->n_params = snet_params(desc->log2_table);
    ShadowNetDev &D = n->dev;
    D.log2T = desc->log2_table;
    const uint64_t T = 1ull << desc->log2_table;
    for (int l = 0; l < kSnetLevels; ++l) {
        D.res[l] = desc->level_res[l];
        const uint64_t s1 = desc->level_res[l] + 1ull;
        if (s1 * s1 * s1 <= T) D.dense_mask |= 1u << l;
    }
    const FieldDev &F = field->dev;
    for (int a = 0; a < 3; ++a) {
        D.lo[a] = F.lo[a];
        D.hi[a] = F.hi[a];
        D.ext_inv[a] = F.ext_inv[a];
    }
    D.has_pose = F.has_pose;
    for (int k = 0; k < 12; ++k) D.to_local[k] = F.to_local[k];
    mrf_status st;
    if ((st = dev_alloc(&n->params, n->n_params, "shadow net parameters")) ||
        (st = dev_alloc(&n->m, n->n_params, "shadow net Adam m")) ||
        (st = dev_alloc(&n->v, n->n_params, "shadow net Adam v")) ||
        (st = dev_alloc(&n->grad, n->n_params, "shadow net gradient")) ||
        (st = dev_alloc(&n->mlp_inf, (size_t)kSnetMlp + 4, "shadow net rendering weights")) ||
        (desc->precision == MRF_PREC_BF16 && (st = dev_alloc(&n->lp, snet_lp_bytes(), "shadow net BF16 weights")))) {
        mrf_shadow_net_destroy(n);
        return st;
    }
    D.table = n->params;
    D.mlp = n->mlp_inf;
    D.lp = n->lp;
    if (desc->params) {
        if (cudaMemcpy(n->params, desc->params, n->n_params * sizeof(float), cudaMemcpyDefault) != cudaSuccess) {
            mrf_shadow_net_destroy(n);
            return fail(MRF_ERR_INVALID_ARG, "mrf_shadow_net_create: cannot read params");
        }
    } else {
        std::vector<float> h(n->n_params, 0.f);
        uint64_t x = desc->seed;
        const uint64_t tbl = n->n_params - kSnetMlp;
        for (uint64_t i = 0; i < tbl; ++i) h[i] = splitmix_uniform(x, 1e-4f);
        float *w = h.data() + tbl;
        const int fan[4][2] = {{kSnetW, kSnetIn}, {kSnetW, kSnetW}, {kSnetW, kSnetW}, {1, kSnetW}};
        const int off[4] = {0, kSnetOffW2, kSnetOffW3, kSnetOffW4};
        for (int L = 0; L < 4; ++L) {
            const float a = (float)std::sqrt(6.0 / (fan[L][0] + fan[L][1]));
            for (int i = 0; i < fan[L][0] * fan[L][1]; ++i) w[off[L] + i] = splitmix_uniform(x, a);
        }
        if (cudaMemcpy(n->params, h.data(), n->n_params * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
            mrf_shadow_net_destroy(n);
            return fail(MRF_ERR_CUDA, "mrf_shadow_net_create: upload");
        }
    }
    if (cudaMemset(n->m, 0, n->n_params * sizeof(float)) != cudaSuccess ||
        cudaMemset(n->v, 0, n->n_params * sizeof(float)) != cudaSuccess ||
        cudaMemset(n->grad, 0, n->n_params * sizeof(unsigned long long)) != cudaSuccess || (st = snet_refresh(n, 0)) ||
        cudaDeviceSynchronize() != cudaSuccess) {
        mrf_shadow_net_destroy(n);
        return st ? st : fail(MRF_ERR_CUDA, "mrf_shadow_net_create: initialisation");
    }
    *out = n;
    return MRF_OK;
}

void mrf_shadow_net_destroy(mrf_shadow_net *n) {
    if (!n) return;
    cudaSetDevice(n->ctx->device);
    cudaFree(n->params);
    cudaFree(n->m);
    cudaFree(n->v);
    cudaFree(n->grad);
    cudaFree(n->mlp_inf);
    cudaFree(n->lp);
    delete n;
}

uint64_t mrf_shadow_net_param_count(const mrf_shadow_net *n) { return n ? n->n_params : 0; }

mrf_status mrf_shadow_net_get_params(const mrf_shadow_net *n, float *out, void *stream) {
    if (!n || !out) return fail(MRF_ERR_INVALID_ARG, "mrf_shadow_net_get_params: NULL argument");
    CUDA_TRY(cudaSetDevice(n->ctx->device), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(out, n->params, n->n_params * sizeof(float), cudaMemcpyDefault, s), "get params");
    if (!is_device_ptr(out)) CUDA_TRY(cudaStreamSynchronize(s), "get params: synchronize");
    return MRF_OK;
}

mrf_status mrf_shadow_net_set_params(mrf_shadow_net *n, const float *in, void *stream) {
    if (!n || !in) return fail(MRF_ERR_INVALID_ARG, "mrf_shadow_net_set_params: NULL argument");
    CUDA_TRY(cudaSetDevice(n->ctx->device), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(n->params, in, n->n_params * sizeof(float), cudaMemcpyDefault, s), "set params");
    CUDA_TRY(cudaMemsetAsync(n->m, 0, n->n_params * sizeof(float), s), "set params");
    CUDA_TRY(cudaMemsetAsync(n->v, 0, n->n_params * sizeof(float), s), "set params");
    n->t = 0;
    mrf_status st = snet_refresh(n, s);
    if (st) return st;
    if (!is_device_ptr(in)) CUDA_TRY(cudaStreamSynchronize(s), "set params: synchronize");
    return MRF_OK;
}

mrf_status mrf_shadow_pairs(mrf_context *ctx, const mrf_field *field, const mrf_render_opts *opts, uint64_t seed,
                            uint64_t first, uint32_t n, float *out, void *stream) {
    if (!ctx || !field || !opts || (!out && n)) return fail(MRF_ERR_INVALID_ARG, "mrf_shadow_pairs: NULL argument");
    if (ctx->n_lights < 1) return fail(MRF_ERR_INVALID_ARG, "mrf_shadow_pairs: the context has no lights");
    if (n && !is_device_ptr(out)) return fail(MRF_ERR_INVALID_ARG, "mrf_shadow_pairs: out must be device memory");
    if (opts->steps_per_segment == 0 && !(opts->dt > 0.f))
        return fail(MRF_ERR_INVALID_ARG, "mrf_shadow_pairs: need steps_per_segment > 0 or dt > 0");
    CUDA_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    RenderParams P{};
    P.F = field->dev;
    P.lights = ctx->lights;
    P.n_lights = ctx->n_lights;
    P.steps = opts->steps_per_segment;
    P.dt = opts->dt;
    P.tmin = opts->tmin;
    P.status = ctx->status;
    CUDA_TRY(launch_snet_pairs(P, seed, first, n, out, (cudaStream_t)stream), "mrf_shadow_pairs");
    return MRF_OK;
}

mrf_status mrf_shadow_net_grad(mrf_shadow_net *n, const float *pairs, uint32_t count, float *grad, float *loss,
                               void *stream) {
    if (!n || !pairs || !grad || !loss || count == 0)
        return fail(MRF_ERR_INVALID_ARG, "mrf_shadow_net_grad: NULL argument or no pairs");
    if (!is_device_ptr(pairs) || !is_device_ptr(grad) || !is_device_ptr(loss))
        return fail(MRF_ERR_INVALID_ARG, "mrf_shadow_net_grad: arrays must be device memory");
    CUDA_TRY(cudaSetDevice(n->ctx->device), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(float), s), "loss clear");
    CUDA_TRY(launch_snet_grad(n->dev, n->params, n->grad, pairs, count, 0, count, loss, s), "mrf_shadow_net_grad");
    CUDA_TRY(launch_snet_grad_out(n->grad, grad, n->n_params, s), "mrf_shadow_net_grad: output");
    return MRF_OK;
}

mrf_status mrf_shadow_net_train(mrf_shadow_net *n, const float *pairs, uint64_t n_pairs, uint32_t batch,
                                uint32_t steps, float *loss, void *stream) {
    if (!n || !pairs || n_pairs == 0 || batch == 0)
        return fail(MRF_ERR_INVALID_ARG, "mrf_shadow_net_train: NULL argument, no pairs or batch 0");
    if (!is_device_ptr(pairs) || (loss && !is_device_ptr(loss)))
        return fail(MRF_ERR_INVALID_ARG, "mrf_shadow_net_train: arrays must be device memory");
    CUDA_TRY(cudaSetDevice(n->ctx->device), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    if (loss) CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(float) * (size_t)steps, s), "loss clear");
    for (uint32_t k = 0; k < steps; ++k) {
        CUDA_TRY(launch_snet_grad(n->dev, n->params, n->grad, pairs, n_pairs, n->cursor % n_pairs, batch,
                                  loss ? loss + k : nullptr, s),
                 "mrf_shadow_net_train: gradient");
        n->cursor = (n->cursor + batch) % n_pairs;
        ++n->t;
        const double c1 = 1.0 - std::pow((double)n->b1, (double)n->t), c2 = 1.0 - std::pow((double)n->b2, (double)n->t);
        const float lr_t = (float)((double)n->lr * std::pow((double)n->decay, (double)(n->t - 1)));
        CUDA_TRY(launch_snet_adam(n->params, n->m, n->v, n->grad, n->n_params, lr_t, n->b1, n->b2, n->eps, c1, c2, s),
                 "mrf_shadow_net_train: Adam");
    }
    return snet_refresh(n, s);
}

mrf_status mrf_shadow_net_eval(mrf_shadow_net *n, const float *pairs, uint32_t count, float *out, void *stream) {
    if (!n || (count && (!pairs || !out))) return fail(MRF_ERR_INVALID_ARG, "mrf_shadow_net_eval: NULL argument");
    if (count && (!is_device_ptr(pairs) || !is_device_ptr(out)))
        return fail(MRF_ERR_INVALID_ARG, "mrf_shadow_net_eval: arrays must be device memory");
    CUDA_TRY(cudaSetDevice(n->ctx->device), "cudaSetDevice");
    CUDA_TRY(launch_snet_eval(n->dev, pairs, count, out, (cudaStream_t)stream), "mrf_shadow_net_eval");
    return MRF_OK;
}


// ------------------------------------------------------------ diagnostics
mrf_status mrf_l2_read_bandwidth(mrf_context *ctx, uint64_t bytes, uint32_t reps, void *stream, double *gbs) {
    if (!ctx || !gbs) return fail(MRF_ERR_INVALID_ARG, "mrf_l2_read_bandwidth: NULL argument");
    if (bytes < (1u << 20) || bytes > (256ull << 20) || bytes % 16 || reps == 0 || reps > 1000)
        return fail(MRF_ERR_INVALID_ARG, "mrf_l2_read_bandwidth: bytes must be a multiple of 16 in [1 MiB, 256 MiB], "
                                         "reps in [1, 1000]");
    CUDA_TRY(cudaSetDevice(ctx->device), "mrf_l2_read_bandwidth: cudaSetDevice");
    mrf_status st = ensure_scratch(ctx, bytes + 256);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    float *sink = reinterpret_cast<float *>(static_cast<char *>(ctx->scratch) + bytes);
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0), "mrf_l2_read_bandwidth: event");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(cudaGetLastError(), "mrf_l2_read_bandwidth: event");
    }
    float ms = 0.f;
    cudaError_t e = launch_l2_fill(ctx->scratch, bytes, sink, s);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch_l2_read(ctx->scratch, bytes, (int)reps, sink, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "mrf_l2_read_bandwidth");
    *gbs = (double)bytes * reps / ((double)ms * 1e-3) / 1e9;
    return MRF_OK;
}

// ------------------------------------------------------------ self tests
void mrf_debug_fail_allocations(uint32_t n) { g_fail_allocs.store(n); }

mrf_status mrf_selftest_timeout(mrf_context *ctx, uint64_t cycles, int32_t wait) {
    if (!ctx) return fail(MRF_ERR_INVALID_ARG, "mrf_selftest_timeout: NULL context");
    if (cycles > (1ull << 32)) return fail(MRF_ERR_INVALID_ARG, "mrf_selftest_timeout: budget above 2^32 cycles");
    CUDA_TRY(cudaSetDevice(ctx->device), "mrf_selftest_timeout: cudaSetDevice");
    CUDA_TRY(launch_selftest_timeout((long long)cycles, ctx->status, 0), "mrf_selftest_timeout: launch");
    if (!wait) return post_status(ctx, 0, "mrf_selftest_timeout: status copy");
    CUDA_TRY(cudaDeviceSynchronize(), "mrf_selftest_timeout: synchronize");
    unsigned st_word = 0;
    CUDA_TRY(cudaMemcpy(&st_word, ctx->status, sizeof(unsigned), cudaMemcpyDeviceToHost), "mrf_selftest_timeout: status");
    if (st_word) {
        cudaMemset(ctx->status, 0, sizeof(unsigned));
        return fail(MRF_ERR_TIMEOUT, "mrf_selftest_timeout: the wait gave up (status 0x%x)", st_word);
    }
    return MRF_OK;
}


// ------------------------------------------------------------ shadow network checkpoints
namespace {
constexpr char kSnetMagic[8] = {'M', 'R', 'F', 'S', 'N', 'E', 'T', '1'};
struct SnetHeader {
    char magic[8];
    uint32_t log2T, res[kSnetLevels];
    uint64_t n_params;
    uint32_t t;
    uint64_t cursor;
    float lr, b1, b2, eps, decay;
    int32_t precision;
};
}  // namespace

mrf_status mrf_shadow_net_save(const mrf_shadow_net *n, const char *path) {
    if (!n || !path) return fail(MRF_ERR_INVALID_ARG, "mrf_shadow_net_save: NULL argument");
    CUDA_TRY(cudaSetDevice(n->ctx->device), "cudaSetDevice");
    CUDA_TRY(cudaDeviceSynchronize(), "mrf_shadow_net_save: synchronize");
    SnetHeader h{};
    std::memcpy(h.magic, kSnetMagic, 8);
    h.log2T = n->dev.log2T;
    for (int l = 0; l < kSnetLevels; ++l) h.res[l] = n->dev.res[l];
    h.n_params = n->n_params;
    h.t = n->t;
    h.cursor = n->cursor;
    h.lr = n->lr;
    h.b1 = n->b1;
    h.b2 = n->b2;
    h.eps = n->eps;
    h.decay = n->decay;
    h.precision = n->precision;
    std::vector<float> buf(n->n_params);
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(MRF_ERR_INVALID_ARG, "mrf_shadow_net_save: cannot open %s", path);
    bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1;
    const float *arrays[3] = {n->params, n->m, n->v};
    for (const float *a : arrays) {
        if (!ok) break;
        if (cudaMemcpy(buf.data(), a, n->n_params * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) {
            std::fclose(f);
            return cuda_fail(cudaGetLastError(), "mrf_shadow_net_save: download");
        }
        ok = std::fwrite(buf.data(), sizeof(float), n->n_params, f) == n->n_params;
    }
    ok = (std::fclose(f) == 0) && ok;
    return ok ? MRF_OK : fail(MRF_ERR_INVALID_ARG, "mrf_shadow_net_save: write to %s failed", path);
}

mrf_status mrf_shadow_net_load(mrf_shadow_net *n, const char *path) {
    if (!n || !path) return fail(MRF_ERR_INVALID_ARG, "mrf_shadow_net_load: NULL argument");
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(MRF_ERR_INVALID_ARG, "mrf_shadow_net_load: cannot open %s", path);
    SnetHeader h{};
    bool ok = std::fread(&h, sizeof(h), 1, f) == 1 && std::memcmp(h.magic, kSnetMagic, 8) == 0;
    ok = ok && h.log2T == n->dev.log2T && h.n_params == n->n_params;
    for (int l = 0; ok && l < kSnetLevels; ++l) ok = h.res[l] == n->dev.res[l];
    if (!ok) {
        std::fclose(f);
        return fail(MRF_ERR_INVALID_ARG, "mrf_shadow_net_load: %s is not a checkpoint of this network shape", path);
    }
    std::vector<float> buf(n->n_params);
    float *arrays[3] = {n->params, n->m, n->v};
    mrf_status st = MRF_OK;
    for (float *a : arrays) {
        if (std::fread(buf.data(), sizeof(float), n->n_params, f) != n->n_params) {
            st = fail(MRF_ERR_INVALID_ARG, "mrf_shadow_net_load: %s is truncated", path);
            break;
        }
        if (cudaMemcpy(a, buf.data(), n->n_params * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
            st = cuda_fail(cudaGetLastError(), "mrf_shadow_net_load: upload");
            break;
        }
    }
    std::fclose(f);
    if (st) return st;
    n->t = h.t;
    n->cursor = h.cursor;
    n->lr = h.lr;
    n->b1 = h.b1;
    n->b2 = h.b2;
    n->eps = h.eps;
    n->decay = h.decay;
    if ((st = snet_refresh(n, 0))) return st;
    CUDA_TRY(cudaDeviceSynchronize(), "mrf_shadow_net_load: synchronize");
    return MRF_OK;
}
