// Device building blocks of the hybrid light-transport loop (FP32 unless noted).
#pragma once
#include <cuda_fp16.h>
#include <cstdint>

#include "common.h"

namespace mrf {

// ------------------------------------------------------------------ vectors
struct V3 {
    float x, y, z;
};
__device__ __forceinline__ V3 v3(float x, float y, float z) { return V3{x, y, z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ V3 operator*(V3 a, float s) { return v3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
    return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ V3 normalize(V3 a) { return a * rsqrtf(dot(a, a)); }
__device__ __forceinline__ float comp(V3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }
__device__ __forceinline__ V3 fma3(V3 a, float s, V3 b) {  // a * s + b
    return v3(fmaf(a.x, s, b.x), fmaf(a.y, s, b.y), fmaf(a.z, s, b.z));
}

struct D3 {
    double x, y, z;
};
__device__ __forceinline__ D3 d3(V3 a) { return D3{a.x, a.y, a.z}; }
__device__ __forceinline__ D3 operator-(D3 a, D3 b) { return D3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ double dot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ D3 cross(D3 a, D3 b) {
    return D3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// ------------------------------------------------------------ Philox4x64-10
// Counter-based generator of Salmon et al. (SC'11), 10 rounds.
__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t m0 = 0xD2E7470EE14C6C93ull, m1 = 0xCA5A826395121157ull;
        uint64_t hi0 = __umul64hi(m0, c[0]), lo0 = m0 * c[0];
        uint64_t hi1 = __umul64hi(m1, c[2]), lo1 = m1 * c[2];
        uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += 0x9E3779B97F4A7C15ull;
        k1 += 0xBB67AE8584CAA73Bull;
    }
}
// 24-bit uniform in [0, 1): exact in FP32
__device__ __forceinline__ float u24(uint64_t x) { return (float)(uint32_t)(x >> 40) * (1.0f / 16777216.0f); }

// ------------------------------------------------------------------ box
// Slab test against [lo, hi]; returns false if the ray misses the box.
__device__ __forceinline__ bool box_interval(const float lo[3], const float hi[3], V3 o, V3 d, float &t0,
                                             float &t1) {
    float a = -INFINITY, b = INFINITY;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float ok = comp(o, k), dk = comp(d, k);
        if (dk == 0.0f) {
            if (ok < lo[k] || ok > hi[k]) return false;
            continue;
        }
        float ta = (lo[k] - ok) / dk, tb = (hi[k] - ok) / dk;
        a = fmaxf(a, fminf(ta, tb));
        b = fminf(b, fmaxf(ta, tb));
    }
    t0 = a;
    t1 = b;
    return b > a;
}

// World ray to the field's local frame (rigid pose; identity when absent):
// o' = R^T (o - t), d' = R^T d.  Ray parameters and lengths are unchanged.
__device__ __forceinline__ void to_field_frame(const FieldDev &F, V3 &o, V3 &d) {
    if (!F.has_pose) return;
    const float *M = F.to_local;
    const V3 q = o, e = d;
    o = v3(fmaf(M[0], q.x, fmaf(M[1], q.y, fmaf(M[2], q.z, M[3]))),
           fmaf(M[4], q.x, fmaf(M[5], q.y, fmaf(M[6], q.z, M[7]))),
           fmaf(M[8], q.x, fmaf(M[9], q.y, fmaf(M[10], q.z, M[11]))));
    d = v3(fmaf(M[0], e.x, fmaf(M[1], e.y, M[2] * e.z)), fmaf(M[4], e.x, fmaf(M[5], e.y, M[6] * e.z)),
           fmaf(M[8], e.x, fmaf(M[9], e.y, M[10] * e.z)));
}

// Local point of the field back to world space: p = R p' + t, with R and t
// recovered from the stored world-to-local [R^T | -R^T t].
__device__ __forceinline__ V3 field_to_world(const FieldDev &F, V3 q) {
    if (!F.has_pose) return q;
    const float *M = F.to_local;
    const V3 t = v3(-(M[0] * M[3] + M[4] * M[7] + M[8] * M[11]), -(M[1] * M[3] + M[5] * M[7] + M[9] * M[11]),
                    -(M[2] * M[3] + M[6] * M[7] + M[10] * M[11]));
    return v3(fmaf(M[0], q.x, fmaf(M[4], q.y, fmaf(M[8], q.z, t.x))),
              fmaf(M[1], q.x, fmaf(M[5], q.y, fmaf(M[9], q.z, t.y))),
              fmaf(M[2], q.x, fmaf(M[6], q.y, fmaf(M[10], q.z, t.z))));
}

// ------------------------------------------------------------- field: analytic
__device__ __forceinline__ bool inside_field_box(const FieldDev &F, V3 p) {
    return p.x >= F.lo[0] && p.x <= F.hi[0] && p.y >= F.lo[1] && p.y <= F.hi[1] && p.z >= F.lo[2] &&
           p.z <= F.hi[2];
}

__device__ __forceinline__ float gauss_field(const FieldDev &F, V3 p, float rgb[3]) {
    float s = 0.f, se0 = 0.f, se1 = 0.f, se2 = 0.f;
    for (int k = 0; k < F.n_blobs; ++k) {
        float4 a = __ldg(F.blob_a + k), b = __ldg(F.blob_b + k);
        float dx = p.x - a.x, dy = p.y - a.y, dz = p.z - a.z;
        float sk = b.x * expf(-(dx * dx + dy * dy + dz * dz) * a.w);
        s += sk;
        se0 = fmaf(sk, b.y, se0);
        se1 = fmaf(sk, b.z, se1);
        se2 = fmaf(sk, b.w, se2);
    }
    if (s > 0.f) {
        float inv = 1.0f / s;
        rgb[0] = se0 * inv; rgb[1] = se1 * inv; rgb[2] = se2 * inv;
    } else {
        rgb[0] = rgb[1] = rgb[2] = 0.f;
    }
    return s;
}

// compact support of the hash field: max_k max(0, 1 - |p - c_k|^2 / r_k^2)
__device__ __forceinline__ float field_support(const FieldDev &F, V3 p) {
    float s = 0.f;
    for (int k = 0; k < F.n_support; ++k) {
        float4 c = __ldg(F.support + k);
        float dx = p.x - c.x, dy = p.y - c.y, dz = p.z - c.z;
        s = fmaxf(s, 1.0f - (dx * dx + dy * dy + dz * dz) * c.w);
    }
    return s;
}

// occupancy bit of the cell containing p (p inside the box)
__device__ __forceinline__ bool occupied(const FieldDev &F, V3 p, int c[3]) {
    const int R = F.occ_res;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int ck = (int)floorf((comp(p, k) - F.lo[k]) * F.occ_scale[k]);
        c[k] = min(max(ck, 0), R - 1);
    }
    uint32_t i = (uint32_t)c[0] + (uint32_t)R * ((uint32_t)c[1] + (uint32_t)R * (uint32_t)c[2]);
    return (__ldg(F.occ + (i >> 5)) >> (i & 31)) & 1u;
}

// ray parameter where the ray leaves occupancy cell c
__device__ __forceinline__ float cell_exit(const FieldDev &F, const int c[3], V3 o, V3 inv_d) {
    float t = INFINITY;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float ik = comp(inv_d, k);
        if (isinf(ik)) continue;
        float edge = F.lo[k] + (float)(c[k] + (ik > 0.f ? 1 : 0)) / F.occ_scale[k];
        t = fminf(t, (edge - comp(o, k)) * ik);
    }
    return t;
}

// --------------------------------------------------------- hash encoding
// Level-l features (2 per level) at p: trilinear blend of the 8 cell corners.
__device__ __forceinline__ float2 hash_level(const FieldDev &F, int l, V3 p) {
    const uint32_t N = F.res[l];
    const uint32_t T = 1u << F.log2T;
    const bool dense = (F.dense_mask >> l) & 1u;
    int c[3];
    float w[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float u = (comp(p, k) - F.lo[k]) * F.ext_inv[k] * (float)N;
        float fl = floorf(u);
        fl = fminf(fmaxf(fl, 0.f), (float)(N - 1));
        c[k] = (int)fl;
        w[k] = u - fl;
    }
    const uint32_t *tab = F.table + (size_t)l * T;
    float f0 = 0.f, f1 = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        uint32_t x = c[0] + (k & 1), y = c[1] + ((k >> 1) & 1), z = c[2] + ((k >> 2) & 1);
        uint32_t idx = dense ? x + (N + 1) * (y + (N + 1) * z) : ((x ^ (y * 2654435761u) ^ (z * 805459861u)) & (T - 1));
        float wt = ((k & 1) ? w[0] : 1.f - w[0]) * (((k >> 1) & 1) ? w[1] : 1.f - w[1]) *
                   (((k >> 2) & 1) ? w[2] : 1.f - w[2]);
        uint32_t e = __ldg(tab + checked_index(idx, T, F.status));
        __half2 h = *reinterpret_cast<__half2 *>(&e);
        float2 v = __half22float2(h);
        f0 = fmaf(wt, v.x, f0);
        f1 = fmaf(wt, v.y, f1);
    }
    return make_float2(f0, f1);
}

__device__ __forceinline__ float softplusf(float x) { return fmaxf(x, 0.f) + log1pf(expf(-fabsf(x))); }

// Real spherical harmonics of bands 0..3 at the unit direction w, orthonormal
// on the sphere, ordered (l, m = -l..l).  Constants: 1/(2 sqrt(pi)),
// sqrt(3/(4 pi)), sqrt(15/pi)/2, sqrt(5/pi)/4, sqrt(15/pi)/4, sqrt(35/(2 pi))/4,
// sqrt(105/pi)/2, sqrt(21/(2 pi))/4, sqrt(7/pi)/4, sqrt(105/pi)/4.
__device__ __forceinline__ void sh16(V3 w, float *Y) {
    const float x = w.x, y = w.y, z = w.z;
    Y[0] = 0.28209479177387814f;
    Y[1] = 0.4886025119029199f * y;
    Y[2] = 0.4886025119029199f * z;
    Y[3] = 0.4886025119029199f * x;
    Y[4] = 1.0925484305920792f * x * y;
    Y[5] = 1.0925484305920792f * y * z;
    Y[6] = 0.31539156525252005f * (3.f * z * z - 1.f);
    Y[7] = 1.0925484305920792f * x * z;
    Y[8] = 0.5462742152960396f * (x * x - y * y);
    Y[9] = 0.5900435899266435f * y * (3.f * x * x - y * y);
    Y[10] = 2.890611442640554f * x * y * z;
    Y[11] = 0.4570457994644658f * y * (5.f * z * z - 1.f);
    Y[12] = 0.3731763325901154f * z * (5.f * z * z - 3.f);
    Y[13] = 0.4570457994644658f * x * (5.f * z * z - 1.f);
    Y[14] = 1.445305721320277f * z * (x * x - y * y);
    Y[15] = 0.5900435899266435f * x * (x * x - 3.f * y * y);
}

// Hash-grid field in FP32: encoding + MLP (weights `w` packed as in mlp_floats,
// normally staged in shared memory).  Returns sigma; fills rgb when want_rgb.
template <bool want_rgb>
__device__ __forceinline__ float hash_field_fp32(const FieldDev &F, const float *__restrict__ w, V3 p, float s,
                                                 float rgb[3]) {
    const int n_in = F.n_in;
    const float *W1T = w, *b1 = w + n_in * 64, *W2 = b1 + 64, *b2 = W2 + 64 * 64, *W3T = b2 + 64, *b3 = W3T + 256;
    float h1[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) h1[j] = b1[j];
    for (int l = 0; l < F.n_levels; ++l) {
        float2 f = hash_level(F, l, p);
        const float4 *ra = reinterpret_cast<const float4 *>(W1T + (2 * l) * 64);
        const float4 *rb = reinterpret_cast<const float4 *>(W1T + (2 * l + 1) * 64);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            float4 a = ra[j], b = rb[j];
            h1[4 * j + 0] = fmaf(a.x, f.x, fmaf(b.x, f.y, h1[4 * j + 0]));
            h1[4 * j + 1] = fmaf(a.y, f.x, fmaf(b.y, f.y, h1[4 * j + 1]));
            h1[4 * j + 2] = fmaf(a.z, f.x, fmaf(b.z, f.y, h1[4 * j + 2]));
            h1[4 * j + 3] = fmaf(a.w, f.x, fmaf(b.w, f.y, h1[4 * j + 3]));
        }
    }
#pragma unroll
    for (int j = 0; j < 64; ++j) h1[j] = fmaxf(h1[j], 0.f);
    float o0 = b3[0], o1 = b3[1], o2 = b3[2], o3 = b3[3];
#pragma unroll 4
    for (int j = 0; j < 64; ++j) {
        const float4 *row = reinterpret_cast<const float4 *>(W2 + j * 64);
        float a = b2[j];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            float4 r = row[i];
            a = fmaf(r.x, h1[4 * i + 0], a);
            a = fmaf(r.y, h1[4 * i + 1], a);
            a = fmaf(r.z, h1[4 * i + 2], a);
            a = fmaf(r.w, h1[4 * i + 3], a);
        }
        a = fmaxf(a, 0.f);
        float4 w3 = *reinterpret_cast<const float4 *>(W3T + 4 * j);
        o0 = fmaf(w3.x, a, o0);
        o1 = fmaf(w3.y, a, o1);
        o2 = fmaf(w3.z, a, o2);
        o3 = fmaf(w3.w, a, o3);
    }
    if (want_rgb) {
        rgb[0] = softplusf(o1);
        rgb[1] = softplusf(o2);
        rgb[2] = softplusf(o3);
    }
    return s * expf(fminf(o0, 15.f));
}

// View-dependent hash field in FP32: layer 1 as above, a 16-output density
// head (sigma from output 0), and when want_rgb a colour network of those 16
// outputs and sh16 of the unit view direction d (field frame): 32 -> 64 ->
// 64 -> 3, r = softplus.  Weights: mlp_floats(n_in) floats, then kViewFloats.
template <bool want_rgb>
__device__ __noinline__ float hash_field_view(const FieldDev &F, const float *__restrict__ w, V3 p, V3 d, float s,
                                              float rgb[3]) {
    const int n_in = F.n_in;
    const float *W1T = w, *b1 = w + n_in * 64;
    const float *WdT = w + mlp_floats(n_in), *bd = WdT + 64 * 16, *Wc1T = bd + 16, *bc1 = Wc1T + 32 * 64,
                *Wc2 = bc1 + 64, *bc2 = Wc2 + 64 * 64, *Wc3T = bc2 + 64, *bc3 = Wc3T + 256;
    float h1[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) h1[j] = b1[j];
    for (int l = 0; l < F.n_levels; ++l) {
        float2 f = hash_level(F, l, p);
        const float4 *ra = reinterpret_cast<const float4 *>(W1T + (2 * l) * 64);
        const float4 *rb = reinterpret_cast<const float4 *>(W1T + (2 * l + 1) * 64);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            float4 a = ra[j], b = rb[j];
            h1[4 * j + 0] = fmaf(a.x, f.x, fmaf(b.x, f.y, h1[4 * j + 0]));
            h1[4 * j + 1] = fmaf(a.y, f.x, fmaf(b.y, f.y, h1[4 * j + 1]));
            h1[4 * j + 2] = fmaf(a.z, f.x, fmaf(b.z, f.y, h1[4 * j + 2]));
            h1[4 * j + 3] = fmaf(a.w, f.x, fmaf(b.w, f.y, h1[4 * j + 3]));
        }
    }
    float x[32];
#pragma unroll
    for (int o = 0; o < 16; ++o) x[o] = bd[o];
#pragma unroll 4
    for (int j = 0; j < 64; ++j) {
        const float h = fmaxf(h1[j], 0.f);
        const float4 *r = reinterpret_cast<const float4 *>(WdT + 16 * j);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 a = r[q];
            x[4 * q + 0] = fmaf(a.x, h, x[4 * q + 0]);
            x[4 * q + 1] = fmaf(a.y, h, x[4 * q + 1]);
            x[4 * q + 2] = fmaf(a.z, h, x[4 * q + 2]);
            x[4 * q + 3] = fmaf(a.w, h, x[4 * q + 3]);
        }
    }
    const float sigma = s * expf(fminf(x[0], 15.f));
    if (!want_rgb) return sigma;
    sh16(normalize(d), x + 16);
    float c1[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) c1[j] = bc1[j];
#pragma unroll 4
    for (int i = 0; i < 32; ++i) {
        const float4 *r = reinterpret_cast<const float4 *>(Wc1T + 64 * i);
        const float xi = x[i];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const float4 a = r[q];
            c1[4 * q + 0] = fmaf(a.x, xi, c1[4 * q + 0]);
            c1[4 * q + 1] = fmaf(a.y, xi, c1[4 * q + 1]);
            c1[4 * q + 2] = fmaf(a.z, xi, c1[4 * q + 2]);
            c1[4 * q + 3] = fmaf(a.w, xi, c1[4 * q + 3]);
        }
    }
#pragma unroll
    for (int j = 0; j < 64; ++j) c1[j] = fmaxf(c1[j], 0.f);
    float o0 = bc3[0], o1 = bc3[1], o2 = bc3[2];
#pragma unroll 4
    for (int j = 0; j < 64; ++j) {
        const float4 *row = reinterpret_cast<const float4 *>(Wc2 + j * 64);
        float a = bc2[j];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            float4 r = row[i];
            a = fmaf(r.x, c1[4 * i + 0], a);
            a = fmaf(r.y, c1[4 * i + 1], a);
            a = fmaf(r.z, c1[4 * i + 2], a);
            a = fmaf(r.w, c1[4 * i + 3], a);
        }
        a = fmaxf(a, 0.f);
        const float4 w3 = *reinterpret_cast<const float4 *>(Wc3T + 4 * j);
        o0 = fmaf(w3.x, a, o0);
        o1 = fmaf(w3.y, a, o1);
        o2 = fmaf(w3.z, a, o2);
    }
    rgb[0] = softplusf(o0);
    rgb[1] = softplusf(o1);
    rgb[2] = softplusf(o2);
    return sigma;
}

// ------------------------------------------------------------- intersection
struct Hit {
    float t;
    uint32_t id;     // original triangle index
    int slot;        // triangle slot in BVH order
};

// Moller-Trumbore in FP64 (edge-inclusive), used to settle near-edge cases.
static __device__ __noinline__ bool mt_fp64(V3 of, V3 df, V3 a, V3 b, V3 c, float tmin, float &t_out) {
    D3 o = d3(of), d = d3(df), v0 = d3(a);
    D3 e1 = d3(b) - v0, e2 = d3(c) - v0;
    D3 pv = cross(d, e2);
    double det = dot(e1, pv);
    if (det == 0.0) return false;
    double inv = 1.0 / det;
    D3 tv = o - v0;
    double u = dot(tv, pv) * inv;
    D3 qv = cross(tv, e1);
    double v = dot(d, qv) * inv;
    double t = dot(e2, qv) * inv;
    if (u >= 0.0 && v >= 0.0 && u + v <= 1.0 && t > (double)tmin) {
        t_out = (float)t;
        return true;
    }
    return false;
}

// FP32 Moller-Trumbore with a margin: clear hits and clear misses are decided in
// FP32; anything within the margin of an edge, of t_min, or at grazing
// incidence is re-tested in FP64 (counted in `retests`).
__device__ __forceinline__ bool tri_test(V3 o, V3 d, V3 v0, V3 v1, V3 v2, float tmin, float tmax, float &t_out,
                                         unsigned &retests) {
    const float M = 1e-4f;
    V3 e1 = v1 - v0, e2 = v2 - v0;
    V3 pv = cross(d, e2);
    float det = dot(e1, pv);
    V3 tv = o - v0;
    V3 qv = cross(tv, e1);
    float inv = 1.0f / det;
    float u = dot(tv, pv) * inv, v = dot(d, qv) * inv, t = dot(e2, qv) * inv;
    V3 n = cross(e1, e2);
    bool grazing = !(det * det > 1e-6f * dot(n, n) * dot(d, d));
    if (!grazing) {
        if (u < -M || v < -M || u + v > 1.f + M) return false;
        if (!(t > tmin - 1e-5f) || t > tmax * (1.f + 1e-5f) + 1e-6f) return false;
        if (u > M && v > M && u + v < 1.f - M && t > tmin + 1e-5f) {
            if (t > tmax) return false;
            t_out = t;
            return true;
        }
    }
    ++retests;
    float t64;
    if (mt_fp64(o, d, v0, v1, v2, tmin, t64) && t64 <= tmax) {
        t_out = t64;
        return true;
    }
    return false;
}

__device__ __forceinline__ void load_tri(const BvhDev &B, int slot, V3 &a, V3 &b, V3 &c, uint32_t &id,
                                         uint32_t &mat) {
    float4 p = __ldg(B.tris + 3 * slot), q = __ldg(B.tris + 3 * slot + 1), r = __ldg(B.tris + 3 * slot + 2);
    a = v3(p.x, p.y, p.z);
    b = v3(q.x, q.y, q.z);
    c = v3(r.x, r.y, r.z);
    id = __float_as_uint(p.w);
    mat = __float_as_uint(q.w);
}

// slab test of a child box, padded so that FP32 rounding never culls a box that
// an FP64 test would hit (robust traversal bound of Ize 2013)
__device__ __forceinline__ bool child_hit(float lx, float ly, float lz, float hx, float hy, float hz, V3 o, V3 inv,
                                          float tmax, float &tnear) {
    float tx0 = (lx - o.x) * inv.x, tx1 = (hx - o.x) * inv.x;
    float ty0 = (ly - o.y) * inv.y, ty1 = (hy - o.y) * inv.y;
    float tz0 = (lz - o.z) * inv.z, tz1 = (hz - o.z) * inv.z;
    float a = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.f));
    float b = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), tmax));
    b = b * (1.0f + 4.0e-7f) + 1e-7f;
    a = a * (1.0f - 4.0e-7f) - 1e-7f;
    tnear = a;
    return a <= b;
}

__device__ __forceinline__ void cswap(float &ka, int &va, float &kb, int &vb) {
    if (kb < ka) {
        const float k = ka;
        ka = kb;
        kb = k;
        const int v = va;
        va = vb;
        vb = v;
    }
}

// Closest hit (any_hit = false) or first hit in (tmin, tmax) (any_hit = true),
// skipping the triangle with original id `skip`, over the wide (four-child)
// BVH: a step loads one node (8 x 16 bytes, one memory round trip), tests its
// four child boxes, tests the triangles of the leaf children, visits the
// nearest inner child and pushes the others far to near.  The closest hit does
// not depend on the order of the steps: the closest triangle's boxes all
// contain its hit point, so it is always tested, and ties go to the lower id.
// A leaf's triangles are loaded in batches of kTriBatch before they are
// tested; every caller uses 1 (a batch of 4 shortens a lone slow ray's chain of
// dependent loads, but its registers cost more occupancy than that gains).
// Adds the nodes visited to `visits` and the ray-triangle tests made to
// `tests`.  Returns false and sets `fault` if the traversal stack overflows.
template <bool any_hit, int kTriBatch = 1>
__device__ bool bvh_trace(const BvhDev &B, V3 o, V3 d, uint32_t skip, float tmin, float tmax, Hit &h,
                          unsigned &retests, unsigned &visits, unsigned &tests, bool &fault) {
    h.t = tmax;
    h.id = kNoHit;
    h.slot = -1;
    if (B.n_tris == 0) return false;
    V3 inv = v3(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);
    int stack[kWideStackSize];
    float stack_t[kWideStackSize];
    int sp = 0;
    int node = 0;
    bool found = false;
    int guard = 4 * B.n_nodes + 64;
    while (true) {
        if (--guard < 0) { fault = true; return found; }
        ++visits;
        const float4 *nd = B.wide + 8 * (size_t)checked_index((uint32_t)node, (uint64_t)B.n_nodes, B.status);
        float4 q[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) q[u] = __ldg(nd + u);
        const int ci[4] = {__float_as_int(q[6].x), __float_as_int(q[6].y), __float_as_int(q[6].z),
                           __float_as_int(q[6].w)};
        const int cc[4] = {__float_as_int(q[7].x), __float_as_int(q[7].y), __float_as_int(q[7].z),
                           __float_as_int(q[7].w)};
        float tn[4];
        bool hit[4];
        hit[0] = child_hit(q[0].x, q[1].x, q[2].x, q[3].x, q[4].x, q[5].x, o, inv, h.t, tn[0]);
        hit[1] = child_hit(q[0].y, q[1].y, q[2].y, q[3].y, q[4].y, q[5].y, o, inv, h.t, tn[1]);
        hit[2] = child_hit(q[0].z, q[1].z, q[2].z, q[3].z, q[4].z, q[5].z, o, inv, h.t, tn[2]);
        hit[3] = child_hit(q[0].w, q[1].w, q[2].w, q[3].w, q[4].w, q[5].w, o, inv, h.t, tn[3]);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (!hit[c] || cc[c] <= 0) continue;
            for (int k0 = ci[c]; k0 < ci[c] + cc[c]; k0 += kTriBatch) {
                const int nb = min(kTriBatch, ci[c] + cc[c] - k0);
                float4 tv[kTriBatch][3];
#pragma unroll
                for (int qq = 0; qq < kTriBatch; ++qq)
                    if (qq < nb) {
                        const float4 *tp = B.tris + 3 * checked_index((uint32_t)(k0 + qq), (uint64_t)B.n_tris, B.status);
                        tv[qq][0] = __ldg(tp);
                        tv[qq][1] = __ldg(tp + 1);
                        tv[qq][2] = __ldg(tp + 2);
                    }
#pragma unroll
                for (int qq = 0; qq < kTriBatch; ++qq) {
                    if (qq >= nb) break;
                    const uint32_t id = __float_as_uint(tv[qq][0].w);
                    if (id == skip) continue;
                    ++tests;
                    float t;
                    const V3 a = v3(tv[qq][0].x, tv[qq][0].y, tv[qq][0].z), b = v3(tv[qq][1].x, tv[qq][1].y, tv[qq][1].z),
                             c3 = v3(tv[qq][2].x, tv[qq][2].y, tv[qq][2].z);
                    if (tri_test(o, d, a, b, c3, tmin, h.t, t, retests)) {
                        if (t < h.t || (t == h.t && id < h.id)) {
                            h.t = t;
                            h.id = id;
                            h.slot = k0 + qq;
                            found = true;
                            if (any_hit) return true;
                        }
                    }
                }
            }
        }
        // inner children, nearest first (absent ones sort last)
        float key[4];
        int val[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const bool inner = hit[c] && cc[c] == 0;
            key[c] = inner ? fminf(tn[c], 3.0e38f) : INFINITY;
            val[c] = inner ? ci[c] : -1;
        }
        cswap(key[0], val[0], key[1], val[1]);
        cswap(key[2], val[2], key[3], val[3]);
        cswap(key[0], val[0], key[2], val[2]);
        cswap(key[1], val[1], key[3], val[3]);
        cswap(key[1], val[1], key[2], val[2]);
        if (val[0] >= 0) {
            if (sp + 3 > kWideStackSize) { fault = true; return found; }
#pragma unroll
            for (int c = 3; c >= 1; --c)
                if (val[c] >= 0) {
                    stack_t[sp] = key[c];
                    stack[sp++] = val[c];
                }
            node = val[0];
        } else {
            // pop the next subtree whose box still starts before the best hit
            bool got = false;
            while (sp > 0) {
                --sp;
                if (stack_t[sp] <= h.t) { node = stack[sp]; got = true; break; }
            }
            if (!got) break;
        }
    }
    return found;
}

}  // namespace mrf
