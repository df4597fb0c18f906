// Path building blocks shared by the megakernel and the wavefront engine:
// statistics counters, field sampling, the segment march (Eqs. 10-11), the
// BSDFs of Sec. 3.3 and primary-ray generation.
#pragma once
#include <cuda_runtime.h>

#include "device.cuh"

namespace mrf {

struct Counters {
    unsigned long long nominal;
    unsigned paths, seg, hits, shadow, evaluated, shadow_eval, retests, fault, net;
    unsigned end_miss, end_tau, end_cap;   // how paths ended: left the scene, throughput below tau, bounce cap
    unsigned nodes, tris;                  // BVH nodes visited, ray-triangle tests
    unsigned long long worst;              // (nodes << 32) | path of this thread's longest closest-hit traversal
};

// Records a closest-hit traversal of `nodes` nodes made for `path`.
__device__ __forceinline__ void note_traversal(Counters &C, unsigned nodes, uint32_t path) {
    const unsigned long long key = ((unsigned long long)nodes << 32) | path;
    if (key > C.worst) C.worst = key;
}

__device__ __forceinline__ void flush_counters(unsigned long long *stats, Counters &C) {
    if (!stats) return;
    unsigned long long v[ST_COUNT] = {C.paths, C.seg, C.hits, C.shadow, C.nominal, C.evaluated, C.shadow_eval,
                                      C.retests, C.fault, C.net, C.end_miss, C.end_tau, C.end_cap, C.nodes, C.tris, 0ull};
    const unsigned mask = __activemask();
#pragma unroll
    for (int k = 0; k < ST_COUNT; ++k) {
        unsigned long long x = v[k];
        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(mask, x, off);
        v[k] = x;
    }
    unsigned long long worst = C.worst;
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long y = __shfl_xor_sync(mask, worst, off);
        if (y > worst) worst = y;
    }
    if ((threadIdx.x & 31) == __ffs(mask) - 1) {
#pragma unroll
        for (int k = 0; k < ST_COUNT; ++k)
            if (v[k] && k != ST_WORST) atomicAdd(stats + k, v[k]);
        if (worst) atomicMax(stats + ST_WORST, worst);
    }
}

// Field sample at p: returns sigma (and radiance if want_rgb).  Sets `evaluated`
// when the field's network (or analytic formula) had to run.
template <bool want_rgb>
__device__ __forceinline__ float field_at(const FieldDev &F, const float *w, V3 p, V3 d, float rgb[3],
                                          bool &evaluated) {
    evaluated = true;
    if (F.kind == MRF_FIELD_HASHGRID) {
        float s = field_support(F, p);
        if (s <= 0.f) {
            evaluated = false;
            if (want_rgb) rgb[0] = rgb[1] = rgb[2] = 0.f;
            return 0.f;
        }
        if (F.view_dep) return hash_field_view<want_rgb>(F, w, p, d, s, rgb);
        return hash_field_fp32<want_rgb>(F, w, p, s, rgb);
    }
    if (F.kind == MRF_FIELD_GAUSS) return gauss_field(F, p, rgb);
    if (want_rgb) { rgb[0] = F.const_rgb[0]; rgb[1] = F.const_rgb[1]; rgb[2] = F.const_rgb[2]; }
    return F.const_sigma;
}

// Shadow mask m(p_t) of Sec. 3.1 at the world point pw: a ray toward each
// light with mask strength r > 0 (position, or an area light's centroid); each
// light a mesh blocks multiplies m by 1 - r.
static __device__ __noinline__ float sample_mask(const RenderParams &P, V3 pw) {
    float m = 1.f;
    for (int l = 0; l < P.n_lights; ++l) {
        const LightDev &L0 = P.lights[l];
        if (!(L0.mask > 0.f)) continue;
        V3 w = v3(L0.target[0], L0.target[1], L0.target[2]) - pw;
        const float D = sqrtf(dot(w, w));
        if (!(D > 0.f)) continue;
        w = w * (1.f / D);
        Hit hs;
        unsigned rs = 0, nv = 0, nt = 0;
        bool fault = false;
        if (bvh_trace<true>(P.B, pw, w, kNoHit, P.tmin, D, hs, rs, nv, nt, fault)) m *= 1.f - L0.mask;
    }
    return m;
}

// Quadrature of Eqs. 10-11 over [a, b] of the ray (o, d).
//   radiance: alpha_i = 1 - exp(-sigma_i delta_i); L += T alpha_i r_i; T *= exp(-sigma_i delta_i);
//             sets `stop` when max(T) falls below tau.
//   otherwise: returns the optical depth sum sigma_i delta_i (shadow transmittance).
// Samples sit at interval midpoints: steps > 0 splits [t0, t1] evenly, else
// intervals of length dt with the last one clipped at t1.  Samples in empty
// occupancy cells are skipped up to the cell exit (their density is zero).
template <bool radiance>
__device__ float march(const RenderParams &P, const float *w, V3 o, V3 d, float a, float b, float T[3], float L[3],
                       bool &stop, Counters &C) {
    const FieldDev &F = P.F;
    const V3 ow = o, dw = d;   // world ray (the shadow mask casts from world points)
    to_field_frame(F, o, d);
    float tb0, tb1;
    if (!box_interval(F.lo, F.hi, o, d, tb0, tb1)) return 0.f;
    const float t0 = fmaxf(a, tb0), t1 = fminf(b, tb1);
    if (!(t1 > t0)) return 0.f;
    int n;
    float h;
    if (P.steps) {
        n = (int)P.steps;
        h = (t1 - t0) / (float)n;
    } else {
        h = P.dt;
        float nf = ceilf((t1 - t0) / h);
        if (nf > 16777216.f) { C.fault |= 2; return 0.f; }
        n = (int)nf;
    }
    C.nominal += (unsigned long long)n;
    const V3 inv = v3(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);
    const bool use_occ = F.kind == MRF_FIELD_HASHGRID && F.occ != nullptr;
    float depth = 0.f;
    for (int i = 0; i < n;) {
        const float lo = fmaf((float)i, h, t0);
        const float hi = P.steps ? fmaf((float)(i + 1), h, t0) : fminf(lo + h, t1);
        const float tm = 0.5f * (lo + hi), delta = hi - lo;
        const V3 p = fma3(d, tm, o);
        if (use_occ) {
            int c[3];
            if (!occupied(F, p, c)) {
                float te = cell_exit(F, c, o, inv);
                int j = (int)ceilf((te - t0) / h - 0.5f);
                i = max(i + 1, j);
                continue;
            }
        }
        float rgb[3];
        bool ev;
        float sigma = field_at<radiance>(F, w, p, d, rgb, ev);
        if (ev) {
            if (radiance) ++C.evaluated;
            else ++C.shadow_eval;
        }
        if (radiance) {
            const float x = sigma * delta;
            const float att = expf(-x);
            float alpha = -expm1f(-x);
            if (P.shadow_mask && sigma > 0.f) alpha *= sample_mask(P, fma3(dw, tm, ow));
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                L[k] = fmaf(T[k] * alpha, rgb[k], L[k]);
                T[k] *= att;
            }
            if (P.tau > 0.f && fmaxf(T[0], fmaxf(T[1], T[2])) < P.tau) {
                stop = true;
                break;
            }
        } else {
            depth = fmaf(sigma, delta, depth);
        }
        ++i;
    }
    return depth;
}

__device__ __forceinline__ V3 reflect(V3 d, V3 n) { return d - n * (2.f * dot(d, n)); }

// unpolarised Fresnel reflectance of a smooth dielectric (TIR -> 1)
__device__ __forceinline__ float fresnel(float cos_i, float eta_i, float eta_t) {
    float r = eta_i / eta_t;
    float s2t = r * r * (1.f - cos_i * cos_i);
    if (s2t >= 1.f) return 1.f;
    float cos_t = sqrtf(1.f - s2t);
    float rs = (eta_i * cos_i - eta_t * cos_t) / (eta_i * cos_i + eta_t * cos_t);
    float rp = (eta_t * cos_i - eta_i * cos_t) / (eta_t * cos_i + eta_i * cos_t);
    return 0.5f * (rs * rs + rp * rp);
}

// cosine-weighted direction around unit n (tangent frame of Duff et al. 2017)
__device__ __forceinline__ V3 sample_cosine(V3 n, float u1, float u2) {
    float sgn = copysignf(1.f, n.z);
    float a = -1.f / (sgn + n.z), b = n.x * n.y * a;
    V3 t1 = v3(1.f + sgn * n.x * n.x * a, sgn * b, -sgn * n.x);
    V3 t2 = v3(b, sgn + n.y * n.y * a, -n.y);
    float r = sqrtf(u1), s, c;
    sincospif(2.f * u2, &s, &c);
    float z = sqrtf(fmaxf(0.f, 1.f - u1));
    return t1 * (r * c) + t2 * (r * s) + n * z;
}

// Pinhole ray through the centre of pixel (px, py) of a W x H image (row 0 at the top).
__device__ __forceinline__ V3 pinhole_dir(V3 f, V3 r, V3 u, float tan_half, float aspect, uint32_t W, uint32_t H,
                                          uint32_t px, uint32_t py) {
    float sx = (2.f * ((float)px + 0.5f) / (float)W - 1.f) * tan_half * aspect;
    float sy = (1.f - 2.f * ((float)py + 0.5f) / (float)H) * tan_half;
    return normalize(f + r * sx + u * sy);
}

__device__ __forceinline__ void primary_ray(const RenderParams &P, uint32_t ray, V3 &o, V3 &d) {
    if (P.n_views) {
        // the view holding this ray: the last one whose first ray is <= ray
        uint32_t lo = 0, hi = P.n_views - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (__ldg(&P.views[mid].offset) <= ray) lo = mid;
            else hi = mid - 1;
        }
        const ViewDev &v = P.views[lo];
        const uint32_t pix = ray - __ldg(&v.offset), W = __ldg(&v.W);
        d = pinhole_dir(v3(__ldg(&v.f[0]), __ldg(&v.f[1]), __ldg(&v.f[2])),
                        v3(__ldg(&v.r[0]), __ldg(&v.r[1]), __ldg(&v.r[2])),
                        v3(__ldg(&v.u[0]), __ldg(&v.u[1]), __ldg(&v.u[2])), __ldg(&v.tan_half), __ldg(&v.aspect), W,
                        __ldg(&v.H), pix % W, pix / W);
        o = v3(__ldg(&v.pos[0]), __ldg(&v.pos[1]), __ldg(&v.pos[2]));
    } else if (P.use_camera) {
        uint32_t px = ray % P.W, py = ray / P.W;
        float sx = (2.f * ((float)px + 0.5f) / (float)P.W - 1.f) * P.tan_half * P.aspect;
        float sy = (1.f - 2.f * ((float)py + 0.5f) / (float)P.H) * P.tan_half;
        V3 f = v3(P.cam_f[0], P.cam_f[1], P.cam_f[2]), r = v3(P.cam_r[0], P.cam_r[1], P.cam_r[2]),
           u = v3(P.cam_u[0], P.cam_u[1], P.cam_u[2]);
        d = normalize(f + r * sx + u * sy);
        o = v3(P.cam_pos[0], P.cam_pos[1], P.cam_pos[2]);
    } else {
        o = v3(P.ray_o[3 * ray], P.ray_o[3 * ray + 1], P.ray_o[3 * ray + 2]);
        d = normalize(v3(P.ray_d[3 * ray], P.ray_d[3 * ray + 1], P.ray_d[3 * ray + 2]));
    }
}


// Surface interaction at the closest hit h of ray (o, d).
struct SurfaceHit {
    V3 p, n, nf;      // hit point, unit geometric normal, normal facing the incoming ray
    float dn;         // d . n
    MaterialDev mat;
    uint32_t id;      // original triangle index
};

__device__ __forceinline__ SurfaceHit surface_at(const RenderParams &P, V3 o, V3 d, const Hit &h) {
    SurfaceHit S;
    V3 a, b, c;
    uint32_t m;
    load_tri(P.B, h.slot, a, b, c, S.id, m);
    S.p = fma3(d, h.t, o);
    S.n = normalize(cross(b - a, c - a));
    S.dn = dot(d, S.n);
    S.nf = S.dn > 0.f ? S.n * -1.f : S.n;
    S.mat = P.mats[min((int)m, P.n_mats - 1)];
    return S;
}

// Uniforms for the surface event ending segment j: Philox4x64-10, counter
// (ray, spp, j, 0), key (seed, 0); top 24 bits of words 0..2.
__device__ __forceinline__ void surface_uniforms(const RenderParams &P, uint32_t ray, uint32_t s, uint32_t j,
                                                 float u[3]) {
    uint64_t ctr[4] = {(uint64_t)ray, (uint64_t)s, (uint64_t)j, 0ull};
    philox4x64_10(ctr, P.seed, 0ull);
    u[0] = u24(ctr[0]);
    u[1] = u24(ctr[1]);
    u[2] = u24(ctr[2]);
}

// Shadow ray k of light l from the diffuse hit S (Sec. 3.1, "Shadow rays"):
// unit direction wl and distance D to the light point, and the next-event
// weight w (to be multiplied by T', the visibility and the field
// transmittance).  Point light: (albedo / pi) cos I / D^2.  Area light: point
// y drawn uniformly on the triangle from Philox counter (ray, spp, j, 1 + q0 + k)
// (square-root barycentric warp), weight (albedo / pi) Le A / N cos_x cos_y / D^2.
// Returns false when the light point is behind the surface or the emitter
// faces away (no shadow ray is cast).
__device__ __forceinline__ bool shadow_ray(const RenderParams &P, const SurfaceHit &S, int l, uint32_t k,
                                           uint32_t ray, uint32_t s, uint32_t j, V3 &wl, float &D, float w[3]) {
    const LightDev &L0 = P.lights[l];
    V3 y;
    float g;
    if (L0.kind == MRF_LIGHT_AREA) {
        uint64_t ctr[4] = {(uint64_t)ray, (uint64_t)s, (uint64_t)j, 1ull + L0.q0 + k};
        philox4x64_10(ctr, P.seed, 0ull);
        const float su = sqrtf(u24(ctr[0])), b0 = 1.f - su, b1 = u24(ctr[1]) * su, b2 = 1.f - b0 - b1;
        y = v3(L0.pos[0], L0.pos[1], L0.pos[2]) * b0 + v3(L0.v1[0], L0.v1[1], L0.v1[2]) * b1 +
            v3(L0.v2[0], L0.v2[1], L0.v2[2]) * b2;
        wl = y - S.p;
        const float D2 = dot(wl, wl);
        D = sqrtf(D2);
        wl = wl * (1.f / D);
        const float cosx = dot(S.nf, wl), cosy = -dot(v3(L0.n[0], L0.n[1], L0.n[2]), wl);
        if (!(cosx > 0.f) || !(cosy > 0.f)) return false;
        g = cosx * cosy / D2 * (L0.area / (float)L0.samples) * 0.31830988618379067f;
    } else {
        wl = v3(L0.pos[0], L0.pos[1], L0.pos[2]) - S.p;
        const float D2 = dot(wl, wl);
        D = sqrtf(D2);
        wl = wl * (1.f / D);
        const float cosl = dot(S.nf, wl);
        if (!(cosl > 0.f)) return false;
        g = cosl / D2 * 0.31830988618379067f;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) w[c] = S.mat.rgb[c] * g * L0.I[c];
    return true;
}

// Samples the BSDF (Eq. 13): returns the new (unnormalised) direction and
// updates the throughput T.  Mirror: T *= rho; glass: Fresnel choice between
// reflection and Snell refraction, T kept; Lambertian: cosine sampling, T *= albedo.
__device__ __forceinline__ V3 bsdf_sample(const SurfaceHit &S, V3 d, const float u[3], float T[3]) {
    if (S.mat.kind == MRF_MAT_MIRROR) {
#pragma unroll
        for (int k = 0; k < 3; ++k) T[k] *= S.mat.rgb[k];
        return reflect(d, S.n);
    }
    if (S.mat.kind == MRF_MAT_GLASS) {
        const bool entering = S.dn < 0.f;
        const float ei = entering ? 1.f : S.mat.ior, et = entering ? S.mat.ior : 1.f;
        const float cos_i = fabsf(S.dn);
        const float F = fresnel(cos_i, ei, et);
        if (u[0] < F) return reflect(d, S.n);
        const float eta = ei / et;
        const float s2t = eta * eta * (1.f - cos_i * cos_i);
        const float cos_t = sqrtf(fmaxf(0.f, 1.f - s2t));
        return d * eta + S.nf * (eta * cos_i - cos_t);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) T[k] *= S.mat.rgb[k];
    return sample_cosine(S.nf, u[1], u[2]);
}

}  // namespace mrf
