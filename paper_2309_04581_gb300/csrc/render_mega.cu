// FP32 megakernel of the hybrid light-transport loop: one thread per ray runs
// the whole path of the paper's Algorithm 1 (cast, march, shadow rays, BSDF
// sample, update, terminate), plus the field-query and ray-cast kernels used to
// test those steps on their own.
#include <cuda_runtime.h>

#include "device.cuh"

namespace mrf {

struct Counters {
    unsigned long long nominal;
    unsigned paths, seg, hits, shadow, evaluated, shadow_eval, retests, fault;
};

__device__ __forceinline__ void flush_counters(unsigned long long *stats, Counters &C) {
    if (!stats) return;
    unsigned long long v[ST_COUNT] = {C.paths, C.seg, C.hits, C.shadow, C.nominal, C.evaluated, C.shadow_eval,
                                      C.retests, C.fault};
    const unsigned mask = __activemask();
#pragma unroll
    for (int k = 0; k < ST_COUNT; ++k) {
        unsigned long long x = v[k];
        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(mask, x, off);
        v[k] = x;
    }
    if ((threadIdx.x & 31) == __ffs(mask) - 1) {
#pragma unroll
        for (int k = 0; k < ST_COUNT; ++k)
            if (v[k]) atomicAdd(stats + k, v[k]);
    }
}

// Field sample at p: returns sigma (and radiance if want_rgb).  Sets `evaluated`
// when the field's network (or analytic formula) had to run.
template <bool want_rgb>
__device__ __forceinline__ float field_at(const FieldDev &F, const float *w, V3 p, float rgb[3], bool &evaluated) {
    evaluated = true;
    if (F.kind == MRF_FIELD_HASHGRID) {
        float s = field_support(F, p);
        if (s <= 0.f) {
            evaluated = false;
            if (want_rgb) rgb[0] = rgb[1] = rgb[2] = 0.f;
            return 0.f;
        }
        return hash_field_fp32<want_rgb>(F, w, p, s, rgb);
    }
    if (F.kind == MRF_FIELD_GAUSS) return gauss_field(F, p, rgb);
    if (want_rgb) { rgb[0] = F.const_rgb[0]; rgb[1] = F.const_rgb[1]; rgb[2] = F.const_rgb[2]; }
    return F.const_sigma;
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
        float sigma = field_at<radiance>(F, w, p, rgb, ev);
        if (ev) {
            if (radiance) ++C.evaluated;
            else ++C.shadow_eval;
        }
        if (radiance) {
            const float x = sigma * delta;
            const float att = expf(-x), alpha = -expm1f(-x);
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

__device__ __forceinline__ void primary_ray(const RenderParams &P, uint32_t ray, V3 &o, V3 &d) {
    if (P.use_camera) {
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

// One path of Algorithm 1.  Writes L (RGB) and the camera segment's opacity.
__device__ void trace_path(const RenderParams &P, const float *w, uint32_t ray, uint32_t s, float L[3], float &alpha0,
                           Counters &C) {
    V3 o, d;
    primary_ray(P, ray, o, d);
    float T[3] = {1.f, 1.f, 1.f};
    L[0] = L[1] = L[2] = 0.f;
    alpha0 = 0.f;
    uint32_t prev = kNoHit, segs = 0;
    const uint64_t path = (uint64_t)ray * P.spp + s;
    ++C.paths;
    for (uint32_t j = 1; j <= P.max_bounces; ++j) {
        Hit h;
        unsigned rt = 0;
        bool fault = false;
        bvh_trace<false>(P.B, o, d, prev, P.tmin, INFINITY, h, rt, fault);
        C.retests += rt;
        if (fault) C.fault |= 1;
        const float T0 = T[0];
        bool stop = false;
        march<true>(P, w, o, d, 0.f, h.t, T, L, stop, C);
        if (j == 1) alpha0 = T0 > 0.f ? 1.f - T[0] / T0 : 0.f;
        segs = j;
        ++C.seg;
        if (P.rec_tri) {
            P.rec_tri[path * P.max_bounces + (j - 1)] = h.id;
            P.rec_t[path * P.max_bounces + (j - 1)] = h.t;
        }
        if (stop || h.id == kNoHit) break;
        ++C.hits;
        V3 a, b, c;
        uint32_t id, m;
        load_tri(P.B, h.slot, a, b, c, id, m);
        const V3 p = fma3(d, h.t, o);
        const V3 n = normalize(cross(b - a, c - a));
        const float dn = dot(d, n);
        const V3 nf = dn > 0.f ? n * -1.f : n;
        const MaterialDev mat = P.mats[min((int)m, P.n_mats - 1)];
        uint64_t ctr[4] = {(uint64_t)ray, (uint64_t)s, (uint64_t)j, 0ull};
        philox4x64_10(ctr, P.seed, 0ull);
        const float u0 = u24(ctr[0]), u1 = u24(ctr[1]), u2 = u24(ctr[2]);
        V3 nd;
        // Eq. 12 adds T' L_e at the hit; every mesh here has L_e = 0.
        if (mat.kind == MRF_MAT_MIRROR) {
            nd = reflect(d, n);
#pragma unroll
            for (int k = 0; k < 3; ++k) T[k] *= mat.rgb[k];
        } else if (mat.kind == MRF_MAT_GLASS) {
            const bool entering = dn < 0.f;
            const float ei = entering ? 1.f : mat.ior, et = entering ? mat.ior : 1.f;
            const float cos_i = fabsf(dn);
            const float F = fresnel(cos_i, ei, et);
            if (u0 < F) {
                nd = reflect(d, n);
            } else {
                const float eta = ei / et;
                const float s2t = eta * eta * (1.f - cos_i * cos_i);
                const float cos_t = sqrtf(fmaxf(0.f, 1.f - s2t));
                nd = d * eta + nf * (eta * cos_i - cos_t);
            }
        } else {
            // next-event estimation: shadow rays toward the point lights
            for (int l = 0; l < P.n_lights; ++l) {
                const LightDev L0 = P.lights[l];
                V3 wl = v3(L0.pos[0], L0.pos[1], L0.pos[2]) - p;
                const float D2 = dot(wl, wl), D = sqrtf(D2);
                wl = wl * (1.f / D);
                const float cosl = dot(nf, wl);
                if (cosl <= 0.f) continue;
                ++C.shadow;
                Hit hs;
                unsigned rs = 0;
                bool f2 = false;
                const bool blocked = bvh_trace<true>(P.B, p, wl, id, P.tmin, D, hs, rs, f2);
                C.retests += rs;
                if (f2) C.fault |= 1;
                if (blocked) continue;
                bool dummy = false;
                const float depth = march<false>(P, w, p, wl, 0.f, D, nullptr, nullptr, dummy, C);
                const float Tf = expf(-depth);
                const float g = cosl / D2 * Tf * 0.31830988618379067f;
#pragma unroll
                for (int k = 0; k < 3; ++k) L[k] = fmaf(T[k] * mat.rgb[k] * g, L0.I[k], L[k]);
            }
            nd = sample_cosine(nf, u1, u2);
#pragma unroll
            for (int k = 0; k < 3; ++k) T[k] *= mat.rgb[k];
        }
        d = normalize(nd);
        o = p;
        prev = id;
        if (P.tau > 0.f && fmaxf(T[0], fmaxf(T[1], T[2])) < P.tau) break;
    }
    if (P.rec_seg) P.rec_seg[path] = segs;
    if (P.rec_tri) {
        for (uint32_t j = segs; j < P.max_bounces; ++j) {
            P.rec_tri[path * P.max_bounces + j] = kNoHit;
            P.rec_t[path * P.max_bounces + j] = INFINITY;
        }
    }
}

__global__ void __launch_bounds__(128) render_megakernel(const RenderParams P) {
    extern __shared__ float smem_w[];
    const FieldDev &F = P.F;
    const float *w = nullptr;
    if (F.kind == MRF_FIELD_HASHGRID) {
        const int nw = mlp_floats(F.n_in);
        for (int i = threadIdx.x; i < nw; i += blockDim.x) smem_w[i] = F.mlp[i];
        __syncthreads();
        w = smem_w;
    }
    const uint32_t ray = blockIdx.x * blockDim.x + threadIdx.x;
    Counters C = {};
    if (ray < P.count) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (uint32_t s = 0; s < P.spp; ++s) {
            float L[3], a0;
            trace_path(P, w, ray, s, L, a0, C);
            acc[0] += L[0]; acc[1] += L[1]; acc[2] += L[2]; acc[3] += a0;
        }
        const float inv = 1.f / (float)P.spp;
        reinterpret_cast<float4 *>(P.out)[ray] = make_float4(acc[0] * inv, acc[1] * inv, acc[2] * inv, acc[3] * inv);
    }
    flush_counters(P.stats, C);
}

cudaError_t launch_render_megakernel(const RenderParams &P, cudaStream_t s) {
    const int threads = 128;
    const size_t smem = P.F.kind == MRF_FIELD_HASHGRID ? (size_t)mlp_floats(P.F.n_in) * sizeof(float) : 0;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(render_megakernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const unsigned blocks = (P.count + threads - 1) / threads;
    render_megakernel<<<blocks, threads, smem, s>>>(P);
    return cudaGetLastError();
}

// ------------------------------------------------------------- field query
__global__ void __launch_bounds__(128) field_query_kernel(const FieldDev F, const float *pts, uint32_t n, float *out) {
    extern __shared__ float smem_w[];
    const float *w = nullptr;
    if (F.kind == MRF_FIELD_HASHGRID) {
        const int nw = mlp_floats(F.n_in);
        for (int i = threadIdx.x; i < nw; i += blockDim.x) smem_w[i] = F.mlp[i];
        __syncthreads();
        w = smem_w;
    }
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const V3 p = v3(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
    float rgb[3] = {0.f, 0.f, 0.f}, sigma = 0.f;
    if (inside_field_box(F, p)) {
        bool ev;
        sigma = field_at<true>(F, w, p, rgb, ev);
    }
    reinterpret_cast<float4 *>(out)[i] = make_float4(sigma, rgb[0], rgb[1], rgb[2]);
}

cudaError_t launch_field_query(const FieldDev &F, const float *pts, uint32_t n, float *out, cudaStream_t s) {
    const size_t smem = F.kind == MRF_FIELD_HASHGRID ? (size_t)mlp_floats(F.n_in) * sizeof(float) : 0;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(field_query_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    field_query_kernel<<<(n + 127) / 128, 128, smem, s>>>(F, pts, n, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------- ray cast
__global__ void __launch_bounds__(128) cast_kernel(const BvhDev B, const float *o, const float *d, const uint32_t *skip,
                                                   uint32_t n, float tmin, float *out_t, uint32_t *out_tri,
                                                   unsigned long long *stats) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    Counters C = {};
    if (i < n) {
        Hit h;
        unsigned rt = 0;
        bool fault = false;
        bvh_trace<false>(B, v3(o[3 * i], o[3 * i + 1], o[3 * i + 2]), v3(d[3 * i], d[3 * i + 1], d[3 * i + 2]),
                         skip ? skip[i] : kNoHit, tmin, INFINITY, h, rt, fault);
        out_t[i] = h.t;
        out_tri[i] = h.id;
        C.retests = rt;
        C.fault = fault ? 1u : 0u;
    }
    flush_counters(stats, C);
}

cudaError_t launch_cast(const BvhDev &B, const float *o, const float *d, const uint32_t *skip, uint32_t n, float tmin,
                        float *out_t, uint32_t *out_tri, unsigned long long *stats, cudaStream_t s) {
    cast_kernel<<<(n + 127) / 128, 128, 0, s>>>(B, o, d, skip, n, tmin, out_t, out_tri, stats);
    return cudaGetLastError();
}

}  // namespace mrf
