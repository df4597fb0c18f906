// Device functions of the shadow-transmittance network: encoding of a
// (point, direction) pair and the thread-level FP32 forward pass.  The network
// stands in for the field march of a shadow ray (Sec. 3.1, "Shadow rays":
// T = exp(-int sigma) toward the light).
#pragma once
#include <cuda_runtime.h>

#include "device.cuh"

namespace mrf {

// Spherical harmonics of the direction input: sh16 (device.cuh).
__device__ __forceinline__ void snet_sh16(V3 w, float *Y) { sh16(w, Y); }

// World point and direction to the field's local frame.
__device__ __forceinline__ void snet_to_local(const ShadowNetDev &N, V3 &p, V3 &w) {
    if (!N.has_pose) return;
    const float *M = N.to_local;
    const V3 q = p, e = w;
    p = v3(fmaf(M[0], q.x, fmaf(M[1], q.y, fmaf(M[2], q.z, M[3]))),
           fmaf(M[4], q.x, fmaf(M[5], q.y, fmaf(M[6], q.z, M[7]))),
           fmaf(M[8], q.x, fmaf(M[9], q.y, fmaf(M[10], q.z, M[11]))));
    w = v3(fmaf(M[0], e.x, fmaf(M[1], e.y, M[2] * e.z)), fmaf(M[4], e.x, fmaf(M[5], e.y, M[6] * e.z)),
           fmaf(M[8], e.x, fmaf(M[9], e.y, M[10] * e.z)));
}

__device__ __forceinline__ bool snet_inside(const ShadowNetDev &N, V3 pl) {
    return pl.x >= N.lo[0] && pl.x <= N.hi[0] && pl.y >= N.lo[1] && pl.y <= N.hi[1] && pl.z >= N.lo[2] &&
           pl.z <= N.hi[2];
}

// Cell of level l holding the local point pl (position scaled to [0,1] by the
// box and clamped): integer corner c and fractional offsets f.
__device__ __forceinline__ void snet_cell(const ShadowNetDev &N, int l, V3 pl, uint32_t c[3], float f[3]) {
    const float Nf = (float)N.res[l];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float u = (comp(pl, a) - N.lo[a]) * N.ext_inv[a];
        u = fminf(fmaxf(u, 0.f), 1.f) * Nf;
        const float fl = fminf(floorf(u), Nf - 1.f);
        c[a] = (uint32_t)fl;
        f[a] = u - fl;
    }
}

// Flat index (in entries, table-wide) of vertex (x, y, z) of level l.
__device__ __forceinline__ uint32_t snet_index(const ShadowNetDev &N, int l, uint32_t x, uint32_t y, uint32_t z) {
    const uint32_t T = 1u << N.log2T;
    uint32_t i;
    if ((N.dense_mask >> l) & 1u) {
        const uint32_t s = N.res[l] + 1;
        i = x + s * (y + s * z);
    } else {
        i = (x ^ (y * 2654435761u) ^ (z * 805459861u)) & (T - 1u);
    }
    return (uint32_t)l * T + i;
}

// The 32 network inputs of the local point pl and local direction wl.
__device__ __forceinline__ void snet_encode(const ShadowNetDev &N, V3 pl, V3 wl, float *x) {
#pragma unroll
    for (int l = 0; l < kSnetLevels; ++l) {
        uint32_t c[3];
        float f[3];
        snet_cell(N, l, pl, c, f);
        float a0 = 0.f, a1 = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t i = snet_index(N, l, c[0] + (k & 1), c[1] + ((k >> 1) & 1), c[2] + ((k >> 2) & 1));
            const float wt = ((k & 1) ? f[0] : 1.f - f[0]) * (((k >> 1) & 1) ? f[1] : 1.f - f[1]) *
                             (((k >> 2) & 1) ? f[2] : 1.f - f[2]);
            const float2 e = __ldg(reinterpret_cast<const float2 *>(N.table) +
                                   checked_index(i, (uint64_t)kSnetLevels << N.log2T, nullptr));
            a0 = fmaf(wt, e.x, a0);
            a1 = fmaf(wt, e.y, a1);
        }
        x[2 * l] = a0;
        x[2 * l + 1] = a1;
    }
    snet_sh16(normalize(wl), x + 2 * kSnetLevels);
}

// Thread-level forward pass with the weights at w (the MLP part of the
// parameter vector): returns sigmoid(z).
__device__ __forceinline__ float snet_mlp(const float *__restrict__ w, const float *x) {
    float h1[kSnetW], h2[kSnetW];
#pragma unroll
    for (int i = 0; i < kSnetW; ++i) {
        const float4 *r = reinterpret_cast<const float4 *>(w + i * kSnetIn);
        float s = w[kSnetOffB1 + i];
#pragma unroll
        for (int k = 0; k < kSnetIn / 4; ++k) {
            const float4 q = r[k];
            s = fmaf(q.x, x[4 * k], s);
            s = fmaf(q.y, x[4 * k + 1], s);
            s = fmaf(q.z, x[4 * k + 2], s);
            s = fmaf(q.w, x[4 * k + 3], s);
        }
        h1[i] = fmaxf(s, 0.f);
    }
#pragma unroll
    for (int i = 0; i < kSnetW; ++i) {
        const float4 *r = reinterpret_cast<const float4 *>(w + kSnetOffW2 + i * kSnetW);
        float s = w[kSnetOffB2 + i];
#pragma unroll
        for (int k = 0; k < kSnetW / 4; ++k) {
            const float4 q = r[k];
            s = fmaf(q.x, h1[4 * k], s);
            s = fmaf(q.y, h1[4 * k + 1], s);
            s = fmaf(q.z, h1[4 * k + 2], s);
            s = fmaf(q.w, h1[4 * k + 3], s);
        }
        h2[i] = fmaxf(s, 0.f);
    }
    float z = w[kSnetOffB4];
#pragma unroll
    for (int i = 0; i < kSnetW; ++i) {
        const float4 *r = reinterpret_cast<const float4 *>(w + kSnetOffW3 + i * kSnetW);
        float s = w[kSnetOffB3 + i];
#pragma unroll
        for (int k = 0; k < kSnetW / 4; ++k) {
            const float4 q = r[k];
            s = fmaf(q.x, h2[4 * k], s);
            s = fmaf(q.y, h2[4 * k + 1], s);
            s = fmaf(q.z, h2[4 * k + 2], s);
            s = fmaf(q.w, h2[4 * k + 3], s);
        }
        z = fmaf(w[kSnetOffW4 + i], fmaxf(s, 0.f), z);
    }
    return 1.f / (1.f + expf(-z));
}

// Network transmittance of the shadow ray leaving world point p along w.
__device__ __forceinline__ float snet_eval(const ShadowNetDev &N, const float *__restrict__ mlp, V3 p, V3 w) {
    snet_to_local(N, p, w);
    float x[kSnetIn];
    snet_encode(N, p, w, x);
    return snet_mlp(mlp, x);
}

}  // namespace mrf
