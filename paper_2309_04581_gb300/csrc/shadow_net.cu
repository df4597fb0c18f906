// Learned shadow transmittance: training pairs, the training step (forward,
// back-propagation, Adam) and inference of the shadow network, all in FP32 on
// the CUDA cores.  The network (shadow_net.cuh) replaces the field march of a
// shadow ray (Sec. 3.1, "Shadow rays"); the march labels its training pairs.
//
// Training step, per block of 256 threads and tile of 64 pairs (persistent
// blocks loop over the batch's tiles):
//   encode   : 4 threads per pair (2 hash levels each; one also writes the
//              spherical harmonics), features stored feature-major X[k][s];
//   forward  : three 64 x 64 (x 32) register-tiled products in shared memory,
//              activations kept for the backward pass;
//   backward : dL/dz = 2 (T - y) T (1 - T) / B, deltas through the layers
//              with the transposed weights, weight gradients accumulated in
//              registers across tiles and added to the global gradient once
//              per block; the hash-table gradient is scattered per pair with
//              float2 atomics (trilinear weights x input gradient).
// Adam then updates every parameter and clears the gradient.
#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "path.cuh"
#include "shadow_net.cuh"
#include "tc.cuh"

namespace mrf {

namespace {

constexpr int kTT = 256;     // training threads per block
constexpr int kTile = 64;    // pairs per tile
constexpr int kSP = 68;      // row stride of the feature-major [feature][pair] arrays (16-byte rows, padded)

struct TrainSmem {
    float Wt1[kSnetIn * kSnetW];     // [k][u]
    float W1[kSnetW * kSnetIn];      // [u][k]
    float Wt2[kSnetW * kSnetW], W2[kSnetW * kSnetW];
    float Wt3[kSnetW * kSnetW], W3[kSnetW * kSnetW];
    float b1[kSnetW], b2[kSnetW], b3[kSnetW], W4[kSnetW];
    float X[kSnetIn * kSP];
    float H1[kSnetW * kSP], H2[kSnetW * kSP], H3[kSnetW * kSP];
    float D3[kSnetW * kSP];          // delta of layer 3, later of layer 1
    float D2[kSnetW * kSP];
    float DX[kSnetIn * kSP];         // gradient of the inputs
    float4 pl[kTile];                // local point (xyz), label (w)
    float zpart[4][kTile];
    float dz[kTile];
    float b4;
};

// acc[i][j] += sum_r A[r][m0 + i] B[r][n0 + j]  (both operands reduction-major)
template <int TM, int TN>
__device__ __forceinline__ void gemm_rr(const float *__restrict__ A, int lda, const float *__restrict__ B, int ldb, int R,
                                        int m0, int n0, float (&acc)[TM][TN]) {
#pragma unroll 4
    for (int r = 0; r < R; ++r) {
        float a[TM], b[TN];
        if constexpr (TM == 4) {
            const float4 q = *reinterpret_cast<const float4 *>(A + r * lda + m0);
            a[0] = q.x; a[1] = q.y; a[2] = q.z; a[3] = q.w;
        } else {
            const float2 q = *reinterpret_cast<const float2 *>(A + r * lda + m0);
            a[0] = q.x; a[1] = q.y;
        }
        const float4 q = *reinterpret_cast<const float4 *>(B + r * ldb + n0);
        b[0] = q.x; b[1] = q.y; b[2] = q.z; b[3] = q.w;
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
}

// acc[i][j] += sum_s A[m0 + i][s] B[n0 + 16 j][s]  (rows of pairs; s over the tile)
template <int TM, int TN>
__device__ __forceinline__ void gemm_mm(const float *__restrict__ A, const float *__restrict__ B, int m0, int n0,
                                        float (&acc)[TM][TN]) {
#pragma unroll 2
    for (int s = 0; s < kTile; s += 4) {
        float4 a[TM], b[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = *reinterpret_cast<const float4 *>(A + (m0 + i) * kSP + s);
#pragma unroll
        for (int j = 0; j < TN; ++j) b[j] = *reinterpret_cast<const float4 *>(B + (n0 + 16 * j) * kSP + s);
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j)
                acc[i][j] = fmaf(a[i].x, b[j].x, fmaf(a[i].y, b[j].y, fmaf(a[i].z, b[j].z, fmaf(a[i].w, b[j].w,
                                                                                                   acc[i][j]))));
    }
}

template <int TM, int TN>
__device__ __forceinline__ void zero(float (&acc)[TM][TN]) {
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
}

// Forward layer: H[u][s] = relu(sum_k Wt[k][u] In[k][s] + b[u]) for the thread's 4 x 4 tile.
__device__ __forceinline__ void forward_layer(const float *Wt, const float *b, const float *In, int K, float *H, int mg,
                                              int ng) {
    float acc[4][4];
    zero(acc);
    gemm_rr<4, 4>(Wt, kSnetW, In, kSP, K, 4 * mg, 4 * ng, acc);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float bb = b[4 * mg + i];
        *reinterpret_cast<float4 *>(H + (4 * mg + i) * kSP + 4 * ng) =
            make_float4(fmaxf(acc[i][0] + bb, 0.f), fmaxf(acc[i][1] + bb, 0.f), fmaxf(acc[i][2] + bb, 0.f),
                        fmaxf(acc[i][3] + bb, 0.f));
    }
}

// Backward through a 64 x 64 layer: Dout[k][s] = [Hk[k][s] > 0] sum_u W[u][k] Din[u][s].
__device__ __forceinline__ void backward_layer(const float *W, const float *Din, const float *Hk, float *Dout, int mg,
                                               int ng) {
    float acc[4][4];
    zero(acc);
    gemm_rr<4, 4>(W, kSnetW, Din, kSP, kSnetW, 4 * mg, 4 * ng, acc);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int k = 4 * mg + i;
        const float4 h = *reinterpret_cast<const float4 *>(Hk + k * kSP + 4 * ng);
        *reinterpret_cast<float4 *>(Dout + k * kSP + 4 * ng) =
            make_float4(h.x > 0.f ? acc[i][0] : 0.f, h.y > 0.f ? acc[i][1] : 0.f, h.z > 0.f ? acc[i][2] : 0.f,
                        h.w > 0.f ? acc[i][3] : 0.f);
    }
}

__device__ __forceinline__ float row_sum(const float *row) {
    float s = 0.f;
    for (int i = 0; i < kTile; i += 4) {
        const float4 q = *reinterpret_cast<const float4 *>(row + i);
        s += (q.x + q.y) + (q.z + q.w);
    }
    return s;
}

// Gradients are summed in 64-bit fixed point with 2^-40 units: integer
// addition is associative, so the sum of a batch does not depend on the order
// in which blocks and threads add their parts, and training reruns and resumes
// bit for bit.  |part| < 2^23 and |sum| < 2^23 hold with a wide margin (the
// loss is a mean of squared errors of a sigmoid, per-pair parts carry 1/B).
constexpr float kGradUnit = 1099511627776.0f;   // 2^40
__device__ __forceinline__ void grad_add(unsigned long long *acc, float x) {
    atomicAdd(acc, (unsigned long long)__float2ll_rn(x * kGradUnit));
}
__device__ __forceinline__ float grad_value(unsigned long long v) {
    return (float)((double)(long long)v * (1.0 / 1099511627776.0));
}

// One pass over pairs [b0, b0 + B) (cyclic in n_pairs) accumulating the loss
// and the gradient of every parameter into the fixed-point sums gacc (which
// the caller cleared).
__global__ void __launch_bounds__(kTT, 1)
snet_train_kernel(const ShadowNetDev N, const float *__restrict__ params, unsigned long long *__restrict__ gacc,
                  const float *__restrict__ pairs, uint64_t n_pairs, uint64_t b0, uint32_t B, float *loss) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem &S = *reinterpret_cast<TrainSmem *>(smem_raw);
    const int tid = threadIdx.x, mg = tid >> 4, ng = tid & 15;
    const float *mlp = params + ((size_t)kSnetLevels << N.log2T) * 2;
    unsigned long long *gmlp = gacc + ((size_t)kSnetLevels << N.log2T) * 2;
    // weights, in both orientations
    for (int i = tid; i < kSnetW * kSnetIn; i += kTT) {
        const int u = i / kSnetIn, k = i % kSnetIn;
        const float w = mlp[i];
        S.W1[i] = w;
        S.Wt1[k * kSnetW + u] = w;
    }
    for (int i = tid; i < kSnetW * kSnetW; i += kTT) {
        const int u = i / kSnetW, k = i % kSnetW;
        const float w2 = mlp[kSnetOffW2 + i], w3 = mlp[kSnetOffW3 + i];
        S.W2[i] = w2;
        S.Wt2[k * kSnetW + u] = w2;
        S.W3[i] = w3;
        S.Wt3[k * kSnetW + u] = w3;
    }
    if (tid < kSnetW) {
        S.b1[tid] = mlp[kSnetOffB1 + tid];
        S.b2[tid] = mlp[kSnetOffB2 + tid];
        S.b3[tid] = mlp[kSnetOffB3 + tid];
        S.W4[tid] = mlp[kSnetOffW4 + tid];
    }
    if (tid == 0) S.b4 = mlp[kSnetOffB4];
    float gW1[4][2], gW2[4][4], gW3[4][4];
    zero(gW1);
    zero(gW2);
    zero(gW3);
    float gb1 = 0.f, gb2 = 0.f, gb3 = 0.f, gW4 = 0.f, gb4 = 0.f, lsum = 0.f;
    const float invB = 1.f / (float)B;
    const uint32_t n_tiles = (B + kTile - 1) / kTile;
    __syncthreads();
    for (uint32_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        // ---- encode
        {
            const int s = tid & 63, part = tid >> 6;
            const uint32_t k = t * kTile + s;
            const bool valid = k < B;
            V3 p = v3(0.f, 0.f, 0.f), w = v3(0.f, 0.f, 1.f);
            float y = 0.f;
            if (valid) {
                const float4 *q = reinterpret_cast<const float4 *>(pairs + 8 * ((b0 + k) % n_pairs));
                const float4 a = __ldg(q), b = __ldg(q + 1);
                p = v3(a.x, a.y, a.z);
                w = v3(a.w, b.x, b.y);
                y = b.w;
            }
            snet_to_local(N, p, w);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int l = 2 * part + h;
                uint32_t c[3];
                float f[3];
                snet_cell(N, l, p, c, f);
                float a0 = 0.f, a1 = 0.f;
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    const uint32_t i =
                        snet_index(N, l, c[0] + (v & 1), c[1] + ((v >> 1) & 1), c[2] + ((v >> 2) & 1));
                    const float wt = ((v & 1) ? f[0] : 1.f - f[0]) * (((v >> 1) & 1) ? f[1] : 1.f - f[1]) *
                                     (((v >> 2) & 1) ? f[2] : 1.f - f[2]);
                    const float2 e = __ldg(reinterpret_cast<const float2 *>(N.table) + i);
                    a0 = fmaf(wt, e.x, a0);
                    a1 = fmaf(wt, e.y, a1);
                }
                S.X[(2 * l) * kSP + s] = valid ? a0 : 0.f;
                S.X[(2 * l + 1) * kSP + s] = valid ? a1 : 0.f;
            }
            if (part == 0) {
                float Y[16];
                snet_sh16(normalize(w), Y);
#pragma unroll
                for (int j = 0; j < 16; ++j) S.X[(2 * kSnetLevels + j) * kSP + s] = valid ? Y[j] : 0.f;
                S.pl[s] = make_float4(p.x, p.y, p.z, valid ? y : -1.f);
            }
        }
        __syncthreads();
        // ---- forward
        forward_layer(S.Wt1, S.b1, S.X, kSnetIn, S.H1, mg, ng);
        __syncthreads();
        forward_layer(S.Wt2, S.b2, S.H1, kSnetW, S.H2, mg, ng);
        __syncthreads();
        forward_layer(S.Wt3, S.b3, S.H2, kSnetW, S.H3, mg, ng);
        __syncthreads();
        {
            const int s = tid & 63, part = tid >> 6;
            float z = 0.f;
#pragma unroll
            for (int u = 16 * part; u < 16 * part + 16; ++u) z = fmaf(S.W4[u], S.H3[u * kSP + s], z);
            S.zpart[part][s] = z;
        }
        __syncthreads();
        if (tid < kTile) {
            const float z = S.b4 + ((S.zpart[0][tid] + S.zpart[1][tid]) + (S.zpart[2][tid] + S.zpart[3][tid]));
            const float y = S.pl[tid].w;
            float d = 0.f;
            if (y >= 0.f) {
                const float T = 1.f / (1.f + expf(-z)), r = T - y;
                lsum = fmaf(r * r, invB, lsum);
                d = 2.f * r * invB * T * (1.f - T);
            }
            S.dz[tid] = d;
        }
        __syncthreads();
        // ---- layer 4 and the delta of layer 3
        if (tid < kSnetW) {
            float s4 = 0.f;
            for (int s = 0; s < kTile; ++s) s4 = fmaf(S.dz[s], S.H3[tid * kSP + s], s4);
            gW4 += s4;
        }
        if (tid == 0) {
            float s4 = 0.f;
            for (int s = 0; s < kTile; ++s) s4 += S.dz[s];
            gb4 += s4;
        }
        for (int i = tid; i < kSnetW * kTile; i += kTT) {
            const int u = i / kTile, s = i % kTile;
            S.D3[u * kSP + s] = S.H3[u * kSP + s] > 0.f ? S.W4[u] * S.dz[s] : 0.f;
        }
        __syncthreads();
        // ---- layer 3: weight gradient, delta of layer 2
        {
            float acc[4][4];
            zero(acc);
            gemm_mm<4, 4>(S.D3, S.H2, 4 * mg, ng, acc);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) gW3[i][j] += acc[i][j];
        }
        if (tid < kSnetW) gb3 += row_sum(S.D3 + tid * kSP);
        backward_layer(S.W3, S.D3, S.H2, S.D2, mg, ng);
        __syncthreads();
        // ---- layer 2: weight gradient, delta of layer 1 (into D3)
        {
            float acc[4][4];
            zero(acc);
            gemm_mm<4, 4>(S.D2, S.H1, 4 * mg, ng, acc);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) gW2[i][j] += acc[i][j];
        }
        if (tid < kSnetW) gb2 += row_sum(S.D2 + tid * kSP);
        backward_layer(S.W2, S.D2, S.H1, S.D3, mg, ng);
        __syncthreads();
        // ---- layer 1: weight gradient and input gradient
        {
            float acc[4][2];
            zero(acc);
            gemm_mm<4, 2>(S.D3, S.X, 4 * mg, ng, acc);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j) gW1[i][j] += acc[i][j];
        }
        if (tid < kSnetW) gb1 += row_sum(S.D3 + tid * kSP);
        {
            float acc[2][4];
            zero(acc);
            gemm_rr<2, 4>(S.W1, kSnetIn, S.D3, kSP, kSnetW, 2 * mg, 4 * ng, acc);
#pragma unroll
            for (int i = 0; i < 2; ++i)
                *reinterpret_cast<float4 *>(S.DX + (2 * mg + i) * kSP + 4 * ng) =
                    make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
        }
        __syncthreads();
        // ---- hash-table gradient: trilinear weight x input gradient, per corner
        for (int task = tid; task < kTile * kSnetLevels; task += kTT) {
            const int s = task & 63, l = task >> 6;
            const float4 q = S.pl[s];
            if (q.w < 0.f) continue;
            uint32_t c[3];
            float f[3];
            snet_cell(N, l, v3(q.x, q.y, q.z), c, f);
            const float g0 = S.DX[(2 * l) * kSP + s], g1 = S.DX[(2 * l + 1) * kSP + s];
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                const uint32_t i = snet_index(N, l, c[0] + (v & 1), c[1] + ((v >> 1) & 1), c[2] + ((v >> 2) & 1));
                const float wt = ((v & 1) ? f[0] : 1.f - f[0]) * (((v >> 1) & 1) ? f[1] : 1.f - f[1]) *
                                 (((v >> 2) & 1) ? f[2] : 1.f - f[2]);
                grad_add(gacc + 2 * (size_t)i, wt * g0);
                grad_add(gacc + 2 * (size_t)i + 1, wt * g1);
            }
        }
        __syncthreads();
    }
    // ---- flush the block's network gradient and loss
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int u = 4 * mg + i;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            grad_add(gmlp + kSnetOffW2 + u * kSnetW + ng + 16 * j, gW2[i][j]);
            grad_add(gmlp + kSnetOffW3 + u * kSnetW + ng + 16 * j, gW3[i][j]);
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) grad_add(gmlp + u * kSnetIn + ng + 16 * j, gW1[i][j]);
    }
    if (tid < kSnetW) {
        grad_add(gmlp + kSnetOffB1 + tid, gb1);
        grad_add(gmlp + kSnetOffB2 + tid, gb2);
        grad_add(gmlp + kSnetOffB3 + tid, gb3);
        grad_add(gmlp + kSnetOffW4 + tid, gW4);
    }
    if (tid == 0) grad_add(gmlp + kSnetOffB4, gb4);
    if (loss && tid < kTile) {   // two full warps hold the per-pair losses
        float x = lsum;
        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        if ((tid & 31) == 0) atomicAdd(loss, x);
    }
}

// Adam (Kingma and Ba) with bias correction c1 = 1 - b1^t, c2 = 1 - b2^t;
// clears the gradient sums.
__global__ void snet_adam_kernel(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                                 unsigned long long *__restrict__ g, uint64_t n, float lr, float b1, float b2,
                                 float eps, float c1, float c2) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const float gi = grad_value(g[i]);
        const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        g[i] = 0ull;
    }
}

// The gradient as FP32 values; clears the sums.
__global__ void snet_grad_out_kernel(unsigned long long *__restrict__ g, float *__restrict__ out, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        out[i] = grad_value(g[i]);
        g[i] = 0ull;
    }
}

// Rendering copy of the MLP part: FP32 values, rounded to BF16 when asked.
__global__ void snet_refresh_kernel(const float *__restrict__ mlp, float *__restrict__ out, int bf16) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kSnetMlp) return;
    const float x = mlp[i];
    out[i] = bf16 ? __bfloat162float(__float2bfloat16_rn(x)) : x;
}

__global__ void __launch_bounds__(128) snet_eval_kernel(const ShadowNetDev N, const float *__restrict__ pairs,
                                                        uint32_t n, float *__restrict__ out) {
    __shared__ __align__(16) float w[kSnetMlp + 3];
    for (int i = threadIdx.x; i < kSnetMlp; i += blockDim.x) w[i] = N.mlp[i];
    __syncthreads();
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float4 *q = reinterpret_cast<const float4 *>(pairs + 8 * (size_t)k);
    const float4 a = __ldg(q), b = __ldg(q + 1);
    out[k] = snet_eval(N, w, v3(a.x, a.y, a.z), v3(a.w, b.x, b.y));
}

// Training pair i (see mrf_shadow_pairs): point uniform in the field box,
// light, point on it, direction, distance and the FP32-marched transmittance.
__global__ void __launch_bounds__(128) snet_pairs_kernel(const RenderParams P, uint64_t seed, uint64_t first,
                                                         uint32_t n, float *__restrict__ out) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint64_t i = first + k;
    uint64_t c0[4] = {i, 0ull, 0ull, 0ull}, c1[4] = {i, 1ull, 0ull, 0ull};
    philox4x64_10(c0, seed, 0x736861646F77ull);
    philox4x64_10(c1, seed, 0x736861646F77ull);
    const FieldDev &F = P.F;
    V3 p = v3(fmaf(u24(c0[0]), F.hi[0] - F.lo[0], F.lo[0]), fmaf(u24(c0[1]), F.hi[1] - F.lo[1], F.lo[1]),
              fmaf(u24(c0[2]), F.hi[2] - F.lo[2], F.lo[2]));
    if (F.has_pose) {
        // local to world: p = R p_l + t, with R = (to_local rotation)^T
        const float *M = F.to_local;
        const V3 q = p;
        const V3 t = v3(-(M[0] * M[3] + M[4] * M[7] + M[8] * M[11]), -(M[1] * M[3] + M[5] * M[7] + M[9] * M[11]),
                        -(M[2] * M[3] + M[6] * M[7] + M[10] * M[11]));
        p = v3(fmaf(M[0], q.x, fmaf(M[4], q.y, fmaf(M[8], q.z, t.x))),
               fmaf(M[1], q.x, fmaf(M[5], q.y, fmaf(M[9], q.z, t.y))),
               fmaf(M[2], q.x, fmaf(M[6], q.y, fmaf(M[10], q.z, t.z))));
    }
    const int l = min((int)(u24(c0[3]) * (float)P.n_lights), P.n_lights - 1);
    const LightDev &L0 = P.lights[l];
    V3 y = v3(L0.pos[0], L0.pos[1], L0.pos[2]);
    if (L0.kind == MRF_LIGHT_AREA) {
        const float su = sqrtf(u24(c1[0])), b0 = 1.f - su, b1 = u24(c1[1]) * su, b2 = 1.f - b0 - b1;
        y = y * b0 + v3(L0.v1[0], L0.v1[1], L0.v1[2]) * b1 + v3(L0.v2[0], L0.v2[1], L0.v2[2]) * b2;
    }
    V3 w = y - p;
    const float D = sqrtf(dot(w, w));
    w = w * (1.f / D);
    Counters C = {};
    bool stop = false;
    const float depth = march<false>(P, F.mlp, p, w, 0.f, D, nullptr, nullptr, stop, C);
    float4 *o = reinterpret_cast<float4 *>(out + 8 * (size_t)k);
    o[0] = make_float4(p.x, p.y, p.z, w.x);
    o[1] = make_float4(w.y, w.z, D, expf(-depth));
}

// ---------------------------------------------------------------------------
// Tensor-core inference (BF16 weights and activations, FP32 accumulators in
// TMEM): four chained tcgen05 MMAs per tile of 128 shadow rays, M = 128 and
// N = 64 (the last layer padded to N = 16), like the field kernel.
constexpr int kLpW1 = 0, kLpW2 = 4096, kLpW3 = 12288, kLpW4 = 20480, kLpBytes = 22528;
constexpr int kTcGroups = 4;   // 128-ray tiles in flight per CTA (256 TMEM columns: two CTAs per SM)
constexpr int kTcBias = kLpBytes, kTcBars = kTcBias + (3 * kSnetW + 4) * 4, kTcSlot = kTcBars + 8 * kTcGroups,
              kTcA = (kTcSlot + 8 + 127) / 128 * 128, kTcBytes = kTcA + kTcGroups * 16384;
static_assert(kTcBias % 16 == 0, "biases are read as float4");

// byte offset of element (r, k) of an R x K operand in the canonical K-major layout
__device__ __forceinline__ uint32_t umma_off(int r, int k, int K) {
    return (uint32_t)((r >> 3) * (K >> 3) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// BF16 copies of W1 (64 x 32), W2, W3 (64 x 64) and W4 (1 x 64, padded to 16
// rows) in the MMA operand layout, from the FP32 MLP part.
__global__ void snet_pack_lp(const float *__restrict__ mlp, uint8_t *__restrict__ lp) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    auto put = [&](uint32_t off, float v) {
        *reinterpret_cast<__nv_bfloat16 *>(lp + off) = __float2bfloat16_rn(v);
    };
    if (i < kSnetW * kSnetIn) put(kLpW1 + umma_off(i / kSnetIn, i % kSnetIn, kSnetIn), mlp[i]);
    if (i < kSnetW * kSnetW) {
        put(kLpW2 + umma_off(i / kSnetW, i % kSnetW, kSnetW), mlp[kSnetOffW2 + i]);
        put(kLpW3 + umma_off(i / kSnetW, i % kSnetW, kSnetW), mlp[kSnetOffW3 + i]);
    }
    if (i < 16 * kSnetW) {
        const int r = i / kSnetW, k = i % kSnetW;
        put(kLpW4 + umma_off(r, k, kSnetW), r == 0 ? mlp[kSnetOffW4 + k] : 0.f);
    }
}

// Network transmittance on the tensor cores.  Queue mode (queue != NULL): ray
// i is queue[i] = slot * K + q with point hp[slot] and direction sdir[idx],
// result to out[idx]; pairs mode: ray i is pairs[8 i ..], result to out[i].
// n = min(*n_dev, n_host) rays (n_dev nullable).
__global__ void __launch_bounds__(128 * kTcGroups, 2)
    snet_tc_kernel(const ShadowNetDev N, const uint8_t *__restrict__ lp, const float *__restrict__ mlp,
                   const uint32_t *__restrict__ queue, const float4 *__restrict__ hp, const float4 *__restrict__ sdir,
                   int K, const float *__restrict__ pairs, const uint32_t *__restrict__ n_dev, uint32_t n_host,
                   float *__restrict__ out, unsigned *__restrict__ status, unsigned long long *stats) {
    using namespace tc;
    extern __shared__ __align__(128) uint8_t smem[];
    float *sBias = reinterpret_cast<float *>(smem + kTcBias);
    uint32_t *sTmem = reinterpret_cast<uint32_t *>(smem + kTcSlot);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int g = tid >> 7, gt = tid & 127, gw = gt >> 5;
    for (int o = tid * 16; o < kLpBytes; o += 128 * kTcGroups * 16)
        *reinterpret_cast<uint4 *>(smem + o) = __ldg(reinterpret_cast<const uint4 *>(lp + o));
    if (tid < kSnetW) {
        sBias[tid] = mlp[kSnetOffB1 + tid];
        sBias[kSnetW + tid] = mlp[kSnetOffB2 + tid];
        sBias[2 * kSnetW + tid] = mlp[kSnetOffB3 + tid];
    }
    if (tid == 0) sBias[3 * kSnetW] = mlp[kSnetOffB4];
    const uint32_t bar = smem_u32(smem + kTcBars + 8 * g);
    if (gt == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(sTmem)),
                     "r"(64 * kTcGroups)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *sTmem;
    const uint32_t t_acc = tmem + 64u * (uint32_t)g;
    const uint32_t t_row = t_acc + ((uint32_t)(gw * 32) << 16);
    uint8_t *sA = smem + kTcA + g * 16384;
    const uint32_t aA = smem_u32(sA), aW1 = smem_u32(smem + kLpW1), aW2 = smem_u32(smem + kLpW2),
                   aW3 = smem_u32(smem + kLpW3), aW4 = smem_u32(smem + kLpW4);
    constexpr uint32_t id64 = instr_desc(true, 128, 64), id16 = instr_desc(true, 128, 16);
    const uint32_t n = n_dev ? min(*n_dev, n_host) : n_host;
    const int bar_id = 1 + g;
    uint32_t phase = 0, evals = 0;
    bool ok = true;
    const tc::TileLoop tl = tc::cta_tiles(n, kTcGroups, g);
    for (uint32_t tile = tl.first; tile < tl.end; tile += tl.step) {
        const uint32_t i = tile * 128u + gt;
        const bool valid = i < n;
        uint32_t dst = i;
        V3 p = v3(0.f, 0.f, 0.f), w = v3(0.f, 0.f, 1.f);
        if (valid) {
            if (queue) {
                dst = queue[i];
                const float4 h4 = hp[dst / (uint32_t)K], sh = sdir[dst];
                p = v3(h4.x, h4.y, h4.z);
                w = v3(sh.x, sh.y, sh.z);
            } else {
                const float4 *q = reinterpret_cast<const float4 *>(pairs + 8 * (size_t)i);
                const float4 a = __ldg(q), b = __ldg(q + 1);
                p = v3(a.x, a.y, a.z);
                w = v3(a.w, b.x, b.y);
            }
            ++evals;
        }
        snet_to_local(N, p, w);
        {
            float x[kSnetIn];
            snet_encode(N, p, w, x);
#pragma unroll
            for (int c = 0; c < kSnetIn / 8; ++c) {
                uint32_t v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = valid ? pack2<true>(x[8 * c + 2 * q], x[8 * c + 2 * q + 1]) : 0u;
                store_chunk(sA, gt, c, (kSnetIn / 8) * 128, make_uint4(v[0], v[1], v[2], v[3]));
            }
        }
        // layer 1: K = 32
        fence_async_smem();
        fence_before_sync();
        if (group_sync_or(bar_id, !ok)) break;
        if (gt == 0) {
            fence_after_sync();
#pragma unroll
            for (int k = 0; k < kSnetIn / 16; ++k)
                mma_f16(t_acc, smem_desc(aA + 256 * k, 128, 512), smem_desc(aW1 + 256 * k, 128, 512), id64, k);
            mma_commit(bar);
        }
        ok &= mbar_wait(bar, phase);
        phase ^= 1;
        fence_after_sync();
        // layers 2 and 3: K = 64, each fed by the previous epilogue
        const uint32_t wl[2] = {aW2, aW3};
#pragma unroll
        for (int L = 0; L < 2; ++L) {
            {
                uint32_t r[32];
                tmem_ld_x32(t_row, r);
                relu_bias_store<true>(r, sBias + 64 * L, sA, gt, 0);
                tmem_ld_x32(t_row + 32, r);
                relu_bias_store<true>(r, sBias + 64 * L + 32, sA, gt, 4);
            }
            fence_async_smem();
            fence_before_sync();
            if (group_sync_or(bar_id, !ok)) { ok = false; break; }
            if (gt == 0) {
                fence_after_sync();
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    mma_f16(t_acc, smem_desc(aA + 256 * k, 128, 1024), smem_desc(wl[L] + 256 * k, 128, 1024), id64, k);
                mma_commit(bar);
            }
            ok &= mbar_wait(bar, phase);
            phase ^= 1;
            fence_after_sync();
        }
        if (!ok) break;
        // layer 4: N = 16 (row 0 is W4)
        {
            uint32_t r[32];
            tmem_ld_x32(t_row, r);
            relu_bias_store<true>(r, sBias + 128, sA, gt, 0);
            tmem_ld_x32(t_row + 32, r);
            relu_bias_store<true>(r, sBias + 160, sA, gt, 4);
        }
        fence_async_smem();
        fence_before_sync();
        if (group_sync_or(bar_id, !ok)) break;
        if (gt == 0) {
            fence_after_sync();
#pragma unroll
            for (int k = 0; k < 4; ++k)
                mma_f16(t_acc, smem_desc(aA + 256 * k, 128, 1024), smem_desc(aW4 + 256 * k, 128, 1024), id16, k);
            mma_commit(bar);
        }
        ok &= mbar_wait(bar, phase);
        phase ^= 1;
        fence_after_sync();
        {
            uint32_t r[16];
            tmem_ld_x16(t_row, r);
            const float z = __uint_as_float(r[0]) + sBias[3 * kSnetW];
            if (valid) out[dst] = 1.f / (1.f + expf(-z));
        }
        fence_before_sync();
    }
    if (!ok && gt == 0 && status) atomicOr(status, 4u);
    if (stats) {
        Counters C = {};
        C.net = evals;
        flush_counters(stats, C);
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64 * kTcGroups)
                     : "memory");
}

}  // namespace

size_t snet_lp_bytes() { return kLpBytes; }

cudaError_t launch_snet_pack_lp(const float *mlp, uint8_t *lp, cudaStream_t s) {
    snet_pack_lp<<<(kSnetW * kSnetW + 255) / 256, 256, 0, s>>>(mlp, lp);
    return cudaGetLastError();
}

cudaError_t launch_snet_tc(const ShadowNetDev &N, const uint8_t *lp, const float *mlp, const uint32_t *queue,
                           const float4 *hp, const float4 *sdir, int K, const float *pairs, const uint32_t *n_dev,
                           uint32_t n_host, float *out, unsigned *status, unsigned long long *stats, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(snet_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcBytes);
    if (e != cudaSuccess) return e;
    snet_tc_kernel<<<152 * 2, 128 * kTcGroups, kTcBytes, s>>>(N, lp, mlp, queue, hp, sdir, K, pairs, n_dev, n_host,
                                                              out, status, stats);
    return cudaGetLastError();
}

size_t snet_train_smem() { return sizeof(TrainSmem); }

cudaError_t launch_snet_pairs(const RenderParams &P, uint64_t seed, uint64_t first, uint32_t n, float *out,
                              cudaStream_t s) {
    if (!n) return cudaSuccess;
    snet_pairs_kernel<<<(n + 127) / 128, 128, 0, s>>>(P, seed, first, n, out);
    return cudaGetLastError();
}

cudaError_t launch_snet_grad(const ShadowNetDev &N, const float *params, unsigned long long *gacc, const float *pairs,
                             uint64_t n_pairs, uint64_t b0, uint32_t B, float *loss, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(snet_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(TrainSmem));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const uint32_t tiles = (B + kTile - 1) / kTile;
    const int grid = (int)std::min<uint32_t>(tiles, 152u);
    snet_train_kernel<<<grid, kTT, sizeof(TrainSmem), s>>>(N, params, gacc, pairs, n_pairs, b0, B, loss);
    return cudaGetLastError();
}

cudaError_t launch_snet_adam(float *p, float *m, float *v, unsigned long long *g, uint64_t n, float lr, float b1,
                             float b2, float eps, double c1, double c2, cudaStream_t s) {
    snet_adam_kernel<<<152 * 8, 256, 0, s>>>(p, m, v, g, n, lr, b1, b2, eps, (float)c1, (float)c2);
    return cudaGetLastError();
}

cudaError_t launch_snet_grad_out(unsigned long long *g, float *out, uint64_t n, cudaStream_t s) {
    snet_grad_out_kernel<<<152 * 8, 256, 0, s>>>(g, out, n);
    return cudaGetLastError();
}

cudaError_t launch_snet_refresh(const float *mlp, float *out, bool bf16, cudaStream_t s) {
    snet_refresh_kernel<<<(kSnetMlp + 255) / 256, 256, 0, s>>>(mlp, out, bf16 ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_snet_eval(const ShadowNetDev &N, const float *pairs, uint32_t n, float *out, cudaStream_t s) {
    if (!n) return cudaSuccess;
    if (N.lp) return launch_snet_tc(N, N.lp, N.mlp, nullptr, nullptr, nullptr, 1, pairs, nullptr, n, out, nullptr, nullptr, s);
    snet_eval_kernel<<<(n + 127) / 128, 128, 0, s>>>(N, pairs, n, out);
    return cudaGetLastError();
}

}  // namespace mrf
