// Tensor-core evaluation of the hash-grid field (the Instant-NGP field the
// paper renders, Sec. 3.3): multiresolution hash encoding on the CUDA cores,
// then the MLP in -> 64 -> 64 -> 4 on the 5th-generation tensor cores
// (tcgen05.mma, FP16 or BF16 operands, FP32 accumulation in tensor memory).
//
// One CTA of 128 threads owns one 128-sample tile at a time (persistent over
// tiles).  Thread r encodes sample r into row r of the A operand in shared
// memory; one thread issues the MMAs of a layer and commits them to an
// mbarrier; every thread then reads its row of the accumulator back from
// tensor memory (warp w owns lanes 32w..32w+31), applies bias and ReLU in FP32
// and writes the next layer's A operand.  All operands use the canonical
// K-major layout without swizzle: 8-row x 16-byte core matrices stored as 128
// contiguous bytes, K-adjacent core matrices 128 bytes apart (LBO) and
// 8-row groups (K/8) * 128 bytes apart (SBO).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "path.cuh"
#include "tc.cuh"

namespace mrf {
namespace {

using namespace tc;

// relu_bias_store with the bias taken from the field's kernel-parameter copy
// (F.bias_c[kOff .. kOff + 32)): constant-bank operands instead of shared loads.
template <bool kBF16, int kOff>
__device__ __forceinline__ void relu_bias_store_c(const uint32_t (&r)[32], const FieldDev &F, uint8_t *A, int row,
                                                  int chunk0) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = 8 * c + 2 * q;
            w[q] = pack2_relu<kBF16>(__uint_as_float(r[k]) + F.bias_c[kOff + k],
                                     __uint_as_float(r[k + 1]) + F.bias_c[kOff + k + 1]);
        }
        store_chunk(A, row, chunk0 + c, 1024, make_uint4(w[0], w[1], w[2], w[3]));
    }
}

// Shared-memory layout of one CTA: weights, biases and support spheres shared
// by its tile groups, then one mbarrier and one 16 KB A operand per group.
constexpr int kSmemW1 = 0, kSmemW2 = 8192, kSmemW3 = 16384, kSmemBias = 18432;
constexpr int kSmemSupport = kSmemBias + 132 * 4;
static_assert(kSmemBias % 16 == 0, "biases are read as float4");
constexpr int kSupportMax = 64;
constexpr int kSmemBars = kSmemSupport + kSupportMax * 16;
constexpr int kABytes = 16384;
template <int G>
struct Layout {
    static constexpr int bars = kSmemBars;
    static constexpr int tmem_slot = kSmemBars + 8 * G;
    static constexpr int a0 = (tmem_slot + 8 + 127) / 128 * 128;
    static constexpr int bytes = a0 + G * kABytes;
    static constexpr uint32_t tmem_cols = 64 * G;   // 64 accumulator columns per group
};
constexpr int kGroups = 8;   // 128-sample tiles in flight per CTA (one CTA per SM, all 512 TMEM columns)

// Table loads.  The gathers hold the L1 load data pipe near its peak, and
// what it spends per warp request grows with the bytes each lane asks for as
// well as with the number of lanes: on the 1920x1080 frame the field kernel
// took 14.47 ms with 16-byte chunk loads for every level, 13.21 ms with the
// 8-byte pairs below for every level, 13.39 ms with one 4-byte load per
// corner, and 12.93 ms with 4-byte loads on the dense levels and 8-byte pairs
// on the hashed ones (the form used).
//
// Hashed level: corner i0 = x0 ^ a and its x-neighbour i1 = (x0 + 1) ^ a share
// the aligned 8-byte pair holding i0 whenever x0 is even (then i1 = i0 ^ 1);
// one 8-byte load serves both there and i1 is fetched on its own otherwise.
__device__ __forceinline__ void load_pair(const uint32_t *__restrict__ tab, uint32_t i0, uint32_t i1, uint32_t &e0,
                                          uint32_t &e1) {
    const uint32_t c0 = i0 & ~1u;
    const uint2 q = __ldg(reinterpret_cast<const uint2 *>(tab + c0));
    e0 = (i0 & 1u) ? q.y : q.x;
    e1 = ((i1 & ~1u) == c0) ? ((i1 & 1u) ? q.y : q.x) : __ldg(tab + i1);
}

// The corner entries (FP16 pairs) of level l around p and the trilinear weights.
__device__ __forceinline__ void level_corners(const FieldDev &F, int l, V3 p, uint32_t (&e)[8], float (&w)[3]) {
    const uint32_t N = F.res[l];
    int c[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        // p lies in the field box (callers encode only samples with support,
        // which is zero outside it), so u >= 0 and only u = N needs clamping
        const float u = (comp(p, k) - F.lo[k]) * F.ext_inv[k] * (float)N;
        const float fl = fminf(floorf(u), (float)(N - 1));
        c[k] = (int)fl;
        w[k] = u - fl;
    }
    uint32_t idx[8];
    if ((F.dense_mask >> l) & 1u) {
        const uint32_t sy = N + 1, sz = sy * sy;
        const uint32_t b = (uint32_t)c[0] + sy * (uint32_t)c[1] + sz * (uint32_t)c[2];
        idx[0] = b;
        idx[1] = b + 1;
        idx[2] = b + sy;
        idx[3] = b + sy + 1;
        idx[4] = b + sz;
        idx[5] = b + sz + 1;
        idx[6] = b + sy + sz;
        idx[7] = b + sy + sz + 1;
    } else {
        const uint32_t mask = (1u << F.log2T) - 1u;
        const uint32_t x0 = (uint32_t)c[0], x1 = x0 + 1u;
        const uint32_t hy0 = (uint32_t)c[1] * 2654435761u, hy1 = hy0 + 2654435761u;
        const uint32_t hz0 = (uint32_t)c[2] * 805459861u, hz1 = hz0 + 805459861u;
        const uint32_t a00 = hy0 ^ hz0, a10 = hy1 ^ hz0, a01 = hy0 ^ hz1, a11 = hy1 ^ hz1;
        idx[0] = (x0 ^ a00) & mask;
        idx[1] = (x1 ^ a00) & mask;
        idx[2] = (x0 ^ a10) & mask;
        idx[3] = (x1 ^ a10) & mask;
        idx[4] = (x0 ^ a01) & mask;
        idx[5] = (x1 ^ a01) & mask;
        idx[6] = (x0 ^ a11) & mask;
        idx[7] = (x1 ^ a11) & mask;
    }
    const uint32_t *tab = F.table + ((size_t)l << F.log2T);
#pragma unroll
    for (int k = 0; k < 8; ++k) idx[k] = checked_index(idx[k], 1ull << F.log2T, F.status);
    if ((F.dense_mask >> l) & 1u) {
#pragma unroll
        for (int k = 0; k < 8; ++k) e[k] = __ldg(tab + idx[k]);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) load_pair(tab, idx[2 * k], idx[2 * k + 1], e[2 * k], e[2 * k + 1]);
    }
}

// Level l of the encoding at p, interpolated in FP32 (FP16 kernels).
__device__ __forceinline__ float2 encode_level_pairs(const FieldDev &F, int l, V3 p) {
    uint32_t e[8];
    float w[3];
    level_corners(F, l, p, e, w);
    float2 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = __half22float2(*reinterpret_cast<const __half2 *>(&e[k]));
    float2 a[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
        a[k] = make_float2(fmaf(w[0], v[2 * k + 1].x - v[2 * k].x, v[2 * k].x),
                           fmaf(w[0], v[2 * k + 1].y - v[2 * k].y, v[2 * k].y));
    const float2 b0 = make_float2(fmaf(w[1], a[1].x - a[0].x, a[0].x), fmaf(w[1], a[1].y - a[0].y, a[0].y));
    const float2 b1 = make_float2(fmaf(w[1], a[3].x - a[2].x, a[2].x), fmaf(w[1], a[3].y - a[2].y, a[2].y));
    return make_float2(fmaf(w[2], b1.x - b0.x, b0.x), fmaf(w[2], b1.y - b0.y, b0.y));
}

// The same level in packed FP16 arithmetic (BF16 kernels): the corner pairs are
// FP16 already and the trilinear weights are rounded to FP16 once, so the seven
// interpolations are a subtraction and a fused multiply-add of a pair each.
// Their rounding (2^-11) stays below the BF16 rounding of the result (2^-8).
__device__ __forceinline__ __half2 encode_level_h2(const FieldDev &F, int l, V3 p) {
    uint32_t e[8];
    float w[3];
    level_corners(F, l, p, e, w);
    __half2 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = *reinterpret_cast<const __half2 *>(&e[k]);
    const __half2 wx = __float2half2_rn(w[0]), wy = __float2half2_rn(w[1]), wz = __float2half2_rn(w[2]);
    __half2 a[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] = __hfma2(wx, __hsub2(v[2 * k + 1], v[2 * k]), v[2 * k]);
    const __half2 b0 = __hfma2(wy, __hsub2(a[1], a[0]), a[0]);
    const __half2 b1 = __hfma2(wy, __hsub2(a[3], a[2]), a[2]);
    return __hfma2(wz, __hsub2(b1, b0), b0);
}

// G tile groups of 128 threads per CTA; group g owns TMEM columns [64g, 64g + 64),
// its own A operand and mbarrier, and synchronises on named barrier 1 + g.
template <bool kBF16, int G>
__global__ void __launch_bounds__(128 * G, 8 / G)
    field_tc_kernel(const FieldDev F, const float *__restrict__ pts, int stride, const uint32_t *__restrict__ n_dev,
                    uint32_t n_host, float4 *__restrict__ out, unsigned *__restrict__ status) {
    using Lo = Layout<G>;
    extern __shared__ __align__(128) uint8_t smem[];
    uint32_t *sTmem = reinterpret_cast<uint32_t *>(smem + Lo::tmem_slot);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int g = tid >> 7, gt = tid & 127, gw = gt >> 5;
    const int n_in = F.n_in, kin = n_in / 16, sbo_in = (n_in / 8) * 128;
    constexpr int kThreadsCta = 128 * G;

    // stage the low-precision weights (already in the canonical layout) and the support spheres
    {
        const int w1_bytes = 64 * n_in * 2;
        const uint8_t *src = reinterpret_cast<const uint8_t *>(F.mlp_lp) + (kBF16 ? w1_bytes + 10240 : 0);
        for (int o = tid * 16; o < w1_bytes; o += kThreadsCta * 16)
            *reinterpret_cast<uint4 *>(smem + kSmemW1 + o) = __ldg(reinterpret_cast<const uint4 *>(src + o));
        for (int o = tid * 16; o < 10240; o += kThreadsCta * 16)
            *reinterpret_cast<uint4 *>(smem + kSmemW2 + o) = __ldg(reinterpret_cast<const uint4 *>(src + w1_bytes + o));
    }
    float4 *sSup = reinterpret_cast<float4 *>(smem + kSmemSupport);
    const bool sup_smem = F.n_support <= kSupportMax;
    if (sup_smem)
        for (int k = tid; k < F.n_support; k += kThreadsCta) sSup[k] = __ldg(F.support + k);
    const float4 *sup = sup_smem ? sSup : F.support;
    const uint32_t bar = smem_u32(smem + Lo::bars + 8 * g);
    if (gt == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(sTmem)),
                     "r"(Lo::tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *sTmem;
    const uint32_t t_acc = tmem + 64u * (uint32_t)g;                       // this group's columns
    const uint32_t t_row = t_acc + ((uint32_t)(gw * 32) << 16);            // this warp's lanes
    uint8_t *sA = smem + Lo::a0 + g * kABytes;
    const uint32_t aA = smem_u32(sA), aW1 = smem_u32(smem + kSmemW1), aW2 = smem_u32(smem + kSmemW2),
                   aW3 = smem_u32(smem + kSmemW3);
    constexpr uint32_t id64 = instr_desc(kBF16, 128, 64), id16 = instr_desc(kBF16, 128, 16);
    const uint32_t n = n_dev ? min(*n_dev, n_host) : n_host;
    const int bar_id = 1 + g;
    uint32_t phase = 0;
    bool ok = true;

    // One warp of the group polls the MMA's mbarrier; the other three wait at the
    // group's named barrier, which also carries the give-up flag, so that the
    // wait costs no shared-memory polls next to the table gathers.  False: the
    // group leaves its loop.
    auto wait_mma = [&]() -> bool {
        if (gw == 0) ok &= mbar_wait(bar, phase);
        phase ^= 1;
        fence_before_sync();
        const bool bad = group_sync_or(bar_id, !ok);
        fence_after_sync();
        return !bad;
    };
    const TileLoop tl = cta_tiles(n, G, g);
    for (uint32_t tile = tl.first; tile < tl.end; tile += tl.step) {
        const uint32_t i = tile * 128u + gt;
        const bool valid = i < n;
        V3 p = v3(0.f, 0.f, 0.f);
        float s = 0.f, dl = 1.f;   // support, interval length (stride 4)
        if (valid) {
            if (stride == 4) {
                const float4 q = reinterpret_cast<const float4 *>(pts)[i];
                p = v3(q.x, q.y, q.z);
                dl = q.w;
            } else {
                p = v3(pts[(size_t)stride * i], pts[(size_t)stride * i + 1], pts[(size_t)stride * i + 2]);
            }
            // support(p): max over the spheres, clamped at 0 (no sphere: no density)
            for (int k = 0; k < F.n_support; ++k) {
                const float4 c = sup[k];
                const float dx = p.x - c.x, dy = p.y - c.y, dz = p.z - c.z;
                s = fmaxf(s, 1.0f - (dx * dx + dy * dy + dz * dz) * c.w);
            }
            if (!inside_field_box(F, p)) s = 0.f;
        }
        // hash encoding -> A (K = n_in)
        for (int c = 0; c < n_in / 8; ++c) {
            uint32_t w[4] = {0u, 0u, 0u, 0u};
            if (s > 0.f) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (kBF16) {
                        const float2 f = __half22float2(encode_level_h2(F, 4 * c + q, p));
                        w[q] = pack2<kBF16>(f.x, f.y);
                    } else {
                        const float2 f = encode_level_pairs(F, 4 * c + q, p);
                        w[q] = pack2<kBF16>(f.x, f.y);
                    }
                }
            }
            store_chunk(sA, gt, c, sbo_in, make_uint4(w[0], w[1], w[2], w[3]));
        }
        fence_async_smem();
        fence_before_sync();
        if (group_sync_or(bar_id, !ok)) break;
        if (gt == 0) {
            fence_after_sync();
            for (int k = 0; k < kin; ++k)
                mma_f16(t_acc, smem_desc(aA + 256 * k, 128, sbo_in), smem_desc(aW1 + 256 * k, 128, sbo_in), id64, k);
            mma_commit(bar);
        }
        if (!wait_mma()) break;
        // layer 1 epilogue -> A (K = 64)
        {
            uint32_t r[32];
            tmem_ld_x32(t_row, r);
            relu_bias_store_c<kBF16, 0>(r, F, sA, gt, 0);
            tmem_ld_x32(t_row + 32, r);
            relu_bias_store_c<kBF16, 32>(r, F, sA, gt, 4);
        }
        fence_async_smem();
        fence_before_sync();
        if (group_sync_or(bar_id, !ok)) break;
        if (gt == 0) {
            fence_after_sync();
#pragma unroll
            for (int k = 0; k < 4; ++k)
                mma_f16(t_acc, smem_desc(aA + 256 * k, 128, 1024), smem_desc(aW2 + 256 * k, 128, 1024), id64, k);
            mma_commit(bar);
        }
        if (!wait_mma()) break;
        // layer 2 epilogue -> A (K = 64)
        {
            uint32_t r[32];
            tmem_ld_x32(t_row, r);
            relu_bias_store_c<kBF16, 64>(r, F, sA, gt, 0);
            tmem_ld_x32(t_row + 32, r);
            relu_bias_store_c<kBF16, 96>(r, F, sA, gt, 4);
        }
        fence_async_smem();
        fence_before_sync();
        if (group_sync_or(bar_id, !ok)) break;
        if (gt == 0) {
            fence_after_sync();
#pragma unroll
            for (int k = 0; k < 4; ++k)
                mma_f16(t_acc, smem_desc(aA + 256 * k, 128, 1024), smem_desc(aW3 + 256 * k, 128, 1024), id16, k);
            mma_commit(bar);
        }
        if (!wait_mma()) break;
        {
            uint32_t r[16];
            tmem_ld_x16(t_row, r);
            const float o0 = __uint_as_float(r[0]) + F.bias_c[128], o1 = __uint_as_float(r[1]) + F.bias_c[129],
                        o2 = __uint_as_float(r[2]) + F.bias_c[130], o3 = __uint_as_float(r[3]) + F.bias_c[131];
            if (valid) {
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (s > 0.f)
                    v = make_float4(s * expf(fminf(o0, 15.f)) * dl, softplusf(o1), softplusf(o2), softplusf(o3));
                out[i] = v;
            }
        }
        fence_before_sync();
    }
    if (!ok && gt == 0 && status) atomicOr(status, 4u);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Lo::tmem_cols)
                     : "memory");
}

// ---------------------------------------------------------------------------
// The same field with every layer's A operand in tensor memory: the thread of
// a row writes the row's encoding (K = 32) and, after each hidden layer, its
// 64 activations (K = 64) with tcgen05.st, and the MMAs read A from tensor
// memory.  No A operand goes through shared memory, whose stores share the L1
// data pipe with the table gathers.  A group needs 64 accumulator and 32
// operand columns: five groups (640 threads) per SM, 480 of the 512 columns.
// A in tensor memory: row r of the tile in lane r, K along the columns, two
// 16-bit elements per 32-bit column (the low half first), so a K = 16 step is 8
// columns.
constexpr int kTmGroups = 5;
constexpr uint32_t kTmGroupCols = 96;   // accumulator [0, 64), A operand [64, 96)
constexpr int kTmBars = kSmemBars;
constexpr int kTmSlot = kTmBars + 8 * kTmGroups;
constexpr int kTmBytes = kTmSlot + 16;

__device__ __forceinline__ void tmem_st_x16(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]) : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// kind::f16 MMA with A read from tensor memory at a_tmem
__device__ __forceinline__ void mma_f16_tmem_a(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                               uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc));
}

// bias (kernel-parameter constant bank) and ReLU of 32 accumulator columns, packed in pairs
template <bool kBF16, int kOff>
__device__ __forceinline__ void relu_bias_pack(const uint32_t (&r)[32], const FieldDev &F, uint32_t (&w)[16]) {
#pragma unroll
    for (int q = 0; q < 16; ++q)
        w[q] = pack2_relu<kBF16>(__uint_as_float(r[2 * q]) + F.bias_c[kOff + 2 * q],
                                 __uint_as_float(r[2 * q + 1]) + F.bias_c[kOff + 2 * q + 1]);
}

template <bool kBF16>
__global__ void __launch_bounds__(128 * kTmGroups, 1)
    field_tc_tmem_kernel(const FieldDev F, const float *__restrict__ pts, int stride,
                         const uint32_t *__restrict__ n_dev, uint32_t n_host, float4 *__restrict__ out,
                         unsigned *__restrict__ status) {
    extern __shared__ __align__(128) uint8_t smem[];
    uint32_t *sTmem = reinterpret_cast<uint32_t *>(smem + kTmSlot);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int g = tid >> 7, gt = tid & 127, gw = gt >> 5;
    const int n_in = F.n_in, kin = n_in / 16, sbo_in = (n_in / 8) * 128;
    constexpr int kThreadsCta = 128 * kTmGroups;
    {
        const int w1_bytes = 64 * n_in * 2;
        const uint8_t *src = reinterpret_cast<const uint8_t *>(F.mlp_lp) + (kBF16 ? w1_bytes + 10240 : 0);
        for (int o = tid * 16; o < w1_bytes; o += kThreadsCta * 16)
            *reinterpret_cast<uint4 *>(smem + kSmemW1 + o) = __ldg(reinterpret_cast<const uint4 *>(src + o));
        for (int o = tid * 16; o < 10240; o += kThreadsCta * 16)
            *reinterpret_cast<uint4 *>(smem + kSmemW2 + o) = __ldg(reinterpret_cast<const uint4 *>(src + w1_bytes + o));
    }
    float4 *sSup = reinterpret_cast<float4 *>(smem + kSmemSupport);
    const bool sup_smem = F.n_support <= kSupportMax;
    if (sup_smem)
        for (int k = tid; k < F.n_support; k += kThreadsCta) sSup[k] = __ldg(F.support + k);
    const float4 *sup = sup_smem ? sSup : F.support;
    const uint32_t bar = smem_u32(smem + kTmBars + 8 * g);
    if (gt == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(sTmem)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *sTmem;
    const uint32_t t_acc = tmem + kTmGroupCols * (uint32_t)g;           // this group's accumulator columns
    const uint32_t t_a = t_acc + 64u;                                   // and its A operand
    const uint32_t lanes = (uint32_t)(gw * 32) << 16;                   // this warp's lanes
    const uint32_t aW1 = smem_u32(smem + kSmemW1), aW2 = smem_u32(smem + kSmemW2), aW3 = smem_u32(smem + kSmemW3);
    constexpr uint32_t id64 = instr_desc(kBF16, 128, 64), id16 = instr_desc(kBF16, 128, 16);
    const uint32_t n = n_dev ? min(*n_dev, n_host) : n_host;
    const int bar_id = 1 + g;
    uint32_t phase = 0;
    bool ok = true;

    auto wait_mma = [&]() -> bool {
        if (gw == 0) ok &= mbar_wait(bar, phase);
        phase ^= 1;
        fence_before_sync();
        const bool bad = group_sync_or(bar_id, !ok);
        fence_after_sync();
        return !bad;
    };
    // the operand written by this group's threads is complete: the MMAs of a layer may read it
    auto operand_ready = [&]() -> bool {
        tmem_st_wait();
        fence_before_sync();
        return !group_sync_or(bar_id, !ok);
    };
    const TileLoop tl = cta_tiles(n, kTmGroups, g);
    for (uint32_t tile = tl.first; tile < tl.end; tile += tl.step) {
        const uint32_t i = tile * 128u + gt;
        const bool valid = i < n;
        V3 p = v3(0.f, 0.f, 0.f);
        float s = 0.f, dl = 1.f;   // support, interval length (stride 4)
        if (valid) {
            if (stride == 4) {
                const float4 q = reinterpret_cast<const float4 *>(pts)[i];
                p = v3(q.x, q.y, q.z);
                dl = q.w;
            } else {
                p = v3(pts[(size_t)stride * i], pts[(size_t)stride * i + 1], pts[(size_t)stride * i + 2]);
            }
            // support(p): max over the spheres, clamped at 0 (no sphere: no density)
            for (int k = 0; k < F.n_support; ++k) {
                const float4 c = sup[k];
                const float dx = p.x - c.x, dy = p.y - c.y, dz = p.z - c.z;
                s = fmaxf(s, 1.0f - (dx * dx + dy * dy + dz * dz) * c.w);
            }
            if (!inside_field_box(F, p)) s = 0.f;
        }
        // hash encoding -> A (K = n_in = 32: 16 columns)
        {
            uint32_t w[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                w[q] = 0u;
                if (s > 0.f) {
                    if (kBF16) {
                        const float2 f = __half22float2(encode_level_h2(F, q, p));
                        w[q] = pack2<kBF16>(f.x, f.y);
                    } else {
                        const float2 f = encode_level_pairs(F, q, p);
                        w[q] = pack2<kBF16>(f.x, f.y);
                    }
                }
            }
            tmem_st_x16(t_a + lanes, w);
        }
        if (!operand_ready()) break;
        if (gt == 0) {
            fence_after_sync();
            for (int k = 0; k < kin; ++k)
                mma_f16_tmem_a(t_acc, t_a + 8u * (uint32_t)k, smem_desc(aW1 + 256 * k, 128, sbo_in), id64, k);
            mma_commit(bar);
        }
        if (!wait_mma()) break;
        // layer 1 epilogue -> A (K = 64: 32 columns)
        {
            uint32_t r[32], w[16];
            tmem_ld_x32(t_acc + lanes, r);
            relu_bias_pack<kBF16, 0>(r, F, w);
            tmem_st_x16(t_a + lanes, w);
            tmem_ld_x32(t_acc + lanes + 32, r);
            relu_bias_pack<kBF16, 32>(r, F, w);
            tmem_st_x16(t_a + lanes + 16, w);
        }
        if (!operand_ready()) break;
        if (gt == 0) {
            fence_after_sync();
#pragma unroll
            for (int k = 0; k < 4; ++k)
                mma_f16_tmem_a(t_acc, t_a + 8u * (uint32_t)k, smem_desc(aW2 + 256 * k, 128, 1024), id64, k);
            mma_commit(bar);
        }
        if (!wait_mma()) break;
        // layer 2 epilogue -> A (K = 64)
        {
            uint32_t r[32], w[16];
            tmem_ld_x32(t_acc + lanes, r);
            relu_bias_pack<kBF16, 64>(r, F, w);
            tmem_st_x16(t_a + lanes, w);
            tmem_ld_x32(t_acc + lanes + 32, r);
            relu_bias_pack<kBF16, 96>(r, F, w);
            tmem_st_x16(t_a + lanes + 16, w);
        }
        if (!operand_ready()) break;
        if (gt == 0) {
            fence_after_sync();
#pragma unroll
            for (int k = 0; k < 4; ++k)
                mma_f16_tmem_a(t_acc, t_a + 8u * (uint32_t)k, smem_desc(aW3 + 256 * k, 128, 1024), id16, k);
            mma_commit(bar);
        }
        if (!wait_mma()) break;
        {
            uint32_t r[16];
            tmem_ld_x16(t_acc + lanes, r);
            const float o0 = __uint_as_float(r[0]) + F.bias_c[128], o1 = __uint_as_float(r[1]) + F.bias_c[129],
                        o2 = __uint_as_float(r[2]) + F.bias_c[130], o3 = __uint_as_float(r[3]) + F.bias_c[131];
            if (valid) {
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (s > 0.f)
                    v = make_float4(s * expf(fminf(o0, 15.f)) * dl, softplusf(o1), softplusf(o2), softplusf(o3));
                out[i] = v;
            }
        }
        fence_before_sync();
    }
    if (!ok && gt == 0 && status) atomicOr(status, 4u);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

// ---------------------------------------------------------------------------
// View-dependent fields: five chained MMAs per 128-sample tile.  Layer 1
// (in -> 64), the density head (64 -> 16, N = 16), then the colour network on
// [head outputs | sh16(view direction)] (32 -> 64 -> 64 -> 3, the last padded
// to N = 16).  Operand block of each precision (bytes): W1 (64 x 32) at 0,
// Wd (16 x 64) at 4096, Wc1 (64 x 32) at 6144, Wc2 (64 x 64) at 10240,
// Wc3 (16 x 64, rows 3.. zero) at 18432; 20,480 bytes.
constexpr int kVW1 = 0, kVWd = 4096, kVWc1 = 6144, kVWc2 = 10240, kVWc3 = 18432, kVWBytes = 20480;
constexpr int kVBias = kVWBytes;                       // b1[64] bd[16] bc1[64] bc2[64] bc3[4]
constexpr int kVSupport = kVBias + 212 * 4;
static_assert(kVBias % 16 == 0, "biases are read as float4");
constexpr int kVBars = kVSupport + kSupportMax * 16;
template <int G>
struct LayoutV {
    static constexpr int bars = kVBars;
    static constexpr int tmem_slot = kVBars + 8 * G;
    static constexpr int a0 = (tmem_slot + 8 + 127) / 128 * 128;
    static constexpr int bytes = a0 + G * kABytes;
    static constexpr uint32_t tmem_cols = 64 * G;
};

template <bool kBF16, int G>
__global__ void __launch_bounds__(128 * G, 8 / G)
    field_tc_view_kernel(const FieldDev F, const float *__restrict__ pts, int stride, const float4 *__restrict__ dirs,
                         const uint32_t *__restrict__ n_dev, uint32_t n_host, float4 *__restrict__ out,
                         unsigned *__restrict__ status) {
    using Lo = LayoutV<G>;
    extern __shared__ __align__(128) uint8_t smem[];
    uint32_t *sTmem = reinterpret_cast<uint32_t *>(smem + Lo::tmem_slot);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int g = tid >> 7, gt = tid & 127, gw = gt >> 5;
    constexpr int kThreadsCta = 128 * G;
    {
        const uint8_t *src = reinterpret_cast<const uint8_t *>(F.mlp_lp) + (kBF16 ? kVWBytes : 0);
        for (int o = tid * 16; o < kVWBytes; o += kThreadsCta * 16)
            *reinterpret_cast<uint4 *>(smem + o) = __ldg(reinterpret_cast<const uint4 *>(src + o));
    }
    float4 *sSup = reinterpret_cast<float4 *>(smem + kVSupport);
    const bool sup_smem = F.n_support <= kSupportMax;
    if (sup_smem)
        for (int k = tid; k < F.n_support; k += kThreadsCta) sSup[k] = __ldg(F.support + k);
    const float4 *sup = sup_smem ? sSup : F.support;
    const uint32_t bar = smem_u32(smem + Lo::bars + 8 * g);
    if (gt == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(sTmem)),
                     "r"(Lo::tmem_cols)
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
    uint8_t *sA = smem + Lo::a0 + g * kABytes;
    const uint32_t aA = smem_u32(sA), aW1 = smem_u32(smem + kVW1), aWd = smem_u32(smem + kVWd),
                   aWc1 = smem_u32(smem + kVWc1), aWc2 = smem_u32(smem + kVWc2), aWc3 = smem_u32(smem + kVWc3);
    constexpr uint32_t id64 = instr_desc(kBF16, 128, 64), id16 = instr_desc(kBF16, 128, 16);
    const uint32_t n = n_dev ? min(*n_dev, n_host) : n_host;
    const int bar_id = 1 + g;
    uint32_t phase = 0;
    bool ok = true;

    // issue the K steps of one layer from a K-major A (sbo) against weights w
    auto layer = [&](uint32_t w, int ksteps, int sbo, uint32_t idesc) {
        fence_async_smem();
        fence_before_sync();
        if (group_sync_or(bar_id, !ok)) return false;
        if (gt == 0) {
            fence_after_sync();
            for (int k = 0; k < ksteps; ++k)
                mma_f16(t_acc, smem_desc(aA + 256 * k, 128, sbo), smem_desc(w + 256 * k, 128, sbo), idesc, k);
            mma_commit(bar);
        }
        ok &= mbar_wait(bar, phase);
        phase ^= 1;
        fence_after_sync();
        return true;
    };

    const TileLoop tl = cta_tiles(n, G, g);
    for (uint32_t tile = tl.first; tile < tl.end; tile += tl.step) {
        const uint32_t i = tile * 128u + gt;
        const bool valid = i < n;
        V3 p = v3(0.f, 0.f, 0.f), dv = v3(0.f, 0.f, 1.f);
        float s = 0.f, dl = 1.f;   // support, interval length (stride 4)
        if (valid) {
            if (stride == 4) {
                const float4 q = reinterpret_cast<const float4 *>(pts)[i];
                p = v3(q.x, q.y, q.z);
                dl = q.w;
            } else {
                p = v3(pts[(size_t)stride * i], pts[(size_t)stride * i + 1], pts[(size_t)stride * i + 2]);
            }
            if (dirs) {
                const float4 q = dirs[i];
                dv = v3(q.x, q.y, q.z);
            }
            // support(p): max over the spheres, clamped at 0 (no sphere: no density)
            for (int k = 0; k < F.n_support; ++k) {
                const float4 c = sup[k];
                const float dx = p.x - c.x, dy = p.y - c.y, dz = p.z - c.z;
                s = fmaxf(s, 1.0f - (dx * dx + dy * dy + dz * dz) * c.w);
            }
            if (!inside_field_box(F, p)) s = 0.f;
        }
        for (int c = 0; c < 4; ++c) {
            uint32_t w[4] = {0u, 0u, 0u, 0u};
            if (s > 0.f) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (kBF16) {
                        const float2 f = __half22float2(encode_level_h2(F, 4 * c + q, p));
                        w[q] = pack2<kBF16>(f.x, f.y);
                    } else {
                        const float2 f = encode_level_pairs(F, 4 * c + q, p);
                        w[q] = pack2<kBF16>(f.x, f.y);
                    }
                }
            }
            store_chunk(sA, gt, c, 512, make_uint4(w[0], w[1], w[2], w[3]));
        }
        if (!layer(aW1, 2, 512, id64)) break;
        {   // layer 1 epilogue -> A (K = 64)
            uint32_t r[32];
            tmem_ld_x32(t_row, r);
            relu_bias_store_c<kBF16, 0>(r, F, sA, gt, 0);
            tmem_ld_x32(t_row + 32, r);
            relu_bias_store_c<kBF16, 32>(r, F, sA, gt, 4);
        }
        if (!layer(aWd, 4, 1024, id16)) break;
        float sigma;
        {   // density head: sigma, and A (K = 32) = [head outputs | sh16(view)]
            uint32_t r[16];
            tmem_ld_x16(t_row, r);
            float x[32];
#pragma unroll
            for (int k = 0; k < 16; ++k) x[k] = __uint_as_float(r[k]) + F.bias_c[64 + k];
            sigma = s * expf(fminf(x[0], 15.f));
            sh16(normalize(dv), x + 16);
#pragma unroll
            for (int c = 0; c < 4; ++c)
                store_chunk(sA, gt, c, 512,
                            make_uint4(pack2<kBF16>(x[8 * c], x[8 * c + 1]), pack2<kBF16>(x[8 * c + 2], x[8 * c + 3]),
                                       pack2<kBF16>(x[8 * c + 4], x[8 * c + 5]),
                                       pack2<kBF16>(x[8 * c + 6], x[8 * c + 7])));
        }
        if (!layer(aWc1, 2, 512, id64)) break;
        {
            uint32_t r[32];
            tmem_ld_x32(t_row, r);
            relu_bias_store_c<kBF16, 80>(r, F, sA, gt, 0);
            tmem_ld_x32(t_row + 32, r);
            relu_bias_store_c<kBF16, 112>(r, F, sA, gt, 4);
        }
        if (!layer(aWc2, 4, 1024, id64)) break;
        {
            uint32_t r[32];
            tmem_ld_x32(t_row, r);
            relu_bias_store_c<kBF16, 144>(r, F, sA, gt, 0);
            tmem_ld_x32(t_row + 32, r);
            relu_bias_store_c<kBF16, 176>(r, F, sA, gt, 4);
        }
        if (!layer(aWc3, 4, 1024, id16)) break;
        {
            uint32_t r[16];
            tmem_ld_x16(t_row, r);
            if (valid) {
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (s > 0.f) {
                    v = make_float4(sigma * dl, softplusf(__uint_as_float(r[0]) + F.bias_c[208]),
                                    softplusf(__uint_as_float(r[1]) + F.bias_c[209]),
                                    softplusf(__uint_as_float(r[2]) + F.bias_c[210]));
                }
                out[i] = v;
            }
        }
        fence_before_sync();
    }
    if (!ok && gt == 0 && status) atomicOr(status, 4u);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Lo::tmem_cols)
                     : "memory");
}

}  // namespace

// CTAs per SM of the persistent launch: 8 groups take all 512 TMEM columns
// (one CTA), 4 groups half of them (two CTAs)
int field_tc_blocks_per_sm(int groups) { return groups == 4 ? 2 : 1; }   // 5 and 8 groups: one CTA per SM

template <int G>
static cudaError_t launch_groups(bool bf16, const FieldDev &F, const float *pts, int stride, const uint32_t *n_dev,
                                 uint32_t n_host, float4 *out, unsigned *status, int grid, cudaStream_t s) {
    auto kern = bf16 ? field_tc_kernel<true, G> : field_tc_kernel<false, G>;
    constexpr int bytes = Layout<G>::bytes;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    if (grid <= 0) grid = 1;
    kern<<<grid, 128 * G, bytes, s>>>(F, pts, stride, n_dev, n_host, out, status);
    return cudaGetLastError();
}

template <int G>
static cudaError_t launch_view_groups(bool bf16, const FieldDev &F, const float *pts, int stride, const float4 *dirs,
                                      const uint32_t *n_dev, uint32_t n_host, float4 *out, unsigned *status, int grid,
                                      cudaStream_t s) {
    auto kern = bf16 ? field_tc_view_kernel<true, G> : field_tc_view_kernel<false, G>;
    constexpr int bytes = LayoutV<G>::bytes;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    if (grid <= 0) grid = 1;
    kern<<<grid, 128 * G, bytes, s>>>(F, pts, stride, dirs, n_dev, n_host, out, status);
    return cudaGetLastError();
}

cudaError_t launch_field_tc_view(const FieldDev &F, bool bf16, const float *pts, int stride, const float4 *dirs,
                                 const uint32_t *n_dev, uint32_t n_host, float4 *out, unsigned *status, int grid,
                                 cudaStream_t s, int groups) {
    if (groups == 4) return launch_view_groups<4>(bf16, F, pts, stride, dirs, n_dev, n_host, out, status, grid, s);
    return launch_view_groups<kGroups>(bf16, F, pts, stride, dirs, n_dev, n_host, out, status, grid, s);
}

cudaError_t launch_field_tc(const FieldDev &F, bool bf16, const float *pts, int stride, const uint32_t *n_dev,
                            uint32_t n_host, float4 *out, unsigned *status, int grid, cudaStream_t s, int groups) {
    if (groups == kTmGroups && F.n_in == 32) {   // A operands in tensor memory (one CTA of five groups per SM)
        auto kern = bf16 ? field_tc_tmem_kernel<true> : field_tc_tmem_kernel<false>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kTmBytes);
        if (e != cudaSuccess) return e;
        kern<<<grid <= 0 ? 1 : grid, 128 * kTmGroups, kTmBytes, s>>>(F, pts, stride, n_dev, n_host, out, status);
        return cudaGetLastError();
    }
    if (groups == 4) return launch_groups<4>(bf16, F, pts, stride, n_dev, n_host, out, status, grid, s);
    return launch_groups<kGroups>(bf16, F, pts, stride, n_dev, n_host, out, status, grid, s);
}

}  // namespace mrf
