// tcgen05 building blocks shared by the tensor-core kernels (field_tc.cu,
// shadow_net.cu): shared-memory and instruction descriptors of kind::f16 MMAs
// with FP32 accumulators in TMEM, commit and bounded mbarrier waits, fences,
// named-barrier OR-reduction, TMEM loads, and the canonical no-swizzle K-major
// operand layout (8-row x 16-byte core matrices, LBO 128 B between K chunks,
// SBO (K/8) x 128 B between 8-row groups).
#pragma once
#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace mrf {
namespace tc {

constexpr long long kWaitCycles = 2000000000ll;  // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory matrix descriptor: start, LBO, SBO (all >> 4),
// descriptor version 1 at bits 46-47, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: D = F32, A = B = F16 (0) or BF16 (1),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t instr_desc(bool bf16, int m, int n) {
    return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// Waits for phase `parity` of the mbarrier for at most `budget` SM cycles;
// false when it gave up.  Each try_wait may suspend the thread for up to
// kSuspendNs (it resumes as soon as the phase completes), so a wait on an MMA
// costs a few polls of the barrier instead of one per scheduling round: the
// polls are shared-memory accesses that compete with the table gathers for the
// L1 data pipe.
constexpr uint32_t kSuspendNs = 20000;
__device__ __forceinline__ bool mbar_wait_budget(uint32_t bar, uint32_t parity, long long budget) {
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity), "r"(kSuspendNs)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > budget) return false;
    }
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) { return mbar_wait_budget(bar, parity, kWaitCycles); }

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// barrier over the 128 threads of one tile group (named barrier `id`), OR-reducing `pred`
__device__ __forceinline__ bool group_sync_or(int id, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "barrier.red.or.pred q, %2, 128, p;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void tmem_ld_x32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld_x16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <bool kBF16>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
    if (kBF16) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    } else {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
}

// pack2 of (max(a, 0), max(b, 0)) in one conversion with ReLU (cvt.rn.relu
// rounds like pack2 and takes negative inputs to zero); a goes to the low half.
template <bool kBF16>
__device__ __forceinline__ uint32_t pack2_relu(float a, float b) {
    uint32_t d;
    if (kBF16)
        asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
    else
        asm("cvt.rn.relu.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
    return d;
}

// 8 consecutive K values of row `row` into the canonical layout (sbo = (K/8)*128)
__device__ __forceinline__ void store_chunk(uint8_t *base, int row, int chunk, int sbo, uint4 v) {
    *reinterpret_cast<uint4 *>(base + (row >> 3) * sbo + chunk * 128 + (row & 7) * 16) = v;
}

// ReLU(accumulator + bias) of 32 columns to four 16-byte chunks of A.  `bias`
// is a 16-byte aligned shared-memory array: every lane reads the same
// addresses, as 128-bit loads (8 instead of 32 shared-memory wavefronts).
template <bool kBF16>
__device__ __forceinline__ void relu_bias_store(const uint32_t (&r)[32], const float *bias, uint8_t *A, int row,
                                                int chunk0) {
    const float4 *b4 = reinterpret_cast<const float4 *>(bias);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float4 bl = b4[2 * c], bh = b4[2 * c + 1];
        const float b[8] = {bl.x, bl.y, bl.z, bl.w, bh.x, bh.y, bh.z, bh.w};
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = 8 * c + 2 * q;
            w[q] = pack2_relu<kBF16>(__uint_as_float(r[k]) + b[2 * q], __uint_as_float(r[k + 1]) + b[2 * q + 1]);
        }
        store_chunk(A, row, chunk0 + c, 1024, make_uint4(w[0], w[1], w[2], w[3]));
    }
}


// The 128-sample tiles of an n-sample launch that group g (of G) of this CTA
// takes: tiles first, first + step, ... below end.  With at least one tile
// per group of the grid, CTA b's groups take tiles b*G .. b*G + G - 1 of each
// round (neighbouring tiles, that is neighbouring rays, share an SM's L1).
// With fewer, every CTA takes a run of ceil(tiles / gridDim.x) <= G tiles, one
// per group, so that every SM gets work: handing consecutive tiles to the
// groups of one CTA queued them behind one SM's L1 data pipe and made a launch
// of a few hundred tiles 2.5 times slower (a run per CTA for every launch cost
// the large ones 1 %).
struct TileLoop {
    uint32_t first, end, step;
};
__device__ __forceinline__ TileLoop cta_tiles(uint32_t n, int G, int g) {
    const uint32_t tiles = (n + 127u) / 128u;
    if (tiles >= gridDim.x * (uint32_t)G) return TileLoop{blockIdx.x * G + g, tiles, gridDim.x * G};
    const uint32_t per = (tiles + gridDim.x - 1u) / gridDim.x;
    const uint32_t b = min(blockIdx.x * per, tiles);
    return TileLoop{b + g, min(b + per, tiles), (uint32_t)G};
}

}  // namespace tc
}  // namespace mrf
