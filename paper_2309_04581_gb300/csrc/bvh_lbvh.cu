// BVH rebuild on the GPU for deforming meshes (same triangles, new vertex
// positions): a linear BVH over the Morton order of the triangle centroids,
// after Karras, "Maximizing Parallelism in the Construction of BVHs, Octrees,
// and k-d Trees" (HPG 2012).  The paper casts rays against its meshes (Eq. 3)
// and syncs them every frame, without naming an acceleration structure.
//
//   1. centroid bounds (block reduction + ordered-integer atomics);
//   2. 30-bit Morton code of every centroid in those bounds;
//   3. stable LSD radix sort of (code, triangle) pairs, 4 bits per pass;
//   4. one thread per internal node finds its key range and split from the
//      common-prefix lengths of the sorted codes (ties broken by position),
//      giving n - 1 internal nodes, root 0, one triangle per leaf;
//   5. leaf slots take the sorted triangles; the bottom-up refit kernel then
//      writes vertices and every box.
// Everything is enqueued on one stream with no host synchronisation.
#include <algorithm>
#include <utility>

#include <cuda_runtime.h>

#include "device.cuh"

namespace mrf {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortTile = 1024;   // keys per block (4 per thread, consecutive)

__device__ __forceinline__ int ordered(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float unordered(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7FFFFFFF); }

__device__ __forceinline__ V3 centroid(const float *verts, const uint32_t *idx, uint32_t t) {
    V3 c = v3(0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float *p = verts + 3 * (size_t)idx[3 * (size_t)t + k];
        c = c + v3(p[0], p[1], p[2]);
    }
    return c * (1.f / 3.f);
}

__global__ void bounds_init(int *bnd) {
    if (threadIdx.x < 3) bnd[threadIdx.x] = ordered(INFINITY);
    else if (threadIdx.x < 6) bnd[threadIdx.x] = ordered(-INFINITY);
}

__global__ void centroid_bounds(const float *verts, const uint32_t *idx, uint32_t n, int *bnd) {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const V3 c = centroid(verts, idx, t);
        for (int a = 0; a < 3; ++a) {
            lo[a] = fminf(lo[a], comp(c, a));
            hi[a] = fmaxf(hi[a], comp(c, a));
        }
    }
    for (int a = 0; a < 3; ++a) {
        for (int off = 16; off > 0; off >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], off));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], off));
        }
    }
    if ((threadIdx.x & 31) == 0)
        for (int a = 0; a < 3; ++a) {
            atomicMin(bnd + a, ordered(lo[a]));
            atomicMax(bnd + 3 + a, ordered(hi[a]));
        }
}

// 10 bits of x spread to every third bit
__device__ __forceinline__ uint32_t spread3(uint32_t x) {
    x &= 0x3FFu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__global__ void morton_codes(const float *verts, const uint32_t *idx, uint32_t n, const int *bnd, uint32_t *key,
                             uint32_t *val) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const V3 c = centroid(verts, idx, t);
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) {
        const float lo = unordered(bnd[a]), hi = unordered(bnd[3 + a]);
        const float ext = hi - lo;
        const float u = ext > 0.f ? (comp(c, a) - lo) / ext : 0.f;
        q[a] = (uint32_t)fminf(fmaxf(u * 1024.f, 0.f), 1023.f);
    }
    key[t] = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
    val[t] = t;
}

// ---- stable LSD radix sort, 4-bit digits
__global__ void __launch_bounds__(kSortThreads) radix_count(const uint32_t *key, uint32_t n, int shift,
                                                             uint32_t *counts, uint32_t nblocks) {
    __shared__ uint32_t c[16];
    if (threadIdx.x < 16) c[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t base = blockIdx.x * kSortTile;
    for (int k = threadIdx.x; k < kSortTile; k += kSortThreads) {
        const uint32_t i = base + k;
        if (i < n) atomicAdd(&c[(key[i] >> shift) & 15u], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 16) counts[threadIdx.x * nblocks + blockIdx.x] = c[threadIdx.x];
}

// exclusive prefix sum of m values in place, one block of 1024 threads
__global__ void __launch_bounds__(1024) radix_scan(uint32_t *a, uint32_t m) {
    __shared__ uint32_t ws[32];
    const uint32_t per = (m + 1023) / 1024, b0 = threadIdx.x * per;
    uint32_t s = 0;
    for (uint32_t i = b0; i < b0 + per && i < m; ++i) s += a[i];
    uint32_t x = s;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t v = ws[lane];
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, v, off);
            if (lane >= off) v += y;
        }
        ws[lane] = v;
    }
    __syncthreads();
    uint32_t run = x - s + (w > 0 ? ws[w - 1] : 0);
    for (uint32_t i = b0; i < b0 + per && i < m; ++i) {
        const uint32_t v = a[i];
        a[i] = run;
        run += v;
    }
}

// block-wide exclusive scan of one value per thread; returns the total
__device__ __forceinline__ uint32_t block_scan(uint32_t x, uint32_t &excl, uint32_t *ws) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = x;
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
    }
    __syncthreads();
    if (lane == 31) ws[w] = inc;
    __syncthreads();
    uint32_t before = 0, total = 0;
    for (int k = 0; k < kSortThreads / 32; ++k) {
        const uint32_t v = ws[k];
        if (k < w) before += v;
        total += v;
    }
    excl = before + inc - x;
    return total;
}

__global__ void __launch_bounds__(kSortThreads) radix_scatter(const uint32_t *key, const uint32_t *val, uint32_t n,
                                                               int shift, const uint32_t *offsets, uint32_t nblocks,
                                                               uint32_t *key_out, uint32_t *val_out) {
    __shared__ uint32_t ws[kSortThreads / 32];
    const uint32_t base = blockIdx.x * kSortTile + 4 * threadIdx.x;
    uint32_t k4[4], v4[4], d4[4];
    bool ok[4];
    for (int e = 0; e < 4; ++e) {
        ok[e] = base + e < n;
        k4[e] = ok[e] ? key[base + e] : 0u;
        v4[e] = ok[e] ? val[base + e] : 0u;
        d4[e] = (k4[e] >> shift) & 15u;
    }
    for (uint32_t dig = 0; dig < 16; ++dig) {
        uint32_t mine = 0;
        for (int e = 0; e < 4; ++e) mine += (ok[e] && d4[e] == dig) ? 1u : 0u;
        uint32_t excl;
        block_scan(mine, excl, ws);
        uint32_t pos = offsets[dig * nblocks + blockIdx.x] + excl;
        for (int e = 0; e < 4; ++e)
            if (ok[e] && d4[e] == dig) {
                key_out[pos] = k4[e];
                val_out[pos] = v4[e];
                ++pos;
            }
    }
}

// ---- hierarchy
__device__ __forceinline__ int delta(const uint32_t *key, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    const uint32_t a = key[i], b = key[j];
    return a != b ? __clz(a ^ b) : 32 + __clz((uint32_t)(i ^ j));
}

__global__ void lbvh_nodes(const uint32_t *key, int n, float4 *nodes, int *parent) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const int d = delta(key, n, i, i + 1) - delta(key, n, i, i - 1) >= 0 ? 1 : -1;
    const int dmin = delta(key, n, i, i - d);
    int lmax = 2;
    while (delta(key, n, i, i + lmax * d) > dmin) lmax *= 2;
    int l = 0;
    for (int t = lmax / 2; t >= 1; t /= 2)
        if (delta(key, n, i, i + (l + t) * d) > dmin) l += t;
    const int j = i + l * d;
    const int dnode = delta(key, n, i, j);
    int s = 0;
    for (int div = 2;; div *= 2) {
        const int t = (l + div - 1) / div;
        if (delta(key, n, i, i + (s + t) * d) > dnode) s += t;
        if (t == 1) break;
    }
    const int g = i + s * d + min(d, 0);
    const int lo = min(i, j), hi = max(i, j);
    const bool left_leaf = lo == g, right_leaf = hi == g + 1;
    float4 *nd = nodes + 4 * i;
    nd[3] = make_float4(__int_as_float(g), __int_as_float(g + 1), __int_as_float(left_leaf ? 1 : 0),
                        __int_as_float(right_leaf ? 1 : 0));
    if (!left_leaf) parent[g] = i;
    if (!right_leaf) parent[g + 1] = i;
    if (i == 0) parent[0] = -1;
}

// single triangle: a root with one leaf child and an empty one
__global__ void lbvh_single(float4 *nodes, int *parent) {
    nodes[3] = make_float4(__int_as_float(0), __int_as_float(-1), __int_as_float(1), __int_as_float(0));
    parent[0] = -1;
}

__global__ void lbvh_leaves(const uint32_t *sorted, const uint32_t *mat, uint32_t n, uint32_t *order, float4 *tris) {
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const uint32_t t = sorted[s];
    order[s] = t;
    tris[3 * (size_t)s].w = __uint_as_float(t);
    tris[3 * (size_t)s + 1].w = __uint_as_float(mat[t]);
    tris[3 * (size_t)s + 2].w = 0.f;
}

}  // namespace

size_t bvh_rebuild_scratch_words(uint32_t n) {
    const uint32_t nblocks = (n + kSortTile - 1) / kSortTile;
    return 4 * (size_t)n + 16 * (size_t)nblocks + 8;
}

// Rebuilds the hierarchy of n triangles (tri_idx, per-triangle materials mat,
// vertices verts already on the device) into nodes (n - 1 internal nodes, or 1
// for n == 1), parent, order and tris, then refits every box.  scratch holds
// bvh_rebuild_scratch_words(n) words.
cudaError_t launch_bvh_rebuild(float4 *nodes, int *parent, int *counters, float4 *tris, uint32_t *order,
                               const uint32_t *tri_idx, const uint32_t *mat, const float *verts, uint32_t n,
                               uint32_t *scratch, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const uint32_t nblocks = (n + kSortTile - 1) / kSortTile;
    uint32_t *k0 = scratch, *v0 = k0 + n, *k1 = v0 + n, *v1 = k1 + n, *cnt = v1 + n;
    int *bnd = reinterpret_cast<int *>(cnt + 16 * (size_t)nblocks);
    cudaError_t e;
    bounds_init<<<1, 32, 0, s>>>(bnd);
    centroid_bounds<<<std::min<uint32_t>((n + 255) / 256, 152u * 8u), 256, 0, s>>>(verts, tri_idx, n, bnd);
    morton_codes<<<(n + 255) / 256, 256, 0, s>>>(verts, tri_idx, n, bnd, k0, v0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int shift = 0; shift < 32; shift += 4) {
        radix_count<<<nblocks, kSortThreads, 0, s>>>(k0, n, shift, cnt, nblocks);
        radix_scan<<<1, 1024, 0, s>>>(cnt, 16 * nblocks);
        radix_scatter<<<nblocks, kSortThreads, 0, s>>>(k0, v0, n, shift, cnt, nblocks, k1, v1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        std::swap(k0, k1);
        std::swap(v0, v1);
    }
    // after 8 passes the sorted pairs are back in the first buffers
    int n_nodes;
    if (n == 1) {
        lbvh_single<<<1, 1, 0, s>>>(nodes, parent);
        n_nodes = 1;
    } else {
        lbvh_nodes<<<(n - 1 + 127) / 128, 128, 0, s>>>(k0, (int)n, nodes, parent);
        n_nodes = (int)n - 1;
    }
    lbvh_leaves<<<(n + 255) / 256, 256, 0, s>>>(v0, mat, n, order, tris);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_bvh_refit(nodes, n_nodes, tris, (int)n, order, tri_idx, verts, parent, counters, nullptr, s);
}

}  // namespace mrf
