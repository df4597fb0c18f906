// BVH refit for moved vertices (same topology), bottom-up in one launch, and
// the four-child copy of the binary BVH that the traversals walk.
//
// One thread per internal node rewrites the triangles of its leaf children and
// their boxes, then "arrives" at its node.  A node is complete after
// (its internal children + 1) arrivals; the thread that completes it writes the
// node's union box into the parent's child slot and arrives at the parent.
// Threads never wait on each other: a thread that is not last simply exits, so
// the launch cannot hang.
#include <cuda_runtime.h>

#include "common.h"

namespace mrf {

__device__ __forceinline__ void box_of_child(const float4 *nodes, int k, int s, float lo[3], float hi[3]) {
    float4 n0 = __ldcg(nodes + 4 * k), n1 = __ldcg(nodes + 4 * k + 1), n2 = __ldcg(nodes + 4 * k + 2);
    if (s == 0) {
        lo[0] = n0.x; lo[1] = n0.y; lo[2] = n0.z; hi[0] = n0.w; hi[1] = n1.x; hi[2] = n1.y;
    } else {
        lo[0] = n1.z; lo[1] = n1.w; lo[2] = n2.x; hi[0] = n2.y; hi[1] = n2.z; hi[2] = n2.w;
    }
}

__device__ __forceinline__ void write_child_box(float4 *nodes, int k, int s, const float lo[3], const float hi[3]) {
    float *f = reinterpret_cast<float *>(nodes + 4 * k);
    float *b = f + (s == 0 ? 0 : 6);
    for (int a = 0; a < 3; ++a) {
        __stcg(b + a, lo[a]);
        __stcg(b + 3 + a, hi[a]);
    }
}

__global__ void bvh_refit_kernel(float4 *nodes, int n_nodes, float4 *tris, const uint32_t *order,
                                 const uint32_t *tri_idx, const float *verts, const int *parent, int *counters) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_nodes) return;
    int4 meta = __ldcg(reinterpret_cast<const int4 *>(nodes + 4 * k + 3));
    int ci[2] = {meta.x, meta.y}, cc[2] = {meta.z, meta.w};
    for (int s = 0; s < 2; ++s) {
        if (cc[s] <= 0) continue;
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int slot = ci[s]; slot < ci[s] + cc[s]; ++slot) {
            const uint32_t t = order[slot];
            float4 *tp = tris + 3 * slot;
            for (int v = 0; v < 3; ++v) {
                const float *p = verts + 3 * (size_t)tri_idx[3 * (size_t)t + v];
                float4 old = tp[v];
                tp[v] = make_float4(p[0], p[1], p[2], old.w);
                for (int a = 0; a < 3; ++a) {
                    lo[a] = fminf(lo[a], p[a]);
                    hi[a] = fmaxf(hi[a], p[a]);
                }
            }
        }
        write_child_box(nodes, k, s, lo, hi);
    }
    int cur = k;
    while (cur >= 0) {
        int4 m = __ldcg(reinterpret_cast<const int4 *>(nodes + 4 * cur + 3));
        const int internal = (m.z == 0 && m.x >= 0) + (m.w == 0 && m.y >= 0);
        __threadfence();
        const int prev = atomicAdd(counters + cur, 1);
        if (prev != internal) return;  // not the last arrival
        __threadfence();
        const int p = parent[cur];
        if (p < 0) return;
        float lo[3], hi[3], lo2[3], hi2[3];
        box_of_child(nodes, cur, 0, lo, hi);
        box_of_child(nodes, cur, 1, lo2, hi2);
        for (int a = 0; a < 3; ++a) {
            lo[a] = fminf(lo[a], lo2[a]);
            hi[a] = fmaxf(hi[a], hi2[a]);
        }
        int4 pm = __ldcg(reinterpret_cast<const int4 *>(nodes + 4 * p + 3));
        write_child_box(nodes, p, (pm.x == cur && pm.z == 0) ? 0 : 1, lo, hi);
        cur = p;
    }
}

cudaError_t launch_bvh_refit(float4 *nodes, int n_nodes, float4 *tris, int n_tris, const uint32_t *tri_order,
                             const uint32_t *tri_idx, const float *verts, const int *parent, int *counters,
                             const int *, cudaStream_t s) {
    if (n_nodes == 0) return cudaSuccess;
    (void)n_tris;
    cudaError_t e = cudaMemsetAsync(counters, 0, sizeof(int) * (size_t)n_nodes, s);
    if (e != cudaSuccess) return e;
    bvh_refit_kernel<<<(n_nodes + 127) / 128, 128, 0, s>>>(nodes, n_nodes, tris, tri_order, tri_idx, verts, parent,
                                                           counters);
    return cudaGetLastError();
}

// Wide (four-child) copy of the BVH, the one every traversal walks.  Wide
// node k stands for binary node k and holds k's grandchildren, or k's children
// where those are leaves, so one traversal step tests four boxes after one
// memory round trip and a ray takes about half as many dependent steps.  Every
// binary node gets its wide copy (those at odd depth are never reached from
// the root, which spares computing depths after a rebuild); one thread per
// node, after every build, refit and rebuild.  Layout, 8 float4 per node:
// [0..5] lo.x, lo.y, lo.z, hi.x, hi.y, hi.z of the four children (one float4
// per coordinate), [6] child index (inner: node, leaf: first triangle slot),
// [7] triangle count (> 0 leaf, 0 inner node, -1 no child: empty box).
struct WideKid {
    float lo[3], hi[3];
    int index, count;
};

__device__ __forceinline__ WideKid kid_of(const float4 *nodes, int k, int s) {
    WideKid r;
    box_of_child(nodes, k, s, r.lo, r.hi);
    const int4 m = __ldcg(reinterpret_cast<const int4 *>(nodes + 4 * k + 3));
    const int ci = s ? m.y : m.x, cc = s ? m.w : m.z;
    r.index = ci;
    r.count = cc > 0 ? cc : ((cc == 0 && ci >= 0) ? 0 : -1);
    return r;
}

__global__ void bvh_widen_kernel(const float4 *nodes, int n_nodes, float4 *wide) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_nodes) return;
    WideKid out[4];
    int n = 0;
    for (int s = 0; s < 2; ++s) {
        const WideKid a = kid_of(nodes, k, s);
        if (a.count > 0) {
            out[n++] = a;
        } else if (a.count == 0) {
            for (int t = 0; t < 2; ++t) {
                const WideKid g = kid_of(nodes, a.index, t);
                if (g.count >= 0) out[n++] = g;
            }
        }
    }
    float f[8][4];
    for (int c = 0; c < 4; ++c) {
        const bool v = c < n;
        for (int a = 0; a < 3; ++a) {
            f[a][c] = v ? out[c].lo[a] : INFINITY;
            f[3 + a][c] = v ? out[c].hi[a] : -INFINITY;
        }
        f[6][c] = __int_as_float(v ? out[c].index : -1);
        f[7][c] = __int_as_float(v ? out[c].count : -1);
    }
    for (int u = 0; u < 8; ++u) wide[8 * (size_t)k + u] = make_float4(f[u][0], f[u][1], f[u][2], f[u][3]);
}

cudaError_t launch_bvh_widen(const float4 *nodes, int n_nodes, float4 *wide, cudaStream_t s) {
    if (n_nodes <= 0) return cudaSuccess;
    bvh_widen_kernel<<<(n_nodes + 127) / 128, 128, 0, s>>>(nodes, n_nodes, wide);
    return cudaGetLastError();
}

}  // namespace mrf
