// Host-side binned-SAH BVH builder (the paper casts rays against its meshes,
// Eq. 3, without naming an acceleration structure; this is the renderer's own).
//
// Output layout (consumed by device.cuh):
//   nodes : 4 x float4 per internal node = both children's boxes +
//           (left, right, left_count, right_count) as int bits.  A child with
//           count > 0 is a leaf covering triangle slots [index, index + count);
//           count == 0 and index >= 0 is an internal node; index < 0 is empty.
//   order : triangle slot -> original triangle index.
//   parent: parent internal node of each internal node (-1 for the root).
// Internal nodes are numbered in depth-first pre-order (parent < child).
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace mrf {

namespace {

constexpr int kLeafMax = 4;
constexpr int kBins = 16;

struct Box {
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX};
    float hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    void grow(const Box &b) {
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], b.lo[k]);
            hi[k] = std::max(hi[k], b.hi[k]);
        }
    }
    void grow(const float p[3]) {
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], p[k]);
            hi[k] = std::max(hi[k], p[k]);
        }
    }
    bool empty() const { return lo[0] > hi[0]; }
    float area() const {
        if (empty()) return 0.f;
        float dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
        return 2.f * (dx * dy + dy * dz + dz * dx);
    }
};

struct Builder {
    const float *verts;
    const uint32_t *tris;
    std::vector<Box> tbox;
    std::vector<float> cen;  // 3 per triangle
    std::vector<uint32_t> prim;
    std::vector<float> nodes;  // 16 floats per node
    std::vector<int> parent;

    Box range_box(int b, int e) const {
        Box r;
        for (int i = b; i < e; ++i) r.grow(tbox[prim[i]]);
        return r;
    }

    // split [b, e): binned SAH over the three axes; median split when all
    // centroids coincide or no bin boundary separates them
    int split(int b, int e) {
        Box cb;
        for (int i = b; i < e; ++i) cb.grow(&cen[3 * prim[i]]);
        float best = FLT_MAX;
        int best_axis = -1, best_bin = -1;
        for (int a = 0; a < 3; ++a) {
            float ext = cb.hi[a] - cb.lo[a];
            if (!(ext > 0.f)) continue;
            Box bb[kBins];
            int bc[kBins] = {0};
            for (int i = b; i < e; ++i) {
                int k = (int)((cen[3 * prim[i] + a] - cb.lo[a]) / ext * kBins);
                k = std::min(std::max(k, 0), kBins - 1);
                bb[k].grow(tbox[prim[i]]);
                ++bc[k];
            }
            Box left[kBins];
            int lc[kBins];
            Box acc;
            int n = 0;
            for (int k = 0; k < kBins; ++k) {
                acc.grow(bb[k]);
                n += bc[k];
                left[k] = acc;
                lc[k] = n;
            }
            Box racc;
            int rn = 0;
            for (int k = kBins - 1; k > 0; --k) {
                racc.grow(bb[k]);
                rn += bc[k];
                int ln = lc[k - 1];
                if (ln == 0 || rn == 0) continue;
                float cost = left[k - 1].area() * ln + racc.area() * rn;
                if (cost < best) {
                    best = cost;
                    best_axis = a;
                    best_bin = k;
                }
            }
        }
        int m;
        if (best_axis < 0) {
            m = (b + e) / 2;
        } else {
            const int a = best_axis;
            const float ext = cb.hi[a] - cb.lo[a];
            auto it = std::partition(prim.begin() + b, prim.begin() + e, [&](uint32_t t) {
                int k = (int)((cen[3 * t + a] - cb.lo[a]) / ext * kBins);
                k = std::min(std::max(k, 0), kBins - 1);
                return k < best_bin;
            });
            m = (int)(it - prim.begin());
            if (m == b || m == e) m = (b + e) / 2;
        }
        return m;
    }

    void set_child(int node, int slot, const Box &bx, int index, int count) {
        float *n = &nodes[16 * node];
        float *bl = slot == 0 ? n : n + 6;  // left: floats 0..5, right: floats 6..11
        bl[0] = bx.lo[0]; bl[1] = bx.lo[1]; bl[2] = bx.lo[2];
        bl[3] = bx.hi[0]; bl[4] = bx.hi[1]; bl[5] = bx.hi[2];
        int32_t iv = index, cv = count;
        std::memcpy(&n[12 + slot], &iv, 4);
        std::memcpy(&n[14 + slot], &cv, 4);
    }

    int new_node(int par) {
        int k = (int)parent.size();
        nodes.resize(16 * (k + 1), 0.f);
        parent.push_back(par);
        Box empty;
        set_child(k, 0, empty, -1, 0);
        set_child(k, 1, empty, -1, 0);
        return k;
    }

    int build(int b, int e, int par) {
        int k = new_node(par);
        int m = split(b, e);
        int rng[2][2] = {{b, m}, {m, e}};
        for (int s = 0; s < 2; ++s) {
            int cb = rng[s][0], ce = rng[s][1];
            Box bx = range_box(cb, ce);
            if (ce - cb <= kLeafMax) {
                set_child(k, s, bx, cb, ce - cb);
            } else {
                int c = build(cb, ce, k);
                set_child(k, s, bx, c, 0);
            }
        }
        return k;
    }
};

}  // namespace

// Builds the BVH of n_tris triangles (vertex indices already validated).
// Returns node floats (16 per node), slot order and parents.
void bvh_build_host(const float *verts, const uint32_t *tris, uint32_t n_tris, std::vector<float> &nodes,
                    std::vector<uint32_t> &order, std::vector<int> &parent) {
    Builder B;
    B.verts = verts;
    B.tris = tris;
    B.tbox.resize(n_tris);
    B.cen.resize(3 * (size_t)n_tris);
    B.prim.resize(n_tris);
    for (uint32_t i = 0; i < n_tris; ++i) {
        for (int v = 0; v < 3; ++v) B.tbox[i].grow(&verts[3 * (size_t)tris[3 * (size_t)i + v]]);
        for (int a = 0; a < 3; ++a) B.cen[3 * i + a] = 0.5f * (B.tbox[i].lo[a] + B.tbox[i].hi[a]);
        B.prim[i] = i;
    }
    if (n_tris > 0) {
        if (n_tris <= (uint32_t)kLeafMax) {
            int k = B.new_node(-1);
            B.set_child(k, 0, B.range_box(0, (int)n_tris), 0, (int)n_tris);
        } else {
            B.build(0, (int)n_tris, -1);
        }
    }
    nodes.swap(B.nodes);
    order.swap(B.prim);
    parent.swap(B.parent);
}

}  // namespace mrf
