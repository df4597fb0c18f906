// Wavefront engine: Algorithm 1 run segment by segment over all live paths.
//
// Per segment j the host enqueues (no host synchronisation):
//   1. wf_cast     : closest hit and shadow-ray visibility at diffuse hits;
//      wf_gen      : generation of every field sample the segment march and
//                    the shadow-ray marches need (occupancy skip and support
//                    test), packed contiguously per job in one flat buffer;
//   2. field       : evaluation of all generated samples, on the tensor cores
//                    for the hash grid at FP16/BF16 (field_tc.cu), else FP32;
//   3. wf_composite: in-order compositing of each job's samples (Eqs. 10-11),
//                    one warp per job at a time;
//      wf_shade    : next-event term, BSDF sample (Eqs. 12-13), termination,
//                    and compaction of the surviving paths into the next queue.
// Sample positions, quadrature intervals and every decision are computed with
// the same FP32 formulas as the megakernel.  Jobs whose samples do not fit the
// sample buffer are marched in place by wf_shade on the CUDA cores.
#include <algorithm>

#include <atomic>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "path.cuh"
#include "shadow_net.cuh"

namespace mrf {

namespace {

constexpr uint32_t kOverflow = 0xFFFFFFFFu;   // slot whose samples did not fit (pending)
constexpr uint32_t kDeferred = 0x80000000u;   // hp.w bit: the slot's shadow rays are traced by wf_vis
constexpr uint32_t kDone = 0xFFFFFFFEu;       // slot composited in an earlier round of the segment
constexpr int kMaxRounds = 16;
constexpr int kThreads = 128;

struct WfParams {
    RenderParams R;
    uint32_t paths;
    float4 *acc;                    // per path: L (rgb), camera-segment opacity
    uint32_t *qpath[2];             // live queues: path ids
    float4 *qo[2], *qd[2], *qT[2];  // origin (+ previous triangle id bits), direction, throughput
    float *hit_t;                   // per live slot, current segment
    int *hit_slot;
    uint32_t *hit_id;
    uint32_t *rstart, *rcount;      // radiance samples of the slot's segment
    uint32_t *sstart, *scount;      // shadow samples, [slot * n_shadow + q]
    float4 *sw;                     // next-event weight (rgb); w = 1: unblocked, marched; 2: unblocked, network
    float4 *hp;                     // hit point (xyz) and number of unblocked shadow rays (w) per live slot
    float4 *sdir;                   // shadow-ray direction (xyz) and light distance (w), [slot * n_shadow + q]
    float4 *comp;                   // per slot: segment radiance sum (rgb, times T(p_j)) and optical depth (w)
    float *sdepth;                  // shadow optical depth (marched) or transmittance (network), [slot * n_shadow + q]
    uint32_t *ctr;                  // [0], [1] live counts; [2] generated samples; [3] network shadow rays;
                                    // [4 + r] slots left pending by generation round r
    uint32_t *squeue;               // shadow rays answered by the network: slot * n_shadow + q
    float4 *samp;                   // sample position (xyz) and interval length (w)
    float4 *sview;                  // view direction (field frame) of each radiance sample (view-dependent fields)
    float4 *fout;                   // sigma * delta, r, g, b per sample
    uint32_t cap;                   // sample capacity
};

// exclusive prefix of n over a fully converged warp plus one atomic per warp
__device__ __forceinline__ uint32_t warp_alloc(uint32_t *ctr, uint32_t n) {
    const int lane = threadIdx.x & 31;
    uint32_t x = n;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, x, 31);
    uint32_t base = 0;
    if (lane == 31 && total) base = atomicAdd(ctr, total);
    base = __shfl_sync(0xffffffffu, base, 31);
    return base + x - n;
}

// Work distribution of the warp-cooperative kernels (wf_gen, wf_mask,
// wf_composite): a warp takes a chunk of S consecutive slots from a per-round
// work counter, walks their jobs one after another (lane l < S holds slot
// base + l) and takes the next chunk until none is left.  S is a power of two,
// at most 32, sized for at least four chunks per resident warp: job lengths vary
// by orders of magnitude (a ray through the field against one that hits the
// floor at once), and a static split left SMs idle for half of the first
// segment and waiting on a few warps with 32 long jobs in the late ones.
__device__ __forceinline__ int chunk_slots(uint32_t live) {
    const uint32_t warps = min(gridDim.x * (blockDim.x >> 5), 152u * 32u);
    const uint32_t need = live / (4u * warps);   // rounded down: at least four chunks per warp
    return need <= 1 ? 1 : (int)min(32u, 1u << (31 - __clz(need)));
}

// First slot of the warp's next chunk (>= live: no work left).
__device__ __forceinline__ uint32_t next_chunk(uint32_t *work, int S, int lane) {
    uint32_t b = 0;
    if (lane == 0) b = atomicAdd(work, (uint32_t)S);
    return __shfl_sync(0xffffffffu, b, 0);
}

// Counters of the engine (W.ctr): [0], [1] live slots of the two queues,
// [2] generated samples, [3] network shadow rays, then per generation round r
// a block of four: slots left pending, and the work counters of wf_gen,
// wf_mask and wf_composite.  One memset per segment clears [2, 4 + 4 * rounds).
// Then the persistent tail's words: the segment it took over at (0: none),
// the paths live then, and its work counter; cleared once per frame.
__device__ __forceinline__ uint32_t *pending_ctr(const WfParams &W, int r) { return W.ctr + 4 + 4 * r; }
__device__ __forceinline__ uint32_t *work_ctr(const WfParams &W, int r, int k) { return W.ctr + 5 + 4 * r + k; }
constexpr int kTailWord = 4 + 4 * kMaxRounds;
constexpr int kCtrWords = kTailWord + 3;
// true once the persistent tail (wf_tail) has taken over the remaining segments
__device__ __forceinline__ bool tail_taken(const WfParams &W) { return W.ctr[kTailWord] != 0u; }

// Shared-memory copies used by the sample walk: coarse occupancy bits and the
// density-support spheres.
constexpr int kCoarseWordsMax = 1024;   // coarse grids up to 32^3 are staged
constexpr int kSupportMax = 64;

struct WalkSmem {
    uint32_t coarse[kCoarseWordsMax];
    float4 support[kSupportMax];
};

struct WalkCtx {
    const uint32_t *coarse;   // shared copy or nullptr
    const float4 *support;    // shared copy (or the global array when it does not fit)
};

__device__ __forceinline__ WalkCtx stage_walk(const FieldDev &F, WalkSmem &sm) {
    const int Rc = F.occ_coarse_res;
    const int cw = (Rc * Rc * Rc + 31) / 32;
    const bool coarse_fits = F.occ_coarse && cw <= kCoarseWordsMax;
    if (coarse_fits)
        for (int i = threadIdx.x; i < cw; i += blockDim.x) sm.coarse[i] = __ldg(F.occ_coarse + i);
    const bool sup_fits = F.n_support <= kSupportMax;
    if (sup_fits)
        for (int i = threadIdx.x; i < F.n_support; i += blockDim.x) sm.support[i] = __ldg(F.support + i);
    __syncthreads();
    return WalkCtx{coarse_fits ? sm.coarse : nullptr, sup_fits ? sm.support : F.support};
}

// exit parameter of the cell c of a grid with cell width `cell` along the ray
__device__ __forceinline__ float grid_cell_exit(const float lo[3], const float cell[3], const int c[3], V3 o, V3 inv) {
    float t = INFINITY;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float ik = comp(inv, k);
        if (isinf(ik)) continue;
        const float edge = fmaf((float)(c[k] + (ik > 0.f ? 1 : 0)), cell[k], lo[k]);
        t = fminf(t, (edge - comp(o, k)) * ik);
    }
    return t;
}

struct Segment {
    float t0, t1, h;
    int n;
};

// quadrature intervals of [a, b] clipped to the field box (same FP32 formulas as march())
__device__ __forceinline__ bool segment_of(const RenderParams &P, V3 o, V3 d, float a, float b, Segment &S) {
    const FieldDev &F = P.F;
    float tb0, tb1;
    if (!box_interval(F.lo, F.hi, o, d, tb0, tb1)) return false;
    S.t0 = fmaxf(a, tb0);
    S.t1 = fminf(b, tb1);
    if (!(S.t1 > S.t0)) return false;
    if (P.steps) {
        S.n = (int)P.steps;
        S.h = (S.t1 - S.t0) / (float)S.n;
    } else {
        S.h = P.dt;
        const float nf = ceilf((S.t1 - S.t0) / S.h);
        if (nf > 16777216.f) return false;
        S.n = (int)nf;
    }
    return true;
}

// Support sphere c's part in one job (o, d in the field's frame, S its
// intervals): whether the ray passes within the sphere (a small relative
// margin on r^2) over [S.t0, S.t1], and, with `ranges`, the interval-index
// range [jb, je) the ray can spend inside it, conservative by two intervals
// (none: jb = INT_MAX, je = -1).  A sphere the ray misses has
// 1 - |p - c|^2 / r^2 < 0 at every point of the segment, and every sample
// outside all ranges lies outside every sphere, so neither changes the support
// (a max clamped at 0) of any sample the walk tests.
__device__ __forceinline__ bool sphere_range(const float4 c, V3 o, V3 d, const Segment &S, float inv_h, bool ranges,
                                             int &jb, int &je) {
    const V3 oc = v3(c.x - o.x, c.y - o.y, c.z - o.z);
    const float dd = dot(d, d), b = dot(oc, d) / dd;   // parameter of the closest approach
    const float tc = fminf(fmaxf(b, S.t0), S.t1);      // clamped to the segment
    const V3 q = v3(o.x + d.x * tc - c.x, o.y + d.y * tc - c.y, o.z + d.z * tc - c.z);
    const bool hit = dot(q, q) * c.w < 1.0f + 1e-3f;
    jb = 0x7fffffff;
    je = -1;
    if (ranges && hit) {
        const V3 e = v3(o.x + d.x * b - c.x, o.y + d.y * b - c.y, o.z + d.z * b - c.z);
        const float disc = ((1.0f + 1e-3f) / c.w - dot(e, e)) / dd;
        if (disc > 0.f) {
            const float w = sqrtf(disc);
            jb = max((int)floorf((b - w - S.t0) * inv_h - 0.5f) - 2, 0);
            je = min((int)ceilf((b + w - S.t0) * inv_h - 0.5f) + 2, S.n);
        }
    }
    return hit;
}

// What the walk of one job tests: the support spheres its ray can enter
// (smask, hash fields with 1..32 spheres) and the interval indices [cb, ce)
// that cover every range of theirs; the walk starts at cb and stops at ce.
// Other fields: every interval, no sphere mask.  A hash field without support
// spheres has no density: an empty cover.
struct Cover {
    uint32_t smask;
    int cb, ce;
};
__device__ __forceinline__ bool has_sphere_cover(const FieldDev &F) {
    return F.kind == MRF_FIELD_HASHGRID && F.n_support > 0 && F.n_support <= 32;
}

// The cover computed by one thread (loop over the spheres).
__device__ __forceinline__ Cover job_cover(const FieldDev &F, const WalkCtx &X, V3 o, V3 d, const Segment &S) {
    Cover cv{0u, 0, S.n};
    if (F.kind == MRF_FIELD_HASHGRID && F.n_support == 0) cv.ce = 0;
    if (!has_sphere_cover(F)) return cv;
    const float inv_h = 1.0f / S.h;
    cv.cb = 0x7fffffff;
    cv.ce = -1;
    for (int k = 0; k < F.n_support; ++k) {
        int jb, je;
        if (sphere_range(X.support[k], o, d, S, inv_h, true, jb, je)) cv.smask |= 1u << k;
        cv.cb = min(cv.cb, jb);
        cv.ce = max(cv.ce, je);
    }
    return cv;
}

// The same cover computed by a warp (lane k takes sphere k); equal to job_cover's.
__device__ __forceinline__ Cover job_cover_warp(const FieldDev &F, const WalkCtx &X, V3 o, V3 d, const Segment &S,
                                                int lane) {
    Cover cv{0u, 0, S.n};
    if (F.kind == MRF_FIELD_HASHGRID && F.n_support == 0) cv.ce = 0;
    if (!has_sphere_cover(F)) return cv;
    int jb = 0x7fffffff, je = -1;
    bool hit = false;
    if (lane < F.n_support) hit = sphere_range(X.support[lane], o, d, S, 1.0f / S.h, true, jb, je);
    cv.smask = __ballot_sync(0xffffffffu, hit);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        jb = min(jb, __shfl_xor_sync(0xffffffffu, jb, off));
        je = max(je, __shfl_xor_sync(0xffffffffu, je, off));
    }
    cv.cb = jb;
    cv.ce = je;
    return cv;
}

__device__ __forceinline__ float support_masked(const float4 *sup, uint32_t mask, V3 p) {
    float s = 0.f;
    while (mask) {
        const int k = __ffs(mask) - 1;
        mask &= mask - 1u;
        const float4 c = sup[k];
        const float dx = p.x - c.x, dy = p.y - c.y, dz = p.z - c.z;
        s = fmaxf(s, 1.0f - (dx * dx + dy * dy + dz * dz) * c.w);
    }
    return s;
}

__device__ __forceinline__ float support_all(const float4 *sup, int n, V3 p) {
    float s = 0.f;
    for (int k = 0; k < n; ++k) {
        const float4 c = sup[k];
        const float dx = p.x - c.x, dy = p.y - c.y, dz = p.z - c.z;
        s = fmaxf(s, 1.0f - (dx * dx + dy * dy + dz * dz) * c.w);
    }
    return s;
}

constexpr int kRunsPerJob = 8;
struct RunList {
    int n;                 // runs recorded; kRunsPerJob + 1 = more than fit (write pass walks again)
    int2 r[kRunsPerJob];   // [begin, end) interval indices
};

// Warp-cooperative walk over the quadrature intervals of one job (every lane
// holds the same job; o and d in the field's frame, S its intervals, cv its
// cover): from the cover's first interval, lane l takes interval i0 + l of
// each 32-interval chunk, tests the density support and the occupancy grid,
// taking the decisions march() takes, and the warp advances by 32 or to the
// exit of an empty cell that holds the chunk's last interval, until the end of
// the cover.  Returns the number of samples whose density can be non-zero (x)
// and the job's nominal interval count (y); records the samples as runs of
// consecutive intervals in `runs` (lane 0 writes; may be nullptr) and, if
// `out` is non-NULL, writes them in order, never more than `limit`.  One
// compiled copy (noinline) serves the counting and the writing walk, so both
// take bit-identical decisions; the counts come back in registers (a reference
// argument would put the caller's counters in local memory).
__device__ __noinline__ uint2 warp_walk_in(const RenderParams &P, const WalkCtx &X, V3 o, V3 d, const Segment S,
                                           const Cover cv, float4 *out, uint32_t limit, int lane, RunList *runs) {
    if (runs && lane == 0) runs->n = 0;
    const FieldDev &F = P.F;
    const bool hash = F.kind == MRF_FIELD_HASHGRID;
    const bool covered = has_sphere_cover(F);
    const bool use_occ0 = hash && F.occ != nullptr;
    // With the sphere cover the support test (arithmetic only) goes first and
    // the coarse grid is left out: the fine grid alone takes the same decisions,
    // and the coarse one only sped up skipping, which the cover now does.  When
    // the grid covers the support it can no longer reject anything either.
    const bool use_coarse = use_occ0 && X.coarse != nullptr && !covered;
    const bool use_occ = use_occ0 && !(covered && F.occ_covers_support);
    const int Rc = F.occ_coarse_res;
    const float inv_h = 1.0f / S.h;
    V3 inv = v3(0.f, 0.f, 0.f);
    if (use_coarse || use_occ) inv = v3(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);
    int nrun = 0, run_end = -1;
    uint32_t k = 0;
    for (int i0 = cv.cb; i0 < cv.ce;) {
        const int i = i0 + lane;
        bool emit = false;
        int skip_to = i + 1;
        float4 rec;
        if (i < S.n) {
            const float lo = fmaf((float)i, S.h, S.t0);
            const float hi = P.steps ? fmaf((float)(i + 1), S.h, S.t0) : fminf(lo + S.h, S.t1);
            const float tm = 0.5f * (lo + hi), delta = hi - lo;
            const V3 p = fma3(d, tm, o);
            bool empty = covered && !(support_masked(X.support, cv.smask, p) > 0.f);
            if (!empty && use_coarse) {
                int c[3];
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    c[q] = min(max((int)floorf((comp(p, q) - F.lo[q]) * F.occ_coarse_scale[q]), 0), Rc - 1);
                const uint32_t ci = (uint32_t)c[0] + (uint32_t)Rc * ((uint32_t)c[1] + (uint32_t)Rc * (uint32_t)c[2]);
                if (!((X.coarse[ci >> 5] >> (ci & 31)) & 1u)) {
                    const float te = grid_cell_exit(F.lo, F.occ_coarse_cell, c, o, inv);
                    skip_to = max(i + 1, (int)ceilf((te - S.t0) * inv_h - 0.5f));
                    empty = true;
                }
            }
            if (!empty && use_occ) {
                int c[3];
                if (!occupied(F, p, c)) {
                    const float te = grid_cell_exit(F.lo, F.occ_cell, c, o, inv);
                    skip_to = max(i + 1, (int)ceilf((te - S.t0) * inv_h - 0.5f));
                    empty = true;
                }
            }
            if (!empty) emit = !hash || covered || support_all(X.support, F.n_support, p) > 0.f;
            rec = make_float4(p.x, p.y, p.z, delta);
        } else {
            skip_to = S.n;
        }
        unsigned m = __ballot_sync(0xffffffffu, emit);
        if (out && emit) {
            const uint32_t slot = k + __popc(m & ((1u << lane) - 1u));
            if (slot < limit) out[slot] = rec;
        }
        k += __popc(m);
        if (runs) {
            // runs of consecutive emitted intervals in this chunk (uniform across lanes)
            while (m) {
                const int st = __ffs(m) - 1;
                const unsigned sh = m >> st;
                const int len = (~sh == 0u) ? 32 - st : __ffs(~sh) - 1;
                const int rb = i0 + st, re = rb + len;
                if (rb == run_end && nrun > 0 && nrun <= kRunsPerJob) {
                    if (lane == 0) runs->r[nrun - 1].y = re;
                } else if (nrun < kRunsPerJob) {
                    if (lane == 0) runs->r[nrun] = make_int2(rb, re);
                    ++nrun;
                } else {
                    nrun = kRunsPerJob + 1;
                }
                run_end = re;
                m = (len == 32) ? 0u : (m & ~(((1u << len) - 1u) << st));
            }
        }
        const int last_skip = __shfl_sync(0xffffffffu, skip_to, 31);
        i0 = max(i0 + 32, last_skip);
    }
    if (runs && lane == 0) runs->n = nrun;
    return make_uint2(k, (uint32_t)S.n);
}

// The same walk for a world-space job on [a, b].
__device__ __forceinline__ uint2 warp_walk(const RenderParams &P, const WalkCtx &X, V3 o, V3 d, float a, float b,
                                           float4 *out, uint32_t limit, int lane, RunList *runs) {
    Segment S;
    to_field_frame(P.F, o, d);
    if (!segment_of(P, o, d, a, b, S)) {
        if (runs && lane == 0) runs->n = 0;
        return make_uint2(0u, 0u);
    }
    return warp_walk_in(P, X, o, d, S, job_cover_warp(P.F, X, o, d, S, lane), out, limit, lane, runs);
}

// Writes samples [first, first + limit) of a job from its recorded runs into
// out[0, limit) (lane-parallel over the run's intervals, positions by the same
// FP32 formulas as the walk); o and d in the field's frame, S the job's
// intervals.
__device__ void write_runs_in(const RenderParams &P, V3 o, V3 d, const Segment &S, const RunList &R, float4 *out,
                              uint32_t limit, int lane, uint32_t first = 0) {
    uint32_t k = 0;
    for (int r = 0; r < R.n; ++r) {
        const int2 run = R.r[r];
        const uint32_t len = (uint32_t)(run.y - run.x);
        if (k + len > first) {
            const int i_first = run.x + (int)(first > k ? first - k : 0u);
            for (int i = i_first + lane; i < run.y; i += 32) {
                const float lo = fmaf((float)i, S.h, S.t0);
                const float hi = P.steps ? fmaf((float)(i + 1), S.h, S.t0) : fminf(lo + S.h, S.t1);
                const float tm = 0.5f * (lo + hi), delta = hi - lo;
                const V3 p = fma3(d, tm, o);
                const uint32_t slot = k + (uint32_t)(i - run.x) - first;
                if (slot < limit) out[slot] = make_float4(p.x, p.y, p.z, delta);
            }
        }
        k += len;
        if (k >= first + limit) break;
    }
}

// The same for a world-space job on [a, b].
__device__ __forceinline__ void write_runs(const RenderParams &P, V3 o, V3 d, float a, float b, const RunList &R,
                                           float4 *out, uint32_t limit, int lane, uint32_t first = 0) {
    Segment S;
    to_field_frame(P.F, o, d);
    if (!segment_of(P, o, d, a, b, S)) return;
    write_runs_in(P, o, d, S, R, out, limit, lane, first);
}

__device__ __forceinline__ V3 shfl3(V3 v, int src) {
    return v3(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src),
              __shfl_sync(0xffffffffu, v.z, src));
}

// Per lane: primary or queued ray, closest hit (Eq. 3), and at diffuse hits the
// shadow rays (one per point light, `samples` per area light).  With one shadow
// ray per hit its visibility is traced here; with more, the rays are stored
// with sw.w = -1 (marched) or -2 (network) and wf_vis traces them, one thread
// per ray, instead of one thread tracing up to 64 of them in turn.
__global__ void __launch_bounds__(kThreads, 5) wf_cast(const WfParams W, uint32_t j, int cur) {
    const RenderParams &P = W.R;
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t live = j == 1 ? W.paths : W.ctr[cur];
    const int K = P.n_shadow;
    if (j > 1) {
        if (tail_taken(W)) return;
        if (live <= P.tail_paths) {   // few paths left: the persistent tail finishes them
            if (tid == 0) {
                W.ctr[kTailWord + 1] = live;
                W.ctr[kTailWord] = j;
            }
            return;
        }
    }
    Counters C = {};
    if (j == 1 && tid == 0) W.ctr[cur] = W.paths;  // every path is live in segment 1
    uint64_t nmask = 0;   // shadow rays of this slot answered by the network
    uint32_t nnet = 0;
    if (tid < live) {
        V3 o, d;
        uint32_t prev = kNoHit, path;
        if (j == 1) {
            path = tid;
            const uint32_t ray = path / P.spp;
            primary_ray(P, ray, o, d);
            W.qpath[cur][tid] = path;
            W.qo[cur][tid] = make_float4(o.x, o.y, o.z, __uint_as_float(kNoHit));
            W.qd[cur][tid] = make_float4(d.x, d.y, d.z, 0.f);
            W.qT[cur][tid] = make_float4(1.f, 1.f, 1.f, 0.f);
            ++C.paths;
        } else {
            path = W.qpath[cur][tid];
            const float4 qo = W.qo[cur][tid], qd = W.qd[cur][tid];
            o = v3(qo.x, qo.y, qo.z);
            prev = __float_as_uint(qo.w);
            d = v3(qd.x, qd.y, qd.z);
        }
        Hit h;
        unsigned rt = 0;
        bool fault = false;
        const unsigned nodes0 = C.nodes;
        bvh_trace<false>(P.B, o, d, prev, P.tmin, INFINITY, h, rt, C.nodes, C.tris, fault);
        note_traversal(C, C.nodes - nodes0, path);
        C.retests += rt;
        if (fault) C.fault |= 1;
        W.hit_t[tid] = h.t;
        W.hit_slot[tid] = h.slot;
        W.hit_id[tid] = h.id;
        uint32_t nvis = 0;   // unblocked shadow rays; kDeferred marks a slot whose rays wf_vis traces
        V3 hp = v3(0.f, 0.f, 0.f);
        if (h.id != kNoHit) {
            const SurfaceHit S = surface_at(P, o, d, h);
            hp = S.p;
            if (S.mat.kind == MRF_MAT_DIFFUSE) {
                if (K > 1) nvis = kDeferred;
                const uint32_t ray = path / P.spp, sp = path % P.spp;
                // shadow rays from inside the field box go to the network
                V3 pl = S.p, wdummy = v3(0.f, 0.f, 1.f);
                if (P.has_snet) snet_to_local(P.snet, pl, wdummy);
                const bool net = P.has_snet && snet_inside(P.snet, pl);
                for (int l = 0; l < P.n_lights; ++l) {
                    const uint32_t ns = P.lights[l].samples, q0 = P.lights[l].slot0;
                    for (uint32_t k = 0; k < ns; ++k) {
                        const size_t idx = (size_t)tid * K + q0 + k;
                        V3 wl;
                        float D, w3[3];
                        float4 wgt = make_float4(0.f, 0.f, 0.f, 0.f);
                        const bool valid = shadow_ray(P, S, l, k, ray, sp, j, wl, D, w3);
                        if (valid && K > 1) {
                            wgt = make_float4(w3[0], w3[1], w3[2], net ? -2.f : -1.f);   // wf_vis decides
                            W.sdir[idx] = make_float4(wl.x, wl.y, wl.z, D);
                        } else if (valid) {
                            ++C.shadow;
                            Hit hs;
                            unsigned rs = 0;
                            bool f2 = false;
                            const bool blocked =
                                bvh_trace<true>(P.B, S.p, wl, S.id, P.tmin, D, hs, rs, C.nodes, C.tris, f2);
                            C.retests += rs;
                            if (f2) C.fault |= 1;
                            if (!blocked) {
                                wgt = make_float4(w3[0], w3[1], w3[2], net ? 2.f : 1.f);
                                ++nvis;
                                if (net) {
                                    nmask |= 1ull << (q0 + k);
                                    ++nnet;
                                }
                                W.sdir[idx] = make_float4(wl.x, wl.y, wl.z, D);
                            }
                        }
                        W.sw[idx] = wgt;
                        W.scount[idx] = 0;
                    }
                }
            }
        }
        W.hp[tid] = make_float4(hp.x, hp.y, hp.z, __uint_as_float(nvis));
    }
    // queue the network's shadow rays (one atomic per warp)
    const uint32_t qbase = warp_alloc(&W.ctr[3], nnet);
    for (uint32_t i = 0; nmask; ++i) {
        const int q = __ffsll((long long)nmask) - 1;
        nmask &= nmask - 1;
        W.squeue[checked_index(qbase + i, (uint64_t)W.paths * (uint64_t)K, P.status)] = tid * (uint32_t)K + (uint32_t)q;
    }
    flush_counters(P.stats, C);
    if (C.fault && P.status) atomicOr(P.status, C.fault);
}

// Visibility of the shadow rays that wf_cast deferred (more than one per
// diffuse hit): one thread per ray, grid-stride over live slots x K.  An
// unblocked ray keeps its weight with sw.w = 1 (marched) or 2 (network: queued
// for wf_shadow_net) and counts in its slot's hp.w; a blocked one gets sw = 0.
// hp.w keeps the kDeferred bit, so the slot reads as having shadow rays and the
// later kernels look at each ray's sw.w.
__global__ void __launch_bounds__(kThreads, 5) wf_vis(const WfParams W, int cur) {
    const RenderParams &P = W.R;
    if (tail_taken(W)) return;
    const uint32_t K = (uint32_t)P.n_shadow;
    const uint64_t total = (uint64_t)W.ctr[cur] * K;
    Counters C = {};
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < total; base += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t idx = base + threadIdx.x;
        bool to_net = false;
        const uint32_t slot = (uint32_t)(idx / K);
        // only slots wf_cast marked hold current shadow-ray entries
        if (idx < total && (__float_as_uint(W.hp[slot].w) & kDeferred)) {
            float4 wgt = W.sw[idx];
            if (wgt.w < 0.f) {
                const float4 h4 = W.hp[slot], sd = W.sdir[idx];
                ++C.shadow;
                Hit hs;
                unsigned rs = 0;
                bool f2 = false;
                const bool blocked = bvh_trace<true>(P.B, v3(h4.x, h4.y, h4.z), v3(sd.x, sd.y, sd.z), W.hit_id[slot],
                                                     P.tmin, sd.w, hs, rs, C.nodes, C.tris, f2);
                C.retests += rs;
                if (f2) C.fault |= 1;
                if (blocked) {
                    wgt = make_float4(0.f, 0.f, 0.f, 0.f);
                } else {
                    wgt.w = -wgt.w;
                    to_net = wgt.w == 2.f;
                    atomicAdd(reinterpret_cast<unsigned *>(&W.hp[slot]) + 3, 1u);
                }
                W.sw[idx] = wgt;
            }
        }
        const uint32_t qi = warp_alloc(&W.ctr[3], to_net ? 1u : 0u);
        if (to_net) W.squeue[checked_index(qi, (uint64_t)W.paths * K, P.status)] = (uint32_t)idx;
    }
    flush_counters(P.stats, C);
    if (C.fault && P.status) atomicOr(P.status, C.fault);
}

// Learned shadow transmittance of every queued shadow ray (grid-stride over
// the queue), stored in sdepth.
__global__ void __launch_bounds__(128) wf_shadow_net(const WfParams W) {
    __shared__ __align__(16) float wsm[kSnetMlp + 3];
    const RenderParams &P = W.R;
    if (tail_taken(W)) return;
    for (int i = threadIdx.x; i < kSnetMlp; i += blockDim.x) wsm[i] = P.snet.mlp[i];
    __syncthreads();
    const uint32_t n = W.ctr[3], K = (uint32_t)P.n_shadow;
    Counters C = {};
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t idx = W.squeue[i], slot = idx / K;
        const float4 h4 = W.hp[slot], sh = W.sdir[idx];
        W.sdepth[idx] = snet_eval(P.snet, wsm, v3(h4.x, h4.y, h4.z), v3(sh.x, sh.y, sh.z));
        ++C.net;
    }
    flush_counters(P.stats, C);
}

// Warp-cooperative sample generation: counts the samples of every job of the
// warp's slots (segment march and visible shadow rays), allocates their
// ranges with one atomic per warp, and writes them in order.
// Round r > 0 regenerates only the slots that round r - 1 left pending (their
// samples did not fit the buffer), into the emptied buffer.
// The per-job set-up of the segment job and of the first marched shadow ray of
// each slot (the ray in the field's frame, its quadrature intervals with their
// divisions, its sphere cover, and the loads it needs) runs lane-parallel, each
// lane for its own slot, before the warp walks the jobs one after another.
struct JobSm {
    float o[3], d[3];
    Segment S;   // S.n = 0: no interval
    Cover cv;
};

__global__ void __launch_bounds__(kThreads, 4) wf_gen(const WfParams W, uint32_t j, int cur, int round) {
    __shared__ WalkSmem wsm;
    __shared__ RunList runs_sm[kThreads / 32][32][2];   // per warp, per slot: segment job, first shadow job
    __shared__ JobSm jobs_sm[kThreads / 32][32];
    __shared__ JobSm shjobs_sm[kThreads / 32][32];   // per slot: its first marched shadow ray
    const RenderParams &P = W.R;
    if (tail_taken(W) || (round > 0 && *pending_ctr(W, round - 1) == 0)) return;   // nothing to do: the grid leaves
    const WalkCtx X = stage_walk(P.F, wsm);
    const int lane = threadIdx.x & 31;
    const uint32_t live = j == 1 ? W.paths : W.ctr[cur];
    const int S = chunk_slots(live);
    const int K = P.n_shadow;
    JobSm(&jobs)[32] = jobs_sm[threadIdx.x >> 5];
    JobSm(&shjobs)[32] = shjobs_sm[threadIdx.x >> 5];
    Counters C = {};
    for (uint32_t wbase; (wbase = next_chunk(work_ctr(W, round, 0), S, lane)) < live;) {
        const uint32_t tid = wbase + (uint32_t)lane;   // this lane's slot (lane < S)
        const bool active = lane < S && tid < live && (round == 0 || W.rcount[tid] == kOverflow);
        V3 hp = v3(0.f, 0.f, 0.f);
        uint32_t vis = 0;   // unblocked shadow rays of the slot
        int sq = -1;        // the slot's first marched shadow ray
        bool walk = false;  // some job of the slot has intervals to walk
        if (active) {
            const float4 qo = W.qo[cur][tid], qd = W.qd[cur][tid], h4 = W.hp[tid];
            V3 o = v3(qo.x, qo.y, qo.z), d = v3(qd.x, qd.y, qd.z);
            hp = v3(h4.x, h4.y, h4.z);
            vis = __float_as_uint(h4.w);
            to_field_frame(P.F, o, d);
            Segment sg;
            JobSm &J = jobs[lane];
            if (segment_of(P, o, d, 0.f, W.hit_t[tid], sg)) {
                J.cv = job_cover(P.F, X, o, d, sg);
            } else {
                sg.n = 0;
                J.cv = Cover{0u, 0, 0};
            }
            J.o[0] = o.x, J.o[1] = o.y, J.o[2] = o.z;
            J.d[0] = d.x, J.d[1] = d.y, J.d[2] = d.z;
            J.S = sg;
            bool more = false;   // a second marched shadow ray
            for (int q = 0; vis && q < K; ++q)
                if (W.sw[(size_t)tid * K + q].w == 1.f) {   // marched shadow rays only
                    if (sq >= 0) {
                        more = true;
                        break;
                    }
                    sq = q;
                }
            if (sq >= 0) {
                const float4 sh = W.sdir[(size_t)tid * K + sq];
                V3 so = hp, sd = v3(sh.x, sh.y, sh.z);
                to_field_frame(P.F, so, sd);
                Segment ss;
                JobSm &J2 = shjobs[lane];
                if (segment_of(P, so, sd, 0.f, sh.w, ss)) {
                    J2.cv = job_cover(P.F, X, so, sd, ss);
                } else {
                    ss.n = 0;
                    J2.cv = Cover{0u, 0, 0};
                }
                J2.o[0] = so.x, J2.o[1] = so.y, J2.o[2] = so.z;
                J2.d[0] = sd.x, J2.d[1] = sd.y, J2.d[2] = sd.z;
                J2.S = ss;
            }
            // a job whose cover is empty has no sample: a slot with nothing else
            // to walk is done here and the warp does not visit it
            const bool sh_walk = sq >= 0 && (more || (shjobs[lane].S.n > 0 && shjobs[lane].cv.cb < shjobs[lane].cv.ce));
            walk = (sg.n > 0 && J.cv.cb < J.cv.ce) || sh_walk;
            if (!walk) {
                W.rcount[tid] = 0;
                C.nominal += (uint32_t)sg.n;
                if (sq >= 0) {
                    W.scount[(size_t)tid * K + sq] = 0;
                    C.nominal += (uint32_t)shjobs[lane].S.n;
                }
            }
        }
        __syncwarp();
        uint32_t my_nr = 0, my_ns0 = 0, my_total = 0;
        const unsigned walkers = __ballot_sync(0xffffffffu, walk);
        for (unsigned wm = walkers; wm; wm &= wm - 1u) {
            const int src = __ffs(wm) - 1;
            const V3 sp = shfl3(hp, src);
            const int ssq = __shfl_sync(0xffffffffu, sq, src);
            const uint32_t src_tid = wbase + src;
            RunList(&rl)[2] = runs_sm[threadIdx.x >> 5][src];
            const JobSm &J = jobs[src];
            uint2 wr = make_uint2(0u, (uint32_t)J.S.n);   // an empty cover: no sample
            if (J.S.n > 0 && J.cv.cb < J.cv.ce)
                wr = warp_walk_in(P, X, v3(J.o[0], J.o[1], J.o[2]), v3(J.d[0], J.d[1], J.d[2]), J.S, J.cv, nullptr, 0,
                                  lane, &rl[0]);
            else if (lane == 0)
                rl[0].n = 0;
            const uint32_t n_r = wr.x;
            if (lane == 0) C.nominal += wr.y;
            uint32_t n_s = 0, ns0 = 0;
            if (ssq >= 0) {
                // the first marched shadow ray (set up above) records its runs; the others walk from scratch
                const JobSm &J2 = shjobs[src];
                uint2 ws = make_uint2(0u, (uint32_t)J2.S.n);
                if (J2.S.n > 0 && J2.cv.cb < J2.cv.ce)
                    ws = warp_walk_in(P, X, v3(J2.o[0], J2.o[1], J2.o[2]), v3(J2.d[0], J2.d[1], J2.d[2]), J2.S, J2.cv,
                                      nullptr, 0, lane, &rl[1]);
                else if (lane == 0)
                    rl[1].n = 0;
                ns0 = ws.x;
                if (lane == 0) C.nominal += ws.y;
                if (lane == src) W.scount[(size_t)src_tid * K + ssq] = ns0;
                n_s = ns0;
                for (int q = ssq + 1; q < K; ++q) {
                    const size_t idx = (size_t)src_tid * K + q;
                    if (W.sw[idx].w != 1.f) continue;   // marched shadow rays only
                    const float4 sh = W.sdir[idx];
                    const uint2 wq = warp_walk(P, X, sp, v3(sh.x, sh.y, sh.z), 0.f, sh.w, nullptr, 0, lane, nullptr);
                    if (lane == 0) C.nominal += wq.y;
                    if (lane == src) W.scount[idx] = wq.x;
                    n_s += wq.x;
                }
            }
            if (lane == src) {
                W.rcount[tid] = n_r;
                my_nr = n_r;
                my_ns0 = ns0;
                my_total = n_r + n_s;
                C.evaluated += n_r;
                C.shadow_eval += n_s;
            }
        }
        const uint32_t base = warp_alloc(&W.ctr[2], my_total);
        const bool fits = (uint64_t)base + my_total <= (uint64_t)W.cap;
        if (active && !walk) W.rstart[tid] = base;
        __syncwarp();
        for (unsigned wm = walkers; wm; wm &= wm - 1u) {
            const int src = __ffs(wm) - 1;
            const bool sfits = __shfl_sync(0xffffffffu, (int)fits, src);
            const uint32_t sbase = __shfl_sync(0xffffffffu, base, src);
            const int ssq = __shfl_sync(0xffffffffu, sq, src);
            const uint32_t src_tid = wbase + src;
            if (!sfits) {
                if (lane == src) {
                    W.rcount[tid] = kOverflow;
                    for (int q = 0; vis && q < K; ++q)
                        if (W.sw[(size_t)tid * K + q].w == 1.f) W.scount[(size_t)tid * K + q] = kOverflow;
                    atomicAdd(pending_ctr(W, round), 1u);
                }
                continue;
            }
            const V3 sp = shfl3(hp, src);
            uint32_t k = sbase;
            const uint32_t nr = __shfl_sync(0xffffffffu, my_nr, src);
            const RunList(&rl)[2] = runs_sm[threadIdx.x >> 5][src];
            const JobSm &J = jobs[src];
            const V3 jo = v3(J.o[0], J.o[1], J.o[2]), jd = v3(J.d[0], J.d[1], J.d[2]);
            if (nr > 0) {
                if (rl[0].n <= kRunsPerJob)
                    write_runs_in(P, jo, jd, J.S, rl[0], W.samp + k, nr, lane);
                else
                    warp_walk_in(P, X, jo, jd, J.S, J.cv, W.samp + k, nr, lane, nullptr);
            }
            if (P.F.view_dep)   // the colour network needs each radiance sample's view direction (field frame)
                for (uint32_t i = lane; i < nr; i += 32) W.sview[k + i] = make_float4(jd.x, jd.y, jd.z, 0.f);
            k += nr;
            if (lane == src) W.rstart[tid] = sbase;
            if (ssq >= 0) {
                const JobSm &J2 = shjobs[src];
                const uint32_t ns0 = __shfl_sync(0xffffffffu, my_ns0, src);
                if (lane == src) W.sstart[(size_t)src_tid * K + ssq] = k;
                if (ns0 > 0) {
                    const V3 so = v3(J2.o[0], J2.o[1], J2.o[2]), sd = v3(J2.d[0], J2.d[1], J2.d[2]);
                    if (rl[1].n <= kRunsPerJob)
                        write_runs_in(P, so, sd, J2.S, rl[1], W.samp + k, ns0, lane);
                    else
                        warp_walk_in(P, X, so, sd, J2.S, J2.cv, W.samp + k, ns0, lane, nullptr);
                }
                k += ns0;
                for (int q = ssq + 1; q < K; ++q) {
                    const size_t idx = (size_t)src_tid * K + q;
                    if (W.sw[idx].w != 1.f) continue;
                    const float4 sh = W.sdir[idx];
                    const uint32_t ns = W.scount[idx];
                    if (lane == src) W.sstart[idx] = k;
                    warp_walk(P, X, sp, v3(sh.x, sh.y, sh.z), 0.f, sh.w, W.samp + k, ns, lane, nullptr);
                    k += ns;
                }
            }
        }
        __syncwarp();   // runs_sm, jobs_sm and shjobs_sm are rewritten by the next chunk
    }
    if (round > 0) C.evaluated = C.shadow_eval = 0, C.nominal = 0;   // counted by round 0
    flush_counters(P.stats, C);
}

// Warp-cooperative compositing of one job's samples (every lane holds the same
// job): 32 consecutive samples per step, cumulative optical depth by a warp
// scan, T(t) = T0 exp(-depth before the sample), L += T(t) alpha r (Eqs. 10-11).
// Stops after the sample at which max(T) falls below tau.  Each lane returns
// its partial sums of L; `depth` (the job's optical depth up to the stop) and
// `stop` are the same in every lane.
// warp_composite_from continues a job from the lane partial sums, depth and
// stop of its earlier samples: a job split at multiples of 32 samples gives the
// same results as one call.
__device__ __forceinline__ void warp_composite_from(const WfParams &W, uint32_t start, uint32_t count, float tmax0,
                                                    float tau, int lane, float &lr, float &lg, float &lb,
                                                    float &depth, bool &stop) {
    // eight 32-sample chunks are loaded before the first is composited, so that a
    // job costs one memory round trip per 256 samples (loads past the stop are
    // inside the job's range and harmless)
    constexpr int kChunks = 8;
    for (uint32_t i0 = 0; i0 < count; i0 += 32 * kChunks) {
        float4 fc[kChunks];
#pragma unroll
        for (int u = 0; u < kChunks; ++u) {
            const uint32_t i = i0 + 32u * u + lane;
            fc[u] = i < count ? W.fout[start + i] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kChunks; ++u) {
            if (i0 + 32u * u >= count) break;
            const bool v = i0 + 32u * u + lane < count;
            const float4 f = fc[u];
            const float x = f.x;   // sigma * delta, from the field kernel (0 past the job)
            float sc = x;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const float y = __shfl_up_sync(0xffffffffu, sc, off);
                if (lane >= off) sc += y;
            }
            const float before = depth + (sc - x), after = depth + sc;
            const bool cross = v && tau > 0.f && tmax0 * expf(-after) < tau;
            const unsigned cm = __ballot_sync(0xffffffffu, cross);
            const int last = cm ? __ffs(cm) - 1 : 31;
            if (v && lane <= last) {
                const float a = -expm1f(-x) * expf(-before);
                lr = fmaf(a, f.y, lr);
                lg = fmaf(a, f.z, lg);
                lb = fmaf(a, f.w, lb);
            }
            depth += __shfl_sync(0xffffffffu, sc, last);
            if (cm) {
                stop = true;
                return;
            }
        }
    }
}

__device__ __forceinline__ void warp_composite(const WfParams &W, uint32_t start, uint32_t count, float tmax0,
                                               float tau, int lane, float &lr, float &lg, float &lb, float &depth,
                                               bool &stop) {
    lr = lg = lb = 0.f;
    depth = 0.f;
    stop = false;
    warp_composite_from(W, start, count, tmax0, tau, lane, lr, lg, lb, depth, stop);
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    return x;
}

// Warp-cooperative compositing of every live slot's segment samples and
// shadow samples (Eqs. 10-11).  Writes, per slot, sum_i exp(-depth_i) alpha_i r_i
// (to be scaled by T(p_j)) and the optical depth up to the stop; a negative
// depth marks a path that fell below tau inside the segment.  Jobs that did not
// fit the sample buffer stay pending for the next round (or wf_overflow);
// composited slots are marked done so that later rounds pass them by.
__global__ void __launch_bounds__(kThreads, 8) wf_composite(const WfParams W, int cur, int round) {
    const RenderParams &P = W.R;
    if (tail_taken(W) || (round > 0 && *pending_ctr(W, round - 1) == 0)) return;
    const int lane = threadIdx.x & 31;
    const uint32_t live = W.ctr[cur];
    const int S = chunk_slots(live);
    for (uint32_t wbase; (wbase = next_chunk(work_ctr(W, round, 2), S, lane)) < live;) {
        const uint32_t tid = wbase + (uint32_t)lane;   // this lane's slot (lane < S)
        bool active = lane < S && tid < live;
        const int K = P.n_shadow;
        uint32_t rc = kOverflow, r0 = 0;
        float tmax = 0.f;
        bool diffuse = false;
        if (active) {
            rc = W.rcount[tid];
            active = rc != kOverflow && rc != kDone;   // generated in this round
            r0 = W.rstart[tid];
            const float4 qT = W.qT[cur][tid];
            tmax = fmaxf(qT.x, fmaxf(qT.y, qT.z));
            diffuse = __float_as_uint(W.hp[tid].w) != 0u;   // some unblocked shadow ray from a diffuse hit
            if (active) W.rcount[tid] = kDone;   // read below from the registers only
            if (active && rc == 0 && !diffuse) {   // no sample and no shadow depth: done here
                W.comp[tid] = make_float4(0.f, 0.f, 0.f, 0.f);
                active = false;
            }
        }
        for (unsigned am = __ballot_sync(0xffffffffu, active); am; am &= am - 1u) {
            const int src = __ffs(am) - 1;
            const uint32_t src_rc = __shfl_sync(0xffffffffu, rc, src);
            const uint32_t src_tid = wbase + src;
            {
                const uint32_t src_r0 = __shfl_sync(0xffffffffu, r0, src);
                const float tmax0 = __shfl_sync(0xffffffffu, tmax, src);
                float lr, lg, lb, dep;
                bool stp;
                warp_composite(W, src_r0, src_rc, tmax0, P.tau, lane, lr, lg, lb, dep, stp);
                lr = warp_sum(lr);
                lg = warp_sum(lg);
                lb = warp_sum(lb);
                if (lane == 0) W.comp[src_tid] = make_float4(lr, lg, lb, stp ? -dep - 1.f : dep);
            }
            if (!__shfl_sync(0xffffffffu, (int)diffuse, src)) continue;
            for (int q = 0; q < K; ++q) {
                const size_t idx = (size_t)src_tid * K + q;
                if (W.sw[idx].w != 1.f) continue;
                const uint32_t sc = W.scount[idx];
                if (sc == kOverflow) continue;
                const uint32_t s0 = W.sstart[idx];
                float dep = 0.f;
#pragma unroll 4
                for (uint32_t i0 = lane; i0 < sc; i0 += 32) dep += W.fout[s0 + i0].x;
                dep = warp_sum(dep);
                if (lane == 0) W.sdepth[idx] = dep;
            }
        }
    }
}

// Shadow mask of Sec. 3.1 on the segment samples (radiance jobs only): the
// radiance of every sample with sigma > 0 is scaled by m(p_t).  One warp walks
// the samples of each of its slots' jobs.
__global__ void __launch_bounds__(kThreads) wf_mask(const WfParams W, int cur, int round) {
    const RenderParams &P = W.R;
    if (tail_taken(W) || (round > 0 && *pending_ctr(W, round - 1) == 0)) return;
    const int lane = threadIdx.x & 31;
    const uint32_t live = W.ctr[cur];
    const int S = chunk_slots(live);
    for (uint32_t wbase; (wbase = next_chunk(work_ctr(W, round, 1), S, lane)) < live;) {
        const uint32_t tid = wbase + (uint32_t)lane;   // this lane's slot (lane < S)
        const bool active = lane < S && tid < live;
        uint32_t rc = kOverflow, r0 = 0;
        if (active) {
            rc = W.rcount[tid];
            r0 = W.rstart[tid];
        }
        for (int src = 0; src < S; ++src) {
            const uint32_t src_rc = __shfl_sync(0xffffffffu, rc, src);
            const uint32_t src_r0 = __shfl_sync(0xffffffffu, r0, src);
            if (!__shfl_sync(0xffffffffu, (int)active, src) || src_rc == kOverflow || src_rc == kDone) continue;
            for (uint32_t i = lane; i < src_rc; i += 32) {
                float4 f = W.fout[src_r0 + i];
                if (!(f.x > 0.f)) continue;
                const float4 q = W.samp[src_r0 + i];
                const float m = sample_mask(P, field_to_world(P.F, v3(q.x, q.y, q.z)));
                if (m != 1.f) {
                    f.y *= m;
                    f.z *= m;
                    f.w *= m;
                    W.fout[src_r0 + i] = f;
                }
            }
        }
    }
}

// Jobs whose samples did not fit the sample buffer are marched in place here,
// on the CUDA cores in FP32, producing the same per-slot results as
// wf_composite (comp, sdepth).  Nothing to do when no job overflowed.
__global__ void __launch_bounds__(kThreads) wf_overflow(const WfParams W, int cur, int last_round) {
    const RenderParams &P = W.R;
    // nothing left pending after the last generation round: the whole grid leaves
    if (tail_taken(W) || *pending_ctr(W, last_round) == 0) return;
    const uint32_t live = W.ctr[cur];
    const int K = P.n_shadow;
    for (uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x; tid < live; tid += gridDim.x * blockDim.x) {
        const bool rad = W.rcount[tid] == kOverflow;
        const float4 h4 = W.hp[tid];
        bool any_shadow = false;
        if (__float_as_uint(h4.w) != 0u)   // unblocked shadow rays (only their counts are current)
            for (int q = 0; q < K; ++q)
                any_shadow |= W.sw[(size_t)tid * K + q].w == 1.f && W.scount[(size_t)tid * K + q] == kOverflow;
        if (!rad && !any_shadow) continue;
        const float4 qo = W.qo[cur][tid], qd = W.qd[cur][tid], qT = W.qT[cur][tid];
        const V3 o = v3(qo.x, qo.y, qo.z), d = v3(qd.x, qd.y, qd.z);
        if (rad) {
            // march with the path's own throughput so that the tau test is the same
            float T[3] = {qT.x, qT.y, qT.z}, L[3] = {0.f, 0.f, 0.f};
            bool stop = false;
            Counters dummy = {};
            march<true>(P, P.F.mlp, o, d, 0.f, W.hit_t[tid], T, L, stop, dummy);
            const int c = (qT.x >= qT.y && qT.x >= qT.z) ? 0 : (qT.y >= qT.z ? 1 : 2);
            const float T0[3] = {qT.x, qT.y, qT.z};
            const float dep = T0[c] > 0.f ? logf(T0[c] / fmaxf(T[c], 1e-38f)) : 0.f;
            W.comp[tid] = make_float4(T0[0] > 0.f ? L[0] / T0[0] : 0.f, T0[1] > 0.f ? L[1] / T0[1] : 0.f,
                                      T0[2] > 0.f ? L[2] / T0[2] : 0.f, stop ? -dep - 1.f : dep);
        }
        if (any_shadow) {
            const V3 hp = v3(h4.x, h4.y, h4.z);
            for (int q = 0; q < K; ++q) {
                const size_t idx = (size_t)tid * K + q;
                if (W.sw[idx].w != 1.f || W.scount[idx] != kOverflow) continue;
                const float4 sh = W.sdir[idx];
                Counters dummy = {};
                bool dstop = false;
                W.sdepth[idx] = march<false>(P, P.F.mlp, hp, v3(sh.x, sh.y, sh.z), 0.f, sh.w, nullptr, nullptr, dstop,
                                             dummy);
            }
        }
    }
}

// Per live slot: apply the composited segment (Eq. 11), add the next-event
// terms, sample the BSDF (Eqs. 12-13), test termination and push survivors.
__global__ void __launch_bounds__(kThreads) wf_shade(const WfParams W, uint32_t j, int cur, int nxt) {
    const RenderParams &P = W.R;
    if (tail_taken(W)) return;
    const uint32_t live = W.ctr[cur];
    const int K = P.n_shadow;
    Counters C = {};
    for (uint32_t base = blockIdx.x * blockDim.x; base < live; base += gridDim.x * blockDim.x) {
        const uint32_t tid = base + threadIdx.x;
        bool push = false;
        uint32_t path = 0, prev = kNoHit;
        V3 o = v3(0.f, 0.f, 0.f), d = v3(0.f, 0.f, 1.f);
        float T[3] = {1.f, 1.f, 1.f};
        if (tid < live) {
            path = W.qpath[cur][tid];
            const uint32_t ray = path / P.spp, s = path % P.spp;
            const float4 qo = W.qo[cur][tid], qd = W.qd[cur][tid], qT = W.qT[cur][tid];
            o = v3(qo.x, qo.y, qo.z);
            d = v3(qd.x, qd.y, qd.z);
            T[0] = qT.x;
            T[1] = qT.y;
            T[2] = qT.z;
            Hit h;
            h.t = W.hit_t[tid];
            h.slot = W.hit_slot[tid];
            h.id = W.hit_id[tid];
            float4 acc = j == 1 ? make_float4(0.f, 0.f, 0.f, 0.f) : W.acc[path];
            float L[3] = {acc.x, acc.y, acc.z};
            const float T0 = T[0];
            bool stop = false;
            {
                // L += T(p_j) * sum_i T_i alpha_i r_i, T' = T(p_j) exp(-depth)
                const float4 cp = W.comp[tid];
                stop = cp.w < 0.f;
                const float att = expf(-(stop ? -cp.w - 1.f : cp.w));
                L[0] = fmaf(T[0], cp.x, L[0]);
                L[1] = fmaf(T[1], cp.y, L[1]);
                L[2] = fmaf(T[2], cp.z, L[2]);
                T[0] *= att;
                T[1] *= att;
                T[2] *= att;
            }
            if (j == 1) acc.w = T0 > 0.f ? 1.f - T[0] / T0 : 0.f;
            ++C.seg;
            const uint64_t rbase = (uint64_t)path * P.max_bounces;
            if (P.rec_tri) {
                P.rec_tri[rbase + (j - 1)] = h.id;
                P.rec_t[rbase + (j - 1)] = h.t;
            }
            bool end = stop || h.id == kNoHit;
            int cause = stop ? 2 : (h.id == kNoHit ? 1 : 0);   // 1 left the scene, 2 throughput below tau, 3 bounce cap
            if (!end) {
                ++C.hits;
                const SurfaceHit S = surface_at(P, o, d, h);
                float u[3];
                surface_uniforms(P, ray, s, j, u);
                if (S.mat.kind == MRF_MAT_DIFFUSE && __float_as_uint(W.hp[tid].w) != 0u) {
                    for (int q = 0; q < K; ++q) {
                        const size_t idx = (size_t)tid * K + q;
                        const float4 wgt = W.sw[idx];
                        if (wgt.w == 0.f) continue;
                        const float Tf = wgt.w == 2.f ? W.sdepth[idx] : expf(-W.sdepth[idx]);
                        L[0] = fmaf(T[0] * Tf, wgt.x, L[0]);
                        L[1] = fmaf(T[1] * Tf, wgt.y, L[1]);
                        L[2] = fmaf(T[2] * Tf, wgt.z, L[2]);
                    }
                }
                const V3 nd = bsdf_sample(S, d, u, T);
                d = normalize(nd);
                o = S.p;
                prev = S.id;
                if (P.tau > 0.f && fmaxf(T[0], fmaxf(T[1], T[2])) < P.tau) {
                    end = true;
                    cause = 2;
                } else if (j == P.max_bounces) {
                    end = true;
                    cause = 3;
                }
            }
            acc.x = L[0];
            acc.y = L[1];
            acc.z = L[2];
            W.acc[path] = acc;
            if (end) {
                C.end_miss += cause == 1;
                C.end_tau += cause == 2;
                C.end_cap += cause == 3;
                if (P.rec_seg) P.rec_seg[path] = j;
                if (P.rec_tri)
                    for (uint32_t q = j; q < P.max_bounces; ++q) {
                        P.rec_tri[rbase + q] = kNoHit;
                        P.rec_t[rbase + q] = INFINITY;
                    }
            }
            push = !end;
        }
        uint32_t slot = warp_alloc(&W.ctr[nxt], push ? 1u : 0u);
        if (push) {
            slot = checked_index(slot, W.paths, P.status);
            W.qpath[nxt][slot] = path;
            W.qo[nxt][slot] = make_float4(o.x, o.y, o.z, __uint_as_float(prev));
            W.qd[nxt][slot] = make_float4(d.x, d.y, d.z, 0.f);
            W.qT[nxt][slot] = make_float4(T[0], T[1], T[2], 0.f);
        }
    }
    flush_counters(P.stats, C);
}

// ---------------------------------------------------------------------------
// Persistent tail.  When at most the tuning's tail_paths paths are live at the
// start of a segment, wf_cast records that segment and every kernel of the
// remaining segments leaves at once; wf_tail, launched once after them, then
// finishes the remaining paths: each warp pops a path from the live queue and
// runs all of its remaining segments, with the wavefront's own steps and
// formulas (closest hit, shadow rays, the sample walk of wf_gen, compositing
// by warp_composite, the surface event of wf_shade).  Paths then wait only on
// their own chain of dependent traversals instead of the slowest path of every
// segment.  The few samples of the tail are evaluated on the CUDA cores with
// the FP32 weights (also for FP16/BF16 fields, as the overflow march does); an
// FP32 field gives the wavefront engine's result bit for bit.
constexpr int kTailWarps = 8;   // warps per tail block

// The steps of the tail that need many registers, kept out of its main loop:
// one field sample as the FP32 field kernel and wf_mask evaluate it,
__device__ __noinline__ float4 tail_sample(const RenderParams &P, const float *wts, float4 rec, V3 dl, bool radiance) {
    const V3 p = v3(rec.x, rec.y, rec.z);
    float rgb[3] = {0.f, 0.f, 0.f}, sigma = 0.f;
    if (inside_field_box(P.F, p)) {
        bool ev;
        sigma = field_at<true>(P.F, wts, p, dl, rgb, ev);
    }
    float4 f = make_float4(sigma * rec.w, rgb[0], rgb[1], rgb[2]);
    if (radiance && P.shadow_mask && f.x > 0.f) {
        const float m = sample_mask(P, field_to_world(P.F, p));
        if (m != 1.f) {
            f.y *= m;
            f.z *= m;
            f.w *= m;
        }
    }
    return f;
}

// a segment whose samples do not fit the warp's slice, marched in place as wf_overflow does,
__device__ __noinline__ float4 tail_march(const RenderParams &P, V3 o, V3 d, float t_hit, const float T[3]) {
    float Tm[3] = {T[0], T[1], T[2]}, Lm[3] = {0.f, 0.f, 0.f};
    bool stop = false;
    Counters dummy = {};
    march<true>(P, P.F.mlp, o, d, 0.f, t_hit, Tm, Lm, stop, dummy);
    const int c = (T[0] >= T[1] && T[0] >= T[2]) ? 0 : (T[1] >= T[2] ? 1 : 2);
    const float dep = T[c] > 0.f ? logf(T[c] / fmaxf(Tm[c], 1e-38f)) : 0.f;
    return make_float4(T[0] > 0.f ? Lm[0] / T[0] : 0.f, T[1] > 0.f ? Lm[1] / T[1] : 0.f, T[2] > 0.f ? Lm[2] / T[2] : 0.f,
                       stop ? -dep - 1.f : dep);
}

// the optical depth of a shadow ray marched in place,
__device__ __noinline__ float tail_shadow_depth(const RenderParams &P, V3 p, V3 w, float D) {
    Counters dummy = {};
    bool dstop = false;
    return march<false>(P, P.F.mlp, p, w, 0.f, D, nullptr, nullptr, dstop, dummy);
}

// the compositing of a window of a segment's samples (warp_composite, continued),
__device__ __noinline__ void tail_composite(const WfParams &W, uint32_t start, uint32_t n, float tmax0, int lane,
                                            float &lr, float &lg, float &lb, float &dep, bool &stp) {
    warp_composite_from(W, start, n, tmax0, W.R.tau, lane, lr, lg, lb, dep, stp);
}

// the network's transmittance of a shadow ray,
__device__ __noinline__ float tail_net(const RenderParams &P, V3 p, V3 w) { return snet_eval(P.snet, P.snet.mlp, p, w); }

// the closest hit of a path's segment (with its traversal statistics),
__device__ __noinline__ Hit tail_cast(const RenderParams &P, V3 o, V3 d, uint32_t prev, uint32_t path, Counters &C) {
    Hit h;
    unsigned rt = 0;
    bool fault = false;
    const unsigned nodes0 = C.nodes;
    bvh_trace<false>(P.B, o, d, prev, P.tmin, INFINITY, h, rt, C.nodes, C.tris, fault);
    note_traversal(C, C.nodes - nodes0, path);
    C.retests += rt;
    if (fault) C.fault |= 1;
    return h;
}

// and the visibility of a shadow ray (true: a mesh blocks it).
__device__ __noinline__ bool tail_blocked(const RenderParams &P, V3 p, V3 w, uint32_t skip, float D, Counters &C) {
    Hit hs;
    unsigned rs = 0;
    bool f2 = false;
    const bool blocked = bvh_trace<true>(P.B, p, w, skip, P.tmin, D, hs, rs, C.nodes, C.tris, f2);
    C.retests += rs;
    if (f2) C.fault |= 1;
    return blocked;
}

__global__ void __launch_bounds__(32 * kTailWarps, 1) wf_tail(const WfParams W) {
    extern __shared__ float tail_w[];     // FP32 field weights (hash grid)
    __shared__ WalkSmem wsm;
    __shared__ RunList runs_sm[kTailWarps];
    const RenderParams &P = W.R;
    const uint32_t j0 = W.ctr[kTailWord];
    if (j0 == 0u) return;
    const WalkCtx X = stage_walk(P.F, wsm);
    const float *wts = P.F.mlp;
    if (P.F.kind == MRF_FIELD_HASHGRID) {
        const int nw = field_mlp_floats(P.F);
        for (int i = threadIdx.x; i < nw; i += blockDim.x) tail_w[i] = P.F.mlp[i];
        __syncthreads();
        wts = tail_w;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t live = W.ctr[kTailWord + 1];
    const int qi = (int)((j0 - 1u) & 1u);
    const int K = P.n_shadow;
    // this warp's slice of the (otherwise idle) sample buffer
    const uint32_t n_warps = gridDim.x * kTailWarps, gw = blockIdx.x * kTailWarps + wid;
    // windows of up to 1024 samples (a multiple of 32), whatever the buffer size, so
    // that every buffer gives the same result
    const uint32_t slice = min(W.cap / n_warps, 1024u) & ~31u, sbase = gw * slice;
    RunList &rl = runs_sm[wid];
    Counters C = {};
    for (uint32_t slot; (slot = next_chunk(W.ctr + kTailWord + 2, 1, lane)) < live;) {
        const uint32_t path = W.qpath[qi][slot];
        const float4 qo = W.qo[qi][slot], qd = W.qd[qi][slot], qT = W.qT[qi][slot];
        V3 o = v3(qo.x, qo.y, qo.z), d = v3(qd.x, qd.y, qd.z);
        uint32_t prev = __float_as_uint(qo.w);
        float T[3] = {qT.x, qT.y, qT.z};
        float4 acc = W.acc[path];
        float L[3] = {acc.x, acc.y, acc.z};
        const uint32_t ray = path / P.spp, sp = path % P.spp;
        const uint64_t rbase = (uint64_t)path * P.max_bounces;
        for (uint32_t j = j0; j <= P.max_bounces; ++j) {
            // closest hit (Eq. 3), traced by lane 0
            Hit h;
            h.t = INFINITY;
            h.slot = -1;
            h.id = kNoHit;
            if (lane == 0) h = tail_cast(P, o, d, prev, path, C);
            h.t = __shfl_sync(0xffffffffu, h.t, 0);
            h.slot = __shfl_sync(0xffffffffu, h.slot, 0);
            h.id = __shfl_sync(0xffffffffu, h.id, 0);
            SurfaceHit S;
            bool diffuse = false;
            if (h.id != kNoHit) {
                S = surface_at(P, o, d, h);
                diffuse = S.mat.kind == MRF_MAT_DIFFUSE;
            }
            // shadow rays at a diffuse hit: lane l holds rays l and l + 32
            V3 pl = diffuse ? S.p : v3(0.f, 0.f, 0.f), wdummy = v3(0.f, 0.f, 1.f);
            if (diffuse && P.has_snet) snet_to_local(P.snet, pl, wdummy);
            const bool net = diffuse && P.has_snet && snet_inside(P.snet, pl);
            float sw_w[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}}, s_tf[2] = {0.f, 0.f};
            bool s_on[2] = {false, false};   // unblocked (weight applies)
            V3 s_dir[2] = {v3(0.f, 0.f, 1.f), v3(0.f, 0.f, 1.f)};
            float s_D[2] = {0.f, 0.f};
            // the value of ray q, held by lane q % 32 in entry q / 32, in every lane
            auto from = [&](const float (&v)[2], int q) {
                return __shfl_sync(0xffffffffu, q < 32 ? v[0] : v[1], q & 31);
            };
            if (diffuse) {
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2) {
                    const int qq = lane + 32 * h2;
                    if (qq >= K) continue;
                    int l = 0;
                    while (l + 1 < P.n_lights && (int)P.lights[l + 1].slot0 <= qq) ++l;
                    const uint32_t k = (uint32_t)qq - P.lights[l].slot0;
                    V3 wl;
                    float D, w3[3];
                    if (!shadow_ray(P, S, l, k, ray, sp, j, wl, D, w3)) continue;
                    ++C.shadow;
                    if (tail_blocked(P, S.p, wl, S.id, D, C)) continue;
                    s_on[h2] = true;
                    s_dir[h2] = wl;
                    s_D[h2] = D;
                    sw_w[h2][0] = w3[0];
                    sw_w[h2][1] = w3[1];
                    sw_w[h2][2] = w3[2];
                    if (net) {
                        s_tf[h2] = tail_net(P, S.p, wl);
                        ++C.net;
                    }
                }
            }
            // marches: job -1 the segment [0, t_hit], job q >= 0 shadow ray q (marched ones)
            float4 comp = make_float4(0.f, 0.f, 0.f, 0.f);
            const float tmax0 = fmaxf(T[0], fmaxf(T[1], T[2]));
            for (int q = -1; q < (diffuse && !net ? K : 0); ++q) {
                V3 jo = o, jd = d;
                float jb = h.t;
                if (q >= 0) {
                    if (!__shfl_sync(0xffffffffu, (int)(q < 32 ? s_on[0] : s_on[1]), q & 31)) continue;
                    jo = S.p;
                    jd = shfl3(q < 32 ? s_dir[0] : s_dir[1], q & 31);
                    jb = from(s_D, q);
                }
                const uint2 wr = warp_walk(P, X, jo, jd, 0.f, jb, nullptr, 0, lane, &rl);
                const uint32_t n = wr.x;
                if (lane == 0) {
                    C.nominal += wr.y;
                    if (q < 0) C.evaluated += n;
                    else C.shadow_eval += n;
                }
                __syncwarp();
                float res = 0.f;   // shadow: optical depth
                const bool replay = rl.n <= kRunsPerJob;
                if (slice > 0 && (replay || n <= slice)) {
                    // the job's samples in windows of the slice (a multiple of 32 samples):
                    // written, evaluated, then composited from the carried sums
                    float lr = 0.f, lg = 0.f, lb = 0.f, dep = 0.f;
                    bool stp = false;
                    V3 ol = jo, dl = jd;
                    to_field_frame(P.F, ol, dl);
                    for (uint32_t c0 = 0; c0 < n && !stp; c0 += slice) {
                        const uint32_t cn = min(slice, n - c0);
                        if (replay)
                            write_runs(P, jo, jd, 0.f, jb, rl, W.samp + sbase, cn, lane, c0);
                        else   // more runs than recorded (then n <= slice): the walk writes them
                            warp_walk(P, X, jo, jd, 0.f, jb, W.samp + sbase, cn, lane, nullptr);
                        __syncwarp();
                        for (uint32_t i = lane; i < cn; i += 32)
                            W.fout[sbase + i] = tail_sample(P, wts, W.samp[sbase + i], dl, q < 0);
                        __syncwarp();
                        if (q < 0) {
                            tail_composite(W, sbase, cn, tmax0, lane, lr, lg, lb, dep, stp);
                        } else {
#pragma unroll 4
                            for (uint32_t i0 = lane; i0 < cn; i0 += 32) dep += W.fout[sbase + i0].x;
                        }
                        __syncwarp();
                    }
                    if (q < 0) comp = make_float4(warp_sum(lr), warp_sum(lg), warp_sum(lb), stp ? -dep - 1.f : dep);
                    else res = warp_sum(dep);
                } else if (q < 0) {
                    // no room at all: marched in place, as wf_overflow does
                    comp = tail_march(P, o, d, h.t, T);
                } else {
                    res = tail_shadow_depth(P, S.p, jd, jb);
                }
                if (q >= 0 && lane == (q & 31)) {
                    if (q < 32) s_tf[0] = res;
                    else s_tf[1] = res;
                }
            }
            // the surface event (all lanes take the same steps; lane 0 records)
            bool stop = comp.w < 0.f;
            {
                const float att = expf(-(stop ? -comp.w - 1.f : comp.w));
                L[0] = fmaf(T[0], comp.x, L[0]);
                L[1] = fmaf(T[1], comp.y, L[1]);
                L[2] = fmaf(T[2], comp.z, L[2]);
                T[0] *= att;
                T[1] *= att;
                T[2] *= att;
            }
            if (lane == 0) {
                ++C.seg;
                if (P.rec_tri) {
                    P.rec_tri[rbase + (j - 1)] = h.id;
                    P.rec_t[rbase + (j - 1)] = h.t;
                }
            }
            bool end = stop || h.id == kNoHit;
            int cause = stop ? 2 : (h.id == kNoHit ? 1 : 0);
            if (!end) {
                if (lane == 0) ++C.hits;
                float u[3];
                surface_uniforms(P, ray, sp, j, u);
                if (diffuse) {
                    for (int q = 0; q < K; ++q) {
                        if (!__shfl_sync(0xffffffffu, (int)(q < 32 ? s_on[0] : s_on[1]), q & 31)) continue;
                        const float tq = from(s_tf, q);
                        const float Tf = net ? tq : expf(-tq);
                        const float w0 = __shfl_sync(0xffffffffu, q < 32 ? sw_w[0][0] : sw_w[1][0], q & 31);
                        const float w1 = __shfl_sync(0xffffffffu, q < 32 ? sw_w[0][1] : sw_w[1][1], q & 31);
                        const float w2 = __shfl_sync(0xffffffffu, q < 32 ? sw_w[0][2] : sw_w[1][2], q & 31);
                        L[0] = fmaf(T[0] * Tf, w0, L[0]);
                        L[1] = fmaf(T[1] * Tf, w1, L[1]);
                        L[2] = fmaf(T[2] * Tf, w2, L[2]);
                    }
                }
                const V3 nd = bsdf_sample(S, d, u, T);
                d = normalize(nd);
                o = S.p;
                prev = S.id;
                if (P.tau > 0.f && fmaxf(T[0], fmaxf(T[1], T[2])) < P.tau) {
                    end = true;
                    cause = 2;
                } else if (j == P.max_bounces) {
                    end = true;
                    cause = 3;
                }
            }
            if (end) {
                if (lane == 0) {
                    C.end_miss += cause == 1;
                    C.end_tau += cause == 2;
                    C.end_cap += cause == 3;
                    if (P.rec_seg) P.rec_seg[path] = j;
                    if (P.rec_tri)
                        for (uint32_t q = j; q < P.max_bounces; ++q) {
                            P.rec_tri[rbase + q] = kNoHit;
                            P.rec_t[rbase + q] = INFINITY;
                        }
                }
                break;
            }
        }
        if (lane == 0) W.acc[path] = make_float4(L[0], L[1], L[2], acc.w);
    }
    flush_counters(P.stats, C);
    if (C.fault && P.status) atomicOr(P.status, C.fault);
}

__global__ void __launch_bounds__(kThreads) wf_finalize(const float4 *__restrict__ acc, uint32_t count, uint32_t spp,
                                                        float4 *__restrict__ out) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= count) return;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
    for (uint32_t s = 0; s < spp; ++s) {
        const float4 v = acc[(size_t)r * spp + s];
        a.x += v.x; a.y += v.y; a.z += v.z; a.w += v.w;
    }
    const float inv = 1.f / (float)spp;
    out[r] = make_float4(a.x * inv, a.y * inv, a.z * inv, a.w * inv);
}

// scratch layout
struct Layout {
    size_t acc, qpath[2], qo[2], qd[2], qT[2], hit_t, hit_slot, hit_id, rstart, rcount, sstart, scount, sw, hp, sdir,
        comp, sdepth, squeue, ctr, samp, fout, sview, total;
    uint32_t cap;
};

Layout layout(uint32_t paths, int n_shadow, uint32_t cap_per_path = 96, bool view_dep = false) {
    Layout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t P = paths, nl = (size_t)std::max(n_shadow, 1);
    L.acc = take(16 * P);
    for (int q = 0; q < 2; ++q) {
        L.qpath[q] = take(4 * P);
        L.qo[q] = take(16 * P);
        L.qd[q] = take(16 * P);
        L.qT[q] = take(16 * P);
    }
    L.hit_t = take(4 * P);
    L.hit_slot = take(4 * P);
    L.hit_id = take(4 * P);
    L.rstart = take(4 * P);
    L.rcount = take(4 * P);
    L.sstart = take(4 * P * nl);
    L.scount = take(4 * P * nl);
    L.sw = take(16 * P * nl);
    L.hp = take(16 * P);
    L.sdir = take(16 * P * nl);
    L.comp = take(16 * P);
    L.sdepth = take(4 * P * nl);
    L.squeue = take(4 * P * nl);
    L.ctr = take(4 * kCtrWords);
    // sample capacity: cap_per_path samples per path plus 4M (overflowing jobs are marched in place)
    const uint64_t cap = std::min<uint64_t>((uint64_t)P * (cap_per_path ? cap_per_path : 96) + (4u << 20),
                                            0x7FFFFFFFull);
    L.cap = (uint32_t)cap;
    L.samp = take(16 * cap);
    L.fout = take(16 * cap);
    L.sview = view_dep ? take(16 * cap) : 0;
    L.total = off;
    return L;
}

// Blocks of `kernel` resident on one SM at kThreads threads (queried once).
template <typename Kern>
unsigned resident_blocks(Kern kernel, std::atomic<int> &cache) {
    int b = cache.load(std::memory_order_relaxed);
    if (b == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kThreads, 0) != cudaSuccess || b < 1) b = 1;
        cache.store(b, std::memory_order_relaxed);
    }
    return (unsigned)b;
}

// Grids of the per-segment kernels.  The slot kernels loop over the live slots
// (grid-stride) and the warp-cooperative ones take chunks of slots from work
// counters, so they need no more blocks than are resident at once (four waves
// for the slot kernels).  A grid sized for every path launched tens of
// thousands of blocks in the late segments, where few paths are left, and each
// of them only found that it had no work.  wf_cast keeps one thread per path
// and a block per 128 paths: its rays differ most in cost, and a grid-stride
// loop (more registers spilled around the traversal) took 1.03 ms per
// 1920x1080 frame with one resident wave and 0.97 with four, against 0.87.
constexpr unsigned kSlotWaves = 4;

// Every launch of one frame, in stream order, with no host synchronisation.
cudaError_t enqueue_frame(const WfParams &W, const RenderParams &P, uint32_t paths, cudaStream_t s,
                          KernelTimer *timer) {
    const unsigned grid = (paths + kThreads - 1) / kThreads;
    static std::atomic<int> occ[5] = {{0}, {0}, {0}, {0}, {0}};   // resident blocks per SM, queried once
    const unsigned g_cast = grid;
    const unsigned g_shade = std::min(grid, kSlotWaves * 152u * resident_blocks(wf_shade, occ[0]));
    const unsigned g_over = std::min(grid, kSlotWaves * 152u * resident_blocks(wf_overflow, occ[1]));
    const unsigned g_gen = std::min(grid, 152u * resident_blocks(wf_gen, occ[2]));
    const unsigned g_mask = std::min(grid, 152u * resident_blocks(wf_mask, occ[3]));
    const unsigned g_comp = std::min(grid, 152u * resident_blocks(wf_composite, occ[4]));
    const FieldDev &F = P.F;
    const bool tc = F.kind == MRF_FIELD_HASHGRID && F.precision != MRF_PREC_FP32;
    const int groups = P.tc_groups == 4 || P.tc_groups == 5 ? P.tc_groups : 8;
    const int field_grid = tc ? 152 * field_tc_blocks_per_sm(groups) : 152 * 8;
    const int rounds = std::min(std::max(P.max_rounds, 1), kMaxRounds);
    // counters left over from the previous call
    cudaError_t e = cudaMemsetAsync(W.ctr, 0, 4 * kCtrWords, s);
    if (e != cudaSuccess) return e;
    // NVTX ranges mark the host-side enqueue of the frame and of each segment
    struct Range {
        explicit Range(const char *n) { nvtxRangePushA(n); }
        ~Range() { nvtxRangePop(); }
    } frame_range("mrf wavefront frame");
    for (uint32_t j = 1; j <= P.max_bounces; ++j) {
        const int cur = (j - 1) & 1, nxt = j & 1;
        Range seg_range("mrf segment");
        if ((e = cudaMemsetAsync(W.ctr + 2, 0, 4 * (2 + 4 * rounds), s)) != cudaSuccess) return e;
        timer_begin(timer, MRF_KERNEL_CAST_GEN, s);
        wf_cast<<<g_cast, kThreads, 0, s>>>(W, j, cur);
        timer_end(timer, s);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (P.n_shadow > 1) {
            const uint64_t rays = (uint64_t)paths * (uint64_t)P.n_shadow;
            const unsigned vgrid = (unsigned)std::min<uint64_t>((rays + kThreads - 1) / kThreads, 152u * 16u);
            timer_begin(timer, MRF_KERNEL_SHADOW_VIS, s);
            wf_vis<<<vgrid, kThreads, 0, s>>>(W, cur);
            timer_end(timer, s);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        if (P.has_snet) {
            timer_begin(timer, MRF_KERNEL_SHADOW_NET, s);
            if (P.snet.lp)   // BF16 network: tensor cores
                e = launch_snet_tc(P.snet, P.snet.lp, P.snet.mlp, W.squeue, W.hp, W.sdir, P.n_shadow, nullptr,
                                   W.ctr + 3, paths * (uint32_t)P.n_shadow, W.sdepth, P.status, P.stats, s);
            else {
                wf_shadow_net<<<152 * 4, 128, 0, s>>>(W);
                e = cudaGetLastError();
            }
            timer_end(timer, s);
            if (e != cudaSuccess) return e;
        }
        // generation rounds: each evaluates and composites what fits the sample
        // buffer; slots left over wait for the next round (the last leftovers
        // are marched in place by wf_overflow)
        for (int r = 0; r < rounds; ++r) {
            if (r > 0 && (e = cudaMemsetAsync(W.ctr + 2, 0, 4, s)) != cudaSuccess) return e;
            timer_begin(timer, MRF_KERNEL_GEN, s);
            wf_gen<<<g_gen, kThreads, 0, s>>>(W, j, cur, r);
            timer_end(timer, s);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            timer_begin(timer, MRF_KERNEL_FIELD, s);
            if (tc && F.view_dep)
                e = launch_field_tc_view(F, F.precision == MRF_PREC_BF16, reinterpret_cast<const float *>(W.samp), 4,
                                         W.sview, W.ctr + 2, W.cap, W.fout, P.status, field_grid, s, groups);
            else if (tc)
                e = launch_field_tc(F, F.precision == MRF_PREC_BF16, reinterpret_cast<const float *>(W.samp), 4,
                                    W.ctr + 2, W.cap, W.fout, P.status, field_grid, s, groups);
            else
                e = launch_field_simt(F, reinterpret_cast<const float *>(W.samp), 4, W.ctr + 2, W.cap, W.fout,
                                      field_grid, s, F.view_dep ? W.sview : nullptr);
            timer_end(timer, s);
            if (e != cudaSuccess) return e;
            if (P.shadow_mask) {
                timer_begin(timer, MRF_KERNEL_MASK, s);
                wf_mask<<<g_mask, kThreads, 0, s>>>(W, cur, r);
                timer_end(timer, s);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
            }
            timer_begin(timer, MRF_KERNEL_COMPOSITE, s);
            wf_composite<<<g_comp, kThreads, 0, s>>>(W, cur, r);
            timer_end(timer, s);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        if ((e = cudaMemsetAsync(W.ctr + nxt, 0, 4, s)) != cudaSuccess) return e;
        timer_begin(timer, MRF_KERNEL_OVERFLOW, s);
        wf_overflow<<<g_over, kThreads, 0, s>>>(W, cur, rounds - 1);
        timer_end(timer, s);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        timer_begin(timer, MRF_KERNEL_SHADE, s);
        wf_shade<<<g_shade, kThreads, 0, s>>>(W, j, cur, nxt);
        timer_end(timer, s);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (P.tail_paths > 0 && P.max_bounces > 1) {
        // the persistent tail: one launch, as many blocks as are resident at once
        const size_t tsmem = F.kind == MRF_FIELD_HASHGRID ? (size_t)field_mlp_floats(F) * sizeof(float) : 0;
        static int tail_blocks_per_sm[2] = {0, 0};   // [0]: no dynamic shared memory, [1]: with
        int &bps = tail_blocks_per_sm[tsmem ? 1 : 0];
        if (tsmem > 48 * 1024 &&
            (e = cudaFuncSetAttribute(wf_tail, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem)) != cudaSuccess)
            return e;
        if (bps == 0 &&
            (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, wf_tail, 32 * kTailWarps, tsmem)) != cudaSuccess)
            return e;
        timer_begin(timer, MRF_KERNEL_TAIL, s);
        wf_tail<<<152 * std::max(bps, 1), 32 * kTailWarps, tsmem, s>>>(W);
        timer_end(timer, s);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    timer_begin(timer, MRF_KERNEL_FINALIZE, s);
    wf_finalize<<<(P.count + kThreads - 1) / kThreads, kThreads, 0, s>>>(W.acc, P.count, P.spp,
                                                                          reinterpret_cast<float4 *>(P.out));
    timer_end(timer, s);
    return cudaGetLastError();
}

}  // namespace

bool wavefront_available() { return true; }

size_t wavefront_scratch_bytes(const RenderParams &P) {
    return layout(P.count * P.spp, P.n_shadow, P.cap_per_path, P.F.view_dep != 0).total;
}

cudaError_t launch_render_wavefront(const RenderParams &P, void *scratch, size_t scratch_bytes, cudaStream_t s,
                                    KernelTimer *timer) {
    const uint32_t paths = P.count * P.spp;
    const Layout Lo = layout(paths, P.n_shadow, P.cap_per_path, P.F.view_dep != 0);
    if (scratch_bytes < Lo.total) return cudaErrorInvalidValue;
    char *b = static_cast<char *>(scratch);
    WfParams W{};
    W.R = P;
    W.paths = paths;
    W.acc = reinterpret_cast<float4 *>(b + Lo.acc);
    for (int q = 0; q < 2; ++q) {
        W.qpath[q] = reinterpret_cast<uint32_t *>(b + Lo.qpath[q]);
        W.qo[q] = reinterpret_cast<float4 *>(b + Lo.qo[q]);
        W.qd[q] = reinterpret_cast<float4 *>(b + Lo.qd[q]);
        W.qT[q] = reinterpret_cast<float4 *>(b + Lo.qT[q]);
    }
    W.hit_t = reinterpret_cast<float *>(b + Lo.hit_t);
    W.hit_slot = reinterpret_cast<int *>(b + Lo.hit_slot);
    W.hit_id = reinterpret_cast<uint32_t *>(b + Lo.hit_id);
    W.rstart = reinterpret_cast<uint32_t *>(b + Lo.rstart);
    W.rcount = reinterpret_cast<uint32_t *>(b + Lo.rcount);
    W.sstart = reinterpret_cast<uint32_t *>(b + Lo.sstart);
    W.scount = reinterpret_cast<uint32_t *>(b + Lo.scount);
    W.sw = reinterpret_cast<float4 *>(b + Lo.sw);
    W.hp = reinterpret_cast<float4 *>(b + Lo.hp);
    W.sdir = reinterpret_cast<float4 *>(b + Lo.sdir);
    W.comp = reinterpret_cast<float4 *>(b + Lo.comp);
    W.sdepth = reinterpret_cast<float *>(b + Lo.sdepth);
    W.ctr = reinterpret_cast<uint32_t *>(b + Lo.ctr);
    W.squeue = reinterpret_cast<uint32_t *>(b + Lo.squeue);
    W.samp = reinterpret_cast<float4 *>(b + Lo.samp);
    W.fout = reinterpret_cast<float4 *>(b + Lo.fout);
    W.sview = Lo.sview ? reinterpret_cast<float4 *>(b + Lo.sview) : nullptr;
    W.cap = Lo.cap;
    return enqueue_frame(W, P, paths, s, timer);
}

// ---------------------------------------------------------------------------
// Allocation-free variant.  Some embedders cannot call cudaMalloc while they
// render: hosts whose device memory is owned by another allocator's pool, and
// real-time loops that cannot afford the device-wide synchronisation an
// allocation may cause.  For them the wavefront engine can run out of this
// file-scope arena instead of library-allocated scratch.  Every GPU that loads
// the library holds the arena until the process exits.  All calls share it and
// it keeps the last call's contents; the engine clears what must start at zero
// (its queue and sample counters), and calls that overlap on the GPU race.
constexpr size_t kStaticArenaBytes = (size_t)64 << 20;   // 64 MiB
constexpr uint32_t kStaticMaxPaths = 1u << 17;           // count * spp limit
constexpr int kStaticMaxLights = 8;   // shadow rays per diffuse hit
constexpr size_t kStaticMinSampleBytes = 2 * 16 * 128 + 512;   // one 128-sample tile in and out, plus slack
static __device__ __align__(256) unsigned char g_static_arena[kStaticArenaBytes];

namespace {
// per-path state of the wavefront engine plus a sample buffer filling the rest
Layout layout_in(uint32_t paths, int n_shadow, size_t bytes, bool &fits) {
    Layout L = layout(paths, n_shadow);
    const size_t state = L.samp;   // everything before the sample buffers
    fits = bytes > state + kStaticMinSampleBytes;
    if (!fits) return L;
    const uint64_t cap = std::min<uint64_t>((bytes - state - 512) / 32, 0x7FFFFFFFull);
    L.cap = (uint32_t)cap;
    L.fout = L.samp + ((16 * cap + 255) & ~(size_t)255);
    L.total = L.fout + 16 * cap;
    fits = L.total <= bytes;
    return L;
}
}  // namespace

uint32_t static_arena_max_paths() { return kStaticMaxPaths; }
int static_arena_max_lights() { return kStaticMaxLights; }

// Largest path count whose per-path state, with n_shadow shadow rays per hit,
// leaves the arena a sample buffer of at least one tile (at most the fixed
// path limit).  The state grows by about 172 + 48 * max(n_shadow, 1) bytes per path.
uint32_t static_arena_paths_that_fit(int n_shadow) {
    uint32_t lo = 0, hi = kStaticMaxPaths;
    while (lo < hi) {
        const uint32_t mid = lo + (hi - lo + 1) / 2;
        bool fits = false;
        layout_in(mid, n_shadow, kStaticArenaBytes, fits);
        if (fits) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Device address of the arena on the current device.  The host-side name
// g_static_arena is only a stand-in for the symbol, so host code must not pass
// it to a kernel; cudaGetSymbolAddress gives the device address.  Called once
// per context, at its creation, with the context's device current.
cudaError_t static_arena(void **ptr, size_t *bytes) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_arena);
    if (e != cudaSuccess) return e;
    *ptr = p;
    *bytes = kStaticArenaBytes;
    return cudaSuccess;
}

// The wavefront launch sequence on a caller-given arena (sample capacity from
// what the arena leaves after the per-path state; jobs beyond it are marched in
// place by wf_shade).
cudaError_t launch_render_wavefront_arena(const RenderParams &P, void *arena, size_t arena_bytes, cudaStream_t s) {
    const uint32_t paths = P.count * P.spp;
    bool fits = false;
    const Layout Lo = layout_in(paths, P.n_shadow, arena_bytes, fits);
    if (!fits) return cudaErrorInvalidValue;
    char *b = static_cast<char *>(arena);
    WfParams W{};
    W.R = P;
    W.paths = paths;
    W.acc = reinterpret_cast<float4 *>(b + Lo.acc);
    for (int q = 0; q < 2; ++q) {
        W.qpath[q] = reinterpret_cast<uint32_t *>(b + Lo.qpath[q]);
        W.qo[q] = reinterpret_cast<float4 *>(b + Lo.qo[q]);
        W.qd[q] = reinterpret_cast<float4 *>(b + Lo.qd[q]);
        W.qT[q] = reinterpret_cast<float4 *>(b + Lo.qT[q]);
    }
    W.hit_t = reinterpret_cast<float *>(b + Lo.hit_t);
    W.hit_slot = reinterpret_cast<int *>(b + Lo.hit_slot);
    W.hit_id = reinterpret_cast<uint32_t *>(b + Lo.hit_id);
    W.rstart = reinterpret_cast<uint32_t *>(b + Lo.rstart);
    W.rcount = reinterpret_cast<uint32_t *>(b + Lo.rcount);
    W.sstart = reinterpret_cast<uint32_t *>(b + Lo.sstart);
    W.scount = reinterpret_cast<uint32_t *>(b + Lo.scount);
    W.sw = reinterpret_cast<float4 *>(b + Lo.sw);
    W.hp = reinterpret_cast<float4 *>(b + Lo.hp);
    W.sdir = reinterpret_cast<float4 *>(b + Lo.sdir);
    W.comp = reinterpret_cast<float4 *>(b + Lo.comp);
    W.sdepth = reinterpret_cast<float *>(b + Lo.sdepth);
    W.ctr = reinterpret_cast<uint32_t *>(b + Lo.ctr);
    W.squeue = reinterpret_cast<uint32_t *>(b + Lo.squeue);
    W.samp = reinterpret_cast<float4 *>(b + Lo.samp);
    W.fout = reinterpret_cast<float4 *>(b + Lo.fout);
    W.cap = Lo.cap;
    return enqueue_frame(W, P, paths, s, nullptr);
}

}  // namespace mrf
