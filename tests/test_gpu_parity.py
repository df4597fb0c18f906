"""CUDA path vs the FP64 oracle, element by element on the same seeded inputs,
through the C ABI.

Tolerances (derived from the FP32 arithmetic of each step):
  - hit triangle ids and segment counts: bit-exact on unflagged pixels, and
    on every pixel the hit ids of the segments before the path's first
    flagged decision (the oracle's first_flag);
  - hit distance: 1e-5 relative to max(t, 1e-2) (coordinates of magnitude
    ~0.5 hold t to ~1e-7 absolute in FP32, so 1e-5 relative is only
    resolvable from t = 1e-2 up);
  - FP32 radiance: 1e-4 relative per pixel, relative to the pixel's largest
    channel, with a floor of 1e-2 x the image peak.  The floor is the FP32
    position error at the fringe of the density support: a sample position
    off by |dp| <= ~5e-7 moves the support s = 1 - |p - c|^2 / r^2 by up to
    2 |dp| / r ~ 1e-5 (r >= 0.1), so a pixel lit by fringe samples carries an
    absolute error up to ~1e-6 x the radiance of the unsupported field,
    about 1e-4 x (1e-2 x the image peak);
  - pixels the oracle flags as ambiguous (a discrete decision within the
    FP32 error bound of its threshold, the bound growing along the path) are
    excluded and must stay below 0.1 % of an image, except in the scenes
    whose own test says why not.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2309_04581_gb300 import scenes as S

pytestmark = pytest.mark.gpu

RTOL_PIX = 1e-4
RTOL_T = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_04581_gb300 import build
    build.build()
    return torch


@pytest.fixture(scope="module")
def M(torch_cuda):
    import paper_2309_04581_gb300.mrf as m
    return m


def _render(M, sc, engine=None, spp=None):
    import torch
    r = M.Renderer(sc)
    rec = r.new_records()
    out, stats = r.render(records=rec, stats=True, engine=engine if engine is not None else M.MRF_ENGINE_AUTO)
    torch.cuda.synchronize()
    res = dict(rgba=out.cpu().numpy().astype(np.float64), stats=stats,
               segments=rec["segments"].cpu().numpy().view(np.uint32).reshape(sc.n_rays, sc.opts.spp),
               tri=rec["tri"].cpu().numpy().view(np.uint32).reshape(sc.n_rays, sc.opts.spp, sc.opts.max_bounces),
               t=rec["t"].cpu().numpy().reshape(sc.n_rays, sc.opts.spp, sc.opts.max_bounces))
    r.close()
    return res


def _trusted(ref):
    """Per path and segment: True where the hit record comes before the path's
    first flagged decision (all segments of paths without one)."""
    ff = ref["first_flag"]
    jj = np.arange(1, ref["tri"].shape[2] + 1)
    return (ff[:, :, None] == 0) | (jj[None, None, :] < ff[:, :, None])


def _compare(gpu, ref, ids=None, rtol=RTOL_PIX, check_records=True, max_flag_frac=1e-3, t_segments=None):
    """Element-wise comparison of a GPU render with the oracle's on the pixels
    `ids`; hit distances are held to RTOL_T on the first `t_segments` segments
    (default: all)."""
    if ids is None:
        ids = np.arange(gpu["rgba"].shape[0])
    g = gpu["rgba"][ids]
    o = ref["rgba"]
    ok = ref["flags"] == 0
    assert (~ok).mean() <= max_flag_frac, f"{(~ok).mean():.4%} ambiguous pixels"
    peak = max(np.abs(o[:, :3]).max(), 1e-30)
    den = np.maximum(np.abs(o[:, :3]).max(1), 1e-2 * peak)
    err = np.abs(g[:, :3] - o[:, :3]).max(1) / den
    worst = int(np.argmax(np.where(ok, err, 0)))
    assert err[ok].max() <= rtol, f"pixel {ids[worst]}: gpu {g[worst]} oracle {o[worst]} rel {err[worst]:.3g}"
    assert np.allclose(g[ok, 3], o[ok, 3], rtol=1e-4, atol=1e-5)
    if check_records:
        seg_g = gpu["segments"][ids]
        assert np.array_equal(seg_g[ok], ref["segments"][ok]), "segment counts differ"
        tri_g = gpu["tri"][ids]
        assert np.array_equal(tri_g[ok], ref["tri"][ok]), "hit triangle ids differ"
        tr = _trusted(ref)
        assert np.array_equal(np.where(tr, tri_g, 0), np.where(tr, ref["tri"], 0)), \
            "hit ids differ before a path's first flagged decision"
        clear = ref["first_flag"] == 0
        assert np.array_equal(seg_g[clear], ref["segments"][clear]), "segment counts differ on unflagged paths"
        tg, to = gpu["t"][ids][ok][:, :, :t_segments], ref["t"][ok][:, :, :t_segments]
        fin = np.isfinite(to)
        assert np.array_equal(np.isfinite(tg), fin)
        assert np.all(np.abs(tg[fin] - to[fin]) <= RTOL_T * np.maximum(to[fin], 1e-2))
    return float(err[ok].max())


# ----------------------------------------------------------------- field
@pytest.mark.parametrize("which", ["const", "gauss", "hash"])
def test_field_query_matches_oracle(M, orc, torch_cuda, which):
    torch = torch_cuda
    sc = {"const": lambda: S.config1(), "gauss": S.config1, "hash": lambda: S.config2(8, 8)}[which]()
    if which == "const":
        sc.field = S.const_field(2.5, [0.25, 1.5, 3.0])
    rng = np.random.default_rng(11)
    if which == "hash":
        # points inside the support spheres (where the network runs) plus uniform ones
        f = sc.field
        k = rng.integers(0, f.support_center.shape[0], 3000)
        pts = f.support_center[k] + rng.uniform(-1, 1, (3000, 3)) * f.support_radius[k, None] * 0.6
        pts = np.concatenate([pts, rng.uniform(-0.5, 0.5, (1000, 3))])
    else:
        pts = rng.uniform(-0.5, 0.5, (4000, 3))
    pts = np.clip(pts, -0.5, 0.5).astype(np.float32)
    osc = orc.OracleScene(sc)
    ref = np.array([[orc.field_eval(osc, p)[0], *orc.field_eval(osc, p)[1]] for p in pts.astype(np.float64)])
    ctx = M.mrf_context_create(0)
    desc, keep = M.field_desc(sc.field)
    fh = M.mrf_field_create(ctx, desc)
    dp = torch.from_numpy(pts).cuda()
    out = torch.empty((pts.shape[0], 4), dtype=torch.float32, device="cuda")
    M.mrf_field_query(ctx, fh, dp.data_ptr(), pts.shape[0], out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    got = out.cpu().numpy().astype(np.float64)
    M.mrf_field_destroy(fh)
    M.mrf_context_destroy(ctx)
    scale = np.abs(ref).max(0)
    assert np.all(np.abs(got - ref) <= 1e-4 * np.abs(ref) + 1e-6 * scale), np.abs(got - ref).max(0)
    if which == "hash":
        assert (ref[:, 0] > 0).sum() > 2000


# ----------------------------------------------------------------- ray casting
def _cast(M, torch, ctx, bvh, o, d, skip=None, tmin=1e-6):
    n = o.shape[0]
    do, dd = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    ds = torch.from_numpy(skip.view(np.int32)).cuda() if skip is not None else None
    ot = torch.empty(n, dtype=torch.float32, device="cuda")
    oi = torch.empty(n, dtype=torch.int32, device="cuda")
    M.mrf_cast(ctx, bvh, do.data_ptr(), dd.data_ptr(), ds.data_ptr() if ds is not None else None, n, tmin,
               ot.data_ptr(), oi.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return ot.cpu().numpy(), oi.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("builder", ["host", "gpu"])
@pytest.mark.parametrize("mesh_name", ["c2", "soup", "tiny", "one"])
def test_bvh_cast_matches_brute_force(M, orc, torch_cuda, mesh_name, builder):
    """Closest hits through the BVH equal the brute-force oracle's, for the
    host SAH tree and for the GPU-rebuilt linear BVH."""
    torch = torch_cuda
    sc = S.config2(8, 8)
    if mesh_name == "soup":
        sc.mesh = S.random_soup(2000, 1)
    elif mesh_name == "tiny":
        sc.mesh = S.random_soup(3, 2)
    elif mesh_name == "one":
        sc.mesh = S.random_soup(1, 3)
    rng = np.random.default_rng(5)
    n = 6000
    o = rng.uniform(-0.6, 0.6, (n, 3)).astype(np.float32)
    tgt = rng.uniform(-0.3, 0.3, (n, 3))
    d = (tgt - o)
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    skip = rng.integers(0, sc.mesh.n_tris, n).astype(np.uint32)
    skip[::3] = 0xFFFFFFFF
    ctx = M.mrf_context_create(0)
    m = sc.mesh
    bvh = M.mrf_bvh_build(ctx, m.verts.ctypes.data, m.verts.shape[0], m.tris.ctypes.data, m.mat.ctypes.data, m.n_tris)
    if builder == "gpu":
        v = np.ascontiguousarray(m.verts)
        M.check(M.lib().mrf_bvh_rebuild(bvh, v.ctypes.data, v.shape[0], None))
    t_g, id_g = _cast(M, torch, ctx, bvh, o, d, skip)
    M.mrf_bvh_destroy(bvh)
    M.mrf_context_destroy(ctx)
    osc = orc.OracleScene(sc)
    flagged = 0
    hits = 0
    for i in range(n):
        tid, t, fl = orc.closest_hit(osc, o[i].astype(np.float64), d[i].astype(np.float64), int(skip[i]))
        if fl:
            flagged += 1
            continue
        assert id_g[i] == tid, (i, id_g[i], tid)
        if tid != orc.NO_HIT:
            hits += 1
            assert abs(t_g[i] - t) <= RTOL_T * max(t, 1e-2), (i, t_g[i], t)
        else:
            assert np.isinf(t_g[i])
    assert flagged <= n * 1e-3
    if mesh_name not in ("tiny", "one"):
        assert hits > n // 10


# ----------------------------------------------------------------- whole paths
def test_config1_full_image(M, orc, torch_cuda):
    sc = S.config1()
    gpu = _render(M, sc)
    ref = orc.render(sc)
    _compare(gpu, ref)
    assert gpu["stats"]["segments"] == int(gpu["segments"].sum())
    assert gpu["stats"]["paths"] == sc.n_rays


def test_occupancy_that_does_not_cover_the_support(M, torch_cuda):
    """Occupancy is an acceleration structure that must cover the density
    support; the library checks the cover when the field is created and lets
    the sample walk skip the grid only then.  With a grid that leaves a slab of
    supported cells empty, the wavefront walk must keep testing it: its image
    then agrees with the megakernel's march (which always tests the grid) and
    differs from the render of the covering grid."""
    import dataclasses
    sc = S.config2(48, 40)
    R = sc.field.occ_res
    i = np.arange(R ** 3, dtype=np.int64)
    clear = ((i % R) >= 56) & ((i % R) < 72)
    bits = sc.field.occ_bits.copy()
    np.bitwise_and.at(bits, i[clear] >> 5, ~(np.uint32(1) << (i[clear] & 31).astype(np.uint32)))
    holes = dataclasses.replace(sc, field=dataclasses.replace(sc.field, occ_bits=bits))
    wf = _render(M, holes, engine=M.MRF_ENGINE_WAVEFRONT)
    mk = _render(M, holes, engine=M.MRF_ENGINE_MEGAKERNEL)
    full = _render(M, sc, engine=M.MRF_ENGINE_WAVEFRONT)
    assert np.abs(wf["rgba"] - full["rgba"]).max() > 1e-2          # the empty slab removes density
    peak = np.abs(mk["rgba"][:, :3]).max()
    assert np.abs(wf["rgba"][:, :3] - mk["rgba"][:, :3]).max() <= 1e-4 * peak
    assert wf["stats"]["samples_evaluated"] == mk["stats"]["samples_evaluated"]


def test_config2_small_full_image(M, orc, torch_cuda):
    sc = S.config2(64, 64)
    gpu = _render(M, sc)
    ref = orc.render(sc)
    _compare(gpu, ref)
    st = gpu["stats"]
    # every path ends by exactly one cause; the causes match the oracle's up to flagged pixels
    assert st["ended_miss"] + st["ended_tau"] + st["ended_cap"] == st["paths"]
    nflag = int((ref["flags"] != 0).sum())
    for k in ("ended_miss", "ended_tau", "ended_cap"):
        assert abs(st[k] - ref["counts"][k]) <= nflag, k
    assert st["bvh_nodes"] >= st["segments"]
    assert st["shadow_rays"] > 0 and st["samples_evaluated"] > 0
    assert st["samples_nominal"] >= st["samples_evaluated"]
    ok = ref["flags"] == 0
    assert abs(st["shadow_rays"] - ref["counts"]["shadow_rays"]) <= (~ok).sum() * sc.opts.max_bounces


def test_traversal_counts_agree_between_engines(M, torch_cuda):
    """The megakernel and the wavefront engine trace the same closest-hit and
    shadow rays with the same FP32 arithmetic, so they visit the same BVH nodes
    and make the same ray-triangle tests; every surface hit needs a test, and a
    visited node holds at most two leaves of at most 4 triangles."""
    sc = S.config2(48, 40)
    a = _render(M, sc, engine=M.MRF_ENGINE_MEGAKERNEL)["stats"]
    b = _render(M, sc, engine=M.MRF_ENGINE_WAVEFRONT)["stats"]
    for k in ("bvh_nodes", "bvh_tri_tests", "segments", "surface_hits", "shadow_rays", "bvh_worst_nodes",
              "bvh_worst_path"):
        assert a[k] == b[k], (k, a[k], b[k])
    assert a["surface_hits"] <= a["bvh_tri_tests"] <= 8 * a["bvh_nodes"]
    assert 1 <= a["bvh_worst_nodes"] <= a["bvh_nodes"] and a["bvh_worst_path"] < a["paths"]


@pytest.mark.parametrize("size", [(800, 800), (1920, 1080)])
def test_config2_full_size_sampled_pixels(M, orc, torch_cuda, size):
    # the benchmark's scene at 800x800 and at the headline's 1920x1080, rendered
    # whole on the GPU (FP32 megakernel); every 16th row and column is
    # recomputed by the oracle
    w, h = size
    sc = S.config2(w, h)
    gpu = _render(M, sc)
    ids = S.strided_pixels(w, h, 16, offset=5)
    ref = orc.render(sc, ids)
    _compare(gpu, ref, ids)


def test_ragged_and_tiny_images(M, orc, torch_cuda):
    for w, h in [(33, 17), (1, 1), (129, 1)]:
        sc = S.config1(w, h)
        _compare(_render(M, sc), orc.render(sc))


def test_spp_and_single_segment_and_no_mesh(M, orc, torch_cuda):
    sc = S.config2(24, 24)
    sc.opts.spp = 3
    _compare(_render(M, sc), orc.render(sc))
    sc = S.config2(24, 24, max_bounces=1)
    _compare(_render(M, sc), orc.render(sc))
    sc = S.config2(24, 24)
    sc.mesh = S.empty_mesh()
    sc.materials = []
    gpu = _render(M, sc)
    _compare(gpu, orc.render(sc))
    assert np.all(gpu["segments"] == 1)


@pytest.mark.parametrize("engine", ["megakernel", "wavefront"])
def test_throughput_threshold(M, orc, torch_cuda, engine):
    # Termination at max(T) < tau: the oracle flags a crossing only where T
    # lies within the FP32 uncertainty of the path's optical depth (which the
    # support's response to FP32 sample positions dominates); that flags
    # fewer than 0.1 % of the pixels, and every other path must stop at the
    # same sample, segment and hit.
    sc = S.config2(48, 48, tau=0.05)
    eng = M.MRF_ENGINE_MEGAKERNEL if engine == "megakernel" else M.MRF_ENGINE_WAVEFRONT
    gpu = _render(M, sc, engine=eng)
    ref = orc.render(sc)
    _compare(gpu, ref)
    assert gpu["stats"]["ended_tau"] > 200          # many paths end at the threshold


def test_mirror_box_series_on_gpu(M, orc, torch_cuda):
    # closed form of the mirror-box series (see the oracle pins), now on the GPU
    sigma, rho, e, z0 = 1.3, 0.9, np.array([1.0, 2.0, 0.5]), 0.1
    sc = S.config1()
    sc.field = S.const_field(sigma, e)
    sc.mesh = S.box_mesh([0, 0, 0], 0.4, 0, inward=True)
    sc.materials = [S.Material(S.MAT_MIRROR, (rho, rho, rho))]
    sc.opts.steps_per_segment = 64
    sc.opts.max_bounces = 9
    xs = [[0.11 + 0.005 * i, 0.137, z0] for i in range(40)]
    scr = S.explicit_rays(sc, xs, [[0, 0, 1]] * 40)
    gpu = _render(M, scr)
    F = lambda v: np.float64(np.float32(v))
    w = F(0.4)
    qa, q = np.exp(-F(sigma) * (w - F(z0))), np.exp(-F(sigma) * 2 * w)
    r = F(rho)
    L = e * (1 - qa) + e * (1 - q) * r * qa * sum((r * q) ** i for i in range(8))
    assert np.allclose(gpu["rgba"][:, :3], L, rtol=1e-5)
    assert np.all(gpu["segments"] == 9)


def test_host_buffers_match_device_buffers(M, orc, torch_cuda):
    torch = torch_cuda
    sc = S.config2(40, 30)
    r = M.Renderer(sc)
    dev, _ = r.render()
    host = torch.empty((sc.n_rays, 4), dtype=torch.float32).pin_memory()
    r.render(out=host)
    assert torch.equal(dev.cpu(), host)
    # explicit rays given in host memory are uploaded by the library
    rng = np.random.default_rng(2)
    o = np.tile(np.array([[0.0, 0.3, 1.6]], np.float32), (500, 1))
    d = rng.normal(size=(500, 3)) * [0.2, 0.2, 1.0] + [0, -0.2, -1]
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    scr = S.explicit_rays(sc, o, d)
    rays = M.mrf_rays()
    rays.origins, rays.dirs, rays.count, rays.spp = o.ctypes.data, d.ctypes.data, 500, 1
    out_h = np.zeros((500, 4), np.float32)
    M.mrf_render(r.ctx, r.field, r.bvh, rays, sc.opts.max_bounces, r.opts_struct(), out_h.ctypes.data, 0)
    ref = orc.render(scr)
    _compare(dict(rgba=out_h.astype(np.float64)), ref, check_records=False)
    r.close()


def test_refit_same_and_moved_vertices(M, orc, torch_cuda):
    torch = torch_cuda
    sc = S.config2(48, 48)
    r = M.Renderer(sc)
    before, _ = r.render()
    v = np.ascontiguousarray(sc.mesh.verts)
    M.mrf_bvh_refit(r.bvh, v.ctypes.data, v.shape[0], torch.cuda.current_stream().cuda_stream)
    same, _ = r.render()
    assert torch.equal(before, same)
    # move the glass sphere and the cube: refit must match the oracle on the moved mesh
    moved = v.copy()
    moved[:, 1] += np.float32(0.05) * np.sin(7.0 * moved[:, 0]).astype(np.float32)
    moved = np.ascontiguousarray(moved.astype(np.float32))
    M.mrf_bvh_refit(r.bvh, moved.ctypes.data, moved.shape[0], torch.cuda.current_stream().cuda_stream)
    rec = r.new_records()
    out, _ = r.render(records=rec)
    torch.cuda.synchronize()
    sc2 = S.config2(48, 48)
    sc2.mesh = S.Mesh(moved, sc.mesh.tris, sc.mesh.mat)
    ref = orc.render(sc2)
    gpu = dict(rgba=out.cpu().numpy().astype(np.float64),
               segments=rec["segments"].cpu().numpy().view(np.uint32).reshape(-1, 1),
               tri=rec["tri"].cpu().numpy().view(np.uint32).reshape(-1, 1, 8),
               t=rec["t"].cpu().numpy().reshape(-1, 1, 8))
    _compare(gpu, ref)
    with pytest.raises(M.MrfError) as ei:
        M.mrf_bvh_refit(r.bvh, moved.ctypes.data, moved.shape[0] - 1, 0)
    assert ei.value.status == M.MRF_ERR_INVALID_ARG
    r.close()


def test_invalid_arguments_on_gpu(M, torch_cuda):
    sc = S.config1(8, 8)
    r = M.Renderer(sc)
    out = np.zeros((64, 4), np.float32)
    opts = r.opts_struct()
    with pytest.raises(M.MrfError) as ei:
        M.mrf_render(r.ctx, r.field, r.bvh, r.rays_struct(), 0, opts, out.ctypes.data)
    assert ei.value.status == M.MRF_ERR_INVALID_ARG
    seg_host = np.zeros(64, np.uint32)
    opts.rec_segments = seg_host.ctypes.data
    with pytest.raises(M.MrfError):
        M.mrf_render(r.ctx, r.field, r.bvh, r.rays_struct(), 4, opts, out.ctypes.data)
    opts = r.opts_struct()
    opts.steps_per_segment, opts.dt = 0, 0.0
    with pytest.raises(M.MrfError):
        M.mrf_render(r.ctx, r.field, r.bvh, r.rays_struct(), 4, opts, out.ctypes.data)
    bad = M.mrf_field_desc()
    bad.kind = 7
    bad.aabb_max[:] = [1, 1, 1]
    with pytest.raises(M.MrfError):
        M.mrf_field_create(r.ctx, bad)
    r.close()


# ----------------------------------------------------------------- tensor-core field
# (sigma relative, radiance absolute); measured on GB300: fp16 6.7e-5 / 4.6e-5, bf16 5.0e-4 / 3.0e-4
TC_TOL = {"fp16": (2e-4, 1e-4), "bf16": (2e-3, 1e-3)}


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("n", [1, 4000, 128 * 1300 + 17])
def test_field_query_tensor_cores(M, orc, torch_cuda, prec, n):
    """tcgen05 MLP (FP16/BF16 operands, FP32 accumulation) vs the FP64 oracle.
    n covers a single sample, a ragged tail and more tiles than resident CTAs."""
    torch = torch_cuda
    sc = S.config2(8, 8)
    f = sc.field
    rng = np.random.default_rng(21)
    k = rng.integers(0, f.support_center.shape[0], n)
    pts = f.support_center[k] + rng.uniform(-1, 1, (n, 3)) * f.support_radius[k, None] * 0.6
    pts = np.clip(pts, -0.5, 0.5).astype(np.float32)
    check = np.arange(n) if n <= 4000 else rng.choice(n, 3000, replace=False)
    osc = orc.OracleScene(sc)
    ref = np.array([[orc.field_eval(osc, p)[0], *orc.field_eval(osc, p)[1]] for p in pts[check].astype(np.float64)])
    ctx = M.mrf_context_create(0)
    desc, keep = M.field_desc(f, {"fp16": M.MRF_PREC_FP16, "bf16": M.MRF_PREC_BF16}[prec])
    fh = M.mrf_field_create(ctx, desc)
    dp = torch.from_numpy(pts).cuda()
    out = torch.full((n, 4), float("nan"), dtype=torch.float32, device="cuda")
    M.mrf_field_query(ctx, fh, dp.data_ptr(), n, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    got = out.cpu().numpy().astype(np.float64)[check]
    M.mrf_field_destroy(fh)
    M.mrf_context_destroy(ctx)
    assert np.all(np.isfinite(got))
    pos = ref[:, 0] > 0
    sig_rel = np.abs(got[pos, 0] - ref[pos, 0]) / ref[pos, 0]
    rgb_abs = np.abs(got[:, 1:] - ref[:, 1:])
    print(f"{prec} n={n}: sigma rel max {sig_rel.max():.3g} mean {sig_rel.mean():.3g}; "
          f"radiance abs max {rgb_abs.max():.3g}")
    assert np.all(got[~pos] == 0)
    assert sig_rel.max() <= TC_TOL[prec][0]
    assert rgb_abs.max() <= TC_TOL[prec][1]


# ----------------------------------------------------------------- wavefront engine
def _psnr(img, ref, ok):
    peak = np.abs(ref[ok, :3]).max()
    mse = np.mean((img[ok, :3] - ref[ok, :3]) ** 2)
    return float("inf") if mse == 0 else 10 * np.log10(peak * peak / mse)


@pytest.mark.parametrize("cfg", ["c1", "c2"])
def test_wavefront_fp32_matches_oracle(M, orc, torch_cuda, cfg):
    sc = S.config1() if cfg == "c1" else S.config2(64, 64)
    gpu = _render(M, sc, engine=M.MRF_ENGINE_WAVEFRONT)
    _compare(gpu, orc.render(sc))


def _render_prec(M, sc, prec, records=True):
    import torch
    r = M.Renderer(sc, precision={"fp16": M.MRF_PREC_FP16, "bf16": M.MRF_PREC_BF16}[prec])
    rec = r.new_records() if records else None
    out, stats = r.render(records=rec, stats=True)
    torch.cuda.synchronize()
    res = dict(rgba=out.cpu().numpy().astype(np.float64), stats=stats)
    if records:
        res.update(segments=rec["segments"].cpu().numpy().view(np.uint32).reshape(sc.n_rays, sc.opts.spp),
                   tri=rec["tri"].cpu().numpy().view(np.uint32).reshape(sc.n_rays, sc.opts.spp, sc.opts.max_bounces),
                   t=rec["t"].cpu().numpy().reshape(sc.n_rays, sc.opts.spp, sc.opts.max_bounces))
    r.close()
    return res


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_wavefront_tensor_core_image_quality(M, orc, torch_cuda, prec):
    """Reduced-precision renders keep every geometric decision of the FP32 path
    (hit ids, segment counts, distances) and reach >= 45 dB PSNR with <= 1e-2
    max absolute error in linear HDR against the FP64 oracle."""
    sc = S.config2(96, 96)
    gpu = _render_prec(M, sc, prec)
    ref = orc.render(sc)
    ok = ref["flags"] == 0
    psnr = _psnr(gpu["rgba"], ref["rgba"], ok)
    maxabs = np.abs(gpu["rgba"][ok, :3] - ref["rgba"][ok, :3]).max()
    print(f"{prec}: PSNR {psnr:.1f} dB, max abs {maxabs:.3g}")
    assert psnr >= 45.0 and maxabs <= 1e-2
    assert np.array_equal(gpu["segments"][ok], ref["segments"][ok])
    assert np.array_equal(gpu["tri"][ok], ref["tri"][ok])


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("size", [(800, 800), (1920, 1080)])
def test_wavefront_tensor_core_full_size_sampled(M, orc, torch_cuda, prec, size):
    # the benchmark's workload in its launch configuration (the 1920x1080 frame
    # is the headline), oracle on every 16th row and column: image error, and
    # the hit ids and segment counts of every sampled path whose course no
    # flagged decision touches
    w, h = size
    sc = S.config2(w, h)
    gpu = _render_prec(M, sc, prec, records=True)
    ids = S.strided_pixels(w, h, 16, offset=3)
    ref = orc.render(sc, ids)
    ok = ref["flags"] == 0
    img = gpu["rgba"][ids]
    psnr = _psnr(img, ref["rgba"], ok)
    maxabs = np.abs(img[ok, :3] - ref["rgba"][ok, :3]).max()
    print(f"{prec} {w}x{h} sampled: PSNR {psnr:.1f} dB, max abs {maxabs:.3g}, {(~ok).mean():.3%} flagged")
    assert psnr >= 45.0 and maxabs <= 1e-2
    assert (~ok).mean() <= 1e-3
    tr = _trusted(ref)
    assert np.array_equal(np.where(tr, gpu["tri"][ids], 0), np.where(tr, ref["tri"], 0))
    clear = ref["first_flag"] == 0
    assert np.array_equal(gpu["segments"][ids][clear], ref["segments"][clear])


# ----------------------------------------------------------------- field pose and tone map
@pytest.mark.parametrize("engine", ["megakernel", "wavefront_fp32", "wavefront_bf16"])
def test_posed_field_matches_oracle(M, orc, torch_cuda, engine):
    """A field moved as a rigid body (Sec. 3.2: queries at t^-1 p) with the
    meshes left in place, through both engines."""
    sc = S.config2(64, 64)
    sc.field.pose = S.rigid_pose([0.2, 1.0, 0.1], 0.5, [0.04, -0.03, 0.06])
    ref = orc.render(sc)
    if engine == "wavefront_bf16":
        gpu = _render_prec(M, sc, "bf16")
        ok = ref["flags"] == 0
        assert _psnr(gpu["rgba"], ref["rgba"], ok) >= 45.0
        assert np.array_equal(gpu["tri"][ok], ref["tri"][ok])
    else:
        eng = M.MRF_ENGINE_MEGAKERNEL if engine == "megakernel" else M.MRF_ENGINE_WAVEFRONT
        _compare(_render(M, sc, engine=eng), ref)


def test_tonemap_matches_oracle(M, orc, torch_cuda):
    torch = torch_cuda
    rng = np.random.default_rng(4)
    hdr = np.concatenate([rng.uniform(-0.1, 1.5, (5000, 4)), [[0.0031308, 0.0, 1.0, 0.5]]]).astype(np.float32)
    ctx = M.mrf_context_create(0)
    din = torch.from_numpy(hdr).cuda()
    out = torch.empty_like(din)
    M.mrf_tonemap(ctx, din.data_ptr(), hdr.shape[0], 1.7, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    got = out.cpu().numpy().astype(np.float64)
    M.mrf_context_destroy(ctx)
    ref = orc.tonemap(hdr[:, :3].astype(np.float64), 1.7)
    assert np.abs(got[:, :3] - ref).max() <= 2e-6
    assert np.array_equal(got[:, 3], hdr[:, 3].astype(np.float64))


# ----------------------------------------------------------------- multi-view batches
@pytest.mark.parametrize("engine", ["megakernel", "wavefront_fp32", "wavefront_bf16"])
def test_multi_view_batch_matches_oracle(M, orc, torch_cuda, engine):
    """Several cameras of uneven sizes (a 1x1 view among them) in one render
    call; rays are numbered view by view, so the oracle renders the same global
    ray indices."""
    sc = S.config2(8, 8)
    sc.cameras = S.orbit_views(5, [(33, 17), (64, 48), (1, 1), (20, 70), (47, 31)])
    ref = orc.render(sc)
    if engine == "wavefront_bf16":
        gpu = _render_prec(M, sc, "bf16")
        ok = ref["flags"] == 0
        assert _psnr(gpu["rgba"], ref["rgba"], ok) >= 45.0
        assert np.array_equal(gpu["tri"][ok], ref["tri"][ok])
        assert np.array_equal(gpu["segments"][ok], ref["segments"][ok])
    else:
        eng = M.MRF_ENGINE_MEGAKERNEL if engine == "megakernel" else M.MRF_ENGINE_WAVEFRONT
        _compare(_render(M, sc, engine=eng), ref)


def test_multi_view_rejections(M, torch_cuda):
    import ctypes as C
    torch = torch_cuda
    sc = S.config2(8, 8)
    sc.cameras = S.orbit_views(3, [(4, 4)])
    r = M.Renderer(sc)
    out = torch.empty((sc.n_rays, 4), dtype=torch.float32, device="cuda")
    rays = r.rays_struct()
    bad = (M.mrf_camera * 3)(*r.views)
    bad[1].width = 0
    rays.camera = C.cast(bad, C.POINTER(M.mrf_camera))
    st = M.lib().mrf_render(r.ctx, r.field, r.bvh, C.byref(rays), 8, C.byref(r.opts_struct()), out.data_ptr(), None,
                            None)
    assert st == M.MRF_ERR_INVALID_ARG and b"camera 1" in M.lib().mrf_last_error()
    st = M.lib().mrf_render_static(r.ctx, r.field, r.bvh, C.byref(r.rays_struct()), 8, C.byref(r.opts_struct()),
                                   out.data_ptr(), None, None)
    assert st == M.MRF_ERR_UNSUPPORTED
    r.close()


# ----------------------------------------------------------------- area lights
@pytest.mark.parametrize("engine", ["megakernel", "wavefront_fp32", "wavefront_bf16"])
def test_area_lights_match_oracle(M, orc, torch_cuda, engine):
    """Four triangle emitters with 16 shadow rays each per diffuse hit (64 in
    all, the wavefront engine's limit); the points on the emitters come from
    the same Philox counters on both sides, so images match pixel by pixel."""
    sc = S.config4(32, 32)
    ref = orc.render(sc)
    if engine == "wavefront_bf16":
        gpu = _render_prec(M, sc, "bf16")
        ok = ref["flags"] == 0
        assert _psnr(gpu["rgba"], ref["rgba"], ok) >= 45.0
        assert np.abs(gpu["rgba"][ok, :3] - ref["rgba"][ok, :3]).max() <= 1e-2
        assert np.array_equal(gpu["tri"][ok], ref["tri"][ok])
    else:
        eng = M.MRF_ENGINE_MEGAKERNEL if engine == "megakernel" else M.MRF_ENGINE_WAVEFRONT
        gpu = _render(M, sc, engine=eng)
        _compare(gpu, ref)
        assert gpu["stats"]["shadow_rays"] == ref["counts"]["shadow_rays"]


def test_area_light_limits(M, torch_cuda):
    import ctypes as C
    torch = torch_cuda
    sc = S.config4(8, 8, samples=17)          # 68 shadow rays per hit > 64
    r = M.Renderer(sc)
    out = torch.empty((sc.n_rays, 4), dtype=torch.float32, device="cuda")
    st = M.lib().mrf_render(r.ctx, r.field, r.bvh, C.byref(r.rays_struct()), 8,
                            C.byref(r.opts_struct(M.MRF_ENGINE_WAVEFRONT)), out.data_ptr(), None, None)
    assert st == M.MRF_ERR_UNSUPPORTED
    st = M.lib().mrf_render_static(r.ctx, r.field, r.bvh, C.byref(r.rays_struct()), 8, C.byref(r.opts_struct()),
                                   out.data_ptr(), None, None)
    assert st == M.MRF_ERR_INVALID_ARG
    bad = (M.mrf_light * 1)()
    bad[0].kind = M.MRF_LIGHT_AREA
    bad[0].samples = 4           # degenerate triangle: all three vertices at the origin
    assert M.lib().mrf_lights_set(r.ctx, bad, 1) == M.MRF_ERR_INVALID_ARG
    bad[0].v1[:] = [1, 0, 0]
    bad[0].v2[:] = [0, 0, 1]
    bad[0].samples = 0
    assert M.lib().mrf_lights_set(r.ctx, bad, 1) == M.MRF_ERR_INVALID_ARG
    r.close()


# ----------------------------------------------------------------- field-sample shadow mask
@pytest.mark.parametrize("engine", ["megakernel", "wavefront_fp32", "wavefront_bf16"])
def test_field_sample_shadow_mask_matches_oracle(M, orc, torch_cuda, engine):
    """Sec. 3.1's shadow mask: every field sample with sigma > 0 casts a ray to
    the light; where a mesh (the mirror cube, the glass sphere) blocks it, the
    sample's radiance is scaled by 1 - r_src."""
    sc = S.config2(48, 48)
    sc.lights = [S.Light(pos=l.pos, intensity=l.intensity, mask_strength=0.8) for l in sc.lights]
    sc.opts.shadow_mask = True
    ref = orc.render(sc)
    plain = S.config2(48, 48)
    assert np.abs(ref["rgba"] - orc.render(plain)["rgba"]).max() > 1e-2   # the mask darkens something
    if engine == "wavefront_bf16":
        gpu = _render_prec(M, sc, "bf16")
        ok = ref["flags"] == 0
        assert _psnr(gpu["rgba"], ref["rgba"], ok) >= 45.0
        assert np.array_equal(gpu["tri"][ok], ref["tri"][ok])
    else:
        eng = M.MRF_ENGINE_MEGAKERNEL if engine == "megakernel" else M.MRF_ENGINE_WAVEFRONT
        # every field sample with sigma > 0 casts a mask ray, hundreds per
        # pixel, each from an FP32 position: about 2 % of the pixels hold one
        # whose error bound reaches a mesh edge (flagged: a decision the FP32
        # ray can take either way).  The mask changes radiance only, so hit
        # ids and segment counts are compared on every unflagged path.
        _compare(_render(M, sc, engine=eng), ref, max_flag_frac=3e-2)


# ----------------------------------------------------------------- view-dependent radiance
@pytest.mark.parametrize("engine", ["megakernel", "wavefront", "wavefront_bf16"])
def test_view_dependent_field_matches_oracle(M, orc, torch_cuda, engine):
    """Instant-NGP network layout: a density head and a colour network of the
    view direction's spherical harmonics (field frame), posed field included;
    BF16 runs the five-MMA tensor-core kernel."""
    sc = S.config2_view(48, 48)
    sc.field.pose = S.rigid_pose([0.2, 1.0, 0.1], 0.4, [0.03, -0.02, 0.05])
    ref = orc.render(sc)
    if engine == "wavefront_bf16":
        gpu = _render_prec(M, sc, "bf16")
        ok = ref["flags"] == 0
        psnr = _psnr(gpu["rgba"], ref["rgba"], ok)
        print(f"view-dependent BF16 tensor cores: PSNR {psnr:.1f} dB")
        assert psnr >= 45.0 and np.abs(gpu["rgba"][ok, :3] - ref["rgba"][ok, :3]).max() <= 1e-2
        assert np.array_equal(gpu["tri"][ok], ref["tri"][ok])
        return
    eng = M.MRF_ENGINE_MEGAKERNEL if engine == "megakernel" else M.MRF_ENGINE_WAVEFRONT
    gpu = _render(M, sc, engine=eng)
    _compare(gpu, ref)
    # the direction matters: the same scene without its colour network's SH inputs differs
    flat = S.config2_view(48, 48)
    flat.field.pose = sc.field.pose
    flat.field.view = dict(flat.field.view, wc1=flat.field.view["wc1"].copy())
    flat.field.view["wc1"][:, 16:] = 0
    assert np.abs(_render(M, flat, engine=eng)["rgba"] - gpu["rgba"]).max() > 1e-3


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_view_dependent_field_query(M, orc, torch_cuda, prec):
    torch = torch_cuda
    sc = S.config2_view(8, 8)
    rng = np.random.default_rng(21)
    pts = rng.uniform(-0.45, 0.45, (5000, 3)).astype(np.float32)
    ctx = M.mrf_context_create(0)
    desc, keep = M.field_desc(sc.field, M.MRF_PREC_BF16 if prec == "bf16" else M.MRF_PREC_FP32)
    f = M.mrf_field_create(ctx, desc)
    dp = torch.from_numpy(pts).cuda()
    out = torch.empty((pts.shape[0], 4), dtype=torch.float32, device="cuda")
    M.mrf_field_query(ctx, f, dp.data_ptr(), pts.shape[0], out.data_ptr())
    got = out.cpu().numpy().astype(np.float64)
    osc = orc.OracleScene(sc)
    ref = np.array([[*orc.field_eval_dir(osc, p.astype(np.float64), [0, 0, 1])[0:1],
                     *orc.field_eval_dir(osc, p.astype(np.float64), [0, 0, 1])[1]] for p in pts])
    assert (ref[:, 0] > 0).sum() > 100
    scale = np.maximum(np.abs(ref).max(0), 1e-6)
    if prec == "fp32":
        assert np.all(np.abs(got - ref) <= 1e-4 * np.abs(ref) + 1e-6 * scale)
    else:   # BF16 operands through five layers: a few 1e-2 relative
        assert np.all(np.abs(got - ref) <= 5e-2 * np.abs(ref) + 5e-3 * scale)
    M.mrf_field_destroy(f)
    M.mrf_context_destroy(ctx)


# ----------------------------------------------------------------- persistent tail
def _render_tuned(M, sc, prec, tail_paths, engine):
    import torch
    r = M.Renderer(sc, precision=prec)
    r.set_tuning(8, 96, 1, tail_paths)
    rec = r.new_records()
    out, stats = r.render(records=rec, stats=True, engine=engine)
    torch.cuda.synchronize()
    res = dict(rgba=out.cpu().numpy().astype(np.float64), stats=stats, img=out.clone(),
               segments=rec["segments"].cpu().numpy().view(np.uint32).reshape(sc.n_rays, sc.opts.spp),
               tri=rec["tri"].cpu().numpy().view(np.uint32).reshape(sc.n_rays, sc.opts.spp, sc.opts.max_bounces),
               t=rec["t"].cpu().numpy().reshape(sc.n_rays, sc.opts.spp, sc.opts.max_bounces))
    r.close()
    return res


@pytest.mark.parametrize("cfg", ["c2", "area", "mask"])
def test_persistent_tail_matches_the_wavefront_and_the_oracle(M, orc, torch_cuda, cfg):
    """The persistent tail (one launch that finishes every path still live,
    a warp per path) takes the wavefront engine's steps: with an FP32 field
    the image, records and statistics equal the per-segment engine's bit for
    bit, and they match the oracle; here it takes over from the second
    segment on."""
    torch = torch_cuda
    if cfg == "c2":
        sc = S.config2(64, 64)
    elif cfg == "area":
        sc = S.config4(32, 32)
    else:
        sc = S.config2(48, 48)
        sc.lights = [S.Light(pos=l.pos, intensity=l.intensity, mask_strength=0.8) for l in sc.lights]
        sc.opts.shadow_mask = True
    W = M.MRF_ENGINE_WAVEFRONT
    plain = _render_tuned(M, sc, M.MRF_PREC_FP32, 0, W)
    tail = _render_tuned(M, sc, M.MRF_PREC_FP32, 1 << 20, W)
    assert torch.equal(tail["img"], plain["img"])
    assert np.array_equal(tail["segments"], plain["segments"]) and np.array_equal(tail["tri"], plain["tri"])
    for k in ("segments", "surface_hits", "shadow_rays", "samples_evaluated", "shadow_samples_evaluated",
              "samples_nominal", "bvh_nodes", "bvh_tri_tests", "ended_miss", "ended_tau", "ended_cap"):
        assert tail["stats"][k] == plain["stats"][k], k
    ref = orc.render(sc)
    _compare(tail, ref, max_flag_frac=3e-2 if cfg == "mask" else 1e-3)
    # the BF16 field through the tail (the tail's samples take the FP32 weights)
    bf = _render_tuned(M, sc, M.MRF_PREC_BF16, 1 << 20, W)
    ok = ref["flags"] == 0
    assert _psnr(bf["rgba"], ref["rgba"], ok) >= 45.0
    assert np.abs(bf["rgba"][ok, :3] - ref["rgba"][ok, :3]).max() <= 1e-2
    assert np.array_equal(bf["tri"][ok], ref["tri"][ok])


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_field_operands_in_tensor_memory_give_the_same_image(M, torch_cuda, prec):
    """field_groups = 5 keeps every layer's A operand in tensor memory (the
    MMAs read A from TMEM) instead of shared memory: the same operands and the
    same accumulation, so the image is the same bit for bit (a ragged frame
    whose last tiles are partial)."""
    torch = torch_cuda
    sc = S.config2(97, 61)
    r = M.Renderer(sc, precision={"fp16": M.MRF_PREC_FP16, "bf16": M.MRF_PREC_BF16}[prec])
    a, st_a = r.render(stats=True)
    a = a.clone()
    r.set_tuning(5, 96, 1)
    b, st_b = r.render(stats=True)
    torch.cuda.synchronize()
    assert st_a["status"] == 0 and st_b["status"] == 0
    assert torch.equal(a, b)
    assert st_a["samples_evaluated"] == st_b["samples_evaluated"]
    r.close()


@pytest.mark.parametrize("n_support", [0, 40, 70])
def test_support_sphere_counts(M, orc, torch_cuda, n_support):
    """Hash fields without a support sphere (support(p) is a max over an empty
    set, so no density anywhere), with more spheres than a warp has lanes (the
    sample walk then tests every sphere at every interval) and with more than
    the shared-memory copy holds: both FP32 engines match the oracle element by
    element, the BF16 wavefront reaches >= 45 dB, and the field queries return
    zero density wherever the support is zero."""
    torch = torch_cuda
    sc = S.config2(48, 48)
    sc.field = S.hash_field(2, n_support=n_support, support_r=(0.05, 0.12))
    ref = orc.render(sc)
    for engine in (M.MRF_ENGINE_MEGAKERNEL, M.MRF_ENGINE_WAVEFRONT):
        gpu = _render(M, sc, engine=engine)
        _compare(gpu, ref)
        if n_support == 0:
            assert gpu["stats"]["samples_evaluated"] == 0
        else:
            assert gpu["stats"]["samples_evaluated"] > 0
    low = _render_prec(M, sc, "bf16")
    ok = ref["flags"] == 0
    assert np.array_equal(low["segments"][ok], ref["segments"][ok])
    diff = np.abs(low["rgba"][ok, :3] - ref["rgba"][ok, :3])
    assert diff.max() <= 1e-2
    if diff.max() > 0:
        assert _psnr(low["rgba"], ref["rgba"], ok) >= 45.0
    # field queries: points spread over the whole box
    rng = np.random.default_rng(5)
    pts = rng.uniform(-0.5, 0.5, (4096, 3)).astype(np.float32)
    osc = orc.OracleScene(sc)
    ref_sig = np.array([orc.field_eval(osc, p)[0] for p in pts.astype(np.float64)])
    ctx = M.mrf_context_create(0)
    for prec in (M.MRF_PREC_FP32, M.MRF_PREC_BF16):
        desc, keep = M.field_desc(sc.field, prec)
        fh = M.mrf_field_create(ctx, desc)
        dp = torch.from_numpy(pts).cuda()
        out = torch.full((len(pts), 4), float("nan"), dtype=torch.float32, device="cuda")
        M.mrf_field_query(ctx, fh, dp.data_ptr(), len(pts), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        sig = out.cpu().numpy()[:, 0]
        M.mrf_field_destroy(fh)
        assert np.all(np.isfinite(sig))
        assert np.all(sig[ref_sig == 0] == 0)
        assert np.all(sig[ref_sig > 0] > 0) or prec != M.MRF_PREC_FP32
    M.mrf_context_destroy(ctx)
