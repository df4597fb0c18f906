"""Closed-form pins of the oracle's march, compositing and whole paths
(Eqs. 10-13 and Algorithm 1 of the paper)."""
import math

import numpy as np
import pytest

from paper_2309_04581_gb300 import scenes as S


def F(v):
    """The FP32 value the scene stores for v (scenes hold FP32 geometry)."""
    return np.float64(np.float32(v))


def _const_scene(sigma, rgb, **opts):
    sc = S.config1()
    sc.field = S.const_field(sigma, rgb)
    sc.mesh = S.empty_mesh()
    sc.materials = []
    for k, v in opts.items():
        setattr(sc.opts, k, v)
    return sc


@pytest.mark.parametrize("mode", ["steps", "dt"])
def test_homogeneous_slab(orc, mode):
    # T = exp(-sigma l), L = e (1 - exp(-sigma l)) exactly, for any step rule
    sigma, e = 3.7, np.array([0.5, 1.25, 2.0])
    sc = _const_scene(sigma, e, steps_per_segment=128 if mode == "steps" else 0, dt=0.0137)
    osc = orc.OracleScene(sc)
    o, d = np.array([0.1, -0.2, 0.9]), np.array([0.0, 0.0, -1.0])
    T, L = orc.march(osc, o, d, 0.0, math.inf)
    l = 1.0   # box z from 0.5 to -0.5
    assert np.allclose(T, math.exp(-sigma * l), rtol=1e-13)
    assert np.allclose(L, e * (1 - math.exp(-sigma * l)), rtol=1e-13)
    # oblique ray, segment cut by a hit at t = 0.7 (ragged last interval)
    d2 = np.array([0.3, 0.4, -0.866])
    d2 /= np.linalg.norm(d2)
    T, L = orc.march(osc, o, d2, 0.0, 0.7)
    ok, t0, t1 = orc.box_interval(osc, o, d2)
    lseg = min(0.7, t1) - max(0.0, t0)
    assert np.allclose(T, math.exp(-sigma * lseg), rtol=1e-13)
    assert np.allclose(L, e * (1 - math.exp(-sigma * lseg)), rtol=1e-12)


def test_throughput_carries_into_segment(orc):
    # T(t) = T(p_j) exp(-int sigma): an incoming throughput scales the segment's radiance
    sc = _const_scene(2.0, [1, 1, 1], steps_per_segment=16)
    osc = orc.OracleScene(sc)
    Tin = np.array([0.5, 0.25, 1.0])
    T, L = orc.march(osc, [0, 0, 0.9], [0, 0, -1], 0.0, math.inf, T=Tin, L=[0.1, 0.2, 0.3])
    q = math.exp(-2.0)
    assert np.allclose(T, Tin * q, rtol=1e-13)
    assert np.allclose(L, np.array([0.1, 0.2, 0.3]) + Tin * (1 - q), rtol=1e-13)


def _single_blob(center, r, peak=50.0, emission=(1.0, 1.0, 1.0)):
    sc = S.config1()
    sc.field = S.gauss_field([center], [r], [peak], [emission])
    sc.mesh = S.empty_mesh()
    sc.materials = []
    return sc


def _gauss_depth_closed_form(peak, r, dperp2, s0, s1):
    # int_{s0}^{s1} peak exp(-(dperp^2 + s^2) / (2 r^2)) ds via erf
    k = r * math.sqrt(2.0)
    return peak * math.exp(-dperp2 / (2 * r * r)) * r * math.sqrt(math.pi / 2) * (
        math.erf(s1 / k) - math.erf(s0 / k))


def test_single_gaussian_midpoint_rule_within_error_bound(orc):
    # The ray starts at the blob's inflection point and runs 0.35 through it.
    # The 128-sample midpoint rule must agree with the erf closed form within
    # the midpoint bound (b - a) h^2 / 24 max|f''|; a left-endpoint rule misses
    # that bound, so a half-step shift of the samples fails this test.
    r, peak = 0.1, 50.0
    c = np.array([0.0, 0.05, 0.0])
    sc = _single_blob(c, r, peak)
    sc.opts.steps_per_segment = 128
    osc = orc.OracleScene(sc)
    o = c + np.array([0.0, 0.0, r])       # distance r from the centre along the ray axis
    d = np.array([0.0, 0.0, -1.0])
    a, b = 0.0, 0.35
    T = orc.transmittance(osc, o, d, a, b)
    # the ray passes through the centre: s measured from the centre, s = t - r
    exact = _gauss_depth_closed_form(peak, r, 0.0, a - r, b - r)
    h = (b - a) / 128
    f2max = peak / r ** 2          # max |d^2/ds^2 peak exp(-s^2/2r^2)| = peak / r^2 at s = 0
    bound = (b - a) * h * h / 24 * f2max
    assert abs(-math.log(T) - exact) <= bound
    # the discriminating check: a left-endpoint rule is off by more than the bound
    ts = a + h * np.arange(128)
    left = sum(peak * math.exp(-((t - r) ** 2) / (2 * r * r)) * h for t in ts)
    assert abs(left - exact) > 3 * bound


def test_constant_colour_telescopes(orc):
    # For any sigma profile with constant radiance e: L = e (1 - T_final)
    e = np.array([2.0, 0.5, 1.5])
    sc = _single_blob([0.05, -0.02, 0.01], 0.12, 40.0, e)
    sc.opts.steps_per_segment = 77
    osc = orc.OracleScene(sc)
    T, L = orc.march(osc, [0.0, 0.0, 0.8], [0.05, -0.03, -1.0], 0.0, math.inf)
    assert np.allclose(L, e * (1 - T), rtol=1e-13)


def test_mirror_box_geometric_series(orc):
    # Camera inside a closed mirror box (inner half-width 0.4, reflectance rho)
    # filled with a homogeneous field: the ray runs along z, so segment 1 has
    # length a = 0.4 - z0 and every later one W = 0.8.  After k segments
    #   L = e (1 - q_a) + e (1 - q) rho q_a sum_{i<k-1} (rho q)^i,  T = q_a rho^(k-1) q^(k-1).
    sigma, rho = 1.3, 0.9
    e = np.array([1.0, 2.0, 0.5])
    sc = _const_scene(sigma, e, steps_per_segment=64)
    sc.mesh = S.box_mesh([0, 0, 0], 0.4, 0, inward=True)
    sc.materials = [S.Material(S.MAT_MIRROR, (rho, rho, rho))]
    z0 = 0.1
    for k in (1, 2, 5, 9):
        sc.opts.max_bounces = k
        sck = S.explicit_rays(sc, [[0.11, 0.137, z0]], [[0.0, 0.0, 1.0]])
        res = orc.render(sck)
        w = F(0.4)
        qa, q = math.exp(-F(sigma) * (w - F(z0))), math.exp(-F(sigma) * 2 * w)
        r = F(rho)
        L = e * (1 - qa) + e * (1 - q) * r * qa * sum((r * q) ** i for i in range(k - 1))
        assert np.allclose(res["rgba"][0, :3], L, rtol=1e-12)
        assert res["segments"][0, 0] == k
        assert res["flags"][0] == 0
        # hits alternate between the z+ and z- walls
        tri = res["tri"][0, 0, :k]
        walls = [int(t) // 2 for t in tri]
        assert walls == [1 if j % 2 == 0 else 0 for j in range(k)]


def _floor_scene(sigma=0.0, occluder=False, albedo=0.5, I=2.0):
    sc = _const_scene(sigma, [0.0, 0.0, 0.0], steps_per_segment=0, dt=0.01)
    meshes = [S.quad_mesh([-0.5, -0.45, -0.5], [-0.5, -0.45, 0.5], [0.5, -0.45, 0.5], [0.5, -0.45, -0.5], 0)]
    if occluder:
        meshes.append(S.quad_mesh([-0.4, 0.1, -0.15], [-0.4, 0.1, 0.15], [-0.1, 0.1, 0.15], [-0.1, 0.1, -0.15], 0))
    sc.mesh = S.merge_meshes(meshes)
    sc.materials = [S.Material(S.MAT_DIFFUSE, (albedo, albedo, albedo))]
    sc.lights = [S.Light(pos=(0.0, 0.45, 0.0), intensity=(I, I, I))]
    sc.opts.max_bounces = 1
    return sc


def test_shadow_ray_point_light_closed_form(orc):
    # Camera ray straight down onto a Lambertian floor, one segment: the only
    # radiance is the next-event term (albedo/pi) cos I / D^2 * V * exp(-sigma l).
    x, z = 0.13, -0.07
    p = np.array([F(x), F(-0.45), F(z)])
    lp = np.array([0.0, F(0.45), 0.0])
    D = np.linalg.norm(lp - p)
    cos = (lp - p)[1] / D
    for sigma in (0.0, 0.8):
        sc = S.explicit_rays(_floor_scene(sigma), [[x, 0.3, z]], [[0, -1, 0]])
        res = orc.render(sc)
        # field transmittance along the camera segment (0.3 -> -0.45 inside the box)
        t_cam = math.exp(-F(sigma) * (F(0.3) - F(-0.45)))
        # the shadow ray runs from the floor to the light; the box ends at y = 0.5 > 0.45
        expect = t_cam * 0.5 / math.pi * cos * 2.0 / D ** 2 * math.exp(-F(sigma) * D)
        assert np.allclose(res["rgba"][0, :3], expect, rtol=1e-12)
        assert res["counts"]["shadow_rays"] == 1
    # an occluder (x in [-0.4, -0.1], y = 0.1) between floor and light blocks the term
    sc = S.explicit_rays(_floor_scene(0.0, occluder=True), [[0.3, 0.3, 0.0]], [[0, -1, 0]])
    assert orc.render(sc)["rgba"][0, :3].max() > 0    # shadow ray passes x = 0.117 at y = 0.1
    d = np.array([0.0, -0.15, -0.3])
    sc = S.explicit_rays(_floor_scene(0.0, occluder=True), [[-0.35, -0.3, 0.3]], [d])
    res = orc.render(sc)
    hitp = np.array([-0.35, -0.3, 0.3]) + res["t"][0, 0, 0] * d / np.linalg.norm(d)
    assert np.allclose(hitp, [-0.35, -0.45, 0.0], atol=1e-7)
    assert np.all(res["rgba"][0, :3] == 0.0)          # shadow ray passes x = -0.136 at y = 0.1


def test_glass_plate_normal_incidence(orc):
    # A glass plate (two inward-facing quads) hit at normal incidence: with the
    # Fresnel draw above F = 0.04 both times, the ray passes straight through
    # with its throughput unchanged, so L equals the slab closed form for the
    # whole box length.  The draw comes from numpy's Philox (the same stream).
    sigma, e = 0.9, np.array([1.0, 0.5, 0.25])
    sc = _const_scene(sigma, e, steps_per_segment=32)
    plate = S.merge_meshes([
        S.quad_mesh([-0.5, -0.5, 0.1], [0.5, -0.5, 0.1], [0.5, 0.5, 0.1], [-0.5, 0.5, 0.1], 0),
        S.quad_mesh([-0.5, -0.5, -0.1], [-0.5, 0.5, -0.1], [0.5, 0.5, -0.1], [0.5, -0.5, -0.1], 0)])
    sc.mesh = plate
    sc.materials = [S.Material(S.MAT_GLASS, ior=1.5)]
    sc.opts.max_bounces = 3
    xs = [[0.1 + 0.01 * i, 0.23, 0.7] for i in range(12)]
    scr = S.explicit_rays(sc, xs, [[0, 0, -1]] * len(xs))
    res = orc.render(scr)
    from tests.test_oracle_units import _numpy_philox_block
    n_checked = 0
    for i in range(len(xs)):
        u1 = int(_numpy_philox_block((i, 0, 1, 0), (sc.opts.seed, 0))[0] >> np.uint64(40)) / 2**24
        u2 = int(_numpy_philox_block((i, 0, 2, 0), (sc.opts.seed, 0))[0] >> np.uint64(40)) / 2**24
        if u1 >= 0.04 and u2 >= 0.04:
            n_checked += 1
            assert np.allclose(res["rgba"][i, :3], e * (1 - math.exp(-F(sigma) * 1.0)), rtol=1e-12)
            assert res["segments"][i, 0] == 3
        elif u1 < 0.04:
            # reflected straight back out of the box: two segments of length 0.4
            q = math.exp(-F(sigma) * (0.5 - F(0.1)))
            assert np.allclose(res["rgba"][i, :3], e * (1 - q) + q * e * (1 - q), rtol=1e-12)
    assert n_checked >= 8


def test_every_path_ends_by_one_cause(orc):
    for sc in (S.config1(24, 24), S.config2(24, 24, tau=0.05), S.config2(16, 16, max_bounces=2)):
        c = orc.render(sc)["counts"]
        assert c["ended_miss"] + c["ended_tau"] + c["ended_cap"] == c["paths"]
    c = orc.render(S.config2(16, 16, max_bounces=2))["counts"]
    assert c["ended_cap"] > 0 and c["ended_tau"] == 0


def test_invariants_on_config_scenes(orc):
    for sc, ids in [(S.config1(), None), (S.config2(96, 96), S.strided_pixels(96, 96, 3))]:
        res = orc.render(sc, ids)
        rgb = res["rgba"][:, :3]
        assert np.all(np.isfinite(rgb)) and np.all(rgb >= 0)
        assert np.all((res["rgba"][:, 3] >= 0) & (res["rgba"][:, 3] <= 1))
        assert res["segments"].max() <= sc.opts.max_bounces and res["segments"].min() >= 1
        assert (res["flags"] != 0).mean() < 0.01
        # every recorded hit precedes the segment count; unused slots stay empty
        for i in range(res["segments"].shape[0]):
            k = res["segments"][i, 0]
            assert np.all(res["tri"][i, 0, k:] == orc.NO_HIT)
            assert np.all(res["tri"][i, 0, :k - 1] != orc.NO_HIT)


def test_tonemap_srgb_transfer(orc):
    # psi: clamp(exposure * L, 0, 1) then the sRGB transfer function; pinned by its
    # end points, the continuity of its two branches at 0.0031308 and the inverse
    # transfer function of the same standard
    assert orc.tonemap(0.0) == 0.0 and orc.tonemap(1.0) == pytest.approx(1.0, abs=1e-15)
    assert orc.tonemap(5.0) == pytest.approx(1.0, abs=1e-15) and orc.tonemap(-1.0) == 0.0
    lo, hi = orc.tonemap(0.0031308), orc.tonemap(0.0031308 * (1 + 1e-9))
    assert abs(lo - hi) < 1e-6
    for c in [0.001, 0.01, 0.2, 0.5, 0.9]:
        v = float(orc.tonemap(c))
        lin = v / 12.92 if v <= 0.04045 else ((v + 0.055) / 1.055) ** 2.4
        assert lin == pytest.approx(c, rel=1e-9)
    assert orc.tonemap(0.25, 2.0) == pytest.approx(float(orc.tonemap(0.5)), rel=1e-15)


def test_field_pose_is_a_change_of_frame(orc):
    # Rendering a field moved by a rigid pose T from camera C equals rendering the
    # unmoved field from the camera moved by T^-1 (no meshes: only the field moves).
    base = S.config2(24, 24)
    base.mesh = S.empty_mesh()
    base.materials = []
    T = S.rigid_pose([0.3, 1.0, -0.2], 0.6, [0.05, -0.1, 0.08])
    R, t = T[:, :3].astype(np.float64), T[:, 3].astype(np.float64)
    moved = S.config2(24, 24)
    moved.mesh = S.empty_mesh()
    moved.materials = []
    moved.field.pose = T
    cam = base.camera
    inv = lambda x: R.T @ (np.asarray(x, np.float64) - t)
    base.camera = S.Camera(pos=S.f32(inv(cam.pos)), look_at=S.f32(inv(cam.look_at)),
                           up=S.f32(R.T @ np.asarray(cam.up, np.float64)), vfov_deg=cam.vfov_deg,
                           width=cam.width, height=cam.height)
    a = orc.render(moved)["rgba"]
    b = orc.render(base)["rgba"]
    peak = np.abs(b[:, :3]).max()
    assert peak > 0.05
    assert np.abs(a - b).max() <= 2e-4 * peak + 1e-7
    # and the pose matters: the same camera without the pose sees something else
    moved.field.pose = None
    c = orc.render(moved)["rgba"]
    assert np.abs(a - c).max() > 0.05 * peak


def test_multi_view_batch_is_the_views_one_after_another(orc):
    # Alg. 1 treats every pixel alone: a batch of views (rays numbered view by
    # view) renders each view exactly as that view rendered alone, whenever the
    # paths draw no random numbers (mirror-only scene); view sizes are uneven
    # and include a 1x1 view, so a wrong view offset or stride fails.
    sizes = [(9, 5), (1, 1), (12, 7), (4, 11)]
    views = S.orbit_views(4, sizes, radius=1.4, height=0.25, vfov=40.0)
    batch = S.config1()
    batch.cameras = views
    got = orc.render(batch)
    assert batch.n_rays == sum(w * h for w, h in sizes) and got["rgba"].shape[0] == batch.n_rays
    off = 0
    images = []
    for cam in views:
        one = S.config1()
        one.camera = cam
        ref = orc.render(one)
        n = cam.width * cam.height
        assert np.array_equal(got["rgba"][off:off + n], ref["rgba"])
        assert np.array_equal(got["segments"][off:off + n], ref["segments"])
        images.append(ref["rgba"])
        off += n
    # the views see different things (the test would pass vacuously otherwise)
    assert not np.allclose(images[0][:4], images[2][:4])
    # a sampled id set indexes the same global numbering
    ids = np.array([0, 44, 45, 46, batch.n_rays - 1], np.uint32)
    sub = orc.render(batch, ids)
    assert np.array_equal(sub["rgba"], got["rgba"][ids])


def test_multi_view_random_numbers_follow_the_global_ray_index(orc):
    # with random draws (glass and diffuse), view 0 of a batch starts at ray 0
    # and equals its render alone; a later view draws with its global ray index,
    # so it equals the render alone only where no path drew anything
    sizes = [(10, 10), (10, 10)]
    views = S.orbit_views(2, sizes)
    views[1] = views[0]
    batch = S.config2(10, 10)
    batch.cameras = views
    got = orc.render(batch)
    one = S.config2(10, 10)
    one.camera = views[0]
    ref = orc.render(one)
    assert np.array_equal(got["rgba"][:100], ref["rgba"])
    same = np.all(got["rgba"][100:] == ref["rgba"], axis=1)
    assert not same.all()


def _polygon_irradiance(p, n, verts, Le):
    """Irradiance at p (normal n) from a uniformly emitting polygon of radiance
    Le facing p: Lambert's closed form E = Le/2 |sum_i theta_i (n . unit(R_i x R_i+1))|."""
    R = [np.asarray(v, np.float64) - p for v in verts]
    R = [r / np.linalg.norm(r) for r in R]
    acc = 0.0
    for i in range(len(R)):
        a, b = R[i], R[(i + 1) % len(R)]
        g = np.cross(a, b)
        acc += math.acos(np.clip(a @ b, -1, 1)) * (g @ n) / np.linalg.norm(g)
    return 0.5 * Le * abs(acc)


def _area_floor_scene(verts, Le, samples, spp, grid=16, half=0.3, y0=0.3):
    sc = _floor_scene()
    sc.lights = [S.area_light(*verts, (Le, Le, Le), samples)]
    sc.opts.spp = spp
    xs = (np.arange(grid) + 0.5) / grid * 2 * half - half
    pts = np.array([[x, y0, z] for z in xs for x in xs])
    return S.explicit_rays(sc, pts, np.tile([0.0, -1.0, 0.0], (pts.shape[0], 1))), pts


def test_area_light_estimator_converges_to_lamberts_formula(orc):
    # A triangle light 0.2 above a Lambertian floor (close, so that cos/D^2
    # varies strongly over it): the mean of the next-event estimates is
    # (albedo/pi) E(p) with E from Lambert's polygon formula; a wrong area, a
    # dropped cosine or non-uniform points on the triangle bias the mean.
    verts = [[-0.1, -0.25, -0.1], [0.15, -0.25, -0.05], [0.0, -0.25, 0.15]]   # front side faces -y
    Le = 3.0
    sc, pts = _area_floor_scene(verts, Le, samples=64, spp=16)
    res = orc.render(sc)
    vf = [S.f32(v).astype(np.float64) for v in verts]
    expect = np.array([0.5 / math.pi * _polygon_irradiance(np.array([F(x), F(-0.45), F(z)]), np.array([0, 1.0, 0]),
                                                           vf, F(Le)) for x, _, z in pts])
    got = res["rgba"][:, 0]
    assert np.all(res["rgba"][:, 0] == res["rgba"][:, 1])
    ratio = got / expect
    assert abs(ratio.mean() - 1.0) <= 6e-3, ratio.mean()
    assert np.abs(ratio - 1.0).max() <= 0.12
    assert res["counts"]["shadow_rays"] == pts.shape[0] * 16 * 64


def test_small_area_light_is_a_point_light(orc):
    # A 2e-3 triangle at the point light's position, facing down, with Le A = I
    # at normal emission: its estimate equals the point light's with intensity
    # I cos(theta_y) (a small Lambertian emitter), cos_y = cos_x for a
    # horizontal floor.
    c = np.array([0.0, 0.45, 0.0])
    h = 1e-3
    verts = [c + [-h, 0, -h], c + [h, 0, -h * 0.5], c + [0, 0, h]]
    vf = [S.f32(v).astype(np.float64) for v in verts]
    A = 0.5 * np.linalg.norm(np.cross(vf[1] - vf[0], vf[2] - vf[0]))
    assert np.cross(vf[1] - vf[0], vf[2] - vf[0])[1] < 0
    I = 2.0
    sc_area, pts = _area_floor_scene(verts, I / A, samples=4, spp=1, grid=6)
    sc_point = S.explicit_rays(_floor_scene(I=I), pts, np.tile([0.0, -1.0, 0.0], (pts.shape[0], 1)))
    sc_point.lights = [S.Light(pos=tuple(S.f32(np.mean(vf, axis=0))), intensity=(I, I, I))]
    a = orc.render(sc_area)["rgba"][:, 0]
    b = orc.render(sc_point)["rgba"][:, 0]
    cos_y = np.array([(F(0.45) - F(-0.45)) / np.linalg.norm(np.mean(vf, axis=0) - [F(x), F(-0.45), F(z)])
                      for x, _, z in pts])
    assert np.allclose(a, b * cos_y, rtol=5e-3)


def test_area_light_back_side_and_occluder(orc):
    # the same light turned over (front side up) sends nothing down; an occluder
    # covering the whole light blocks every shadow ray
    verts = [[-0.1, -0.25, -0.1], [0.0, -0.25, 0.15], [0.15, -0.25, -0.05]]
    sc, _ = _area_floor_scene(verts, 3.0, samples=8, spp=1, grid=4, half=0.05)
    res = orc.render(sc)
    assert np.all(res["rgba"][:, :3] == 0.0) and res["counts"]["shadow_rays"] == 0
    verts = [[-0.1, 0.25, -0.1], [0.15, 0.25, -0.05], [0.0, 0.25, 0.15]]
    sc, _ = _area_floor_scene(verts, 3.0, samples=8, spp=1, grid=4, half=0.05, y0=0.0)
    open_ = orc.render(sc)["rgba"][:, 0]
    sc.mesh = S.merge_meshes([sc.mesh, S.quad_mesh([-0.3, 0.1, -0.3], [-0.3, 0.1, 0.3], [0.3, 0.1, 0.3],
                                                   [0.3, 0.1, -0.3], 0)])
    shut = orc.render(sc)["rgba"][:, 0]
    assert open_.min() > 0 and np.all(shut == 0.0)


def test_field_sample_shadow_mask_closed_form(orc):
    # Sec. 3.1's shadow mask: a homogeneous slab seen along +x at y = 0 under a
    # point light at (0, 0.45, 0); an occluder quad (x in [-0.5, 0], y = 0.3)
    # blocks the light for exactly the samples with x < 0 (their shadow rays
    # cross y = 0.3 at x/3).  With mask strength r those samples emit (1 - r) r(p):
    #   L = e [(1 - r)(1 - exp(-sigma/2)) + exp(-sigma/2)(1 - exp(-sigma/2))].
    sigma, e, r = 2.3, np.array([0.4, 1.1, 2.0]), 0.75
    sc = _const_scene(sigma, e, steps_per_segment=128)
    sc.mesh = S.quad_mesh([-0.5, 0.3, -0.3], [-0.5, 0.3, 0.3], [0.0, 0.3, 0.3], [0.0, 0.3, -0.3], 0)
    sc.materials = [S.Material(S.MAT_DIFFUSE, (0.5, 0.5, 0.5))]
    sc.lights = [S.Light(pos=(0.0, 0.45, 0.0), intensity=(1.0, 1.0, 1.0), mask_strength=r)]
    sc.opts.max_bounces = 1
    sc.opts.shadow_mask = True
    sc = S.explicit_rays(sc, [[-0.6, 0.0, 0.0]], [[1.0, 0.0, 0.0]])
    got = orc.render(sc)["rgba"][0, :3]
    s2 = F(sigma) * 0.5
    h = math.exp(-s2)
    rF = F(r)
    expect = S.f32(e).astype(np.float64) * ((1 - rF) * (1 - h) + h * (1 - h))
    assert np.allclose(got, expect, rtol=1e-12)
    # mask off, or strength 0: the plain slab
    sc.opts.shadow_mask = False
    plain = orc.render(sc)["rgba"][0, :3]
    assert np.allclose(plain, S.f32(e).astype(np.float64) * (1 - h * h), rtol=1e-12)


def test_view_dependent_field_pose_uses_the_field_frame(orc):
    # the colour network sees the view direction in the field's own frame: a
    # posed view-dependent field seen from a camera equals the unposed field
    # seen from the inversely moved camera
    T = S.rigid_pose([0.3, 1.0, -0.2], 0.6, [0.05, -0.1, 0.08])
    R, t = T[:, :3].astype(np.float64), T[:, 3].astype(np.float64)
    moved = S.config2_view(24, 24)
    moved.mesh = S.empty_mesh()
    moved.materials = []
    moved.field.pose = T
    base = S.config2_view(24, 24)
    base.mesh = S.empty_mesh()
    base.materials = []
    cam = base.camera
    inv = lambda x: R.T @ (np.asarray(x, np.float64) - t)
    base.camera = S.Camera(pos=S.f32(inv(cam.pos)), look_at=S.f32(inv(cam.look_at)),
                           up=S.f32(R.T @ np.asarray(cam.up, np.float64)), vfov_deg=cam.vfov_deg,
                           width=cam.width, height=cam.height)
    a = orc.render(moved)["rgba"]
    b = orc.render(base)["rgba"]
    peak = np.abs(b[:, :3]).max()
    assert peak > 0.05
    assert np.abs(a - b).max() <= 2e-4 * peak + 1e-7


def _mirror_margin_recurrence(t_first, t_next, n):
    """Edge margins the oracle's FP32 error bounds give the n segments of a ray
    bouncing at normal incidence between two parallel mirrors (base 2e-7;
    camera ray: 2.4e-7 lateral, 4e-7 rad; per mirror bounce +2.4e-7 lateral
    and +4e-7 rad; lateral error grows by t times the angular one)."""
    lat, ang, out = 2.4e-7, 4e-7, []
    for j in range(n):
        t = t_first if j == 0 else t_next
        out.append(2e-7 + lat + t * ang)
        lat, ang = lat + t * ang + 2.4e-7, ang + 4e-7
    return out


@pytest.mark.parametrize("delta,expect", [(5e-6, None), (1e-4, 0)])
def test_edge_margin_grows_along_a_mirror_path(orc, delta, expect):
    # A ray along z between the z+ and z- walls of a mirror box hits both
    # walls at the same point, delta from the diagonal edge of their
    # triangles.  The camera segment is clear of the margin; the first flagged
    # segment is the one whose accumulated FP32 error bound reaches delta, and
    # every hit before it is the wall the closed form names.
    sc = _const_scene(0.0, [0.0, 0.0, 0.0], steps_per_segment=4)
    sc.mesh = S.box_mesh([0, 0, 0], 0.4, 0, inward=True)
    sc.materials = [S.Material(S.MAT_MIRROR, (1.0, 1.0, 1.0))]
    sc.opts.max_bounces = 9
    x0, z0 = np.float32(0.1), np.float32(0.1)
    y0 = np.float32(np.float64(x0) - delta * math.sqrt(2.0))
    d_edge = abs(np.float64(x0) - np.float64(y0)) / math.sqrt(2.0)     # exact distance to the line y = x
    res = orc.render(S.explicit_rays(sc, [[x0, y0, z0]], [[0.0, 0.0, 1.0]]))
    margins = _mirror_margin_recurrence(F(0.4) - np.float64(z0), 2 * F(0.4), 9)
    first = next((j + 1 for j, m in enumerate(margins) if m >= d_edge), 0)
    if expect is None:
        assert 1 < first <= 9
    else:
        assert first == expect
    assert res["first_flag"][0, 0] == first
    k = (first - 1) if first else 9
    walls = [int(t) // 2 for t in res["tri"][0, 0, :k]]
    assert walls == [1 if j % 2 == 0 else 0 for j in range(k)]


def test_fp32_error_bounds_cover_a_float32_mirror_path():
    # The error bounds behind the flags, checked against an actual FP32
    # computation: rays bouncing 16 times inside a rotated mirror box, once in
    # float32 (every operation rounded) and once in float64 from the same FP32
    # start and the same FP32 wall normals.  Every float32 hit point lies
    # within the bound on the hit point's in-plane error.
    rng = np.random.default_rng(3)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    n32 = np.concatenate([q, -q]).astype(np.float32)          # six walls n . x = 0.4, normals pointing out
    n64 = n32.astype(np.float64)
    n64 /= np.linalg.norm(n64, axis=1, keepdims=True)
    n32 = n64.astype(np.float32)
    worst = 0.0
    for _ in range(300):
        o = rng.uniform(-0.25, 0.25, 3).astype(np.float32)
        d = rng.normal(size=3)
        d = (d / np.linalg.norm(d)).astype(np.float32)
        p64, d64, p32, d32 = o.astype(np.float64), d.astype(np.float64), o.copy(), d.copy()
        lat, ang = 2.4e-7, 4e-7
        for _j in range(16):
            den64 = n64 @ d64
            t64 = np.where(den64 > 1e-9, (0.4 - n64 @ p64) / np.where(den64 > 1e-9, den64, 1.0), np.inf)
            k = int(np.argmin(t64))
            den32 = (n32 @ d32).astype(np.float32)
            t32 = np.where(den32 > np.float32(1e-9),
                           (np.float32(0.4) - (n32 @ p32).astype(np.float32)) / np.where(den32 > 0, den32,
                                                                                          np.float32(1)),
                           np.float32(np.inf)).astype(np.float32)
            if int(np.argmin(t32)) != k:
                break                               # near a corner: the walls differ, the path ends here
            cos = max(float(den64[k]), 0.01)
            h64 = p64 + t64[k] * d64
            h32 = (p32 + t32[k] * d32).astype(np.float32)
            bound = (lat + t64[k] * ang) / cos + 2.4e-7
            err = float(np.linalg.norm(h32.astype(np.float64) - h64))
            worst = max(worst, err / bound)
            assert err <= bound, (err, bound)
            lat, ang = lat + t64[k] * ang + 2.4e-7, ang + 4e-7
            d64 = d64 - 2 * (d64 @ n64[k]) * n64[k]
            d64 /= np.linalg.norm(d64)
            r32 = (d32 - np.float32(2) * np.float32(d32 @ n32[k]) * n32[k]).astype(np.float32)
            d32 = (r32 / np.float32(np.linalg.norm(r32))).astype(np.float32)
            p64, p32 = h64, h32
    assert worst > 1e-3    # the bound is not vacuous
