"""Pins of the FP64 oracle's building blocks against things other than itself:
IEEE formats, a library generator, closed-form optics and geometry, library
linear algebra, and exact-arithmetic special cases."""
import math

import numpy as np
import pytest
import torch

from paper_2309_04581_gb300 import scenes as S


# --------------------------------------------------------------- binary16
def test_half_decode_matches_numpy_for_every_pattern(orc):
    bits = np.arange(65536, dtype=np.uint32)
    ref = bits.astype(np.uint16).view(np.float16).astype(np.float64)
    got = np.array([orc.half_to_double(int(b)) for b in bits])
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan], ref[~nan])


# --------------------------------------------------------------- Philox4x64-10
def _numpy_philox_block(ctr, key):
    """numpy's Philox increments its 256-bit counter before each block."""
    c = 0
    for i, w in enumerate(ctr):
        c |= int(w) << (64 * i)
    c = (c - 1) % (1 << 256)
    words = [(c >> (64 * i)) & ((1 << 64) - 1) for i in range(4)]
    bg = np.random.Philox(counter=np.array(words, dtype=np.uint64), key=np.array([int(k) for k in key], dtype=np.uint64))
    return bg.random_raw(4)


@pytest.mark.parametrize("ctr,key", [
    ((1, 0, 0, 0), (0, 0)), ((0, 1, 0, 0), (0, 0)), ((12345, 7, 3, 0), (2, 0)),
    ((2**64 - 1, 2**63, 17, 2**40), (2**64 - 5, 99)), ((640000, 3, 8, 0), (20230908, 0)),
])
def test_philox_matches_numpy(orc, ctr, key):
    assert np.array_equal(orc.philox4x64(ctr, key), _numpy_philox_block(ctr, key))


def test_philox_uniforms_are_uniform(orc):
    # top-24-bit uniforms: mean 1/2, variance 1/12 within 5 sigma over 20k draws
    u = np.array([orc.philox4x64((i, 0, 0, 0), (7, 0))[0] >> np.uint64(40) for i in range(20000)],
                 np.float64) / 2**24
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / u.size)
    assert abs(u.var() - 1 / 12) < 0.01


# --------------------------------------------------------------- camera
def test_pinhole_camera_geometry(orc):
    sc = S.config1(width=33, height=21)
    osc = orc.OracleScene(sc)
    W, H = 33, 21
    fwd = np.array([0, -0.3, -1.6]) / np.linalg.norm([0, -0.3, -1.6])
    o, d = orc.camera_ray(osc, (H // 2) * W + W // 2)
    assert np.allclose(o, [0, 0.3, 1.6])
    assert np.allclose(d, fwd, atol=1e-15)
    # vertical extent: angle between top and bottom pixel-centre rays of the centre column
    _, dt = orc.camera_ray(osc, 0 * W + W // 2)
    _, db = orc.camera_ray(osc, (H - 1) * W + W // 2)
    half = math.radians(45.0) / 2
    expect = 2 * math.atan((1 - 1 / H) * math.tan(half))
    assert math.isclose(math.acos(np.clip(dt @ db, -1, 1)), expect, rel_tol=1e-12)
    # horizontal extent scales with the aspect ratio
    _, dl = orc.camera_ray(osc, (H // 2) * W + 0)
    _, dr = orc.camera_ray(osc, (H // 2) * W + W - 1)
    expect_h = 2 * math.atan((1 - 1 / W) * math.tan(half) * W / H)
    assert math.isclose(math.acos(np.clip(dl @ dr, -1, 1)), expect_h, rel_tol=1e-12)
    # top row leans toward +y, left column toward -x (right-handed, y up)
    assert dt[1] > d[1] and dl[0] < 0 < dr[0]
    for pix in range(0, W * H, 37):
        assert abs(np.linalg.norm(orc.camera_ray(osc, pix)[1]) - 1) < 1e-15


# --------------------------------------------------------------- hash grid
def _table_scene(level_res, log2_T=19, fill=None):
    f = S.hash_field(99, n_support=1, occ_res=32)
    L = len(level_res)
    T = 1 << log2_T
    tab = np.zeros((L, T, 2), np.float16) if fill is None else fill
    f.level_res = np.asarray(level_res, np.uint32)
    f.table = tab
    f.log2_table_size = log2_T
    f.w1 = S.f32(np.zeros((64, 2 * L)))
    sc = S.config1()
    sc.field = f
    return sc


def test_dense_level_reproduces_linear_function_exactly(orc):
    # Trilinear interpolation reproduces any linear function of the vertex
    # coordinates; values are multiples of 2^-10 so FP16 stores them exactly.
    N = 16
    T = 1 << 19
    tab = np.zeros((1, T, 2), np.float16)
    g = np.arange(N + 1)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    idx = (x + (N + 1) * (y + (N + 1) * z)).reshape(-1)
    tab[0, idx, 0] = (x / 64 + y / 128 - z / 256).reshape(-1)
    tab[0, idx, 1] = (2 * z / 64 - x / 128).reshape(-1)
    sc = _table_scene([N], fill=tab)
    osc = orc.OracleScene(sc)
    rng = np.random.default_rng(0)
    for p in rng.uniform(-0.5, 0.5, size=(200, 3)):
        u = (p + 0.5) * N
        feat = orc.hash_encode(osc, p)
        assert abs(feat[0] - (u[0] / 64 + u[1] / 128 - u[2] / 256)) < 1e-14
        assert abs(feat[1] - (2 * u[2] / 64 - u[0] / 128)) < 1e-14


def test_hashed_level_along_x_axis_and_at_vertices(orc):
    # Level 2048 does not fit densely (2049^3 > 2^19) so it is hashed; on the
    # line y = z = 0 of the level grid the hash reduces to x (x * 1 mod T), so a
    # table linear in the index interpolates exactly along that line.
    N, T = 2048, 1 << 19
    tab = np.zeros((1, T, 2), np.float16)
    ix = np.arange(N + 1)
    tab[0, ix, 0] = ix / 4096
    tab[0, ix, 1] = (N - ix) / 4096
    sc = _table_scene([N], fill=tab)
    osc = orc.OracleScene(sc)
    for ux in [0.0, 0.25, 3.5, 1000.125, 2047.75]:
        p = np.array([ux / N - 0.5, -0.5, -0.5])
        feat = orc.hash_encode(osc, p)
        assert abs(feat[0] - ux / 4096) < 1e-12
        assert abs(feat[1] - (N - ux) / 4096) < 1e-12
    # at any grid vertex the encoding is one table entry (no blending)
    rng = np.random.default_rng(1)
    tab2 = rng.uniform(-0.5, 0.5, size=(1, T, 2)).astype(np.float16)
    sc2 = _table_scene([N], fill=tab2)
    osc2 = orc.OracleScene(sc2)
    vals = set(map(tuple, tab2[0].astype(np.float64)))
    for v in rng.integers(0, N, size=(20, 3)):
        feat = orc.hash_encode(osc2, v / N - 0.5)
        assert tuple(feat) in vals


def test_level_resolution_table():
    # N_l = floor(16 * b^l), b = 128^(1/15): 16 levels from 16 to 2048
    assert S.level_resolutions(16, 16, 2048).tolist() == [
        16, 22, 30, 42, 58, 80, 111, 153, 212, 294, 406, 561, 776, 1072, 1482, 2048]


def test_mlp_matches_torch_fp64_chain(orc):
    sc = S.config2(8, 8)
    osc = orc.OracleScene(sc)
    f = sc.field
    rng = np.random.default_rng(3)
    lin = lambda w, b: (torch.tensor(w, dtype=torch.float64), torch.tensor(b, dtype=torch.float64))
    (w1, b1), (w2, b2), (w3, b3) = lin(f.w1, f.b1), lin(f.w2, f.b2), lin(f.w3, f.b3)
    for x in rng.uniform(-1, 1, size=(20, 32)):
        t = torch.tensor(x)
        ref = torch.nn.functional.linear(torch.relu(torch.nn.functional.linear(
            torch.relu(torch.nn.functional.linear(t, w1, b1)), w2, b2)), w3, b3)
        assert np.allclose(orc.mlp(osc, x), ref.numpy(), rtol=0, atol=1e-13)


def test_hash_field_heads(orc):
    # sigma = support * exp(min(o0, 15)); radiance = softplus(o1..3)
    sc = S.config2(8, 8)
    osc = orc.OracleScene(sc)
    c = sc.field.support_center[0].astype(np.float64)
    for p in [c, c + 0.03, c - [0.02, 0.0, 0.05]]:
        o = orc.mlp(osc, orc.hash_encode(osc, p))
        sig, rgb = orc.field_eval(osc, p)
        s = orc.support(osc, p)
        assert s > 0
        assert math.isclose(sig, s * math.exp(min(o[0], 15.0)), rel_tol=1e-14)
        sp = torch.nn.functional.softplus(torch.tensor(o[1:], dtype=torch.float64)).numpy()
        assert np.allclose(rgb, sp, rtol=1e-14)
    # outside every support sphere the density is exactly zero
    far = np.array([0.49, 0.49, 0.49])
    d = np.linalg.norm(sc.field.support_center - far, axis=1)
    assert np.all(d > sc.field.support_radius)
    assert orc.field_eval(osc, far)[0] == 0.0


def test_support_is_covered_by_occupancy(orc):
    # every point with non-zero density lies in an occupied cell, so skipping
    # empty cells never drops a contribution
    sc = S.config2(8, 8)
    osc = orc.OracleScene(sc)
    f = sc.field
    R = f.occ_res
    bits = np.unpackbits(f.occ_bits.view(np.uint8), bitorder="little").astype(bool)
    rng = np.random.default_rng(5)
    k = rng.integers(0, f.support_center.shape[0], size=4000)
    dirs = rng.normal(size=(4000, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    pts = f.support_center[k] + dirs * (f.support_radius[k] * rng.uniform(0, 1.0, 4000))[:, None]
    pts = np.clip(pts, -0.4999, 0.4999)
    for p in pts:
        if orc.support(osc, p) > 0:
            c = np.floor((p + 0.5) * R).astype(int)
            assert bits[c[0] + R * (c[1] + R * c[2])]


def test_gauss_field_closed_forms(orc):
    sc = S.config1()
    sc.field = S.gauss_field([[0.1, 0.0, 0.0]], [0.1], [50.0], [[1.0, 2.0, 3.0]])
    osc = orc.OracleScene(sc)
    sig, rgb = orc.field_eval(osc, [0.1, 0.0, 0.0])
    assert sig == pytest.approx(50.0, rel=1e-15)
    sig, _ = orc.field_eval(osc, [0.1 + 0.1, 0.0, 0.0])     # one radius away: peak * e^-1/2
    assert sig == pytest.approx(50.0 * math.exp(-0.5), rel=1e-7)
    # two equal blobs: colour at the midpoint is the mean of the emissions
    sc.field = S.gauss_field([[-0.1, 0, 0], [0.1, 0, 0]], [0.1, 0.1], [50, 50], [[1, 0, 0], [0, 0, 4]])
    osc = orc.OracleScene(sc)
    _, rgb = orc.field_eval(osc, [0.0, 0.0, 0.0])
    assert np.allclose(rgb, [0.5, 0, 2.0], rtol=1e-15)


# --------------------------------------------------------------- intersection
def test_moller_trumbore_recovers_barycentrics(orc):
    rng = np.random.default_rng(7)
    for _ in range(200):
        v = rng.uniform(-1, 1, size=(3, 3))
        b1, b2 = rng.uniform(0, 0.5, size=2)
        p = (1 - b1 - b2) * v[0] + b1 * v[1] + b2 * v[2]
        o = rng.uniform(-3, 3, size=3)
        d = (p - o) / np.linalg.norm(p - o)
        hit, t, g1, g2 = orc.intersect_tri(o, d, *v)
        assert hit
        assert abs(g1 - b1) < 1e-9 and abs(g2 - b2) < 1e-9
        assert abs(t - np.linalg.norm(p - o)) < 1e-9


def test_intersection_edge_inclusive_and_misses(orc):
    v0, v1, v2 = [0, 0, 0], [1, 0, 0], [0, 1, 0]
    d = [0, 0, -1]
    assert orc.intersect_tri([0.5, 0.0, 1.0], d, v0, v1, v2)[0]        # on edge v0-v1
    assert orc.intersect_tri([0.5, 0.5, 1.0], d, v0, v1, v2)[0]        # on the hypotenuse
    assert orc.intersect_tri([0.0, 0.0, 1.0], d, v0, v1, v2)[0]        # at a vertex
    assert not orc.intersect_tri([0.5, -1e-12, 1.0], d, v0, v1, v2)[0]
    assert not orc.intersect_tri([0.6, 0.6, 1.0], d, v0, v1, v2)[0]
    assert not orc.intersect_tri([0.2, 0.2, 1.0], [1, 0, 0], v0, v1, v2)[0]   # parallel
    assert not orc.intersect_tri([0.2, 0.2, -1.0], d, v0, v1, v2)[0]          # behind
    hit, t, _, _ = orc.intersect_tri([0.2, 0.2, 1.0], d, v0, v1, v2)
    assert hit and t == 1.0


def test_closest_hit_brute_force(orc):
    # three stacked squares (2 triangles each) at z = 0, -1, -2
    quads = [S.quad_mesh([-1, -1, z], [1, -1, z], [1, 1, z], [-1, 1, z], 0) for z in (0.0, -1.0, -2.0)]
    sc = S.config1()
    sc.mesh = S.merge_meshes(quads)
    osc = orc.OracleScene(sc)
    tid, t, fl = orc.closest_hit(osc, [0.3, -0.2, 1.0], [0, 0, -1])
    assert tid in (0, 1) and t == 1.0 and fl == 0
    tid2, t2, _ = orc.closest_hit(osc, [0.3, -0.2, 1.0], [0, 0, -1], skip=tid)
    assert tid2 in (2, 3) and t2 == 2.0      # skipping the first square's triangle
    tid3, t3, _ = orc.closest_hit(osc, [0.3, -0.2, 1.0], [0, 0, 1])
    assert tid3 == orc.NO_HIT and math.isinf(t3)
    # a hit on the shared diagonal: both triangles tie, the lower id wins and the pixel is flagged
    tid4, _, fl4 = orc.closest_hit(osc, [0.25, 0.25, 1.0], [0, 0, -1])
    assert tid4 == 0 and fl4 & orc.FLAG_EDGE


# --------------------------------------------------------------- BSDFs
def test_mirror_reflection_laws(orc):
    rng = np.random.default_rng(11)
    for _ in range(100):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        r = orc.reflect(d, n)
        assert abs(np.linalg.norm(r) - 1) < 1e-14
        assert abs(r @ n + d @ n) < 1e-14                       # d'.n = -d.n
        assert np.allclose(r - (r @ n) * n, d - (d @ n) * n)    # tangential part kept


def test_fresnel_closed_forms(orc):
    assert orc.fresnel(1.0, 1.0, 1.5) == pytest.approx(0.04, abs=1e-15)
    assert orc.fresnel(1.0, 1.5, 1.0) == pytest.approx(0.04, abs=1e-15)
    # Brewster angle: p-polarised reflectance vanishes, so F = r_s^2 / 2 with theta_t = 90 deg - theta_i
    tb = math.atan(1.5)
    ci, ct = math.cos(tb), math.cos(math.pi / 2 - tb)
    rs = (ci - 1.5 * ct) / (ci + 1.5 * ct)
    assert orc.fresnel(ci, 1.0, 1.5) == pytest.approx(rs * rs / 2, rel=1e-12)
    # total internal reflection beyond asin(1/1.5) = 41.81 deg inside the glass
    crit = math.asin(1 / 1.5)
    assert orc.fresnel(math.cos(crit + 1e-6), 1.5, 1.0) == 1.0
    assert orc.fresnel(math.cos(crit - 1e-3), 1.5, 1.0) < 1.0
    # grazing incidence reflects everything; reflectance grows with angle
    assert orc.fresnel(1e-9, 1.0, 1.5) == pytest.approx(1.0, abs=1e-8)
    fs = [orc.fresnel(math.cos(math.radians(a)), 1.0, 1.5) for a in range(0, 89, 4)]
    assert all(a <= b + 1e-15 for a, b in zip(fs[10:], fs[11:]))


def test_snell_refraction(orc):
    for deg in [0, 10, 30, 45, 60, 80]:
        th = math.radians(deg)
        d = np.array([math.sin(th), 0, -math.cos(th)])
        ok, t = orc.refract(d, [0, 0, 1], 1 / 1.5)
        assert ok
        assert abs(np.linalg.norm(t) - 1) < 1e-14
        assert math.isclose(math.hypot(t[0], t[1]), math.sin(th) / 1.5, rel_tol=1e-12, abs_tol=1e-15)
        assert t[2] < 0
    # from inside beyond the critical angle: TIR
    th = math.radians(45)
    ok, _ = orc.refract(np.array([math.sin(th), 0, -math.cos(th)]), [0, 0, 1], 1.5)
    assert not ok


@pytest.mark.parametrize("n", [[0, 0, 1], [0, 0, -1], [0, 1, 0], [0.6, 0, 0.8], [-0.48, 0.6, -0.64]])
def test_cosine_hemisphere_sampling(orc, n):
    n = np.asarray(n, np.float64) / np.linalg.norm(n)
    k = 64
    us = (np.arange(k) + 0.5) / k
    cos = []
    for u1 in us:
        for u2 in us:
            w = orc.sample_cosine(n, u1, u2)
            assert abs(np.linalg.norm(w) - 1) < 1e-13
            cos.append(w @ n)
    cos = np.array(cos)
    assert cos.min() > 0
    # E[cos theta] = 2/3 for the cosine-weighted pdf; cos^2 theta is uniform on [0, 1]
    assert abs(cos.mean() - 2 / 3) < 2e-3
    hist, _ = np.histogram(cos ** 2, bins=8, range=(0, 1))
    assert np.all(np.abs(hist - cos.size / 8) <= 1)


# --------------------------------------------------------------- view-dependent radiance
def test_view_networks_match_torch_layers(orc):
    torch = pytest.importorskip("torch")
    sc = S.config2_view(8, 8)
    osc = orc.OracleScene(sc)
    f, v = sc.field, sc.field.view
    rng = np.random.default_rng(12)
    F = torch.nn.functional
    T = lambda a: torch.tensor(np.asarray(a, np.float64))
    for _ in range(8):
        feat = rng.uniform(-0.5, 0.5, 32)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        lg, rgb = orc.mlp_view(osc, feat, d)
        h = F.relu(F.linear(T(feat), T(f.w1), T(f.b1)))
        dn = F.linear(h, T(v["wd2"]), T(v["bd2"]))
        x = torch.cat([dn, T(orc.sh16(d))])
        c = F.relu(F.linear(x, T(v["wc1"]), T(v["bc1"])))
        c = F.relu(F.linear(c, T(v["wc2"]), T(v["bc2"])))
        out = F.softplus(F.linear(c, T(v["wc3"]), T(v["bc3"])))
        assert lg == pytest.approx(float(dn[0]), rel=1e-13, abs=1e-13)
        assert np.allclose(rgb, out.numpy(), rtol=1e-13, atol=1e-14)


def test_view_dependence_is_only_in_the_colour(orc):
    sc = S.config2_view(8, 8)
    osc = orc.OracleScene(sc)
    p = None
    rng = np.random.default_rng(13)
    for _ in range(200):   # a point with density
        q = rng.uniform(-0.4, 0.4, 3)
        if orc.field_eval_dir(osc, q, [0, 0, 1])[0] > 1.0:
            p = q
            break
    assert p is not None
    s1, c1 = orc.field_eval_dir(osc, p, [0, 0, 1])
    s2, c2 = orc.field_eval_dir(osc, p, [1, 0, 0])
    assert s1 == s2 and np.abs(c1 - c2).max() > 1e-3
    # zero SH columns of the colour network: no view dependence at all
    sc.field.view["wc1"] = sc.field.view["wc1"].copy()
    sc.field.view["wc1"][:, 16:] = 0
    osc = orc.OracleScene(sc)
    _, c1 = orc.field_eval_dir(osc, p, [0, 0, 1])
    _, c2 = orc.field_eval_dir(osc, p, [0.6, -0.8, 0])
    assert np.array_equal(c1, c2)
