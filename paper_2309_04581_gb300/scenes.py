"""Seeded synthetic scenes for the hybrid mesh + radiance-field renderer.

This module only *generates inputs*: cameras, field parameters, meshes,
materials, lights and render options.  It holds none of the renderer's
arithmetic (no ray generation, no field evaluation, no intersection, no
shading); the CUDA library and the FP64 CPU oracle each implement those on
their own and both consume the arrays produced here.

All floating-point scene values are rounded to FP32 here, so that the FP32
GPU path and the FP64 oracle start from bit-identical parameters (the oracle
widens them exactly).

The scene shapes follow the paper's workloads (a bounded radiance field with
inserted mirror, glass and diffuse meshes, Fig. 1 and Sec. 3.1 of the paper);
the captured datasets the paper uses are not available, so every scene is
synthetic and seeded from ``MASTER_SEED`` through SplitMix64 sub-seeds.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field as dc_field
from typing import List, Optional

import numpy as np

MASTER_SEED = 20230908
_M64 = (1 << 64) - 1

# material kinds (Sec. 3.3 names refractive, reflective and Lambertian BSDFs)
MAT_MIRROR = 0
MAT_GLASS = 1
MAT_DIFFUSE = 2

# field kinds
FIELD_CONST = 0
FIELD_GAUSS = 1
FIELD_HASH = 2

# light kinds
LIGHT_POINT = 0
LIGHT_AREA = 1


def splitmix64(x: int) -> int:
    """One SplitMix64 output for state ``x`` (Steele, Lea, Flood 2014)."""
    x = (x + 0x9E3779B97F4A7C15) & _M64
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def subseed(config: int, purpose: int, master: int = MASTER_SEED) -> int:
    """Sub-seed for (config, purpose), derived from the master seed."""
    return splitmix64(splitmix64(splitmix64(master) ^ config) ^ (purpose * 0x632BE59BD9B4E019 & _M64))


def _rng(config: int, purpose: int) -> np.random.Generator:
    return np.random.default_rng(subseed(config, purpose))


def f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))


# ---------------------------------------------------------------------------
# scene containers
# ---------------------------------------------------------------------------
@dataclass
class Camera:
    pos: np.ndarray
    look_at: np.ndarray
    up: np.ndarray
    vfov_deg: float
    width: int
    height: int


@dataclass
class Field:
    kind: int
    aabb_min: np.ndarray
    aabb_max: np.ndarray
    # FIELD_CONST
    const_sigma: float = 0.0
    const_rgb: np.ndarray = dc_field(default_factory=lambda: f32([0, 0, 0]))
    # FIELD_GAUSS: sigma(x) = sum_k peak_k exp(-|x-c_k|^2 / (2 r_k^2)); emission-weighted colour
    blob_center: Optional[np.ndarray] = None   # (K,3) f32
    blob_radius: Optional[np.ndarray] = None   # (K,)  f32
    blob_peak: Optional[np.ndarray] = None     # (K,)  f32
    blob_emission: Optional[np.ndarray] = None  # (K,3) f32
    # FIELD_HASH: multiresolution hash grid + MLP
    level_res: Optional[np.ndarray] = None     # (L,) uint32
    log2_table_size: int = 19
    n_features: int = 2
    table: Optional[np.ndarray] = None         # (L, T, F) float16
    w1: Optional[np.ndarray] = None            # (64, L*F) f32
    b1: Optional[np.ndarray] = None
    w2: Optional[np.ndarray] = None            # (64, 64)
    b2: Optional[np.ndarray] = None
    w3: Optional[np.ndarray] = None            # (4, 64)
    b3: Optional[np.ndarray] = None
    support_center: Optional[np.ndarray] = None  # (S,3) f32: compact support of the density
    support_radius: Optional[np.ndarray] = None  # (S,)
    occ_res: int = 0
    occ_bits: Optional[np.ndarray] = None      # (occ_res^3 / 32,) uint32, cell x + R*(y + R*z)
    # rigid pose of the field, 3x4 local-to-world [R | t] f32 (None = identity)
    pose: Optional[np.ndarray] = None
    # view-dependent radiance: dict of the density head wd2 (16x64), bd2 and the
    # colour network wc1 (64x32), bc1, wc2 (64x64), bc2, wc3 (3x64), bc3 (None = off)
    view: Optional[dict] = None


@dataclass
class Mesh:
    verts: np.ndarray   # (V,3) f32
    tris: np.ndarray    # (N,3) uint32
    mat: np.ndarray     # (N,)  uint32 material index

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])


@dataclass
class Material:
    kind: int
    rgb: tuple = (1.0, 1.0, 1.0)  # mirror reflectance rho / diffuse albedo
    ior: float = 1.5              # glass index of refraction


@dataclass
class Light:
    pos: tuple                    # point light: position; area light: vertex v0
    intensity: tuple              # point light: intensity I; area light: radiance Le of the front side
    kind: int = LIGHT_POINT
    v1: Optional[tuple] = None    # area light: the other two vertices (front normal (v1-v0) x (v2-v0))
    v2: Optional[tuple] = None
    samples: int = 1              # area light: shadow rays per diffuse hit
    mask_strength: float = 0.0    # r_src of the field-sample shadow mask (0 = casts no mask)


def area_light(v0, v1, v2, radiance, samples: int) -> "Light":
    return Light(pos=tuple(f32(v0)), intensity=tuple(f32(radiance)), kind=LIGHT_AREA, v1=tuple(f32(v1)),
                 v2=tuple(f32(v2)), samples=int(samples))


@dataclass
class RenderOpts:
    max_bounces: int = 4          # maximum segments per path (camera segment = 1)
    spp: int = 1
    seed: int = 0
    steps_per_segment: int = 0    # >0: that many midpoint samples per segment
    dt: float = 0.0               # steps_per_segment == 0: fixed step length
    tau: float = 0.0              # throughput termination threshold (0 = off)
    tmin: float = 1e-6            # smallest accepted ray-triangle distance
    shadow_mask: bool = False     # scale field samples blocked from a light by 1 - r_src


@dataclass
class Scene:
    name: str
    camera: Camera
    field: Field
    mesh: Mesh
    materials: List[Material]
    lights: List[Light]
    opts: RenderOpts
    ray_o: Optional[np.ndarray] = None   # explicit rays (n,3) f32; overrides the camera
    ray_d: Optional[np.ndarray] = None
    cameras: Optional[List[Camera]] = None  # several views in one batch; overrides `camera`

    @property
    def n_rays(self) -> int:
        if self.ray_o is not None:
            return int(self.ray_o.shape[0])
        if self.cameras:
            return sum(c.width * c.height for c in self.cameras)
        return self.camera.width * self.camera.height


# ---------------------------------------------------------------------------
# meshes
# ---------------------------------------------------------------------------
def empty_mesh() -> Mesh:
    return Mesh(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.uint32), np.zeros((0,), np.uint32))


def merge_meshes(meshes: List[Mesh]) -> Mesh:
    vs, ts, ms, off = [], [], [], 0
    for m in meshes:
        vs.append(m.verts)
        ts.append(m.tris + off)
        ms.append(m.mat)
        off += m.verts.shape[0]
    return Mesh(f32(np.concatenate(vs)), np.ascontiguousarray(np.concatenate(ts).astype(np.uint32)),
                np.ascontiguousarray(np.concatenate(ms).astype(np.uint32)))


def box_mesh(center, half, mat: int, inward: bool = False) -> Mesh:
    """Axis-aligned box of 12 triangles; outward-facing winding unless ``inward``."""
    c = np.asarray(center, np.float64)
    h = np.broadcast_to(np.asarray(half, np.float64), (3,))
    corners = np.array([[x, y, z] for z in (-1, 1) for y in (-1, 1) for x in (-1, 1)], np.float64)
    verts = c + corners * h
    # vertex index = x + 2y + 4z with x,y,z in {0,1}
    quads = [(0, 2, 3, 1), (4, 5, 7, 6),   # z-, z+
             (0, 1, 5, 4), (2, 6, 7, 3),   # y-, y+
             (0, 4, 6, 2), (1, 3, 7, 5)]   # x-, x+
    tris = []
    for a, b, cc, d in quads:
        t1, t2 = (a, b, cc), (a, cc, d)
        if inward:
            t1, t2 = (a, cc, b), (a, d, cc)
        tris += [t1, t2]
    return Mesh(f32(verts), np.array(tris, np.uint32), np.full(len(tris), mat, np.uint32))


def quad_mesh(p0, p1, p2, p3, mat: int) -> Mesh:
    verts = np.array([p0, p1, p2, p3], np.float64)
    return Mesh(f32(verts), np.array([[0, 1, 2], [0, 2, 3]], np.uint32), np.full(2, mat, np.uint32))


def icosphere_faces(level: int):
    """Unit icosphere after ``level`` 1:4 subdivisions (normalised midpoints)."""
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(p, np.float64) / np.linalg.norm(p) for p in v]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
             (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5),
             (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    return np.array(verts), np.array(faces, np.int64)


def glass_icosphere_10240(center, radius, mat: int) -> Mesh:
    """10,240-triangle sphere: the level-4 icosphere (5,120 faces) with every face
    split in two at the midpoint of its longest edge.  The midpoint stays on the
    chord (it is not pushed onto the sphere), so the surface is exactly the
    level-4 polyhedron and stays closed where neighbouring faces split
    different edges."""
    verts, faces = icosphere_faces(4)
    verts = list(verts)
    cache = {}
    out = []
    for a, b, c in faces:
        e = [(np.linalg.norm(verts[a] - verts[b]), 0), (np.linalg.norm(verts[b] - verts[c]), 1),
             (np.linalg.norm(verts[c] - verts[a]), 2)]
        k = max(e)[1]
        tri = (a, b, c)
        p, q, r = tri[k], tri[(k + 1) % 3], tri[(k + 2) % 3]   # longest edge p-q, opposite r
        key = (min(p, q), max(p, q))
        if key not in cache:
            verts.append(0.5 * (verts[p] + verts[q]))
            cache[key] = len(verts) - 1
        m = cache[key]
        out += [(p, m, r), (m, q, r)]
    v = np.asarray(center, np.float64) + radius * np.array(verts)
    tris = np.array(out, np.uint32)
    assert tris.shape[0] == 10240
    return Mesh(f32(v), tris, np.full(tris.shape[0], mat, np.uint32))


def random_soup(n_tris: int, seed_purpose: int, scale: float = 0.3, tri_size: float = 0.15) -> Mesh:
    """Random triangle soup inside [-scale, scale]^3 (for intersection tests)."""
    rng = _rng(900, seed_purpose)
    c = rng.uniform(-scale, scale, size=(n_tris, 1, 3))
    v = c + rng.uniform(-tri_size, tri_size, size=(n_tris, 3, 3))
    verts = v.reshape(-1, 3)
    tris = np.arange(n_tris * 3, dtype=np.uint32).reshape(-1, 3)
    return Mesh(f32(verts), tris, np.zeros(n_tris, np.uint32))


# ---------------------------------------------------------------------------
# fields
# ---------------------------------------------------------------------------
UNIT_BOX_MIN = f32([-0.5, -0.5, -0.5])
UNIT_BOX_MAX = f32([0.5, 0.5, 0.5])


def const_field(sigma: float, rgb, aabb_min=UNIT_BOX_MIN, aabb_max=UNIT_BOX_MAX) -> Field:
    return Field(kind=FIELD_CONST, aabb_min=f32(aabb_min), aabb_max=f32(aabb_max),
                 const_sigma=float(np.float32(sigma)), const_rgb=f32(rgb))


def gauss_field(centers, radii, peaks, emission, aabb_min=UNIT_BOX_MIN, aabb_max=UNIT_BOX_MAX) -> Field:
    return Field(kind=FIELD_GAUSS, aabb_min=f32(aabb_min), aabb_max=f32(aabb_max),
                 blob_center=f32(np.reshape(centers, (-1, 3))), blob_radius=f32(np.reshape(radii, (-1,))),
                 blob_peak=f32(np.reshape(peaks, (-1,))), blob_emission=f32(np.reshape(emission, (-1, 3))))


def level_resolutions(n_levels: int, n_min: int, n_max: int) -> np.ndarray:
    """Per-level grid resolution N_l = floor(N_min * b^l), b = exp((ln N_max - ln N_min)/(L-1))
    (the multiresolution hash encoding the paper takes from Instant-NGP).  Evaluated in
    FP64 with a 1e-9 guard so that the exact endpoint N_max is not lost to rounding."""
    b = math.exp((math.log(n_max) - math.log(n_min)) / (n_levels - 1))
    return np.array([math.floor(n_min * b ** l + 1e-9) for l in range(n_levels)], np.uint32)


def occupancy_from_spheres(centers, radii, res: int, aabb_min, aabb_max, margin: float) -> np.ndarray:
    """Occupancy bitfield: a cell is set when its closed box, grown by ``margin``,
    meets any sphere.  Bit for cell (x, y, z) is word (i >> 5), bit (i & 31) with
    i = x + res*(y + res*z)."""
    lo = np.asarray(aabb_min, np.float64)
    ext = np.asarray(aabb_max, np.float64) - lo
    edges = [lo[a] + ext[a] * np.arange(res + 1) / res for a in range(3)]
    occ = np.zeros((res, res, res), bool)  # [z, y, x]
    for c, r in zip(np.asarray(centers, np.float64), np.asarray(radii, np.float64)):
        d = []
        for a in range(3):
            cl, ch = edges[a][:-1] - margin, edges[a][1:] + margin
            d.append(np.maximum(np.maximum(cl - c[a], c[a] - ch), 0.0))
        d2 = d[2][:, None, None] ** 2 + d[1][None, :, None] ** 2 + d[0][None, None, :] ** 2
        occ |= d2 <= r * r
    bits = occ.reshape(-1)  # x fastest
    words = np.zeros(res ** 3 // 32, np.uint32)
    idx = np.nonzero(bits)[0]
    np.bitwise_or.at(words, idx >> 5, (np.uint32(1) << (idx & 31).astype(np.uint32)))
    return words


def hash_field(config: int, n_levels=16, log2_T=19, n_feat=2, n_min=16, n_max=2048, width=64,
               n_support=8, support_r=(0.1, 0.25), support_c=0.3, occ_res=128, sigma_bias=3.0,
               aabb_min=UNIT_BOX_MIN, aabb_max=UNIT_BOX_MAX) -> Field:
    """Hash-grid field of the paper's default Instant-NGP shape: seeded table
    U(-a_l, a_l) with a_l = 0.5 * N_0 / N_l in FP16, seeded Xavier-uniform MLP
    32 -> 64 -> 64 -> 4, and a
    compact density support made of ``n_support`` seeded spheres whose
    conservative cover is the occupancy bitfield."""
    T = 1 << log2_T
    rng_t = _rng(config, 1)
    res = level_resolutions(n_levels, n_min, n_max)
    # amplitude 0.5 * N_0 / N_l: every level contributes the same feature gradient
    # (a 1/f spectrum, like a trained field), instead of white noise at 2048^3
    amp = 0.5 * n_min / res.astype(np.float64)
    table = (rng_t.uniform(-1.0, 1.0, size=(n_levels, T, n_feat)) * amp[:, None, None]).astype(np.float16)
    rng_w = _rng(config, 2)
    d_in = n_levels * n_feat

    def xavier(o, i):
        a = math.sqrt(6.0 / (i + o))
        return f32(rng_w.uniform(-a, a, size=(o, i)))

    w1, w2, w3 = xavier(width, d_in), xavier(width, width), xavier(4, width)
    b3 = f32([sigma_bias, 0, 0, 0])
    rng_s = _rng(config, 3)
    sc = f32(rng_s.uniform(-support_c, support_c, size=(n_support, 3)))
    sr = f32(rng_s.uniform(support_r[0], support_r[1], size=(n_support,)))
    occ = occupancy_from_spheres(sc, sr, occ_res, aabb_min, aabb_max, margin=1e-4)
    return Field(kind=FIELD_HASH, aabb_min=f32(aabb_min), aabb_max=f32(aabb_max),
                 level_res=res, log2_table_size=log2_T,
                 n_features=n_feat, table=np.ascontiguousarray(table),
                 w1=w1, b1=f32(np.zeros(width)), w2=w2, b2=f32(np.zeros(width)), w3=w3, b3=b3,
                 support_center=sc, support_radius=sr, occ_res=occ_res, occ_bits=occ)


# ---------------------------------------------------------------------------
# configurations
# ---------------------------------------------------------------------------
def default_camera(width: int, height: int) -> Camera:
    return Camera(pos=f32([0.0, 0.3, 1.6]), look_at=f32([0, 0, 0]), up=f32([0, 1, 0]),
                  vfov_deg=45.0, width=width, height=height)


def config1(width: int = 64, height: int = 64) -> Scene:
    """Plain method, analytic field: 8 seeded Gaussian blobs (radius U(0.05,0.15),
    peak sigma 50, constant linear-HDR emission U(0,4)) in [-1/2,1/2]^3, one
    12-triangle perfect-mirror cube of half-size 0.2 at the origin, 4 segments per
    path, 128 midpoint samples per segment."""
    rng = _rng(1, 0)
    centers = rng.uniform(-0.35, 0.35, size=(8, 3))
    radii = rng.uniform(0.05, 0.15, size=8)
    emission = rng.uniform(0.0, 4.0, size=(8, 3))
    field = gauss_field(centers, radii, np.full(8, 50.0), emission)
    mesh = box_mesh([0, 0, 0], 0.2, 0)
    return Scene(name="c1_gauss_mirror_64", camera=default_camera(width, height), field=field, mesh=mesh,
                 materials=[Material(MAT_MIRROR, (1.0, 1.0, 1.0))], lights=[],
                 opts=RenderOpts(max_bounces=4, spp=1, seed=1, steps_per_segment=128, tau=0.0))


DT_C2 = float(np.float32(math.sqrt(3.0) / 1024.0))


def config2(width: int = 800, height: int = 800, tau: float = 0.0, max_bounces: int = 8) -> Scene:
    """Hash-grid field (16 levels, 2^19 entries, 2 FP16 features, resolutions 16..2048,
    MLP 32-64-64-4 with exp density and softplus radiance), 128^3 occupancy, a
    10,240-triangle glass sphere (IOR 1.5), a mirror cube, a diffuse floor and one
    point light; up to 8 segments per path, fixed step sqrt(3)/1024."""
    field = hash_field(2)
    glass = glass_icosphere_10240([0.2, 0.0, 0.0], 0.15, 1)
    cube = box_mesh([-0.2, 0.0, 0.0], 0.1, 0)
    floor = quad_mesh([-0.5, -0.45, -0.5], [-0.5, -0.45, 0.5], [0.5, -0.45, 0.5], [0.5, -0.45, -0.5], 2)
    mesh = merge_meshes([glass, cube, floor])
    mats = [Material(MAT_MIRROR, (1.0, 1.0, 1.0)), Material(MAT_GLASS, ior=1.5),
            Material(MAT_DIFFUSE, (0.5, 0.5, 0.5))]
    lights = [Light(pos=(0.0, 0.45, 0.3), intensity=(2.0, 2.0, 2.0))]
    return Scene(name=f"c2_hash_glass_{width}x{height}", camera=default_camera(width, height), field=field,
                 mesh=mesh, materials=mats, lights=lights,
                 opts=RenderOpts(max_bounces=max_bounces, spp=1, seed=2, steps_per_segment=0, dt=DT_C2,
                                 tau=tau))


def seeded_area_lights(n: int = 4, samples: int = 16, config: int = 4):
    """n emitter triangles above the field box (y in [0.55, 0.75], outside it),
    equilateral with circumradius U(0.06, 0.12), random yaw, front side facing
    down, radiance U(30, 90) per channel (HDR emitters)."""
    rng = _rng(config, 7)
    out = []
    for _ in range(n):
        c = np.array([rng.uniform(-0.35, 0.35), rng.uniform(0.55, 0.75), rng.uniform(-0.35, 0.35)])
        r, yaw = rng.uniform(0.06, 0.12), rng.uniform(0, 2 * math.pi)
        # counter-clockwise seen from below: normal (v1 - v0) x (v2 - v0) points to -y
        vs = [c + r * np.array([math.cos(yaw - k * 2 * math.pi / 3), 0.0, math.sin(yaw - k * 2 * math.pi / 3)])
              for k in range(3)]
        if np.cross(vs[1] - vs[0], vs[2] - vs[0])[1] > 0:
            vs = [vs[0], vs[2], vs[1]]
        out.append(area_light(vs[0], vs[1], vs[2], rng.uniform(30.0, 90.0, 3), samples))
    return out


def config4(width: int = 1920, height: int = 1080, samples: int = 16, max_bounces: int = 8) -> Scene:
    """The hash-grid scene of config2 lit by 4 seeded area-light triangles with
    `samples` shadow rays each per diffuse hit, 1 spp."""
    sc = config2(width, height, max_bounces=max_bounces)
    sc.name = f"c4_area_lights_{width}x{height}"
    sc.lights = seeded_area_lights(4, samples)
    sc.opts.seed = 4
    return sc


def explicit_rays(scene: Scene, origins, dirs) -> Scene:
    """Copy of ``scene`` traced along the given rays instead of its camera."""
    d = np.asarray(dirs, np.float64)
    d = d / np.linalg.norm(d, axis=1, keepdims=True)
    return Scene(name=scene.name + "_rays", camera=scene.camera, field=scene.field, mesh=scene.mesh,
                 materials=scene.materials, lights=scene.lights, opts=scene.opts,
                 ray_o=f32(np.reshape(origins, (-1, 3))), ray_d=f32(d))


def strided_pixels(width: int, height: int, stride: int, offset: int = 0) -> np.ndarray:
    """Pixel indices (y*width + x) of every ``stride``-th row and column."""
    ys = np.arange(offset % stride, height, stride)
    xs = np.arange(offset % stride, width, stride)
    return np.ascontiguousarray((ys[:, None] * width + xs[None, :]).reshape(-1).astype(np.uint32))


def rigid_pose(axis, angle_rad: float, translation) -> np.ndarray:
    """3x4 local-to-world [R | t] (Rodrigues rotation about `axis`, then translation), in f32."""
    k = np.asarray(axis, np.float64)
    k = k / np.linalg.norm(k)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    R = np.eye(3) + math.sin(angle_rad) * K + (1 - math.cos(angle_rad)) * K @ K
    return f32(np.concatenate([R, np.asarray(translation, np.float64).reshape(3, 1)], axis=1))


def orbit_views(n: int, sizes, radius: float = 1.6, height: float = 0.3, vfov: float = 45.0):
    """n cameras on a circle around the origin looking at it, with the given (width, height) sizes."""
    cams = []
    for k in range(n):
        a = 2 * math.pi * k / n
        w, h = sizes[k % len(sizes)]
        cams.append(Camera(pos=f32([radius * math.sin(a), height, radius * math.cos(a)]), look_at=f32([0, 0, 0]),
                           up=f32([0, 1, 0]), vfov_deg=vfov, width=int(w), height=int(h)))
    return cams


def seeded_view_sizes(n: int, purpose: int = 0, lo=(256, 256), hi=(1920, 1080)):
    """n view sizes with log-uniform pixel counts between lo and hi (aspect interpolated)."""
    rng = _rng(3, purpose)
    out = []
    for _ in range(n):
        t = rng.uniform(0, 1)
        w = int(round(math.exp(math.log(lo[0]) + t * (math.log(hi[0]) - math.log(lo[0])))))
        h = int(round(math.exp(math.log(lo[1]) + t * (math.log(hi[1]) - math.log(lo[1])))))
        out.append((w, h))
    return out


# ---------------------------------------------------------------------------
# shadow-transmittance surrogate: hyper-parameters and seeded initial values
# ---------------------------------------------------------------------------
SNET_LEVELS = 8
SNET_LOG2_T = 17
SNET_WIDTH = 64
SNET_IN = 32


def snet_level_resolutions(n_levels: int = SNET_LEVELS, base: int = 16, finest: int = 181) -> np.ndarray:
    """floor(base * b^l) with b = (finest/base)^(1/(n_levels-1)) = sqrt(2): 16, 22, 32, 45, 64, 90, 128, 181."""
    return level_resolutions(n_levels, base, finest)


def snet_n_params(log2_T: int = SNET_LOG2_T, n_levels: int = SNET_LEVELS) -> int:
    W, D = SNET_WIDTH, SNET_IN
    return n_levels * (1 << log2_T) * 2 + W * D + W + 2 * (W * W + W) + W + 1


def snet_init(seed: int = 5, log2_T: int = SNET_LOG2_T, n_levels: int = SNET_LEVELS,
              table_scale: float = 1e-4) -> np.ndarray:
    """Flat FP32 parameter vector: table U(-1e-4, 1e-4); W1, W2, W3, W4
    Xavier-uniform; biases 0 (layout: table, W1, b1, W2, b2, W3, b3, W4, b4)."""
    rng = _rng(5, seed)
    W, D = SNET_WIDTH, SNET_IN
    parts = [rng.uniform(-table_scale, table_scale, n_levels * (1 << log2_T) * 2)]
    for fan_out, fan_in in ((W, D), (W, W), (W, W), (1, W)):
        lim = math.sqrt(6.0 / (fan_in + fan_out))
        parts.append(rng.uniform(-lim, lim, fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    return f32(np.concatenate(parts))


# ---------------------------------------------------------------------------
# dynamic sequence: a deforming cloth and moving rigid bodies, frame by frame
# ---------------------------------------------------------------------------
def cloth_grid(n: int, half: float, y: float, mat: int) -> Mesh:
    """(n+1)^2 vertices on the square [-half, half]^2 at height y, 2 n^2 triangles."""
    g = np.linspace(-half, half, n + 1)
    xx, zz = np.meshgrid(g, g, indexing="xy")
    verts = np.stack([xx.ravel(), np.full(xx.size, y), zz.ravel()], axis=1)
    i = np.arange(n)
    a = (i[None, :] + (n + 1) * i[:, None]).ravel()
    tris = np.concatenate([np.stack([a, a + n + 1, a + 1], 1), np.stack([a + 1, a + n + 1, a + n + 2], 1)])
    return Mesh(f32(verts), tris.astype(np.uint32), np.full(tris.shape[0], mat, np.uint32))


def torus_mesh(R: float, r: float, nu: int, nv: int, mat: int) -> Mesh:
    """Torus around the y axis, nu x nv quads split into 2 nu nv triangles."""
    u = np.arange(nu) * 2 * math.pi / nu
    v = np.arange(nv) * 2 * math.pi / nv
    uu, vv = np.meshgrid(u, v, indexing="ij")
    verts = np.stack([(R + r * np.cos(vv)) * np.cos(uu), r * np.sin(vv), (R + r * np.cos(vv)) * np.sin(uu)], -1)
    iu, iv = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
    a = iu * nv + iv
    b = ((iu + 1) % nu) * nv + iv
    c = ((iu + 1) % nu) * nv + (iv + 1) % nv
    d = iu * nv + (iv + 1) % nv
    tris = np.concatenate([np.stack([a, b, c], -1).reshape(-1, 3), np.stack([a, c, d], -1).reshape(-1, 3)])
    return Mesh(f32(verts.reshape(-1, 3)), tris.astype(np.uint32), np.full(tris.shape[0], mat, np.uint32))


class DynamicSequence:
    """A cloth grid (n x n quads) with seeded sinusoid-plus-noise motion and
    `bodies` rigid tori (2,048 triangles each) with seeded rigid motion, inside
    the config-2 field and its meshes; `vertices(k)` gives frame k's vertex
    array (topology fixed), `scene` frame 0."""

    def __init__(self, width=1920, height=1080, spp=4, cloth_n=256, bodies=64, lights=4, max_bounces=8):
        rng = _rng(5, 11)
        base = config2(width, height, max_bounces=max_bounces)
        self.static = base.mesh
        self.cloth = cloth_grid(cloth_n, 0.45, -0.3, 2)
        self.torus = torus_mesh(0.03, 0.012, 32, 32, 0)
        self.n_bodies = bodies
        self.body_center = rng.uniform(-0.35, 0.35, (bodies, 3))
        self.body_center[:, 1] = rng.uniform(-0.2, 0.35, bodies)
        self.body_axis = rng.normal(size=(bodies, 3))
        self.body_axis /= np.linalg.norm(self.body_axis, axis=1, keepdims=True)
        self.body_spin = rng.uniform(0.5, 2.0, bodies)
        self.body_orbit = rng.uniform(0.02, 0.08, (bodies, 3))
        self.body_freq = rng.uniform(0.3, 1.2, (bodies, 3))
        self.cloth_phase = rng.uniform(0, 2 * math.pi, self.cloth.verts.shape[0])
        mats = list(base.materials)            # 0 mirror, 1 glass, 2 diffuse
        body_mat = rng.integers(0, 3, bodies).astype(np.uint32)
        tris, mat, off = [self.static.tris], [self.static.mat], self.static.verts.shape[0]
        tris.append(self.cloth.tris + off)
        mat.append(self.cloth.mat)
        off += self.cloth.verts.shape[0]
        nv = self.torus.verts.shape[0]
        for b in range(bodies):
            tris.append(self.torus.tris + off + b * nv)
            mat.append(np.full(self.torus.tris.shape[0], body_mat[b], np.uint32))
        self.tris = np.ascontiguousarray(np.concatenate(tris).astype(np.uint32))
        self.mat = np.ascontiguousarray(np.concatenate(mat).astype(np.uint32))
        lights = [Light(pos=tuple(f32([rng.uniform(-0.4, 0.4), rng.uniform(0.42, 0.48), rng.uniform(-0.4, 0.4)])),
                        intensity=tuple(f32(rng.uniform(0.5, 1.5, 3)))) for _ in range(lights)]
        self.scene = Scene(name=f"dynamic_{width}x{height}", camera=default_camera(width, height), field=base.field,
                           mesh=Mesh(self.vertices(0), self.tris, self.mat), materials=mats, lights=lights,
                           opts=RenderOpts(max_bounces=max_bounces, spp=spp, seed=5, steps_per_segment=0, dt=DT_C2))

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])

    def vertices(self, k: int, fps: float = 30.0) -> np.ndarray:
        t = k / fps
        cv = self.cloth.verts.astype(np.float64).copy()
        cv[:, 1] += 0.04 * np.sin(6.0 * cv[:, 0] + 2.0 * t) * np.cos(5.0 * cv[:, 2] - 1.5 * t) \
            + 0.004 * np.sin(9.0 * t + self.cloth_phase)
        tv = self.torus.verts.astype(np.float64)
        out = [self.static.verts.astype(np.float64), cv]
        for b in range(self.n_bodies):
            ang = self.body_spin[b] * t
            k_ = self.body_axis[b]
            K = np.array([[0, -k_[2], k_[1]], [k_[2], 0, -k_[0]], [-k_[1], k_[0], 0]])
            R = np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K
            c = self.body_center[b] + self.body_orbit[b] * np.sin(self.body_freq[b] * t * 2 * math.pi)
            out.append(tv @ R.T + c)
        return f32(np.concatenate(out))


def view_networks(seed: int = 9, width: int = 64, sigma_bias: float = 3.0) -> dict:
    """Seeded Xavier-uniform weights of the view-dependent heads (density head
    16 x 64 with bias[0] = sigma_bias, colour network 32 -> 64 -> 64 -> 3)."""
    rng = _rng(6, seed)

    def xavier(fo, fi):
        lim = math.sqrt(6.0 / (fi + fo))
        return f32(rng.uniform(-lim, lim, (fo, fi)))

    bd2 = np.zeros(16)
    bd2[0] = sigma_bias
    return {"wd2": xavier(16, width), "bd2": f32(bd2), "wc1": xavier(width, 32), "bc1": f32(np.zeros(width)),
            "wc2": xavier(width, width), "bc2": f32(np.zeros(width)), "wc3": xavier(3, width), "bc3": f32(np.zeros(3))}


def config2_view(width: int = 800, height: int = 800, max_bounces: int = 8) -> Scene:
    """config2 with view-dependent radiance: the hash grid and first layer of
    config2 feed a 16-output density head and a colour network of those outputs
    and the view direction's spherical harmonics (the Instant-NGP layout)."""
    sc = config2(width, height, max_bounces=max_bounces)
    sc.field.view = view_networks()
    sc.name = f"c2_view_{width}x{height}"
    return sc


# ---------------------------------------------------------------------------
# batched views in a mirror room
# ---------------------------------------------------------------------------
def displaced_sphere(center, radius: float, level: int, mat: int, seed_purpose: int, amp: float = 0.1) -> Mesh:
    """Icosphere whose vertices move radially by amp * radius * n(x), n a seeded
    smooth noise (a sum of 6 random plane waves, values in [-1, 1])."""
    rng = _rng(7, seed_purpose)
    verts, faces = icosphere_faces(level)
    k = rng.normal(size=(6, 3)) * 3.0
    ph = rng.uniform(0, 2 * math.pi, 6)
    noise = np.sin(verts @ k.T + ph).sum(1) / 6.0
    v = np.asarray(center, np.float64) + verts * (radius * (1.0 + amp * noise))[:, None]
    return Mesh(f32(v), np.ascontiguousarray(faces, np.uint32), np.full(faces.shape[0], mat, np.uint32))


class MultiViewScene:
    """32 seeded views (log-uniform sizes from 256x256 to 1920x1080) inside a
    mirror room around the hash-grid field, with 13 noise-displaced spheres
    (5,120 triangles each, mixed materials) and a 128 x 128 cloth grid whose
    vertices move every frame; up to 16 segments per path."""

    def __init__(self, n_views: int = 32, scale: float = 1.0, max_bounces: int = 16, spheres: int = 13):
        rng = _rng(3, 21)
        base = config2(8, 8, max_bounces=max_bounces)
        room = box_mesh([0.0, 0.0, 0.0], 0.62, 0, inward=True)
        meshes = [room]
        for i in range(spheres):
            c = rng.uniform(-0.38, 0.38, 3)
            meshes.append(displaced_sphere(c, rng.uniform(0.05, 0.1), 4, int(rng.integers(0, 3)), i))
        self.static = merge_meshes(meshes)
        self.cloth = cloth_grid(128, 0.45, -0.4, 2)
        self.cloth_phase = rng.uniform(0, 2 * math.pi, self.cloth.verts.shape[0])
        mesh = merge_meshes([self.static, self.cloth])
        sizes = seeded_view_sizes(n_views, 4)
        sizes = [(max(1, int(round(w * scale))), max(1, int(round(h * scale)))) for w, h in sizes]
        views = orbit_views(n_views, sizes, radius=0.58, height=0.1, vfov=60.0)
        self.scene = Scene(name=f"views{n_views}", camera=views[0], field=base.field, mesh=mesh,
                           materials=base.materials, lights=base.lights, cameras=views,
                           opts=RenderOpts(max_bounces=max_bounces, spp=1, seed=3, steps_per_segment=0, dt=DT_C2))

    @property
    def n_tris(self) -> int:
        return int(self.scene.mesh.tris.shape[0])

    def vertices(self, k: int, fps: float = 30.0) -> np.ndarray:
        t = k / fps
        cv = self.cloth.verts.astype(np.float64).copy()
        cv[:, 1] += 0.03 * np.sin(7.0 * cv[:, 0] + 2.0 * t) * np.cos(6.0 * cv[:, 2] - 1.3 * t) \
            + 0.003 * np.sin(8.0 * t + self.cloth_phase)
        return f32(np.concatenate([self.static.verts.astype(np.float64), cv]))
