"""FP64 CPU oracle of the hybrid mesh + radiance-field light-transport loop.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The CUDA library never imports,
links or calls anything in this directory.

The arithmetic lives in ``mrf_oracle.c`` (plain C, double precision, written
step by step from the paper's Algorithm 1 and Eqs. 3, 10-13) and in
``shadow_net.c`` (the learned shadow-transmittance surrogate: encoding,
network, loss, back-propagation and Adam, in FP64).  This module only compiles
them with gcc and marshals numpy arrays from a ``scenes.Scene`` into the C
struct ``orc_scene``.

Every function here is pinned by a ``-m "not gpu"`` test (closed forms,
invariants, brute force, library routines) except the whole-image composition,
for which the paper gives no worked example: "parity unpinned" beyond its
pinned parts.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mrf_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "shadow_net.c")]
_LIB_PATH = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

NO_HIT = 0xFFFFFFFF
FLAG_EDGE, FLAG_SHADOW, FLAG_FRESNEL, FLAG_TAU, FLAG_BASIS, FLAG_TMIN = 1, 2, 4, 8, 16, 32
COUNT_NAMES = ("segments", "shadow_rays", "samples_nominal", "samples_supported", "surface_hits", "paths",
               "ended_miss", "ended_tau", "ended_cap")

_fp = C.POINTER(C.c_float)
_u32p = C.POINTER(C.c_uint32)
_u16p = C.POINTER(C.c_uint16)
_i32p = C.POINTER(C.c_int32)
_dp = C.POINTER(C.c_double)
_u64p = C.POINTER(C.c_uint64)


class OrcScene(C.Structure):
    _fields_ = [
        ("cam_pos", C.c_float * 3), ("cam_look", C.c_float * 3), ("cam_up", C.c_float * 3),
        ("vfov_deg", C.c_float), ("width", C.c_uint32), ("height", C.c_uint32),
        ("ray_o", _fp), ("ray_d", _fp), ("n_rays", C.c_uint32),
        ("field_kind", C.c_int32), ("aabb_min", C.c_float * 3), ("aabb_max", C.c_float * 3),
        ("const_sigma", C.c_float), ("const_rgb", C.c_float * 3),
        ("n_blobs", C.c_uint32), ("blob_c", _fp), ("blob_r", _fp), ("blob_peak", _fp), ("blob_e", _fp),
        ("n_levels", C.c_uint32), ("log2_T", C.c_uint32), ("n_feat", C.c_uint32),
        ("level_res", _u32p), ("table", _u16p), ("mlp_width", C.c_uint32),
        ("w1", _fp), ("b1", _fp), ("w2", _fp), ("b2", _fp), ("w3", _fp), ("b3", _fp),
        ("n_support", C.c_uint32), ("sup_c", _fp), ("sup_r", _fp),
        ("n_verts", C.c_uint32), ("verts", _fp), ("n_tris", C.c_uint32), ("tris", _u32p), ("tri_mat", _u32p),
        ("n_mats", C.c_uint32), ("mat_kind", _i32p), ("mat_rgb", _fp), ("mat_ior", _fp),
        ("n_lights", C.c_uint32), ("light_pos", _fp), ("light_I", _fp),
        ("max_bounces", C.c_uint32), ("spp", C.c_uint32), ("seed", C.c_uint64),
        ("steps_per_segment", C.c_uint32), ("dt", C.c_float), ("tau", C.c_float), ("tmin", C.c_float),
        ("margin_dist", C.c_double), ("margin_t", C.c_double), ("margin_fresnel", C.c_double),
        ("field_pose", _fp),
        ("n_views", C.c_uint32), ("view_cam", _fp), ("view_size", _u32p),
        ("light_kind", _i32p), ("light_v1", _fp), ("light_v2", _fp), ("light_samples", _u32p),
        ("shadow_net", C.c_void_p), ("shadow_mask", C.c_int32), ("light_mask", _fp),
        ("view_dep", C.c_int32), ("wd2", _fp), ("bd2", _fp), ("wc1", _fp), ("bc1", _fp), ("wc2", _fp), ("bc2", _fp),
        ("wc3", _fp), ("bc3", _fp), ("margin_tau", C.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, strict IEEE double, no contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or any(os.path.getmtime(_LIB_PATH) < os.path.getmtime(f)
                                                         for f in _SRCS):
            tmp = _LIB_PATH + f".{os.getpid()}.tmp"
            cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                   "-fno-fast-math", "-Wall", "-Wno-unused-function", "-o", tmp, *_SRCS, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        L.orc_half_to_double.restype = C.c_double
        L.orc_half_to_double.argtypes = [C.c_uint16]
        L.orc_philox4x64.argtypes = [_u64p, _u64p, _u64p]
        L.orc_camera_ray.argtypes = [C.POINTER(OrcScene), C.c_uint32, _dp, _dp]
        L.orc_hash_encode.argtypes = [C.POINTER(OrcScene), _dp, _dp]
        L.orc_mlp.argtypes = [C.POINTER(OrcScene), _dp, _dp]
        L.orc_support.restype = C.c_double
        L.orc_support.argtypes = [C.POINTER(OrcScene), _dp]
        L.orc_field_eval.restype = C.c_int
        L.orc_field_eval.argtypes = [C.POINTER(OrcScene), _dp, _dp, _dp]
        L.orc_field_eval_dir.restype = C.c_int
        L.orc_field_eval_dir.argtypes = [C.POINTER(OrcScene), _dp, _dp, _dp, _dp]
        L.orc_mlp_view.argtypes = [C.POINTER(OrcScene), _dp, _dp, _dp, _dp]
        L.orc_box_interval.restype = C.c_int
        L.orc_box_interval.argtypes = [C.POINTER(OrcScene), _dp, _dp, _dp, _dp]
        L.orc_transmittance.restype = C.c_double
        L.orc_transmittance.argtypes = [C.POINTER(OrcScene), _dp, _dp, C.c_double, C.c_double, _u64p]
        L.orc_march.argtypes = [C.POINTER(OrcScene), _dp, _dp, C.c_double, C.c_double, _dp, _dp]
        L.orc_intersect_tri.restype = C.c_int
        L.orc_intersect_tri.argtypes = [_dp, _dp, _dp, _dp, _dp, C.c_double, _dp, _dp, _dp]
        L.orc_closest_hit.restype = C.c_uint32
        L.orc_closest_hit.argtypes = [C.POINTER(OrcScene), _dp, _dp, C.c_uint32, _dp, _u32p]
        L.orc_reflect.argtypes = [_dp, _dp, _dp]
        L.orc_fresnel.restype = C.c_double
        L.orc_fresnel.argtypes = [C.c_double, C.c_double, C.c_double]
        L.orc_refract.restype = C.c_int
        L.orc_refract.argtypes = [_dp, _dp, C.c_double, _dp]
        L.orc_sample_cosine.argtypes = [_dp, C.c_double, C.c_double, _dp]
        L.orc_render.restype = C.c_int
        L.orc_render.argtypes = [C.POINTER(OrcScene), _u32p, C.c_uint32, _dp, _u32p, _u32p, _dp, _u32p, _u64p,
                                 C.c_int]
        L.orc_render_ex.restype = C.c_int
        L.orc_render_ex.argtypes = [C.POINTER(OrcScene), _u32p, C.c_uint32, _dp, _u32p, _u32p, _dp, _u32p, _u64p,
                                    C.c_int, _u32p]
        L.orc_num_threads.restype = C.c_int
        L.orc_tonemap.restype = C.c_double
        L.orc_tonemap.argtypes = [C.c_double, C.c_double]
        L.orc_shadow_pairs.argtypes = [C.POINTER(OrcScene), C.c_uint64, C.c_uint64, C.c_uint32, _dp]
        L.orc_sh16.argtypes = [_dp, _dp]
        L.orc_snet_n_params.restype = C.c_uint64
        L.orc_snet_n_params.argtypes = [C.POINTER(OrcSnet)]
        L.orc_snet_encode.argtypes = [C.POINTER(OrcSnet), _dp, _dp, _dp]
        L.orc_snet_forward.restype = C.c_double
        L.orc_snet_forward.argtypes = [C.POINTER(OrcSnet), _dp, _dp]
        L.orc_snet_relu_margin.restype = C.c_double
        L.orc_snet_relu_margin.argtypes = [C.POINTER(OrcSnet), _dp, _dp]
        L.orc_snet_loss_grad.restype = C.c_double
        L.orc_snet_loss_grad.argtypes = [C.POINTER(OrcSnet), _dp, _dp, C.c_uint32, _dp]
        L.orc_adam_step.argtypes = [_dp, _dp, _dp, _dp, C.c_uint64, C.c_uint32, C.c_double, C.c_double, C.c_double,
                                    C.c_double]
        _lib = L
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(t) if a is not None else None


class OracleScene:
    """A ``scenes.Scene`` marshalled into an ``orc_scene`` (keeps its arrays alive)."""

    def __init__(self, scene, margin_dist=2e-7, margin_t=1e-5, margin_fresnel=1e-5, margin_tau=2e-6, shadow_net=None):
        self.scene = scene
        self.shadow_net = shadow_net
        keep = []

        def arr(a, dt):
            if a is None:
                return None
            x = np.ascontiguousarray(np.asarray(a).astype(dt, copy=False))
            keep.append(x)
            return x

        s = OrcScene()
        cam = scene.camera
        s.cam_pos[:] = list(map(float, cam.pos))
        s.cam_look[:] = list(map(float, cam.look_at))
        s.cam_up[:] = list(map(float, cam.up))
        s.vfov_deg = cam.vfov_deg
        s.width, s.height = cam.width, cam.height
        if scene.ray_o is not None:
            s.ray_o = _ptr(arr(scene.ray_o, np.float32), _fp)
            s.ray_d = _ptr(arr(scene.ray_d, np.float32), _fp)
            s.n_rays = scene.ray_o.shape[0]
        f = scene.field
        s.field_kind = f.kind
        s.aabb_min[:] = list(map(float, f.aabb_min))
        s.aabb_max[:] = list(map(float, f.aabb_max))
        s.const_sigma = f.const_sigma
        s.const_rgb[:] = list(map(float, f.const_rgb))
        if f.blob_center is not None:
            s.n_blobs = f.blob_center.shape[0]
            s.blob_c = _ptr(arr(f.blob_center, np.float32), _fp)
            s.blob_r = _ptr(arr(f.blob_radius, np.float32), _fp)
            s.blob_peak = _ptr(arr(f.blob_peak, np.float32), _fp)
            s.blob_e = _ptr(arr(f.blob_emission, np.float32), _fp)
        if f.table is not None:
            s.n_levels = f.level_res.shape[0]
            s.log2_T = f.log2_table_size
            s.n_feat = f.n_features
            s.level_res = _ptr(arr(f.level_res, np.uint32), _u32p)
            s.table = _ptr(arr(f.table.view(np.uint16), np.uint16), _u16p)
            s.mlp_width = f.w1.shape[0]
            for nm in ("w1", "b1", "w2", "b2", "w3", "b3"):
                setattr(s, nm, _ptr(arr(getattr(f, nm), np.float32), _fp))
            s.n_support = f.support_center.shape[0]
            s.sup_c = _ptr(arr(f.support_center, np.float32), _fp)
            s.sup_r = _ptr(arr(f.support_radius, np.float32), _fp)
            if getattr(f, "view", None) is not None:
                s.view_dep = 1
                for nm in ("wd2", "bd2", "wc1", "bc1", "wc2", "bc2", "wc3", "bc3"):
                    setattr(s, nm, _ptr(arr(f.view[nm], np.float32), _fp))
        m = scene.mesh
        s.n_verts = m.verts.shape[0]
        s.verts = _ptr(arr(m.verts, np.float32), _fp)
        s.n_tris = m.tris.shape[0]
        s.tris = _ptr(arr(m.tris, np.uint32), _u32p)
        s.tri_mat = _ptr(arr(m.mat, np.uint32), _u32p)
        mats = scene.materials or []
        s.n_mats = len(mats)
        s.mat_kind = _ptr(arr(np.array([x.kind for x in mats] or [0], np.int32), np.int32), _i32p)
        s.mat_rgb = _ptr(arr(np.array([x.rgb for x in mats] or [(0, 0, 0)], np.float32), np.float32), _fp)
        s.mat_ior = _ptr(arr(np.array([x.ior for x in mats] or [1.0], np.float32), np.float32), _fp)
        lights = scene.lights or []
        s.n_lights = len(lights)
        s.light_pos = _ptr(arr(np.array([x.pos for x in lights] or [(0, 0, 0)], np.float32), np.float32), _fp)
        s.light_I = _ptr(arr(np.array([x.intensity for x in lights] or [(0, 0, 0)], np.float32), np.float32), _fp)
        if getattr(scene.opts, "shadow_mask", False):
            s.shadow_mask = 1
            s.light_mask = _ptr(arr(np.array([x.mask_strength for x in lights] or [0.0], np.float32), np.float32), _fp)
        if any(x.kind != 0 for x in lights):
            s.light_kind = _ptr(arr(np.array([x.kind for x in lights], np.int32), np.int32), _i32p)
            s.light_v1 = _ptr(arr(np.array([x.v1 if x.v1 is not None else (0, 0, 0) for x in lights], np.float32),
                                  np.float32), _fp)
            s.light_v2 = _ptr(arr(np.array([x.v2 if x.v2 is not None else (0, 0, 0) for x in lights], np.float32),
                                  np.float32), _fp)
            s.light_samples = _ptr(arr(np.array([x.samples for x in lights], np.uint32), np.uint32), _u32p)
        o = scene.opts
        s.max_bounces, s.spp, s.seed = o.max_bounces, o.spp, o.seed
        s.steps_per_segment, s.dt, s.tau, s.tmin = o.steps_per_segment, o.dt, o.tau, o.tmin
        s.margin_dist, s.margin_t, s.margin_fresnel = margin_dist, margin_t, margin_fresnel
        s.margin_tau = margin_tau
        if getattr(f, "pose", None) is not None:
            s.field_pose = _ptr(arr(f.pose, np.float32), _fp)
        views = getattr(scene, "cameras", None)
        if views:
            s.n_views = len(views)
            s.view_cam = _ptr(arr(np.array([[*v.pos, *v.look_at, *v.up, v.vfov_deg] for v in views], np.float32),
                                  np.float32), _fp)
            s.view_size = _ptr(arr(np.array([[v.width, v.height] for v in views], np.uint32), np.uint32), _u32p)
        if shadow_net is not None:
            s.shadow_net = C.cast(C.pointer(shadow_net.s), C.c_void_p)
        self.s = s
        self._keep = keep

    @property
    def ref(self):
        return C.byref(self.s)


def render(scene, ids=None, threads: int = 0, records: bool = True, shadow_net=None, **margins):
    """Render ``ids`` (pixel or explicit-ray indices; default all) in FP64.

    Returns a dict: rgba (n,4) f64, segments (n,spp) u32, tri (n,spp,B) u32,
    t (n,spp,B) f64, flags (n,) u32, first_flag (n,spp) u32 (the segment of
    each path's first ambiguity flag, 0 = none), counts {name: int}."""
    L = lib()
    os_ = OracleScene(scene, shadow_net=shadow_net, **margins)
    n_all = scene.n_rays
    ids = np.arange(n_all, dtype=np.uint32) if ids is None else np.ascontiguousarray(np.asarray(ids, np.uint32))
    n = ids.shape[0]
    spp, B = scene.opts.spp, scene.opts.max_bounces
    rgba = np.zeros((n, 4), np.float64)
    segs = np.zeros((n, spp), np.uint32)
    tri = np.zeros((n, spp, B), np.uint32) if records else None
    tt = np.zeros((n, spp, B), np.float64) if records else None
    flags = np.zeros(n, np.uint32)
    first = np.zeros((n, spp), np.uint32)
    counts = np.zeros(len(COUNT_NAMES), np.uint64)
    L.orc_render_ex(os_.ref, _ptr(ids, _u32p), n, _ptr(rgba, _dp), _ptr(segs, _u32p), _ptr(tri, _u32p),
                    _ptr(tt, _dp), _ptr(flags, _u32p), _ptr(counts, _u64p), int(threads), _ptr(first, _u32p))
    return dict(rgba=rgba, segments=segs, tri=tri, t=tt, flags=flags, first_flag=first, ids=ids,
                counts={k: int(v) for k, v in zip(COUNT_NAMES, counts)})


# ---- thin wrappers of the unit functions (used by the pin tests) ----------
def _d(x, n=3):
    return np.ascontiguousarray(np.asarray(x, np.float64).reshape(n))


def half_to_double(bits: int) -> float:
    return lib().orc_half_to_double(int(bits))


def philox4x64(ctr, key):
    c = np.ascontiguousarray(np.asarray(ctr, np.uint64))
    k = np.ascontiguousarray(np.asarray(key, np.uint64))
    out = np.zeros(4, np.uint64)
    lib().orc_philox4x64(_ptr(c, _u64p), _ptr(k, _u64p), _ptr(out, _u64p))
    return out


def camera_ray(oscene: OracleScene, pix: int):
    o, d = np.zeros(3), np.zeros(3)
    lib().orc_camera_ray(oscene.ref, int(pix), _ptr(o, _dp), _ptr(d, _dp))
    return o, d


def hash_encode(oscene: OracleScene, p):
    f = oscene.scene.field
    feat = np.zeros(f.level_res.shape[0] * f.n_features)
    lib().orc_hash_encode(oscene.ref, _ptr(_d(p), _dp), _ptr(feat, _dp))
    return feat


def mlp(oscene: OracleScene, feat):
    out = np.zeros(4)
    lib().orc_mlp(oscene.ref, _ptr(np.ascontiguousarray(np.asarray(feat, np.float64)), _dp), _ptr(out, _dp))
    return out


def support(oscene: OracleScene, p) -> float:
    return lib().orc_support(oscene.ref, _ptr(_d(p), _dp))


def field_eval(oscene: OracleScene, p):
    sig = np.zeros(1)
    rgb = np.zeros(3)
    lib().orc_field_eval(oscene.ref, _ptr(_d(p), _dp), _ptr(sig, _dp), _ptr(rgb, _dp))
    return float(sig[0]), rgb


def field_eval_dir(oscene: OracleScene, p, d):
    sig = np.zeros(1)
    rgb = np.zeros(3)
    lib().orc_field_eval_dir(oscene.ref, _ptr(_d(p), _dp), _ptr(_d(d), _dp), _ptr(sig, _dp), _ptr(rgb, _dp))
    return float(sig[0]), rgb


def mlp_view(oscene: OracleScene, feat, d):
    """View-dependent networks on given encoder features: (sigma logit, rgb)."""
    f = np.ascontiguousarray(np.asarray(feat, np.float64))
    lg, rgb = np.zeros(1), np.zeros(3)
    lib().orc_mlp_view(oscene.ref, _ptr(f, _dp), _ptr(_d(d), _dp), _ptr(lg, _dp), _ptr(rgb, _dp))
    return float(lg[0]), rgb


def box_interval(oscene: OracleScene, o, d):
    t0, t1 = np.zeros(1), np.zeros(1)
    ok = lib().orc_box_interval(oscene.ref, _ptr(_d(o), _dp), _ptr(_d(d), _dp), _ptr(t0, _dp), _ptr(t1, _dp))
    return bool(ok), float(t0[0]), float(t1[0])


def transmittance(oscene: OracleScene, o, d, a, b) -> float:
    return lib().orc_transmittance(oscene.ref, _ptr(_d(o), _dp), _ptr(_d(d), _dp), float(a), float(b), None)


def march(oscene: OracleScene, o, d, a, b, T=(1.0, 1.0, 1.0), L=(0.0, 0.0, 0.0)):
    Tv, Lv = _d(T).copy(), _d(L).copy()
    lib().orc_march(oscene.ref, _ptr(_d(o), _dp), _ptr(_d(d), _dp), float(a), float(b), _ptr(Tv, _dp), _ptr(Lv, _dp))
    return Tv, Lv


def intersect_tri(o, d, v0, v1, v2, tmin=1e-6):
    t, b1, b2 = np.zeros(1), np.zeros(1), np.zeros(1)
    hit = lib().orc_intersect_tri(_ptr(_d(o), _dp), _ptr(_d(d), _dp), _ptr(_d(v0), _dp), _ptr(_d(v1), _dp),
                                  _ptr(_d(v2), _dp), float(tmin), _ptr(t, _dp), _ptr(b1, _dp), _ptr(b2, _dp))
    return bool(hit), float(t[0]), float(b1[0]), float(b2[0])


def closest_hit(oscene: OracleScene, o, d, skip=NO_HIT):
    t = np.zeros(1)
    fl = np.zeros(1, np.uint32)
    tid = lib().orc_closest_hit(oscene.ref, _ptr(_d(o), _dp), _ptr(_d(d), _dp), int(skip), _ptr(t, _dp),
                                _ptr(fl, _u32p))
    return int(tid), float(t[0]), int(fl[0])


def reflect(d, n):
    out = np.zeros(3)
    lib().orc_reflect(_ptr(_d(d), _dp), _ptr(_d(n), _dp), _ptr(out, _dp))
    return out


def fresnel(cos_i, eta_i, eta_t) -> float:
    return lib().orc_fresnel(float(cos_i), float(eta_i), float(eta_t))


def refract(d, n, eta):
    out = np.zeros(3)
    ok = lib().orc_refract(_ptr(_d(d), _dp), _ptr(_d(n), _dp), float(eta), _ptr(out, _dp))
    return bool(ok), out


def sample_cosine(n, u1, u2):
    out = np.zeros(3)
    lib().orc_sample_cosine(_ptr(_d(n), _dp), float(u1), float(u2), _ptr(out, _dp))
    return out


def num_threads() -> int:
    return lib().orc_num_threads()


def tonemap(L, exposure=1.0):
    """psi applied channel-wise to an array of linear radiance values."""
    f = lib().orc_tonemap
    a = np.asarray(L, np.float64)
    return np.vectorize(lambda v: f(float(v), float(exposure)))(a)


# ---- the shadow-transmittance surrogate (shadow_net.c) ----------------------
class OrcSnet(C.Structure):
    _fields_ = [("n_levels", C.c_uint32), ("log2_T", C.c_uint32), ("level_res", _u32p),
                ("aabb_min", C.c_float * 3), ("aabb_max", C.c_float * 3), ("field_pose", _fp), ("params", _dp)]


class OracleShadowNet:
    """The surrogate's hyper-parameters and an FP64 copy of a flat parameter vector."""

    def __init__(self, level_res, log2_T, params, aabb_min=(-0.5, -0.5, -0.5), aabb_max=(0.5, 0.5, 0.5),
                 pose=None):
        self.level_res = np.ascontiguousarray(np.asarray(level_res, np.uint32))
        self.params = np.ascontiguousarray(np.asarray(params, np.float64))
        self.pose = None if pose is None else np.ascontiguousarray(np.asarray(pose, np.float32))
        s = OrcSnet()
        s.n_levels = self.level_res.shape[0]
        s.log2_T = int(log2_T)
        s.level_res = _ptr(self.level_res, _u32p)
        s.aabb_min[:] = [float(x) for x in aabb_min]
        s.aabb_max[:] = [float(x) for x in aabb_max]
        s.field_pose = _ptr(self.pose, _fp) if self.pose is not None else None
        s.params = _ptr(self.params, _dp)
        self.s = s
        assert lib().orc_snet_n_params(C.byref(s)) == self.params.shape[0], "parameter count"

    @property
    def ref(self):
        return C.byref(self.s)

    def encode(self, p, w):
        x = np.zeros(32)
        lib().orc_snet_encode(self.ref, _ptr(_d(p), _dp), _ptr(_d(w), _dp), _ptr(x, _dp))
        return x

    def forward(self, p, w) -> float:
        return lib().orc_snet_forward(self.ref, _ptr(_d(p), _dp), _ptr(_d(w), _dp))

    def relu_margin(self, p, w) -> float:
        return lib().orc_snet_relu_margin(self.ref, _ptr(_d(p), _dp), _ptr(_d(w), _dp))

    def loss_grad(self, pw, y, grad=True):
        pw = np.ascontiguousarray(np.asarray(pw, np.float64).reshape(-1, 6))
        y = np.ascontiguousarray(np.asarray(y, np.float64).reshape(-1))
        g = np.zeros_like(self.params) if grad else None
        loss = lib().orc_snet_loss_grad(self.ref, _ptr(pw, _dp), _ptr(y, _dp), pw.shape[0], _ptr(g, _dp))
        return loss, g


def snet_n_params(n_levels: int, log2_T: int, width: int = 64, n_in: int = 32) -> int:
    return n_levels * (1 << log2_T) * 2 + width * n_in + width + 2 * (width * width + width) + width + 1


def sh16(w):
    out = np.zeros(16)
    lib().orc_sh16(_ptr(_d(w), _dp), _ptr(out, _dp))
    return out


def adam_step(theta, m, v, g, t, lr, b1=0.9, b2=0.99, eps=1e-15):
    """In place on the FP64 arrays theta, m, v."""
    lib().orc_adam_step(_ptr(theta, _dp), _ptr(m, _dp), _ptr(v, _dp), _ptr(np.ascontiguousarray(g, np.float64), _dp),
                        theta.shape[0], int(t), float(lr), float(b1), float(b2), float(eps))


def shadow_pairs(scene, seed: int, first: int, n: int) -> np.ndarray:
    """n x 8 (point, direction, distance, FP64 marched transmittance)."""
    os_ = OracleScene(scene)
    out = np.zeros((n, 8), np.float64)
    lib().orc_shadow_pairs(os_.ref, int(seed), int(first), int(n), _ptr(out, _dp))
    return out
