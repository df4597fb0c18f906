"""ctypes binding of the C ABI in include/mrf.h (argument marshalling only).

Every function named ``mrf_*`` here calls the library function of the same
name; all rendering work runs in the CUDA library ``libmrf.so``.  There is no
CPU fallback: if the library or a CUDA device is missing, the calls raise.

``Renderer`` is a convenience wrapper that uploads a ``scenes.Scene`` and
renders it into torch tensors (torch provides device memory and streams).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import scenes as S

_HERE = os.path.dirname(os.path.abspath(__file__))
# MRF_LIB selects another in-tree build (the bounds-checked libmrf_checked.so)
LIB_PATH = os.environ.get("MRF_LIB") or os.path.join(_HERE, "libmrf.so")
_lib = None
_lock = threading.Lock()

MRF_OK, MRF_ERR_INVALID_ARG, MRF_ERR_CUDA, MRF_ERR_OOM, MRF_ERR_TIMEOUT, MRF_ERR_NOT_READY, MRF_ERR_UNSUPPORTED = range(7)
MRF_FIELD_CONST, MRF_FIELD_GAUSS, MRF_FIELD_HASHGRID = 0, 1, 2
MRF_PREC_FP32, MRF_PREC_FP16, MRF_PREC_BF16 = 0, 1, 2
MRF_MAT_MIRROR, MRF_MAT_GLASS, MRF_MAT_DIFFUSE = 0, 1, 2
MRF_LIGHT_POINT, MRF_LIGHT_AREA = 0, 1
MRF_ENGINE_AUTO, MRF_ENGINE_MEGAKERNEL, MRF_ENGINE_WAVEFRONT = 0, 1, 2
KERNEL_NAMES = ("render_megakernel", "wf_cast", "field", "wf_shade", "wf_finalize", "wf_gen", "wf_composite",
                "wf_shadow_net", "wf_vis", "wf_overflow", "wf_mask", "wf_tail")
NO_HIT = 0xFFFFFFFF

# every entry point declared in include/mrf.h
EXPORTS = ("mrf_context_create", "mrf_context_destroy", "mrf_last_error", "mrf_version", "mrf_field_create",
           "mrf_field_destroy", "mrf_field_set_precision", "mrf_field_query", "mrf_bvh_build", "mrf_bvh_refit",
           "mrf_bvh_destroy", "mrf_bvh_rebuild", "mrf_cast", "mrf_materials_set", "mrf_lights_set", "mrf_render", "mrf_render_static",
           "mrf_tonemap", "mrf_shadow_net_create", "mrf_shadow_net_destroy", "mrf_shadow_net_param_count",
           "mrf_shadow_net_get_params", "mrf_shadow_net_set_params", "mrf_shadow_pairs", "mrf_shadow_net_grad",
           "mrf_shadow_net_train", "mrf_shadow_net_eval", "mrf_frame_capture", "mrf_frame_replay", "mrf_frame_stats",
           "mrf_frame_destroy", "mrf_tuning_get", "mrf_tuning_set", "mrf_autotune", "mrf_selftest_timeout",
           "mrf_debug_fail_allocations", "mrf_shadow_net_save", "mrf_shadow_net_load", "mrf_sync_status",
           "mrf_l2_read_bandwidth")

_fp = C.POINTER(C.c_float)
_u32p = C.POINTER(C.c_uint32)
_u16p = C.POINTER(C.c_uint16)
_vp = C.c_void_p


class mrf_field_desc(C.Structure):
    _fields_ = [
        ("kind", C.c_int32), ("aabb_min", C.c_float * 3), ("aabb_max", C.c_float * 3),
        ("const_sigma", C.c_float), ("const_rgb", C.c_float * 3),
        ("n_blobs", C.c_uint32), ("blob_center", _fp), ("blob_radius", _fp), ("blob_peak", _fp),
        ("blob_emission", _fp),
        ("n_levels", C.c_uint32), ("log2_table_size", C.c_uint32), ("n_features", C.c_uint32),
        ("level_res", _u32p), ("table", _u16p), ("mlp_width", C.c_uint32),
        ("w1", _fp), ("b1", _fp), ("w2", _fp), ("b2", _fp), ("w3", _fp), ("b3", _fp),
        ("n_support", C.c_uint32), ("support_center", _fp), ("support_radius", _fp),
        ("occ_res", C.c_uint32), ("occ_bits", _u32p), ("precision", C.c_int32), ("pose", _fp),
        ("view_dependent", C.c_int32), ("wd2", _fp), ("bd2", _fp), ("wc1", _fp), ("bc1", _fp), ("wc2", _fp),
        ("bc2", _fp), ("wc3", _fp), ("bc3", _fp),
    ]


class mrf_material(C.Structure):
    _fields_ = [("kind", C.c_int32), ("rgb", C.c_float * 3), ("ior", C.c_float)]


class mrf_light(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pos", C.c_float * 3), ("intensity", C.c_float * 3), ("v1", C.c_float * 3),
                ("v2", C.c_float * 3), ("samples", C.c_uint32), ("mask_strength", C.c_float)]


class mrf_camera(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("look_at", C.c_float * 3), ("up", C.c_float * 3),
                ("vfov_deg", C.c_float), ("width", C.c_uint32), ("height", C.c_uint32)]


class mrf_rays(C.Structure):
    _fields_ = [("camera", C.POINTER(mrf_camera)), ("origins", _vp), ("dirs", _vp), ("count", C.c_uint32),
                ("spp", C.c_uint32), ("n_cameras", C.c_uint32)]


class mrf_render_opts(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("steps_per_segment", C.c_uint32), ("dt", C.c_float), ("tau", C.c_float),
                ("tmin", C.c_float), ("engine", C.c_int32), ("rec_segments", _vp), ("rec_tri", _vp),
                ("rec_t", _vp), ("kernel_ms", C.POINTER(C.c_float)), ("kernel_launches", C.POINTER(C.c_uint32)),
                ("shadow_net", _vp), ("shadow_mask", C.c_int32)]


class mrf_shadow_net_desc(C.Structure):
    _fields_ = [("log2_table", C.c_uint32), ("level_res", C.c_uint32 * 8), ("params", _vp), ("seed", C.c_uint64),
                ("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("precision", C.c_int32), ("lr_decay", C.c_float)]


class mrf_tuning(C.Structure):
    _fields_ = [("field_groups", C.c_uint32), ("samples_per_path", C.c_uint32), ("rounds", C.c_uint32),
                ("tail_paths", C.c_uint32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class mrf_stats(C.Structure):
    _fields_ = [("paths", C.c_uint64), ("segments", C.c_uint64), ("surface_hits", C.c_uint64),
                ("shadow_rays", C.c_uint64), ("samples_nominal", C.c_uint64), ("samples_evaluated", C.c_uint64),
                ("shadow_samples_evaluated", C.c_uint64), ("fp64_retests", C.c_uint64), ("status", C.c_uint64),
                ("shadow_net_evals", C.c_uint64), ("ended_miss", C.c_uint64), ("ended_tau", C.c_uint64),
                ("ended_cap", C.c_uint64), ("bvh_nodes", C.c_uint64),
                ("bvh_tri_tests", C.c_uint64), ("bvh_worst_nodes", C.c_uint64), ("bvh_worst_path", C.c_uint64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class MrfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"mrf status {status}: {msg}")
        self.status = status


def lib():
    """Loads libmrf.so (built in-tree by ``build.py``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run paper_2309_04581_gb300.build.build())")
            L = C.CDLL(LIB_PATH)
            L.mrf_last_error.restype = C.c_char_p
            L.mrf_version.restype = C.c_char_p
            for name in EXPORTS:
                fn = getattr(L, name)
                if name not in ("mrf_last_error", "mrf_version"):
                    fn.restype = C.c_int
            for name in ("mrf_context_destroy", "mrf_field_destroy", "mrf_bvh_destroy", "mrf_shadow_net_destroy",
                         "mrf_frame_destroy", "mrf_debug_fail_allocations"):
                getattr(L, name).restype = None
            L.mrf_selftest_timeout.argtypes = [_vp, C.c_uint64, C.c_int32]
            L.mrf_sync_status.argtypes = [_vp, C.POINTER(C.c_uint32)]
            L.mrf_l2_read_bandwidth.argtypes = [_vp, C.c_uint64, C.c_uint32, _vp, C.POINTER(C.c_double)]
            L.mrf_shadow_net_save.argtypes = [_vp, C.c_char_p]
            L.mrf_shadow_net_load.argtypes = [_vp, C.c_char_p]
            L.mrf_debug_fail_allocations.argtypes = [C.c_uint32]
            L.mrf_frame_capture.argtypes = [_vp, _vp, _vp, C.POINTER(mrf_rays), C.c_uint32, C.POINTER(mrf_render_opts),
                                            _vp, C.POINTER(_vp)]
            L.mrf_frame_replay.argtypes = [_vp, _vp]
            L.mrf_tuning_get.argtypes = [_vp, C.POINTER(mrf_tuning)]
            L.mrf_tuning_set.argtypes = [_vp, C.POINTER(mrf_tuning)]
            L.mrf_autotune.argtypes = [_vp, _vp, _vp, C.POINTER(mrf_rays), C.c_uint32, C.POINTER(mrf_render_opts),
                                       _vp, _vp, C.c_uint32, C.POINTER(mrf_tuning), C.POINTER(C.c_float)]
            L.mrf_frame_stats.argtypes = [_vp, _vp, C.POINTER(mrf_stats)]
            L.mrf_frame_destroy.argtypes = [_vp]
            L.mrf_shadow_net_param_count.restype = C.c_uint64
            L.mrf_shadow_net_param_count.argtypes = [_vp]
            L.mrf_shadow_net_create.argtypes = [_vp, _vp, C.POINTER(mrf_shadow_net_desc), C.POINTER(_vp)]
            L.mrf_shadow_net_destroy.argtypes = [_vp]
            L.mrf_shadow_net_get_params.argtypes = [_vp, _vp, _vp]
            L.mrf_shadow_net_set_params.argtypes = [_vp, _vp, _vp]
            L.mrf_shadow_pairs.argtypes = [_vp, _vp, C.POINTER(mrf_render_opts), C.c_uint64, C.c_uint64, C.c_uint32,
                                           _vp, _vp]
            L.mrf_shadow_net_grad.argtypes = [_vp, _vp, C.c_uint32, _vp, _vp, _vp]
            L.mrf_shadow_net_train.argtypes = [_vp, _vp, C.c_uint64, C.c_uint32, C.c_uint32, _vp, _vp]
            L.mrf_shadow_net_eval.argtypes = [_vp, _vp, C.c_uint32, _vp, _vp]
            L.mrf_context_create.argtypes = [C.c_int, C.POINTER(_vp)]
            L.mrf_field_create.argtypes = [_vp, C.POINTER(mrf_field_desc), C.POINTER(_vp)]
            L.mrf_field_set_precision.argtypes = [_vp, C.c_int32]
            L.mrf_field_query.argtypes = [_vp, _vp, _vp, C.c_uint32, _vp, _vp]
            L.mrf_bvh_build.argtypes = [_vp, _vp, C.c_uint32, _vp, _vp, C.c_uint32, C.POINTER(_vp)]
            L.mrf_bvh_refit.argtypes = [_vp, _vp, C.c_uint32, _vp]
            L.mrf_bvh_rebuild.argtypes = [_vp, _vp, C.c_uint32, _vp]
            L.mrf_cast.argtypes = [_vp, _vp, _vp, _vp, _vp, C.c_uint32, C.c_float, _vp, _vp, _vp]
            L.mrf_materials_set.argtypes = [_vp, C.POINTER(mrf_material), C.c_uint32]
            L.mrf_lights_set.argtypes = [_vp, C.POINTER(mrf_light), C.c_uint32]
            L.mrf_render.argtypes = [_vp, _vp, _vp, C.POINTER(mrf_rays), C.c_uint32, C.POINTER(mrf_render_opts), _vp,
                                     _vp, C.POINTER(mrf_stats)]
            L.mrf_render_static.argtypes = [_vp, _vp, _vp, C.POINTER(mrf_rays), C.c_uint32, C.POINTER(mrf_render_opts),
                                            _vp, _vp, C.POINTER(mrf_stats)]
            L.mrf_tonemap.argtypes = [_vp, _vp, C.c_uint32, C.c_float, _vp, _vp]
            L.mrf_context_destroy.argtypes = [_vp]
            L.mrf_field_destroy.argtypes = [_vp]
            L.mrf_bvh_destroy.argtypes = [_vp]
            _lib = L
    return _lib


def check(status: int):
    if status != MRF_OK:
        raise MrfError(status, lib().mrf_last_error().decode())


# ---------------------------------------------------------------- raw ABI
def mrf_context_create(device: int = 0) -> int:
    h = _vp()
    check(lib().mrf_context_create(device, C.byref(h)))
    return h.value


def mrf_context_destroy(ctx: int):
    lib().mrf_context_destroy(ctx)


def mrf_field_create(ctx: int, desc: mrf_field_desc) -> int:
    h = _vp()
    check(lib().mrf_field_create(ctx, C.byref(desc), C.byref(h)))
    return h.value


def mrf_field_destroy(f: int):
    lib().mrf_field_destroy(f)


def mrf_field_set_precision(f: int, precision: int):
    check(lib().mrf_field_set_precision(f, precision))


def mrf_field_query(ctx: int, f: int, points_ptr: int, n: int, out_ptr: int, stream: int = 0):
    check(lib().mrf_field_query(ctx, f, points_ptr, n, out_ptr, stream))


def mrf_bvh_build(ctx: int, verts_ptr: int, n_verts: int, tris_ptr: int, mat_ptr: int, n_tris: int) -> int:
    h = _vp()
    check(lib().mrf_bvh_build(ctx, verts_ptr, n_verts, tris_ptr, mat_ptr, n_tris, C.byref(h)))
    return h.value


def mrf_bvh_refit(bvh: int, verts_ptr: int, n_verts: int, stream: int = 0):
    check(lib().mrf_bvh_refit(bvh, verts_ptr, n_verts, stream))


def mrf_bvh_destroy(bvh: int):
    lib().mrf_bvh_destroy(bvh)


def mrf_cast(ctx, bvh, o_ptr, d_ptr, skip_ptr, n, tmin, t_ptr, tri_ptr, stream=0):
    check(lib().mrf_cast(ctx, bvh, o_ptr, d_ptr, skip_ptr, n, tmin, t_ptr, tri_ptr, stream))


def mrf_materials_set(ctx: int, mats):
    arr = (mrf_material * max(1, len(mats)))()
    for i, m in enumerate(mats):
        arr[i].kind = m.kind
        arr[i].rgb[:] = [float(x) for x in m.rgb]
        arr[i].ior = float(m.ior)
    check(lib().mrf_materials_set(ctx, arr, len(mats)))


def mrf_lights_set(ctx: int, lights):
    arr = (mrf_light * max(1, len(lights)))()
    for i, l in enumerate(lights):
        arr[i].kind = l.kind
        arr[i].pos[:] = [float(x) for x in l.pos]
        arr[i].intensity[:] = [float(x) for x in l.intensity]
        if getattr(l, "v1", None) is not None:
            arr[i].v1[:] = [float(x) for x in l.v1]
            arr[i].v2[:] = [float(x) for x in l.v2]
        arr[i].samples = int(getattr(l, "samples", 1))
        arr[i].mask_strength = float(getattr(l, "mask_strength", 0.0))
    check(lib().mrf_lights_set(ctx, arr, len(lights)))


def mrf_render(ctx, field, bvh, rays: mrf_rays, max_bounces: int, opts: mrf_render_opts, out_ptr: int, stream: int = 0,
               stats: mrf_stats | None = None):
    check(lib().mrf_render(ctx, field, bvh, C.byref(rays), max_bounces, C.byref(opts), out_ptr, stream,
                           C.byref(stats) if stats is not None else None))


# ---------------------------------------------------------------- helpers
def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def field_desc(field: S.Field, precision: int = MRF_PREC_FP32):
    """mrf_field_desc for a scenes.Field (host arrays; returns desc and the arrays it points to)."""
    d = mrf_field_desc()
    keep = []

    def arr(a, dt):
        x = np.ascontiguousarray(np.asarray(a).astype(dt, copy=False))
        keep.append(x)
        return x

    d.kind = field.kind
    d.aabb_min[:] = [float(x) for x in field.aabb_min]
    d.aabb_max[:] = [float(x) for x in field.aabb_max]
    d.const_sigma = field.const_sigma
    d.const_rgb[:] = [float(x) for x in field.const_rgb]
    d.precision = precision
    if getattr(field, "pose", None) is not None:
        d.pose = _p(arr(field.pose, np.float32), _fp)
    if getattr(field, "view", None) is not None:
        d.view_dependent = 1
        for nm in ("wd2", "bd2", "wc1", "bc1", "wc2", "bc2", "wc3", "bc3"):
            setattr(d, nm, _p(arr(field.view[nm], np.float32), _fp))
    if field.blob_center is not None:
        d.n_blobs = field.blob_center.shape[0]
        d.blob_center = _p(arr(field.blob_center, np.float32), _fp)
        d.blob_radius = _p(arr(field.blob_radius, np.float32), _fp)
        d.blob_peak = _p(arr(field.blob_peak, np.float32), _fp)
        d.blob_emission = _p(arr(field.blob_emission, np.float32), _fp)
    if field.table is not None:
        d.n_levels = field.level_res.shape[0]
        d.log2_table_size = field.log2_table_size
        d.n_features = field.n_features
        d.level_res = _p(arr(field.level_res, np.uint32), _u32p)
        d.table = _p(arr(field.table.view(np.uint16), np.uint16), _u16p)
        d.mlp_width = field.w1.shape[0]
        for nm in ("w1", "b1", "w2", "b2", "w3", "b3"):
            setattr(d, nm, _p(arr(getattr(field, nm), np.float32), _fp))
        if field.support_center is not None:
            d.n_support = field.support_center.shape[0]
            d.support_center = _p(arr(field.support_center, np.float32), _fp)
            d.support_radius = _p(arr(field.support_radius, np.float32), _fp)
        if field.occ_bits is not None and field.occ_res:
            d.occ_res = field.occ_res
            d.occ_bits = _p(arr(field.occ_bits, np.uint32), _u32p)
    return d, keep


def camera_struct(cam: S.Camera) -> mrf_camera:
    c = mrf_camera()
    c.pos[:] = [float(x) for x in cam.pos]
    c.look_at[:] = [float(x) for x in cam.look_at]
    c.up[:] = [float(x) for x in cam.up]
    c.vfov_deg = float(cam.vfov_deg)
    c.width, c.height = cam.width, cam.height
    return c


class Renderer:
    """Uploads a scenes.Scene once and renders it on ``device`` with torch-owned buffers."""

    def __init__(self, scene: S.Scene, device: int = 0, precision: int = MRF_PREC_FP32):
        import torch
        self.torch = torch
        self.scene = scene
        self.device = device
        self.ctx = mrf_context_create(device)
        desc, keep = field_desc(scene.field, precision)
        self.field = mrf_field_create(self.ctx, desc)
        del keep
        m = scene.mesh
        v = np.ascontiguousarray(m.verts, np.float32)
        t = np.ascontiguousarray(m.tris, np.uint32)
        mt = np.ascontiguousarray(m.mat, np.uint32)
        self.bvh = mrf_bvh_build(self.ctx, v.ctypes.data, v.shape[0], t.ctypes.data, mt.ctypes.data, t.shape[0])
        if scene.materials:
            mrf_materials_set(self.ctx, scene.materials)
        mrf_lights_set(self.ctx, scene.lights)
        self.cam = camera_struct(scene.camera)
        self.views = None
        if scene.cameras:
            self.views = (mrf_camera * len(scene.cameras))(*[camera_struct(c) for c in scene.cameras])
        self._rays_dev = None
        if scene.ray_o is not None:
            dev = torch.device("cuda", device)
            self._rays_dev = (torch.from_numpy(scene.ray_o).to(dev), torch.from_numpy(scene.ray_d).to(dev))

    def tuning(self) -> dict:
        t = mrf_tuning()
        check(lib().mrf_tuning_get(self.ctx, C.byref(t)))
        return t.as_dict()

    def set_tuning(self, field_groups: int, samples_per_path: int, rounds: int = 1, tail_paths: int = 0):
        t = mrf_tuning(field_groups, samples_per_path, rounds, tail_paths)
        check(lib().mrf_tuning_set(self.ctx, C.byref(t)))

    def autotune(self, out=None, reps: int = 2, engine=MRF_ENGINE_AUTO, shadow_net=None):
        """Runs the autotuner on this renderer's request; returns (best tuning, [12 frame times in ms])."""
        torch = self.torch
        if out is None:
            out = torch.empty((self.scene.n_rays, 4), dtype=torch.float32, device=torch.device("cuda", self.device))
        best = mrf_tuning()
        ms = (C.c_float * 12)()
        opts = self.opts_struct(engine, None, shadow_net)
        check(lib().mrf_autotune(self.ctx, self.field, self.bvh, C.byref(self.rays_struct()),
                                 self.scene.opts.max_bounces, C.byref(opts), out.data_ptr(),
                                 torch.cuda.current_stream(self.device).cuda_stream, reps, C.byref(best), ms))
        return best.as_dict(), [float(x) for x in ms]

    def set_vertices(self, verts, rebuild=False, stream=None):
        """New vertex positions for the mesh (same topology): a refit of the BVH
        (mrf_bvh_refit), rebuild="gpu" a GPU rebuild in place (mrf_bvh_rebuild),
        both enqueued on `stream`, or rebuild="host" (or True) a host SAH build
        that replaces the BVH handle (captured frames keep the old one)."""
        v = np.ascontiguousarray(verts, np.float32)
        s = stream if stream is not None else self.torch.cuda.current_stream(self.device).cuda_stream
        if rebuild == "gpu":
            check(lib().mrf_bvh_rebuild(self.bvh, v.ctypes.data, v.shape[0], s))
        elif rebuild:
            m = self.scene.mesh
            t = np.ascontiguousarray(m.tris, np.uint32)
            mt = np.ascontiguousarray(m.mat, np.uint32)
            new = mrf_bvh_build(self.ctx, v.ctypes.data, v.shape[0], t.ctypes.data, mt.ctypes.data, t.shape[0])
            mrf_bvh_destroy(self.bvh)
            self.bvh = new
        else:
            mrf_bvh_refit(self.bvh, v.ctypes.data, v.shape[0], s)

    def close(self):
        if getattr(self, "ctx", None):
            mrf_bvh_destroy(self.bvh)
            mrf_field_destroy(self.field)
            mrf_context_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rays_struct(self) -> mrf_rays:
        r = mrf_rays()
        if self.views is not None:
            r.camera = C.cast(self.views, C.POINTER(mrf_camera))
            r.n_cameras = len(self.views)
            r.count = self.scene.n_rays
        elif self._rays_dev is None:
            r.camera = C.pointer(self.cam)
            r.count = self.scene.n_rays
        else:
            r.origins = self._rays_dev[0].data_ptr()
            r.dirs = self._rays_dev[1].data_ptr()
            r.count = self._rays_dev[0].shape[0]
        r.spp = self.scene.opts.spp
        return r

    def opts_struct(self, engine=MRF_ENGINE_AUTO, records=None, shadow_net=None) -> mrf_render_opts:
        o = self.scene.opts
        s = mrf_render_opts()
        s.shadow_net = shadow_net.handle if shadow_net is not None else None
        s.shadow_mask = 1 if getattr(o, "shadow_mask", False) else 0
        s.seed, s.steps_per_segment, s.dt, s.tau, s.tmin = o.seed, o.steps_per_segment, o.dt, o.tau, o.tmin
        s.engine = engine
        if records is not None:
            s.rec_segments = records["segments"].data_ptr()
            s.rec_tri = records["tri"].data_ptr()
            s.rec_t = records["t"].data_ptr()
        return s

    def new_records(self):
        torch = self.torch
        dev = torch.device("cuda", self.device)
        n, spp, B = self.scene.n_rays, self.scene.opts.spp, self.scene.opts.max_bounces
        return {"segments": torch.zeros(n * spp, dtype=torch.int32, device=dev),
                "tri": torch.zeros(n * spp * B, dtype=torch.int32, device=dev),
                "t": torch.zeros(n * spp * B, dtype=torch.float32, device=dev)}

    def render(self, out=None, engine=MRF_ENGINE_AUTO, records=None, stats=False, stream=None, timing=None,
               shadow_net=None):
        """Renders into ``out`` (count x 4 float32 CUDA tensor, allocated if None).
        Returns (out, stats dict or None).  If ``timing`` is a dict, it receives
        per-kernel CUDA-event milliseconds and launch counts of this call.
        ``shadow_net`` (a ShadowNet of this renderer) answers shadow rays."""
        torch = self.torch
        n = self.scene.n_rays
        if out is None:
            out = torch.empty((n, 4), dtype=torch.float32, device=torch.device("cuda", self.device))
        st = mrf_stats() if stats else None
        s = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        opts = self.opts_struct(engine, records, shadow_net)
        if timing is not None:
            ms = (C.c_float * len(KERNEL_NAMES))()
            cnt = (C.c_uint32 * len(KERNEL_NAMES))()
            opts.kernel_ms = ms
            opts.kernel_launches = cnt
        mrf_render(self.ctx, self.field, self.bvh, self.rays_struct(), self.scene.opts.max_bounces, opts,
                   out.data_ptr(), s, st)
        if timing is not None:
            for k, name in enumerate(KERNEL_NAMES):
                timing[name] = (float(ms[k]), int(cnt[k]))
        return out, (st.as_dict() if st is not None else None)


class Frame:
    """A Renderer's render call captured into a CUDA graph (mrf_frame_capture) for replay."""

    def __init__(self, renderer: "Renderer", out, engine=MRF_ENGINE_AUTO, records=None, shadow_net=None):
        self.r = renderer
        self.out = out
        opts = renderer.opts_struct(engine, records, shadow_net)
        h = _vp()
        check(lib().mrf_frame_capture(renderer.ctx, renderer.field, renderer.bvh, C.byref(renderer.rays_struct()),
                                      renderer.scene.opts.max_bounces, C.byref(opts), out.data_ptr(), C.byref(h)))
        self.handle = h.value

    def replay(self, stream=None):
        s = stream if stream is not None else self.r.torch.cuda.current_stream(self.r.device).cuda_stream
        check(lib().mrf_frame_replay(self.handle, s))

    def stats(self, stream=None) -> dict:
        s = stream if stream is not None else self.r.torch.cuda.current_stream(self.r.device).cuda_stream
        st = mrf_stats()
        check(lib().mrf_frame_stats(self.handle, s, C.byref(st)))
        return st.as_dict()

    def close(self):
        if getattr(self, "handle", None):
            lib().mrf_frame_destroy(self.handle)
            self.handle = None


def mrf_l2_read_bandwidth(ctx: int, nbytes: int, reps: int, stream: int = 0) -> float:
    """L2 read bandwidth in GB/s over an L2-resident buffer of nbytes (see include/mrf.h)."""
    g = C.c_double()
    check(lib().mrf_l2_read_bandwidth(ctx, nbytes, reps, stream, C.byref(g)))
    return g.value


def mrf_tonemap(ctx: int, in_ptr: int, n: int, exposure: float, out_ptr: int, stream: int = 0):
    check(lib().mrf_tonemap(ctx, in_ptr, n, exposure, out_ptr, stream))


class ShadowNet:
    """The learned shadow-transmittance network of a Renderer's field (the C ABI's mrf_shadow_net)."""

    def __init__(self, renderer: "Renderer", params=None, precision: int = MRF_PREC_FP32, log2_table: int = S.SNET_LOG2_T,
                 level_res=None, lr: float = 1e-2, betas=(0.9, 0.99), eps: float = 1e-15, seed: int = 0,
                 lr_decay: float = 1.0):
        self.r = renderer
        torch = renderer.torch
        d = mrf_shadow_net_desc()
        d.log2_table = log2_table
        d.level_res[:] = [int(x) for x in (level_res if level_res is not None else S.snet_level_resolutions())]
        keep = None
        if params is not None:
            keep = torch.as_tensor(np.asarray(params, np.float32)).to(torch.device("cuda", renderer.device))
            d.params = keep.data_ptr()
        d.seed = seed
        d.lr, d.beta1, d.beta2, d.eps = lr, betas[0], betas[1], eps
        d.precision = precision
        d.lr_decay = lr_decay
        h = _vp()
        check(lib().mrf_shadow_net_create(renderer.ctx, renderer.field, C.byref(d), C.byref(h)))
        self.handle = h.value
        self.n_params = int(lib().mrf_shadow_net_param_count(self.handle))
        del keep

    def close(self):
        if getattr(self, "handle", None):
            lib().mrf_shadow_net_destroy(self.handle)
            self.handle = None

    def _stream(self):
        return self.r.torch.cuda.current_stream(self.r.device).cuda_stream

    def params(self):
        torch = self.r.torch
        out = torch.empty(self.n_params, dtype=torch.float32, device=torch.device("cuda", self.r.device))
        check(lib().mrf_shadow_net_get_params(self.handle, out.data_ptr(), self._stream()))
        return out

    def set_params(self, p):
        torch = self.r.torch
        t = torch.as_tensor(p, dtype=torch.float32).to(torch.device("cuda", self.r.device)).contiguous()
        check(lib().mrf_shadow_net_set_params(self.handle, t.data_ptr(), self._stream()))
        torch.cuda.synchronize(self.r.device)

    def pairs(self, seed: int, first: int, n: int):
        """n x 8 float32 CUDA tensor of training pairs labelled by the FP32 march."""
        torch = self.r.torch
        out = torch.empty((n, 8), dtype=torch.float32, device=torch.device("cuda", self.r.device))
        opts = self.r.opts_struct()
        check(lib().mrf_shadow_pairs(self.r.ctx, self.r.field, C.byref(opts), seed, first, n, out.data_ptr(),
                                     self._stream()))
        return out

    def grad(self, pairs):
        torch = self.r.torch
        dev = torch.device("cuda", self.r.device)
        g = torch.empty(self.n_params, dtype=torch.float32, device=dev)
        loss = torch.empty(1, dtype=torch.float32, device=dev)
        check(lib().mrf_shadow_net_grad(self.handle, pairs.data_ptr(), pairs.shape[0], g.data_ptr(), loss.data_ptr(),
                                        self._stream()))
        return g, loss

    def train(self, pairs, batch: int, steps: int):
        torch = self.r.torch
        loss = torch.empty(max(steps, 1), dtype=torch.float32, device=torch.device("cuda", self.r.device))
        check(lib().mrf_shadow_net_train(self.handle, pairs.data_ptr(), pairs.shape[0], batch, steps, loss.data_ptr(),
                                         self._stream()))
        return loss[:steps]

    def save(self, path: str):
        check(lib().mrf_shadow_net_save(self.handle, os.fsencode(path)))

    def load(self, path: str):
        check(lib().mrf_shadow_net_load(self.handle, os.fsencode(path)))

    def eval(self, pairs):
        torch = self.r.torch
        out = torch.empty(pairs.shape[0], dtype=torch.float32, device=torch.device("cuda", self.r.device))
        check(lib().mrf_shadow_net_eval(self.handle, pairs.data_ptr(), pairs.shape[0], out.data_ptr(), self._stream()))
        return out
