"""mrf_render_static, the allocation-free render entry point, against mrf_render.

mrf_render_static serves callers that cannot call cudaMalloc while rendering
(their device memory belongs to another allocator's pool, or their loop cannot
afford an allocation's device-wide synchronisation): it runs the wavefront
engine out of a 64 MiB arena that lives in the library's static device memory.
This file is collected last so that a run stopping at its first failure has
run every other test before it; it passes alone in a fresh process as well.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2309_04581_gb300 import scenes as S

pytestmark = pytest.mark.gpu

RTOL_PIX = 1e-4   # the per-pixel bar of the parity tests (relative, floor 1e-2 x image peak)


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_04581_gb300 import build
    build.build()
    import paper_2309_04581_gb300.mrf as M
    return torch, M


def _close(a, b):
    peak = max(np.abs(b[:, :3]).max(), 1e-30)
    den = np.maximum(np.abs(b[:, :3]).max(1), 1e-2 * peak)
    return float((np.abs(a[:, :3] - b[:, :3]).max(1) / den).max())


def _render_both(torch, M, sc, precision, calls=2):
    r = M.Renderer(sc, precision=precision)
    n, B = sc.n_rays, sc.opts.max_bounces
    ref = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    rec_ref = r.new_records()
    M.mrf_render(r.ctx, r.field, r.bvh, r.rays_struct(), B, r.opts_struct(M.MRF_ENGINE_WAVEFRONT, rec_ref),
                 ref.data_ptr(), 0)
    outs = []
    for _ in range(calls):
        out = torch.full((n, 4), float("nan"), dtype=torch.float32, device="cuda")
        rec = r.new_records()
        st = M.mrf_stats()
        # through the C ABI directly
        status = M.lib().mrf_render_static(r.ctx, r.field, r.bvh, C.byref(r.rays_struct()), B,
                                           C.byref(r.opts_struct(M.MRF_ENGINE_AUTO, rec)), out.data_ptr(), None,
                                           C.byref(st))
        assert status == M.MRF_OK, M.lib().mrf_last_error().decode()
        torch.cuda.synchronize()
        outs.append((out.cpu().numpy().astype(np.float64), rec, st.as_dict()))
    torch.cuda.synchronize()
    return r, ref.cpu().numpy().astype(np.float64), rec_ref, outs


@pytest.mark.parametrize("precision", ["bf16", "fp32"])
def test_static_arena_matches_mrf_render_twice(env, precision):
    torch, M = env
    prec = {"bf16": M.MRF_PREC_BF16, "fp32": M.MRF_PREC_FP32}[precision]
    sc = S.config2(96, 96)
    r, ref, rec_ref, outs = _render_both(torch, M, sc, prec, calls=2)
    for img, rec, st in outs:
        assert np.all(np.isfinite(img))
        assert _close(img, ref) <= RTOL_PIX
        assert torch.equal(rec["segments"], rec_ref["segments"])
        assert torch.equal(rec["tri"], rec_ref["tri"])
        assert st["paths"] == sc.n_rays and st["segments"] == int(rec["segments"].sum())
    r.close()


def test_static_arena_after_a_different_call(env):
    # the arena keeps the last call's contents: a smaller render in between must not leak into the next one
    torch, M = env
    small = S.config1(16, 16)
    r0 = M.Renderer(small)
    out0 = torch.empty((small.n_rays, 4), dtype=torch.float32, device="cuda")
    assert M.lib().mrf_render_static(r0.ctx, r0.field, r0.bvh, C.byref(r0.rays_struct()), small.opts.max_bounces,
                                     C.byref(r0.opts_struct()), out0.data_ptr(), None, None) == M.MRF_OK
    torch.cuda.synchronize()
    r0.close()
    sc = S.config2(64, 48)
    r, ref, _, outs = _render_both(torch, M, sc, M.MRF_PREC_BF16, calls=1)
    assert _close(outs[0][0], ref) <= RTOL_PIX
    r.close()


def test_static_arena_rejects_oversize_and_host_output(env):
    torch, M = env
    sc = S.config2(400, 400)          # 160,000 paths > 131,072
    r = M.Renderer(sc, precision=M.MRF_PREC_BF16)
    out = torch.empty((sc.n_rays, 4), dtype=torch.float32, device="cuda")
    st = M.lib().mrf_render_static(r.ctx, r.field, r.bvh, C.byref(r.rays_struct()), 8, C.byref(r.opts_struct()),
                                   out.data_ptr(), None, None)
    assert st == M.MRF_ERR_INVALID_ARG
    assert b"static arena" in M.lib().mrf_last_error()
    host = np.zeros((sc.n_rays, 4), np.float32)
    st = M.lib().mrf_render_static(r.ctx, r.field, r.bvh, C.byref(r.rays_struct()), 8, C.byref(r.opts_struct()),
                                   host.ctypes.data, None, None)
    assert st == M.MRF_ERR_INVALID_ARG
    r.close()


def test_static_arena_overflow_is_marched_in_place(env):
    # 129,600 paths: the arena's sample buffer (~1.3M samples after the per-path
    # state) is smaller than the first segment's ~7M samples, so most jobs take
    # the in-place FP32 march; the image must still match mrf_render's.
    torch, M = env
    sc = S.config2(360, 360)
    for prec, tol in ((M.MRF_PREC_FP32, RTOL_PIX), (M.MRF_PREC_BF16, 2e-3)):
        r, ref, rec_ref, outs = _render_both(torch, M, sc, prec, calls=1)
        img, rec, _ = outs[0]
        assert _close(img, ref) <= tol
        assert torch.equal(rec["segments"], rec_ref["segments"])
        r.close()


def test_static_arena_rounds_match_mrf_render_exactly(env):
    # with enough generation rounds every job of the 129,600 paths is evaluated
    # from the arena's small sample buffer in turns, none is marched in place:
    # the image is mrf_render's bit for bit
    torch, M = env
    sc = S.config2(360, 360)
    for prec in (M.MRF_PREC_BF16, M.MRF_PREC_FP32):
        r = M.Renderer(sc, precision=prec)
        r.set_tuning(8, 96, 16)
        ref = torch.empty((sc.n_rays, 4), dtype=torch.float32, device="cuda")
        M.mrf_render(r.ctx, r.field, r.bvh, r.rays_struct(), 8, r.opts_struct(M.MRF_ENGINE_WAVEFRONT), ref.data_ptr(),
                     0)
        out = torch.full_like(ref, float("nan"))
        st = M.mrf_stats()
        assert M.lib().mrf_render_static(r.ctx, r.field, r.bvh, C.byref(r.rays_struct()), 8, C.byref(r.opts_struct()),
                                         out.data_ptr(), None, C.byref(st)) == M.MRF_OK
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
        r.close()


def _eight_lights(sc):
    l0 = sc.lights[0]
    sc.lights = [S.Light(pos=(l0.pos[0] + 0.05 * (k - 3.5), l0.pos[1], l0.pos[2]),
                         intensity=tuple(x / 8 for x in l0.intensity)) for k in range(8)]
    return sc


def test_static_arena_limit_depends_on_the_light_count(env):
    # eight point lights make the per-path state 556 B: 125,316 paths no longer
    # fit the 64 MiB arena (a clear MRF_ERR_INVALID_ARG, not a launch failure),
    # while 90,000 paths still render and match mrf_render
    torch, M = env
    sc = _eight_lights(S.config2(354, 354))
    r = M.Renderer(sc)
    out = torch.empty((sc.n_rays, 4), dtype=torch.float32, device="cuda")
    st = M.lib().mrf_render_static(r.ctx, r.field, r.bvh, C.byref(r.rays_struct()), 8, C.byref(r.opts_struct()),
                                   out.data_ptr(), None, None)
    assert st == M.MRF_ERR_INVALID_ARG
    assert b"do not fit the static arena" in M.lib().mrf_last_error()
    r.close()
    sc = _eight_lights(S.config2(300, 300))
    r, ref, rec_ref, outs = _render_both(torch, M, sc, M.MRF_PREC_FP32, calls=1)
    img, rec, st = outs[0]
    assert _close(img, ref) <= RTOL_PIX
    assert torch.equal(rec["segments"], rec_ref["segments"])
    assert st["shadow_rays"] > 0
    r.close()
