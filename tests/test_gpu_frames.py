"""Captured frames (mrf_frame_capture / mrf_frame_replay): a render call
captured once into a CUDA graph replays to the same image as mrf_render, and
follows the scene's device memory (a BVH refit) between replays."""
import ctypes as C

import numpy as np
import pytest

from paper_2309_04581_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_04581_gb300 import build
    build.build()
    import paper_2309_04581_gb300.mrf as M
    return torch, M


@pytest.mark.parametrize("prec,engine", [("bf16", "wavefront"), ("fp32", "megakernel"), ("fp32", "wavefront")])
def test_replay_matches_render(env, prec, engine):
    torch, M = env
    sc = S.config2(96, 80)
    sc.cameras = S.orbit_views(3, [(96, 80), (33, 17), (1, 1)])   # a multi-view batch: table copied at capture
    r = M.Renderer(sc, precision=M.MRF_PREC_BF16 if prec == "bf16" else M.MRF_PREC_FP32)
    eng = M.MRF_ENGINE_WAVEFRONT if engine == "wavefront" else M.MRF_ENGINE_MEGAKERNEL
    ref, st_ref = r.render(engine=eng, stats=True)
    out = torch.full_like(ref, float("nan"))
    f = M.Frame(r, out, engine=eng)
    for _ in range(3):
        f.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
        st = f.stats()
        for k in ("paths", "segments", "surface_hits", "shadow_rays", "samples_evaluated", "shadow_samples_evaluated"):
            assert st[k] == st_ref[k], k
    f.close()
    r.close()


def test_replay_follows_refit_and_keeps_captured_lights(env):
    torch, M = env
    sc = S.config2(64, 64)
    r = M.Renderer(sc, precision=M.MRF_PREC_BF16)
    out = torch.empty((sc.n_rays, 4), dtype=torch.float32, device="cuda")
    f = M.Frame(r, out)
    f.replay()
    torch.cuda.synchronize()
    first = out.clone()
    # deform the meshes: the replay reads the refitted BVH
    moved = sc.mesh.verts.copy()
    moved[:, 1] += np.float32(0.05) * np.sin(7.0 * moved[:, 0]).astype(np.float32)
    moved = np.ascontiguousarray(moved.astype(np.float32))
    M.mrf_bvh_refit(r.bvh, moved.ctypes.data, moved.shape[0], torch.cuda.current_stream().cuda_stream)
    ref, _ = r.render()
    f.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, ref) and not torch.equal(out, first)
    # lights were copied at capture: switching them off afterwards changes mrf_render only
    dark = [S.Light(pos=l.pos, intensity=(0.0, 0.0, 0.0)) for l in sc.lights]
    M.mrf_lights_set(r.ctx, dark)
    ref_dark, _ = r.render()
    f.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, ref) and not torch.equal(ref_dark, ref)
    f.close()
    r.close()


def test_capture_rejects_host_outputs(env):
    torch, M = env
    sc = S.config1(16, 16)
    r = M.Renderer(sc)
    host = np.zeros((sc.n_rays, 4), np.float32)
    h = C.c_void_p()
    st = M.lib().mrf_frame_capture(r.ctx, r.field, r.bvh, C.byref(r.rays_struct()), 4, C.byref(r.opts_struct()),
                                   host.ctypes.data, C.byref(h))
    assert st == M.MRF_ERR_INVALID_ARG and not h.value
    r.close()


def test_autotuner_picks_a_candidate_and_keeps_results(env):
    """The autotuner times the six launch-shape / queue-size candidates on the
    request and keeps the fastest; none of them changes the image."""
    torch, M = env
    sc = S.config2(256, 256)
    r = M.Renderer(sc, precision=M.MRF_PREC_BF16)
    assert r.tuning() == {"field_groups": 8, "samples_per_path": 96, "rounds": 1, "tail_paths": 0}
    before, st0 = r.render(stats=True)
    best, ms = r.autotune(reps=2)
    assert best == r.tuning()
    cands = [(g, c, k) for g in (8, 4) for c in (48, 96, 192) for k in (1, 8)]
    assert (best["field_groups"], best["samples_per_path"], best["rounds"]) in cands
    assert all(x > 0 for x in ms) and min(ms) == pytest.approx(
        ms[cands.index((best["field_groups"], best["samples_per_path"], best["rounds"]))])
    print("autotune ms", ms, "best", best)
    for g in (4, 8):
        for c in (48, 192):
            r.set_tuning(g, c, 8)
            img, st = r.render(stats=True)
            torch.cuda.synchronize()
            assert torch.equal(img, before), (g, c)
            assert st["samples_evaluated"] == st0["samples_evaluated"]
    with pytest.raises(M.MrfError):
        r.set_tuning(6, 96)
    r.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_mirror_room_views_match_oracle(env, orc, prec):
    """The batched-view workload at a tiny scale: five views of uneven size in a
    mirror room with displaced spheres and a cloth, 16 segments per path,
    through a captured frame after a cloth refit, against the oracle.

    Every segment of a 16-bounce mirror path carries the FP32 error of all
    the bounces before it (the angular error grows by every reflection, the
    lateral one by the distance travelled times the angular one), so the
    oracle's error bound reaches the edges of the spheres' small facets on a
    fifth of the paths, mostly in their late segments.  Hence: on every pixel
    the hit ids of all segments before the path's first flagged decision; on
    unflagged pixels every segment's hit id, the segment counts and the
    radiance (FP32: 1e-4 per pixel; BF16: >= 45 dB and <= 1e-2 max abs)."""
    torch, M = env
    from tests.test_gpu_parity import _compare, _trusted
    mv = S.MultiViewScene(n_views=5, scale=0.02)   # 25x16, 25x16, 23x15, 17x12, 8x7
    r = M.Renderer(mv.scene, precision=M.MRF_PREC_FP32 if prec == "fp32" else M.MRF_PREC_BF16)
    v = mv.vertices(5)
    r.set_vertices(v)
    out = torch.empty((mv.scene.n_rays, 4), dtype=torch.float32, device="cuda")
    rec = r.new_records()
    f = M.Frame(r, out, engine=M.MRF_ENGINE_WAVEFRONT, records=rec)
    f.replay()
    torch.cuda.synchronize()
    sc = mv.scene
    sc2 = S.Scene(name="moved", camera=sc.camera, field=sc.field, mesh=S.Mesh(v, sc.mesh.tris, sc.mesh.mat),
                  materials=sc.materials, lights=sc.lights, opts=sc.opts, cameras=sc.cameras)
    ref = orc.render(sc2)
    B = sc.opts.max_bounces
    gpu = dict(rgba=out.cpu().numpy().astype(np.float64),
               segments=rec["segments"].cpu().numpy().view(np.uint32).reshape(-1, 1),
               tri=rec["tri"].cpu().numpy().view(np.uint32).reshape(-1, 1, B),
               t=rec["t"].cpu().numpy().reshape(-1, 1, B))
    ok = ref["flags"] == 0
    frac = float((~ok).mean())
    print(f"{prec}: {frac:.1%} of the pixels flagged; first flagged segment histogram "
          f"{np.bincount(ref['first_flag'][:, 0], minlength=B + 1).tolist()}")
    assert frac <= 0.3
    assert ref["segments"].mean() > 8     # long mirror-room paths
    tr = _trusted(ref)
    assert tr.mean() > 0.8
    assert np.array_equal(np.where(tr, gpu["tri"], 0), np.where(tr, ref["tri"], 0))
    assert np.array_equal(gpu["tri"][ok], ref["tri"][ok])
    assert np.array_equal(gpu["segments"][ok], ref["segments"][ok])
    if prec == "fp32":
        # hit distances: the 1e-5 relative bar on the camera segment; later ones
        # carry the FP32 error of every bounce before them (the hit point's
        # bound reaches about 5e-5 world units after 16 mirror bounces) and are
        # held to 1e-4 absolute
        _compare(gpu, ref, max_flag_frac=0.3, t_segments=1)
        tg, to = gpu["t"][ok], ref["t"][ok]
        fin = np.isfinite(to)
        assert np.array_equal(np.isfinite(tg), fin)
        dt = np.where(fin, np.abs(np.where(fin, tg, 0) - np.where(fin, to, 0)), 0)
        print("fp32 mirror room: largest hit-distance difference per segment",
              [f"{x:.2g}" for x in dt.max(axis=(0, 1))])
        assert dt.max() <= 1e-4
    else:
        a, b = gpu["rgba"][ok, :3], ref["rgba"][ok, :3]
        peak = np.abs(b).max()
        psnr = 10 * np.log10(peak * peak / np.mean((a - b) ** 2))
        print(f"bf16 mirror room: PSNR {psnr:.1f} dB, max abs {np.abs(a - b).max():.3g}")
        assert psnr >= 45.0 and np.abs(a - b).max() <= 1e-2
    f.close()
    r.close()


def test_bounded_wait_gives_up_cleanly(env):
    """A wait on a barrier nothing arrives at runs out of its budget, the
    status word reports it as MRF_ERR_TIMEOUT, and the context renders on."""
    torch, M = env
    sc = S.config1(16, 16)
    r = M.Renderer(sc)
    before, _ = r.render()
    st = M.lib().mrf_selftest_timeout(r.ctx, 20000, 1)
    assert st == M.MRF_ERR_TIMEOUT and b"gave up" in M.lib().mrf_last_error()
    after, stats = r.render(stats=True)
    torch.cuda.synchronize()
    assert stats["status"] == 0 and torch.equal(before, after)
    r.close()


def test_sync_status_reports_a_wait_that_gave_up(env):
    """Without waiting, a kernel that gave up is reported later: by
    mrf_sync_status, which waits for the device, or by the next render call
    once the status copy that the earlier call enqueued has landed; either
    clears the word and the context renders on."""
    torch, M = env
    sc = S.config1(16, 16)
    r = M.Renderer(sc)
    before, _ = r.render()
    torch.cuda.synchronize()
    w = C.c_uint32(0)
    assert M.lib().mrf_sync_status(r.ctx, C.byref(w)) == M.MRF_OK and w.value == 0
    # reported by mrf_sync_status
    assert M.lib().mrf_selftest_timeout(r.ctx, 20000, 0) == M.MRF_OK
    assert M.lib().mrf_sync_status(r.ctx, C.byref(w)) == M.MRF_ERR_TIMEOUT and w.value != 0
    assert b"gave up" in M.lib().mrf_last_error()
    assert M.lib().mrf_sync_status(r.ctx, C.byref(w)) == M.MRF_OK and w.value == 0
    # reported by the next render call, without a host wait in that call
    assert M.lib().mrf_selftest_timeout(r.ctx, 20000, 0) == M.MRF_OK
    torch.cuda.synchronize()
    out = torch.empty_like(before)
    st = M.lib().mrf_render(r.ctx, r.field, r.bvh, C.byref(r.rays_struct()), sc.opts.max_bounces,
                            C.byref(r.opts_struct()), out.data_ptr(), None, None)
    assert st == M.MRF_ERR_TIMEOUT and b"earlier kernel gave up" in M.lib().mrf_last_error()
    after, stats = r.render(stats=True)
    torch.cuda.synchronize()
    assert stats["status"] == 0 and torch.equal(before, after)
    # the same through the allocation-free entry point
    assert M.lib().mrf_selftest_timeout(r.ctx, 20000, 0) == M.MRF_OK
    torch.cuda.synchronize()
    st = M.lib().mrf_render_static(r.ctx, r.field, r.bvh, C.byref(r.rays_struct()), sc.opts.max_bounces,
                                   C.byref(r.opts_struct()), out.data_ptr(), None, None)
    assert st == M.MRF_ERR_TIMEOUT
    assert M.lib().mrf_sync_status(r.ctx, C.byref(w)) == M.MRF_OK
    r.close()


def test_injected_allocation_failure(env):
    torch, M = env
    sc = S.config2(8, 8)
    ctx = M.mrf_context_create(0)
    desc, keep = M.field_desc(sc.field)
    M.lib().mrf_debug_fail_allocations(1)
    with pytest.raises(M.MrfError) as ei:
        M.mrf_field_create(ctx, desc)
    assert ei.value.status == M.MRF_ERR_OOM and "injected" in str(ei.value)
    f = M.mrf_field_create(ctx, desc)          # the next one succeeds
    M.mrf_field_destroy(f)
    M.lib().mrf_debug_fail_allocations(0)
    M.mrf_context_destroy(ctx)
