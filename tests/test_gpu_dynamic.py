"""Deforming meshes frame by frame: per-frame BVH refit against a rebuild from
the same vertices, and a refitted frame against the FP64 oracle."""
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


def test_refit_sequence_matches_rebuild_and_oracle(env, orc):
    torch, M = env
    seq = S.DynamicSequence(48, 40, spp=1, cloth_n=24, bodies=3, lights=2)
    a = M.Renderer(seq.scene)      # refitted every frame
    b = M.Renderer(seq.scene)      # rebuilt on the host every frame
    c = M.Renderer(seq.scene)      # rebuilt on the GPU every frame
    for k in range(1, 5):
        v = seq.vertices(k, fps=4.0)   # large steps: the boxes move a lot between frames
        a.set_vertices(v)
        b.set_vertices(v, rebuild="host")
        c.set_vertices(v, rebuild="gpu")
        ia, _ = a.render()
        ib, _ = b.render()
        ic, _ = c.render()
        torch.cuda.synchronize()
        # same closest hits whichever tree finds them: identical images
        assert torch.equal(ia, ib), k
        assert torch.equal(ia, ic), k
    c.close()
    sc = S.Scene(name="frame4", camera=seq.scene.camera, field=seq.scene.field,
                 mesh=S.Mesh(seq.vertices(4, fps=4.0), seq.tris, seq.mat), materials=seq.scene.materials,
                 lights=seq.scene.lights, opts=seq.scene.opts)
    ref = orc.render(sc)
    img = ia.cpu().numpy().astype(np.float64)
    ok = ref["flags"] == 0
    assert ok.mean() > 0.99
    peak = np.abs(ref["rgba"][:, :3]).max()
    den = np.maximum(np.abs(ref["rgba"][:, :3]).max(1), 1e-2 * peak)
    assert (np.abs(img[:, :3] - ref["rgba"][:, :3]).max(1) / den)[ok].max() <= 1e-4
    a.close()
    b.close()
