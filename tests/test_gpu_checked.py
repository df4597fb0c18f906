"""The bounds-checked build (libmrf_checked.so: every table, node and
triangle index tested before use, a bad one reported in the status word)
renders the benchmark scenes with no bad index and the same image as the
release build.  It stands in for a memory checker, which this pool does not
offer."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import hashlib, json, sys
sys.path.insert(0, ROOT)
import torch
import paper_2309_04581_gb300.mrf as M
from paper_2309_04581_gb300 import scenes as S
res = {}
for name, sc, prec in [("c2_bf16", S.config2(160, 120), M.MRF_PREC_BF16), ("c2_fp32", S.config2(96, 64), M.MRF_PREC_FP32),
                       ("c4_bf16", S.config4(64, 48), M.MRF_PREC_BF16)]:
    r = M.Renderer(sc, precision=prec)
    out, st = r.render(stats=True)
    torch.cuda.synchronize()
    res[name] = {"status": st["status"], "hash": hashlib.sha256(out.cpu().numpy().tobytes()).hexdigest()}
    r.close()
print(json.dumps(res))
"""


def _run(lib):
    env = dict(os.environ, MRF_LIB=lib)
    out = subprocess.run([sys.executable, "-c", SCRIPT.replace("ROOT", repr(ROOT))], env=env, capture_output=True,
                         text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_bounds_checked_build_finds_no_bad_index():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_04581_gb300 import build
    rel = build.build()
    chk = build.build(checked=True)
    a, b = _run(rel), _run(chk)
    for k in a:
        assert b[k]["status"] == 0, (k, b[k])
        assert a[k]["hash"] == b[k]["hash"], k
