"""The debug build (-DCF_DEBUG_BOUNDS: in-kernel checks of pair layouts,
scratch slots and staged neighbour indices that record a status and skip the
access) on a clean run: a forward over pairs of every execution class and an
adjoint, in a subprocess that loads the debug library through CFSIM_LIBRARY.
The status words stay CF_OK and the outputs equal the product library's."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RUN = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from gen import config2, config4
from paper_1707_02423_gb300 import api
dev = "cuda:0"
w = config2(40)
pa = api.Pack(w.cfgs_a, w.F, device=dev)
om = torch.linspace(0.5, 1.5, w.F, device=dev)
res = api.similarity(pa, pa, w.pairs, om, 0.8, 40, want_x=True, want_match=True)  # checks the status word
g = config4(8)
pg = api.Pack(g.cfgs_a, g.F, device=dev)
og = torch.ones(g.F, device=dev)
rg = api.similarity(pg, pg, g.pairs, og, 0.8, 40, want_match=True)
gw, _, go = api.similarity_backward(pg, pg, g.pairs, og, rg.match, torch.ones(len(g.pairs), device=dev), 0.8, 40)
np.savez(sys.argv[2], X=res.X.cpu().numpy(), s=res.scores.cpu().numpy(), m=res.match.cpu().numpy(),
         gw=gw.cpu().numpy(), go=go.cpu().numpy())
"""


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02423_gb300 import build

    build.build()


def _run(lib, out):
    env = dict(os.environ)
    if lib:
        env["CFSIM_LIBRARY"] = lib
    else:
        env.pop("CFSIM_LIBRARY", None)
    r = subprocess.run([sys.executable, "-c", RUN, ROOT, out], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return np.load(out)


def test_debug_bounds_build_runs_clean(tmp_path):
    from paper_1707_02423_gb300 import build

    dbg = build.build(variant="debug_bounds")
    a = _run(dbg, str(tmp_path / "debug.npz"))
    b = _run(None, str(tmp_path / "product.npz"))
    assert np.abs(a["X"] - b["X"]).max() <= 1e-6
    assert np.abs(a["s"] - b["s"]).max() <= 1e-6
    assert np.array_equal(a["m"], b["m"])
    for k in ("gw", "go"):
        assert np.abs(a[k] - b[k]).max() <= 1e-6 * max(1.0, float(np.abs(b[k]).max()))
