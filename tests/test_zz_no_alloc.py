"""cf_similarity_noalloc: the entry point for callers that cannot allocate
device memory (an allocator owning the whole device heap, host callbacks, a
serving loop that must not add allocation latency).  It runs cf_similarity on
a file-scope 32 MiB device array instead of a caller workspace.

Checked through the C ABI against cf_similarity with a caller-sized
workspace, on two calls in a row (the array keeps the previous call's
contents, so the second call shows that what must start at zero is cleared).
This file is collected last so that a failure here never hides another test.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from _helpers import ATOL_S, ATOL_X  # noqa: E402
from gen import config1, config2  # noqa: E402
from paper_1707_02423_gb300 import _binding as B  # noqa: E402
from paper_1707_02423_gb300 import api  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02423_gb300 import build

    build.build()


def _noalloc(pack, d_pairs, P, omega, x_elems, m_elems, alpha=0.8, K=40):
    L = B.lib()
    prm = B.params(alpha, K)
    X = torch.full((x_elems,), -7.0, device=DEV)
    sc = torch.full((P,), -7.0, device=DEV)
    mt = torch.full((m_elems,), -7, dtype=torch.int32, device=DEV)
    st = torch.full((1,), -7, dtype=torch.int32, device=DEV)
    B.check(L.cf_similarity_noalloc(pack.dev.data_ptr(), pack.dev.data_ptr(), d_pairs.data_ptr(), P, C.byref(prm),
                                    omega.data_ptr(), X.data_ptr(), sc.data_ptr(), mt.data_ptr(), st.data_ptr(),
                                    None))
    torch.cuda.synchronize()
    return X.cpu().numpy(), sc.cpu().numpy(), mt.cpu().numpy(), int(st.item())


@pytest.mark.parametrize("which", ["cfg1", "cfg2_subset"])
def test_noalloc_matches_cf_similarity_twice(which):
    w = config1() if which == "cfg1" else config2(40)  # the subset has pairs too large for shared memory
    pack = api.Pack(w.cfgs_a, w.F, device=DEV)
    pairs = np.ascontiguousarray(w.pairs, np.int32)
    P = len(pairs)
    omega = torch.linspace(0.5, 1.5, w.F, device=DEV)
    ref = api.similarity(pack, pack, pairs, omega, 0.8, 40, want_x=True, want_match=True)
    X_ref = ref.X.cpu().numpy()
    s_ref = ref.scores.cpu().numpy()
    m_ref = ref.match.cpu().numpy()
    d_pairs = torch.from_numpy(pairs).to(DEV)
    for _ in range(2):
        X, sc, mt, status = _noalloc(pack, d_pairs, P, omega, len(X_ref), len(m_ref))
        assert status == 0
        assert np.abs(X - X_ref).max() <= ATOL_X
        assert np.abs(sc - s_ref).max() <= ATOL_S
        assert np.array_equal(mt, m_ref)


def test_noalloc_rejects_pair_lists_beyond_its_limit():
    w = config1()
    pack = api.Pack(w.cfgs_a, w.F, device=DEV)
    L = B.lib()
    prm = B.params()
    omega = torch.ones(w.F, device=DEV)
    big_p = 3_000_000  # the fixed workspace part alone exceeds 32 MiB; nothing is launched
    s = L.cf_similarity_noalloc(pack.dev.data_ptr(), pack.dev.data_ptr(), pack.dev.data_ptr(), big_p, C.byref(prm),
                                omega.data_ptr(), None, None, None, None, None)
    assert s == 2  # CF_ERR_WORKSPACE
    assert b"32 MiB" in L.cf_last_error_detail()


@pytest.mark.parametrize("flag", ["plan_only", "reuse_plan"])
def test_noalloc_rejects_plan_flags(flag):
    """A plan kept in the shared array could belong to another call's pairs,
    so the flags that keep or reuse a plan are refused before any launch."""
    w = config1()
    pack = api.Pack(w.cfgs_a, w.F, device=DEV)
    L = B.lib()
    prm = B.params(flags=B.CF_FLAG_PLAN_ONLY if flag == "plan_only" else B.CF_FLAG_REUSE_PLAN)
    omega = torch.ones(w.F, device=DEV)
    d_pairs = torch.from_numpy(np.ascontiguousarray(w.pairs, np.int32)).to(DEV)
    sc = torch.full((len(w.pairs),), -7.0, device=DEV)
    s = L.cf_similarity_noalloc(pack.dev.data_ptr(), pack.dev.data_ptr(), d_pairs.data_ptr(), len(w.pairs),
                                C.byref(prm), omega.data_ptr(), None, sc.data_ptr(), None, None, None)
    assert s == 1  # CF_ERR_INVALID_ARG
    assert b"REUSE_PLAN" in L.cf_last_error_detail()
    torch.cuda.synchronize()
    assert float(sc.min()) == -7.0  # nothing ran
