"""cf_score_matrix and cf_ward (Ward linkage of similarity profiles) against
the FP64 oracle (oracle/ward.py, pinned in test_oracle_ward.py).

Bar: a valid, monotone linkage whose cophenetic distances and sorted merge
heights are within 1e-4 (relative to the largest height) of scipy's on the
same FP32 points; on small sets with well-separated heights every merge
(cluster ids, size) equals scipy's; the score-matrix scatter is bit-exact."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gen import config2  # noqa: E402
from oracle import ward as OW  # noqa: E402
from paper_1707_02423_gb300 import _binding as B  # noqa: E402
from paper_1707_02423_gb300 import api  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02423_gb300 import build

    build.build()


def gpu_linkage(X):
    merge, height, size = api.ward(torch.tensor(X, dtype=torch.float32, device=DEV))
    return np.column_stack([merge.cpu().numpy(), height.cpu().numpy(), size.cpu().numpy()]).astype(np.float64)


def compare_linkage(X, exact):
    """Cophenetic distances (the height at which two points first share a
    cluster: unchanged when near-tied merges swap order) within 1e-4 of the
    largest height; with `exact`, every merge equal to scipy's."""
    from scipy.cluster.hierarchy import cophenet, is_valid_linkage

    Zg = gpu_linkage(X)
    Z = OW.linkage(X.astype(np.float32).astype(np.float64))
    assert is_valid_linkage(Zg)
    assert np.all(np.diff(Zg[:, 2]) >= -1e-6 * Zg[:, 2].max())  # monotone heights
    if len(X) > 2:
        assert np.abs(cophenet(Zg) - cophenet(Z)).max() <= 1e-4 * Z[:, 2].max()
    assert np.allclose(np.sort(Zg[:, 2]), np.sort(Z[:, 2]), rtol=1e-4, atol=1e-6)
    if exact:
        assert np.array_equal(Zg[:, [0, 1, 3]], Z[:, [0, 1, 3]]), (Zg[:4], Z[:4])


@pytest.mark.parametrize("n,dim,seed,exact", [(2, 1, 0, True), (3, 2, 1, True), (17, 5, 2, True),
                                              (64, 8, 3, False), (200, 200, 4, False)])
def test_random_points(n, dim, seed, exact):
    X = np.random.default_rng(seed).random((n, dim))
    compare_linkage(X, exact)


def test_single_point_has_no_merges():
    merge, height, size = api.ward(torch.ones(1, 3, device=DEV))
    assert merge.numel() == 0 and height.numel() == 0


def test_score_matrix_scatter_and_bad_pair():
    pairs = np.array([[0, 1], [2, 2], [1, 3]], np.int32)
    sc = torch.tensor([0.5, 1.25, 0.75], device=DEV)
    S = api.score_matrix(pairs, sc, 4).cpu().numpy()
    assert np.array_equal(S, OW.score_matrix(4, pairs, [0.5, 1.25, 0.75]))
    R = api.score_matrix(pairs, sc, 3, 4, symmetric=False).cpu().numpy()
    assert R.shape == (3, 4) and R[0, 1] == 0.5 and R[1, 3] == 0.75 and R[2, 2] == 1.25
    assert R[1, 0] == 0.0  # not mirrored
    with pytest.raises(B.CfsimError):
        api.score_matrix(np.array([[0, 9]], np.int32), sc[:1], 4)


def test_profiles_of_all_pair_scores():
    # the paper's use: cluster CFGs by their rows of the all-pairs score matrix
    w = config2(24)
    n = len(w.cfgs_a)
    pairs = np.array([(i, j) for i in range(n) for j in range(i, n)], np.int32)  # with self pairs
    pa = api.Pack(w.cfgs_a, w.F, device=DEV)
    res = api.similarity(pa, pa, pairs, torch.ones(w.F, device=DEV))
    S = api.score_matrix(pairs, res.scores, n)
    assert torch.equal(S, S.T)
    compare_linkage(S.cpu().numpy().astype(np.float64), exact=False)
