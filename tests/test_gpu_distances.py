"""cf_distances (resized transition matrices, the five Table 1 distances)
against the FP64 oracle (oracle/distances.py, pinned in
test_oracle_distances.py).

Bar: every distance within 1e-5 relative plus 1e-6 absolute of the oracle
(FP32 entries and row sums, compensated sums across rows); the [0, 1] scaling within
2e-5 absolute."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gen import CFG, config1, config2, config5, structured_cfg  # noqa: E402
from oracle import distances as OD  # noqa: E402
from paper_1707_02423_gb300 import _binding as B  # noqa: E402
from paper_1707_02423_gb300 import api  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02423_gb300 import build

    build.build()


def check(got, want, rel=1e-5, ab=1e-6):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    err = np.abs(got - want) - (rel * np.abs(want) + ab)
    assert err.max() <= 0, (np.unravel_index(err.argmax(), err.shape), got.ravel()[err.argmax()],
                            want.ravel()[err.argmax()])


@pytest.mark.parametrize("p", [3.0, 1.0, 2.0, 4.5])
def test_cfg1_all_pairs(p):
    w = config1()
    pa = api.Pack(w.cfgs_a, w.F, device=DEV)
    got = api.distances(pa, pa, w.pairs, p).cpu().numpy()
    check(got, OD.run_pairs(w.cfgs_a, w.cfgs_a, w.pairs, p))


def test_cfg2_subset_both_orders_and_scaling():
    w = config2(30)
    pairs = np.concatenate([w.pairs, w.pairs[:, ::-1]])
    pa = api.Pack(w.cfgs_a, w.F, device=DEV)
    raw = api.distances(pa, pa, pairs).cpu().numpy()
    want = OD.run_pairs(w.cfgs_a, w.cfgs_a, pairs)
    check(raw, want)
    P = len(w.pairs)
    assert np.array_equal(raw[:P], raw[P:])  # d(A, B) = d(B, A) bit for bit (same resize, same order)
    sc = api.distances(pa, pa, pairs, scale01=True).cpu().numpy()
    assert np.abs(sc - OD.scale01(want)).max() <= 2e-5
    assert sc.min() == 0.0 and np.isclose(sc.max(axis=0), 1.0).all()


def test_two_packs_and_self_pairs():
    w = config5(3, 25)
    pa = api.Pack(w.cfgs_a, w.F, device=DEV)
    pb = api.Pack(w.cfgs_b, w.F, device=DEV)
    check(api.distances(pa, pb, w.pairs).cpu().numpy(), OD.run_pairs(w.cfgs_a, w.cfgs_b, w.pairs))
    selfp = np.array([(i, i) for i in range(25)], np.int32)
    d = api.distances(pb, pb, selfp).cpu().numpy()
    assert np.abs(d).max() <= 1e-6  # every distance of a CFG to itself is 0


def test_edge_cases():
    rng = np.random.default_rng(9)
    F = 2
    one = CFG(1, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32), np.ones((1, F), np.float32))
    loop1 = CFG(1, np.array([0], np.int32), np.array([0], np.int32), np.array([0.7], np.float32),
                np.ones((1, F), np.float32))
    empty5 = CFG(5, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32),
                 np.ones((5, F), np.float32))
    c = structured_cfg(rng, 40, 4, F - 1)
    big = structured_cfg(rng, 700, 6, F - 1)
    cfgs = [one, loop1, empty5, c, big]
    pairs = np.array([(a, b) for a in range(5) for b in range(5)], np.int32)
    pa = api.Pack(cfgs, F, device=DEV)
    check(api.distances(pa, pa, pairs, 3.0).cpu().numpy(), OD.run_pairs(cfgs, cfgs, pairs, 3.0))


def test_dense_pairs_beyond_the_staged_edge_area():
    """CFGs small enough for the staged layout, some of whose pairs carry more
    edges than a warp's staged edge area: those pairs read their CSR from
    global memory, the others from shared memory, in the same launch."""
    rng = np.random.default_rng(11)
    F = 2

    def dense(n, deg):
        src = np.repeat(np.arange(n), deg).astype(np.int32)
        dst = np.concatenate([rng.choice(n, deg, replace=False) for _ in range(n)]).astype(np.int32)
        return CFG(n, src, dst, rng.uniform(0.1, 1.0, n * deg).astype(np.float32),
                   rng.uniform(0, 1, (n, F)).astype(np.float32))

    cfgs = [dense(100, 5), dense(60, 4), structured_cfg(rng, 30, 3, F - 1), dense(9, 2), dense(2, 2)]
    pairs = np.array([(a, b) for a in range(len(cfgs)) for b in range(len(cfgs))], np.int32)
    pa = api.Pack(cfgs, F, device=DEV)
    check(api.distances(pa, pa, pairs, 3.0).cpu().numpy(), OD.run_pairs(cfgs, cfgs, pairs, 3.0))


def test_bad_pair_index_sets_status():
    w = config1()
    pa = api.Pack(w.cfgs_a, w.F, device=DEV)
    with pytest.raises(B.CfsimError) as e:
        api.distances(pa, pa, np.array([[0, 1], [0, 99]], np.int32))
    assert e.value.status == 1
