"""k-NN graph parity against the FP64 oracle (gpu)."""
import numpy as np
import pytest

import datagen
from gpu_util import check_knn, drgb_module
from oracle import knn as oknn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def drgb():
    return drgb_module()


def _run(drgb, X, k, mode):
    import torch
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    idx, dist = drgb.knn_graph(Xd, k, mode=mode)
    torch.cuda.synchronize()
    return idx.cpu().numpy(), dist.cpu().numpy()


CASES = [
    (16, 50, 15),      # n = k + 1: every other point is a neighbour
    (64, 50, 15),
    (500, 3, 15),
    (777, 100, 7),     # d > one 32-wide tile, ragged in both n and d
    (1000, 64, 32),    # maximum k
    (2000, 50, 15),    # the 2,000-point workload
    (333, 1, 1),       # k = 1, d = 1
]


def _tc_supported(d, k):
    return d + 3 <= 64 and k < 32


@pytest.mark.parametrize("mode", [1, 0, 2, 3])
@pytest.mark.parametrize("n,d,k", CASES)
def test_knn_matches_oracle(drgb, n, d, k, mode):
    X, _ = datagen.mixture(n, d, 10, seed=n + d)
    if mode in (2, 3) and not _tc_supported(d, k):
        with pytest.raises(drgb.DrgbError):
            _run(drgb, X, k, mode)
        return
    gi, gd = _run(drgb, X, k, mode)
    oi, od = oknn.knn(X, k)
    check_knn(X, np.arange(n), gi, gd, oi, od, k)


@pytest.mark.parametrize("mode", [2, 3])
@pytest.mark.parametrize("n,d,k", [(4097, 50, 15), (5000, 61, 31), (9000, 8, 10), (130, 50, 15)])
def test_tensor_core_ragged_tiles(drgb, n, d, k, mode):
    # n not a multiple of the 128-row query block or the 256-row database tile
    X, _ = datagen.aniso_mixture(n, d, 20, seed=n)
    gi, gd = _run(drgb, X, k, mode)
    rows = np.unique(np.concatenate([np.arange(0, n, 7), np.arange(max(0, n - 300), n)]))
    oi, od = oknn.knn_rows(X, rows, k)
    check_knn(X, rows, gi[rows], gd[rows], oi, od, k)


@pytest.mark.parametrize("mode", [2, 3])
@pytest.mark.parametrize("d", [50, 49])
def test_tensor_core_matches_exact_scan_bitwise(drgb, mode, d):
    # both paths finish with the same FP32 arithmetic on the same candidates,
    # and the rows the certificate leaves are re-scanned over the cells they
    # can reach (an odd d as well as an even one)
    X, _ = datagen.mixture(6000, d, 12, seed=5)
    gi2, gd2 = _run(drgb, X, 15, mode)
    unc = drgb.knn_uncertified()
    gi1, gd1 = _run(drgb, X, 15, 1)
    assert np.array_equal(gi1, gi2) and np.array_equal(gd1, gd2)
    if mode == 2:
        assert unc > 0   # the BF16 certificate leaves rows to the re-scan


@pytest.mark.parametrize("mode", [2, 3])
def test_tensor_core_far_from_origin(drgb, mode):
    # a large common offset: centring keeps the 16-bit pass accurate; whatever
    # it cannot certify goes through the exact scan, so results stay exact
    X, _ = datagen.mixture(5000, 50, 10, seed=8)
    X = X + np.float32(1000.0)
    gi, gd = _run(drgb, X, 15, mode)
    rows = np.arange(0, 5000, 11)
    oi, od = oknn.knn_rows(X, rows, 15)
    check_knn(X, rows, gi[rows], gd[rows], oi, od, 15)
    assert drgb.knn_uncertified() <= 5000


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_planted_duplicates_resolve_by_index(drgb, mode):
    g = np.random.default_rng(7)
    base = g.normal(size=(300, 50)).astype(np.float32)
    X = np.concatenate([base, base[:40], base[:40], base[:5]])   # exact duplicates
    gi, gd = _run(drgb, X, 15, mode)
    oi, od = oknn.knn(X, 15)
    assert np.array_equal(gi, oi)          # exact ties are broken by index on both sides
    assert np.all(gd[:40, 0] == 0.0) and np.all(gd[:5, 2] == 0.0)


@pytest.mark.parametrize("mode", [2, 3])
def test_many_exact_copies_through_the_rescan(drgb, mode):
    # 40 copies of one point among 6,000: for each copy the other copies fill
    # all 32 candidate slots at distance 0, so no certificate can hold and
    # the row goes to the exact re-scan with a k-th distance of 0; the
    # re-scan must still admit the points at distance exactly 0
    g = np.random.default_rng(11)
    X = g.normal(size=(6000, 20)).astype(np.float32)
    copies = np.arange(100, 6000, 150)[:40]
    X[copies] = X[copies[0]]
    gi, gd = _run(drgb, X, 15, mode)
    oi, od = oknn.knn_rows(X, copies, 15)
    assert np.array_equal(gi[copies], oi) and np.all(gd[copies] == 0.0)
    rows = np.arange(0, 6000, 97)
    oi, od = oknn.knn_rows(X, rows, 15)
    check_knn(X, rows, gi[rows], gd[rows], oi, od, 15)


def test_all_points_identical(drgb):
    X = np.ones((50, 8), np.float32)
    gi, gd = _run(drgb, X, 10, 1)
    oi, od = oknn.knn(X, 10)
    assert np.array_equal(gi, oi) and np.all(gd == 0)


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_70k_sampled_rows(drgb, mode):
    # mode 2 (BF16) leaves most of the 70K rows uncertified: more rows than
    # the cell re-scan's partial lists hold (about 15,000 with 34 cells), so
    # they go through the chunked scan of all points
    X, _ = datagen.config_70k(seed=0)
    gi, gd = _run(drgb, X, 15, mode)
    rows = np.linspace(0, len(X) - 1, 300).astype(np.int64)
    oi, od = oknn.knn_rows(X, rows, 15)
    check_knn(X, rows, gi[rows], gd[rows], oi, od, 15)
    if mode == 3:
        # the FP16 certificate holds for nearly every row of this workload
        assert drgb.knn_uncertified() < 0.05 * len(X)
    if mode == 2:
        assert drgb.knn_uncertified() > 20000


def test_rejects_bad_sizes(drgb):
    import torch
    X = torch.zeros((15, 4), device="cuda")
    with pytest.raises(drgb.DrgbError) as e:
        drgb.knn_graph(X, 15)
    assert e.value.code == -1
    with pytest.raises(drgb.DrgbError):
        drgb.knn_graph(torch.zeros((100, 4), device="cuda"), 33)
    raw = torch.zeros(100 * 4 * 4 + 4, dtype=torch.uint8, device="cuda")
    rc = drgb._lib.load().drgb_knn_graph(drgb.context(), drgb._ptr(raw[2:]), 100, 4, 5, 1,
                                         drgb._ptr(raw), drgb._ptr(raw), None)
    assert rc == -1   # 2-byte offset: not even float-aligned, refused on the host
    flat = torch.zeros(100 * 4 + 1, device="cuda")  # a 4-byte offset (a row slice) is fine
    idx, _ = drgb.knn_graph(flat[1:].view(100, 4), 5)
    assert idx.shape == (100, 5)
