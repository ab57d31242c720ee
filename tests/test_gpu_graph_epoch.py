"""Fuzzy graph, initialisation and SGD epoch parity against the oracle (gpu)."""
import numpy as np
import pytest

import datagen
from gpu_util import drgb_module, epoch_tolerance
from oracle import fuzzy as ofuzzy, knn as oknn, sgd as osgd
from oracle.fuzzy import Q_ONE

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def drgb():
    return drgb_module()


def _t(x, dtype=None):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x if dtype is None else x.astype(dtype))).cuda()


def _np(t):
    return t.cpu().numpy()


def _gpu_graph(drgb, X, k, T):
    import torch
    idx, dist = drgb.knn_graph(_t(X, np.float32), k)
    g = drgb.fuzzy_weights(idx, dist, T, with_rho_sigma=True)
    torch.cuda.synchronize()
    return idx, dist, g


# ---------------------------------------------------------------- fuzzy graph
@pytest.mark.parametrize("n,k,T", [(2000, 15, 200), (500, 7, 500), (300, 32, 50), (16, 15, 200)])
def test_fuzzy_graph_matches_oracle(drgb, n, k, T):
    X, _ = datagen.mixture(n, 50, 10, seed=n)
    idx, dist, g = _gpu_graph(drgb, X, k, T)
    gi, gd = _np(idx).astype(np.int64), _np(dist).astype(np.float64)
    o = ofuzzy.build_csr(gi, gd, T, k)     # oracle on the same (FP32) neighbour lists
    np.testing.assert_array_equal(_np(g.rho), o["rho"])
    np.testing.assert_allclose(_np(g.sigma), o["sigma"], rtol=1e-4)
    rp, col, q = (_np(x).astype(np.int64) for x in (g.row_ptr, g.col, g.q))
    w = _np(g.w).astype(np.float64)
    W_TOL = 1e-5
    # GPU schedule words are consistent with its own weights (w_max = 1):
    # q = round-half-even(2^24 w), an exact operation on an FP32 w
    assert o["w_max"] == 1.0
    np.testing.assert_array_equal(q, np.rint(Q_ONE * w).astype(np.int64))
    # structure: same (head, tail) pairs, except entries whose weight lies
    # within the weight tolerance of the pruning boundary w = 1 / T
    gpu_pairs = {}
    for i in range(n):
        for e in range(rp[i], rp[i + 1]):
            gpu_pairs[(i, int(col[e]))] = e
    o_heads = np.repeat(np.arange(n), np.diff(o["row_ptr"]))
    o_pairs = {(int(i), int(c)): e for e, (i, c) in enumerate(zip(o_heads, o["col"]))}
    S = o["union"]
    for key in set(gpu_pairs) ^ set(o_pairs):
        assert abs(S[key[0], key[1]] - 1.0 / T) <= W_TOL + 2.0 / Q_ONE, f"structural mismatch {key}"
    for i in range(n):
        assert np.all(np.diff(col[rp[i]:rp[i + 1]]) > 0)
    common = sorted(set(gpu_pairs) & set(o_pairs))
    ge = np.array([gpu_pairs[p] for p in common])
    oe = np.array([o_pairs[p] for p in common])
    np.testing.assert_allclose(w[ge], o["w"][oe], atol=W_TOL)
    # exact symmetry of the GPU weights and schedule words
    for (i, c), e in gpu_pairs.items():
        e2 = gpu_pairs[(c, i)]
        assert w[e] == w[e2] and q[e] == q[e2]
    assert int(rp[-1]) == len(col)


def test_fuzzy_reports_a_neighbour_listed_twice(drgb):
    import torch
    X, _ = datagen.mixture(300, 50, 5, seed=7)
    idx, dist = drgb.knn_graph(_t(X, np.float32), 15)
    bad = idx.clone()
    bad[3, 1] = bad[3, 0]
    lib, ctx = drgb._lib.load(), drgb.context(0)
    stream = torch.cuda.current_stream().cuda_stream
    assert lib.drgb_sync(ctx, stream) == 0
    drgb.fuzzy_weights(bad, dist, 200)           # runs; the status word records the error
    assert lib.drgb_sync(ctx, stream) == drgb._lib.ERR_INVALID
    drgb.fuzzy_weights(idx, dist, 200)           # well-formed lists: no error, status cleared
    assert lib.drgb_sync(ctx, stream) == 0


def test_fuzzy_row_sums(drgb):
    X, _ = datagen.mixture(3000, 50, 10, seed=3)
    idx, dist, g = _gpu_graph(drgb, X, 15, 200)
    gd = _np(dist).astype(np.float64)
    rho, sig = _np(g.rho).astype(np.float64), _np(g.sigma).astype(np.float64)
    s = np.exp(-np.maximum(0, gd - rho[:, None]) / sig[:, None]).sum(1)
    free = sig > 1e-3 * gd.mean(1) * (1 + 1e-6)
    np.testing.assert_allclose(s[free], np.log2(15), atol=2e-5)


# ---------------------------------------------------------------- init
def test_init_bit_exact(drgb):
    for n, seed, R in [(1, 0, 10.0), (1000, 1, 10.0), (70001, 123456789012, 3.5)]:
        Y = _np(drgb.init_embedding(n, R, seed))
        assert np.array_equal(Y, osgd.init_embedding(n, seed, R).astype(np.float32))


# ---------------------------------------------------------------- epoch
def _oracle_graph(n, k, T, seed, d=50):
    X, _ = datagen.mixture(n, d, 10, seed=seed)
    oi, od = oknn.knn(X, k)
    return X, ofuzzy.build_csr(oi, od, T, k)


def _graph_tensors(drgb, rp, col, q, w=None):
    return drgb.Graph(_t(rp, np.int32), _t(col, np.int32),
                      _t(np.zeros(len(col)) if w is None else w, np.float32), _t(q, np.int32))


def _compare_epoch(drgb, Y, rp, col, q, a, b, lr, neg, t, seed):
    n = Y.shape[0]
    g = _graph_tensors(drgb, rp, col, q)
    Yg = _np(drgb.embed_epoch(_t(Y, np.float32), g, a, b, lr, neg, t, seed))
    ref = osgd.epoch(Y.astype(np.float32), rp, col, q.astype(np.uint64), a, b, lr, neg, t, seed)
    err = np.abs(Yg - ref)
    tol = epoch_tolerance(ref)
    assert np.all(err <= tol), f"max rel err {np.max(err / np.maximum(np.abs(ref), 1))}"
    return Yg, ref


@pytest.mark.parametrize("neg", [0, 1, 5, 8])
@pytest.mark.parametrize("t", [0, 3, 117])
def test_epoch_matches_oracle(drgb, neg, t):
    X, o = _oracle_graph(2000, 15, 200, 0)
    a, b = drgb.find_ab(1.0, 0.1)
    Y = np.random.default_rng(t).uniform(-10, 10, size=(2000, 2)).astype(np.float32)
    lr = 1.0 * (1 - t / 200)
    _compare_epoch(drgb, Y, o["row_ptr"], o["col"], o["q"], a, b, lr, neg, t, 2)


def test_epoch_contracted_embedding(drgb):
    # a late-stage embedding: points in tight clusters, many clipped terms
    X, o = _oracle_graph(1500, 15, 500, 5)
    lab = np.arange(1500) % 10
    g = np.random.default_rng(0)
    Y = (g.normal(size=(10, 2)) * 5)[lab] + g.normal(scale=0.05, size=(1500, 2))
    _compare_epoch(drgb, Y.astype(np.float32), o["row_ptr"], o["col"], o["q"], 1.577, 0.895,
                   0.3, 5, 250, 77)


def test_epoch_hub_row_and_empty_rows(drgb):
    # star: row 0 has 3000 entries (a hub far above 1024), rows 1..3000 one entry;
    # rows 3001..3099 are empty.
    n = 3100
    heads = np.concatenate([np.zeros(3000, np.int64), np.arange(1, 3001)])
    cols = np.concatenate([np.arange(1, 3001), np.zeros(3000, np.int64)])
    order = np.lexsort((cols, heads))
    heads, cols = heads[order], cols[order]
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, heads + 1, 1)
    rp = np.cumsum(rp)
    q = np.random.default_rng(1).integers(Q_ONE // 200, Q_ONE + 1, size=len(cols)).astype(np.uint64)
    Y = np.random.default_rng(2).uniform(-10, 10, size=(n, 2)).astype(np.float32)
    Yg, ref = _compare_epoch(drgb, Y, rp, cols, q, 1.577, 0.895, 1.0, 5, 7, 3)
    assert np.array_equal(Yg[3001:], Y[3001:]) or np.allclose(Yg[3001:], Y[3001:])


def test_epoch_coincident_points(drgb):
    n = 64
    rp = np.arange(n + 1) * 1
    col = (np.arange(n) + 1) % n
    q = np.full(n, Q_ONE, np.uint64)
    Y = np.zeros((n, 2), np.float32)
    Y[: n // 2] = 1.25   # half the points coincide with their neighbour
    _compare_epoch(drgb, Y, rp, col, q, 1.577, 0.895, 1.0, 5, 0, 9)


def test_epoch_two_points(drgb):
    rp = np.array([0, 1, 2])
    col = np.array([1, 0])
    q = np.array([Q_ONE, Q_ONE], np.uint64)
    Y = np.array([[0.0, 0.0], [3.0, 4.0]], np.float32)
    _compare_epoch(drgb, Y, rp, col, q, 1.0, 1.0, 0.5, 8, 0, 7)


def test_epoch_loop_resume_is_bit_identical(drgb):
    import torch
    X, o = _oracle_graph(1200, 15, 60, 11)
    g = _graph_tensors(drgb, o["row_ptr"], o["col"], o["q"])
    a, b = drgb.find_ab(1.0, 0.1)
    Y0 = drgb.init_embedding(1200, 10.0, 1)
    full = Y0.clone()
    drgb.embed_epochs(full, g, a, b, 1.0, 5, 0, 60, 60, 2)
    part = Y0.clone()
    drgb.embed_epochs(part, g, a, b, 1.0, 5, 0, 23, 60, 2)
    drgb.embed_epochs(part, g, a, b, 1.0, 5, 23, 60, 60, 2)
    step = Y0.clone()
    for t in range(60):
        step = drgb.embed_epoch(step, g, a, b, float(np.float32(1.0 * (1 - t / 60))), 5, t, 2)
    torch.cuda.synchronize()
    assert torch.equal(full, part)
    assert torch.equal(full, step)


def test_epoch_loop_tracks_oracle_for_a_few_epochs(drgb):
    X, o = _oracle_graph(1000, 15, 200, 4)
    g = _graph_tensors(drgb, o["row_ptr"], o["col"], o["q"])
    a, b = drgb.find_ab(1.0, 0.1)
    Y = drgb.init_embedding(1000, 10.0, 1)
    drgb.embed_epochs(Y, g, a, b, 1.0, 5, 0, 3, 200, 2)
    ref = osgd.init_embedding(1000, 1, 10.0)
    for t in range(3):
        ref = osgd.epoch(ref, o["row_ptr"], o["col"], o["q"], a, b, 1.0 * (1 - t / 200), 5, t, 2)
    err = np.abs(_np(Y) - ref)
    assert np.all(err <= 3 * epoch_tolerance(ref))


def test_epoch_rejects_bad_arguments(drgb):
    import torch
    X, o = _oracle_graph(100, 5, 50, 1)
    g = _graph_tensors(drgb, o["row_ptr"], o["col"], o["q"])
    Y = torch.zeros((100, 2), device="cuda")
    with pytest.raises(drgb.DrgbError):
        drgb.embed_epoch(Y, g, 1.0, 1.0, 1.0, 5, 0, 0, out=Y)        # aliasing
    with pytest.raises(drgb.DrgbError):
        drgb.embed_epoch(Y, g, 1.0, 1.0, 1.0, -1, 0, 0)              # negative neg
    with pytest.raises(drgb.DrgbError):
        drgb.embed_epochs(Y, g, 1.0, 1.0, 1.0, 5, 10, 5, 50, 0)      # bad range


def _star_graph(n_hub=3000, n_empty=100, seed=1):
    """Row 0 has n_hub entries, rows 1..n_hub one entry each, then n_empty empty rows."""
    n = n_hub + 1 + n_empty
    heads = np.concatenate([np.zeros(n_hub, np.int64), np.arange(1, n_hub + 1)])
    cols = np.concatenate([np.arange(1, n_hub + 1), np.zeros(n_hub, np.int64)])
    order = np.lexsort((cols, heads))
    heads, cols = heads[order], cols[order]
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, heads + 1, 1)
    q = np.random.default_rng(seed).integers(Q_ONE // 200, Q_ONE + 1, size=len(cols)).astype(np.uint64)
    return n, np.cumsum(rp), cols, q


@pytest.mark.parametrize("graph", ["mixture", "star"])
def test_epoch_every_tuning_choice_is_bit_identical(drgb, graph):
    """The force-kernel width changes the speed only: every choice must give
    the same bits, and those bits must stay within the oracle tolerance."""
    import torch
    from paper_2603_04035_gb300 import _lib
    if graph == "mixture":
        X, o = _oracle_graph(2000, 15, 200, 0)
        n, rp, col, q = 2000, o["row_ptr"], o["col"], o["q"]
    else:
        n, rp, col, q = _star_graph()
    g = _graph_tensors(drgb, rp, col, q)
    Y = np.random.default_rng(5).uniform(-10, 10, size=(n, 2)).astype(np.float32)
    Yd = _t(Y)
    saved = drgb.get_tuning(_lib.TUNE_EPOCH_WARPS), drgb.get_tuning(_lib.TUNE_EPOCH_PIPE)
    outs = {}
    try:
        for pipe in (0, 1):   # flat and pipelined forms
            drgb.set_tuning(_lib.TUNE_EPOCH_PIPE, pipe)
            for warps in (4, 8):
                drgb.set_tuning(_lib.TUNE_EPOCH_WARPS, warps)
                for neg in (5, 6):   # the fixed-count and the generic force paths
                    outs[(pipe, warps, neg)] = drgb.embed_epoch(Yd, g, 1.577, 0.895, 0.7, neg, 13, 4).clone()
        torch.cuda.synchronize()
    finally:
        drgb.set_tuning(_lib.TUNE_EPOCH_WARPS, saved[0])
        drgb.set_tuning(_lib.TUNE_EPOCH_PIPE, saved[1])
    for neg in (5, 6):
        for key in ((0, 4, neg), (0, 8, neg), (1, 8, neg)):
            assert torch.equal(outs[(1, 4, neg)], outs[key]), key
        ref = osgd.epoch(Y, rp, col, q.astype(np.uint64), 1.577, 0.895, 0.7, neg, 13, 4)
        assert np.all(np.abs(_np(outs[(1, 4, neg)]) - ref) <= epoch_tolerance(ref))


def test_set_tuning_rejects_unsupported_values(drgb):
    from paper_2603_04035_gb300 import _lib
    for bad in (0, 2, 16, 32):
        with pytest.raises(drgb.DrgbError):
            drgb.set_tuning(_lib.TUNE_EPOCH_WARPS, bad)
    for bad in (-1, 2):
        with pytest.raises(drgb.DrgbError):
            drgb.set_tuning(_lib.TUNE_EPOCH_PIPE, bad)
    with pytest.raises(drgb.DrgbError):
        drgb.set_tuning(99, 4)



def test_gather_probe(drgb):
    # the epoch's roofline denominator: random 8-byte loads per second; an
    # array that fits in L1 is served at least as fast as one that only fits in L2
    import torch
    small = torch.randn((70_000, 2), device="cuda")
    big = torch.randn((8_000_000, 2), device="cuda")
    rs, rb = drgb.gather_probe(small, rounds=32), drgb.gather_probe(big, rounds=32)
    assert 1e9 < rb and 1e9 < rs < 1e13, (rs, rb)
    assert rs > 0.8 * rb
    with pytest.raises(drgb.DrgbError):
        drgb.gather_probe(small, rounds=0)
    with pytest.raises(drgb.DrgbError):
        drgb.gather_probe(small.view(-1)[1:-1].view(-1, 2), rounds=4)   # not 8-byte aligned
