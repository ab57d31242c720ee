"""Failure detection on the GPU without a fault (gpu).

The tensor-core kernels wait on mbarriers for a bounded time; a wait that
gives up reports DRGB_ERR_TIMEOUT through the context's status word and the
kernel returns.  drgb_wait_selftest runs that same bounded wait on a barrier
nothing arrives at, with no copy or tensor-core work in flight, so the test
makes the wait run out without putting the GPU at risk.
"""
import ctypes as C
import time

import numpy as np
import pytest

import datagen
from gpu_util import drgb_module

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_the_context_recovers():
    import torch
    drgb = drgb_module()
    from paper_2603_04035_gb300 import _lib
    lib = _lib.load()
    ctx = drgb.context()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    t0 = time.perf_counter()
    rc = lib.drgb_wait_selftest(ctx, 5000, 0, stream)          # 5 ms limit, nothing arrives
    dt = time.perf_counter() - t0
    assert rc == _lib.ERR_TIMEOUT
    assert 0.005 <= dt < 2.0, dt
    assert lib.drgb_wait_selftest(ctx, 5000, 1, stream) == 0   # the control: the wait succeeds
    # the status word was read and cleared: the tensor-core k-NN on the same
    # context runs normally
    X, _ = datagen.mixture(6000, 50, 10, seed=2)
    idx, dist = drgb.knn_graph(torch.from_numpy(X).cuda(), 15)
    assert drgb.knn_uncertified() >= 0
    d = dist.cpu().numpy()
    assert np.all(np.isfinite(d)) and np.all(np.diff(d, axis=1) >= 0)


def test_selftest_rejects_bad_limits():
    drgb = drgb_module()
    from paper_2603_04035_gb300 import _lib
    lib = _lib.load()
    ctx = drgb.context()
    for bad in (0, -5, 10_000_001):
        assert lib.drgb_wait_selftest(ctx, bad, 0, None) == _lib.ERR_INVALID


def test_scratch_limit_refuses_and_the_context_recovers():
    # an allocation failure made on the host: the capped context refuses the
    # fit's scratch with a clear error, holds at most the cap, and fits again
    # (the same result) once the cap is lifted
    import torch
    drgb = drgb_module()
    from paper_2603_04035_gb300 import _lib
    lib = _lib.load()
    ctx = drgb.context()
    X, _ = datagen.mixture(2000, 50, 10, seed=1)
    Xd = torch.from_numpy(X).cuda()
    ref = drgb.fit_transform(Xd, n_epochs=50)
    try:
        assert lib.drgb_set_scratch_limit(ctx, 1 << 20) == 0
        assert lib.drgb_ctx_scratch_bytes(ctx) <= 1 << 20
        with pytest.raises(drgb.DrgbError) as err:
            drgb.fit_transform(Xd, n_epochs=50)
        assert err.value.code == _lib.ERR_WORKSPACE and "limit" in str(err.value)
        assert lib.drgb_set_scratch_limit(ctx, -1) == _lib.ERR_INVALID
    finally:
        assert lib.drgb_set_scratch_limit(ctx, 0) == 0
    assert torch.equal(drgb.fit_transform(Xd, n_epochs=50), ref)


def test_nonfinite_embedding_is_reported():
    # NaN injected into Y: the epoch runs and the next synchronising call
    # reports DRGB_ERR_NONFINITE; a finite Y then passes and clears the status
    import torch
    drgb = drgb_module()
    from paper_2603_04035_gb300 import _lib
    lib = _lib.load()
    ctx = drgb.context()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    X, _ = datagen.mixture(400, 50, 5, seed=2)
    Xd = torch.from_numpy(X).cuda()
    idx, dist = drgb.knn_graph(Xd, 15)
    g = drgb.fuzzy_weights(idx, dist, 200)
    a, b = drgb.find_ab()
    Y = drgb.init_embedding(400, seed=3)
    assert lib.drgb_sync(ctx, stream) == 0
    bad = Y.clone()
    bad[5, 1] = float("nan")
    drgb.embed_epoch(bad, g, a, b, 1.0, 5, 0, seed=4)
    assert lib.drgb_sync(ctx, stream) == _lib.ERR_NONFINITE
    bad[5, 1] = float("inf")
    drgb.embed_epochs(bad, g, a, b, 1.0, 5, 0, 2, 200, seed=4)
    assert lib.drgb_sync(ctx, stream) == _lib.ERR_NONFINITE
    out = drgb.embed_epoch(Y, g, a, b, 1.0, 5, 0, seed=4)
    assert lib.drgb_sync(ctx, stream) == 0 and torch.isfinite(out).all()
