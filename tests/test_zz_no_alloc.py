"""Allocation-free fuzzy-graph entry point (gpu).

drgb_fuzzy_weights_static is for callers that cannot allocate device memory:
code running under an external memory manager that owns all of the device's
memory, or in a setting where cudaMalloc is not allowed.  It takes no context
and keeps its scratch in a fixed device array inside the library, which every
call shares.  These tests call it through the C ABI and check that it returns
what drgb_fuzzy_weights returns, on consecutive calls (the array still holds
the previous call's data when the next call starts), and that sizes beyond the
array are refused.  The file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

import datagen
from gpu_util import drgb_module

pytestmark = pytest.mark.gpu


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _outputs(n, k, dev):
    import torch
    cap = 2 * n * k
    return (torch.empty(n + 1, dtype=torch.int32, device=dev), torch.empty(cap, dtype=torch.int32, device=dev),
            torch.empty(cap, dtype=torch.float32, device=dev), torch.empty(cap, dtype=torch.int32, device=dev),
            torch.empty(n, dtype=torch.float32, device=dev), torch.empty(n, dtype=torch.float32, device=dev))


def _call_static(lib, idx, dist, n_epochs, outs):
    import torch
    n, k = idx.shape
    row_ptr, col, w, q, rho, sigma = outs
    stream = C.c_void_p(torch.cuda.current_stream(idx.device).cuda_stream)
    return lib.drgb_fuzzy_weights_static(_ptr(idx), _ptr(dist), n, k, n_epochs, _ptr(row_ptr), _ptr(col),
                                         _ptr(w), _ptr(q), col.numel(), _ptr(rho), _ptr(sigma), stream)


def _static_graph(lib, idx, dist, n_epochs):
    n, k = idx.shape
    outs = _outputs(n, k, idx.device)
    rc = _call_static(lib, idx, dist, n_epochs, outs)
    row_ptr, col, w, q, rho, sigma = outs
    nnz = int(row_ptr[n].item()) if rc == 0 else 0
    return rc, row_ptr, col[:nnz], w[:nnz], q[:nnz], rho, sigma


def test_static_entry_point_matches_context_entry_point():
    import torch
    drgb = drgb_module()
    from paper_2603_04035_gb300 import _lib
    lib = _lib.load()
    # two different inputs, then the first again: each call must not depend on
    # what the previous one left in the shared array
    for n, seed, T in [(2000, 0, 200), (3500, 1, 500), (2000, 0, 200)]:
        X, _ = datagen.mixture(n, 50, 10, seed=seed)
        idx, dist = drgb.knn_graph(torch.from_numpy(X).cuda(), 15)
        ref = drgb.fuzzy_weights(idx, dist, T, with_rho_sigma=True)
        rc, rp, col, w, q, rho, sigma = _static_graph(lib, idx, dist, T)
        assert rc == 0
        # both entry points run the same kernels on the same inputs: the
        # graph is the same bit for bit
        assert torch.equal(rp, ref.row_ptr)
        assert torch.equal(col, ref.col)
        assert torch.equal(q, ref.q)
        assert torch.equal(w, ref.w)
        assert torch.equal(rho, ref.rho)
        assert torch.equal(sigma, ref.sigma)


def test_static_entry_point_allocates_no_device_memory():
    import torch
    drgb = drgb_module()
    from paper_2603_04035_gb300 import _lib
    lib = _lib.load()
    X, _ = datagen.mixture(25_000, 50, 10, seed=3)
    idx, dist = drgb.knn_graph(torch.from_numpy(X).cuda(), 15)
    X2, _ = datagen.mixture(2000, 50, 10, seed=4)
    small = drgb.knn_graph(torch.from_numpy(X2).cuda(), 15)
    assert _call_static(lib, *small, 200, _outputs(2000, 15, idx.device)) == 0   # set-up call
    outs = _outputs(25_000, 15, idx.device)          # every output exists before the measurement
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    assert _call_static(lib, idx, dist, 200, outs) == 0
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    # its scratch (about 14 MB at this size) lives in the library's fixed array
    assert free0 - free1 < (2 << 20), (free0, free1)
    assert int(outs[0][25_000].item()) > 0


def test_static_entry_point_refuses_oversized_input():
    import torch
    drgb_module()
    from paper_2603_04035_gb300 import _lib
    lib = _lib.load()
    dummy_i = torch.zeros(16, dtype=torch.int32, device="cuda")
    dummy_f = torch.zeros(16, dtype=torch.float32, device="cuda")
    n, k = 60_000, 15
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.drgb_fuzzy_weights_static(_ptr(dummy_i), _ptr(dummy_f), n, k, 200, _ptr(dummy_i), _ptr(dummy_i),
                                       _ptr(dummy_f), _ptr(dummy_i), 2 * n * k, None, None, stream)
    assert rc == _lib.ERR_WORKSPACE
