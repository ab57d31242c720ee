"""GB300-native UMAP-style neighbour embedding (the hot path of mlx-vis,
arXiv 2603.04035): exact k-NN graph, fuzzy simplicial-set graph, a,b fit and
the synchronous negative-sampling SGD epoch, as hand-written CUDA for sm_103a
behind the C ABI of include/drgb.h.

This module only marshals arguments: PyTorch provides device memory and
streams, every step runs in libdrgb's kernels.  There is no CPU fallback; the
functions raise if the library is not built or no GB300 is present.

Public API (names follow the C ABI):

    knn_graph(X, k)                      -> (idx int32 n x k, dist float32 n x k)
    fuzzy_weights(idx, dist, n_epochs)   -> Graph(row_ptr, col, w, q)
    find_ab(spread, min_dist)            -> (a, b)
    init_embedding(n, init_range, seed)  -> Y float32 n x 2
    embed_epoch(Y, graph, a, b, lr, neg, epoch, seed) -> Y'
    embed_epochs(Y, graph, a, b, lr0, neg, t_begin, t_end, n_epochs, seed)  (in place)
    fit_transform(X, **params)           -> Y
    eval_recall(X, Y, k, n_query) / eval_trust(X, Y, k, n_query) -> float
    UMAP(**params).fit_transform(X)      (Section 2.1's class-based API)
"""
from __future__ import annotations

import atexit
import ctypes as C
import os
from dataclasses import dataclass

import torch

from . import _lib
from ._lib import MAX_K, Params  # noqa: F401

__all__ = ["DrgbError", "Graph", "UMAP", "knn_graph", "fuzzy_weights", "find_ab",
           "init_embedding", "embed_epoch", "embed_epochs", "fit_transform", "eval_recall",
           "eval_trust", "eval_recall_heldout", "spectral_init", "pca", "knn_nndescent", "gather_probe", "render", "default_params", "context", "knn_uncertified", "launch_count",
           "set_profiling", "stage_times", "set_tuning", "get_tuning", "set_tuning_cache",
           "tuning_cache_lookup", "tuning_cache_store", "knn_tiles", "fit_transform_batched",
           "autotune_epoch", "mlp_param_count", "mlp_init", "mlp_sample", "mlp_grad", "mlp_train",
           "mlp_embed", "ParametricUMAP", "transform"]


class DrgbError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"drgb error {code} ({_lib.ERROR_NAMES.get(code, '?')}): {msg}")
        self.code = code


_contexts: dict[int, int] = {}


def _destroy_all():
    lib = _lib._lib
    if lib is None:
        return
    for h in list(_contexts.values()):
        lib.drgb_ctx_destroy(h)
    _contexts.clear()


atexit.register(_destroy_all)


def context(device: int | None = None) -> int:
    """Opaque drgb_ctx handle for a CUDA device (created on first use)."""
    lib = _lib.load()
    dev = torch.cuda.current_device() if device is None else int(device)
    h = _contexts.get(dev)
    if h is None:
        out = C.c_void_p()
        rc = lib.drgb_ctx_create(dev, C.byref(out))
        if rc != 0:
            raise DrgbError(rc, f"cannot create a context on cuda:{dev} (needs a GB300, sm_103)")
        h = _contexts[dev] = out.value
    return h


def _check(rc: int, ctx) -> None:
    if rc != 0:
        msg = _lib.load().drgb_last_error(ctx)
        raise DrgbError(rc, msg.decode() if msg else "")


def _ptr(t: torch.Tensor | None):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(dev: torch.device):
    return C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def _cuda(t: torch.Tensor, dtype, name: str, ndim: int | None = None) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if ndim is not None and t.dim() != ndim:
        raise ValueError(f"{name} must have {ndim} dimensions")
    return t.contiguous()


@dataclass
class Graph:
    """Head-sorted CSR of the fuzzy graph (device tensors)."""
    row_ptr: torch.Tensor   # int32 n+1
    col: torch.Tensor       # int32 nnz
    w: torch.Tensor         # float32 nnz
    q: torch.Tensor         # int32 nnz holding uint32 schedule words (< 2^25)
    rho: torch.Tensor | None = None
    sigma: torch.Tensor | None = None

    @property
    def n(self) -> int:
        return self.row_ptr.numel() - 1

    @property
    def nnz(self) -> int:
        return self.col.numel()


def default_params() -> dict:
    p = Params()
    _lib.load().drgb_default_params(C.byref(p))
    return {f: getattr(p, f) for f, _ in Params._fields_}


def launch_count(device=None) -> int:
    """Kernels launched so far by the library on this device's context."""
    return int(_lib.load().drgb_launch_count(context(device)))


def set_tuning(param: int, value: int, device=None) -> None:
    """Set a performance knob of the device's context (see include/drgb.h)."""
    ctx = context(device)
    _check(_lib.load().drgb_set_tuning(ctx, param, value), ctx)


def get_tuning(param: int, device=None) -> int:
    """Current value of a performance knob of the device's context."""
    ctx = context(device)
    v = C.c_int32(0)
    _check(_lib.load().drgb_get_tuning(ctx, param, C.byref(v)), ctx)
    return int(v.value)


def set_tuning_cache(path: str | None, device=None) -> None:
    """Use (or with None stop using) a JSON tuning cache for the device's
    context: autotuned batched fits reuse its settings (see include/drgb.h)."""
    ctx = context(device)
    _check(_lib.load().drgb_set_tuning_cache(ctx, None if path is None else os.fsencode(path)), ctx)


def tuning_cache_lookup(path: str, key: str) -> tuple[int, int] | None:
    """(force-kernel width, form) stored for `key` in the tuning cache, or None."""
    v, p = C.c_int32(0), C.c_int32(0)
    rc = _lib.load().drgb_tuning_cache_lookup(os.fsencode(path), key.encode("ascii"), C.byref(v), C.byref(p))
    return (int(v.value), int(p.value)) if rc == 0 else None


def tuning_cache_store(path: str, key: str, epoch_warps: int, epoch_pipe: int = 1) -> None:
    """Add or replace the entry of `key` in the tuning cache."""
    rc = _lib.load().drgb_tuning_cache_store(os.fsencode(path), key.encode("ascii"), epoch_warps, epoch_pipe)
    if rc != 0:
        raise DrgbError(rc, f"tuning cache: cannot store {key!r} = ({epoch_warps}, {epoch_pipe}) in {path}")


def set_profiling(on: bool, device=None) -> None:
    _check(_lib.load().drgb_set_profiling(context(device), int(bool(on))), context(device))


STAGES = ("knn", "fuzzy", "init", "epochs", "knn_gemm", "knn_prep", "knn_rerank", "knn_rescan")


def stage_times(device=None) -> dict:
    """Per-stage milliseconds of the last profiled fit_transform (synchronous)."""
    ms = (C.c_float * 8)()
    ctx = context(device)
    m = _lib.load().drgb_stage_times(ctx, ms, 8)
    if m < 0:
        _check(m, ctx)
    return {STAGES[i] if i < len(STAGES) else f"stage{i}": ms[i] for i in range(m)}


# ---------------------------------------------------------------- k-NN
def knn_graph(X: torch.Tensor, k: int = 15, mode: int = 0):
    """Exact k-NN graph of the rows of X (self excluded): (idx int32, dist float32)."""
    X = _cuda(X, torch.float32, "X", 2)
    n, d = X.shape
    idx = torch.empty((n, k), dtype=torch.int32, device=X.device)
    dist = torch.empty((n, k), dtype=torch.float32, device=X.device)
    ctx = context(X.device.index)
    _check(_lib.load().drgb_knn_graph(ctx, _ptr(X), n, d, k, mode, _ptr(idx), _ptr(dist),
                                      _stream(X.device)), ctx)
    return idx, dist


def knn_nndescent(X: torch.Tensor, k: int = 15, seed: int = 1, delta: float = 0.015, max_iter: int = 30,
                  reverse: bool = False):
    """Approximate k-NN graph by NNDescent: (idx int32, dist float32, update
    rate of each iteration run); reverse=True joins over general neighbours
    (own list and reverse neighbours, k <= 16)."""
    X = _cuda(X, torch.float32, "X", 2)
    n, d = X.shape
    idx = torch.empty((n, k), dtype=torch.int32, device=X.device)
    dist = torch.empty((n, k), dtype=torch.float32, device=X.device)
    it = C.c_int32(0)
    rates = (C.c_double * max(1, max_iter))()
    ctx = context(X.device.index)
    _check(_lib.load().drgb_knn_nndescent(ctx, _ptr(X), n, d, k, seed, delta, max_iter, int(reverse), _ptr(idx),
                                          _ptr(dist), C.byref(it), rates, _stream(X.device)), ctx)
    return idx, dist, [rates[t] for t in range(it.value)]


def gather_probe(Y: torch.Tensor, rounds: int = 256, seed: int = 1) -> float:
    """Random 8-byte gathers per second from the rows of Y (n x 2 FP32, CUDA)."""
    Y = _cuda(Y, torch.float32, "Y", 2)
    out = C.c_double()
    ctx = context(Y.device.index)
    _check(_lib.load().drgb_gather_probe(ctx, _ptr(Y), Y.shape[0], rounds, seed, C.byref(out),
                                         _stream(Y.device)), ctx)
    return out.value


def knn_uncertified(device=None) -> int:
    ctx = context(device)
    out = C.c_int64()
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    _check(_lib.load().drgb_knn_uncertified(ctx, C.byref(out), _stream(dev)), ctx)
    return out.value


def knn_tiles(device=None) -> tuple[int, int]:
    """(tile products computed, tile products of a full scan) of the last
    tensor-core k-NN call on the device."""
    ctx = context(device)
    done, total = C.c_int64(), C.c_int64()
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    _check(_lib.load().drgb_knn_tiles(ctx, C.byref(done), C.byref(total), _stream(dev)), ctx)
    return done.value, total.value


# ---------------------------------------------------------------- fuzzy graph
def fuzzy_weights(idx: torch.Tensor, dist: torch.Tensor, n_epochs: int,
                  with_rho_sigma: bool = False) -> Graph:
    idx = _cuda(idx, torch.int32, "idx", 2)
    dist = _cuda(dist, torch.float32, "dist", 2)
    n, k = idx.shape
    dev = idx.device
    cap = 2 * n * k
    row_ptr = torch.empty(n + 1, dtype=torch.int32, device=dev)
    col = torch.empty(cap, dtype=torch.int32, device=dev)
    w = torch.empty(cap, dtype=torch.float32, device=dev)
    q = torch.empty(cap, dtype=torch.int32, device=dev)
    rho = torch.empty(n, dtype=torch.float32, device=dev) if with_rho_sigma else None
    sigma = torch.empty(n, dtype=torch.float32, device=dev) if with_rho_sigma else None
    ctx = context(dev.index)
    _check(_lib.load().drgb_fuzzy_weights(ctx, _ptr(idx), _ptr(dist), n, k, n_epochs, _ptr(row_ptr),
                                          _ptr(col), _ptr(w), _ptr(q), cap, _ptr(rho), _ptr(sigma),
                                          _stream(dev)), ctx)
    nnz = int(row_ptr[n].item())
    return Graph(row_ptr, col[:nnz], w[:nnz], q[:nnz], rho, sigma)


def find_ab(spread: float = 1.0, min_dist: float = 0.1):
    a, b = C.c_float(), C.c_float()
    rc = _lib.load().drgb_find_ab(spread, min_dist, C.byref(a), C.byref(b))
    if rc != 0:
        raise DrgbError(rc, "find_ab: invalid spread/min_dist")
    return a.value, b.value


# ---------------------------------------------------------------- embedding
def init_embedding(n: int, init_range: float = 10.0, seed: int = 1, device=None) -> torch.Tensor:
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    Y = torch.empty((n, 2), dtype=torch.float32, device=dev)
    ctx = context(dev.index)
    _check(_lib.load().drgb_init_embedding(ctx, n, init_range, seed, _ptr(Y), _stream(dev)), ctx)
    return Y


def _graph_args(g: Graph):
    return (_ptr(_cuda(g.row_ptr, torch.int32, "row_ptr")), _ptr(_cuda(g.col, torch.int32, "col")),
            _ptr(_cuda(g.q, torch.int32, "q")))


def spectral_init(g: Graph, init_range: float = 10.0, seed: int = 1):
    """Spectral initial layout of the graph (n x 2 FP32) and the three leading
    eigenvalues of its normalised adjacency."""
    n = g.n
    Y = torch.empty((n, 2), dtype=torch.float32, device=g.row_ptr.device)
    ev = (C.c_double * 3)()
    ctx = context(Y.device.index)
    _check(_lib.load().drgb_spectral_init(ctx, _ptr(g.row_ptr), _ptr(g.col), _ptr(g.w), n, init_range, seed,
                                          _ptr(Y), ev, _stream(Y.device)), ctx)
    return Y, [ev[0], ev[1], ev[2]]


def pca(X: torch.Tensor, dim: int = 50):
    """PCA of the rows of X (n x D, FP32 on the GPU) to `dim` components:
    (Z n x dim, components dim x D, mean D, eigenvalues of the covariance)."""
    X = _cuda(X, torch.float32, "X", 2)
    n, D = X.shape
    Z = torch.empty((n, dim), dtype=torch.float32, device=X.device)
    comps = torch.empty((dim, D), dtype=torch.float32, device=X.device)
    mu = torch.empty((D,), dtype=torch.float32, device=X.device)
    ev = (C.c_double * max(dim, 1))()
    ctx = context(X.device.index)
    _check(_lib.load().drgb_pca(ctx, _ptr(X), n, D, dim, _ptr(Z), _ptr(comps), _ptr(mu), ev,
                                _stream(X.device)), ctx)
    return Z, comps, mu, [ev[k] for k in range(dim)]


def embed_epoch(Y: torch.Tensor, g: Graph, a: float, b: float, lr: float, neg: int, epoch: int,
                seed: int, out: torch.Tensor | None = None) -> torch.Tensor:
    Y = _cuda(Y, torch.float32, "Y", 2)
    n = Y.shape[0]
    out = torch.empty_like(Y) if out is None else out
    ctx = context(Y.device.index)
    _check(_lib.load().drgb_embed_epoch(ctx, _ptr(Y), _ptr(out), *_graph_args(g), n, a, b, lr, neg,
                                        epoch, seed, _stream(Y.device)), ctx)
    return out


def embed_epochs(Y: torch.Tensor, g: Graph, a: float, b: float, lr0: float, neg: int, t_begin: int,
                 t_end: int, n_epochs: int, seed: int, tmp: torch.Tensor | None = None) -> torch.Tensor:
    """Epochs [t_begin, t_end) of a T-epoch schedule, in place on Y (contiguous)."""
    if not Y.is_contiguous():
        raise ValueError("Y must be contiguous (updated in place)")
    Y = _cuda(Y, torch.float32, "Y", 2)
    tmp = torch.empty_like(Y) if tmp is None else tmp
    ctx = context(Y.device.index)
    _check(_lib.load().drgb_embed_epochs(ctx, _ptr(Y), _ptr(tmp), *_graph_args(g), Y.shape[0], a, b,
                                         lr0, neg, t_begin, t_end, n_epochs, seed,
                                         _stream(Y.device)), ctx)
    return Y


def _params(**kw) -> Params:
    p = Params()
    _lib.load().drgb_default_params(C.byref(p))
    alias = {"n_neighbors": "k", "negative_sample_rate": "neg", "learning_rate": "lr0"}
    for key, v in kw.items():
        key = alias.get(key, key)
        if key not in dict(Params._fields_):
            raise TypeError(f"unknown parameter {key}")
        setattr(p, key, v)
    return p


def fit_transform(X: torch.Tensor, epoch_callback=None, out: torch.Tensor | None = None,
                  init: str = "random", **params) -> torch.Tensor:
    """Embed the rows of X (n x d FP32, CUDA) into n x 2; synchronous.
    init: "random" (uniform in [-init_range, init_range]^2) or "spectral"
    (the spectral layout of the fuzzy graph, see spectral_init)."""
    X = _cuda(X, torch.float32, "X", 2)
    n, d = X.shape
    if init not in ("random", "spectral"):
        raise ValueError(f"init must be 'random' or 'spectral', not {init!r}")
    p = _params(**params)
    if init == "spectral":
        p.flags |= _lib.FLAG_INIT_SPECTRAL
    Y = torch.empty((n, 2), dtype=torch.float32, device=X.device) if out is None else out
    ctx = context(X.device.index)
    if epoch_callback is None:
        cb = _lib.EPOCH_CB()  # NULL function pointer
    else:
        def _cb(t, ptr, nn, user):
            return int(bool(epoch_callback(t, Y)))
        cb = _lib.EPOCH_CB(_cb)
    _check(_lib.load().drgb_fit_transform(ctx, _ptr(X), n, d, C.byref(p), _ptr(Y), cb, None,
                                          _stream(X.device)), ctx)
    return Y


def fit_transform_batched(X_cat: torch.Tensor, offsets, seeds_init=None, seeds_neg=None,
                          autotune: bool = False, out: torch.Tensor | None = None, **params) -> torch.Tensor:
    """Embed many instances at once: rows offsets[b]:offsets[b+1] of X_cat are
    instance b.  Each instance's result equals fit_transform of its rows alone
    with seeds (seeds_init[b], seeds_neg[b]).  Synchronous."""
    X_cat = _cuda(X_cat, torch.float32, "X_cat", 2)
    off = [int(v) for v in offsets]
    count = len(off) - 1
    p = _params(**params)
    if autotune:
        p.flags |= _lib.FLAG_AUTOTUNE
    Y = torch.empty((X_cat.shape[0], 2), dtype=torch.float32, device=X_cat.device) if out is None else out
    off_arr = (C.c_int64 * (count + 1))(*off)
    si = (C.c_uint64 * count)(*[int(v) for v in seeds_init]) if seeds_init is not None else None
    sn = (C.c_uint64 * count)(*[int(v) for v in seeds_neg]) if seeds_neg is not None else None
    ctx = context(X_cat.device.index)
    _check(_lib.load().drgb_fit_transform_batched(ctx, _ptr(X_cat), off_arr, count, X_cat.shape[1], C.byref(p),
                                                  si, sn, _ptr(Y), _stream(X_cat.device)), ctx)
    return Y


def autotune_epoch(Y: torch.Tensor, g: Graph, a: float, b: float, neg: int = 5, n_epochs: int = 200,
                   seed: int = 2, trials: int = 3):
    """Time the epoch force-kernel settings on this graph; keeps and returns
    the fastest ((warps per CTA, form), microseconds per epoch)."""
    Y = _cuda(Y, torch.float32, "Y", 2)
    choice = (C.c_int32 * 3)()
    us = C.c_float()
    ctx = context(Y.device.index)
    _check(_lib.load().drgb_autotune_epoch(ctx, _ptr(Y), *_graph_args(g), Y.shape[0], a, b, neg, n_epochs, seed,
                                           trials, choice, C.byref(us), _stream(Y.device)), ctx)
    return (int(choice[0]), int(choice[1])), us.value


# ---------------------------------------------------------------- learned embedder
def mlp_param_count() -> int:
    return int(_lib.load().drgb_mlp_param_count())


def mlp_init(d: int, seed: int = 0, device=None) -> torch.Tensor:
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    P = torch.empty(mlp_param_count(), dtype=torch.float32, device=dev)
    ctx = context(dev.index)
    _check(_lib.load().drgb_mlp_init(ctx, _ptr(P), d, seed, _stream(dev)), ctx)
    return P


def mlp_sample(g: Graph, n_edges: int, neg: int = 5, step: int = 0, seed: int = 0) -> torch.Tensor:
    dev = g.row_ptr.device
    rows = torch.empty(n_edges * (2 + neg), dtype=torch.int32, device=dev)
    ctx = context(dev.index)
    _check(_lib.load().drgb_mlp_sample(ctx, *_graph_args(g), g.n, g.nnz, n_edges, neg, step, seed, _ptr(rows),
                                       _stream(dev)), ctx)
    return rows


def mlp_grad(params: torch.Tensor, X: torch.Tensor, rows: torch.Tensor, n_edges: int, neg: int, a: float,
             b: float):
    """(gradient vector, mean batch loss) for explicit rows (n_edges * (2 + neg))."""
    X = _cuda(X, torch.float32, "X", 2)
    rows = _cuda(rows, torch.int32, "rows")
    grad = torch.empty_like(params)
    loss = torch.empty(1, dtype=torch.float32, device=X.device)
    ctx = context(X.device.index)
    _check(_lib.load().drgb_mlp_grad(ctx, _ptr(params), _ptr(X), X.shape[0], X.shape[1], _ptr(rows), n_edges, neg,
                                     a, b, _ptr(grad), _ptr(loss), _stream(X.device)), ctx)
    return grad, float(loss.item())


def mlp_train(X: torch.Tensor, g: Graph, a: float, b: float, params: torch.Tensor, adam_m: torch.Tensor,
              adam_v: torch.Tensor, steps: int, batch_edges: int = 4096, neg: int = 5, lr: float = 1e-3,
              seed: int = 0, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8) -> torch.Tensor:
    """Run `steps` Adam steps in place; returns the per-step losses (device)."""
    X = _cuda(X, torch.float32, "X", 2)
    mp = _lib.MlpParams(steps, batch_edges, neg, lr, beta1, beta2, eps, seed)
    losses = torch.zeros(max(1, steps), dtype=torch.float32, device=X.device)
    ctx = context(X.device.index)
    _check(_lib.load().drgb_mlp_train(ctx, _ptr(X), X.shape[0], X.shape[1], *_graph_args(g), g.nnz, a, b,
                                      C.byref(mp), _ptr(params), _ptr(adam_m), _ptr(adam_v), _ptr(losses),
                                      _stream(X.device)), ctx)
    return losses[:steps]


def mlp_embed(params: torch.Tensor, X: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    X = _cuda(X, torch.float32, "X", 2)
    Y = torch.empty((X.shape[0], 2), dtype=torch.float32, device=X.device) if out is None else out
    ctx = context(X.device.index)
    _check(_lib.load().drgb_mlp_embed(ctx, _ptr(params), _ptr(X), X.shape[0], X.shape[1], _ptr(Y),
                                      _stream(X.device)), ctx)
    return Y


def transform(X_train: torch.Tensor, Y_train: torch.Tensor, X_new: torch.Tensor, **params) -> torch.Tensor:
    """Embed new points by plain optimisation against a fixed training embedding."""
    X_train = _cuda(X_train, torch.float32, "X_train", 2)
    Y_train = _cuda(Y_train, torch.float32, "Y_train", 2)
    X_new = _cuda(X_new, torch.float32, "X_new", 2)
    p = _params(**params)
    Y = torch.empty((X_new.shape[0], 2), dtype=torch.float32, device=X_new.device)
    ctx = context(X_new.device.index)
    _check(_lib.load().drgb_transform(ctx, _ptr(X_train), _ptr(Y_train), X_train.shape[0], _ptr(X_new),
                                      X_new.shape[0], X_new.shape[1], C.byref(p), _ptr(Y), _stream(X_new.device)),
           ctx)
    return Y


class ParametricUMAP:
    """Learned embedder: fit(X) builds the fuzzy graph and trains the MLP on
    it; transform(X_new) embeds new points with one forward pass."""

    def __init__(self, n_neighbors: int = 15, n_epochs: int = 200, passes: float = 50.0,
                 batch_edges: int = 4096, neg: int = 5, lr: float = 1e-3, min_dist: float = 0.1,
                 spread: float = 1.0, seed: int = 0):
        self.k, self.T, self.passes, self.B = n_neighbors, n_epochs, passes, batch_edges
        self.neg, self.lr, self.seed = neg, lr, seed
        self.a, self.b = find_ab(spread, min_dist)
        self.params = None

    def fit(self, X: torch.Tensor):
        X = _cuda(X, torch.float32, "X", 2)
        idx, dist = knn_graph(X, self.k)
        g = fuzzy_weights(idx, dist, self.T)
        self.params = mlp_init(X.shape[1], self.seed, X.device.index)
        m, v = torch.zeros_like(self.params), torch.zeros_like(self.params)
        steps = max(1, int(round(self.passes * g.nnz / self.B)))
        self.losses = mlp_train(X, g, self.a, self.b, self.params, m, v, steps, self.B, self.neg, self.lr,
                                self.seed + 1)
        return self

    def transform(self, X: torch.Tensor) -> torch.Tensor:
        return mlp_embed(self.params, X)


# ---------------------------------------------------------------- metrics
def eval_recall(X: torch.Tensor, Y: torch.Tensor, k: int = 15, n_query: int = 0) -> float:
    X = _cuda(X, torch.float32, "X", 2)
    Y = _cuda(Y, torch.float32, "Y", 2)
    out = C.c_double()
    ctx = context(X.device.index)
    _check(_lib.load().drgb_eval_recall(ctx, _ptr(X), _ptr(Y), X.shape[0], X.shape[1], k, n_query,
                                        C.byref(out), _stream(X.device)), ctx)
    return out.value


def eval_trust(X: torch.Tensor, Y: torch.Tensor, k: int = 15, n_query: int = 0) -> float:
    X = _cuda(X, torch.float32, "X", 2)
    Y = _cuda(Y, torch.float32, "Y", 2)
    out = C.c_double()
    ctx = context(X.device.index)
    _check(_lib.load().drgb_eval_trust(ctx, _ptr(X), _ptr(Y), X.shape[0], X.shape[1], k, n_query,
                                       C.byref(out), _stream(X.device)), ctx)
    return out.value


def eval_recall_heldout(X_train: torch.Tensor, Y_train: torch.Tensor, X_new: torch.Tensor, Y_new: torch.Tensor,
                        k: int = 15, n_query: int = 0) -> float:
    """Held-out k-NN preservation of new points against the training set."""
    Xt = _cuda(X_train, torch.float32, "X_train", 2)
    Yt = _cuda(Y_train, torch.float32, "Y_train", 2)
    Xn = _cuda(X_new, torch.float32, "X_new", 2)
    Yn = _cuda(Y_new, torch.float32, "Y_new", 2)
    if Xt.shape[1] != Xn.shape[1] or Yt.shape[1] != 2 or Yn.shape[1] != 2 or Yt.shape[0] != Xt.shape[0] \
            or Yn.shape[0] != Xn.shape[0]:
        raise ValueError("eval_recall_heldout: shape mismatch")
    out = C.c_double()
    ctx = context(Xt.device.index)
    _check(_lib.load().drgb_eval_recall_heldout(ctx, _ptr(Xt), _ptr(Yt), Xt.shape[0], _ptr(Xn), _ptr(Yn),
                                                Xn.shape[0], Xt.shape[1], k, n_query, C.byref(out),
                                                _stream(Xt.device)), ctx)
    return out.value


def render(Y: torch.Tensor, rgb: torch.Tensor, width: int = 1000, height: int = 1000, radius: float = 2.0,
           alpha: float = 1.0, background=(1.0, 1.0, 1.0), view=None, out: torch.Tensor | None = None,
           return_view: bool = False):
    """Circle-splatting render of the embedding Y (n x 2) with per-point
    colours rgb (n x 3 in [0, 1]) into a height x width x 3 uint8 frame on the
    device.  view = (x0, y0, scale) or None (fitted to the points)."""
    Y = _cuda(Y, torch.float32, "Y", 2)
    rgb = _cuda(rgb, torch.float32, "rgb", 2)
    if Y.shape[1] != 2 or rgb.shape != (Y.shape[0], 3):
        raise ValueError("render: Y must be n x 2 and rgb n x 3")
    frame = torch.empty((height, width, 3), dtype=torch.uint8, device=Y.device) if out is None else out
    bg = (C.c_float * 3)(*background)
    vin = (C.c_float * 3)(*view) if view is not None else None
    vout = (C.c_float * 3)()
    ctx = context(Y.device.index)
    _check(_lib.load().drgb_render(ctx, _ptr(Y), _ptr(rgb), Y.shape[0], width, height, radius, alpha, bg, vin,
                                   vout if return_view else None, _ptr(frame), _stream(Y.device)), ctx)
    if return_view:
        return frame, (vout[0], vout[1], vout[2])
    return frame


class UMAP:
    """Class-based front end mirroring Section 2.1: instantiate with
    hyper-parameters, call fit_transform(X) on an n x d array, receive n x 2."""

    def __init__(self, n_neighbors: int = 15, n_epochs: int = 200, min_dist: float = 0.1,
                 spread: float = 1.0, negative_sample_rate: int = 5, learning_rate: float = 1.0,
                 init_range: float = 10.0, seed: int = 0, knn_mode: int = 0, epoch_callback=None):
        self.params = dict(k=n_neighbors, n_epochs=n_epochs, min_dist=min_dist, spread=spread,
                           neg=negative_sample_rate, lr0=learning_rate, init_range=init_range,
                           seed_init=seed + 1, seed_neg=seed + 2, knn_mode=knn_mode)
        self.epoch_callback = epoch_callback
        self.embedding_ = None

    def fit_transform(self, X) -> torch.Tensor:
        if not isinstance(X, torch.Tensor):
            X = torch.as_tensor(X, dtype=torch.float32)
        if not X.is_cuda:
            X = X.to("cuda", dtype=torch.float32)
        self.embedding_ = fit_transform(X, epoch_callback=self.epoch_callback, **self.params)
        return self.embedding_
