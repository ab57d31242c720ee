"""The C ABI library builds, loads and exports every declared entry point;
host-side behaviour that needs no GPU (not gpu)."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

from conftest import ROOT
from oracle import curve


@pytest.fixture(scope="module")
def lib():
    from paper_2603_04035_gb300 import _lib, build
    build.build()
    return _lib.load()


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(drgb_\w+)\s*\(", src))
    return sorted(n for n in names if n != "drgb_epoch_cb")


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


def test_binding_declares_every_symbol():
    from paper_2603_04035_gb300 import _lib
    assert set(declared_symbols()) <= set(_lib.SIGNATURES)


def test_version_and_defaults(lib):
    from paper_2603_04035_gb300 import _lib
    assert lib.drgb_version() >= 10000
    p = _lib.Params()
    assert lib.drgb_default_params(C.byref(p)) == 0
    assert (p.k, p.n_epochs, p.neg, p.lr0, p.init_range) == (15, 200, 5, 1.0, 10.0)
    assert p.pca_dim == 0                      # no PCA unless asked for
    assert C.sizeof(p) == 64                   # the C struct: 56 bytes of fields, pca_dim, padding
    assert lib.drgb_default_params(None) == _lib.ERR_INVALID


@pytest.mark.parametrize("spread,min_dist", [(1.0, 0.1), (1.0, 0.5), (2.0, 0.25), (1.0, 0.01)])
def test_host_find_ab_matches_oracle(lib, spread, min_dist):
    a, b = C.c_float(), C.c_float()
    assert lib.drgb_find_ab(spread, min_dist, C.byref(a), C.byref(b)) == 0
    a_o, b_o = curve.find_ab(spread, np.float32(min_dist).item())
    assert abs(a.value - a_o) < 1e-5 * a_o and abs(b.value - b_o) < 1e-5 * b_o


def test_find_ab_rejects_bad_arguments(lib):
    from paper_2603_04035_gb300 import _lib
    a, b = C.c_float(), C.c_float()
    assert lib.drgb_find_ab(0.0, 0.1, C.byref(a), C.byref(b)) == _lib.ERR_INVALID
    assert lib.drgb_find_ab(1.0, -0.1, C.byref(a), C.byref(b)) == _lib.ERR_INVALID
    assert lib.drgb_find_ab(1.0, 0.1, None, C.byref(b)) == _lib.ERR_INVALID


def test_null_context_is_rejected_without_touching_a_gpu(lib):
    from paper_2603_04035_gb300 import _lib
    E = _lib.ERR_INVALID
    assert lib.drgb_knn_graph(None, None, 10, 2, 3, 0, None, None, None) == E
    assert lib.drgb_fuzzy_weights(None, None, None, 10, 3, 10, None, None, None, None, 60, None,
                                  None, None) == E
    assert lib.drgb_embed_epoch(None, None, None, None, None, None, 10, 1.0, 1.0, 1.0, 5, 0, 0,
                                None) == E
    assert lib.drgb_embed_epochs(None, None, None, None, None, None, 10, 1.0, 1.0, 1.0, 5, 0, 1, 1,
                                 0, None) == E
    assert lib.drgb_init_embedding(None, 10, 10.0, 0, None, None) == E
    assert lib.drgb_fit_transform(None, None, 10, 2, None, None, _lib.EPOCH_CB(), None, None) == E
    assert lib.drgb_pca(None, None, 10, 4, 2, None, None, None, None, None) == E
    assert lib.drgb_set_scratch_limit(None, 0) == E
    assert lib.drgb_sync(None, None) == E
    assert lib.drgb_ctx_create(0, None) == E
    assert lib.drgb_ctx_destroy(None) == 0
    assert lib.drgb_last_error(None) == b"null context"


@pytest.mark.skipif(os.path.exists("/dev/nvidia0"), reason="host has a GPU")
def test_ctx_create_without_gpu_reports_device_error(lib):
    from paper_2603_04035_gb300 import _lib
    h = C.c_void_p()
    assert lib.drgb_ctx_create(0, C.byref(h)) == _lib.ERR_DEVICE
    assert h.value is None


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2603_04035_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if path.endswith((".py", ".cu", ".cuh", ".h")):
            text = open(path).read()
            assert "oracle" not in re.sub(r"#.*|//.*", "", text).replace("oracle.", ""), path
            assert "import oracle" not in text and "from oracle" not in text, path


def test_wait_selftest_needs_a_context(lib):
    from paper_2603_04035_gb300 import _lib
    assert lib.drgb_wait_selftest(None, 1000, 0, None) == _lib.ERR_INVALID


def test_tuning_cache_round_trip(lib, tmp_path):
    import json
    from paper_2603_04035_gb300 import _lib
    path = str(tmp_path / "tune.json").encode()
    v, pp = C.c_int32(0), C.c_int32(0)
    key = b"NVIDIA GB300|152 SMs|rows 2^21|instances 2^8|k 15"
    assert lib.drgb_tuning_cache_lookup(path, key, C.byref(v), C.byref(pp)) == _lib.ERR_INVALID   # no file yet
    assert lib.drgb_tuning_cache_store(path, key, 8, 1) == 0
    assert lib.drgb_tuning_cache_store(path, b"other|1", 4, 0) == 0
    assert lib.drgb_tuning_cache_lookup(path, key, C.byref(v), C.byref(pp)) == 0 and (v.value, pp.value) == (8, 1)
    assert lib.drgb_tuning_cache_store(path, key, 4, 0) == 0                              # replaced
    assert lib.drgb_tuning_cache_lookup(path, key, C.byref(v), C.byref(pp)) == 0 and (v.value, pp.value) == (4, 0)
    with open(path) as f:
        assert json.load(f) == {key.decode(): {"epoch_warps": 4, "epoch_pipe": 0},
                                "other|1": {"epoch_warps": 4, "epoch_pipe": 0}}
    assert lib.drgb_tuning_cache_lookup(path, b"missing", C.byref(v), C.byref(pp)) == _lib.ERR_INVALID


def test_tuning_cache_rejects_bad_keys_values_and_paths(lib, tmp_path):
    from paper_2603_04035_gb300 import _lib
    path = str(tmp_path / "tune.json").encode()
    for bad in (b"", b'a"b', b"a\\b", b"tab\there", b"x" * 256):
        assert lib.drgb_tuning_cache_store(path, bad, 8, 1) == _lib.ERR_INVALID, bad
    for warps in (0, 5, 16):
        assert lib.drgb_tuning_cache_store(path, b"k", warps, 1) == _lib.ERR_INVALID, warps
    for pipe in (-1, 2):
        assert lib.drgb_tuning_cache_store(path, b"k", 8, pipe) == _lib.ERR_INVALID, pipe
    assert not os.path.exists(path)
    assert lib.drgb_tuning_cache_store(str(tmp_path / "no" / "dir.json").encode(), b"k", 8, 1) == _lib.ERR_INVALID
    assert lib.drgb_set_tuning_cache(None, path) == _lib.ERR_INVALID


def test_tuning_cache_reads_only_its_own_lines(lib, tmp_path):
    from paper_2603_04035_gb300 import _lib
    p = tmp_path / "tune.json"
    p.write_text('{\n  garbage line\n  "a": {"epoch_warps": 6},\n  "b": {"epoch_warps": 4},\n'
                 '  "c": {"epoch_warps": 8, "epoch_pipe": 0},\n  "d": {"epoch_warps": 8, "epoch_pipe": 7}\n}\n')
    v, pp = C.c_int32(0), C.c_int32(0)
    f = str(p).encode()
    assert lib.drgb_tuning_cache_lookup(f, b"b", C.byref(v), C.byref(pp)) == 0 and (v.value, pp.value) == (4, 1)
    assert lib.drgb_tuning_cache_lookup(f, b"c", C.byref(v), C.byref(pp)) == 0 and (v.value, pp.value) == (8, 0)
    assert lib.drgb_tuning_cache_lookup(f, b"a", C.byref(v), C.byref(pp)) == _lib.ERR_INVALID  # unsupported
    assert lib.drgb_tuning_cache_lookup(f, b"d", C.byref(v), C.byref(pp)) == _lib.ERR_INVALID  # bad form


def test_tuning_cache_python_wrappers(lib, tmp_path):
    import paper_2603_04035_gb300 as drgb
    path = str(tmp_path / "t.json")
    assert drgb.tuning_cache_lookup(path, "k") is None
    drgb.tuning_cache_store(path, "k", 8)
    assert drgb.tuning_cache_lookup(path, "k") == (8, 1)
    drgb.tuning_cache_store(path, "k", 4, 0)
    assert drgb.tuning_cache_lookup(path, "k") == (4, 0)
    with pytest.raises(drgb.DrgbError):
        drgb.tuning_cache_store(path, "k", 3)


def test_params_aliases_and_umap_defaults(lib):
    import paper_2603_04035_gb300 as drgb
    p = drgb._params(n_neighbors=10, negative_sample_rate=7, learning_rate=0.5, n_epochs=300)
    assert (p.k, p.neg, p.n_epochs) == (10, 7, 300) and abs(p.lr0 - 0.5) < 1e-7
    with pytest.raises(TypeError):
        drgb._params(no_such_parameter=1)
    u = drgb.UMAP(n_neighbors=12, seed=4, min_dist=0.25)
    assert u.params["k"] == 12 and u.params["min_dist"] == 0.25
    assert (u.params["seed_init"], u.params["seed_neg"]) == (5, 6)   # data seed s: init s+1, negatives s+2
