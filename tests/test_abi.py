"""The C ABI library builds, loads and exports every entry point declared in
include/rp.h.  No compute call is made, so this runs without a GPU."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    # function declarations; "rp_status (*field)(...)" inside a struct is a callback type, not an entry point
    names = set(re.findall(r"\b(rp_[a-z_0-9]+)\s*\(", src)) - {"rp_status"}
    return sorted(names)


@pytest.fixture(scope="module")
def lib_path():
    from paper_2602_08097_gb300 import build as b
    return b.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("rp_load_graph", "rp_tune", "rp_tune_batch", "rp_search", "rp_graph_export", "rp_knn",
                 "rp_recall", "rp_build_knn_base", "rp_create", "rp_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (rp_[a-z_0-9]+)\b", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"


def test_library_loads_without_a_gpu(lib_path):
    import paper_2602_08097_gb300 as rp
    lib = rp.load_library()
    for n in _declared():
        assert hasattr(lib, n)


def test_binding_has_the_same_names():
    import paper_2602_08097_gb300 as rp
    for n in _declared():
        if n == "rp_stats_t":
            continue
        assert hasattr(rp, n), n


def test_missing_library_fails_loudly(tmp_path):
    import paper_2602_08097_gb300 as rp
    with pytest.raises(ImportError):
        rp.load_library.__wrapped__(str(tmp_path / "nope.so")) if hasattr(rp.load_library, "__wrapped__") else \
            _load_fresh(rp, str(tmp_path / "nope.so"))


def _load_fresh(rp, path):
    saved = rp._lib
    rp._lib = None
    try:
        return rp.load_library(path)
    finally:
        rp._lib = saved



def test_no_alloc_binding_rejects_host_arrays_before_the_call(lib_path):
    """rp_search_noalloc hands its pointers straight to a kernel, so the binding
    refuses host memory (numpy arrays, CPU tensors) before the library sees a
    pointer; this needs no GPU."""
    import numpy as np
    torch = pytest.importorskip("torch")
    import paper_2602_08097_gb300 as rp
    X = np.zeros((10, 16), dtype=np.uint8)
    row_ptr = np.zeros(11, dtype=np.int64)
    col = np.zeros(1, dtype=np.int32)
    with pytest.raises(TypeError):
        rp.rp_search_noalloc(X, row_ptr, col, 0, X[:2], 8, 4)
    with pytest.raises(TypeError):
        rp.rp_search_noalloc(torch.from_numpy(X), torch.from_numpy(row_ptr), torch.from_numpy(col), 0,
                             torch.from_numpy(X[:2]), 8, 4)
