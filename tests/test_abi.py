"""The C-ABI library loads and exports every entry point include/farm.h declares
(no compute call: these run without a GPU)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_path():
    import __graft_entry__ as g
    g.build()
    from paper_2606_15476_gb300 import _build
    return _build.LIB


def declared_symbols():
    with open(os.path.join(ROOT, "include", "farm.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(farm_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary_calls():
    names = declared_symbols()
    for must in ("farm_memory_upload", "farm_query_batch", "farm_topk"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = C.CDLL(lib_path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib_path):
    import paper_2606_15476_gb300 as F
    assert set(declared_symbols()) <= set(F.farm.exported_symbols())
    for n in declared_symbols():
        assert callable(getattr(F, n))


def test_default_params_match_the_paper(lib_path):
    import paper_2606_15476_gb300 as F
    p = F.farm_default_params()
    # App. D.2: mu = 5, w = 0.5, class factor 0.3, Near sigma 0.5 m
    assert (p.mu, p.w, p.class_mis, p.sigma_near) == (5.0, 0.5, pytest.approx(0.3), 0.5)
    assert p.k_anchor == 16 and p.k_max == 10


def test_null_context_is_rejected_without_touching_the_gpu(lib_path):
    lib = C.CDLL(lib_path)
    lib.farm_sync.argtypes = [C.c_void_p]
    lib.farm_destroy.argtypes = [C.c_void_p]
    assert lib.farm_sync(None) == 1
    assert lib.farm_destroy(None) == 1
    lib.farm_create.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
    assert lib.farm_create(None, 0, None, None) == 1


def test_bad_params_are_rejected_before_any_cuda_call(lib_path):
    import paper_2606_15476_gb300 as F
    for field, bad in [("w", 1.5), ("class_mis", 0.0), ("tau_v", 0.0), ("k_anchor", 0),
                       ("k_anchor", 1000), ("z_min", -1.0), ("k_max", 0)]:
        p = F.farm_default_params()
        setattr(p, field, bad)
        with pytest.raises(F.FarmError) as ei:
            F.farm_create(0, None, p)
        assert ei.value.status == 1, field
    p = F.farm_default_params()
    p.class_mis = 0.01     # rank bound (5+10)/(0.5*0.01)-5 far above 512
    with pytest.raises(F.FarmError):
        F.farm_create(0, None, p)


def test_version_string(lib_path):
    import paper_2606_15476_gb300 as F
    assert "sm_103a" in F.farm_version()
