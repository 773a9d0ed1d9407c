"""C-ABI checks that need no GPU: the library builds, loads, exports every entry point
include/lbmd.h declares, and rejects invalid arguments before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "lbmd.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lbmd_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1306_0788_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    from paper_1306_0788_gb300 import lbmd
    assert sorted(lbmd.EXPORTS) == names


def test_binding_has_the_same_names():
    from paper_1306_0788_gb300 import lbmd
    for n in _declared():
        assert callable(getattr(lbmd, n)), n


@pytest.mark.parametrize("field,value", [("nx", 0), ("tau_r", 0.5), ("dt", 0.5), ("kT", -1.0), ("storage", 7)])
def test_create_rejects_invalid_params_without_device(field, value):
    from paper_1306_0788_gb300 import lbmd
    p = lbmd.params((4, 4, 4))
    setattr(p, field, value)
    with pytest.raises(lbmd.LbmdError) as e:
        lbmd.lbmd_create(p)
    assert e.value.code == lbmd.LBMD_E_INVALID_ARG
    assert lbmd.lbmd_last_error(None)


def test_product_path_has_no_oracle_or_cpu_fallback():
    """The library binding must not import the oracle and must fail loudly without the .so."""
    src = open(os.path.join(ROOT, "paper_1306_0788_gb300", "lbmd.py")).read()
    assert "oracle" not in src.replace("oracle-free", "")
    csrc = os.path.join(ROOT, "paper_1306_0788_gb300", "csrc")
    for f in os.listdir(csrc):
        assert "lbmd_oracle" not in open(os.path.join(csrc, f)).read()
    assert "raise ImportError" in src


@pytest.mark.parametrize("storage,max_slots", [(7, 4), (0, 0), (0, 70000)])
def test_batch_create_rejects_invalid_arguments_without_device(storage, max_slots):
    from paper_1306_0788_gb300 import lbmd
    with pytest.raises(lbmd.LbmdError) as e:
        lbmd.lbmd_batch_create(0, storage, max_slots)
    assert e.value.code == lbmd.LBMD_E_INVALID_ARG
    assert lbmd.lbmd_batch_last_error(None)


@pytest.mark.parametrize("field,value", [("collision", 5), ("lambda_bulk", 0.0), ("lambda_mom", -2.0),
                                         ("lambda_ghost", 0.3)])
def test_create_rejects_invalid_collision_without_device(field, value):
    from paper_1306_0788_gb300 import lbmd
    p = lbmd.params((4, 4, 4), collision=lbmd.LBMD_COLLISION_MRT)
    setattr(p, field, value)
    with pytest.raises(lbmd.LbmdError) as e:
        lbmd.lbmd_create(p)
    assert e.value.code == lbmd.LBMD_E_INVALID_ARG


@pytest.mark.parametrize("k", [0, 257])
def test_create_rejects_invalid_substeps_without_device(k):
    from paper_1306_0788_gb300 import lbmd
    p = lbmd.params((4, 4, 4), md_substeps=k)
    with pytest.raises(lbmd.LbmdError) as e:
        lbmd.lbmd_create(p)
    assert e.value.code == lbmd.LBMD_E_INVALID_ARG


@pytest.mark.parametrize("diag_every,tol", [(-1, 0.0), (5, 0.0), (5, -1e-3), (5, float("inf")), (5, float("nan"))])
def test_create_rejects_invalid_drift_check_without_device(diag_every, tol):
    from paper_1306_0788_gb300 import lbmd
    p = lbmd.params((4, 4, 4), diag_every=diag_every, drift_tol=tol)
    with pytest.raises(lbmd.LbmdError) as e:
        lbmd.lbmd_create(p)
    assert e.value.code == lbmd.LBMD_E_INVALID_ARG
    assert "diag_every" in lbmd.lbmd_last_error(None)


def test_every_entry_point_refuses_a_null_handle_without_device():
    """Each call that takes a context or a batch returns LBMD_E_INVALID_ARG (the counters -1)
    for a NULL handle, before touching the device; destroy(NULL) is a no-op."""
    import ctypes
    from paper_1306_0788_gb300 import lbmd
    lib = lbmd._lib
    no_handle = {"lbmd_create", "lbmd_batch_create", "lbmd_fluid_moments_static", "lbmd_last_error",
                 "lbmd_batch_last_error", "lbmd_destroy", "lbmd_batch_destroy"}
    checked = 0
    for name in lbmd.EXPORTS:
        if name in no_handle:
            continue
        fn = getattr(lib, name)
        args = [0 if a in (ctypes.c_int, ctypes.c_int64, ctypes.c_size_t) else 1.0 if a is ctypes.c_double else None
                for a in fn.argtypes]
        assert fn(*args) == lbmd.LBMD_E_INVALID_ARG, name  # -1 for the counters too
        checked += 1
    assert checked >= 35
    lib.lbmd_destroy(None)
    lib.lbmd_batch_destroy(None)
