"""The C-ABI library loads and exports every entry point include/cs_hsi.h declares;
argument errors that need no device are reported (CPU only, no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2401_14762_gb300 import build, cs
    build.build()
    return cs.load_library()


def declared():
    hdr = open(os.path.join(ROOT, "include", "cs_hsi.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(cs_[a-z_0-9]+)\s*\(", hdr)))


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    from paper_2401_14762_gb300 import cs
    assert sorted(cs.EXPORTED) == names


def test_defaults(lib):
    from paper_2401_14762_gb300 import cs
    o = cs.cs_opts_default()
    assert o.eps == 1e-8 and o.max_iters == 100 and o.prec == cs.CS_FP32 and o.mu == 0.1
    assert o.iters_out is None and o.converged_out is None and o.kappa_per_pixel is None
    assert o.cycle_skip == 1


def test_errors_before_any_device_work(lib):
    from paper_2401_14762_gb300 import cs
    h = ctypes.c_void_p()
    assert lib.cs_create(ctypes.byref(h), 10, 5, None, None, None, 0.0, None) == cs.CS_ERR_SHAPE
    assert lib.cs_create(ctypes.byref(h), 129, 200, None, None, None, 0.0, None) == cs.CS_ERR_SHAPE
    assert lib.cs_create(ctypes.byref(h), 10, 257, None, None, None, 0.0, None) == cs.CS_ERR_SHAPE
    assert lib.cs_create(ctypes.byref(h), 10, 20, None, None, None, 0.0, None) == cs.CS_ERR_ARG
    assert lib.cs_create(None, 10, 20, None, None, None, 0.0, None) == cs.CS_ERR_ARG
    assert lib.cs_recover_gomp(None, None, None, 0, 4, 2, None) == cs.CS_ERR_ARG
    assert lib.cs_get_lipschitz(None, None) == cs.CS_ERR_ARG
    assert lib.cs_sync(None) == cs.CS_ERR_ARG
    assert "ctx" in cs.cs_last_error()
    lib.cs_destroy(None)
    # batches: empty, NULL parameters or an unknown algorithm are argument errors
    prm = cs.cs_algo_params(1e-3, 1.0, 10, 4, 2)
    items = (cs.cs_batch_item * 1)()
    assert lib.cs_recover_batch(None, 1, cs.CS_ALGO_GOMP, ctypes.byref(prm), None) == cs.CS_ERR_ARG
    assert lib.cs_recover_batch(items, 0, cs.CS_ALGO_GOMP, ctypes.byref(prm), None) == cs.CS_ERR_ARG
    assert lib.cs_recover_batch(items, 1, cs.CS_ALGO_GOMP, None, None) == cs.CS_ERR_ARG
    assert lib.cs_recover_batch(items, 1, 7, ctypes.byref(prm), None) == cs.CS_ERR_ARG
    # sparsification: a NULL context is an argument error
    assert lib.cs_sparsify(None, None, None, 0, 0.1, 1, None, None) == cs.CS_ERR_ARG
    # complex contexts: shape limits and a NULL dictionary are reported before any device
    # work (the real form doubles M and N: M <= 64, N <= 128)
    assert lib.cs_create_complex(ctypes.byref(h), 65, 128, None, 0.0, None) == cs.CS_ERR_ARG
    A = (ctypes.c_double * (2 * 65 * 130))()
    assert lib.cs_create_complex(ctypes.byref(h), 65, 130, A, 0.0, None) == cs.CS_ERR_SHAPE
    assert lib.cs_create_complex(ctypes.byref(h), 8, 4, A, 0.0, None) == cs.CS_ERR_SHAPE
    assert lib.cs_create_complex(None, 8, 16, A, 0.0, None) == cs.CS_ERR_ARG
