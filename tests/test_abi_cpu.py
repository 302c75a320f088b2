"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point include/qn.h declares, validates arguments before touching
the device, and its host-only Error metric (Eq. 1) agrees with the oracle's."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(qn_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def qn():
    from paper_2210_15874_gb300 import build
    build.build()
    from paper_2210_15874_gb300 import qn as mod
    return mod


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("qn_batch_create", "qn_batch_set_stream", "qn_batch_set_allocator", "qn_run_qaoa",
                     "qn_expectation", "qn_probs", "qn_grad", "qn_traj_debug", "qn_last_error",
                     "qn_batch_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(qn):
    lib = ctypes.CDLL(qn.LIBRARY_PATH)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert set(declared_symbols()) == set(qn.EXPORTED)


def test_create_validates_before_device_work(qn):
    h = ctypes.c_void_p()
    assert qn.qn_batch_create(0, 10, 1, ctypes.byref(h)) == qn.QN_EINVAL
    assert b"n = 0" in qn.qn_last_error()
    assert qn.qn_batch_create(31, 10, 1, ctypes.byref(h)) == qn.QN_EINVAL
    assert qn.qn_batch_create(4, 0, 1, ctypes.byref(h)) == qn.QN_EINVAL
    assert qn.qn_batch_create(4, 8, 1, None) == qn.QN_EINVAL
    assert qn.qn_batch_create(4, 8, 1, ctypes.byref(h)) == qn.QN_OK
    m, s = ctypes.c_double(), ctypes.c_double()
    assert qn.qn_expectation(h, ctypes.byref(m), ctypes.byref(s)) == qn.QN_ESTATE
    assert qn.qn_batch_set_launch_batch(h, -1) == qn.QN_EINVAL
    for bad in (-1, 3):
        assert qn.qn_batch_set_launch_mode(h, bad) == qn.QN_EINVAL
    for good in (0, 1, 2):
        assert qn.qn_batch_set_launch_mode(h, good) == qn.QN_OK
    c, r, u = ctypes.c_int64(-1), ctypes.c_int64(-1), ctypes.c_int64(-1)
    assert qn.qn_graph_info(h, ctypes.byref(c), ctypes.byref(r), ctypes.byref(u)) == qn.QN_OK
    assert (c.value, r.value, u.value) == (0, 0, 0)
    assert qn.qn_graph_info(h, None, None, None) == qn.QN_OK
    assert qn.qn_graph_info(None, None, None, None) == qn.QN_EINVAL
    qn.qn_batch_destroy(h)
    qn.qn_batch_destroy(None)


def test_fidelity_error_matches_oracle(qn):
    import oracle
    rng = np.random.default_rng(0)
    for d in (2, 16, 256):
        a = rng.random(d); a /= a.sum()
        b = rng.random(d); b /= b.sum()
        assert abs(qn.fidelity_error(a, b) - oracle.error(a, b)) < 1e-15
    with pytest.raises(qn.QnError):
        qn.fidelity_error([-0.1, 1.1], [0.5, 0.5])
