"""The C-ABI library builds, loads without a GPU and exports every symbol the header
declares; the header and the binding agree on the list."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_symbols():
    src = open(os.path.join(ROOT, "include", "locpir.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lp_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2407_19871_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(built_lib):
    L = ctypes.CDLL(built_lib)
    syms = _header_symbols()
    assert len(syms) >= 20
    for s in syms:
        assert hasattr(L, s), s


def test_binding_lists_every_declared_symbol():
    from paper_2407_19871_gb300 import locpir
    assert sorted(locpir.EXPORTS) == _header_symbols()


def test_host_only_entry_points_without_gpu(built_lib):
    from paper_2407_19871_gb300 import locpir
    L = locpir.lib()
    p = locpir.params_default()
    assert (p.n, p.N, p.k, p.Bgbit, p.lg, p.basebit, p.t) == (630, 1024, 1, 10, 3, 2, 8)
    assert L.lp_strerror(locpir.LP_ETIMEOUT) == b"device wait timed out"
    # Argument validation happens before any device call.
    bad = locpir.lp_params(630, 2048, 1, 10, 3, 2, 8)
    h = ctypes.c_void_p()
    assert L.lp_create(ctypes.byref(bad), 0, ctypes.byref(h)) == locpir.LP_EINVAL
    assert b"unsupported" in L.lp_last_error()
    assert L.lp_gate_batch(None, 0, None, None, None, None, 1, None) == locpir.LP_EINVAL
