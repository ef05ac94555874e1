"""Host-side checks of the C ABI (no GPU): the library builds, loads and exports
every entry point declared in include/mlmc.h; argument errors are reported as
status codes before any device work."""
import ctypes as C
import os
import re

import pytest

from paper_1911_06066_gb300 import binding as B
from paper_1911_06066_gb300 import build as Bd
from paper_1911_06066_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "mlmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mlmc_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    Bd.build()
    return B.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(B.exported_symbols()) == names


def test_invalid_configs_rejected_on_host(lib):
    cfg = B.make_config(W.MC2D_32)
    for field, bad in [("dim", 4), ("n_levels", 0), ("n_levels", 9), ("m0", 0), ("kl_modes", 0),
                       ("precision", 7), ("newton_max", 0), ("lin_rtol", 0.0), ("kl_ell", -1.0)]:
        c = B.make_config(W.MC2D_32)
        setattr(c, field, bad)
        h = C.c_void_p()
        st = lib.mlmc_create(C.byref(c), C.byref(h))
        assert st == -1 and not h.value, field
        assert lib.mlmc_last_error(None)
    assert lib.mlmc_create(None, None) == -1


def test_null_context_rejected(lib):
    assert lib.mlmc_xi(None, 0, 0, None, 0, None, None) == -1
    assert lib.mlmc_solve(None, 0, None, 0, None, None, None, None, 0, None) == -1
    assert lib.mlmc_estimate(None, None, None, None, None, None, None, None, None) == -1
    b = C.c_size_t()
    assert lib.mlmc_workspace_bytes(None, 0, 1, C.byref(b)) == -1


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(B, "_lib", None)
    monkeypatch.setattr(B, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        B.lib()
