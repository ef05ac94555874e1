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
                       ("precision", 7), ("newton_max", 0), ("lin_rtol", 0.0), ("kl_ell", -1.0),
                       ("precond", 2), ("mg_nu", 9), ("mg_nu", -1), ("mg_coarse_sweeps", 65)]:
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


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the header's structs have the C sizes and field
    offsets (compiled with the host C compiler from include/mlmc.h)."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no host C compiler")
    structs = [("mlmc_config", B.mlmc_config), ("mlmc_sample_info", B.mlmc_sample_info),
               ("mlmc_server_config", B.mlmc_server_config), ("mlmc_request", B.mlmc_request),
               ("mlmc_result", B.mlmc_result)]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mlmc.h"', "int main(void) {"]
    for name, cls in structs:
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for f in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, f[0], name, f[0]))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)]).decode().splitlines())
    for name, cls in structs:
        assert int(got[name]) == C.sizeof(cls), name
        for f in cls._fields_:
            assert int(got[name + "." + f[0]]) == getattr(cls, f[0]).offset, (name, f[0])


def test_server_rejects_bad_arguments_without_device_work(lib):
    assert lib.mlmc_server_create(None, None, None) == -1
    assert lib.mlmc_server_submit(None, None, 0) == -1
    cnt = C.c_int()
    assert lib.mlmc_server_poll(None, None, 0, C.byref(cnt), None, None, 0, 0.0) == -1
    assert lib.mlmc_server_drain(None, 1.0) == -1
    lib.mlmc_server_destroy(None)


def test_merge_is_host_only(lib):
    # runs with no device present: the cross-device merge needs none
    import numpy as np
    Na, Nb = np.array([2], np.int64), np.array([2], np.int64)
    ma, mb = np.array([1.0, 3.0]), np.array([3.0, 5.0])
    za, zb = np.zeros(2), np.zeros(2)
    qa, qb = np.ones(2), np.full(2, 3.0)
    p = lambda a: a.ctypes.data_as(C.c_void_p)
    assert lib.mlmc_merge_states(1, 2, p(Na), p(ma), p(za), p(qa), p(Nb), p(mb), p(zb), p(qb)) == 0
    assert Na[0] == 4 and list(ma) == [2.0, 4.0] and list(za) == [4.0, 4.0] and list(qa) == [2.0, 2.0]
