"""The C ABI library loads and exports every function include/rpca.h declares (CPU only:
no compute call is made without a GPU)."""
import ctypes

import pytest

P = pytest.importorskip("paper_1711_05519_gb300")


@pytest.fixture(scope="module")
def lib():
    from paper_1711_05519_gb300 import build

    build.build()
    return P.lib()


def test_exports_every_declared_function(lib):
    names = P.header_functions()
    assert len(names) >= 10
    missing = [f for f in names if not hasattr(lib, f)]
    assert not missing, missing


def test_host_only_calls(lib):
    p = P.rpca.Params()
    assert lib.rpca_params_default(ctypes.byref(p)) == P.OK
    assert (p.max_iter, p.trim, p.precision, p.zeta_mode) == (100, 1, 1, 0)
    assert P.status_string(P.CAPACITY) == "RPCA_ERR_CAPACITY"
    assert P.status_string(99) == "RPCA_UNKNOWN_STATUS"
    assert lib.rpca_create(None, None, None) == P.INVALID_ARG
    assert lib.rpca_params_default(None) == P.INVALID_ARG
    ctx = ctypes.c_void_p()
    bad = P.rpca.Params()
    lib.rpca_params_default(ctypes.byref(bad))
    bad.beta, bad.gamma, bad.tol = 0.1, 1.5, 1e-5  # gamma must be < 1
    assert lib.rpca_create(ctypes.byref(ctx), ctypes.byref(bad), None) == P.INVALID_ARG
    assert lib.rpca_solve_host(None, 10, 10, 1, 0.1, 0.5, 1e-5, None, None, None, None, None, 0, None, None,
                               None) == P.INVALID_ARG
    assert lib.rpca_set_lowrank(None, None, None, None, 0, 0.0, 0) == P.INVALID_ARG
    assert lib.rpca_get_state(None, None, None, None) == P.INVALID_ARG
    assert lib.rpca_selftest_waits(None, None) == P.INVALID_ARG
    lib.rpca_solve_host_release()  # nothing kept yet: a no-op


def test_struct_layouts_match_the_header(tmp_path):
    # the ctypes mirrors of rpca_params and rpca_iter_stats against the C compiler's layout
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    root = P.rpca._HERE.rsplit("/", 1)[0]
    fields = {"rpca_params": [f for f, _ in P.rpca.Params._fields_],
              "rpca_iter_stats": [f for f, _ in P.rpca.IterStats._fields_]}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "rpca.h"', "int main(void) {"]
    for st, fs in fields.items():
        lines.append(f'  printf("{st} size %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'  printf("{st} {f} %zu\\n", offsetof({st}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-std=c99", "-I", root + "/include", str(src), "-o", str(exe)])
    got = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        st, f, v = line.split()
        got[(st, f)] = int(v)
    for st, cls in (("rpca_params", P.rpca.Params), ("rpca_iter_stats", P.rpca.IterStats)):
        assert got[(st, "size")] == ctypes.sizeof(cls), st
        for f in fields[st]:
            assert got[(st, f)] == getattr(cls, f).offset, (st, f)
