"""The C ABI library loads without a GPU, exports every declared entry point,
and its struct layouts match the Python binding."""
import ctypes as ct
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ppd.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1701_01748_gb300 import build
    path = build.build()
    return ct.CDLL(path)


def declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"PPD_API[^;(]*?\b(ppd_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for core in ("ppd_create", "ppd_set_visibilities", "ppd_set_weights", "ppd_iterate", "ppd_get_image"):
        assert core in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    from paper_1701_01748_gb300 import ppd
    cfg = ppd.ppd_config_default(n0=64, n1=64)
    assert cfg.oversample == 2 and cfg.kernel_width == 8 and cfg.wavelet_levels == 4
    assert abs(cfg.tau - 0.49) < 1e-15 and cfg.lambda_ == 1.0 and abs(cfg.kappa - 1e-4) < 1e-20
    assert cfg.n_itr == 1 and cfg.precond == 1
    assert ppd.ppd_status_string(-6) == "call out of order"
    assert ppd.ppd_status_string(0) == "ok"
    # argument checks happen before any device work
    h = ct.c_void_p()
    bad = ppd.ppd_config_default(n0=100, n1=100)
    assert ppd._lib().ppd_create(ct.byref(h), ct.byref(bad)) == ppd.PPD_ERR_UNSUPPORTED
    bad = ppd.ppd_config_default(n0=64, n1=64, lambda_=0.5)
    assert ppd._lib().ppd_create(ct.byref(h), ct.byref(bad)) == ppd.PPD_ERR_INVALID_ARG
    assert ppd._lib().ppd_create(None, ct.byref(bad)) == ppd.PPD_ERR_INVALID_ARG
    assert ppd._lib().ppd_iterate(None, 1, None) == ppd.PPD_ERR_INVALID_ARG
    assert ppd._lib().ppd_launch_count(None) == 0


def test_struct_layout_matches_binding(tmp_path):
    from paper_1701_01748_gb300 import ppd
    prog = tmp_path / "layout.c"
    fields = {"ppd_config": [f for f, _ in ppd.ppd_config._fields_],
              "ppd_stats": [f for f, _ in ppd.ppd_stats._fields_],
              "ppd_params": [f for f, _ in ppd.ppd_params._fields_]}
    lines = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{HEADER}"', "int main(void){"]
    for s, fs in fields.items():
        lines.append(f'printf("%zu\\n", sizeof({s}));')
        for f in fs:
            cf = "lambda" if f == "lambda_" else f
            lines.append(f'printf("%zu\\n", offsetof({s}, {cf}));')
    lines.append("return 0;}")
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", str(prog), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = []
    for s, fs in fields.items():
        cls = getattr(ppd, s)
        want.append(ct.sizeof(cls))
        want.extend(getattr(cls, f).offset for f in fs)
    assert got == want
