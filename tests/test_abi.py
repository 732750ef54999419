"""CPU checks of the C ABI: the library builds, loads without a GPU and
exports every entry point declared in include/mpk.h; host-only helpers agree
with the oracle."""
import re

import numpy as np

import oracle
import paper_2205_01598_gb300 as mpk


def _declared():
    text = open(mpk.HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mpk_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    mpk.build()
    lib = mpk.load()
    names = _declared()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name


def test_strerror_and_defaults_need_no_gpu():
    assert mpk.mpk_strerror(0) == "ok"
    assert "timed out" in mpk.mpk_strerror(mpk.MPK_ERR_TIMEOUT)
    o = mpk.mpk_opts_default()
    assert o.safety_f == 0.5 and o.nrhs == 1 and o.root == 0 and o.prec == mpk.MPK_F64


def test_schroedinger_coefficients_match_oracle():
    for M, c, r, dt in [(64, 0.01, 14.25, 50 / 14.25), (10, -2.0, 3.0, 0.4)]:
        got = mpk.mpk_cheb_coeffs_schroedinger(M, c, r, dt)
        ref = oracle.cheb_coeffs_schroedinger(M, c, r, dt)
        assert np.max(np.abs(got - ref)) <= 1e-15


def test_product_path_does_not_touch_the_oracle():
    """The library package neither imports nor loads anything under oracle/."""
    import os
    pkg = os.path.dirname(mpk.__file__)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(root, f)).read()
                assert "import oracle" not in src and "oracle/" not in src and "mpk_oracle" not in src, f


def test_ctypes_structs_match_the_header(tmp_path):
    """The binding's ctypes structures have the C header's sizes and field
    offsets (compiled with the host C compiler), so appended fields such as
    mpk_opts.sweep land where the library reads them."""
    import ctypes as C
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        import pytest
        pytest.skip("no host C compiler")
    structs = {"mpk_opts": mpk.mpk_opts, "mpk_plan_stats": mpk.mpk_plan_stats,
               "mpk_tune_candidate": mpk.mpk_tune_candidate}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{mpk.HEADER}"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{name}.{field} %zu\\n", offsetof({name}, {field}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", str(src), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                          text=True).stdout.split("\n") if l)
    for name, cls in structs.items():
        assert int(out[name]) == C.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(out[f"{name}.{field}"]) == getattr(cls, field).offset, f"{name}.{field}"
