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
