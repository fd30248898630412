"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every entry point include/ckks_kan.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b((?:ckks|kan)_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    n = declared()
    for f in ("ckks_keygen", "ckks_encrypt", "ckks_decrypt", "ckks_add", "ckks_mul_relin",
              "ckks_rescale", "ckks_rotate", "kan_layer_eval", "kan_infer"):
        assert f in n


def test_library_exports_every_declared_symbol():
    from paper_2409_07751_gb300 import build
    path = build.build()
    L = ctypes.CDLL(path)
    missing = [n for n in sorted(declared()) if not hasattr(L, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_2409_07751_gb300 import ckks
    assert declared() <= set(ckks.SIGNATURES)


def test_model_descriptor_b0_forms_and_stages():
    """Both forms of the order-0 basis (Algorithm 2's product, the difference
    of knot comparisons) and both matvec forms (hoisted, double hoisted)
    marshal; another form, or a composite mixing f_n orders with coefficient
    lists, is refused."""
    import numpy as np
    import pytest
    from paper_2409_07751_gb300 import ckks, workloads as W
    m = W.make_model("t", widths=[3, 2], G=3, k=2)
    d = ckks._descs(m, [])
    assert d[0].b0_form == 0 and d[0].n_comp_poly == 0
    m[0]["b0"] = "difference"
    m[0]["comp"] = [np.array([1.5, -0.5]), np.array([2.0])]
    d = ckks._descs(m, [])
    assert d[0].b0_form == 1 and d[0].n_comp_poly == 2
    m[0]["b0"] = "ratio"
    with pytest.raises(ValueError):
        ckks._descs(m, [])
    m[0]["b0"] = "product"
    m[0]["comp"] = [3, np.array([1.0])]
    with pytest.raises(ValueError):
        ckks._descs(m, [])
    m[0]["comp"] = [3]
    m[0]["bsgs"] = "double"
    assert ckks._descs(m, [])[0].bsgs_form == 1
    m[0]["bsgs"] = "triple"
    with pytest.raises(ValueError):
        ckks._descs(m, [])
