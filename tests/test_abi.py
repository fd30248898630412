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


def test_model_descriptor_rejects_unsupported_b0_form():
    """Layers asking for the difference form of the order-0 basis are
    refused by the binding instead of being evaluated in another form."""
    import pytest
    from paper_2409_07751_gb300 import ckks, workloads as W
    m = W.make_model("t", widths=[3, 2], G=3, k=2)
    ckks._descs(m, [])  # the product form builds
    m[0]["b0"] = "difference"
    with pytest.raises(ValueError):
        ckks._descs(m, [])
