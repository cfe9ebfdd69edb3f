"""The C-ABI library builds, loads without a GPU and exports every function
declared in include/galnb.h; the binding declares the same names."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \*]*?\b(gnb_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_exports_header_symbols():
    from paper_2510_23330_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_has_same_names():
    from paper_2510_23330_gb300 import galnb
    for n in _declared():
        assert callable(getattr(galnb, n)), n


def test_config_defaults_without_gpu():
    from paper_2510_23330_gb300 import galnb
    cfg = galnb.gnb_config()
    galnb.gnb_config_default(cfg)
    assert cfg.G == 1.0 and cfg.theta == 0.5 and cfg.n_leaf == 16 and cfg.n_ngb == 64
    assert abs(cfg.gamma - 5.0 / 3.0) < 1e-15 and cfg.multipole == 1


def test_null_context_errors_without_gpu():
    from paper_2510_23330_gb300 import galnb
    L = galnb.lib()
    assert L.gnb_build_tree(None) == galnb.GNB_EINVAL
    assert L.gnb_compute_gravity(None, 0) == galnb.GNB_EINVAL
    assert galnb.gnb_last_error(None) == "null context"
    cfg = galnb.gnb_config()
    galnb.gnb_config_default(cfg)
    cfg.n_ngb = 32
    h = ctypes.c_void_p()
    assert galnb.gnb_create(ctypes.byref(h), cfg) == galnb.GNB_EINVAL
