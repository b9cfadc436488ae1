"""The C-ABI library loads and exports every entry point include/bsvd.h
declares. No compute call is made, so this runs without a GPU."""
import ctypes
import os
import re

import paper_1907_07410_gb300 as bs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(bsvd_[a-z_0-9]+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    lib = bs.load()
    declared = declared_symbols()
    assert "bsvd_partition" in declared and "bsvd_factor" in declared
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared <= set(bs.EXPORTS) | declared
    assert set(bs.EXPORTS) <= declared


def test_config_layout_matches_header():
    cfg = bs.bsvd_config_default()
    assert cfg.cheb_degree == 8 and cfg.max_iters == 30
    assert cfg.tol == 0.0          # per-precision default in bsvd_create
    assert cfg.clamp_lo == 1.0 and cfg.clamp_hi == 5.0
    # int32 x2, float x2, int32 x6, double, uint64, pointer, int32 x2
    assert ctypes.sizeof(bs.Config) == 72
    assert bs.Config.tol.offset == 40 and bs.Config.stream.offset == 56
    assert bs.Config.panel_path.offset == 64 and cfg.panel_path == 0


def test_sgd_params_layout_matches_header():
    prm = bs.SgdParams()
    prm.precision = 7
    prm.max_steps = -3
    bs.load().bsvd_sgd_params_default(ctypes.byref(prm))
    assert prm.k == 13 and prm.max_steps == 100 and prm.a_user == 0.019
    # the last field is written where the binding reads it
    assert prm.precision == bs.SGD_FP64 == 0 and bs.SGD_FP32 == 1
    # double x9, int32 x3, padded to 8
    assert ctypes.sizeof(bs.SgdParams) == 88
    assert bs.SgdParams.precision.offset == 80


def test_binding_signatures_match_header_arity():
    """Every declared function has ctypes argument types, as many as the
    header's parameter list (a missing one would silently convert a pointer
    to a C int)."""
    lib = bs.load()
    text = ""
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text += open(os.path.join(ROOT, "include", fn)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    decls = re.findall(r"\b(bsvd_[a-z_0-9]+)\s*\(([^)]*)\)\s*;", text)
    assert len(decls) >= 20
    for name, params in decls:
        params = params.strip()
        arity = 0 if params in ("", "void") else params.count(",") + 1
        f = getattr(lib, name)
        assert f.argtypes is not None, name
        assert len(f.argtypes) == arity, (name, len(f.argtypes), arity)
