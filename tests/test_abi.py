"""CPU checks of the C ABI library and of the oracle/product separation (no GPU calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "chebmg.h")
PKG = os.path.join(ROOT, "paper_2210_03179_gb300")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(chebmg_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def built():
    import __graft_entry__ as g
    g.build()
    import paper_2210_03179_gb300 as cm
    return cm


def test_library_exports_every_declared_symbol(built):
    names = declared_functions()
    assert len(names) >= 18
    handle = ctypes.CDLL(str(built.LIB_PATH))
    missing = [n for n in names if not hasattr(handle, n)]
    assert not missing, missing


def test_binding_covers_the_header(built):
    assert set(declared_functions()) == set(built._SIGNATURES)


def test_host_only_entry_points(built):
    L = built.lib()
    assert L.chebmg_strerror(built.CHEBMG_ENOTCONV).decode() == "not converged"
    o = built.chebmg_opts()
    L.chebmg_default_opts(ctypes.byref(o))
    assert (o.kind, o.order, o.sided, o.prec, o.lanczos_steps) == (5, 2, 1, 0, 30)
    assert o.lmin_ratio == 0.1 and o.coarse_rtol == 1e-10
    # argument validation happens before any device call
    ctx = ctypes.c_void_p()
    assert L.chebmg_setup_fd2d(62, 1.0, 1.0, 2, 7, ctypes.byref(o), ctypes.byref(ctx)) == built.CHEBMG_EINVAL
    bad = built.chebmg_opts()
    L.chebmg_default_opts(ctypes.byref(bad))
    bad.order = 9          # one-sided order 18 > 16 tabulated betas
    assert L.chebmg_setup_fd2d(63, 1.0, 1.0, 2, 7, ctypes.byref(bad), ctypes.byref(ctx)) == built.CHEBMG_EINVAL
    assert L.chebmg_apply_A(None, 0, 0, None, None) == built.CHEBMG_EINVAL


def test_struct_layout_matches_header():
    import paper_2210_03179_gb300 as cm
    # int x4, double x2, int (+pad), ptr, double, int (+pad), ptr  -> 72 bytes on LP64
    assert ctypes.sizeof(cm.chebmg_opts) == 72


def _sources(top, exts):
    for d, _, files in os.walk(top):
        for f in files:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_product_never_touches_the_oracle():
    pat = re.compile(r"\boracle\b")
    for path in _sources(PKG, (".py", ".cu", ".cuh", ".cpp", ".h")):
        text = open(path).read()
        assert not pat.search(text), f"{path} mentions the oracle"
    for path in _sources(os.path.join(ROOT, "include"), (".h",)):
        assert not pat.search(open(path).read())


def test_oracle_never_imports_the_product():
    for path in _sources(os.path.join(ROOT, "oracle"), (".py",)):
        text = open(path).read()
        assert "paper_2210_03179_gb300" not in text and "chebmg" not in text.lower(), path


def test_beta_tables_agree_between_sides():
    # Both sides transcribe Table 5 independently; compare the text of the two copies.
    from oracle.chebyshev import BETA_TABLE
    src = open(os.path.join(PKG, "csrc", "api.cu")).read()
    block = src[src.index("kBeta[16][16]"):]
    block = block[: block.index("};")]
    rows = re.findall(r"\{([^{}]*)\}", block)
    assert len(rows) == 16
    for k, row in enumerate(rows, start=1):
        vals = [float(v) for v in row.split(",") if v.strip()]
        assert vals == list(BETA_TABLE[k])
