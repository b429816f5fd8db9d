"""The C-ABI library loads without a GPU and exports every entry point that
include/bfc.h declares; host-only calls behave as documented."""
import ctypes
import os
import re

import pytest

import paper_2510_17734_gb300 as bfc
from paper_2510_17734_gb300 import build as bfc_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    bfc_build.build()
    return bfc.load()


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(bfc_\w+)\s*\(", text, flags=re.M)
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("bfc_create", "bfc_eval", "bfc_als_sweep", "bfc_grad", "bfc_complete"):
        assert must in names
    assert sorted(names) == sorted(bfc.exported_symbols)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_num_params_host_only(lib):
    assert bfc.bfc_num_params(256, 4, 16, 4) == 4096
    assert bfc.bfc_num_params(4096, 8, 16, 6) == 196608
    assert bfc.bfc_num_params(65536, 12, 16, 8) == 7340032
    assert bfc.bfc_num_params(100, 2, 16, 4) == -1


def test_create_validates_sizes_before_touching_a_device(lib):
    import numpy as np
    i = np.zeros(4, np.int32)
    t = np.zeros(4, np.complex128)
    bad = [dict(n=100, L=2, b=16, r=4), dict(n=64, L=2, b=16, r=0), dict(n=64, L=2, b=16, r=13)]
    for kw in bad:
        prm = bfc.Params(lam=1e-6, prec=0, **kw)
        with pytest.raises(bfc.BfcError, match="EINVAL"):
            bfc.bfc_create(prm, i, i, t)
    prm = bfc.Params(n=64, L=2, b=16, r=2, lam=-1.0)
    with pytest.raises(bfc.BfcError, match="lambda"):
        bfc.bfc_create(prm, i, i, t)
    assert "lambda" in bfc.bfc_last_error(None)
    prm = bfc.Params(n=64, L=2, b=16, r=2, lam=1e-6, prec=1, gram_impl=3)
    with pytest.raises(bfc.BfcError, match="gram_impl"):
        bfc.bfc_create(prm, i, i, t)
