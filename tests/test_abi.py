"""The C-ABI library builds, loads and exports every function include/gsr.h
declares (no GPU needed: nothing here launches a kernel)."""
import os
import re

from paper_2212_11675_gb300 import _lib

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")


def declared():
    names = set()
    for f in os.listdir(HDR):
        if f.endswith(".h"):
            txt = open(os.path.join(HDR, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(gsr_\w+)\s*\(", txt))
    return names


def test_header_declares_the_boundary():
    names = declared()
    for must in ("gsr_create", "gsr_destroy", "gsr_aprod1", "gsr_aprod2", "gsr_lsqr_solve",
                 "gsr_precondition", "gsr_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol():
    L = _lib.lib()
    missing = [n for n in sorted(declared()) if not hasattr(L, n)]
    assert not missing, missing
    assert set(_lib.EXPORTS) <= declared()


def test_strerror_and_null_handling_without_gpu():
    L = _lib.lib()
    assert L.gsr_strerror(_lib.GSR_ERR_INDEX) == b"matrix structure out of range"
    assert L.gsr_strerror(12345) == b"unknown error"
    # argument checks happen before any CUDA call
    assert L.gsr_aprod1(None, None, None, None) == _lib.GSR_ERR_ARG
    assert L.gsr_lsqr_solve(None, None, 1, 0.0, 0.0, None, None, None, None) == _lib.GSR_ERR_ARG
    assert L.gsr_destroy(None) == _lib.GSR_OK


def test_create_checks_the_product_form_before_any_cuda_call():
    import ctypes

    import numpy as np
    L = _lib.lib()
    sp = np.array([0, 1], dtype=np.uint32)
    att = np.zeros(1, dtype=np.uint32)
    ins = np.arange(6, dtype=np.uint16)
    val = np.ones(24)
    h = ctypes.c_void_p()

    def create(n_instr, products):
        d = _lib.Dims(1, 8, n_instr, 1)
        cfg = _lib.Config()
        L.gsr_config_default(ctypes.byref(cfg))
        assert cfg.products == _lib.GSR_PRODUCTS_AUTO
        cfg.products = products
        return L.gsr_create(ctypes.byref(h), ctypes.byref(d), sp.ctypes.data, att.ctypes.data,
                            ins.ctypes.data, val.ctypes.data, ctypes.byref(cfg))

    assert create(60, 7) == _lib.GSR_ERR_ARG
    assert create(60, -1) == _lib.GSR_ERR_ARG
    # the attitude split forms exclude each other and have no kernel with the
    # split star units, nor (axes 1 and 2) with the split instrument units
    M = _lib.GSR_PRODUCTS_MASK
    assert create(60, M | _lib.GSR_SPLIT_APROD2_ATT | _lib.GSR_SPLIT_APROD2_ATT2) == _lib.GSR_ERR_ARG
    assert (create(60, M | _lib.GSR_SPLIT_APROD2_ATT | _lib.GSR_SPLIT_APROD2_STARS)
            == _lib.GSR_ERR_UNSUPPORTED)
    assert (create(60, M | _lib.GSR_SPLIT_APROD2_ATT2 | _lib.GSR_SPLIT_APROD2_INSTR)
            == _lib.GSR_ERR_UNSUPPORTED)
    # the astrometric split extends aprod 1's split form
    assert create(60, M | _lib.GSR_SPLIT_APROD1_ASTRO) == _lib.GSR_ERR_ARG
    assert create(60, M | 64) == _lib.GSR_ERR_ARG
    # split products keep x in shared memory: at most 3072 instruments
    assert create(4000, _lib.GSR_PRODUCTS_SPLIT) == _lib.GSR_ERR_UNSUPPORTED
    assert not h.value
