"""The C ABI: the built library exports every entry point include/gfcc.h declares (CPU only, no compute)."""
import ctypes
import os
import re

import pytest

from paper_2010_04768_gb300 import build as gbuild
from paper_2010_04768_gb300 import gfcc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "gfcc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gfcc_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(gfcc.LIB_PATH):
        gbuild.build()
    return ctypes.CDLL(gfcc.LIB_PATH)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gfcc_create", "gfcc_solve", "gfcc_destroy", "gfcc_set_option", "gfcc_last_stats"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_last_error_is_empty_string_initially(lib):
    lib.gfcc_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.gfcc_last_error(), bytes)


def test_null_arguments_are_rejected_without_a_gpu(lib):
    # argument checks happen before any CUDA call
    typed = gfcc.load()
    h = ctypes.c_void_p()
    assert typed.gfcc_create(0, 4, 4, None, None, None, None, None, ctypes.byref(h)) == gfcc.ERR_ARG
    assert b"o >= 1" in typed.gfcc_last_error()
    assert typed.gfcc_set_option(None, 1, 1.0) == gfcc.ERR_ARG
    assert typed.gfcc_residual_stats(None, None, None, None) == gfcc.ERR_ARG
    cnt = ctypes.c_int(0)
    assert typed.gfcc_refine_stats(None, ctypes.byref(cnt), None) == gfcc.ERR_ARG
    typed.gfcc_destroy(None)


def test_guess_model_arguments_are_rejected_without_a_gpu(lib):
    typed = gfcc.load()
    h = ctypes.c_void_p()
    assert typed.gfcc_mlp_create(256, gfcc.MLP_FP32, None, ctypes.byref(h)) == gfcc.ERR_ARG
    assert typed.gfcc_mlp_create(0, gfcc.MLP_FP32, None, ctypes.byref(h)) == gfcc.ERR_ARG
    loss = ctypes.c_double()
    assert typed.gfcc_mlp_train(None, 10, 32, 1e-3, 0, ctypes.byref(loss)) == gfcc.ERR_ARG
    assert typed.gfcc_mlp_collect(None, None, 1, 0, None) == gfcc.ERR_ARG
    assert typed.gfcc_set_guess_model(None, None) == gfcc.ERR_ARG
    assert typed.gfcc_mlp_num_params(None) == 0
    typed.gfcc_mlp_destroy(None)


def test_process_options_and_block_solve_arguments_without_a_gpu(lib):
    # process-wide options are host state; bad keys, values and NULL contexts are rejected before any
    # CUDA call
    typed = gfcc.load()
    assert typed.gfcc_set_process_option(999, 1.0) == gfcc.ERR_ARG
    assert typed.gfcc_set_process_option(gfcc.OPT_WAIT_NS, 0.0) == gfcc.ERR_ARG
    assert typed.gfcc_set_process_option(gfcc.OPT_TEST_NO_LOADS, 2.0) == gfcc.ERR_ARG
    assert typed.gfcc_set_process_option(gfcc.OPT_SETUP_EMULATE_FLOPS, -1.0) == gfcc.ERR_ARG
    assert typed.gfcc_set_process_option(gfcc.OPT_WAIT_NS, 1e9) == gfcc.OK
    assert typed.gfcc_set_process_option(gfcc.OPT_TEST_NO_LOADS, 0.0) == gfcc.OK
    assert typed.gfcc_set_process_option(gfcc.OPT_SETUP_EMULATE_FLOPS, 4e12) == gfcc.OK
    om = (ctypes.c_double * 1)(0.1)
    orb = (ctypes.c_int * 1)(0)
    G = (ctypes.c_double * 2)()
    assert typed.gfcc_solve_block(None, 1, om, 0.01, 1, orb, 1, orb, 1e-8, G) == gfcc.ERR_ARG


def test_ccsd_arguments_are_rejected_without_a_gpu(lib):
    # sizes, NULL inputs, tol, max_iter and unknown flags are checked before any CUDA call
    typed = gfcc.load()
    f = (ctypes.c_double * 4)()
    ch = (ctypes.c_double * 4)()
    t1 = (ctypes.c_double * 1)()
    t2 = (ctypes.c_double * 1)()
    assert typed.gfcc_ccsd(0, 1, 1, f, ch, 1e-8, 10, 0, t1, t2, None, None) == gfcc.ERR_ARG
    assert typed.gfcc_ccsd(1, 1, 1, None, ch, 1e-8, 10, 0, t1, t2, None, None) == gfcc.ERR_ARG
    assert typed.gfcc_ccsd(1, 1, 1, f, ch, 0.0, 10, 0, t1, t2, None, None) == gfcc.ERR_ARG
    assert typed.gfcc_ccsd(1, 1, 1, f, ch, 1e-8, 0, 0, t1, t2, None, None) == gfcc.ERR_ARG
    assert typed.gfcc_ccsd(1, 1, 1, f, ch, 1e-8, 10, 4, t1, t2, None, None) == gfcc.ERR_ARG
    assert typed.gfcc_ccsd(1, 1, 1, f, ch, 1e-8, 10, 0, None, t2, None, None) == gfcc.ERR_ARG


def test_closed_shell_create_arguments_are_rejected_without_a_gpu(lib):
    typed = gfcc.load()
    h = ctypes.c_void_p()
    f = (ctypes.c_double * 4)()
    assert typed.gfcc_create_rhf(0, 1, 1, f, f, f, f, None, ctypes.byref(h)) == gfcc.ERR_ARG
    assert typed.gfcc_create_rhf(1, 1, 1, None, f, f, f, None, ctypes.byref(h)) == gfcc.ERR_ARG
    assert typed.gfcc_create_rhf(1, 1, 1, f, f, f, f, None, None) == gfcc.ERR_ARG


def test_checkpoint_arguments_are_rejected_without_a_gpu(lib, tmp_path):
    typed = gfcc.load()
    om = (ctypes.c_double * 1)(0.1)
    orb = (ctypes.c_int * 1)(0)
    G = (ctypes.c_double * 2)()
    path = str(tmp_path / "ck.bin").encode()
    assert typed.gfcc_solve_checkpoint(None, 1, om, 0.01, 1, orb, 1e-8, path, None, G) == gfcc.ERR_ARG
    assert not (tmp_path / "ck.bin").exists()
