"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/ctm.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

import paper_2607_15158_gb300 as pkg
from paper_2607_15158_gb300 import build as B

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "include", "ctm.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(pkg.LIB_PATH):
        B.build()
    return ctypes.CDLL(pkg.LIB_PATH)


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ctm_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("ctm_init", "ctm_move", "ctm_converge", "ctm_expect", "ctm_free"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_default_opts_without_gpu(lib):
    o = pkg.ctm_default_opts()
    assert (o.p, o.si_rounds, o.warmup_iters, o.warmup_rounds, o.method, o.prec,
            o.normalize, o.sign_fix) == (5, 1, 5, 8, 0, 0, 1, 1)
    assert o.svd_rel_cutoff == 1e-12
    assert (o.svd_max_sweeps, o.init_mode, o.recycle_sin2, o.min_si_steps) == (80, 0, 0.0, 3)
    assert (o.absorb_tc, o.si_coupled, o.warmup_rsvd, o.svd_presolve, o.fp64_tc) == (0, 0, 0, 1, 1)
    assert o.split_refine == 0.0


def test_bad_options_are_rejected_before_device_work(lib):
    pkg.load()
    A = (ctypes.c_void_p * 1)(ctypes.c_void_p(16))
    for kw in (dict(svd_max_sweeps=0), dict(init_mode=2), dict(recycle_sin2=-1.0),
               dict(min_si_steps=-1), dict(svd_presolve=2), dict(fp64_tc=-1),
               dict(split_refine=-1e-6), dict(split_refine=float("nan"))):
        o = pkg.ctm_default_opts(**kw)
        ptr = ctypes.c_void_p()
        st = pkg._lib.ctm_init(ctypes.byref(ptr), 1, 1, A, None, 0, 2, 2, 4, ctypes.byref(o))
        assert st == pkg.CTM_EINVAL, kw


def test_argument_errors_are_reported_before_device_work(lib):
    pkg.load()
    ptr = ctypes.c_void_p()
    st = pkg._lib.ctm_init(ctypes.byref(ptr), 0, 1, None, None, 0, 2, 2, 4, None)
    assert st == pkg.CTM_EINVAL
    assert b"must be >= 1" in pkg._lib.ctm_last_error(None)


def test_footprint_is_host_arithmetic(lib):
    # no device work: grows with chi and D, split precision adds the slice caches
    f = [pkg.ctm_footprint(1, 1, 2, 3, chi, False) for chi in (9, 18, 27)]
    assert f[0] < f[1] < f[2]
    assert pkg.ctm_footprint(1, 1, 2, 4, 27, False) > f[2]
    split = pkg.ctm_default_opts(prec=pkg.CTM_PREC_SPLIT_BF16)
    assert pkg.ctm_footprint(1, 1, 2, 3, 27, False, split) > f[2]
    n = ctypes.c_size_t(0)
    assert pkg._lib.ctm_footprint(1, 1, 2, 0, 8, 0, None, ctypes.byref(n)) == pkg.CTM_EINVAL
    # cfg3 (3x3, complex D = 6, chi = 144, three lanes) fits several times in the 280 GB
    assert pkg.ctm_footprint(3, 3, 2, 6, 144, True, split) < 60e9
    # the refinement adds its exact-digit operands and the unfused lane pipelines
    refine = pkg.ctm_default_opts(prec=pkg.CTM_PREC_SPLIT_BF16, split_refine=1e-5)
    fr = pkg.ctm_footprint(3, 3, 2, 6, 144, True, refine)
    assert pkg.ctm_footprint(3, 3, 2, 6, 144, True, split) < fr < 120e9


def test_noalloc_rejects_oversize_before_device_work(lib):
    pkg.load()
    fake = ctypes.c_void_p(16)
    st = pkg._lib.ctm_svdvals_noalloc(fake, 257, pkg.CTM_C128, fake, None)
    assert st == pkg.CTM_EINVAL
    assert b"exceeds" in pkg._lib.ctm_noalloc_last_error()
