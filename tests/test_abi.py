"""The C-ABI library builds for sm_103a, loads, exports every symbol include/ks.h
declares, and rejects bad parameters on the host (no GPU needed for these)."""
import ctypes
import os
import re

import pytest

from paper_2603_16692_gb300 import build, ks
from paper_2603_16692_gb300 import workload as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "ks.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ks_[a-z_]+)\s*\(", src)))


def test_library_builds_and_exports_header_symbols():
    so = build.build()
    assert os.path.exists(so)
    lib = ctypes.CDLL(so)
    names = header_functions()
    assert "ks_switch" in names and "ks_keygen" in names and "ks_switch_batch" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(ks.SYMBOLS) | set(names)
    assert set(ks.SYMBOLS) <= set(names)


def test_strerror_names_every_code():
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert ks.strerror(code) and ks.strerror(code) != "unknown error"
    assert ks.strerror(-99) == "unknown error"


def _create(dnum, logn, L, q, p):
    try:
        h = ks.ks_context_create(dnum, logn, L, q, p)
    except ks.KSError as e:
        return e.code
    ks.ks_context_destroy(h)
    return 0


def test_context_rejects_bad_parameters_on_host():
    prm = W.make_params(2, 5, 3)
    q, p = list(prm.q), list(prm.p)
    assert _create(2, 5, 3, q[:-1], p) == ks.KS_EINVAL          # nq != L+1
    assert _create(2, 5, 3, q, p + p[:1]) == ks.KS_EINVAL        # np != alpha
    assert _create(0, 5, 3, q, p) == ks.KS_EINVAL                # dnum 0
    assert _create(2, 18, 3, q, p) == ks.KS_EINVAL               # N > 2^17
    assert _create(2, 5, 3, q[:-1] + [q[0] + 64 * 2], p) in (ks.KS_EPRIME,)  # not prime/dup
    bad = list(q)
    bad[1] = q[0]                                                # repeated prime
    assert _create(2, 5, 3, bad, p) == ks.KS_EPRIME
    bad = list(q)
    bad[2] = 1000003                                             # prime, 3 mod 64
    assert _create(2, 5, 3, bad, p) == ks.KS_EPRIME
    bad = list(q)
    bad[0] = (1 << 62) + 1                                       # too large
    assert _create(2, 5, 3, bad, p) == ks.KS_EPRIME
    bad = list(q)
    bad[3] = 7 * 64 * 64 + 1                                     # 1 mod 64 but composite
    assert _create(2, 5, 3, bad, p) == ks.KS_EPRIME


def test_switch_rejects_null_context():
    lib = ks.load()
    assert lib.ks_switch(None, None, None, None, 0, 0, None, 0, None) == ks.KS_EINVAL
    assert lib.ks_keygen(None, None, None, None, None, None, None) == ks.KS_EINVAL
    assert lib.ks_switch_batch(None, -1, 0, None) == ks.KS_EINVAL


def test_new_entry_points_reject_bad_arguments_on_host():
    """Argument checks that run before any CUDA call."""
    lib = ks.load()
    d = ctypes.c_double()
    assert lib.ks_calibrate(0, 16, ctypes.byref(d), None) == ks.KS_EINVAL
    assert lib.ks_calibrate(ks.KS_CAL_MAC, 0, ctypes.byref(d), None) == ks.KS_EINVAL
    assert lib.ks_calibrate(ks.KS_CAL_BUTTERFLY, 16, None, None) == ks.KS_EINVAL
    assert lib.ks_selector_load(None) == ks.KS_EINVAL
    assert lib.ks_select(None, None, None, None) == ks.KS_EINVAL
    assert lib.ks_switch_host_async(None, None, None, None, 0, 0, None) == ks.KS_EINVAL
    assert lib.ks_switch_host_async_ws(None, None, None, None, 0, 0, None, 0, None) == \
        ks.KS_EINVAL
    n = ctypes.c_size_t()
    assert lib.ks_host_workspace_size(None, 0, 0, ctypes.byref(n)) == ks.KS_EINVAL
    sel = ks.ks_selector()
    for k in range(6):
        sel.x_std[k] = 1.0
    for k in range(4):
        sel.t_std[k] = 1.0
        sel.variant[k] = ks.KS_DPOB
    sel.x_std[2] = 0.0  # a zero standard deviation is refused before anything is copied
    assert lib.ks_selector_load(ctypes.byref(sel)) == ks.KS_EINVAL
    sel.x_std[2] = 1.0
    sel.variant[1] = 7  # not a dataflow
    assert lib.ks_selector_load(ctypes.byref(sel)) == ks.KS_EINVAL


def test_plan_flags_match_the_header():
    """Every plan flag of the binding has the value include/ks.h gives it, and the plan
    names spell the tensor-core flags."""
    text = open(os.path.join(ROOT, "include", "ks.h")).read()
    defs = dict(re.findall(r"#define (KS_\w+) (0x[0-9a-fA-F]+|\d+)\b", text))
    for name in ("KS_UNFUSED", "KS_RADIX4", "KS_RADIX16", "KS_BCONV_TC", "KS_BCONV_TC_DOWN",
                 "KS_SPLIT_DOWN", "KS_COLALT_INV", "KS_COLALT_UPC", "KS_COLALT_DNC"):
        assert getattr(ks, name) == int(defs[name], 0), name
    assert ks.variant_name(ks.KS_DPOB | ks.KS_BCONV_TC_DOWN) == "DPOB-tcdown"
    assert ks.variant_name(ks.KS_DPOB | ks.KS_BCONV_TC_DOWN | ks.KS_BCONV_TC) == "DPOB-tc"
