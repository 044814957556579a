"""The C-ABI library loads on a CPU-only host and exports every declared symbol;
argument errors are reported before any CUDA work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2605_14103_gb300 import build as B
from paper_2605_14103_gb300 import feeders as F
from paper_2605_14103_gb300 import zbus

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return zbus.lib()


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(zbus_\w+)\s*\(", txt))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("zbus_network_create", "zbus_solve", "zbus_network_destroy",
                 "zbus_status_string"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    for code, name in zbus.STATUS.items():
        assert zbus.zbus_status_string(code) == name


def test_opts_default(lib):
    o = zbus.zbus_solve_opts_default()
    assert o.precision == 0 and o.conv_rule == 0
    assert o.mismatch_tol == 1e-6 and o.max_correction == 8


def _create(lib, n_total, row, col, val, slack, vs):
    h = C.c_void_p()
    row = np.ascontiguousarray(row, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.complex128)
    slack = np.ascontiguousarray(slack, dtype=np.int32)
    vs = np.ascontiguousarray(vs, dtype=np.complex128)
    st = lib.zbus_network_create(n_total, row.size, row.ctypes.data, col.ctypes.data,
                                 val.ctypes.data, slack.ctypes.data, vs.ctypes.data, None,
                                 C.byref(h))
    return st, h.value


def test_create_rejects_bad_arguments(lib):
    vs = np.ones(3, dtype=np.complex128)
    ok_row, ok_col, ok_val = [0, 1, 2, 3], [0, 1, 2, 3], [1, 1, 1, 1]
    cases = [
        (3, ok_row, ok_col, ok_val, [0, 1, 2]),            # too small
        (4, [0, 9], [0, 0], [1, 1], [0, 1, 2]),            # row out of range
        (4, ok_row, ok_col, ok_val, [0, 1, 1]),            # repeated slack
        (4, ok_row, ok_col, ok_val, [0, 1, 7]),            # slack out of range
        (4, [0], [0], [np.nan], [0, 1, 2]),                # non-finite value
    ]
    for n_total, r, c, v, s in cases:
        st, h = _create(lib, n_total, r, c, v, s, vs)
        assert st == 1, (n_total, r, s, zbus.zbus_last_error())
        assert not h
        assert zbus.zbus_last_error()


def test_solve_rejects_null_network(lib):
    st = lib.zbus_solve(None, 4, None, None, None, 1e-8, 50, None, None, None, None, None)
    assert st == 1
    assert "NULL" in zbus.zbus_last_error()
    assert lib.zbus_network_size(None) == -1
    lib.zbus_network_destroy(None)   # ignored


def test_create_phased_rejects_bad_maps(lib):
    f = F.make_partial_feeder(12, 5, lateral_frac=1.0)
    row = np.ascontiguousarray(f.Y_row, np.int32)
    col = np.ascontiguousarray(f.Y_col, np.int32)
    val = np.ascontiguousarray(f.Y_val, np.complex128)
    sl = np.array([0, 1, 2], np.int32)
    vs = np.ascontiguousarray(f.v_slack)
    out = C.c_void_p()

    def call(bp):
        bp = np.ascontiguousarray(bp, np.int32)
        return lib.zbus_network_create_phased(f.n_total, row.size, row.ctypes.data,
                                              col.ctypes.data, val.ctypes.data, sl.ctypes.data,
                                              vs.ctypes.data, bp.ctypes.data, None,
                                              C.byref(out))

    bp = f.bus_phase.copy()
    dup = bp.copy()
    dup[5] = dup[4]                         # two indices on one bus-phase
    assert call(dup) == 1
    swapped = bp.copy()
    swapped[[0, 1]] = swapped[[1, 0]]       # slack phases out of order
    assert call(swapped) == 1
    onslack = bp.copy()
    onslack[4] = 0                          # a load phase on the slack bus (duplicate too)
    assert call(onslack) == 1
    neg = bp.copy()
    neg[7] = -3
    assert call(neg) == 1
    assert lib.zbus_network_create_phased(f.n_total, row.size, row.ctypes.data, col.ctypes.data,
                                          val.ctypes.data, sl.ctypes.data, vs.ctypes.data,
                                          None, None, C.byref(out)) == 1
    assert not out.value


def test_tune_variants_and_override_without_a_gpu(lib):
    """The contraction variants are listed and an override is checked on the
    host: a pair that is not compiled, or a precision without tensor-core
    tiles, is refused; BN = 0 clears an entry."""
    fp16 = zbus.zbus_tune_variants("fp16_scaled")
    bf16 = zbus.zbus_tune_variants("bf16x2")
    assert fp16 and bf16 and zbus.zbus_tune_variants("fp64") == []
    assert all(bn in (64, 128, 256) and st >= 2 for bn, st in fp16 + bf16)
    assert lib.zbus_tune_variants(2, None, None, -1) == -1
    bn, st = fp16[0]
    zbus.zbus_tune_set("fp16_scaled", 381, 4096, bn, st)
    zbus.zbus_tune_set("fp16_scaled", 381, 4096, 0, 0)
    for args in (("fp16_scaled", 381, 4096, 96, 4), ("fp64", 381, 4096, bn, st),
                 ("tree", 381, 4096, bn, st), ("fp16_scaled", 0, 4096, bn, st),
                 ("fp16_scaled", 381, 0, bn, st)):
        with pytest.raises(zbus.ZbusError) as ei:
            zbus.zbus_tune_set(*args)
        assert ei.value.status == 1


def test_new_entry_points_refuse_bad_arguments_without_a_gpu(lib):
    """Argument checks that run before any CUDA work: the FP64 probe with no
    output, the serving footprint of a NULL network or a non-serving
    precision, the wait limit outside the checked build, and the
    allocation-free solve of a NULL network."""
    assert lib.zbus_probe_fp64_rate(None, None, None) == 1
    a = C.c_uint64(0)
    assert lib.zbus_serve_footprint(None, 2, C.byref(a), None, None) == 1
    assert lib.zbus_checked_set_wait(0) == 7                 # normal build: unsupported
    assert lib.zbus_solve_noalloc(None, 4, None, None, None, 1e-8, 50, 0, None, None, None,
                                  None) == 1
    o = zbus.zbus_solve_opts_default()
    assert o.max_correction == 8                            # FP64 correction sweeps by default

