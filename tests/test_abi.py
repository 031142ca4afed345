"""The C-ABI library loads and exports every function include/hepacc.h
declares; host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

from paper_1906_06242_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def declared_functions():
    names = set()
    for fn in os.listdir(HEADER_DIR):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(HEADER_DIR, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\*?\s*(hepacc_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    path = B.build()
    return ctypes.CDLL(path)


def test_header_declares_the_paper_kernels():
    names = declared_functions()
    for required in ("hepacc_sum_in_offsets", "hepacc_max_in_offsets", "hepacc_get_in_offsets",
                     "hepacc_mask_deltar", "hepacc_fill_histogram", "hepacc_run_chain"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_host_side_errors_without_gpu(lib):
    lib.hepacc_last_error.restype = ctypes.c_char_p
    lib.hepacc_status_string.restype = ctypes.c_char_p
    lib.hepacc_version.restype = ctypes.c_char_p
    assert b"hepacc" in lib.hepacc_version()
    dummy = ctypes.c_void_p(16)
    # negative size
    st = lib.hepacc_sum_in_offsets(dummy, 0, dummy, 6, ctypes.c_int64(-1), None, None, dummy, 0, None)
    assert st == 1 and b"n_rows" in lib.hepacc_last_error()
    # missing output pointer
    st = lib.hepacc_sum_in_offsets(dummy, 0, dummy, 6, ctypes.c_int64(5), None, None, None, 0, None)
    assert st == 1
    # bad offsets dtype
    st = lib.hepacc_sum_in_offsets(dummy, 0, dummy, 0, ctypes.c_int64(5), None, None, dummy, 0, None)
    assert st == 2 and lib.hepacc_status_string(st) == b"HEPACC_ERR_DTYPE"
    # empty input is a no-op
    assert lib.hepacc_sum_in_offsets(None, 0, None, 6, ctypes.c_int64(0), None, None, None, 0, None) == 0
    # nbins out of range
    st = lib.hepacc_fill_histogram(dummy, 0, None, None, ctypes.c_int64(4), dummy, 0, dummy, None, None, None)
    assert st == 1
    # chain: null config
    assert lib.hepacc_run_chain(None, None, None, None) == 1


def test_plan_host_side_errors_without_gpu(lib):
    from paper_1906_06242_gb300 import hepacc as H
    from paper_1906_06242_gb300 import synth
    C = H.ChainConfig(synth.CUTS, synth.HIST_SPECS, [1.0])
    cfg = C.c_struct()

    def batch(offsets=H.I64, kin=H.F32, btag=H.F32):
        b = H.EventBatchC()
        b.n_events = 10
        b.offsets_type, b.kin_type, b.btag_type = offsets, kin, btag
        for f in H.COLUMNS + ("jet_offsets", "mu_offsets", "el_offsets", "weight"):
            setattr(b, f, 16)
        return b

    out = H.ChainOutputsC()
    out.counts = out.sumw = 16
    plan = ctypes.c_void_p()

    def create(b, o, flags=0, n=1, p=ctypes.byref(plan)):
        return lib.hepacc_plan_create(ctypes.byref(cfg), n, ctypes.byref(b), ctypes.byref(o), flags, None, p)

    assert create(batch(), out, p=None) == 1                 # no plan pointer
    assert create(batch(), out, n=0) == 1                    # no samples
    assert create(batch(), out, flags=1 << 10) == 1          # unknown flag
    per_event = H.ChainOutputsC()
    per_event.counts = per_event.sumw = per_event.ev_pass = 16
    assert create(batch(), per_event) == 1                   # plans write no per-event outputs
    assert create(batch(offsets=H.I32), out) == 2            # int64 offsets only
    assert create(batch(kin=H.BF16, btag=H.F32), out) == 2   # half kinematics take half btag
    no_counts = H.ChainOutputsC()
    assert create(batch(), no_counts) == 1
    assert plan.value is None
    lib.hepacc_plan_destroy(None)


def test_histogram_nd_host_side_errors_without_gpu(lib):
    lib.hepacc_last_error.restype = ctypes.c_char_p
    dummy = 16

    def call(ndim, types, nbins, n=10, counts=dummy):
        k = max(1, len(types))
        data = (ctypes.c_void_p * k)(*([dummy] * k))
        edges = (ctypes.c_void_p * k)(*([dummy] * k))
        tt = (ctypes.c_int * k)(*(types or [0]))
        nb = (ctypes.c_int32 * k)(*(nbins or [1]))
        return lib.hepacc_fill_histogram_nd(ctypes.c_int32(ndim), data, tt, edges, nb, None, None,
                                            ctypes.c_int64(n), ctypes.c_void_p(counts), None, None, None)

    assert call(0, [0], [4]) == 1                          # no axis
    assert call(5, [0] * 5, [4] * 5) == 1                  # more than HEPACC_MAX_HIST_DIMS
    assert call(2, [0, 6], [4, 4]) == 2                    # int64 data is not a histogram axis
    assert call(2, [0, 0], [4, 0]) == 1                    # an axis without bins
    assert call(2, [0, 0], [4095, 4095]) == 1 and b"2^24" in lib.hepacc_last_error()   # 4097^2 cells
    assert call(2, [0, 0], [4, 4], n=-1) == 1
    assert call(2, [0, 0], [4, 4], counts=None) == 1       # counts required
    assert call(2, [0, 0], [4, 4], n=0, counts=None) == 0  # empty input is a no-op
