"""Python front of the CPU oracle (``hepacc_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
CPU-baseline leg of the benchmark. The GPU library never imports it, and it
imports nothing from the GPU library; it takes plain numpy arrays (the seeded
inputs) and returns numpy arrays.

Histogram edges and jet-pt scales are derived here, independently of the GPU
binding, from the plain parameters (low, high, bins) and shifts k:
edge_b = float32(low + (high - low) * b / bins) evaluated in binary64, and
scale_k = float32(1 + 0.01 k).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hepacc_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libhepacc_oracle.so")

F32, F16, BF16, I8, U8, I32, I64 = 0, 1, 2, 3, 4, 5, 6
_NP_CODE = {np.dtype(np.float32): F32, np.dtype(np.int8): I8, np.dtype(np.uint8): U8,
            np.dtype(np.int32): I32, np.dtype(np.int64): I64}
N_VARS = 20


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-Wall",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def use_library(path):
    """Point this module at another build of the oracle source (the mutation
    tests load deliberately broken copies); ``None`` restores the default."""
    global _lib
    _lib = None if path is None else _setup(ctypes.CDLL(path))


def _setup(handle):
    handle.oracle_dr2.restype = ctypes.c_float
    handle.oracle_dr2.argtypes = [ctypes.c_float] * 4
    handle.oracle_mass2.restype = ctypes.c_double
    handle.oracle_mass2.argtypes = [ctypes.c_double] * 8
    handle.oracle_bin_of.restype = ctypes.c_int
    handle.oracle_bin_of.argtypes = [ctypes.c_double, ctypes.c_void_p, ctypes.c_int]
    return handle


def compile_source(src_path, out_path):
    """Compile an oracle source file with the same flags as ``build``."""
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", out_path, src_path, "-lm"]
    subprocess.check_call(cmd)
    return out_path


def lib():
    global _lib
    if _lib is None:
        _lib = _setup(ctypes.CDLL(build()))
    return _lib




# ----------------------------------------------------------------------------
# marshalling helpers
# ----------------------------------------------------------------------------

def _p(a):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"], "oracle inputs must be contiguous"
    # the returned pointer keeps the array alive (masks converted on the fly
    # are temporaries)
    return a.ctypes.data_as(ctypes.c_void_p)


def _code(a, fmt=None):
    """dtype code of a column: float32/int arrays by dtype; uint16 arrays are
    half bit patterns and need ``fmt`` ('bf16' or 'f16')."""
    if a.dtype == np.uint16:
        if fmt == "bf16":
            return BF16
        if fmt == "f16":
            return F16
        raise ValueError("uint16 column needs fmt='bf16' or 'f16'")
    return _NP_CODE[a.dtype]


def _i64(x):
    return ctypes.c_int64(int(x))


def _u8(m):
    if m is None:
        return None
    return np.ascontiguousarray(m, dtype=np.uint8)


# ----------------------------------------------------------------------------
# generic kernels
# ----------------------------------------------------------------------------

def sum_in_offsets(x, offsets, mask_rows=None, mask_content=None, out=None, fmt=None):
    """Listing 1 semantics (+= into ``out``); float content -> float32 out,
    integer content -> int64 out."""
    n = len(offsets) - 1
    mask_rows, mask_content = _u8(mask_rows), _u8(mask_content)
    integer = x.dtype in (np.int8, np.uint8, np.int32, np.int64)
    if out is None:
        out = np.zeros(n, dtype=np.int64 if integer else np.float32)
    f = lib().oracle_sum_in_offsets_i if integer else lib().oracle_sum_in_offsets_f
    f(_p(x), _code(x, fmt), _p(offsets), _code(offsets), _i64(n), _p(mask_rows), _p(mask_content), _p(out))
    return out


def minmax_in_offsets(x, offsets, want_max=True, mask_rows=None, mask_content=None,
                      empty=-np.inf, out=None, arg=None, fmt=None):
    n = len(offsets) - 1
    mask_rows, mask_content = _u8(mask_rows), _u8(mask_content)
    if out is None:
        out = np.full(n, np.nan, dtype=np.float32)
    if arg is None:
        arg = np.full(n, -7, dtype=np.int32)
    lib().oracle_minmax_in_offsets(_p(x), _code(x, fmt), _p(offsets), _code(offsets), _i64(n),
                                   _p(mask_rows), _p(mask_content), ctypes.c_int(int(want_max)),
                                   ctypes.c_float(empty), _p(out), _p(arg))
    return out, arg


def get_in_offsets(x, offsets, nth=0, mask_rows=None, mask_content=None, default=np.nan,
                   out=None, idx=None, fmt=None):
    n = len(offsets) - 1
    mask_rows, mask_content = _u8(mask_rows), _u8(mask_content)
    nth_arr = None
    nth_scalar = 0
    if np.ndim(nth) == 0:
        nth_scalar = int(nth)
    else:
        nth_arr = np.ascontiguousarray(nth, dtype=np.int32)
    if out is None:
        out = np.full(n, np.nan, dtype=np.float32)
    if idx is None:
        idx = np.full(n, -7, dtype=np.int32)
    lib().oracle_get_in_offsets(_p(x), _code(x, fmt), _p(offsets), _code(offsets), _i64(n),
                                _p(nth_arr), ctypes.c_int32(nth_scalar), _p(mask_rows),
                                _p(mask_content), ctypes.c_float(default), _p(out), _p(idx))
    return out, idx


def set_in_offsets(x, offsets, nth=0, value=0, mask_rows=None, mask_content=None):
    """In place on a uint8 or float32 array ``x``."""
    n = len(offsets) - 1
    mask_rows, mask_content = _u8(mask_rows), _u8(mask_content)
    nth_arr = None
    nth_scalar = 0
    if np.ndim(nth) == 0:
        nth_scalar = int(nth)
    else:
        nth_arr = np.ascontiguousarray(nth, dtype=np.int32)
    assert x.dtype in (np.uint8, np.float32)
    lib().oracle_set_in_offsets(_p(x), _code(x), _p(offsets), _code(offsets), _i64(n), _p(nth_arr),
                                ctypes.c_int32(nth_scalar), _p(mask_rows), _p(mask_content),
                                ctypes.c_double(value))
    return x


def select_range(x, lo=-np.inf, hi=np.inf, scale=1.0, use_abs=False, mask_in=None, fmt=None):
    m = len(x)
    out = np.zeros(m, dtype=np.uint8)
    lib().oracle_select_range(_p(x), _code(x, fmt), _i64(m), ctypes.c_float(scale), ctypes.c_float(lo),
                              ctypes.c_float(hi), ctypes.c_int(int(use_abs)), _p(_u8(mask_in)), _p(out))
    return out


def scale(x, s, fmt=None):
    out = np.zeros(len(x), dtype=np.float32)
    lib().oracle_scale(_p(x), _code(x, fmt), _i64(len(x)), ctypes.c_float(s), _p(out))
    return out


def dr2(eta1, phi1, eta2, phi2):
    return lib().oracle_dr2(eta1, phi1, eta2, phi2)


def mask_deltar(eta1, phi1, off1, eta2, phi2, off2, mask_rows=None, mask1_in=None, mask2=None,
                dr2_cut=0.16, out=None, fmt1=None, fmt2=None):
    n = len(off1) - 1
    assert len(off2) == n + 1 and off1.dtype == off2.dtype
    if out is None:
        out = np.full(len(eta1), 7, dtype=np.uint8)
    lib().oracle_mask_deltar(_p(eta1), _p(phi1), _code(eta1, fmt1), _p(off1), _p(eta2), _p(phi2),
                             _code(eta2, fmt2), _p(off2), _code(off1), _i64(n), _p(_u8(mask_rows)),
                             _p(_u8(mask1_in)), _p(_u8(mask2)), ctypes.c_float(dr2_cut), _p(out))
    return out


def hist_edges(lo, hi, nbins):
    """float32 edges float32(lo + (hi - lo) * b / nbins), b = 0..nbins."""
    return np.array([np.float32(lo + (hi - lo) * b / nbins) for b in range(nbins + 1)],
                    dtype=np.float32)


def bin_of(v, edges):
    edges = np.ascontiguousarray(edges, dtype=np.float32)
    return lib().oracle_bin_of(float(v), _p(edges), len(edges) - 1)


def fill_histogram(x, edges, weights=None, mask=None, counts=None, sumw=None, sumw2=None, fmt=None):
    edges = np.ascontiguousarray(edges, dtype=np.float32)
    nb = len(edges) - 1
    if counts is None:
        counts = np.zeros(nb + 2, dtype=np.uint64)
    if sumw is None:
        sumw = np.zeros(nb + 2, dtype=np.float64)
    if sumw2 is None:
        sumw2 = np.zeros(nb + 2, dtype=np.float64)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float32)
    lib().oracle_fill_histogram(_p(x), _code(x, fmt), _p(w), _p(_u8(mask)), _i64(len(x)), _p(edges),
                                ctypes.c_int(nb), _p(counts), _p(sumw), _p(sumw2))
    return counts, sumw, sumw2


def fill_histogram_nd(xs, edges, weights=None, mask=None, fmts=None):
    """Histogram over len(xs) variables; returns counts, sumw, sumw2 shaped
    (nbins_0 + 2, nbins_1 + 2, ...), axis 0 slowest in memory."""
    k = len(xs)
    fmts = fmts or [None] * k
    edges = [np.ascontiguousarray(e, dtype=np.float32) for e in edges]
    nbs = [len(e) - 1 for e in edges]
    shape = tuple(nb + 2 for nb in nbs)
    counts = np.zeros(shape, dtype=np.uint64)
    sumw = np.zeros(shape, dtype=np.float64)
    sumw2 = np.zeros(shape, dtype=np.float64)
    xs = [np.ascontiguousarray(x) for x in xs]
    xp = (ctypes.c_void_p * k)(*[x.ctypes.data for x in xs])
    xt = (ctypes.c_int * k)(*[_code(x, f) for x, f in zip(xs, fmts)])
    ep = (ctypes.c_void_p * k)(*[e.ctypes.data for e in edges])
    nb = (ctypes.c_int * k)(*nbs)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float32)
    n = len(xs[0])
    assert all(len(x) == n for x in xs)
    lib().oracle_fill_histogram_nd(ctypes.c_int(k), xp, xt, ep, nb, _p(w), _p(_u8(mask)), _i64(n), _p(counts),
                                   _p(sumw), _p(sumw2))
    return counts, sumw, sumw2


def pair_mass(pt, eta, phi, mass, offsets, ia, ib, mask_rows=None, fmt=None):
    n = len(offsets) - 1
    out = np.full(n, np.nan, dtype=np.float64)
    ia = np.ascontiguousarray(ia, dtype=np.int32)
    ib = np.ascontiguousarray(ib, dtype=np.int32)
    lib().oracle_pair_mass(_p(pt), _p(eta), _p(phi), _p(mass), _code(pt, fmt), _p(offsets),
                           _code(offsets), _i64(n), _p(ia), _p(ib), _p(_u8(mask_rows)), _p(out))
    return out


def mass2(pt1, eta1, phi1, m1, pt2, eta2, phi2, m2):
    return lib().oracle_mass2(pt1, eta1, phi1, m1, pt2, eta2, phi2, m2)


def max_pt_trijet(pt, eta, phi, mass, offsets, mask_rows=None, mask_content=None, fmt=None):
    n = len(offsets) - 1
    m = np.full(n, np.nan)
    ptj = np.full(n, np.nan)
    idx = np.full((n, 3), -7, dtype=np.int32)
    gap = np.full(n, np.nan)
    lib().oracle_max_pt_trijet(_p(pt), _p(eta), _p(phi), _p(mass), _code(pt, fmt), _p(offsets),
                               _code(offsets), _i64(n), _p(_u8(mask_rows)), _p(_u8(mask_content)),
                               _p(m), _p(ptj), _p(idx), _p(gap))
    return m, ptj, idx, gap


# ----------------------------------------------------------------------------
# the analysis chain
# ----------------------------------------------------------------------------

class _Batch(ctypes.Structure):
    _fields_ = [("n_events", ctypes.c_int64), ("offset_type", ctypes.c_int),
                ("jet_off", ctypes.c_void_p), ("mu_off", ctypes.c_void_p), ("el_off", ctypes.c_void_p),
                ("kin_type", ctypes.c_int), ("btag_type", ctypes.c_int),
                ("jet_pt", ctypes.c_void_p), ("jet_eta", ctypes.c_void_p), ("jet_phi", ctypes.c_void_p),
                ("jet_mass", ctypes.c_void_p), ("jet_btag", ctypes.c_void_p),
                ("mu_pt", ctypes.c_void_p), ("mu_eta", ctypes.c_void_p), ("mu_phi", ctypes.c_void_p),
                ("mu_iso", ctypes.c_void_p), ("mu_tight", ctypes.c_void_p),
                ("el_pt", ctypes.c_void_p), ("el_eta", ctypes.c_void_p), ("el_phi", ctypes.c_void_p),
                ("el_iso", ctypes.c_void_p), ("el_tight", ctypes.c_void_p),
                ("weight", ctypes.c_void_p)]


class _Config(ctypes.Structure):
    _fields_ = [("lep_pt_min", ctypes.c_float), ("lep_abseta_max", ctypes.c_float),
                ("lep_iso_max", ctypes.c_float), ("jet_pt_min", ctypes.c_float),
                ("jet_abseta_max", ctypes.c_float), ("dr2_cut", ctypes.c_float),
                ("btag_min", ctypes.c_float), ("n_var", ctypes.c_int), ("scales", ctypes.c_void_p),
                ("n_hist", ctypes.c_int), ("nbins", ctypes.c_void_p), ("edges", ctypes.c_void_p),
                ("jec_neta", ctypes.c_int), ("jec_npt", ctypes.c_int), ("jec_eta_edges", ctypes.c_void_p),
                ("jec_pt_edges", ctypes.c_void_p), ("jec_contents", ctypes.c_void_p)]


class _Outputs(ctypes.Structure):
    _fields_ = [("counts", ctypes.c_void_p), ("sumw", ctypes.c_void_p), ("sumw2", ctypes.c_void_p),
                ("ev_pass", ctypes.c_void_p), ("ev_nlep", ctypes.c_void_p),
                ("ev_njet", ctypes.c_void_p), ("ev_nb", ctypes.c_void_p), ("ev_idx", ctypes.c_void_p),
                ("ev_vars", ctypes.c_void_p), ("ev_gap", ctypes.c_void_p), ("ev_idx2", ctypes.c_void_p)]


def trijet_closest_mass(pt, eta, phi, mass, offsets, target=172.0, mask_rows=None, mask_content=None, fmt=None):
    """Per event: the triplet of masked-in objects whose FP64 mass is closest
    to ``target`` (Section IV top candidate). Returns (mass, idx3 [N,3],
    gap) with gap = |m_second - target| - |m_best - target|."""
    n = len(offsets) - 1
    m = np.full(n, np.nan)
    idx = np.full((n, 3), -7, dtype=np.int32)
    gap = np.full(n, np.nan)
    L = lib()
    L.oracle_trijet_closest_mass(_p(pt), _p(eta), _p(phi), _p(mass), _code(pt, fmt), _p(offsets), _code(offsets),
                                 _i64(n), _p(_u8(mask_rows)), _p(_u8(mask_content)), ctypes.c_double(target),
                                 _p(m), _p(idx), _p(gap))
    return m, idx, gap


def select_opposite_sign(charge, offsets, mask_rows=None, mask_in=None, out=None):
    """Per event: keep the first two masked-in objects of opposite charge
    (Section III specialised kernel); ``out`` (uint8, content size) is
    written only for events with mask_rows set."""
    n = len(offsets) - 1
    charge = np.ascontiguousarray(charge, dtype=np.int8)
    if out is None:
        out = np.zeros(len(charge), dtype=np.uint8)
    lib().oracle_select_opposite_sign(_p(charge), _p(offsets), _code(offsets), _i64(n), _p(_u8(mask_rows)),
                                      _p(_u8(mask_in)), _p(out))
    return out


def get_bin_contents(x, edges, contents, interpolate=False, fmt=None):
    """Lookup of ``contents`` (nbins+2 float32, under/overflow included) at
    the bins of ``x`` (Section III kernel list), or the binary32 linear
    interpolation between bin centres."""
    edges = np.ascontiguousarray(edges, dtype=np.float32)
    contents = np.ascontiguousarray(contents, dtype=np.float32)
    out = np.empty(len(x), dtype=np.float32)
    lib().oracle_get_bin_contents(_p(x), _code(x, fmt), _i64(len(x)), _p(edges), ctypes.c_int(len(edges) - 1),
                                  _p(contents), ctypes.c_int(1 if interpolate else 0), _p(out))
    return out


def run_chain(batch, cuts, hist_specs, shifts, per_event=True, kin_fmt=None, btag_fmt=None, jec=None):
    """Run the benchmark chain on a seeded batch (the object made by the input
    generator, read through its attributes only). ``shifts`` are the integer k
    of the jet-pt scales 1 + 0.01 k. Returns a dict of numpy arrays:
    counts/sumw/sumw2 [n_var, total_bins]; with ``per_event`` also pass,
    nlep, njet, nb, idx [n_var, 5, N], vars [n_var, 20, N] (float64),
    gap [n_var, N] and idx2 [n_var, 3, N]. ``jec`` (optional): jet-energy
    correction tables, dict of eta_edges, pt_edges and contents
    [n_var][n_eta + 2][n_pt + 2] (float32); the variations then correct each
    jet's pt by its table instead of scaling it."""
    n = int(batch.n_events)
    c = batch.cols
    kin_fmt = kin_fmt or getattr(batch, "kin_fmt", None)
    btag_fmt = btag_fmt or getattr(batch, "btag_fmt", None)
    keep = []

    def P(a):
        a = np.ascontiguousarray(a)
        keep.append(a)
        return a.ctypes.data

    b = _Batch()
    b.n_events = n
    b.offset_type = _code(batch.jet_offsets)
    b.jet_off, b.mu_off, b.el_off = P(batch.jet_offsets), P(batch.mu_offsets), P(batch.el_offsets)
    b.kin_type = _code(c["jet_pt"], kin_fmt)
    b.btag_type = _code(c["jet_btag"], btag_fmt if c["jet_btag"].dtype == np.uint16 else None)
    for coll in ("jet", "mu", "el"):
        for v in ("pt", "eta", "phi"):
            setattr(b, f"{coll}_{v}", P(c[f"{coll}_{v}"]))
    b.jet_mass = P(c["jet_mass"])
    b.jet_btag = P(c["jet_btag"])
    for coll in ("mu", "el"):
        setattr(b, f"{coll}_iso", P(np.asarray(c[f"{coll}_iso"], dtype=np.float32)))
        setattr(b, f"{coll}_tight", P(np.asarray(c[f"{coll}_tight"], dtype=np.uint8)))
    b.weight = P(batch.weight)

    cfg = _Config()
    cfg.lep_pt_min = cuts["lep_pt_min"]
    cfg.lep_abseta_max = cuts["lep_abseta_max"]
    cfg.lep_iso_max = cuts["lep_iso_max"]
    cfg.jet_pt_min = cuts["jet_pt_min"]
    cfg.jet_abseta_max = cuts["jet_abseta_max"]
    cfg.dr2_cut = cuts["dr2_cut"]
    cfg.btag_min = cuts["btag_min"]
    scales = np.array([np.float32(1.0 + 0.01 * k) for k in shifts], dtype=np.float32)
    nv = len(scales)
    cfg.n_var = nv
    cfg.scales = P(scales)
    nbins = np.array([s[3] for s in hist_specs], dtype=np.int32)
    edges = np.concatenate([hist_edges(s[1], s[2], s[3]) for s in hist_specs])
    cfg.n_hist = len(hist_specs)
    cfg.nbins = P(nbins)
    cfg.edges = P(edges)
    if jec is not None:
        # jet-energy corrections: eta_edges, pt_edges (float32) and contents
        # [n_var][len(eta_edges) + 1][len(pt_edges) + 1] (float32)
        ee = np.ascontiguousarray(jec["eta_edges"], dtype=np.float32)
        pe = np.ascontiguousarray(jec["pt_edges"], dtype=np.float32)
        ct = np.ascontiguousarray(jec["contents"], dtype=np.float32)
        assert ct.shape == (nv, len(ee) + 1, len(pe) + 1), ct.shape
        cfg.jec_neta, cfg.jec_npt = len(ee) - 1, len(pe) - 1
        cfg.jec_eta_edges, cfg.jec_pt_edges, cfg.jec_contents = P(ee), P(pe), P(ct)
    total_bins = int((nbins + 2).sum())

    out = {"counts": np.zeros((nv, total_bins), dtype=np.uint64),
           "sumw": np.zeros((nv, total_bins)), "sumw2": np.zeros((nv, total_bins)),
           "edges": edges, "nbins": nbins, "scales": scales}
    o = _Outputs()
    o.counts, o.sumw, o.sumw2 = (out["counts"].ctypes.data, out["sumw"].ctypes.data,
                                 out["sumw2"].ctypes.data)
    if per_event:
        out["pass"] = np.zeros((nv, n), dtype=np.uint8)
        out["nlep"] = np.zeros(n, dtype=np.int32)
        out["njet"] = np.zeros((nv, n), dtype=np.int32)
        out["nb"] = np.zeros((nv, n), dtype=np.int32)
        out["idx"] = np.zeros((nv, 5, n), dtype=np.int32)
        out["vars"] = np.zeros((nv, N_VARS, n))
        out["gap"] = np.zeros((nv, n))
        out["idx2"] = np.zeros((nv, 3, n), dtype=np.int32)
        o.ev_pass, o.ev_nlep = out["pass"].ctypes.data, out["nlep"].ctypes.data
        o.ev_njet, o.ev_nb = out["njet"].ctypes.data, out["nb"].ctypes.data
        o.ev_idx, o.ev_vars = out["idx"].ctypes.data, out["vars"].ctypes.data
        o.ev_gap, o.ev_idx2 = out["gap"].ctypes.data, out["idx2"].ctypes.data
    lib().oracle_run_chain(ctypes.byref(b), ctypes.byref(cfg), ctypes.byref(o))
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
