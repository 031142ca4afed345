"""Thin Python binding of the hepacc C ABI (include/hepacc.h).

Argument marshalling only: every function here passes device pointers of
torch tensors, sizes and the current CUDA stream to the function of the same
name in libhepacc.so; all computation happens in the library's kernels.
There is no CPU path: if the library cannot be loaded, calls raise.
"""
from __future__ import annotations

import ctypes
import json
import math
import os

import numpy as np
import torch

from . import build as _build

F32, F16, BF16, I8, U8, I32, I64, F64 = 0, 1, 2, 3, 4, 5, 6, 7
NVARS = 20
MAX_VARIATIONS = 64
MAX_EDGES = 4096

_TORCH_CODE = {torch.float32: F32, torch.float16: F16, torch.bfloat16: BF16, torch.int8: I8,
               torch.uint8: U8, torch.int32: I32, torch.int64: I64, torch.float64: F64}

_c_void_p = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_f32 = ctypes.c_float


class HepaccError(RuntimeError):
    """A hepacc call returned a non-OK status."""

    def __init__(self, status, message):
        super().__init__(f"{message} [status {status}]")
        self.status = status


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libhepacc.so (building it first when missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"hepacc library not built: {_build.LIB}")
    L = ctypes.CDLL(_build.LIB)
    L.hepacc_version.restype = ctypes.c_char_p
    L.hepacc_last_error.restype = ctypes.c_char_p
    L.hepacc_status_string.restype = ctypes.c_char_p
    L.hepacc_status_string.argtypes = [ctypes.c_int]
    for name in ("hepacc_sum_in_offsets", "hepacc_max_in_offsets", "hepacc_min_in_offsets",
                 "hepacc_get_in_offsets", "hepacc_set_in_offsets", "hepacc_select_range", "hepacc_scale",
                 "hepacc_mask_deltar", "hepacc_fill_histogram", "hepacc_pair_mass", "hepacc_max_pt_trijet",
                 "hepacc_run_chain", "hepacc_validate_offsets", "hepacc_device_error",
                 "hepacc_selftest_wait_timeout", "hepacc_plan_create", "hepacc_plan_run",
                 "hepacc_plan_describe", "hepacc_trijet_closest_mass", "hepacc_select_opposite_sign",
                 "hepacc_get_bin_contents", "hepacc_fill_histogram_nd"):
        getattr(L, name).restype = ctypes.c_int
    L.hepacc_plan_destroy.restype = None
    L.hepacc_plan_destroy.argtypes = [ctypes.c_void_p]
    L.hepacc_plan_run.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p]
    L.hepacc_plan_describe.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int32]
    _lib = L
    return L


def _check(status: int):
    if status != 0:
        L = load()
        raise HepaccError(status, f"{L.hepacc_status_string(status).decode()}: {L.hepacc_last_error().decode()}")


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return _c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


_EMPTY = {}


def _addr(t) -> int:
    """Device address of a tensor; empty tensors (which torch gives address 0)
    get a small placeholder allocation, never read since nothing is in it."""
    if t.numel() == 0:
        key = t.device.index
        if key not in _EMPTY:
            _EMPTY[key] = torch.zeros(64, dtype=torch.uint8, device=t.device)
        return _EMPTY[key].data_ptr()
    return t.data_ptr()


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("hepacc arrays must be CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("hepacc arrays must be contiguous")
    return _c_void_p(_addr(t))


def _code(t):
    return _TORCH_CODE[t.dtype]


def version() -> str:
    return load().hepacc_version().decode()


def device_error() -> int:
    """Read and clear the device error word (synchronises the device)."""
    v = ctypes.c_uint32(0)
    _check(load().hepacc_device_error(ctypes.byref(v)))
    return v.value


def hepacc_selftest_wait_timeout(limit_cycles=1_000_000, stream=None):
    """Run the bounded-wait self-test kernel (sets the device error word)."""
    _check(load().hepacc_selftest_wait_timeout(_i64(limit_cycles), _stream(stream)))


# ---------------------------------------------------------------------------
# generic kernels (Section III)
# ---------------------------------------------------------------------------

def hepacc_sum_in_offsets(content, offsets, mask_rows=None, mask_content=None, out=None, out_dtype=None,
                          stream=None):
    n = offsets.numel() - 1
    if out is None:
        if out_dtype is None:
            out_dtype = torch.float32 if content.is_floating_point() else torch.int64
        out = torch.zeros(n, dtype=out_dtype, device=content.device)
    _check(load().hepacc_sum_in_offsets(_ptr(content), _code(content), _ptr(offsets), _code(offsets), _i64(n),
                                        _ptr(mask_rows), _ptr(mask_content), _ptr(out), _code(out),
                                        _stream(stream)))
    return out


def _minmax(fn, content, offsets, mask_rows, mask_content, empty, out, arg, stream):
    n = offsets.numel() - 1
    if out is None:
        out = torch.full((n,), float("nan"), dtype=torch.float32, device=content.device)
    if arg is None:
        arg = torch.full((n,), -7, dtype=torch.int32, device=content.device)
    _check(fn(_ptr(content), _code(content), _ptr(offsets), _code(offsets), _i64(n), _ptr(mask_rows),
              _ptr(mask_content), _f32(empty), _ptr(out), _ptr(arg), _stream(stream)))
    return out, arg


def hepacc_max_in_offsets(content, offsets, mask_rows=None, mask_content=None, empty=-math.inf, out=None,
                          arg=None, stream=None):
    return _minmax(load().hepacc_max_in_offsets, content, offsets, mask_rows, mask_content, empty, out, arg, stream)


def hepacc_min_in_offsets(content, offsets, mask_rows=None, mask_content=None, empty=math.inf, out=None,
                          arg=None, stream=None):
    return _minmax(load().hepacc_min_in_offsets, content, offsets, mask_rows, mask_content, empty, out, arg, stream)


def hepacc_get_in_offsets(content, offsets, nth=0, mask_rows=None, mask_content=None, default=math.nan,
                          out=None, index=None, stream=None):
    n = offsets.numel() - 1
    nth_t = nth if torch.is_tensor(nth) else None
    if out is None:
        out = torch.full((n,), float("nan"), dtype=torch.float32, device=content.device)
    if index is None:
        index = torch.full((n,), -7, dtype=torch.int32, device=content.device)
    _check(load().hepacc_get_in_offsets(_ptr(content), _code(content), _ptr(offsets), _code(offsets), _i64(n),
                                        _ptr(nth_t), _i32(0 if nth_t is not None else int(nth)), _ptr(mask_rows),
                                        _ptr(mask_content), _f32(default), _ptr(out), _ptr(index),
                                        _stream(stream)))
    return out, index


def hepacc_set_in_offsets(content, offsets, nth=0, value=0, mask_rows=None, mask_content=None, stream=None):
    n = offsets.numel() - 1
    nth_t = nth if torch.is_tensor(nth) else None
    _check(load().hepacc_set_in_offsets(_ptr(content), _code(content), _ptr(offsets), _code(offsets), _i64(n),
                                        _ptr(nth_t), _i32(0 if nth_t is not None else int(nth)), _ptr(mask_rows),
                                        _ptr(mask_content), ctypes.c_double(value), _stream(stream)))
    return content


def hepacc_select_range(content, lo=-math.inf, hi=math.inf, scale=1.0, use_abs=False, mask_in=None,
                        mask_out=None, stream=None):
    n = content.numel()
    if mask_out is None:
        mask_out = torch.empty(n, dtype=torch.uint8, device=content.device)
    _check(load().hepacc_select_range(_ptr(content), _code(content), _i64(n), _f32(scale), _f32(lo), _f32(hi),
                                      ctypes.c_int(int(use_abs)), _ptr(mask_in), _ptr(mask_out), _stream(stream)))
    return mask_out


def hepacc_scale(content, scale, out=None, stream=None):
    n = content.numel()
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=content.device)
    _check(load().hepacc_scale(_ptr(content), _code(content), _i64(n), _f32(scale), _ptr(out), _stream(stream)))
    return out


def hepacc_mask_deltar(eta1, phi1, offsets1, eta2, phi2, offsets2, mask_rows=None, mask1_in=None, mask2=None,
                       dr2_cut=0.16, mask1_out=None, stream=None):
    n = offsets1.numel() - 1
    if mask1_out is None:
        mask1_out = torch.full((eta1.numel(),), 7, dtype=torch.uint8, device=eta1.device)
    _check(load().hepacc_mask_deltar(_ptr(eta1), _ptr(phi1), _code(eta1), _ptr(offsets1), _ptr(eta2), _ptr(phi2),
                                     _code(eta2), _ptr(offsets2), _code(offsets1), _i64(n), _ptr(mask_rows),
                                     _ptr(mask1_in), _ptr(mask2), _f32(dr2_cut), _ptr(mask1_out),
                                     _stream(stream)))
    return mask1_out


def hepacc_fill_histogram(data, edges, weights=None, mask=None, counts=None, sumw=None, sumw2=None,
                          with_sumw2=True, stream=None):
    nb = edges.numel() - 1
    dev = data.device
    if counts is None:
        counts = torch.zeros(nb + 2, dtype=torch.int64, device=dev)
    if sumw is None:
        sumw = torch.zeros(nb + 2, dtype=torch.float64, device=dev)
    if sumw2 is None and with_sumw2:
        sumw2 = torch.zeros(nb + 2, dtype=torch.float64, device=dev)
    _check(load().hepacc_fill_histogram(_ptr(data), _code(data), _ptr(weights), _ptr(mask), _i64(data.numel()),
                                        _ptr(edges), _i32(nb), _ptr(counts), _ptr(sumw), _ptr(sumw2),
                                        _stream(stream)))
    return counts, sumw, sumw2


def hepacc_fill_histogram_nd(data, edges, weights=None, mask=None, counts=None, sumw=None, sumw2=None,
                             with_sumw2=True, stream=None):
    """Histogram over len(data) variables; the outputs are shaped
    (nbins_0 + 2, nbins_1 + 2, ...), axis 0 slowest."""
    k = len(data)
    if k != len(edges):
        raise ValueError("one edges tensor per axis")
    shape = tuple(e.numel() + 1 for e in edges)
    dev = data[0].device
    if counts is None:
        counts = torch.zeros(shape, dtype=torch.int64, device=dev)
    if sumw is None:
        sumw = torch.zeros(shape, dtype=torch.float64, device=dev)
    if sumw2 is None and with_sumw2:
        sumw2 = torch.zeros(shape, dtype=torch.float64, device=dev)
    n = data[0].numel()
    if any(x.numel() != n for x in data):
        raise ValueError("all axes need the same number of elements")
    ptrs = (ctypes.c_void_p * k)(*[_ptr(x) for x in data])
    types = (ctypes.c_int * k)(*[_code(x) for x in data])
    eptrs = (ctypes.c_void_p * k)(*[_ptr(e) for e in edges])
    nbs = (ctypes.c_int32 * k)(*[e.numel() - 1 for e in edges])
    _check(load().hepacc_fill_histogram_nd(_i32(k), ptrs, types, eptrs, nbs, _ptr(weights), _ptr(mask),
                                           _i64(n), _ptr(counts), _ptr(sumw), _ptr(sumw2), _stream(stream)))
    return counts, sumw, sumw2


def hepacc_pair_mass(pt, eta, phi, mass, offsets, idx_a, idx_b, mask_rows=None, out=None, stream=None):
    n = offsets.numel() - 1
    if out is None:
        out = torch.full((n,), float("nan"), dtype=torch.float32, device=pt.device)
    _check(load().hepacc_pair_mass(_ptr(pt), _ptr(eta), _ptr(phi), _ptr(mass), _code(pt), _ptr(offsets),
                                   _code(offsets), _i64(n), _ptr(idx_a), _ptr(idx_b), _ptr(mask_rows), _ptr(out),
                                   _stream(stream)))
    return out


def hepacc_max_pt_trijet(pt, eta, phi, mass, offsets, mask_rows=None, mask_content=None, out_mass=None,
                         out_pt=None, out_idx3=None, stream=None):
    n = offsets.numel() - 1
    dev = pt.device
    if out_mass is None:
        out_mass = torch.full((n,), float("nan"), dtype=torch.float32, device=dev)
    if out_pt is None:
        out_pt = torch.full((n,), float("nan"), dtype=torch.float32, device=dev)
    if out_idx3 is None:
        out_idx3 = torch.full((n, 3), -7, dtype=torch.int32, device=dev)
    _check(load().hepacc_max_pt_trijet(_ptr(pt), _ptr(eta), _ptr(phi), _ptr(mass), _code(pt), _ptr(offsets),
                                       _code(offsets), _i64(n), _ptr(mask_rows), _ptr(mask_content),
                                       _ptr(out_mass), _ptr(out_pt), _ptr(out_idx3), _stream(stream)))
    return out_mass, out_pt, out_idx3


def hepacc_trijet_closest_mass(pt, eta, phi, mass, offsets, target=172.0, mask_rows=None, mask_content=None,
                               out_mass=None, out_idx3=None, stream=None):
    """Top candidate: the triplet of masked-in objects with mass closest to
    ``target``; returns (mass [N] float32, idx3 [N,3] int32)."""
    n = offsets.numel() - 1
    if out_mass is None:
        out_mass = torch.full((n,), float("nan"), dtype=torch.float32, device=pt.device)
    if out_idx3 is None:
        out_idx3 = torch.full((n, 3), -7, dtype=torch.int32, device=pt.device)
    _check(load().hepacc_trijet_closest_mass(_ptr(pt), _ptr(eta), _ptr(phi), _ptr(mass), _code(pt), _ptr(offsets),
                                             _code(offsets), _i64(n), _ptr(mask_rows), _ptr(mask_content),
                                             _f32(target), _ptr(out_mass), _ptr(out_idx3), _stream(stream)))
    return out_mass, out_idx3


def hepacc_select_opposite_sign(charge, offsets, mask_rows=None, mask_in=None, mask_out=None, stream=None):
    """Keep the first two masked-in objects of opposite charge per event."""
    n = offsets.numel() - 1
    if mask_out is None:
        mask_out = torch.zeros(charge.numel(), dtype=torch.uint8, device=charge.device)
    _check(load().hepacc_select_opposite_sign(_ptr(charge), _ptr(offsets), _code(offsets), _i64(n),
                                              _ptr(mask_rows), _ptr(mask_in), _ptr(mask_out), _stream(stream)))
    return mask_out


def hepacc_get_bin_contents(data, edges, contents, interpolate=False, out=None, stream=None):
    """Histogram lookup (bin contents, or binary32 linear interpolation
    between bin centres); edges and contents are float32 device tensors."""
    if out is None:
        out = torch.empty(data.numel(), dtype=torch.float32, device=data.device)
    _check(load().hepacc_get_bin_contents(_ptr(data), _code(data), _i64(data.numel()), _ptr(edges),
                                          _i32(edges.numel() - 1), _ptr(contents), _i32(1 if interpolate else 0),
                                          _ptr(out), _stream(stream)))
    return out


def hepacc_validate_offsets(offsets, content_len, first_bad=None, stream=None):
    n = offsets.numel() - 1
    if first_bad is None:
        first_bad = torch.zeros(1, dtype=torch.int64, device=offsets.device)
    _check(load().hepacc_validate_offsets(_ptr(offsets), _code(offsets), _i64(n), _i64(content_len),
                                          _ptr(first_bad), _stream(stream)))
    return first_bad


# ---------------------------------------------------------------------------
# the fused chain (Section IV)
# ---------------------------------------------------------------------------

class EventBatchC(ctypes.Structure):
    _fields_ = [("n_events", ctypes.c_int64), ("offsets_type", ctypes.c_int),
                ("jet_offsets", _c_void_p), ("mu_offsets", _c_void_p), ("el_offsets", _c_void_p),
                ("kin_type", ctypes.c_int), ("btag_type", ctypes.c_int),
                ("jet_pt", _c_void_p), ("jet_eta", _c_void_p), ("jet_phi", _c_void_p), ("jet_mass", _c_void_p),
                ("jet_btag", _c_void_p),
                ("mu_pt", _c_void_p), ("mu_eta", _c_void_p), ("mu_phi", _c_void_p), ("mu_iso", _c_void_p),
                ("mu_tight", _c_void_p),
                ("el_pt", _c_void_p), ("el_eta", _c_void_p), ("el_phi", _c_void_p), ("el_iso", _c_void_p),
                ("el_tight", _c_void_p),
                ("weight", _c_void_p), ("jets_per_event", ctypes.c_float),
                ("muons_per_event", ctypes.c_float), ("electrons_per_event", ctypes.c_float),
                ("jet_len", ctypes.c_int64), ("mu_len", ctypes.c_int64), ("el_len", ctypes.c_int64)]


class ChainConfigC(ctypes.Structure):
    _fields_ = [("lep_pt_min", ctypes.c_float), ("lep_abseta_max", ctypes.c_float),
                ("lep_iso_max", ctypes.c_float), ("jet_pt_min", ctypes.c_float),
                ("jet_abseta_max", ctypes.c_float), ("dr2_cut", ctypes.c_float), ("btag_min", ctypes.c_float),
                ("n_var", ctypes.c_int32), ("scales", _c_void_p), ("nbins", ctypes.c_int32 * NVARS),
                ("edges", _c_void_p), ("jec_neta", ctypes.c_int32), ("jec_npt", ctypes.c_int32),
                ("jec_eta_edges", _c_void_p), ("jec_pt_edges", _c_void_p), ("jec_contents", _c_void_p)]


class ChainOutputsC(ctypes.Structure):
    _fields_ = [("counts", _c_void_p), ("sumw", _c_void_p), ("sumw2", _c_void_p), ("ev_pass", _c_void_p),
                ("ev_nlep", _c_void_p), ("ev_njet", _c_void_p), ("ev_nb", _c_void_p), ("ev_idx", _c_void_p),
                ("ev_vars", _c_void_p)]


COLUMNS = ("jet_pt", "jet_eta", "jet_phi", "jet_mass", "jet_btag", "mu_pt", "mu_eta", "mu_phi", "mu_iso",
           "mu_tight", "el_pt", "el_eta", "el_phi", "el_iso", "el_tight")


class DeviceBatch:
    """Device-resident columns of one sample (torch tensors) and the C struct
    pointing at them."""

    def __init__(self, n_events, offsets, cols, weight, objects=None):
        self.n_events = int(n_events)
        self.offsets = offsets      # dict jet/mu/el -> tensor
        self.cols = cols            # dict name -> tensor
        self.weight = weight
        self._objects = objects     # dict jet/mu/el -> objects in these events (None: read from the offsets)
        self._c = None

    @classmethod
    def from_host(cls, batch, device="cuda", non_blocking=False):
        """Copy a host batch (numpy columns; half columns as uint16 bit
        patterns with ``kin_fmt``/``btag_fmt`` attributes) to the device."""
        kin_fmt = getattr(batch, "kin_fmt", None)
        btag_fmt = getattr(batch, "btag_fmt", None)
        half = {"bf16": torch.bfloat16, "f16": torch.float16}

        def up(a, fmt=None):
            t = torch.from_numpy(np.ascontiguousarray(a))
            if a.dtype == np.uint16:
                t = t.view(torch.int16).view(half[fmt])
            return t.to(device, non_blocking=non_blocking)

        offsets = {k: up(v) for k, v in batch.offsets.items()}
        cols = {}
        for name in COLUMNS:
            a = batch.cols[name]
            fmt = btag_fmt if name == "jet_btag" else kin_fmt
            cols[name] = up(a, fmt)
        objects = {k: int(v[-1] - v[0]) if len(v) else 0 for k, v in batch.offsets.items()}
        return cls(batch.n_events, offsets, cols, up(batch.weight), objects=objects)

    def objects(self) -> dict:
        """Objects per collection in this batch's events (offsets[n] -
        offsets[0]; a slice of a larger batch shares its columns): as given
        at construction, else read once from the device offsets."""
        if getattr(self, "_objects", None) is None:
            if self.n_events == 0:
                self._objects = {k: 0 for k in self.offsets}
            else:
                self._objects = {k: int((v[-1] - v[0]).item()) for k, v in self.offsets.items()}
        return self._objects

    def nbytes_read(self) -> int:
        """Bytes of every array the chain reads: offsets, the 15 columns, weight."""
        tot = sum(t.numel() * t.element_size() for t in self.offsets.values())
        tot += sum(t.numel() * t.element_size() for t in self.cols.values())
        return tot + self.weight.numel() * 4

    def c_struct(self):
        c = EventBatchC()
        c.n_events = self.n_events
        c.offsets_type = _code(self.offsets["jet"])
        c.jet_offsets = _addr(self.offsets["jet"])
        c.mu_offsets = _addr(self.offsets["mu"])
        c.el_offsets = _addr(self.offsets["el"])
        c.kin_type = _code(self.cols["jet_pt"])
        c.btag_type = _code(self.cols["jet_btag"])
        for name in COLUMNS:
            setattr(c, name, _addr(self.cols[name]))
        c.weight = _addr(self.weight)
        n = max(1, self.n_events)
        objs = self.objects()
        c.jets_per_event = objs["jet"] / n
        c.muons_per_event = objs["mu"] / n
        c.electrons_per_event = objs["el"] / n
        c.jet_len = self.cols["jet_pt"].numel()
        c.mu_len = self.cols["mu_pt"].numel()
        c.el_len = self.cols["el_pt"].numel()
        self._c = c
        return c


def hist_edges(lo, hi, nbins):
    """binary32 edges float32(lo + (hi - lo) * b / nbins), b = 0..nbins, with
    the arithmetic in binary64."""
    b = np.arange(nbins + 1, dtype=np.float64)
    return (lo + (hi - lo) * b / nbins).astype(np.float32)


class ChainConfig:
    """Cuts, jet-pt scales and histogram edges of the chain (host memory);
    optionally jet-energy correction tables (``jec``: dict of eta_edges,
    pt_edges (host, float32) and contents, a float32 tensor
    [n_var][n_eta + 2][n_pt + 2], moved to the device)."""

    def __init__(self, cuts, hist_specs, scales, jec=None):
        if len(hist_specs) != NVARS:
            raise ValueError(f"the chain fills exactly {NVARS} histograms")
        self.cuts = dict(cuts)
        self.hist_specs = list(hist_specs)
        self.scales = np.asarray(scales, dtype=np.float32)
        self.nbins = np.array([h[3] for h in hist_specs], dtype=np.int32)
        self.edges = np.concatenate([hist_edges(h[1], h[2], h[3]) for h in hist_specs]).astype(np.float32)
        self.total_bins = int((self.nbins + 2).sum())
        self.bin_offsets = np.concatenate([[0], np.cumsum(self.nbins + 2)[:-1]]).astype(np.int64)
        self.jec = None
        if jec is not None:
            ee = np.ascontiguousarray(jec["eta_edges"], dtype=np.float32)
            pe = np.ascontiguousarray(jec["pt_edges"], dtype=np.float32)
            ct = torch.as_tensor(np.asarray(jec["contents"], dtype=np.float32)).contiguous().cuda()
            if tuple(ct.shape) != (len(self.scales), len(ee) + 1, len(pe) + 1):
                raise ValueError(f"correction contents must be [n_var][n_eta + 2][n_pt + 2], got {tuple(ct.shape)}")
            self.jec = (ee, pe, ct)

    @property
    def n_var(self):
        return len(self.scales)

    def c_struct(self):
        c = ChainConfigC()
        for k in ("lep_pt_min", "lep_abseta_max", "lep_iso_max", "jet_pt_min", "jet_abseta_max", "dr2_cut",
                  "btag_min"):
            setattr(c, k, float(self.cuts[k]))
        c.n_var = self.n_var
        c.scales = self.scales.ctypes.data
        for h in range(NVARS):
            c.nbins[h] = int(self.nbins[h])
        c.edges = self.edges.ctypes.data
        if self.jec is not None:
            ee, pe, ct = self.jec
            c.jec_neta, c.jec_npt = len(ee) - 1, len(pe) - 1
            c.jec_eta_edges, c.jec_pt_edges, c.jec_contents = ee.ctypes.data, pe.ctypes.data, ct.data_ptr()
        return c


class ChainOutputs:
    """Histogram outputs [n_var, total_bins] and optional per-event arrays."""

    def __init__(self, cfg: ChainConfig, n_events: int, per_event=False, sumw2=True, device="cuda"):
        nv, tb = cfg.n_var, cfg.total_bins
        self.counts = torch.zeros((nv, tb), dtype=torch.int64, device=device)
        self.sumw = torch.zeros((nv, tb), dtype=torch.float64, device=device)
        self.sumw2 = torch.zeros((nv, tb), dtype=torch.float64, device=device) if sumw2 else None
        self.per_event = per_event
        if per_event:
            n = n_events
            self.ev_pass = torch.full((nv, n), 7, dtype=torch.uint8, device=device)
            self.ev_nlep = torch.full((n,), -7, dtype=torch.int32, device=device)
            self.ev_njet = torch.full((nv, n), -7, dtype=torch.int32, device=device)
            self.ev_nb = torch.full((nv, n), -7, dtype=torch.int32, device=device)
            self.ev_idx = torch.full((nv, 5, n), -7, dtype=torch.int32, device=device)
            self.ev_vars = torch.full((nv, NVARS, n), -7.0, dtype=torch.float32, device=device)

    def zero_(self):
        self.counts.zero_()
        self.sumw.zero_()
        if self.sumw2 is not None:
            self.sumw2.zero_()

    def c_struct(self):
        c = ChainOutputsC()
        c.counts = self.counts.data_ptr()
        c.sumw = self.sumw.data_ptr()
        c.sumw2 = self.sumw2.data_ptr() if self.sumw2 is not None else None
        if self.per_event:
            c.ev_pass = self.ev_pass.data_ptr()
            c.ev_nlep = self.ev_nlep.data_ptr()
            c.ev_njet = self.ev_njet.data_ptr()
            c.ev_nb = self.ev_nb.data_ptr()
            c.ev_idx = self.ev_idx.data_ptr()
            c.ev_vars = self.ev_vars.data_ptr()
        return c


def hepacc_run_chain(batch: DeviceBatch, cfg: ChainConfig, out: ChainOutputs, stream=None, _structs=None):
    """Run the fused chain; histograms in ``out`` accumulate."""
    if _structs is None:
        _structs = (batch.c_struct(), cfg.c_struct(), out.c_struct())
    bc, cc, oc = _structs
    _check(load().hepacc_run_chain(ctypes.byref(bc), ctypes.byref(cc), ctypes.byref(oc), _stream(stream)))
    return out


PLAN_AUTOTUNE = 1
PLAN_GRAPH = 2
PLAN_HIST_BLOCK, PLAN_HIST_CLUSTER8, PLAN_HIST_CLUSTER16, PLAN_HIST_GLOBAL = 4, 8, 16, 32
PLAN_VALIDATE = 64


class Plan:
    """A batched chain plan (``hepacc_plan_create``): samples, their outputs
    and the launch configuration, run with :meth:`run`. Keeps the Python
    objects whose device memory the plan points at alive."""

    def __init__(self, handle, batches, outputs, cfg):
        self._h = handle
        self.batches = batches
        self.outputs = outputs
        self.cfg = cfg

    def run(self, stream=None):
        """Run the samples and outputs the plan was created with."""
        _check(load().hepacc_plan_run(self._h, 0, None, None, _stream(stream)))

    def run_batch(self, batches, outputs, stream=None, _structs=None):
        """Run the plan's configuration (and graph) over another batch of as
        many samples: ``batches[i]`` adds to ``outputs[i]``. The tensors must
        stay alive until the run is done; the returned structs can be passed
        back as ``_structs`` to skip rebuilding them."""
        if _structs is None:
            if len(batches) != len(outputs):
                raise ValueError("one output per sample")
            n = len(batches)
            _structs = (n, (EventBatchC * n)(*[b.c_struct() for b in batches]),
                        (ChainOutputsC * n)(*[o.c_struct() for o in outputs]))
        n, bs, os_ = _structs
        _check(load().hepacc_plan_run(self._h, n, bs, os_, _stream(stream)))
        return _structs

    def describe(self) -> dict:
        buf = ctypes.create_string_buffer(16384)
        _check(load().hepacc_plan_describe(self._h, buf, len(buf)))
        return json.loads(buf.value.decode())

    def close(self):
        if self._h:
            load().hepacc_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hepacc_plan_create(cfg: ChainConfig, batches, outputs, flags=PLAN_AUTOTUNE | PLAN_GRAPH, stream=None) -> Plan:
    """Plan the chain over many samples (``batches[i]`` adds to
    ``outputs[i]``); see :class:`Plan`."""
    if len(batches) != len(outputs) or not batches:
        raise ValueError("one output per sample, at least one sample")
    n = len(batches)
    bs = (EventBatchC * n)(*[b.c_struct() for b in batches])
    os_ = (ChainOutputsC * n)(*[o.c_struct() for o in outputs])
    cc = cfg.c_struct()
    h = ctypes.c_void_p()
    _check(load().hepacc_plan_create(ctypes.byref(cc), n, bs, os_, int(flags), _stream(stream), ctypes.byref(h)))
    return Plan(h, list(batches), list(outputs), cfg)
