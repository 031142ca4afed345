"""The Section IV chain composed from the per-operation kernels.

This is the paper's own way of running an analysis: one library call per step
(object selection masks, segmented sums/maxima, get/set within offsets, Delta R
masking, masses, one fill_histogram call per histogram), with masks and
per-event arrays passed between calls through device memory. Every step is a
hepacc kernel; torch only allocates the intermediate arrays. It produces the
same histograms as the fused hepacc_run_chain and exists to measure the cost
of running the chain as separate calls.
"""
from __future__ import annotations

import math

import torch

from . import hepacc as H

NAN = float("nan")


class PerOpWorkspace:
    """Intermediate device arrays for one batch shape."""

    def __init__(self, batch: H.DeviceBatch):
        dev = batch.weight.device
        n = batch.n_events
        mj = batch.cols["jet_pt"].numel()
        mm = batch.cols["mu_pt"].numel()
        me = batch.cols["el_pt"].numel()
        f = lambda k: torch.empty(k, dtype=torch.float32, device=dev)
        i = lambda k: torch.empty(k, dtype=torch.int32, device=dev)
        u = lambda k: torch.empty(k, dtype=torch.uint8, device=dev)
        self.mu_sel, self.el_sel = u(mm), u(me)
        self.jet_acc, self.sel, self.sel2, self.bsel = u(mj), u(mj), u(mj), u(mj)
        self.ptk = f(mj)
        self.nlep, self.nmu, self.njet, self.nb = i(n), i(n), i(n), i(n)
        self.has_mu, self.pas, self.pas3 = u(n), u(n), u(n)
        self.lead_idx, self.sub_idx = i(n), i(n)
        self.v = {name: f(n) for name in ("ht", "lead_pt", "lead_eta", "lead_phi", "lead_mass", "lead_btag",
                                           "sub_pt", "m_jj", "max_btag", "m_jjj", "pt_jjj", "lep_pt", "lep_eta",
                                           "lep_phi", "lep_iso", "st", "sum_mass")}
        # float32 copies of half kinematic columns for the mass kernels
        kin = batch.cols["jet_eta"].dtype
        self.wide = kin != torch.float32
        if self.wide:
            self.jet_eta32, self.jet_phi32, self.jet_mass32 = f(mj), f(mj), f(mj)


def run_chain_per_op(b: H.DeviceBatch, cfg: H.ChainConfig, out: H.ChainOutputs, ws: PerOpWorkspace = None,
                     stream=None):
    """Accumulate the chain's histograms into ``out`` with per-operation calls."""
    if ws is None:
        ws = PerOpWorkspace(b)
    c = cfg.cuts
    C = b.cols
    jo, mo, eo = b.offsets["jet"], b.offsets["mu"], b.offsets["el"]
    inf = math.inf
    kw = {"stream": stream}

    # leptons: pt, |eta|, tight, iso selections (variation independent)
    for coll, sel in (("mu", ws.mu_sel), ("el", ws.el_sel)):
        H.hepacc_select_range(C[f"{coll}_pt"], lo=c["lep_pt_min"], hi=inf, mask_out=sel, **kw)
        H.hepacc_select_range(C[f"{coll}_eta"], lo=-inf, hi=c["lep_abseta_max"], use_abs=True, mask_in=sel,
                              mask_out=sel, **kw)
        H.hepacc_select_range(C[f"{coll}_tight"], lo=0.0, hi=inf, mask_in=sel, mask_out=sel, **kw)
        H.hepacc_select_range(C[f"{coll}_iso"], lo=-inf, hi=c["lep_iso_max"], mask_in=sel, mask_out=sel, **kw)
    ws.nlep.zero_()
    ws.nmu.zero_()
    H.hepacc_sum_in_offsets(ws.mu_sel, mo, out=ws.nlep, **kw)
    H.hepacc_sum_in_offsets(ws.el_sel, eo, out=ws.nlep, **kw)
    H.hepacc_sum_in_offsets(ws.mu_sel, mo, out=ws.nmu, **kw)
    # the lepton: first selected muon, else first selected electron
    H.hepacc_select_range(ws.nmu, lo=0.0, hi=inf, mask_out=ws.has_mu, **kw)
    for var, col in (("lep_pt", "pt"), ("lep_eta", "eta"), ("lep_phi", "phi"), ("lep_iso", "iso")):
        H.hepacc_get_in_offsets(C[f"el_{col}"], eo, 0, mask_content=ws.el_sel, default=NAN, out=ws.v[var],
                                index=_scratch_idx(ws), **kw)
        H.hepacc_get_in_offsets(C[f"mu_{col}"], mo, 0, mask_rows=ws.has_mu, mask_content=ws.mu_sel, default=NAN,
                                out=ws.v[var], index=_scratch_idx(ws), **kw)
    # jets: |eta| and Delta R to the selected leptons of both flavours
    H.hepacc_select_range(C["jet_eta"], lo=-inf, hi=c["jet_abseta_max"], use_abs=True, mask_out=ws.jet_acc, **kw)
    H.hepacc_mask_deltar(C["jet_eta"], C["jet_phi"], jo, C["mu_eta"], C["mu_phi"], mo, mask1_in=ws.jet_acc,
                         mask2=ws.mu_sel, dr2_cut=c["dr2_cut"], mask1_out=ws.jet_acc, **kw)
    H.hepacc_mask_deltar(C["jet_eta"], C["jet_phi"], jo, C["el_eta"], C["el_phi"], eo, mask1_in=ws.jet_acc,
                         mask2=ws.el_sel, dr2_cut=c["dr2_cut"], mask1_out=ws.jet_acc, **kw)
    if ws.wide:
        H.hepacc_scale(C["jet_eta"], 1.0, out=ws.jet_eta32, **kw)
        H.hepacc_scale(C["jet_phi"], 1.0, out=ws.jet_phi32, **kw)
        H.hepacc_scale(C["jet_mass"], 1.0, out=ws.jet_mass32, **kw)
        eta32, phi32, mass32 = ws.jet_eta32, ws.jet_phi32, ws.jet_mass32
    else:
        eta32, phi32, mass32 = C["jet_eta"], C["jet_phi"], C["jet_mass"]

    v = ws.v
    for k in range(cfg.n_var):
        s = float(cfg.scales[k])
        H.hepacc_scale(C["jet_pt"], s, out=ws.ptk, **kw)
        H.hepacc_select_range(ws.ptk, lo=c["jet_pt_min"], hi=inf, mask_in=ws.jet_acc, mask_out=ws.sel, **kw)
        H.hepacc_select_range(C["jet_btag"], lo=c["btag_min"], hi=inf, mask_in=ws.sel, mask_out=ws.bsel, **kw)
        ws.njet.zero_()
        ws.nb.zero_()
        H.hepacc_sum_in_offsets(ws.sel, jo, out=ws.njet, **kw)
        H.hepacc_sum_in_offsets(ws.bsel, jo, out=ws.nb, **kw)
        H.hepacc_select_range(ws.nlep, lo=0.5, hi=1.5, mask_out=ws.pas, **kw)
        H.hepacc_select_range(ws.njet, lo=1.5, hi=inf, mask_in=ws.pas, mask_out=ws.pas, **kw)
        H.hepacc_select_range(ws.nb, lo=0.5, hi=inf, mask_in=ws.pas, mask_out=ws.pas, **kw)
        H.hepacc_select_range(ws.njet, lo=2.5, hi=inf, mask_in=ws.pas, mask_out=ws.pas3, **kw)
        for name in ("ht", "st", "sum_mass"):
            v[name].zero_()
        H.hepacc_sum_in_offsets(ws.ptk, jo, mask_content=ws.sel, out=v["ht"], **kw)
        H.hepacc_sum_in_offsets(ws.ptk, jo, mask_content=ws.sel, out=v["st"], **kw)
        H.hepacc_sum_in_offsets(C["mu_pt"], mo, mask_content=ws.mu_sel, out=v["st"], **kw)
        H.hepacc_sum_in_offsets(C["el_pt"], eo, mask_content=ws.el_sel, out=v["st"], **kw)
        H.hepacc_sum_in_offsets(C["jet_mass"], jo, mask_content=ws.sel, out=v["sum_mass"], **kw)
        H.hepacc_max_in_offsets(ws.ptk, jo, mask_content=ws.sel, empty=NAN, out=v["lead_pt"], arg=ws.lead_idx, **kw)
        # sub-leading: the same maximum with the leading jet masked out
        H.hepacc_select_range(ws.ptk, lo=-inf, hi=inf, mask_in=ws.sel, mask_out=ws.sel2, **kw)
        H.hepacc_set_in_offsets(ws.sel2, jo, nth=ws.lead_idx, value=0, **kw)
        H.hepacc_max_in_offsets(ws.ptk, jo, mask_content=ws.sel2, empty=NAN, out=v["sub_pt"], arg=ws.sub_idx, **kw)
        for var, col in (("lead_eta", "jet_eta"), ("lead_phi", "jet_phi"), ("lead_mass", "jet_mass"),
                         ("lead_btag", "jet_btag")):
            H.hepacc_get_in_offsets(C[col], jo, ws.lead_idx, default=NAN, out=v[var], index=_scratch_idx(ws), **kw)
        H.hepacc_max_in_offsets(C["jet_btag"], jo, mask_content=ws.sel, empty=NAN, out=v["max_btag"],
                                arg=_scratch_idx(ws), **kw)
        H.hepacc_pair_mass(ws.ptk, eta32, phi32, mass32, jo, ws.lead_idx, ws.sub_idx, out=v["m_jj"], **kw)
        H.hepacc_max_pt_trijet(ws.ptk, eta32, phi32, mass32, jo, mask_content=ws.sel, out_mass=v["m_jjj"],
                               out_pt=v["pt_jjj"], out_idx3=_scratch_idx3(ws), **kw)
        data = [v["ht"], v["lead_pt"], v["lead_eta"], v["lead_phi"], v["lead_mass"], v["lead_btag"], v["sub_pt"],
                v["m_jj"], ws.njet, ws.nb, v["max_btag"], v["m_jjj"], v["pt_jjj"], v["lep_pt"], v["lep_eta"],
                v["lep_phi"], v["lep_iso"], v["st"], v["sum_mass"], b.weight]
        for h in range(H.NVARS):
            lo = int(cfg.bin_offsets[h])
            hi = lo + int(cfg.nbins[h]) + 2
            e0 = int(sum(cfg.nbins[:h] + 1))
            edges = _edges_dev(cfg, b.weight.device)[e0:e0 + int(cfg.nbins[h]) + 1]
            mask = ws.pas3 if h in (11, 12) else ws.pas
            H.hepacc_fill_histogram(data[h], edges, weights=b.weight, mask=mask, counts=out.counts[k, lo:hi],
                                    sumw=out.sumw[k, lo:hi],
                                    sumw2=None if out.sumw2 is None else out.sumw2[k, lo:hi],
                                    with_sumw2=out.sumw2 is not None, **kw)
    return out


def dimuon_mass(pt, eta, phi, mass, charge, offsets, mask_in=None, stream=None):
    """Dimuon candidate per event (Section III, select_opposite_sign_muons,
    then a pair mass): the first opposite-charge pair among the muons with
    mask_in set, its two local indices (get_in_offsets with n = 0 and 1 over
    the pair mask) and its invariant mass; NaN and -1, -1 without a pair.
    Returns (mass, idx_a, idx_b, pair_mask)."""
    pair = H.hepacc_select_opposite_sign(charge, offsets, mask_in=mask_in, stream=stream)
    _, ia = H.hepacc_get_in_offsets(pt, offsets, nth=0, mask_content=pair, stream=stream)
    _, ib = H.hepacc_get_in_offsets(pt, offsets, nth=1, mask_content=pair, stream=stream)
    m = H.hepacc_pair_mass(pt, eta, phi, mass, offsets, ia, ib, stream=stream)
    return m, ia, ib, pair


def _scratch_idx(ws):
    if not hasattr(ws, "_idx_scratch"):
        ws._idx_scratch = torch.empty_like(ws.lead_idx)
    return ws._idx_scratch


def _scratch_idx3(ws):
    if not hasattr(ws, "_idx3_scratch"):
        ws._idx3_scratch = torch.empty((ws.lead_idx.numel(), 3), dtype=torch.int32, device=ws.lead_idx.device)
    return ws._idx3_scratch


_EDGE_CACHE = {}


def _edges_dev(cfg, device):
    key = (id(cfg), str(device))
    if key not in _EDGE_CACHE:
        _EDGE_CACHE[key] = torch.from_numpy(cfg.edges).to(device)
    return _EDGE_CACHE[key]
