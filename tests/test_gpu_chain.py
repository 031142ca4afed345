"""GPU parity of the fused chain (hepacc_run_chain) and of the per-operation
chain against the oracle (Section IV benchmark analysis)."""
import json
import os

import numpy as np
import pytest
import torch

from paper_1906_06242_gb300 import synth
from tests import chain_check as CC

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_events.json")


@pytest.fixture(scope="module")
def H():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1906_06242_gb300 import hepacc
    hepacc.load()
    return hepacc


def run_gpu(H, batch, shifts, per_event=True, sumw2=True, jec=None):
    cfg = H.ChainConfig(synth.CUTS, synth.HIST_SPECS, synth.variation_scales(1) if shifts is None else
                        [np.float32(1.0 + 0.01 * k) for k in shifts], jec=jec)
    db = H.DeviceBatch.from_host(batch)
    out = H.ChainOutputs(cfg, batch.n_events, per_event=per_event, sumw2=sumw2)
    H.hepacc_run_chain(db, cfg, out)
    torch.cuda.synchronize()
    res = {"counts": out.counts.cpu().numpy().view(np.uint64), "sumw": out.sumw.cpu().numpy(),
           "sumw2": None if out.sumw2 is None else out.sumw2.cpu().numpy(), "cfg": cfg}
    if per_event:
        res.update(pass_=out.ev_pass.cpu().numpy(), nlep=out.ev_nlep.cpu().numpy(), njet=out.ev_njet.cpu().numpy(),
                   nb=out.ev_nb.cpu().numpy(), idx=out.ev_idx.cpu().numpy(), vars=out.ev_vars.cpu().numpy())
        res["pass"] = res.pop("pass_")
    return res


def check(H, orc, batch, shifts, per_event=True, jec=None):
    o = orc.run_chain(batch, synth.CUTS, synth.HIST_SPECS, shifts, jec=jec)
    g = run_gpu(H, batch, shifts, per_event=per_event, jec=jec)
    stats = {}
    if per_event:
        stats.update(CC.compare_per_event(g, o, shifts))
    stats.update(CC.compare_hists(g["counts"], g["sumw"], g["sumw2"], o, batch.weight, o["nbins"], o["edges"]))
    assert H.device_error() == 0
    return stats


def test_chain_golden_events(H, orc):
    with open(GOLDEN) as f:
        g = json.load(f)
    batch = synth.hand_batch(g["events"])
    check(H, orc, batch, g["shifts"])


def test_chain_plain_100k_int32(H, orc):
    batch = synth.generate(100_000, 1, offset_dtype=np.int32)
    stats = check(H, orc, batch, [0])
    print("plain_100k", stats)


@pytest.mark.parametrize("fmt", ["f32", "bf16", "f16"])
def test_chain_variations(H, orc, fmt):
    batch = synth.generate(30_011, 3)
    if fmt != "f32":
        batch = synth.reduced_precision(batch, fmt)
    stats = check(H, orc, batch, synth.variation_shifts(7))
    print(fmt, stats)


def test_chain_many_jets_and_leptons(H, orc):
    # dense events (Poisson 12 jets, 2.5 muons): tiles overflow the stage
    # capacity sometimes, more leptons per event
    batch = synth.generate(20_011, 5, lam_jet=12.0, lam_mu=2.5)
    check(H, orc, batch, [0, 4, -4])


def test_chain_nan_phi_jets(H, orc):
    """Jets with a NaN phi are selected (NaN is not closer than the Delta R
    cut) and make the ranking value of every triplet that contains them NaN;
    a NaN value never wins, so events whose triplets are all NaN-ranked have
    no trijet on either side (per event and in the histograms)."""
    batch = synth.generate(20_011, 7)
    phi = batch.cols["jet_phi"].copy()
    phi[np.random.default_rng(8).random(len(phi)) < 0.2] = np.nan
    cols = dict(batch.cols)
    cols["jet_phi"] = phi
    nb = synth.EventBatch(n_events=batch.n_events, jet_offsets=batch.jet_offsets, mu_offsets=batch.mu_offsets,
                          el_offsets=batch.el_offsets, cols=cols, weight=batch.weight, seed=batch.seed)
    check(H, orc, nb, [0, 3])
    o = orc.run_chain(nb, synth.CUTS, synth.HIST_SPECS, [0, 3])
    assert ((o["pass"] == 1) & (o["njet"] >= 3) & (o["idx"][:, 2] < 0)).sum() > 0   # the case occurs
    # the per-operation kernel on the same jets
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    om, _opt, oidx, _gap = orc.max_pt_trijet(cols["jet_pt"], cols["jet_eta"], phi, cols["jet_mass"], batch.jet_offsets)
    gm, _gpt, gidx = H.hepacc_max_pt_trijet(d(cols["jet_pt"]), d(cols["jet_eta"]), d(phi), d(cols["jet_mass"]),
                                            d(batch.jet_offsets))
    torch.cuda.synchronize()
    gidx = gidx.cpu().numpy()
    np.testing.assert_array_equal(gidx[:, 0] < 0, oidx[:, 0] < 0)
    assert (np.isnan(gm.cpu().numpy()) == np.isnan(om)).all()
    assert H.device_error() == 0


def test_chain_histograms_without_per_event_outputs(H, orc):
    # the launch the benchmark times (no per-event outputs) against the oracle
    batch = synth.generate(200_003, 7)
    for shifts in ([0], synth.variation_shifts(21)):
        o = orc.run_chain(batch, synth.CUTS, synth.HIST_SPECS, shifts)
        g = run_gpu(H, batch, shifts, per_event=False)
        CC.compare_hists(g["counts"], g["sumw"], g["sumw2"], o, batch.weight, o["nbins"], o["edges"])
    assert H.device_error() == 0


def test_chain_accumulates(H, orc):
    batch = synth.generate(10_000, 8)
    cfg = H.ChainConfig(synth.CUTS, synth.HIST_SPECS, [1.0])
    db = H.DeviceBatch.from_host(batch)
    out = H.ChainOutputs(cfg, batch.n_events)
    H.hepacc_run_chain(db, cfg, out)
    H.hepacc_run_chain(db, cfg, out)
    o = orc.run_chain(batch, synth.CUTS, synth.HIST_SPECS, [0], per_event=False)
    np.testing.assert_array_equal(out.counts.cpu().numpy().view(np.uint64), 2 * o["counts"])


def test_chain_empty_and_tiny(H, orc):
    for n in (0, 1, 31, 33):
        batch = synth.generate(n, 9)
        if n == 0:
            cfg = H.ChainConfig(synth.CUTS, synth.HIST_SPECS, [1.0])
            out = H.ChainOutputs(cfg, 0)
            H.hepacc_run_chain(H.DeviceBatch.from_host(batch), cfg, out)
            assert int(out.counts.sum()) == 0
        else:
            check(H, orc, batch, [0, 2])


@pytest.mark.parametrize("fmt", ["f32", "bf16"])
def test_per_op_chain_matches_oracle(H, orc, fmt):
    from paper_1906_06242_gb300 import perop
    batch = synth.generate(50_021, 12)
    if fmt != "f32":
        batch = synth.reduced_precision(batch, fmt)
    shifts = [0, 1, -1]
    o = orc.run_chain(batch, synth.CUTS, synth.HIST_SPECS, shifts)
    cfg = H.ChainConfig(synth.CUTS, synth.HIST_SPECS, [np.float32(1.0 + 0.01 * k) for k in shifts])
    db = H.DeviceBatch.from_host(batch)
    out = H.ChainOutputs(cfg, batch.n_events)
    perop.run_chain_per_op(db, cfg, out)
    torch.cuda.synchronize()
    CC.compare_hists(out.counts.cpu().numpy().view(np.uint64), out.sumw.cpu().numpy(), out.sumw2.cpu().numpy(),
                     o, batch.weight, o["nbins"], o["edges"])
    assert H.device_error() == 0


def test_chain_full_size_plain_10m(H, orc):
    # the benchmark's workload and launch: 10M events, FP32, int64 offsets,
    # no per-event outputs; every histogram bin against the oracle's
    batch = synth.generate(10_000_000, 1)
    o = orc.run_chain(batch, synth.CUTS, synth.HIST_SPECS, [0])
    g = run_gpu(H, batch, [0], per_event=False)
    stats = CC.compare_hists(g["counts"], g["sumw"], g["sumw2"], o, batch.weight, o["nbins"], o["edges"])
    print("plain_10m", stats)
    assert H.device_error() == 0


def test_chain_too_dense_for_any_stage(H, orc):
    # 60 jets and 6 muons per event: a stage sized for that density does not
    # fit in shared memory; the call lays out smaller stages and the tiles
    # that do not fit them are read from global memory (per-event outputs
    # and histograms, against the oracle)
    batch = synth.generate(1_501, 91, lam_jet=60.0, lam_mu=6.0)
    check(H, orc, batch, [0, 5])



@pytest.mark.parametrize("fmt", ["f32", "bf16"])
def test_chain_jet_energy_corrections(H, orc, fmt):
    # variations that correct each jet's pt by an (eta, pt) table
    # (Section IV), per event and per histogram against the oracle
    batch = synth.generate(40_013, 17, offset_dtype=np.int32)
    if fmt != "f32":
        batch = synth.reduced_precision(batch, fmt)
    shifts = synth.variation_shifts(5)
    print(fmt, check(H, orc, batch, shifts, jec=synth.jec_tables(shifts)))


@pytest.mark.parametrize("lam_jet,n", [(4.0, 60_013), (60.0, 1_201)])
def test_chain_jet_energy_corrections_histograms_only(H, orc, lam_jet, n):
    # without per-event outputs only the pairs whose corrected jets pass are
    # queued; events of more than 64 jets take the unbuffered path
    batch = synth.generate(n, 29, lam_jet=lam_jet)
    shifts = synth.variation_shifts(9)
    print(lam_jet, check(H, orc, batch, shifts, per_event=False, jec=synth.jec_tables(shifts)))


def test_chain_constant_corrections_equal_scales(H):
    # a table whose every entry is float32(1 + 0.01 k) is the scale variation k
    batch = synth.generate(30_007, 19)
    shifts = [0, 2, -2]
    t = synth.jec_tables(shifts)
    t["contents"] = np.stack([np.full_like(t["contents"][0], np.float32(1.0 + 0.01 * k)) for k in shifts])
    a = run_gpu(H, batch, shifts, jec=t)
    b = run_gpu(H, batch, shifts)
    for key in ("pass", "njet", "nb", "idx", "counts"):
        np.testing.assert_array_equal(a[key], b[key], err_msg=key)
    # the two are separate kernel builds: the variables computed in a fixed
    # order of binary32 operations agree bit for bit, the masses and |sum pT|
    # (whose products the compiler may fuse differently) to the mass tolerance
    loose = list(CC.MASS_VARS) + [CC.PTJJJ]
    exact = [h for h in range(synth.N_HIST) if h not in loose]
    np.testing.assert_array_equal(a["vars"][:, exact], b["vars"][:, exact])
    np.testing.assert_allclose(a["vars"][:, loose], b["vars"][:, loose], rtol=CC.REL_MASS, atol=0)
    assert H.device_error() == 0
