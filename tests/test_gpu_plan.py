"""GPU parity of batched chain plans (hepacc_plan_*) against the oracle: many
samples of uneven size, each with its jet-pt variations, in one persistent
launch (the Section IV benchmark runs the chain over such a sample set),
for every histogram placement, with and without CUDA-graph replay."""
import numpy as np
import pytest
import torch

from paper_1906_06242_gb300 import synth
from tests import chain_check as CC

pytestmark = pytest.mark.gpu

BLOCK, CL8, CL16, GLOBAL = 4, 8, 16, 32


@pytest.fixture(scope="module")
def H():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1906_06242_gb300 import hepacc
    hepacc.load()
    return hepacc


def config(H, shifts):
    return H.ChainConfig(synth.CUTS, synth.HIST_SPECS, [np.float32(1.0 + 0.01 * k) for k in shifts])


def run_plan(H, samples, shifts, flags, runs=1):
    cfg = config(H, shifts)
    dbs = [H.DeviceBatch.from_host(s) for s in samples]
    outs = [H.ChainOutputs(cfg, s.n_events) for s in samples]
    plan = H.hepacc_plan_create(cfg, dbs, outs, flags=flags)
    for _ in range(runs):
        plan.run()
    torch.cuda.synchronize()
    desc = plan.describe()
    plan.close()
    assert H.device_error() == 0
    res = [(o.counts.cpu().numpy().view(np.uint64), o.sumw.cpu().numpy(), o.sumw2.cpu().numpy()) for o in outs]
    return res, desc


def check_samples(orc, samples, shifts, res, runs=1):
    for s, (c, w, w2) in zip(samples, res):
        o = orc.run_chain(s, synth.CUTS, synth.HIST_SPECS, shifts)
        if runs == 1:
            CC.compare_hists(c, w, w2, o, s.weight, o["nbins"], o["edges"])
        else:
            # accumulation: every run adds the same integer counts
            assert (c % runs == 0).all()
            CC.compare_hists(c // runs, w / runs, w2 / runs, o, s.weight, o["nbins"], o["edges"])


@pytest.mark.parametrize("fmt", ["f32", "bf16", "f16"])
def test_plan_12_samples_21_variations(H, orc, fmt):
    # the benchmark's sample set scaled down (sizes 1k .. 54k events)
    samples = synth.batched_samples(12, size_scale=0.005 if fmt == "bf16" else 0.002)
    if fmt != "f32":
        samples = [synth.reduced_precision(s, fmt) for s in samples]
    shifts = synth.variation_shifts(21)
    res, desc = run_plan(H, samples, shifts, flags=1 | 2)
    print(fmt, desc)
    assert desc["graph"] and desc["launches"] == 1
    check_samples(orc, samples, shifts, res)


@pytest.mark.parametrize("placement", [BLOCK, CL8, CL16, GLOBAL])
def test_plan_placements_one_variation(H, orc, placement):
    samples = [synth.generate(n, 40 + i, offset_dtype=np.int64) for i, n in enumerate([9_001, 0, 20_011, 313, 1])]
    res, desc = run_plan(H, samples, [0], flags=placement)
    want = {BLOCK: "block", CL8: "cluster", CL16: "cluster", GLOBAL: "global"}[placement]
    assert desc["chosen"]["histograms"] == want
    if placement in (CL8, CL16):
        assert desc["chosen"]["cluster"] == placement
    check_samples(orc, samples, [0], res)


@pytest.mark.parametrize("placement", [CL8, CL16, GLOBAL])
def test_plan_placements_seven_variations(H, orc, placement):
    samples = [synth.reduced_precision(synth.generate(n, 50 + i, offset_dtype=np.int64), "bf16")
               for i, n in enumerate([12_007, 3_001, 700])]
    shifts = synth.variation_shifts(7)
    res, desc = run_plan(H, samples, shifts, flags=placement | 2, runs=2)
    check_samples(orc, samples, shifts, res, runs=2)


def test_plan_block_placement_too_large_is_rejected(H):
    # 21 variations x 2040 bins x 20 bytes do not fit in one block's shared memory
    samples = [synth.generate(100, 1, offset_dtype=np.int64)]
    with pytest.raises(H.HepaccError):
        run_plan(H, samples, synth.variation_shifts(21), flags=BLOCK)


def test_plan_more_than_16_samples(H, orc):
    samples = [synth.generate(n, 60 + i, offset_dtype=np.int64) for i, n in enumerate(range(500, 500 + 37 * 20, 37))]
    shifts = synth.variation_shifts(3)
    res, desc = run_plan(H, samples, shifts, flags=1 | 2)
    assert desc["launches"] == 2
    check_samples(orc, samples, shifts, res)


def test_plan_dense_events(H, orc):
    # tiles that overflow the stage capacity are read from global memory
    samples = [synth.generate(8_011, 70, lam_jet=12.0, lam_mu=2.5, offset_dtype=np.int64),
               synth.generate(5_003, 71, offset_dtype=np.int64)]
    shifts = synth.variation_shifts(5)
    res, _ = run_plan(H, samples, shifts, flags=CL16)
    check_samples(orc, samples, shifts, res)


def test_plan_matches_single_sample_calls(H):
    # a plan and one hepacc_run_chain per sample give the same counts
    samples = [synth.generate(n, 80 + i, offset_dtype=np.int64) for i, n in enumerate([30_000, 7_000])]
    shifts = synth.variation_shifts(9)
    res, _ = run_plan(H, samples, shifts, flags=1)
    cfg = config(H, shifts)
    for s, (c, w, _) in zip(samples, res):
        db = H.DeviceBatch.from_host(s)
        out = H.ChainOutputs(cfg, s.n_events)
        H.hepacc_run_chain(db, cfg, out)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.counts.cpu().numpy().view(np.uint64), c)
        np.testing.assert_allclose(out.sumw.cpu().numpy(), w, rtol=1e-12, atol=1e-9)


def test_plan_rejects_bad_samples(H):
    cfg = config(H, [0])
    s = synth.generate(100, 1, offset_dtype=np.int64)
    db = H.DeviceBatch.from_host(s)
    with pytest.raises(H.HepaccError):   # per-event outputs
        H.hepacc_plan_create(cfg, [db], [H.ChainOutputs(cfg, 100, per_event=True)])
    s32 = synth.generate(100, 1, offset_dtype=np.int32)
    with pytest.raises(H.HepaccError):   # int32 offsets
        H.hepacc_plan_create(cfg, [H.DeviceBatch.from_host(s32)], [H.ChainOutputs(cfg, 100)])
    sb = synth.reduced_precision(s, "bf16")
    with pytest.raises(H.HepaccError):   # mixed column types
        H.hepacc_plan_create(cfg, [db, H.DeviceBatch.from_host(sb)], [H.ChainOutputs(cfg, 100)] * 2)
    with pytest.raises(H.HepaccError):   # unknown flag
        H.hepacc_plan_create(cfg, [db], [H.ChainOutputs(cfg, 100)], flags=1 << 10)
    assert H.device_error() == 0


@pytest.mark.parametrize("flags", [1 | 2, GLOBAL | 2, CL16 | 2, GLOBAL])
def test_plan_reused_over_batches(H, orc, flags):
    # one plan (tuned and captured on the first set) run over three sets of
    # the same number of samples and column types, with other event counts
    # and contents (Section II: the cache is processed batch after batch);
    # each run equals the oracle on its own set
    shifts = synth.variation_shifts(5)
    cfg = config(H, shifts)
    sets = [[synth.generate(n, 300 + 10 * b + i, offset_dtype=np.int64) for i, n in enumerate(sizes)]
            for b, sizes in enumerate([(20_011, 3_001, 512), (4_003, 25_013, 1), (9_001, 0, 17_077)])]
    dbs = [[H.DeviceBatch.from_host(s) for s in st] for st in sets]
    outs = [[H.ChainOutputs(cfg, s.n_events) for s in st] for st in sets]
    plan = H.hepacc_plan_create(cfg, dbs[0], outs[0], flags=flags)
    plan.run()
    for b in (1, 2):
        plan.run_batch(dbs[b], outs[b])
    torch.cuda.synchronize()
    desc = plan.describe()
    # a batch of another sample count or column type is refused
    with pytest.raises(H.HepaccError):
        plan.run_batch(dbs[1][:2], outs[1][:2])
    bf = [H.DeviceBatch.from_host(synth.reduced_precision(s, "bf16")) for s in sets[1]]
    with pytest.raises(H.HepaccError):
        plan.run_batch(bf, outs[1])
    plan.close()
    assert H.device_error() == 0
    print(flags, desc["chosen"])
    for st, os_ in zip(sets, outs):
        res = [(o.counts.cpu().numpy().view(np.uint64), o.sumw.cpu().numpy(), o.sumw2.cpu().numpy()) for o in os_]
        check_samples(orc, st, shifts, res)



def test_plan_with_jet_energy_corrections(H, orc):
    # a plan whose variations correct jets by table lookup (compacting kernel)
    samples = [synth.generate(n, 500 + i, offset_dtype=np.int64) for i, n in enumerate([15_013, 4_001, 9_007])]
    shifts = synth.variation_shifts(7)
    jec = synth.jec_tables(shifts)
    cfg = H.ChainConfig(synth.CUTS, synth.HIST_SPECS, [np.float32(1.0 + 0.01 * k) for k in shifts], jec=jec)
    dbs = [H.DeviceBatch.from_host(s) for s in samples]
    outs = [H.ChainOutputs(cfg, s.n_events) for s in samples]
    plan = H.hepacc_plan_create(cfg, dbs, outs, flags=1 | 2)
    plan.run()
    torch.cuda.synchronize()
    assert plan.describe()["chosen"]["kernel"] == "compacting"
    plan.close()
    assert H.device_error() == 0
    for s, o in zip(samples, outs):
        ref = orc.run_chain(s, synth.CUTS, synth.HIST_SPECS, shifts, jec=jec)
        CC.compare_hists(o.counts.cpu().numpy().view(np.uint64), o.sumw.cpu().numpy(), o.sumw2.cpu().numpy(), ref,
                         s.weight, ref["nbins"], ref["edges"])


def test_plan_autotune_cache(H, orc):
    # a second autotuned plan of the same shape takes the first one's choice
    # without timing; another configuration is tuned afresh
    samples = [synth.generate(n, 700 + i, offset_dtype=np.int64) for i, n in enumerate([30_011, 8_009])]
    shifts = synth.variation_shifts(3)
    cfg = config(H, shifts)
    dbs = [H.DeviceBatch.from_host(s) for s in samples]
    flags = H.PLAN_AUTOTUNE | H.PLAN_HIST_GLOBAL
    outs_a = [H.ChainOutputs(cfg, s.n_events) for s in samples]
    a = H.hepacc_plan_create(cfg, dbs, outs_a, flags=flags)
    da = a.describe()
    outs_b = [H.ChainOutputs(cfg, s.n_events) for s in samples]
    b = H.hepacc_plan_create(cfg, dbs, outs_b, flags=flags)
    db_ = b.describe()
    assert db_["tuned_from_cache"] and db_["tried"] == []
    assert db_["chosen"] == da["chosen"]
    b.run()
    torch.cuda.synchronize()
    cfg2 = config(H, synth.variation_shifts(5))
    c = H.hepacc_plan_create(cfg2, dbs, [H.ChainOutputs(cfg2, s.n_events) for s in samples], flags=flags)
    assert not c.describe()["tuned_from_cache"]
    for p in (a, b, c):
        p.close()
    assert H.device_error() == 0
    res = [(o.counts.cpu().numpy().view(np.uint64), o.sumw.cpu().numpy(), o.sumw2.cpu().numpy()) for o in outs_b]
    check_samples(orc, samples, shifts, res)
