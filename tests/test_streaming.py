"""Streaming the chain from host memory: the range split (host logic, CPU)
and the streamed result against the resident run and the oracle (GPU)."""
import numpy as np
import pytest

from paper_1906_06242_gb300 import streaming, synth
from tests import chain_check as CC


def test_event_bytes_add_up():
    b = synth.generate(5_000, 3, offset_dtype=np.int64)
    per = streaming.event_bytes(b)
    jets = int(b.jet_offsets[-1]); mus = int(b.mu_offsets[-1]); els = int(b.el_offsets[-1])
    # offsets 3 x 8 B + weight 4 B per event; jets 5 x 4 B; leptons 4 x 4 B + 1 B
    assert per.sum() == b.n_events * (24 + 4) + jets * 20 + (mus + els) * 17


@pytest.mark.parametrize("budget", [1, 2_000, 50_000, 10 ** 12])
def test_split_ranges_cover_and_respect_budget(budget):
    b = synth.generate(3_001, 4, lam_jet=12.0, offset_dtype=np.int64)
    per = streaming.event_bytes(b)
    rs = streaming.split_ranges(b, budget)
    assert rs[0][0] == 0 and rs[-1][1] == b.n_events
    for (a0, b0), (a1, _) in zip(rs, rs[1:]):
        assert b0 == a1 and b0 > a0
    for a, z in rs:
        assert per[a:z].sum() <= budget or z - a == 1
        if z < b.n_events:   # greedy: the next event would not have fitted
            assert per[a:z + 1].sum() > budget


def test_split_ranges_empty_batch():
    assert streaming.split_ranges(synth.generate(0, 1), 1000) == []


def test_host_range_rebases_offsets():
    b = synth.generate(2_000, 5, offset_dtype=np.int32)
    a, z = 700, 1_300
    r = streaming.host_range(b, a, z)
    for coll in ("jet", "mu", "el"):
        off = b.offsets[coll]
        ro = r["off_" + coll]
        assert ro.dtype == off.dtype and ro[0] == 0
        np.testing.assert_array_equal(ro, off[a:z + 1] - off[a])
    np.testing.assert_array_equal(r["jet_pt"], b.cols["jet_pt"][b.jet_offsets[a]:b.jet_offsets[z]])
    np.testing.assert_array_equal(r["el_tight"], b.cols["el_tight"][b.el_offsets[a]:b.el_offsets[z]])
    np.testing.assert_array_equal(r["weight"], b.weight[a:z])


@pytest.mark.gpu
@pytest.mark.parametrize("fmt", ["f32", "bf16"])
def test_streamed_equals_resident_and_oracle(orc, fmt):
    import torch
    from paper_1906_06242_gb300 import hepacc as H
    assert torch.cuda.is_available()
    b = synth.generate_chunked(60_000, 5, chunk=25_000, lam_jet=12.0, lam_mu=2.5, offset_dtype=np.int64)
    if fmt != "f32":
        b = synth.reduced_precision(b, fmt)
    shifts = [0, 1, -1]
    cfg = H.ChainConfig(synth.CUTS, synth.HIST_SPECS, [np.float32(1.0 + 0.01 * k) for k in shifts])
    resident = H.ChainOutputs(cfg, b.n_events)
    H.hepacc_run_chain(H.DeviceBatch.from_host(b), cfg, resident)
    out = H.ChainOutputs(cfg, b.n_events)
    sc = streaming.StreamedChain(b, cfg, out, batch_bytes=3 << 20)
    assert len(sc.ranges) >= 4
    sc.run()
    sc.run()   # a second pass reuses the buffers and adds the same again
    torch.cuda.synchronize()
    assert H.device_error() == 0
    np.testing.assert_array_equal(out.counts.cpu().numpy(), 2 * resident.counts.cpu().numpy())
    np.testing.assert_allclose(out.sumw.cpu().numpy(), 2 * resident.sumw.cpu().numpy(), rtol=1e-12, atol=1e-9)
    copy_ms, chain_ms = sc.run_serial()   # the measurement pass adds the same once more
    assert copy_ms > 0 and chain_ms > 0
    np.testing.assert_array_equal(out.counts.cpu().numpy(), 3 * resident.counts.cpu().numpy())
    o = orc.run_chain(b, synth.CUTS, synth.HIST_SPECS, shifts)
    CC.compare_hists(out.counts.cpu().numpy().view(np.uint64) // 3, out.sumw.cpu().numpy() / 3,
                     out.sumw2.cpu().numpy() / 3, o, b.weight, o["nbins"], o["edges"])
