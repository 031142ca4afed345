"""The sharded chain on the device: a batch split into K contiguous event
ranges (shard.shard_device_batch: sliced offsets, shared columns), each run
by hepacc_run_chain into its own outputs, the outputs summed on the host (the
one exchange of the multi-GPU chain, here without a collective). Counts must
equal the unsharded run bit for bit, weighted sums to 1e-9, and both the
oracle."""
import numpy as np
import pytest
import torch

from paper_1906_06242_gb300 import shard, synth
from tests import chain_check as CC

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1906_06242_gb300 import hepacc
    hepacc.load()
    return hepacc


@pytest.mark.parametrize("fmt,off", [("f32", np.int64), ("bf16", np.int64), ("f32", np.int32)])
def test_device_shards_add_up(H, orc, fmt, off):
    b = synth.generate(90_017, 33, offset_dtype=off)
    if fmt != "f32":
        b = synth.reduced_precision(b, fmt)
    shifts = [0, 2, -2]
    cfg = H.ChainConfig(synth.CUTS, synth.HIST_SPECS, [np.float32(1.0 + 0.01 * k) for k in shifts])
    db = H.DeviceBatch.from_host(b)
    whole = H.ChainOutputs(cfg, b.n_events)
    H.hepacc_run_chain(db, cfg, whole)
    o = orc.run_chain(b, synth.CUTS, synth.HIST_SPECS, shifts)
    for k in (2, 3, 8):
        parts = []
        for r in range(k):
            sb = shard.shard_device_batch(db, r, k)
            out = H.ChainOutputs(cfg, sb.n_events)
            H.hepacc_run_chain(sb, cfg, out)
            parts.append(out)
        torch.cuda.synchronize()
        counts = sum(p.counts.cpu().numpy().view(np.uint64) for p in parts)
        sumw = sum(p.sumw.cpu().numpy() for p in parts)
        sumw2 = sum(p.sumw2.cpu().numpy() for p in parts)
        np.testing.assert_array_equal(counts, whole.counts.cpu().numpy().view(np.uint64))
        ref = whole.sumw.cpu().numpy()
        assert (np.abs(sumw - ref) <= 1e-9 * np.maximum(np.abs(ref), 1.0)).all()
        CC.compare_hists(counts, sumw, sumw2, o, b.weight, o["nbins"], o["edges"])
    assert H.device_error() == 0
