"""Full-size parity of the benchmarked forms: the sizes and launch
configurations bench.py times, against the oracle run in spawned worker
processes over event ranges (tests/oracle_pool.py). Histograms only (the
per-event outputs of tens of millions of events are not kept): counts exact
except for the net flow across bin edges within the mass tolerance, weighted
sums to 1e-9 relative (tests/chain_check.py)."""
import numpy as np
import pytest
import torch

from paper_1906_06242_gb300 import streaming, synth
from tests import chain_check as CC
from tests.oracle_pool import oracle_hists

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1906_06242_gb300 import hepacc
    hepacc.load()
    return hepacc


def gpu_hists(out):
    torch.cuda.synchronize()
    return (out.counts.cpu().numpy().view(np.uint64), out.sumw.cpu().numpy(),
            None if out.sumw2 is None else out.sumw2.cpu().numpy())


def check_against_oracle(batch, shifts, g):
    c, w, w2, allow, nbins, _ = oracle_hists(batch, shifts)
    return CC.check_hists(g[0], g[1], g[2], c, w, w2, allow, nbins)


@pytest.fixture(scope="module")
def plain10m():
    w = synth.WORKLOADS["plain_10m"]
    return synth.generate(w["n_events"], w["seed"], offset_dtype=w["offset_dtype"])


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_fullsize_half_precision_10m(H, plain10m, fmt):
    # the 10M-event set with pt/eta/phi/mass in BF16 or FP16 and btag FP16,
    # as the benchmark's fused_bf16 / fused_f16 forms run it
    b = synth.reduced_precision(plain10m, fmt)
    cfg = H.ChainConfig(synth.CUTS, synth.HIST_SPECS, [1.0])
    out = H.ChainOutputs(cfg, b.n_events)
    H.hepacc_run_chain(H.DeviceBatch.from_host(b), cfg, out)
    g = gpu_hists(out)
    assert H.device_error() == 0
    print(fmt, check_against_oracle(b, [0], g))


def test_fullsize_batched_plan_12x21(H):
    # the batching form: 12 uneven samples (50.04M events), 21 variations,
    # BF16 kinematics, one autotuned plan replayed as a CUDA graph
    samples = [synth.reduced_precision(s, "bf16") for s in synth.batched_samples(12, workers=12)]
    shifts = synth.variation_shifts(21)
    cfg = H.ChainConfig(synth.CUTS, synth.HIST_SPECS, [np.float32(1.0 + 0.01 * k) for k in shifts])
    dbs = [H.DeviceBatch.from_host(s) for s in samples]
    outs = [H.ChainOutputs(cfg, s.n_events) for s in samples]
    plan = H.hepacc_plan_create(cfg, dbs, outs, flags=H.PLAN_AUTOTUNE | H.PLAN_GRAPH)
    plan.run()
    res = [gpu_hists(o) for o in outs]
    print(plan.describe()["chosen"])
    plan.close()
    del dbs
    torch.cuda.empty_cache()
    assert H.device_error() == 0
    for s, g in zip(samples, res):
        check_against_oracle(s, shifts, g)


def test_fullsize_dense_chunk_resident_and_streamed(H):
    # one 5M-event chunk of the dense scale set (Poisson 12 jets, 2.5
    # muons), resident and streamed from pinned host memory in ranges of at
    # most 2 GB and of 256 MB
    w = synth.WORKLOADS["scale_60m"]
    b = synth.generate_chunked(5_000_000, w["seed"], chunk=5_000_000, lam_jet=w["lam_jet"], lam_mu=w["lam_mu"],
                               lam_el=w["lam_el"], offset_dtype=w["offset_dtype"])
    cfg = H.ChainConfig(synth.CUTS, synth.HIST_SPECS, [1.0])
    out = H.ChainOutputs(cfg, b.n_events)
    H.hepacc_run_chain(H.DeviceBatch.from_host(b), cfg, out)
    resident = gpu_hists(out)
    for budget in (2 << 30, 256 << 20):
        o2 = H.ChainOutputs(cfg, b.n_events)
        sc = streaming.StreamedChain(b, cfg, o2, batch_bytes=budget)
        sc.run(torch.cuda.current_stream())
        g = gpu_hists(o2)
        np.testing.assert_array_equal(g[0], resident[0])
        del sc
    assert H.device_error() == 0
    print(check_against_oracle(b, [0], resident))
