"""Debug checks of the offsets before a chain launch (device-side check,
reported through the device error word as HEPACC_ERR_DEVICE_CHECK): plans
with the validate flag, and hepacc_run_chain with HEPACC_DEBUG set (in a
child process, since the variable is read once). A rejected batch is never
handed to the chain kernel."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_1906_06242_gb300 import synth

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DEVICE_CHECK = 6


def decreasing(batch, coll="jet", at=1234):
    """Copy of a host batch whose offsets of `coll` decrease at event `at`."""
    offs = {k: v.copy() for k, v in batch.offsets.items()}
    offs[coll][at] = offs[coll][at + 1] + 1
    return synth.EventBatch(n_events=batch.n_events, jet_offsets=offs["jet"], mu_offsets=offs["mu"],
                            el_offsets=offs["el"], cols=batch.cols, weight=batch.weight, seed=batch.seed)


@pytest.fixture(scope="module")
def H():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1906_06242_gb300 import hepacc
    hepacc.load()
    return hepacc


def test_plan_validate_flag(H):
    b = synth.generate(5_000, 9, offset_dtype=np.int64)
    cfg = H.ChainConfig(synth.CUTS, synth.HIST_SPECS, [1.0])
    for coll in ("jet", "mu", "el"):
        bad = H.DeviceBatch.from_host(decreasing(b, coll))
        with pytest.raises(H.HepaccError) as ei:
            H.hepacc_plan_create(cfg, [H.DeviceBatch.from_host(b), bad], [H.ChainOutputs(cfg, 5_000)] * 2,
                                 flags=H.PLAN_VALIDATE | H.PLAN_HIST_GLOBAL)
        assert ei.value.status == DEVICE_CHECK
    assert H.device_error() == 0   # the check consumed its bit
    # valid samples pass the check and give the unchecked plan's result
    outs = [H.ChainOutputs(cfg, 5_000) for _ in range(2)]
    for flags, out in zip((H.PLAN_VALIDATE | H.PLAN_HIST_GLOBAL, H.PLAN_HIST_GLOBAL), outs):
        p = H.hepacc_plan_create(cfg, [H.DeviceBatch.from_host(b)], [out], flags=flags)
        p.run()
        p.close()
    torch.cuda.synchronize()
    assert torch.equal(outs[0].counts, outs[1].counts)


CHILD = r"""
import numpy as np, torch
from paper_1906_06242_gb300 import hepacc as H, synth
from tests.test_gpu_validate import decreasing
H.load()
b = synth.generate(5_000, 9, offset_dtype=np.int32)
cfg = H.ChainConfig(synth.CUTS, synth.HIST_SPECS, [1.0])
out = H.ChainOutputs(cfg, 5_000)
H.hepacc_run_chain(H.DeviceBatch.from_host(b), cfg, out)
torch.cuda.synchronize()
good = out.counts.clone()
try:
    H.hepacc_run_chain(H.DeviceBatch.from_host(decreasing(b, "mu", 77)), cfg, out)
    print("not rejected")
except H.HepaccError as e:
    assert e.status == 6, e
torch.cuda.synchronize()
assert torch.equal(out.counts, good), "the rejected batch reached the chain"
assert H.device_error() == 0
print("ok")
"""


def test_run_chain_debug_env(H):
    env = dict(os.environ, HEPACC_DEBUG="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
