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


def short_columns(H, batch, coll="jet", cut=16):
    """Device batch whose `coll` columns are views 16 elements shorter than
    offsets[n] (the views end inside the full tensors, so nothing outside
    an allocation is ever addressable)."""
    db = H.DeviceBatch.from_host(batch)
    prefix = {"jet": "jet_", "mu": "mu_", "el": "el_"}[coll]
    cols = {k: (v[:-cut] if k.startswith(prefix) else v) for k, v in db.cols.items()}
    return H.DeviceBatch(db.n_events, db.offsets, cols, db.weight, objects=db.objects())


def test_plan_validate_content_length(H):
    # offsets[n] beyond a collection's content length is rejected before
    # the chain runs (the check compares with the length in the batch)
    b = synth.generate(4_000, 19, offset_dtype=np.int64)
    cfg = H.ChainConfig(synth.CUTS, synth.HIST_SPECS, [1.0])
    for coll in ("jet", "mu", "el"):
        with pytest.raises(H.HepaccError) as ei:
            H.hepacc_plan_create(cfg, [short_columns(H, b, coll)], [H.ChainOutputs(cfg, 4_000)],
                                 flags=H.PLAN_VALIDATE | H.PLAN_HIST_GLOBAL)
        assert ei.value.status == DEVICE_CHECK
    assert H.device_error() == 0


CHILD_LEN = r"""
import numpy as np, torch
from paper_1906_06242_gb300 import hepacc as H, synth
from tests.test_gpu_validate import short_columns
H.load()
b = synth.generate(3_000, 21, offset_dtype=np.int32)
cfg = H.ChainConfig(synth.CUTS, synth.HIST_SPECS, [1.0])
out = H.ChainOutputs(cfg, 3_000)
try:
    H.hepacc_run_chain(short_columns(H, b, "mu"), cfg, out)
    print("not rejected")
except H.HepaccError as e:
    assert e.status == 6, e
torch.cuda.synchronize()
assert int(out.counts.sum().item()) == 0, "the rejected batch reached the chain"
assert H.device_error() == 0
print("ok")
"""


def test_run_chain_debug_content_length(H):
    env = dict(os.environ, HEPACC_DEBUG="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD_LEN], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr

