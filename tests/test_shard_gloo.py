"""The sharded chain on world_size-2 gloo ranks (CPU): every rank runs the
oracle chain on its event range, the histograms are summed with
all_reduce, and the sum equals the unsharded run (counts exactly, weighted
sums up to rounding order)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1906_06242_gb300 import shard, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n, shifts, outdir):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    from oracle import oracle
    batch = synth.generate(n, 31)
    part = shard.shard_host_batch(batch, rank, world)
    o = oracle.run_chain(part, synth.CUTS, synth.HIST_SPECS, shifts, per_event=False)
    t = [torch.from_numpy(o["counts"].astype(np.int64)), torch.from_numpy(o["sumw"]), torch.from_numpy(o["sumw2"])]
    shard.allreduce_histograms(t)
    if rank == 0:
        np.save(os.path.join(outdir, "counts.npy"), t[0].numpy())
        np.save(os.path.join(outdir, "sumw.npy"), t[1].numpy())
        np.save(os.path.join(outdir, "sumw2.npy"), t[2].numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_shard_ranges_cover_events():
    for n in (0, 1, 7, 1000, 10_000_001):
        for w in (1, 2, 3, 8):
            r = [shard.shard_range(n, k, w) for k in range(w)]
            assert r[0][0] == 0 and r[-1][1] == n
            assert all(r[i][1] == r[i + 1][0] for i in range(w - 1))
            assert max(b - a for a, b in r) - min(b - a for a, b in r) <= 1


def test_sharded_chain_gloo_two_ranks(orc, tmp_path):
    n, shifts = 30_011, [0, 2, -2]
    mp.spawn(_worker, args=(2, _free_port(), n, shifts, str(tmp_path)), nprocs=2, join=True)
    full = orc.run_chain(synth.generate(n, 31), synth.CUTS, synth.HIST_SPECS, shifts, per_event=False)
    np.testing.assert_array_equal(np.load(tmp_path / "counts.npy"), full["counts"].astype(np.int64))
    np.testing.assert_allclose(np.load(tmp_path / "sumw.npy"), full["sumw"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(np.load(tmp_path / "sumw2.npy"), full["sumw2"], rtol=1e-12, atol=1e-12)
