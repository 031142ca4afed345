"""The oracle on large batches for the full-size GPU tests: event ranges of
the batch run by the unchanged oracle in spawned worker processes (started
with spawn, so that no worker inherits a CUDA context), each returning its
histograms and its part of the comparison allowance (tests/chain_check.py),
which add up over ranges."""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np

from paper_1906_06242_gb300 import streaming, synth


def _shard(arrays, n_events, shifts, kin_fmt, btag_fmt):
    from oracle import oracle
    from tests import chain_check as CC
    oracle.build()
    b = synth.EventBatch(n_events=n_events, jet_offsets=arrays["off_jet"], mu_offsets=arrays["off_mu"],
                         el_offsets=arrays["off_el"], cols=arrays, weight=arrays["weight"])
    o = oracle.run_chain(b, synth.CUTS, synth.HIST_SPECS, shifts, per_event=True, kin_fmt=kin_fmt, btag_fmt=btag_fmt)
    allow = CC.hist_allowance(o, b.weight, o["nbins"], o["edges"])
    return o["counts"], o["sumw"], o["sumw2"], allow, o["nbins"], o["edges"]


def oracle_hists(batch, shifts, events_per_shard=200_000, workers=None):
    """(counts, sumw, sumw2, allowance, nbins, edges) of the oracle over the
    whole batch."""
    workers = workers or max(1, min(32, os.cpu_count() or 1))
    n = batch.n_events
    bounds = list(range(0, n, events_per_shard)) + [n]
    kin_fmt = getattr(batch, "kin_fmt", None)
    btag_fmt = getattr(batch, "btag_fmt", None)
    tot = None
    from tests import chain_check as CC
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        futs = [ex.submit(_shard, streaming.host_range(batch, a, z), z - a, list(shifts), kin_fmt, btag_fmt)
                for a, z in zip(bounds[:-1], bounds[1:]) if z > a]
        for f in futs:
            c, w, w2, allow, nbins, edges = f.result()
            if tot is None:
                tot = [c.astype(np.uint64), w.copy(), w2.copy(), allow, nbins, edges]
            else:
                tot[0] += c.astype(np.uint64)
                tot[1] += w
                tot[2] += w2
                tot[3] = CC.add_allowances(tot[3], allow)
    return tuple(tot)
