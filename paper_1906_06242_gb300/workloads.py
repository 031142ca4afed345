"""Run one workload a few times (for profilers and quick timings).

  python -m paper_1906_06242_gb300.workloads plain --events 2000000 --runs 3
  python -m paper_1906_06242_gb300.workloads plain --events 2000000 --kin bf16
  python -m paper_1906_06242_gb300.workloads batched --scale 0.02 --runs 3
  python -m paper_1906_06242_gb300.workloads op --op sum_in_offsets --events 2000000

``plain``: one sample of the benchmark generator (int64 offsets), one
variation, hepacc_run_chain. ``batched``: the 12-sample set with 21 jet-pt
variations as one plan (no autotuning, no graph, so that every launch is a
plain kernel launch); ``--placement`` picks the histogram placement.
``op``: one per-operation kernel on the jets of the plain sample (sum, max,
get, select, scale, mask_deltar, fill_histogram, max_pt_trijet,
trijet_closest_mass, fill_histogram_nd over jet pt and eta). One untimed
run, then ``--runs`` timed runs; prints the mean device time per run.
"""
from __future__ import annotations

import argparse
import sys

import numpy as np
import torch

from . import hepacc as H
from . import synth

PLACEMENTS = {"block": 4, "cluster8": 8, "cluster16": 16, "global": 32}


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("workload", choices=["plain", "batched", "op"])
    p.add_argument("--op", default="sum_in_offsets")
    p.add_argument("--events", type=int, default=2_000_000)
    p.add_argument("--kin", choices=["f32", "bf16", "f16"], default="f32")
    p.add_argument("--scale", type=float, default=0.02)
    p.add_argument("--variations", type=int, default=21)
    p.add_argument("--placement", choices=sorted(PLACEMENTS), default="global")
    p.add_argument("--runs", type=int, default=3)
    a = p.parse_args(argv)
    H.load()
    if a.workload == "op":
        batch = synth.generate(a.events, 1)
        db = H.DeviceBatch.from_host(batch)
        C, jo, mo = db.cols, db.offsets["jet"], db.offsets["mu"]
        n = batch.n_events
        f = torch.zeros(n, dtype=torch.float32, device="cuda")
        i = torch.zeros(n, dtype=torch.int32, device="cuda")
        i3 = torch.zeros((n, 3), dtype=torch.int32, device="cuda")
        mj = torch.empty(C["jet_pt"].numel(), dtype=torch.uint8, device="cuda")
        mm = torch.ones(C["mu_pt"].numel(), dtype=torch.uint8, device="cuda")
        ej = torch.empty(C["jet_pt"].numel(), dtype=torch.float32, device="cuda")
        edges = torch.from_numpy(H.hist_edges(20.0, 500.0, 100)).cuda()
        hc = torch.zeros(102, dtype=torch.int64, device="cuda")
        hw = torch.zeros(102, dtype=torch.float64, device="cuda")
        edges_eta = torch.from_numpy(H.hist_edges(-2.5, 2.5, 30)).cuda()
        hc2 = torch.zeros((102, 32), dtype=torch.int64, device="cuda")
        hw2 = torch.zeros((102, 32), dtype=torch.float64, device="cuda")
        ops = {
            "sum_in_offsets": lambda: H.hepacc_sum_in_offsets(C["jet_pt"], jo, out=f),
            "max_in_offsets": lambda: H.hepacc_max_in_offsets(C["jet_pt"], jo, out=f, arg=i),
            "get_in_offsets": lambda: H.hepacc_get_in_offsets(C["jet_pt"], jo, 0, out=f, index=i),
            "select_range": lambda: H.hepacc_select_range(C["jet_pt"], lo=30.0, mask_out=mj),
            "scale": lambda: H.hepacc_scale(C["jet_pt"], 1.01, out=ej),
            "mask_deltar": lambda: H.hepacc_mask_deltar(C["jet_eta"], C["jet_phi"], jo, C["mu_eta"], C["mu_phi"], mo,
                                                        mask2=mm, mask1_out=mj),
            "fill_histogram": lambda: H.hepacc_fill_histogram(C["jet_pt"], edges, counts=hc, sumw=hw, sumw2=None,
                                                              with_sumw2=False),
            "max_pt_trijet": lambda: H.hepacc_max_pt_trijet(C["jet_pt"], C["jet_eta"], C["jet_phi"], C["jet_mass"], jo,
                                                            out_mass=f, out_idx3=i3),
            "trijet_closest_mass": lambda: H.hepacc_trijet_closest_mass(C["jet_pt"], C["jet_eta"], C["jet_phi"],
                                                                        C["jet_mass"], jo, out_mass=f, out_idx3=i3),
            "fill_histogram_nd": lambda: H.hepacc_fill_histogram_nd([C["jet_pt"], C["jet_eta"]], [edges, edges_eta],
                                                                    counts=hc2, sumw=hw2, with_sumw2=False),
        }
        run = ops[a.op]
    elif a.workload == "plain":
        batch = synth.generate(a.events, 1)
        if a.kin != "f32":
            batch = synth.reduced_precision(batch, a.kin)
        cfg = H.ChainConfig(synth.CUTS, synth.HIST_SPECS, [1.0])
        db = H.DeviceBatch.from_host(batch)
        out = H.ChainOutputs(cfg, batch.n_events)
        st = (db.c_struct(), cfg.c_struct(), out.c_struct())

        def run():
            H.hepacc_run_chain(db, cfg, out, _structs=st)
        n = batch.n_events
    else:
        samples = synth.batched_samples(12, size_scale=a.scale)
        if a.kin != "f32":
            samples = [synth.reduced_precision(s, a.kin) for s in samples]
        shifts = synth.variation_shifts(a.variations)
        cfg = H.ChainConfig(synth.CUTS, synth.HIST_SPECS, [np.float32(1.0 + 0.01 * k) for k in shifts])
        dbs = [H.DeviceBatch.from_host(s) for s in samples]
        outs = [H.ChainOutputs(cfg, s.n_events) for s in samples]
        plan = H.hepacc_plan_create(cfg, dbs, outs, flags=PLACEMENTS[a.placement])
        run = plan.run
        n = sum(s.n_events for s in samples)
    run()   # first launch: module load and launch set-up
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(a.runs):
        run()
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / max(1, a.runs)
    print(f"{a.workload} events={n} ms_per_run={ms:.3f} events_per_s={n / (ms * 1e-3):.4g} "
          f"device_error={H.device_error()}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
