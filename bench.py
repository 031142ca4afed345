"""Benchmark of the fused analysis chain on GB300.

One step = one pass of the whole chain (lepton and jet selection, Delta R
masking, counts, HT, leading jets, pair and trijet masses, 20 weighted
histograms) over a resident batch of 10M synthetic events (float32 columns,
int64 offsets) in one hepacc_run_chain launch. Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun every rank runs its own batch (weak scaling, no collective in
the timed region). ``--impl reference`` times the CPU oracle on the host
cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "plain_10m"
METRIC = "events/s and HBM GB/s (% of peak) for the full chain, plain vs BF16+batched, 1 GB300"
N_EVENTS = 10_000_000

# The paper's own rates (Sections III and IV), other hardware and other
# workloads: context for the figures, not a baseline of this workload.
PAPER_CONTEXT = {
    "hardware": "Numba kernels; CPU Xeon E5-2687W v4 @ 3.00 GHz, GPU GeForce Titan X",
    "kernels_events_per_s": {"value": 1e7, "note": "order of magnitude (tens of MHz) per kernel, ~11M preloaded "
                                                     "events, GPU ~20-30x one CPU thread"},
    "delta_r_mask_events_per_s": {"cpu_1_thread": 7e6, "gpu": 7e6 * 14},
    "full_analysis_events_per_s": {"partial_systematics": {"cpu_1_thread": 50e3, "cpu_4_threads": 119e3,
                                                           "gpu": 440e3},
                                   "full_systematics": {"cpu_1_thread": 1.4e3, "cpu_4_threads": 4.0e3,
                                                        "gpu": 20e3},
                                   "note": "CMS Open Data analysis with a DNN and ~1000 histograms"},
}
N_VARIATIONS_BATCHED = 21


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="hepacc", choices=["hepacc", "reference"])
    p.add_argument("--events", type=int, default=N_EVENTS)
    p.add_argument("--no-extra", action="store_true", help="skip the secondary forms")
    p.add_argument("--batched-scale", type=float, default=1.0,
                   help="size factor of the 12-sample batched set (1.0: 0.2M to 20M events per sample)")
    p.add_argument("--dense-events", type=int, default=60_000_000,
                   help="events of the dense scale set (12 jets, 2.5 muons per event); 0 skips it")
    # profiler-target mode: run one workload a few times, print its device time
    p.add_argument("--profile", choices=["plain", "batched", "dense", "op"], default=None,
                   help="run one workload --runs times (a target for ncu) instead of the benchmark")
    p.add_argument("--op", default="sum_in_offsets", help="--profile op: the per-operation kernel")
    p.add_argument("--kin", choices=["f32", "bf16", "f16"], default="f32", help="--profile: kinematic column type")
    p.add_argument("--variations", type=int, default=1, help="--profile: jet-pt variations")
    p.add_argument("--runs", type=int, default=3, help="--profile: runs after one untimed run")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def algorithmic_bytes(batch) -> int:
    """Bytes the chain must read once: three offsets arrays, the 15 object
    columns it uses and the event weights."""
    tot = sum(a.nbytes for a in batch.offsets.values())
    for name in ("jet_pt", "jet_eta", "jet_phi", "jet_mass", "jet_btag", "mu_pt", "mu_eta", "mu_phi", "mu_iso",
                 "mu_tight", "el_pt", "el_eta", "el_phi", "el_iso", "el_tight"):
        tot += batch.cols[name].nbytes
    return tot + batch.weight.nbytes


def kernel_source_sha():
    """Hash of the chain kernel's code (comments and blank space removed, so
    that a comment edit leaves recorded counters valid)."""
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1906_06242_gb300", "csrc")
    for fn in ("chain.cu", "chain_kernel.cuh", "fused_kernel.cuh", "hepacc_tiles.cuh", "hepacc_device.cuh"):
        src = open(os.path.join(csrc, fn), encoding="utf-8").read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def profile_counters():
    """Per-event counters of the fused chain kernel, one ncu capture per
    form (profiles/counters.json; the captures and their commands are in the
    summaries beside it): DRAM bytes read + written and warp instructions
    per event. Valid only while the kernel sources hash to the recorded
    value; {} otherwise."""
    try:
        with open(os.path.join(ROOT, "profiles", "counters.json")) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return {}
    if d.get("kernel_source_sha") != kernel_source_sha():
        return {}
    return d.get("forms", {})


def issue_roofline(events, ms, form, clock_mhz):
    """Roofline of an issue-bound form: warp instructions per second (the
    events times the form's instructions per event from profile_counters)
    against the SMs' issue peak, one warp instruction per scheduler per
    cycle: SMs x 4 x the SM clock sampled under load. None without
    counters for the form."""
    import torch
    c = profile_counters().get(form)
    if not c or not ms or not clock_mhz:
        return None
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peak = sms * 4 * clock_mhz * 1e6
    achieved = events * c["warp_instructions_per_event"] / (ms * 1e-3)
    return {"bound": "issue", "achieved": achieved, "peak": peak, "unit": "warp instructions/s",
            "frac": achieved / peak, "warp_instructions_per_event": c["warp_instructions_per_event"],
            "peak_from": f"{sms} SMs x 4 schedulers x {clock_mhz:.0f} MHz (sampled)",
            "counters_from": c.get("capture")}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.t0 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        self.t0 = time.time()

    def elapsed(self):
        return time.time() - self.t0

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(batch, n_sample, shifts=(0,)):
    """The oracle, as it is, on a bounded sample of the workload (the first
    n_sample events), single-threaded on the host."""
    from oracle import oracle
    from paper_1906_06242_gb300 import synth
    n = min(n_sample, batch.n_events)
    sub = synth.EventBatch(n_events=n, jet_offsets=batch.jet_offsets[:n + 1], mu_offsets=batch.mu_offsets[:n + 1],
                           el_offsets=batch.el_offsets[:n + 1], cols=batch.cols, weight=batch.weight[:n])
    t0 = time.perf_counter()
    oracle.run_chain(sub, synth.CUTS, synth.HIST_SPECS, list(shifts), per_event=False)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "events/s", "cores": 1, "kind": "oracle",
            "sample": f"first {n} events of the {batch.n_events}-event workload, {len(shifts)} variation(s), "
                      f"{dt:.2f} s single-threaded"}


def _oracle_shard(arrays, n_events):
    """Worker: the oracle, as it is, on one shard; returns its seconds."""
    from oracle import oracle
    from paper_1906_06242_gb300 import synth
    b = synth.EventBatch(n_events=n_events, jet_offsets=arrays["off_jet"], mu_offsets=arrays["off_mu"],
                         el_offsets=arrays["off_el"], cols=arrays, weight=arrays["weight"])
    oracle.build()
    t0 = time.perf_counter()
    oracle.run_chain(b, synth.CUTS, synth.HIST_SPECS, [0], per_event=False)
    return time.perf_counter() - t0


def cpu_oracle_all_cores(batch, n_sample):
    """The same oracle on all host cores: the first n_sample events cut into
    one contiguous shard per core, each run by the unchanged oracle in its
    own spawned process (per-process histograms, as the paper's
    multithreaded CPU backend keeps per-thread ones). Rate = events / the
    slowest shard's compute time."""
    import concurrent.futures as cf
    import multiprocessing as mp
    from paper_1906_06242_gb300 import streaming
    cores = os.cpu_count() or 1
    n = min(n_sample, batch.n_events)
    bounds = [n * r // cores for r in range(cores + 1)]
    shards = [streaming.host_range(batch, bounds[r], bounds[r + 1]) for r in range(cores)]
    with cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as ex:
        times = list(ex.map(_oracle_shard, shards, [bounds[r + 1] - bounds[r] for r in range(cores)]))
    worst = max(times)
    return {"value": n / worst, "unit": "events/s", "cores": cores, "kind": "oracle, one process per core",
            "sample": f"first {n} events of the {batch.n_events}-event workload in {cores} shards, "
                      f"slowest shard {worst:.2f} s"}


def headline_config(n_events, world):
    """The headline workload's config (both arms)."""
    return {"workload": WORKLOAD, "events_per_gpu": n_events, "offsets": "int64", "columns": "float32",
            "variations": 1, "histograms": 20, "bins": 100, "l2": "inputs larger than L2 (no flush needed)",
            "parallelism": f"dp{world} (independent event shards)"}


def run_reference(args, rank, world):
    """The oracle (the reference of this method) on the headline workload:
    each step the next 300k-event window of the same 10M events, single
    threaded on the host. Rank 0 only."""
    if rank != 0:
        return
    from paper_1906_06242_gb300 import synth
    per_step = 300_000
    batch = synth.generate(args.events, 1)
    per_step = min(per_step, batch.n_events)
    from oracle import oracle
    oracle.build()
    times = []
    for i in range(args.warmup + args.steps):
        a = (i * per_step) % max(1, batch.n_events - per_step + 1)
        # events [a, a + per_step): offsets sliced, columns shared (event i
        # owns [off[i], off[i+1]) of the full columns)
        sub = synth.EventBatch(n_events=per_step, jet_offsets=batch.jet_offsets[a:a + per_step + 1],
                               mu_offsets=batch.mu_offsets[a:a + per_step + 1],
                               el_offsets=batch.el_offsets[a:a + per_step + 1], cols=batch.cols,
                               weight=batch.weight[a:a + per_step])
        t0 = time.perf_counter()
        oracle.run_chain(sub, synth.CUTS, synth.HIST_SPECS, [0], per_event=False)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = per_step * len(times) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": headline_config(batch.n_events, world),
            "cpu_baseline": {"value": value, "unit": "events/s", "cores": 1, "kind": "oracle",
                             "sample": f"per step the next {per_step}-event window of the {batch.n_events}-event "
                                       f"{WORKLOAD} workload, 1 variation, single-threaded"},
            "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_profile(args):
    """One workload, one untimed run then ``--runs`` runs, for profiler
    captures: ``plain`` (one sample of the benchmark generator, int64
    offsets, ``--events``), ``dense`` (the dense scale set's generator:
    Poisson 12 jets, 2.5 muons), ``batched`` (the 12-sample set scaled by
    ``--batched-scale`` as one plan without autotuning or graph, every
    launch a plain kernel launch), ``op`` (one per-operation kernel on the
    jets of the plain sample). Prints the mean device time per run."""
    import numpy as np
    import torch
    from paper_1906_06242_gb300 import hepacc as H
    from paper_1906_06242_gb300 import synth
    H.load()
    shifts = synth.variation_shifts(args.variations)
    cfg = H.ChainConfig(synth.CUTS, synth.HIST_SPECS, [np.float32(1.0 + 0.01 * k) for k in shifts])
    if args.profile in ("plain", "dense"):
        if args.profile == "plain":
            batch = synth.generate(args.events, 1)
        else:
            w = synth.WORKLOADS["scale_60m"]
            batch = synth.generate(args.events, w["seed"], lam_jet=w["lam_jet"], lam_mu=w["lam_mu"],
                                   lam_el=w["lam_el"], offset_dtype=w["offset_dtype"])
        if args.kin != "f32":
            batch = synth.reduced_precision(batch, args.kin)
        db = H.DeviceBatch.from_host(batch)
        out = H.ChainOutputs(cfg, batch.n_events)
        st = (db.c_struct(), cfg.c_struct(), out.c_struct())

        def run():
            H.hepacc_run_chain(db, cfg, out, _structs=st)
        n = batch.n_events
    elif args.profile == "batched":
        samples = synth.batched_samples(12, size_scale=args.batched_scale)
        if args.kin != "f32":
            samples = [synth.reduced_precision(s, args.kin) for s in samples]
        dbs = [H.DeviceBatch.from_host(s) for s in samples]
        outs = [H.ChainOutputs(cfg, s.n_events) for s in samples]
        plan = H.hepacc_plan_create(cfg, dbs, outs, flags=H.PLAN_HIST_GLOBAL)
        run = plan.run
        n = sum(s.n_events for s in samples)
    else:
        batch = synth.generate(args.events, 1)
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
            "max_pt_trijet": lambda: H.hepacc_max_pt_trijet(C["jet_pt"], C["jet_eta"], C["jet_phi"], C["jet_mass"],
                                                            jo, out_mass=f, out_idx3=i3),
            "trijet_closest_mass": lambda: H.hepacc_trijet_closest_mass(C["jet_pt"], C["jet_eta"], C["jet_phi"],
                                                                        C["jet_mass"], jo, out_mass=f, out_idx3=i3),
            "fill_histogram_nd": lambda: H.hepacc_fill_histogram_nd([C["jet_pt"], C["jet_eta"]], [edges, edges_eta],
                                                                    counts=hc2, sumw=hw2, with_sumw2=False),
        }
        run = ops[args.op]
    run()   # first run: module load and launch set-up
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(args.runs):
        run()
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / max(1, args.runs)
    print(json.dumps({"profile": args.profile, "events": int(n), "ms_per_run": ms, "device_error": H.device_error()}))


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.profile:
        return run_profile(args)
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    from paper_1906_06242_gb300 import hepacc as H
    from paper_1906_06242_gb300 import synth

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    H.load()

    batch = synth.generate(args.events, 1 + rank)
    cfg = H.ChainConfig(synth.CUTS, synth.HIST_SPECS, [1.0])
    db = H.DeviceBatch.from_host(batch)
    out = H.ChainOutputs(cfg, batch.n_events, per_event=False, sumw2=True)
    structs = (db.c_struct(), cfg.c_struct(), out.c_struct())
    stream = torch.cuda.current_stream()
    alg_bytes = algorithmic_bytes(batch)

    def step():
        H.hepacc_run_chain(db, cfg, out, stream=stream, _structs=structs)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    clock = ClockSampler(local)
    clock.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(args.steps):
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    # keep the same work running until the clock sampler has seen >= 1 s of load
    while clock.elapsed() < 1.2:
        for _ in range(50):
            step()
        torch.cuda.synchronize()
    clocks = clock.stop()
    if H.device_error():
        raise RuntimeError("the chain kernel set the device error word during the timed steps")
    total_ms = t_start.elapsed_time(t_end)
    kern_ms = [a.elapsed_time(b) for a, b in ev]
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        # the one exchange of the sharded chain: sum of the histograms
        from paper_1906_06242_gb300 import shard
        shard.allreduce_histograms([out.counts, out.sumw, out.sumw2])
    ms_per_step = total_ms / args.steps
    value = world * batch.n_events / (ms_per_step * 1e-3)
    avg_kernel_ms = sum(kern_ms) / len(kern_ms)
    hbm, peak_kind = peaks()
    achieved = alg_bytes / (avg_kernel_ms * 1e-3) / 1e9

    # end to end: pinned host columns -> device, chain, histograms -> host
    e2e = None
    if True:
        pinned = {}
        for k, a in list(batch.offsets.items()):
            pinned["off_" + k] = torch.from_numpy(a).pin_memory()
        for name in H.COLUMNS:
            pinned[name] = torch.from_numpy(batch.cols[name]).pin_memory()
        pinned["weight"] = torch.from_numpy(batch.weight).pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in pinned.values())
        res_host = [torch.empty_like(out.counts, device="cpu").pin_memory(),
                    torch.empty_like(out.sumw, device="cpu").pin_memory(),
                    torch.empty_like(out.sumw2, device="cpu").pin_memory()]
        d2h = sum(t.numel() * t.element_size() for t in res_host)
        dev_bufs = {k: torch.empty_like(t, device="cuda") for k, t in pinned.items()}
        db2 = H.DeviceBatch(batch.n_events, {k: dev_bufs["off_" + k] for k in ("jet", "mu", "el")},
                            {name: dev_bufs[name] for name in H.COLUMNS}, dev_bufs["weight"],
                            objects={k: int(v[-1] - v[0]) for k, v in batch.offsets.items()})
        out2 = H.ChainOutputs(cfg, batch.n_events, per_event=False, sumw2=True)
        s2 = (db2.c_struct(), cfg.c_struct(), out2.c_struct())

        def e2e_step():
            for k, t in pinned.items():
                dev_bufs[k].copy_(t, non_blocking=True)
            out2.zero_()
            H.hepacc_run_chain(db2, cfg, out2, stream=stream, _structs=s2)
            res_host[0].copy_(out2.counts, non_blocking=True)
            res_host[1].copy_(out2.sumw, non_blocking=True)
            res_host[2].copy_(out2.sumw2, non_blocking=True)

        for _ in range(3):
            e2e_step()
        torch.cuda.synchronize()
        k2 = max(3, min(args.steps, 20))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k2):
            e2e_step()
        b.record(stream)
        torch.cuda.synchronize()
        serial_ms = a.elapsed_time(b) / k2
        serial = {"value": world * batch.n_events / (serial_ms * 1e-3), "ms_per_step": serial_ms,
                  "h2d_bytes_per_step": h2d, "form": "all columns copied, then one chain call"}
        del dev_bufs, db2, out2, s2
        # the headline form, through the streaming API: the copies of range i
        # overlap the chain on range i-1 (ranges of about 1/8 of the columns)
        from paper_1906_06242_gb300 import streaming
        out3 = H.ChainOutputs(cfg, batch.n_events, per_event=False, sumw2=True)
        sc = streaming.StreamedChain(batch, cfg, out3, batch_bytes=max(1 << 20, alg_bytes // 8))

        def e2e_streamed():
            out3.zero_()
            sc.run(stream)
            res_host[0].copy_(out3.counts, non_blocking=True)
            res_host[1].copy_(out3.sumw, non_blocking=True)
            res_host[2].copy_(out3.sumw2, non_blocking=True)

        for _ in range(3):
            e2e_streamed()
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(k2):
            e2e_streamed()
        b.record(stream)
        torch.cuda.synchronize()
        e2e_ms = a.elapsed_time(b) / k2
        e2e = {"value": world * batch.n_events / (e2e_ms * 1e-3), "unit": "events/s",
               "h2d_bytes_per_step": int(sc.h2d_bytes), "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
               "form": "streaming.StreamedChain: %d host ranges, copies overlapping the chain" % len(sc.ranges),
               "serial": serial}
        del sc, out3
        if H.device_error():
            raise RuntimeError("the chain kernel set the device error word in the end-to-end forms")

    extra = {}
    if not args.no_extra and rank == 0:
        # the streamed dense form first: its host-to-device copies ran at a
        # third of the link's rate when measured after the other forms
        mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz")
        if args.dense_events > 0:
            extra.update(dense_forms(H, synth, torch, stream, args.dense_events, mhz))
        extra.update(secondary_forms(H, synth, batch, torch, stream))
        extra["kernels"] = kernel_forms(H, batch, torch, stream)
        extra.update(batched_forms(H, synth, torch, stream, args.batched_scale, mhz))

    if H.device_error():
        raise RuntimeError("a kernel set the device error word in the secondary forms")
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = cpu_baseline(batch, 4_000_000) if world == 1 else None
    # DRAM traffic of one launch: bytes per event of the committed capture
    # (a smaller case of the same kernel, traffic proportional to the events)
    counters = profile_counters()
    traffic = None
    if "plain_f32" in counters:
        traffic = counters["plain_f32"]["dram_bytes_per_event"] * batch.n_events
    if world == 1 and not args.no_extra:
        extra["cpu_oracle_all_cores"] = cpu_oracle_all_cores(batch, 4_000_000)
    line = {
        "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": headline_config(batch.n_events, world),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "peak_source": f"{peak_kind} hbm_gbs",
                     "traffic": traffic, "traffic_from": counters.get("plain_f32", {}).get("capture"),
                     "kernel": "k_fused",
                     "algorithmic_bytes_per_launch": int(alg_bytes),
                     "avg_kernel_ms": avg_kernel_ms,
                     "median_kernel_ms": sorted(kern_ms)[len(kern_ms) // 2], "min_kernel_ms": min(kern_ms)},
        "issue_roofline": issue_roofline(batch.n_events, avg_kernel_ms, "plain_f32", clocks.get("sm_mhz")),
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": args.steps,
        "clocks": clocks,
        "paper_context": PAPER_CONTEXT,
    }
    if extra:
        line["forms"] = extra
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def secondary_forms(H, synth, batch, torch, stream):
    """The other forms of the headline metric, each timed the same way:
    the chain as separate per-operation calls (FP32), the fused chain on
    BF16 kinematic columns."""
    from paper_1906_06242_gb300 import perop
    res = {}
    cfg = H.ChainConfig(synth.CUTS, synth.HIST_SPECS, [1.0])

    def timeit(fn, k=10, w=2):
        for _ in range(w):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / k

    db = H.DeviceBatch.from_host(batch)
    out = H.ChainOutputs(cfg, batch.n_events, per_event=False)
    ws = perop.PerOpWorkspace(db)
    ms = timeit(lambda: perop.run_chain_per_op(db, cfg, out, ws, stream=stream), k=5, w=1)
    res["per_op_fp32"] = {"events_per_s": batch.n_events / (ms * 1e-3), "ms_per_step": ms}
    del ws, db
    # reference decisions and histograms of the FP32 columns (per-event outputs)
    db = H.DeviceBatch.from_host(batch)
    ref = H.ChainOutputs(cfg, batch.n_events, per_event=True)
    H.hepacc_run_chain(db, cfg, ref, stream=stream)
    ref_pass = ref.ev_pass.clone()
    ref_counts = ref.counts.clone()
    del ref, db
    # 21 variations as jet-pt scales and as (eta, pt) correction tables
    # (Section IV: corrections looked up in binned tables, interpolated)
    shifts21 = synth.variation_shifts(N_VARIATIONS_BATCHED)
    db = H.DeviceBatch.from_host(batch)
    for name, jec in (("fused_scales_21", None), ("fused_jec_tables_21", synth.jec_tables(shifts21))):
        c21 = H.ChainConfig(synth.CUTS, synth.HIST_SPECS, [np.float32(1.0 + 0.01 * k) for k in shifts21], jec=jec)
        o21 = H.ChainOutputs(c21, batch.n_events)
        s21 = (db.c_struct(), c21.c_struct(), o21.c_struct())
        ms = timeit(lambda: H.hepacc_run_chain(db, c21, o21, stream=stream, _structs=s21), k=10, w=2)
        res[name] = {"events_per_s": batch.n_events / (ms * 1e-3), "ms_per_step": ms,
                     "event_variations_per_s": N_VARIATIONS_BATCHED * batch.n_events / (ms * 1e-3),
                     "variations": N_VARIATIONS_BATCHED,
                     "form": "FP32 columns, one call" + (", per-jet table lookups" if jec else ", scales")}
        del o21
    del db
    for fmt in ("bf16", "f16"):
        hb = synth.reduced_precision(batch, fmt)
        dh = H.DeviceBatch.from_host(hb)
        oh = H.ChainOutputs(cfg, batch.n_events, per_event=False)
        s = (dh.c_struct(), cfg.c_struct(), oh.c_struct())
        ms = timeit(lambda: H.hepacc_run_chain(dh, cfg, oh, stream=stream, _structs=s), k=20, w=3)
        nbytes = algorithmic_bytes(hb)
        # changed event decisions and histogram deltas against the FP32 columns
        pe = H.ChainOutputs(cfg, batch.n_events, per_event=True)
        H.hepacc_run_chain(dh, cfg, pe, stream=stream)
        changed = int((pe.ev_pass != ref_pass).sum().item())
        l1 = int((pe.counts - ref_counts).abs().sum().item())
        res[f"fused_{fmt}"] = {"events_per_s": batch.n_events / (ms * 1e-3), "ms_per_step": ms,
                               "algorithmic_gbs": nbytes / (ms * 1e-3) / 1e9,
                               "algorithmic_bytes": int(nbytes),
                               "changed_decisions_vs_f32": changed,
                               "passing_f32": int(ref_pass.sum().item()),
                               "hist_count_l1_vs_f32": l1}
        del dh, pe
    return res


def kernel_forms(H, batch, torch, stream):
    """Each per-operation kernel alone on the 10M workload's device columns:
    device time, algorithmic bytes (every array the call must read or write,
    once) and the fraction of the measured HBM copy bandwidth."""
    import math
    hbm, _ = peaks()
    db = H.DeviceBatch.from_host(batch)
    C = db.cols
    jo, mo = db.offsets["jet"], db.offsets["mu"]
    n, mj, mm = batch.n_events, C["jet_pt"].numel(), C["mu_pt"].numel()
    ob = 8 * (n + 1)
    dev = "cuda"
    out_f = torch.zeros(n, dtype=torch.float32, device=dev)
    out_f2 = torch.zeros(n, dtype=torch.float32, device=dev)
    idx = torch.zeros(n, dtype=torch.int32, device=dev)
    idx3 = torch.zeros((n, 3), dtype=torch.int32, device=dev)
    mask_j = torch.empty(mj, dtype=torch.uint8, device=dev)
    mask_m = torch.ones(mm, dtype=torch.uint8, device=dev)
    edges = torch.from_numpy(H.hist_edges(20.0, 500.0, 100)).to(dev)
    counts = torch.zeros(102, dtype=torch.int64, device=dev)
    sumw = torch.zeros(102, dtype=torch.float64, device=dev)
    sumw2 = torch.zeros(102, dtype=torch.float64, device=dev)
    n_first = int((np.diff(batch.jet_offsets) > 0).sum())   # events with a first jet
    q_mu = torch.from_numpy(batch.cols["mu_charge"]).to(dev)
    mask_os = torch.empty(mm, dtype=torch.uint8, device=dev)
    table = torch.linspace(0.9, 1.1, 102, device=dev)
    corr = torch.empty(mj, dtype=torch.float32, device=dev)
    edges_pt = torch.from_numpy(H.hist_edges(20.0, 500.0, 60)).to(dev)
    edges_eta = torch.from_numpy(H.hist_edges(-2.5, 2.5, 50)).to(dev)
    counts2 = torch.zeros((62, 52), dtype=torch.int64, device=dev)
    sumw2d = torch.zeros((62, 52), dtype=torch.float64, device=dev)
    ops = {
        "sum_in_offsets": (lambda: H.hepacc_sum_in_offsets(C["jet_pt"], jo, out=out_f, stream=stream),
                           4 * mj + ob + 8 * n),
        "max_in_offsets": (lambda: H.hepacc_max_in_offsets(C["jet_pt"], jo, out=out_f, arg=idx, stream=stream),
                           4 * mj + ob + 8 * n),
        "get_in_offsets": (lambda: H.hepacc_get_in_offsets(C["jet_pt"], jo, 0, out=out_f, index=idx, stream=stream),
                           ob + 4 * n_first + 8 * n),
        "select_range": (lambda: H.hepacc_select_range(C["jet_pt"], lo=30.0, hi=math.inf, mask_out=mask_j,
                                                       stream=stream), 5 * mj),
        "mask_deltar": (lambda: H.hepacc_mask_deltar(C["jet_eta"], C["jet_phi"], jo, C["mu_eta"], C["mu_phi"], mo,
                                                     mask2=mask_m, dr2_cut=0.16, mask1_out=mask_j, stream=stream),
                        8 * mj + 9 * mm + 2 * ob + mj),
        "fill_histogram": (lambda: H.hepacc_fill_histogram(C["jet_pt"], edges, counts=counts, sumw=sumw,
                                                           sumw2=sumw2, stream=stream), 4 * mj),
        "max_pt_trijet": (lambda: H.hepacc_max_pt_trijet(C["jet_pt"], C["jet_eta"], C["jet_phi"], C["jet_mass"], jo,
                                                         out_mass=out_f, out_pt=out_f2, out_idx3=idx3,
                                                         stream=stream), 16 * mj + ob + 20 * n),
        "trijet_closest_mass": (lambda: H.hepacc_trijet_closest_mass(C["jet_pt"], C["jet_eta"], C["jet_phi"],
                                                                     C["jet_mass"], jo, target=172.0, out_mass=out_f,
                                                                     out_idx3=idx3, stream=stream),
                                16 * mj + ob + 16 * n),
        "select_opposite_sign": (lambda: H.hepacc_select_opposite_sign(q_mu, mo, mask_out=mask_os, stream=stream),
                                 2 * mm + ob),
        "get_bin_contents": (lambda: H.hepacc_get_bin_contents(C["jet_pt"], edges, table, interpolate=True, out=corr,
                                                               stream=stream), 8 * mj),
        "fill_histogram_nd": (lambda: H.hepacc_fill_histogram_nd([C["jet_pt"], C["jet_eta"]], [edges_pt, edges_eta],
                                                                 counts=counts2, sumw=sumw2d, with_sumw2=False,
                                                                 stream=stream), 8 * mj),
    }
    res = {}
    for name, (fn, nbytes) in ops.items():
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(20):
            fn()
        e.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(e) / 20
        gbs = nbytes / (ms * 1e-3) / 1e9
        res[name] = {"ms": ms, "algorithmic_bytes": int(nbytes), "gbs": gbs, "hbm_frac": gbs / hbm}
    return res


def batched_forms(H, synth, torch, stream, scale, mhz=None):
    """The batching form: 12 samples of uneven size (log-uniform 0.2M to 20M
    events, seeds 11 to 22), each with 21 jet-pt variations, BF16 kinematic
    columns and FP16 btag, in one autotuned persistent launch replayed as a
    CUDA graph; next to it the plain forms of the same work on FP32
    columns: one fused hepacc_run_chain call per sample, and the chain as
    separate per-operation library calls."""
    import numpy as np
    t0 = time.perf_counter()
    samples = synth.batched_samples(12, size_scale=scale, workers=min(12, os.cpu_count() or 1))
    gen_s = time.perf_counter() - t0
    n_tot = sum(s.n_events for s in samples)
    shifts = synth.variation_shifts(N_VARIATIONS_BATCHED)
    cfg = H.ChainConfig(synth.CUTS, synth.HIST_SPECS, [np.float32(1.0 + 0.01 * k) for k in shifts])

    def timeit(fn, k, w=2):
        for _ in range(w):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / k

    res = {}
    # plain form: FP32 columns, one call per sample
    dbs = [H.DeviceBatch.from_host(s) for s in samples]
    outs = [H.ChainOutputs(cfg, s.n_events) for s in samples]
    structs = [(d.c_struct(), cfg.c_struct(), o.c_struct()) for d, o in zip(dbs, outs)]

    def per_sample():
        for d, o, st in zip(dbs, outs, structs):
            H.hepacc_run_chain(d, cfg, o, stream=stream, _structs=st)

    ms = timeit(per_sample, k=5)
    nbytes = sum(d.nbytes_read() for d in dbs)
    res["plain_calls_12x21"] = {"events_per_s": n_tot / (ms * 1e-3), "ms_per_step": ms,
                                "roofline": issue_roofline(n_tot, ms, "calls_f32_21", mhz),
                                "event_variations_per_s": N_VARIATIONS_BATCHED * n_tot / (ms * 1e-3),
                                "algorithmic_gbs": nbytes / (ms * 1e-3) / 1e9, "launches": len(samples),
                                "form": "FP32 columns, one fused hepacc_run_chain call per sample"}
    # the per-operation form: every step of the chain a separate library call
    from paper_1906_06242_gb300 import perop
    wss = [perop.PerOpWorkspace(d) for d in dbs]

    def per_op():
        for d, o, w in zip(dbs, outs, wss):
            perop.run_chain_per_op(d, cfg, o, w, stream=stream)

    ms_op = timeit(per_op, k=1, w=1)
    res["per_op_calls_12x21"] = {"events_per_s": n_tot / (ms_op * 1e-3), "ms_per_step": ms_op,
                                 "event_variations_per_s": N_VARIATIONS_BATCHED * n_tot / (ms_op * 1e-3),
                                 "form": "FP32 columns, the chain as separate per-operation library calls"}
    del dbs, outs, structs, wss
    # batched form: BF16 columns, one plan
    hs = [synth.reduced_precision(s, "bf16") for s in samples]
    del samples
    dbs = [H.DeviceBatch.from_host(s) for s in hs]
    outs = [H.ChainOutputs(cfg, s.n_events) for s in hs]
    t0 = time.perf_counter()
    plan = H.hepacc_plan_create(cfg, dbs, outs, flags=H.PLAN_AUTOTUNE | H.PLAN_GRAPH, stream=stream)
    tune_s = time.perf_counter() - t0
    ms = timeit(plan.run, k=10)
    nbytes = sum(d.nbytes_read() for d in dbs)
    res["batched_bf16_12x21"] = {"events_per_s": n_tot / (ms * 1e-3), "ms_per_step": ms,
                                 "roofline": issue_roofline(n_tot, ms, "batched_bf16_21", mhz),
                                 "event_variations_per_s": N_VARIATIONS_BATCHED * n_tot / (ms * 1e-3),
                                 "algorithmic_gbs": nbytes / (ms * 1e-3) / 1e9, "algorithmic_bytes": int(nbytes),
                                 "events": int(n_tot), "samples": [int(s.n_events) for s in hs],
                                 "variations": N_VARIATIONS_BATCHED, "plan": plan.describe(),
                                 "autotune_s": tune_s, "generation_s": gen_s, "size_scale": scale,
                                 "speedup_vs_fused_calls": res["plain_calls_12x21"]["ms_per_step"] / ms,
                                 "speedup_vs_per_op_calls": res["per_op_calls_12x21"]["ms_per_step"] / ms}
    plan.close()
    return res


def dense_forms(H, synth, torch, stream, n_events, mhz=None):
    """The scale form: dense events (Poisson 12 jets, 2.5 muons, 0.8
    electrons; drawn in 5M-event chunks from seed 5) resident in HBM as FP32
    and as BF16 columns, and the FP32 set streamed from pinned host memory
    in 2 GB batches on a copy stream overlapped with the chain."""
    import numpy as np
    from paper_1906_06242_gb300 import streaming
    t0 = time.perf_counter()
    w = synth.WORKLOADS["scale_60m"]
    b = synth.generate_chunked(n_events, w["seed"], chunk=5_000_000, workers=min(12, os.cpu_count() or 1),
                               lam_jet=w["lam_jet"], lam_mu=w["lam_mu"], lam_el=w["lam_el"],
                               offset_dtype=np.int64)
    gen_s = time.perf_counter() - t0
    cfg = H.ChainConfig(synth.CUTS, synth.HIST_SPECS, [1.0])
    hbm, _ = peaks()

    def timeit(fn, k, w=2):
        for _ in range(w):
            fn()
        torch.cuda.synchronize()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            fn()
        e.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(e) / k

    res = {}

    def resident(batch, name):
        db = H.DeviceBatch.from_host(batch)
        out = H.ChainOutputs(cfg, batch.n_events)
        st = (db.c_struct(), cfg.c_struct(), out.c_struct())
        ms = timeit(lambda: H.hepacc_run_chain(db, cfg, out, stream=stream, _structs=st), k=10)
        nbytes = db.nbytes_read()
        out.zero_()
        H.hepacc_run_chain(db, cfg, out, stream=stream, _structs=st)
        res[name] = {"events_per_s": batch.n_events / (ms * 1e-3), "ms_per_step": ms,
                     "algorithmic_gbs": nbytes / (ms * 1e-3) / 1e9, "algorithmic_bytes": int(nbytes),
                     "hbm_frac": nbytes / (ms * 1e-3) / 1e9 / hbm, "events": int(batch.n_events),
                     "roofline": issue_roofline(batch.n_events, ms, name.replace("_resident", ""), mhz)}
        return out

    ref = resident(b, "dense_resident_f32")
    ref_counts = ref.counts.clone()
    del ref
    torch.cuda.empty_cache()
    out = H.ChainOutputs(cfg, b.n_events)
    t0 = time.perf_counter()
    sc = streaming.StreamedChain(b, cfg, out, batch_bytes=2 << 30)
    pin_s = time.perf_counter() - t0
    ms = timeit(lambda: sc.run(stream), k=3, w=1)
    # the two halves without overlap: every range copied, then its chain
    copy_ms, compute_ms = sc.run_serial(stream)
    out.zero_()
    sc.run(stream)
    torch.cuda.synchronize()
    res["dense_streamed_f32"] = {"events_per_s": b.n_events / (ms * 1e-3), "ms_per_step": ms,
                                 "h2d_bytes_per_step": int(sc.h2d_bytes),
                                 "h2d_gbs": sc.h2d_bytes / (ms * 1e-3) / 1e9, "batches": len(sc.ranges),
                                 "batch_bytes": 2 << 30, "pinning_s": pin_s,
                                 "copies_only_ms": copy_ms, "copies_only_gbs": sc.h2d_bytes / (copy_ms * 1e-3) / 1e9,
                                 "chain_only_ms": compute_ms,
                                 "overlap": max(copy_ms, compute_ms) / ms,
                                 "counts_equal_resident": bool(torch.equal(out.counts, ref_counts))}
    del sc, out
    torch.cuda.empty_cache()
    hb = synth.reduced_precision(b, "bf16")
    del b
    resident(hb, "dense_resident_bf16")
    res["dense_resident_bf16"]["generation_s"] = gen_s
    return res


if __name__ == "__main__":
    main()
