"""The chain over a batch that stays in host memory, streamed to the GPU.

The host batch is cut into contiguous event ranges whose columns take at
most ``batch_bytes`` each (offsets of every range rebased to start at 0),
held in pinned host memory. ``run`` copies range i into one of two device
buffer sets on a copy stream while the chain runs on range i-1 from the
other set on the compute stream; stream events order the reuse of a set.
The histograms of every range add into the same outputs (the chain
accumulates), so the result equals the resident run up to the order of the
binary64 additions.

Only the arrays the chain reads are copied: the three offsets arrays, the
15 object columns (``hepacc.COLUMNS``) and the event weights.
"""
from __future__ import annotations

import numpy as np

from . import hepacc as H

COLLECTIONS = ("jet", "mu", "el")


def event_bytes(batch) -> np.ndarray:
    """Bytes the chain reads for each event of a host batch (its offsets
    entries, its objects' columns, its weight)."""
    n = batch.n_events
    per = np.zeros(n, dtype=np.int64)
    for coll in COLLECTIONS:
        off = batch.offsets[coll].astype(np.int64)
        per += off.dtype.itemsize
        obj = sum(batch.cols[name].dtype.itemsize for name in H.COLUMNS if name.startswith(coll + "_"))
        per += obj * np.diff(off)
    return per + batch.weight.dtype.itemsize


def split_ranges(batch, batch_bytes: int):
    """Contiguous [a, b) event ranges covering the batch, each reading at
    most ``batch_bytes`` (an event larger than that forms a range alone)."""
    n = batch.n_events
    if n == 0:
        return []
    cum = np.concatenate([[0], np.cumsum(event_bytes(batch))])
    ranges = []
    a = 0
    while a < n:
        b = int(np.searchsorted(cum, cum[a] + batch_bytes, side="right")) - 1
        b = max(b, a + 1)
        b = min(b, n)
        ranges.append((a, b))
        a = b
    return ranges


def host_range(batch, a: int, b: int) -> dict:
    """The arrays of events [a, b): offsets rebased to 0, column slices."""
    out = {}
    for coll in COLLECTIONS:
        off = batch.offsets[coll]
        lo, hi = int(off[a]), int(off[b])
        out["off_" + coll] = (off[a:b + 1] - off[a]).astype(off.dtype)
        for name in H.COLUMNS:
            if name.startswith(coll + "_"):
                out[name] = batch.cols[name][lo:hi]
    out["weight"] = batch.weight[a:b]
    return out


class StreamedChain:
    """Double-buffered host-to-device streaming of the chain (see module
    docstring). ``out`` (hepacc.ChainOutputs) receives the histograms of
    every ``run``."""

    def __init__(self, batch, cfg: H.ChainConfig, out: H.ChainOutputs, batch_bytes: int = 2 << 30,
                 device: str = "cuda"):
        import torch
        self.torch = torch
        self.cfg = cfg
        self.out = out
        kin_fmt = getattr(batch, "kin_fmt", None)
        btag_fmt = getattr(batch, "btag_fmt", None)
        half = {"bf16": torch.bfloat16, "f16": torch.float16}

        def pinned(name, a):
            t = torch.from_numpy(np.ascontiguousarray(a))
            if a.dtype == np.uint16:
                t = t.view(torch.int16).view(half[btag_fmt if name == "jet_btag" else kin_fmt])
            return t.pin_memory()

        self.ranges = split_ranges(batch, batch_bytes)
        self.parts = []
        for a, b in self.ranges:
            self.parts.append({k: pinned(k, v) for k, v in host_range(batch, a, b).items()})
        # two device sets, each as large as the largest range of every array
        self.bufs = []
        for _ in range(2 if len(self.parts) > 1 else 1):
            bufs = {}
            for k in (self.parts[0] if self.parts else {}):
                m = max(p[k].numel() for p in self.parts)
                bufs[k] = torch.empty(max(1, m), dtype=self.parts[0][k].dtype, device=device)
            self.bufs.append(bufs)
        # per range: device views and the C structs pointing at them
        self.views = []
        for i, p in enumerate(self.parts):
            buf = self.bufs[i % len(self.bufs)]
            v = {k: buf[k][:t.numel()] for k, t in p.items()}
            n = p["weight"].numel()
            objects = {c: int(p["off_" + c][-1]) if n else 0 for c in COLLECTIONS}   # host offsets rebased to 0
            db = H.DeviceBatch(n, {c: v["off_" + c] for c in COLLECTIONS}, {name: v[name] for name in H.COLUMNS},
                               v["weight"], objects=objects)
            self.views.append((v, db, (db.c_struct(), cfg.c_struct(), out.c_struct())))
        self.copy_stream = torch.cuda.Stream(device=device)
        self.copied = [torch.cuda.Event() for _ in self.bufs]
        self.free = [torch.cuda.Event() for _ in self.bufs]

    @property
    def h2d_bytes(self) -> int:
        return sum(t.numel() * t.element_size() for p in self.parts for t in p.values())

    def run_serial(self, stream=None):
        """One pass with no overlap (each range copied, then its chain, on
        one stream); returns the milliseconds spent in copies and in the
        chain. For measurement only."""
        torch = self.torch
        compute = stream if stream is not None else torch.cuda.current_stream()
        marks = []
        for p, (v, db, structs) in zip(self.parts, self.views):
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(compute)
            with torch.cuda.stream(compute):
                for k, t in p.items():
                    v[k].copy_(t, non_blocking=True)
            e1.record(compute)
            H.hepacc_run_chain(db, self.cfg, self.out, stream=compute, _structs=structs)
            e2.record(compute)
            marks.append((e0, e1, e2))
        torch.cuda.synchronize()
        copy_ms = sum(a.elapsed_time(b) for a, b, _ in marks)
        chain_ms = sum(b.elapsed_time(c) for _, b, c in marks)
        return copy_ms, chain_ms

    def run(self, stream=None):
        """One pass over the whole batch; enqueued on ``stream`` (default:
        the current stream) and the copy stream."""
        torch = self.torch
        compute = stream if stream is not None else torch.cuda.current_stream()
        # the copy of the first range may not overtake earlier work on the buffers
        for ev in self.free:
            ev.record(compute)
        for i, (p, (v, db, structs)) in enumerate(zip(self.parts, self.views)):
            j = i % len(self.bufs)
            self.copy_stream.wait_event(self.free[j])
            with torch.cuda.stream(self.copy_stream):
                for k, t in p.items():
                    v[k].copy_(t, non_blocking=True)
            self.copied[j].record(self.copy_stream)
            compute.wait_event(self.copied[j])
            H.hepacc_run_chain(db, self.cfg, self.out, stream=compute, _structs=structs)
            self.free[j].record(compute)


__all__ = ["event_bytes", "split_ranges", "host_range", "StreamedChain"]
