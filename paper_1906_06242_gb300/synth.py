"""Seeded synthetic jagged-array events and the workload definitions.

This module only draws random numbers and lays them out as columns; it holds
none of the analysis arithmetic (no cuts, no reductions, no masses, no
binning). It is the one piece shared by the GPU path and the CPU oracle, which
both receive exactly the arrays made here.

Data layout (Section II of the paper): N events, M objects per collection, an
offsets array of N+1 entries per collection and one flat array of M entries per
object feature. Three collections are drawn: jets, muons, electrons.

Generator recipe (the stand-in for the CMS Open Data the paper analyses, which
is not available): numpy ``default_rng(seed)`` (PCG64), draws in this order:

1. per-event counts: jets ~ Poisson(lam_jet), muons ~ Poisson(lam_mu),
   electrons ~ Poisson(lam_el);
2. for jets, then muons, then electrons: pt = 20 + Exp(mean 30) GeV,
   eta ~ N(0, 1.5) clipped to +-4.7, phi ~ U(-pi, pi),
   mass ~ LogNormal(ln 5, 0.5); then for jets btag ~ U(0, 1); for leptons
   charge = +-1 (int8), iso ~ Exp(mean 0.1), tight ~ Bernoulli(0.8) (uint8);
3. event weight ~ N(1, 0.1);
4. objects sorted by descending pt inside each event (stable), in float64;
5. floating columns cast to float32 (round to nearest even).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ----------------------------------------------------------------------------
# Workload definitions: parameters only.
# ----------------------------------------------------------------------------

#: Object and event selection thresholds of the benchmark chain (Section IV:
#: jet and lepton selection on pt and eta, jet-lepton Delta R matching).
CUTS = {
    "lep_pt_min": 20.0,      # lepton pt > 20
    "lep_abseta_max": 2.4,   # |eta| < 2.4
    "lep_iso_max": 0.15,     # iso < 0.15 (and tight id)
    "jet_pt_min": 30.0,      # jet pt (after scale) > 30
    "jet_abseta_max": 2.5,   # |eta| < 2.5
    "dr2_cut": 0.16,         # jet masked if Delta R^2 < 0.16 to a selected lepton
    "btag_min": 0.8,         # b-tagged jet: btag > 0.8
}

#: The 20 histogrammed event variables: (name, low edge, high edge, bins).
HIST_SPECS = [
    ("ht", 0.0, 2000.0, 100),
    ("lead_jet_pt", 0.0, 1000.0, 100),
    ("lead_jet_eta", -2.5, 2.5, 100),
    ("lead_jet_phi", -math.pi, math.pi, 100),
    ("lead_jet_mass", 0.0, 100.0, 100),
    ("lead_jet_btag", 0.0, 1.0, 100),
    ("sublead_jet_pt", 0.0, 1000.0, 100),
    ("m_jj", 0.0, 2000.0, 100),
    ("n_jet", 0.0, 100.0, 100),
    ("n_bjet", 0.0, 100.0, 100),
    ("max_btag", 0.0, 1.0, 100),
    ("m_jjj", 0.0, 3000.0, 100),
    ("pt_jjj", 0.0, 2000.0, 100),
    ("lep_pt", 0.0, 500.0, 100),
    ("lep_eta", -2.5, 2.5, 100),
    ("lep_phi", -math.pi, math.pi, 100),
    ("lep_iso", 0.0, 0.15, 100),
    ("st", 0.0, 2500.0, 100),
    ("sum_jet_mass", 0.0, 500.0, 100),
    ("weight", 0.0, 2.0, 100),
]
N_HIST = len(HIST_SPECS)

#: Indices of the two trijet variables (filled only for events with >= 3 jets).
TRIJET_VARS = (11, 12)


def variation_shifts(n_var: int) -> list[int]:
    """Jet-pt scale shifts k (scale 1 + 0.01 k): nominal first, then +1, -1,
    +2, -2, ... (Section IV: jet energy systematics)."""
    ks = [0]
    k = 1
    while len(ks) < n_var:
        ks.append(k)
        if len(ks) < n_var:
            ks.append(-k)
        k += 1
    return ks


def variation_scales(n_var: int) -> list[float]:
    """Python-float (binary64) scale factors 1 + 0.01 k for ``variation_shifts``."""
    return [1.0 + 0.01 * k for k in variation_shifts(n_var)]


# ----------------------------------------------------------------------------
# Event generation
# ----------------------------------------------------------------------------

@dataclass
class EventBatch:
    """One sample of N events in columnar (offsets + flat content) form."""
    n_events: int
    jet_offsets: np.ndarray
    mu_offsets: np.ndarray
    el_offsets: np.ndarray
    cols: dict = field(default_factory=dict)   # name -> flat numpy array
    weight: np.ndarray | None = None
    seed: int | None = None

    @property
    def offsets(self):
        return {"jet": self.jet_offsets, "mu": self.mu_offsets, "el": self.el_offsets}

    def n_objects(self, coll: str) -> int:
        off = self.offsets[coll]
        return int(off[-1] - off[0])

    def nbytes(self) -> int:
        tot = self.jet_offsets.nbytes + self.mu_offsets.nbytes + self.el_offsets.nbytes
        tot += sum(a.nbytes for a in self.cols.values())
        tot += self.weight.nbytes
        return tot


def _sort_perm_desc(counts: np.ndarray, key: np.ndarray, chunk: int = 1 << 20) -> np.ndarray:
    """Permutation that orders ``key`` descending inside each event (stable)."""
    n = counts.shape[0]
    starts = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=starts[1:])
    perm = np.empty(int(starts[-1]), dtype=np.int64)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        c = counts[a:b]
        s0, s1 = int(starts[a]), int(starts[b])
        if s1 == s0:
            continue
        kmax = int(c.max())
        rel = starts[a:b] - s0
        ev = np.repeat(np.arange(b - a), c)
        pos = np.arange(s1 - s0) - np.repeat(rel, c)
        if kmax <= 1:
            perm[s0:s1] = np.arange(s0, s1)
            continue
        dense = np.full((b - a, kmax), np.inf)
        dense[ev, pos] = -key[s0:s1]
        order = np.argsort(dense, axis=1, kind="stable")
        perm[s0:s1] = s0 + rel[ev] + order[ev, pos]
    return perm


def _draw_collection(rng, total: int, kind: str):
    out = {}
    out["pt"] = 20.0 + rng.exponential(30.0, total)
    out["eta"] = np.clip(rng.normal(0.0, 1.5, total), -4.7, 4.7)
    out["phi"] = rng.uniform(-math.pi, math.pi, total)
    out["mass"] = rng.lognormal(math.log(5.0), 0.5, total)
    if kind == "jet":
        out["btag"] = rng.uniform(0.0, 1.0, total)
    else:
        out["charge"] = np.where(rng.integers(0, 2, total) == 1, 1, -1).astype(np.int8)
        out["iso"] = rng.exponential(0.1, total)
        out["tight"] = (rng.random(total) < 0.8).astype(np.uint8)
    return out


def generate(n_events: int, seed: int, lam_jet: float = 5.0, lam_mu: float = 1.0,
             lam_el: float = 0.8, offset_dtype=np.int64, rng=None) -> EventBatch:
    """Draw ``n_events`` events with the recipe in the module docstring."""
    if rng is None:
        rng = np.random.default_rng(seed)
    n = int(n_events)
    counts = {
        "jet": rng.poisson(lam_jet, n).astype(np.int64),
        "mu": rng.poisson(lam_mu, n).astype(np.int64),
        "el": rng.poisson(lam_el, n).astype(np.int64),
    }
    cols = {}
    offsets = {}
    for coll in ("jet", "mu", "el"):
        c = counts[coll]
        total = int(c.sum())
        cols[coll] = _draw_collection(rng, total, "jet" if coll == "jet" else "lep")
    weight = rng.normal(1.0, 0.1, n)
    batch_cols = {}
    for coll in ("jet", "mu", "el"):
        c = counts[coll]
        perm = _sort_perm_desc(c, cols[coll]["pt"])
        off = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(c, out=off[1:])
        offsets[coll] = off.astype(offset_dtype)
        for name, arr in cols[coll].items():
            arr = arr[perm]
            if arr.dtype == np.float64:
                arr = arr.astype(np.float32)
            batch_cols[f"{coll}_{name}"] = np.ascontiguousarray(arr)
    return EventBatch(n_events=n, jet_offsets=offsets["jet"], mu_offsets=offsets["mu"],
                      el_offsets=offsets["el"], cols=batch_cols,
                      weight=weight.astype(np.float32), seed=seed)


# ----------------------------------------------------------------------------
# Reduced-precision storage of the kinematic columns (mixed-precision storage,
# Section I). Rounding is IEEE round-to-nearest-even, done once on the host.
# Half columns are returned as uint16 bit patterns.
# ----------------------------------------------------------------------------

KINEMATIC = ("pt", "eta", "phi", "mass")


def to_half_bits(x: np.ndarray, fmt: str) -> np.ndarray:
    """float32 array -> uint16 bit patterns of bf16 or f16 (round to nearest even)."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
    if fmt == "bf16":
        h = t.to(torch.bfloat16)
    elif fmt == "f16":
        h = t.to(torch.float16)
    else:
        raise ValueError(fmt)
    return h.view(torch.int16).numpy().view(np.uint16).copy()


def reduced_precision(batch: EventBatch, kin_fmt: str, btag_fmt: str = "f16") -> EventBatch:
    """Copy of ``batch`` whose jet and lepton pt/eta/phi/mass columns are stored
    as ``kin_fmt`` (bf16 or f16) and jet btag as ``btag_fmt``; lepton iso stays
    float32 and tight stays uint8."""
    cols = dict(batch.cols)
    for coll in ("jet", "mu", "el"):
        for v in KINEMATIC:
            cols[f"{coll}_{v}"] = to_half_bits(batch.cols[f"{coll}_{v}"], kin_fmt)
    if btag_fmt != "f32":
        cols["jet_btag"] = to_half_bits(batch.cols["jet_btag"], btag_fmt)
    out = EventBatch(n_events=batch.n_events, jet_offsets=batch.jet_offsets,
                     mu_offsets=batch.mu_offsets, el_offsets=batch.el_offsets,
                     cols=cols, weight=batch.weight, seed=batch.seed)
    out.kin_fmt = kin_fmt
    out.btag_fmt = btag_fmt
    return out


# ----------------------------------------------------------------------------
# The five benchmark workloads
# ----------------------------------------------------------------------------

WORKLOADS = {
    "plain_100k": dict(n_events=100_000, seed=1, offset_dtype=np.int32),
    "plain_10m": dict(n_events=10_000_000, seed=1, offset_dtype=np.int64),
    # drawn in chunks (generate_chunked), so that it can be generated in parallel
    "scale_60m": dict(n_events=60_000_000, seed=5, offset_dtype=np.int64,
                      lam_jet=12.0, lam_mu=2.5, lam_el=0.8),
}


def _one_sample(i: int, first_seed: int, lo: float, hi: float, size_scale: float) -> EventBatch:
    rng = np.random.default_rng(first_seed + i)
    size = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
    size = max(0, int(round(size * size_scale)))
    return generate(size, first_seed + i, rng=rng, offset_dtype=np.int64)


def _pool(workers: int):
    import concurrent.futures as cf
    import multiprocessing as mp
    return cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))


def batched_samples(n_samples: int = 12, first_seed: int = 11, lo: float = 2e5,
                    hi: float = 2e7, size_scale: float = 1.0, workers: int = 1):
    """The uneven-size sample set: sample i uses ``default_rng(first_seed + i)``;
    its first draw fixes its size round(exp(U(ln lo, ln hi))) (times
    ``size_scale``, for reduced test versions), and the events follow from the
    same generator. ``workers`` > 1 draws the samples in that many spawned
    processes (same arrays)."""
    args = [(i, first_seed, lo, hi, size_scale) for i in range(n_samples)]
    if workers <= 1:
        return [_one_sample(*a) for a in args]
    with _pool(workers) as ex:
        return list(ex.map(_one_sample, *zip(*args)))


def _one_chunk(n: int, seed: int, i: int, kw: dict) -> EventBatch:
    return generate(n, seed, rng=np.random.default_rng([seed, i]), **kw)


def concat_batches(parts) -> EventBatch:
    """Events of ``parts`` one after the other (offsets rebased)."""
    n = sum(p.n_events for p in parts)
    offsets = {}
    for coll in ("jet", "mu", "el"):
        dt = parts[0].offsets[coll].dtype
        off = np.zeros(n + 1, dtype=np.int64)
        at, base = 0, 0
        for p in parts:
            o = p.offsets[coll].astype(np.int64)
            off[at + 1:at + p.n_events + 1] = o[1:] - o[0] + base
            at += p.n_events
            base += int(o[-1] - o[0])
        offsets[coll] = off.astype(dt)
    cols = {k: np.concatenate([p.cols[k] for p in parts]) for k in parts[0].cols}
    return EventBatch(n_events=n, jet_offsets=offsets["jet"], mu_offsets=offsets["mu"], el_offsets=offsets["el"],
                      cols=cols, weight=np.concatenate([p.weight for p in parts]), seed=parts[0].seed)


def generate_chunked(n_events: int, seed: int, chunk: int = 5_000_000, workers: int = 1, **kw) -> EventBatch:
    """``n_events`` events drawn as consecutive chunks of ``chunk`` events,
    chunk i from ``default_rng([seed, i])`` with the recipe of ``generate``
    (the large scale set, so that its chunks can be drawn in parallel)."""
    sizes = [min(chunk, n_events - a) for a in range(0, n_events, chunk)]
    if workers <= 1:
        parts = [_one_chunk(m, seed, i, kw) for i, m in enumerate(sizes)]
    else:
        with _pool(workers) as ex:
            parts = list(ex.map(_one_chunk, sizes, [seed] * len(sizes), range(len(sizes)), [kw] * len(sizes)))
    return concat_batches(parts) if parts else generate(0, seed, **kw)


def hand_batch(events, offset_dtype=np.int64) -> EventBatch:
    """Build a batch from explicit per-event object lists (for small hand-made
    cases). ``events`` is a list of dicts with keys 'jet', 'mu', 'el' (lists of
    per-object dicts) and 'weight'."""
    cols = {}
    offsets = {}
    fields = {"jet": ("pt", "eta", "phi", "mass", "btag"),
              "mu": ("pt", "eta", "phi", "mass", "charge", "iso", "tight"),
              "el": ("pt", "eta", "phi", "mass", "charge", "iso", "tight")}
    for coll, names in fields.items():
        counts = [len(ev.get(coll, [])) for ev in events]
        off = np.zeros(len(events) + 1, dtype=np.int64)
        np.cumsum(counts, out=off[1:])
        offsets[coll] = off.astype(offset_dtype)
        for nm in names:
            vals = [obj.get(nm, 0) for ev in events for obj in ev.get(coll, [])]
            if nm == "charge":
                arr = np.array(vals, dtype=np.int8)
            elif nm == "tight":
                arr = np.array(vals, dtype=np.uint8)
            else:
                arr = np.array(vals, dtype=np.float32)
            cols[f"{coll}_{nm}"] = arr
    w = np.array([ev.get("weight", 1.0) for ev in events], dtype=np.float32)
    return EventBatch(n_events=len(events), jet_offsets=offsets["jet"], mu_offsets=offsets["mu"],
                      el_offsets=offsets["el"], cols=cols, weight=w)


def jec_tables(shifts, seed: int = 101, n_eta: int = 8, n_pt: int = 24):
    """Synthetic jet-energy correction tables (inputs standing in for the
    experiment's correction files, which are not available): eta edges
    uniform over [-2.5, 2.5], pt edges log-uniform over [20, 1000] GeV, and
    for variation k (shift k) contents 1 + 0.01 k plus a smooth random
    (eta, pt) dependence of a few per cent, float32, shape [n_var][n_eta +
    2][n_pt + 2] (rows and columns for under- and overflow included)."""
    rng = np.random.default_rng(seed)
    eta_edges = np.linspace(-2.5, 2.5, n_eta + 1).astype(np.float32)
    pt_edges = np.geomspace(20.0, 1000.0, n_pt + 1).astype(np.float32)
    a = rng.uniform(-0.03, 0.03, size=(n_eta + 2, 1))
    b = rng.uniform(-0.02, 0.02, size=(1, n_pt + 2))
    shape = np.sin(np.linspace(0.0, 3.0, n_pt + 2))[None, :]
    base = 1.0 + a + b * shape
    contents = np.stack([(base + 0.01 * k).astype(np.float32) for k in shifts])
    return {"eta_edges": eta_edges, "pt_edges": pt_edges, "contents": contents}
