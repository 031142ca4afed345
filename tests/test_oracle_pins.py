"""Pins of the CPU oracle to things other than itself.

Each check below is fixed by the paper's definitions (Section II data model,
Section III kernels and Listing 1, Section IV chain) and by mathematics:
hand-made events with answers worked out by hand (tests/golden), closed
forms (two-body decay momentum, massless pair identity, balanced three-body
system), invariants (segment counts sum to the content length, Delta R
symmetry, total histogram weight), numpy.histogram for the binning, and
brute force on tiny inputs written with a different structure (itertools,
complex transverse momenta, pairwise mass formula).
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from paper_1906_06242_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
F32 = np.float32
VAR = {name: i for i, (name, *_r) in enumerate(synth.HIST_SPECS)}


def _jagged(rng, n, lam, off_dtype=np.int64, first=0):
    counts = rng.poisson(lam, n)
    off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    off += first
    return counts, off.astype(off_dtype)


# ---------------------------------------------------------------------------
# golden hand-made events through the chain
# ---------------------------------------------------------------------------

def _golden():
    with open(os.path.join(GOLDEN, "hand_events.json")) as f:
        return json.load(f)


def test_golden_events_chain(orc):
    g = _golden()
    evs = g["events"]
    batch = synth.hand_batch(evs)
    out = orc.run_chain(batch, synth.CUTS, synth.HIST_SPECS, g["shifts"])
    for i, ev in enumerate(evs):
        ex = ev["expect"]
        why = ev["why"]
        assert out["nlep"][i] == ex["nlep"], why
        for k in range(len(g["shifts"])):
            if "njet" in ex:
                assert out["njet"][k, i] == ex["njet"][k], why
            if "nb" in ex:
                assert out["nb"][k, i] == ex["nb"][k], why
            if "pass" in ex:
                assert out["pass"][k, i] == ex["pass"][k], why
        if "lead" in ex:
            assert out["idx"][0, 0, i] == ex["lead"], why
        if "sub" in ex:
            assert out["idx"][0, 1, i] == ex["sub"], why
        if "tri" in ex:
            assert list(out["idx"][0, 2:, i]) == ex["tri"], why
        for name, val in ex.get("vars", {}).items():
            got = out["vars"][0, VAR[name], i]
            if val is None:
                assert math.isnan(got), (why, name)
            elif name in ("m_jj", "m_jjj"):
                assert got == pytest.approx(val, rel=1e-7), (why, name)
            else:
                assert got == float(F32(val)), (why, name, got, val)


def test_golden_ht_histogram(orc):
    g = _golden()
    batch = synth.hand_batch(g["events"])
    out = orc.run_chain(batch, synth.CUTS, synth.HIST_SPECS, g["shifts"])
    h = g["ht_hist_nominal"]
    counts = out["counts"][0, :102]
    sumw = out["sumw"][0, :102]
    exp_c = np.zeros(102, dtype=np.uint64)
    exp_w = np.zeros(102)
    for b, c in h["counts"].items():
        exp_c[int(b)] = c
    for b, w in h["sumw"].items():
        exp_w[int(b)] = w
    np.testing.assert_array_equal(counts, exp_c)
    np.testing.assert_allclose(sumw, exp_w, rtol=0, atol=0)


# ---------------------------------------------------------------------------
# sum_in_offsets (Listing 1)
# ---------------------------------------------------------------------------

def test_sum_counts_invariant(orc):
    rng = np.random.default_rng(3)
    for off_dtype in (np.int32, np.int64):
        counts, off = _jagged(rng, 1000, 3.0, off_dtype, first=17)
        m = int(off[-1])
        ones = np.ones(m, dtype=np.uint8)
        got = orc.sum_in_offsets(ones, off)
        np.testing.assert_array_equal(got, counts)
        assert got.sum() == off[-1] - off[0]


def test_sum_integer_valued_is_exact(orc):
    # integer values below 2^24 summed in any order are exact in FP32
    rng = np.random.default_rng(4)
    counts, off = _jagged(rng, 2000, 6.0)
    x = rng.integers(0, 1000, int(off[-1])).astype(np.float32)
    mask = (rng.random(len(x)) < 0.7).astype(np.uint8)
    got = orc.sum_in_offsets(x, off, mask_content=mask)
    exact = np.zeros(2000, dtype=np.int64)
    np.add.at(exact, np.repeat(np.arange(2000), counts), x.astype(np.int64) * mask)
    np.testing.assert_array_equal(got.astype(np.int64), exact)


def test_sum_listing1_semantics(orc):
    # masked events are skipped and keep their previous value; others accumulate (+=)
    off = np.array([0, 2, 2, 5], dtype=np.int64)
    x = np.array([1.5, 2.5, 4.0, 8.0, 16.0], dtype=np.float32)
    out = np.array([100.0, 7.0, -1.0], dtype=np.float32)
    orc.sum_in_offsets(x, off, mask_rows=np.array([1, 1, 0]), out=out)
    np.testing.assert_array_equal(out, [104.0, 7.0, -1.0])
    orc.sum_in_offsets(x, off, mask_content=np.array([0, 1, 1, 0, 1]), out=out)
    np.testing.assert_array_equal(out, [106.5, 7.0, 19.0])


def test_sum_fp32_sequential_order(orc):
    # 1e8 + 1 + 1 + ... in FP32 element order: each +1 is lost (ulp(1e8) = 8)
    off = np.array([0, 5], dtype=np.int64)
    x = np.array([1e8, 1, 1, 1, 1], dtype=np.float32)
    got = orc.sum_in_offsets(x, off)
    assert got[0] == F32(1e8)
    x2 = np.array([1, 1, 1, 1, 1e8], dtype=np.float32)
    assert orc.sum_in_offsets(x2, off)[0] == F32(1e8 + 4)


# ---------------------------------------------------------------------------
# max / min / get / set in offsets
# ---------------------------------------------------------------------------

def test_minmax_hand_cases(orc):
    off = np.array([0, 4, 7, 7, 9, 11], dtype=np.int32)
    x = np.array([3, 5, 5, 1, 2, 1, 1, np.nan, np.nan, np.nan, 4], dtype=np.float32)
    mx, amx = orc.minmax_in_offsets(x, off, True)
    mn, amn = orc.minmax_in_offsets(x, off, False)
    assert list(amx) == [1, 0, -1, -1, 1]      # tie -> first; empty -> -1; NaN never chosen
    np.testing.assert_array_equal(mx[[0, 1, 4]], [5, 2, 4])
    assert mx[2] == -np.inf and mx[3] == -np.inf
    assert list(amn) == [3, 1, -1, -1, 1]
    np.testing.assert_array_equal(mn[[0, 1, 4]], [1, 1, 4])


def test_minmax_brute_force(orc):
    rng = np.random.default_rng(5)
    counts, off = _jagged(rng, 500, 4.0)
    x = rng.integers(-5, 6, int(off[-1])).astype(np.float32)   # many ties
    mask = (rng.random(len(x)) < 0.6).astype(np.uint8)
    rows = (rng.random(500) < 0.8).astype(np.uint8)
    for want_max in (True, False):
        out = np.full(500, 99.0, dtype=np.float32)
        arg = np.full(500, 99, dtype=np.int32)
        orc.minmax_in_offsets(x, off, want_max, rows, mask, -1e30, out, arg)
        for e in range(500):
            if not rows[e]:
                assert out[e] == 99.0 and arg[e] == 99
                continue
            vals = [(float(x[i]), i - off[e]) for i in range(off[e], off[e + 1]) if mask[i]]
            if not vals:
                assert out[e] == F32(-1e30) and arg[e] == -1
                continue
            best = max(v for v, _ in vals) if want_max else min(v for v, _ in vals)
            assert out[e] == best
            assert arg[e] == next(j for v, j in vals if v == best)


def test_max_equals_get0_on_sorted(orc):
    b = synth.generate(3000, 9)
    pt, off = b.cols["jet_pt"], b.jet_offsets
    mask = (b.cols["jet_btag"] > 0.3).astype(np.uint8)
    mx, amx = orc.minmax_in_offsets(pt, off, True, mask_content=mask, empty=-1.0)
    g, gi = orc.get_in_offsets(pt, off, 0, mask_content=mask, default=-1.0)
    np.testing.assert_array_equal(mx, g)
    np.testing.assert_array_equal(amx, gi)


def test_get_set_brute_force(orc):
    rng = np.random.default_rng(6)
    counts, off = _jagged(rng, 400, 3.0, np.int32)
    x = rng.random(int(off[-1])).astype(np.float32)
    mask = (rng.random(len(x)) < 0.7).astype(np.uint8)
    nth = rng.integers(-1, 4, 400).astype(np.int32)
    out, idx = orc.get_in_offsets(x, off, nth, mask_content=mask, default=-5.0)
    for e in range(400):
        sel = [i for i in range(off[e], off[e + 1]) if mask[i]]
        if 0 <= nth[e] < len(sel):
            assert out[e] == x[sel[nth[e]]] and idx[e] == sel[nth[e]] - off[e]
        else:
            assert out[e] == F32(-5.0) and idx[e] == -1
    m2 = mask.copy()
    orc.set_in_offsets(m2, off, nth, 0, mask_content=mask)
    expect = mask.copy()
    for e in range(400):
        sel = [i for i in range(off[e], off[e + 1]) if mask[i]]
        if 0 <= nth[e] < len(sel):
            expect[sel[nth[e]]] = 0
    np.testing.assert_array_equal(m2, expect)


def test_select_range_edges(orc):
    x = np.array([30.0, np.nextafter(F32(30), F32(100)), 29.0, -3.0, 3.0, np.nan], dtype=np.float32)
    np.testing.assert_array_equal(orc.select_range(x, lo=30.0), [0, 1, 0, 0, 0, 0])
    np.testing.assert_array_equal(orc.select_range(x, hi=2.5, use_abs=True, lo=-1), [0, 0, 0, 0, 0, 0])
    np.testing.assert_array_equal(orc.select_range(x, hi=3.5, use_abs=True, lo=-1), [0, 0, 0, 1, 1, 0])
    # scale is applied as one FP32 product before the comparison
    np.testing.assert_array_equal(orc.select_range(np.array([30.2], np.float32), lo=30.0, scale=0.99), [0])


# ---------------------------------------------------------------------------
# Delta R
# ---------------------------------------------------------------------------

def test_dr2_exact_boundary_and_wrap(orc):
    # |Delta eta| = 0.5 exactly: Delta R^2 = 0.25 exactly, not below a 0.25 cut
    assert orc.dr2(0.75, 0.0, 0.25, 0.0) == 0.25
    off = np.array([0, 2], dtype=np.int64)
    off2 = np.array([0, 1], dtype=np.int64)
    eta1 = np.array([0.75, np.nextafter(F32(0.75), F32(0))], dtype=np.float32)
    phi1 = np.zeros(2, dtype=np.float32)
    m = orc.mask_deltar(eta1, phi1, off, np.array([0.25], np.float32), np.zeros(1, np.float32), off2,
                        dr2_cut=0.25)
    np.testing.assert_array_equal(m, [1, 0])
    # phi 3.0 and -3.0 are 2*pi - 6 = 0.283 apart
    d = orc.dr2(0.0, 3.0, 0.0, -3.0)
    assert d == pytest.approx((2 * math.pi - 6.0) ** 2, rel=1e-5)
    assert orc.dr2(0.0, -3.0, 0.0, 3.0) == d


def test_dr2_symmetric_and_matches_fp64(orc):
    rng = np.random.default_rng(7)
    e1, e2 = rng.normal(0, 2, (2, 2000)).astype(np.float32)
    p1, p2 = rng.uniform(-math.pi, math.pi, (2, 2000)).astype(np.float32)
    for i in range(2000):
        a = orc.dr2(e1[i], p1[i], e2[i], p2[i])
        b = orc.dr2(e2[i], p2[i], e1[i], p1[i])
        assert a == b
        # independent FP64 distance, the angle difference folded by the complex argument
        dphi = np.angle(np.exp(1j * (float(p1[i]) - float(p2[i]))))
        ref = (float(e1[i]) - float(e2[i])) ** 2 + dphi ** 2
        assert a == pytest.approx(ref, rel=2e-6, abs=1e-6)


def test_mask_deltar_brute_force(orc):
    rng = np.random.default_rng(8)
    n = 300
    _, off1 = _jagged(rng, n, 4.0)
    _, off2 = _jagged(rng, n, 1.5)
    m1, m2 = int(off1[-1]), int(off2[-1])
    eta1 = rng.normal(0, 1, m1).astype(np.float32)
    phi1 = rng.uniform(-math.pi, math.pi, m1).astype(np.float32)
    eta2 = rng.normal(0, 1, m2).astype(np.float32)
    phi2 = rng.uniform(-math.pi, math.pi, m2).astype(np.float32)
    mk1 = (rng.random(m1) < 0.8).astype(np.uint8)
    mk2 = (rng.random(m2) < 0.8).astype(np.uint8)
    got = orc.mask_deltar(eta1, phi1, off1, eta2, phi2, off2, mask1_in=mk1, mask2=mk2, dr2_cut=0.5)
    for e in range(n):
        for i in range(off1[e], off1[e + 1]):
            near = False
            for j in range(off2[e], off2[e + 1]):
                if not mk2[j]:
                    continue
                dphi = np.angle(np.exp(1j * (float(phi1[i]) - float(phi2[j]))))
                d = (float(eta1[i]) - float(eta2[j])) ** 2 + dphi ** 2
                if abs(d - 0.5) < 1e-5:
                    pytest.skip("random case too close to the cut for an FP64 comparison")
                near |= d < 0.5
            assert got[i] == (mk1[i] and not near)


# ---------------------------------------------------------------------------
# invariant masses
# ---------------------------------------------------------------------------

def _two_body(M, m1, m2):
    return math.sqrt((M * M - (m1 + m2) ** 2) * (M * M - (m1 - m2) ** 2)) / (2 * M)


def test_mass_two_body_decay_closed_form(orc):
    rng = np.random.default_rng(10)
    for _ in range(300):
        M = rng.uniform(10, 500)
        m1, m2 = rng.uniform(0, 0.45 * M, 2)
        p = _two_body(M, m1, m2)
        theta = rng.uniform(0.05, math.pi - 0.05)
        phi = rng.uniform(-math.pi, math.pi)
        pt = p * math.sin(theta)
        eta = -math.log(math.tan(theta / 2))
        got = orc.mass2(pt, eta, phi, m1, pt, -eta, phi + math.pi, m2)
        assert got == pytest.approx(M, rel=1e-10)


def test_mass_massless_pair_identity(orc):
    rng = np.random.default_rng(11)
    for _ in range(300):
        pt1, pt2 = rng.uniform(1, 500, 2)
        e1, e2 = rng.normal(0, 2, 2)
        f1, f2 = rng.uniform(-math.pi, math.pi, 2)
        ref = math.sqrt(2 * pt1 * pt2 * (math.cosh(e1 - e2) - math.cos(f1 - f2)))
        got = orc.mass2(pt1, e1, f1, 0.0, pt2, e2, f2, 0.0)
        assert got == pytest.approx(ref, rel=1e-9)


def test_mass_single_object_and_rotation(orc):
    rng = np.random.default_rng(12)
    for _ in range(200):
        pt, eta, phi, m = rng.uniform(1, 300), rng.normal(0, 2), rng.uniform(-3, 3), rng.uniform(0, 50)
        assert orc.mass2(pt, eta, phi, m, 0.0, 0.0, 0.0, 0.0) == pytest.approx(m, rel=1e-9, abs=1e-9)
        a = (pt, eta, phi, m)
        b = (rng.uniform(1, 300), rng.normal(0, 2), rng.uniform(-3, 3), rng.uniform(0, 50))
        r = rng.uniform(-1, 1)
        m_ab = orc.mass2(*a, *b)
        m_rot = orc.mass2(a[0], a[1], a[2] + r, a[3], b[0], b[1], b[2] + r, b[3])
        assert m_rot == pytest.approx(m_ab, rel=1e-9)


def _pairwise_mass(objs):
    """m^2 = sum m_i^2 + 2 sum_{i<j} (E_i E_j - p_i . p_j), from (pt, eta, phi, m)."""
    vecs = []
    for pt, eta, phi, m in objs:
        p = np.array([pt * math.cos(phi), pt * math.sin(phi), pt * math.sinh(eta)])
        vecs.append((math.sqrt(p @ p + m * m), p, m))
    m2 = sum(m * m for _, _, m in vecs)
    for (ea, pa, _), (eb, pb, _) in itertools.combinations(vecs, 2):
        m2 += 2 * (ea * eb - pa @ pb)
    return math.sqrt(max(m2, 0.0))


def test_trijet_brute_force(orc):
    b = synth.generate(4000, 13)
    off = b.jet_offsets
    c = b.cols
    mask = (np.abs(c["jet_eta"]) < 2.5).astype(np.uint8)
    m, ptj, idx, gap = orc.max_pt_trijet(c["jet_pt"], c["jet_eta"], c["jet_phi"], c["jet_mass"], off,
                                         mask_content=mask)
    checked = 0
    for e in range(b.n_events):
        sel = [i for i in range(off[e], off[e + 1]) if mask[i]]
        if len(sel) > 6:
            continue
        if len(sel) < 3:
            assert math.isnan(m[e]) and list(idx[e]) == [-1, -1, -1]
            continue
        best, best_v = None, -1.0
        for t in itertools.combinations(sel, 3):
            v = abs(sum(float(c["jet_pt"][i]) * np.exp(1j * float(c["jet_phi"][i])) for i in t))
            if v > best_v:
                best, best_v = t, v
        if gap[e] < 1e-9:
            continue
        assert [i - off[e] for i in best] == list(idx[e])
        assert ptj[e] == pytest.approx(best_v, rel=1e-9)
        objs = [(float(c["jet_pt"][i]), float(c["jet_eta"][i]), float(c["jet_phi"][i]),
                 float(c["jet_mass"][i])) for i in best]
        assert m[e] == pytest.approx(_pairwise_mass(objs), rel=1e-8)
        checked += 1
    assert checked > 1000


def test_trijet_balanced_three_body(orc):
    # three massless jets of equal pt at 120 degrees: zero momentum, m = 3 pt
    off = np.array([0, 3], dtype=np.int64)
    for pt in (10.0, 55.0, 400.0):
        x = np.full(3, pt, dtype=np.float32)
        phi = np.array([0.3, 0.3 + 2 * math.pi / 3, 0.3 - 2 * math.pi / 3], dtype=np.float32)
        m, ptj, idx, gap = orc.max_pt_trijet(x, np.zeros(3, np.float32), phi, np.zeros(3, np.float32), off)
        assert m[0] == pytest.approx(3 * pt, rel=1e-7)
        assert ptj[0] < 1e-4 * pt


# ---------------------------------------------------------------------------
# histograms
# ---------------------------------------------------------------------------

def test_histogram_vs_numpy(orc):
    rng = np.random.default_rng(14)
    edges = orc.hist_edges(-1.0, 3.0, 40)
    x = rng.normal(1.0, 1.5, 50000).astype(np.float32)
    x[:10] = edges[[0, 5, 17, 40, 40, 39, 0, 1, 2, 3]]     # values exactly on edges
    x[10] = np.inf
    x[11] = -np.inf
    x[12] = np.nan
    w = rng.normal(1, 0.2, len(x)).astype(np.float32)
    mask = (rng.random(len(x)) < 0.9).astype(np.uint8)
    counts, sumw, sumw2 = orc.fill_histogram(x, edges, w, mask)
    ok = mask.astype(bool) & ~np.isnan(x)
    xv, wv = x[ok].astype(np.float64), w[ok].astype(np.float64)
    inner = (xv >= edges[0]) & (xv < edges[-1])
    ref_c, _ = np.histogram(xv[inner], bins=edges.astype(np.float64))
    ref_w, _ = np.histogram(xv[inner], bins=edges.astype(np.float64), weights=wv[inner])
    ref_w2, _ = np.histogram(xv[inner], bins=edges.astype(np.float64), weights=wv[inner] ** 2)
    np.testing.assert_array_equal(counts[1:-1], ref_c)
    assert counts[0] == np.sum(xv < edges[0])
    assert counts[-1] == np.sum(xv >= edges[-1])
    np.testing.assert_allclose(sumw[1:-1], ref_w, rtol=1e-12)
    np.testing.assert_allclose(sumw2[1:-1], ref_w2, rtol=1e-12)
    assert counts.sum() == ok.sum()
    assert sumw.sum() == pytest.approx(wv.sum(), rel=1e-12)


def test_histogram_edges_are_float32_of_binary64(orc):
    e = orc.hist_edges(-math.pi, math.pi, 100)
    assert e.dtype == np.float32 and len(e) == 101
    assert e[0] == F32(-math.pi) and e[-1] == F32(math.pi) and e[50] == 0.0
    assert orc.bin_of(float(e[7]), e) == 8           # lower edge is inside the bin
    assert orc.bin_of(float(np.nextafter(e[7], F32(-10))), e) == 7
    assert orc.bin_of(float(e[-1]), e) == 101         # upper edge is overflow


def _numpy_nd(cols, edges, w):
    """numpy.histogramdd with outer edges at +-1e300 added on every axis, so
    that its cells are the under/overflow layout of the fill (the last numpy
    bin is closed, which only matters at 1e300); infinities map to +-1e299."""
    pts = np.stack([np.clip(c.astype(np.float64), -1e299, 1e299) for c in cols], axis=1)
    bins = [np.concatenate([[-1e300], e.astype(np.float64), [1e300]]) for e in edges]
    c, _ = np.histogramdd(pts, bins=bins)
    sw, _ = np.histogramdd(pts, bins=bins, weights=w)
    sw2, _ = np.histogramdd(pts, bins=bins, weights=w * w)
    return c.astype(np.uint64), sw, sw2


def test_histogram_nd_vs_numpy(orc):
    """Three axes of different sizes and types (float32, int32, bf16), values
    on edges, infinities, NaNs on each axis, a mask and weights."""
    rng = np.random.default_rng(41)
    n = 60_000
    e0 = orc.hist_edges(-2.0, 2.0, 7)
    e1 = np.array([-0.5, 0.5, 1.5, 2.5, 4.0, 7.0], np.float32)        # 5 bins
    e2 = orc.hist_edges(0.0, 1.0, 3)
    x0 = rng.normal(0, 1.5, n).astype(np.float32)
    x1 = rng.poisson(2.5, n).astype(np.int32) - 1
    x2f = rng.uniform(-0.2, 1.2, n).astype(np.float32)
    x0[:8] = e0[[0, 1, 3, 7, 7, 6, 2, 5]]
    x2f[:4] = e2[[0, 1, 2, 3]]
    x0[8], x0[9] = np.inf, -np.inf
    x0[10] = np.nan
    x1[11] = 4                                   # an int on an edge
    x2f[12] = np.nan
    x2 = synth.to_half_bits(x2f, "bf16")
    x2v = (x2.astype(np.uint32) << 16).view(np.float32)      # bf16 = the top half of a binary32
    w = rng.normal(1, 0.2, n).astype(np.float32)
    mask = (rng.random(n) < 0.9).astype(np.uint8)
    counts, sumw, sumw2 = orc.fill_histogram_nd([x0, x1, x2], [e0, e1, e2], w, mask, fmts=[None, None, "bf16"])
    assert counts.shape == (9, 7, 5)
    ok = mask.astype(bool) & ~np.isnan(x0) & ~np.isnan(x2v)
    rc, rw, rw2 = _numpy_nd([x0[ok], x1[ok], x2v[ok]], [e0, e1, e2], w[ok].astype(np.float64))
    np.testing.assert_array_equal(counts, rc)
    np.testing.assert_allclose(sumw, rw, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(sumw2, rw2, rtol=1e-12, atol=1e-12)
    assert counts.sum() == ok.sum()
    # the element on an exact int edge sits above it, the infinities at the ends
    assert counts[:, 5, :].sum() == np.sum(ok & (x1 >= 4) & (x1 < 7))
    assert counts[-1].sum() == np.sum(ok & (x0 >= e0[-1]))


def test_histogram_nd_reduces_to_1d(orc):
    """One axis is the one-dimensional fill; a second axis with a single
    all-covering bin leaves the first axis' histogram unchanged."""
    rng = np.random.default_rng(42)
    x = rng.normal(0, 2, 20_000).astype(np.float32)
    x[:3] = [np.nan, np.inf, -np.inf]
    w = rng.normal(1, 0.1, len(x)).astype(np.float32)
    e = orc.hist_edges(-3, 3, 11)
    c1, w1, q1 = orc.fill_histogram(x, e, w)
    cn, wn, qn = orc.fill_histogram_nd([x], [e], w)
    np.testing.assert_array_equal(cn, c1)
    np.testing.assert_array_equal(wn, w1)
    y = np.zeros_like(x)
    c2, w2, _ = orc.fill_histogram_nd([x, y], [e, np.array([-1, 1], np.float32)], w)
    np.testing.assert_array_equal(c2[:, 1], c1)
    assert c2[:, [0, 2]].sum() == 0
    np.testing.assert_array_equal(w2[:, 1], w1)


# ---------------------------------------------------------------------------
# the chain on generated events
# ---------------------------------------------------------------------------

def test_chain_histogram_invariants(orc):
    b = synth.generate(20000, 21)
    shifts = synth.variation_shifts(5)
    out = orc.run_chain(b, synth.CUTS, synth.HIST_SPECS, shifts)
    nb = 102
    for k in range(len(shifts)):
        passed = out["pass"][k].astype(bool)
        tri = passed & (out["njet"][k] >= 3)
        wsum = b.weight[passed].astype(np.float64).sum()
        for h in range(synth.N_HIST):
            c = out["counts"][k, h * nb:(h + 1) * nb]
            s = out["sumw"][k, h * nb:(h + 1) * nb]
            want = tri if h in synth.TRIJET_VARS else passed
            assert c.sum() == want.sum()
            assert s.sum() == pytest.approx(b.weight[want].astype(np.float64).sum(), rel=1e-12)
            s2 = out["sumw2"][k, h * nb:(h + 1) * nb]
            assert s2.sum() == pytest.approx((b.weight[want].astype(np.float64) ** 2).sum(), rel=1e-12)
        assert out["counts"][k, :nb].sum() == passed.sum()
        assert out["sumw"][k, :nb].sum() == pytest.approx(wsum, rel=1e-12)
        assert (out["nb"][k] <= out["njet"][k]).all()


def _brute_chain(b, shifts):
    """The Section IV chain written out per event with Python lists and numpy
    float32 scalars (FP32 cut arithmetic), itertools for triplets, complex
    numbers for transverse momenta and the pairwise mass formula."""
    cut = {k: F32(v) for k, v in synth.CUTS.items()}
    pi_f, two_pi_f = F32(3.14159265358979), F32(6.28318530717959)
    c = b.cols
    res = []
    for e in range(b.n_events):
        leps = []
        for coll in ("mu", "el"):
            off = b.offsets[coll]
            for i in range(off[e], off[e + 1]):
                if (c[f"{coll}_pt"][i] > cut["lep_pt_min"] and abs(c[f"{coll}_eta"][i]) < cut["lep_abseta_max"]
                        and c[f"{coll}_tight"][i] and c[f"{coll}_iso"][i] < cut["lep_iso_max"]):
                    leps.append((c[f"{coll}_pt"][i], c[f"{coll}_eta"][i], c[f"{coll}_phi"][i]))
        o = b.jet_offsets
        per_k = []
        for k in shifts:
            s = F32(1.0 + 0.01 * k)
            jets = []
            for i in range(o[e], o[e + 1]):
                ptk = c["jet_pt"][i] * s
                eta, phi = c["jet_eta"][i], c["jet_phi"][i]
                if not (ptk > cut["jet_pt_min"] and abs(eta) < cut["jet_abseta_max"]):
                    continue
                close = False
                for _lpt, leta, lphi in leps:
                    dphi = phi - lphi
                    if dphi > pi_f:
                        dphi = dphi - two_pi_f
                    elif dphi < -pi_f:
                        dphi = dphi + two_pi_f
                    deta = eta - leta
                    close |= (deta * deta + dphi * dphi) < cut["dr2_cut"]
                if not close:
                    jets.append((i - o[e], ptk, eta, phi, c["jet_mass"][i], c["jet_btag"][i]))
            ht = F32(0)
            for j in jets:
                ht = ht + j[1]
            nbj = sum(1 for j in jets if j[5] > cut["btag_min"])
            order = sorted(range(len(jets)), key=lambda q: (-float(jets[q][1]), q))
            r = {"njet": len(jets), "nb": nbj, "ht": ht,
                 "pass": int(len(leps) == 1 and len(jets) >= 2 and nbj >= 1),
                 "lead": jets[order[0]][0] if jets else -1,
                 "sub": jets[order[1]][0] if len(jets) > 1 else -1}
            if len(jets) > 1:
                a, bb = jets[order[0]], jets[order[1]]
                r["m_jj"] = _pairwise_mass([(float(a[1]), float(a[2]), float(a[3]), float(a[4])),
                                            (float(bb[1]), float(bb[2]), float(bb[3]), float(bb[4]))])
            if len(jets) > 2:
                vals = [(abs(sum(float(jets[q][1]) * np.exp(1j * float(jets[q][3])) for q in t)), t)
                        for t in itertools.combinations(range(len(jets)), 3)]
                bv = max(v for v, _ in vals)
                t = next(t for v, t in vals if v == bv)
                r["tri"] = [jets[q][0] for q in t]
                r["m_jjj"] = _pairwise_mass([tuple(float(jets[q][z]) for z in (1, 2, 3, 4)) for q in t])
                r["pt_jjj"] = bv
            per_k.append(r)
        res.append((len(leps), per_k))
    return res


def test_chain_vs_brute_force(orc):
    b = synth.generate(600, 22)
    shifts = [0, 3, -3]
    out = orc.run_chain(b, synth.CUTS, synth.HIST_SPECS, shifts)
    ref = _brute_chain(b, shifts)
    for e, (nlep, per_k) in enumerate(ref):
        assert out["nlep"][e] == nlep
        for k, r in enumerate(per_k):
            assert out["njet"][k, e] == r["njet"]
            assert out["nb"][k, e] == r["nb"]
            assert out["pass"][k, e] == r["pass"]
            assert out["vars"][k, VAR["ht"], e] == float(r["ht"])
            assert out["idx"][k, 0, e] == r["lead"] and out["idx"][k, 1, e] == r["sub"]
            if "m_jj" in r:
                assert out["vars"][k, VAR["m_jj"], e] == pytest.approx(r["m_jj"], rel=1e-8)
            if "tri" in r and out["gap"][k, e] > 1e-9:
                assert list(out["idx"][k, 2:, e]) == r["tri"]
                assert out["vars"][k, VAR["m_jjj"], e] == pytest.approx(r["m_jjj"], rel=1e-8)
                assert out["vars"][k, VAR["pt_jjj"], e] == pytest.approx(r["pt_jjj"], rel=1e-9)


def test_chain_reduced_precision_inputs_are_widened(orc):
    # a half-precision batch gives exactly the chain of its float32 widening
    b = synth.generate(3000, 23)
    for fmt in ("bf16", "f16"):
        h = synth.reduced_precision(b, fmt)
        wide = synth.EventBatch(n_events=h.n_events, jet_offsets=h.jet_offsets, mu_offsets=h.mu_offsets,
                                el_offsets=h.el_offsets, cols=dict(h.cols), weight=h.weight)
        import torch
        tdt = torch.bfloat16 if fmt == "bf16" else torch.float16
        for name, a in h.cols.items():
            if a.dtype == np.uint16:
                dt = tdt if name != "jet_btag" else torch.float16
                wide.cols[name] = torch.from_numpy(a.view(np.int16)).view(dt).float().numpy()
        o1 = orc.run_chain(h, synth.CUTS, synth.HIST_SPECS, [0, 1])
        o2 = orc.run_chain(wide, synth.CUTS, synth.HIST_SPECS, [0, 1])
        np.testing.assert_array_equal(o1["counts"], o2["counts"])
        np.testing.assert_array_equal(o1["vars"], o2["vars"])


def test_f16_decode_special_values(orc):
    bits = np.array([0x0000, 0x8000, 0x0001, 0x03ff, 0x0400, 0x3c00, 0xc000, 0x7bff, 0x7c00, 0xfc00],
                    dtype=np.uint16)
    off = np.array([0] + list(range(1, 11)), dtype=np.int64)
    got, _ = orc.get_in_offsets(bits, off, 0, fmt="f16")
    want = [0.0, -0.0, 2.0 ** -24, 1023 * 2.0 ** -24, 2.0 ** -14, 1.0, -2.0, 65504.0, np.inf, -np.inf]
    np.testing.assert_array_equal(got, np.array(want, dtype=np.float32))


def test_trijet_exact_tie_goes_to_first(orc):
    # jets 1, 2, 3 are identical, so triplets (0,1,2), (0,1,3), (0,2,3) tie exactly
    off = np.array([0, 4], dtype=np.int64)
    pt = np.array([100, 50, 50, 50], dtype=np.float32)
    z = np.zeros(4, dtype=np.float32)
    _m, _pt, idx, gap = orc.max_pt_trijet(pt, z, z, z, off)
    assert list(idx[0]) == [0, 1, 2] and gap[0] == 0.0


def test_mass_of_nan_coordinates_is_nan(orc):
    """Invariant masses propagate a NaN coordinate (the clamp at zero is for
    rounding below zero only)."""
    assert math.isnan(orc.mass2(50.0, 0.0, float("nan"), 5.0, 40.0, 1.0, 1.0, 5.0))
    assert math.isnan(orc.mass2(50.0, float("nan"), 0.0, 5.0, 40.0, 1.0, 1.0, 5.0))
    assert orc.mass2(50.0, 0.3, 0.2, 0.0, 50.0, 0.3, 0.2, 0.0) == 0.0   # collinear massless pair


def test_trijet_nan_phi_never_wins(orc):
    """A NaN phi makes the ranking value of every triplet containing that
    object NaN; such a triplet is never chosen, and with no comparable
    triplet there is none (NaN outputs, indices -1)."""
    nan = np.nan
    pt = np.array([50, 40, 30, 50, 40, 30, 20, 50, 40, 30, 20], np.float32)
    phi = np.array([0, nan, 1, 0, 1, nan, 2, nan, 1, nan, 2], np.float32)
    z = np.zeros_like(pt)
    mass = np.full_like(pt, 5.0)
    off = np.array([0, 3, 7, 11], np.int64)
    m, ptj, idx, _gap = orc.max_pt_trijet(pt, z, phi, mass, off)
    assert np.isnan(m[0]) and np.isnan(ptj[0]) and list(idx[0]) == [-1, -1, -1]
    assert list(idx[1]) == [0, 1, 3] and np.isfinite(m[1]) and np.isfinite(ptj[1])
    assert np.isnan(m[2]) and np.isnan(ptj[2]) and list(idx[2]) == [-1, -1, -1]


def test_chain_nan_phi_jet_leaves_no_trijet(orc):
    """A selected jet with a NaN phi (it passes the Delta R cut: NaN is not
    closer than 0.4) in an event with three selected jets: the event passes,
    its trijet variables are NaN and its trijet histograms get nothing,
    while the same event with a finite phi fills them."""
    lep = {"pt": 40, "eta": 0.0, "phi": 0.0, "mass": 0.1, "charge": 1, "iso": 0.01, "tight": 1}
    evs = []
    for p in (np.nan, 2.5):
        evs.append({"weight": 1.0, "mu": [lep], "el": [],
                    "jet": [{"pt": 60, "eta": 1.5, "phi": 1.5, "mass": 5, "btag": 0.9},
                            {"pt": 50, "eta": -1.5, "phi": float(p), "mass": 5, "btag": 0.1},
                            {"pt": 40, "eta": 1.0, "phi": -2.0, "mass": 5, "btag": 0.1}]})
    out = orc.run_chain(synth.hand_batch(evs), synth.CUTS, synth.HIST_SPECS, [0])
    assert list(out["pass"][0]) == [1, 1] and list(out["njet"][0]) == [3, 3]
    v = out["vars"][0]
    assert np.isnan(v[11, 0]) and np.isnan(v[12, 0]) and list(out["idx"][0, 2:, 0]) == [-1, -1, -1]
    assert np.isfinite(v[11, 1]) and np.isfinite(v[12, 1]) and list(out["idx"][0, 2:, 1]) == [0, 1, 2]
    nb = [h[3] for h in synth.HIST_SPECS]
    start = np.concatenate([[0], np.cumsum([b + 2 for b in nb])])
    c = out["counts"][0]
    assert c[start[0]:start[1]].sum() == 2                # HT: both events
    assert c[start[11]:start[12]].sum() == 1              # trijet mass: the finite one only
    assert c[start[12]:start[13]].sum() == 1              # trijet |sum pT|


def test_chain_dr2_equal_to_cut_keeps_jet(orc):
    # Delta eta = 0.1f, Delta phi = 0.38729832f give Delta R^2 == 0.16f exactly in
    # IEEE binary32 (checked here with numpy's float32 arithmetic); "closer than"
    # is strict, so the jet stays; one float closer it is masked.
    deta, dphi = F32(0.1), F32(0.38729832)
    assert deta * deta + dphi * dphi == F32(0.16)
    closer = np.nextafter(dphi, F32(0))
    assert deta * deta + closer * closer < F32(0.16)
    lep = {"pt": 40, "eta": 0.0, "phi": 0.0, "mass": 0.1, "charge": 1, "iso": 0.01, "tight": 1}
    evs = []
    for p in (dphi, closer):
        evs.append({"weight": 1.0, "mu": [lep], "el": [],
                    "jet": [{"pt": 50, "eta": float(deta), "phi": float(p), "mass": 5, "btag": 0.9},
                            {"pt": 40, "eta": -2.0, "phi": 2.0, "mass": 5, "btag": 0.1}]})
    out = orc.run_chain(synth.hand_batch(evs), synth.CUTS, synth.HIST_SPECS, [0])
    assert list(out["njet"][0]) == [2, 1]
    assert list(out["pass"][0]) == [1, 0]


# --- next rows: top candidate closest to the top mass, opposite-sign muons,
# --- histogram lookups (Sections III and IV)

def _closest_brute(pt, eta, phi, mass, off, target):
    """Per event: (mass, local indices, gap) of the triplet whose pairwise-
    formula mass is closest to target; combinations are lexicographic, so a
    strict comparison keeps the first on ties."""
    res = []
    for e in range(len(off) - 1):
        a, b = int(off[e]), int(off[e + 1])
        objs = [(float(pt[i]), float(eta[i]), float(phi[i]), float(mass[i])) for i in range(a, b)]
        best = None
        for c in itertools.combinations(range(len(objs)), 3):
            m = _pairwise_mass([objs[i] for i in c])
            d = abs(m - target)
            if best is None or d < best[0]:
                best = (d, m, c)
        res.append(best)
    return res


def test_trijet_closest_mass_brute_force(orc):
    rng = np.random.default_rng(31)
    n = 300
    _, off = _jagged(rng, n, 5.0)
    m = int(off[-1])
    pt = (20 + rng.exponential(60, m)).astype(np.float32)
    eta = rng.normal(0, 1.5, m).astype(np.float32)
    phi = rng.uniform(-np.pi, np.pi, m).astype(np.float32)
    mass = rng.lognormal(np.log(8), 0.5, m).astype(np.float32)
    om, idx, gap = orc.trijet_closest_mass(pt, eta, phi, mass, off, target=172.0)
    for e, best in enumerate(_closest_brute(pt, eta, phi, mass, off, 172.0)):
        if best is None:
            assert np.isnan(om[e]) and (idx[e] == -1).all()
            continue
        _, mb, c = best
        if gap[e] > 1e-6:   # the two FP64 formulas agree far below this
            assert tuple(idx[e]) == c, (e, idx[e], c)
        assert abs(om[e] - mb) <= 1e-9 * mb


def test_trijet_closest_mass_closed_form_and_tie(orc):
    # three massless objects at eta = 0, 120 degrees apart, pt = 172/3 each:
    # no net momentum, E = 172, so their mass is 172; a fourth, harder object
    # makes every other triplet heavier; the fifth repeats the third, so
    # (0, 1, 2) and (0, 1, 4) tie exactly: the first wins
    p = 172.0 / 3.0
    pt = np.array([p, p, p, 400.0, p], np.float32)
    eta = np.zeros(5, np.float32)
    phi = np.array([0.0, 2 * np.pi / 3, -2 * np.pi / 3, 0.3, -2 * np.pi / 3], np.float32)
    mass = np.zeros(5, np.float32)
    off = np.array([0, 5, 7], np.int64)
    pt2 = np.concatenate([pt, [50.0, 60.0]]).astype(np.float32)
    eta2 = np.concatenate([eta, [0.1, 0.2]]).astype(np.float32)
    phi2 = np.concatenate([phi, [0.1, 0.2]]).astype(np.float32)
    mass2 = np.concatenate([mass, [1.0, 1.0]]).astype(np.float32)
    om, idx, gap = orc.trijet_closest_mass(pt2, eta2, phi2, mass2, off, target=172.0)
    assert tuple(idx[0]) == (0, 1, 2)
    assert abs(om[0] - 172.0) < 1e-3   # float32 inputs: the triangle closes to ~1e-5 relative
    assert gap[0] == 0.0
    assert np.isnan(om[1]) and (idx[1] == -1).all() and np.isinf(gap[1])


def _first_opposite_pair(q, on):
    for i, j in itertools.combinations([k for k in range(len(q)) if on[k]], 2):
        if q[i] * q[j] < 0:
            return i, j
    return None


def test_select_opposite_sign_hand_cases(orc):
    events = [[1, 1, -1], [1, 1], [-1, 1, 1, -1], [], [0, 1, -1], [1], [1, -1], [0, 0, 1]]
    q = np.array([c for ev in events for c in ev], np.int8)
    off = np.concatenate([[0], np.cumsum([len(ev) for ev in events])]).astype(np.int64)
    out = orc.select_opposite_sign(q, off)
    want = [[1, 0, 1], [0, 0], [1, 1, 0, 0], [], [0, 1, 1], [0], [1, 1], [0, 0, 0]]
    np.testing.assert_array_equal(out, np.array([c for ev in want for c in ev], np.uint8))
    # masked-in objects only; rows with mask_rows unset keep their values
    mask_in = np.ones(len(q), np.uint8)
    mask_in[off[2]] = 0                   # event 2 without its first muon: (1, 3) is the first pair
    rows = np.ones(len(events), np.uint8)
    rows[0] = 0
    out = np.full(len(q), 7, np.uint8)
    orc.select_opposite_sign(q, off, mask_rows=rows, mask_in=mask_in, out=out)
    np.testing.assert_array_equal(out[off[0]:off[1]], [7, 7, 7])
    np.testing.assert_array_equal(out[off[2]:off[3]], [0, 1, 0, 1])


def test_select_opposite_sign_brute_force(orc):
    rng = np.random.default_rng(41)
    n = 2000
    _, off = _jagged(rng, n, 2.5)
    m = int(off[-1])
    q = rng.choice(np.array([-1, 0, 1], np.int8), m, p=[0.45, 0.1, 0.45])
    mask_in = (rng.random(m) < 0.8).astype(np.uint8)
    out = orc.select_opposite_sign(q, off, mask_in=mask_in)
    for e in range(n):
        a, b = int(off[e]), int(off[e + 1])
        want = np.zeros(b - a, np.uint8)
        pair = _first_opposite_pair([int(x) for x in q[a:b]], mask_in[a:b])
        if pair:
            want[list(pair)] = 1
        np.testing.assert_array_equal(out[a:b], want)


def test_get_bin_contents_step_matches_numpy(orc):
    rng = np.random.default_rng(51)
    edges = np.sort(rng.uniform(-5, 5, 41)).astype(np.float32)     # uneven bins
    contents = rng.normal(size=42).astype(np.float32)
    x = np.concatenate([rng.uniform(-6, 6, 5000), edges, [np.nan, np.inf, -np.inf]]).astype(np.float32)
    out = orc.get_bin_contents(x, edges, contents)
    b = np.searchsorted(edges.astype(np.float64), x.astype(np.float64), side="right")
    ok = ~np.isnan(x)
    np.testing.assert_array_equal(out[ok], contents[b[ok]])
    assert np.isnan(out[~ok]).all()


def test_get_bin_contents_interpolation(orc):
    rng = np.random.default_rng(52)
    edges = np.linspace(0, 10, 11).astype(np.float32)
    centres = ((edges[:-1] + edges[1:]) * np.float32(0.5)).astype(np.float32)
    y = rng.normal(size=10).astype(np.float32)
    contents = np.concatenate([[99.0], y, [-99.0]]).astype(np.float32)
    # exact at the bin centres, clamped outside the first and last centre
    np.testing.assert_array_equal(orc.get_bin_contents(centres, edges, contents, interpolate=True), y)
    out = orc.get_bin_contents(np.array([-3, 0.2, 9.7, 40], np.float32), edges, contents, interpolate=True)
    np.testing.assert_array_equal(out, [y[0], y[0], y[-1], y[-1]])
    # between two centres the value lies between their contents
    v = rng.uniform(0.5, 9.5, 4000).astype(np.float32)
    out = orc.get_bin_contents(v, edges, contents, interpolate=True)
    b = np.clip(np.floor(v.astype(np.float64) - 0.5).astype(int), 0, 8)
    lo, hi = np.minimum(y[b], y[b + 1]), np.maximum(y[b], y[b + 1])
    assert ((out >= lo - 1e-6) & (out <= hi + 1e-6)).all()
    # contents linear in the centre are reproduced up to binary32 rounding
    lin = np.concatenate([[0.0], 2.0 + 0.5 * centres, [0.0]]).astype(np.float32)
    np.testing.assert_allclose(orc.get_bin_contents(v, edges, lin, interpolate=True),
                               2.0 + 0.5 * v.astype(np.float64), rtol=1e-6, atol=1e-6)
    # one bin: its content everywhere
    one = orc.get_bin_contents(np.array([-1, 0.5, 3], np.float32), np.array([0, 1], np.float32),
                               np.array([5, 6, 7], np.float32), interpolate=True)
    np.testing.assert_array_equal(one, [6, 6, 6])


def test_get_bin_contents_interpolation_matches_numpy_interp(orc):
    # uneven (log-spaced, as the correction tables' pt bins) edges: linear
    # interpolation between bin centres, clamped at the first and last
    # centre, is numpy.interp over the centres (binary64 there, binary32 in
    # the oracle: equal to a few ulp of the contents)
    rng = np.random.default_rng(53)
    edges = np.geomspace(20.0, 1000.0, 25).astype(np.float32)
    centres = ((edges[:-1] + edges[1:]) * np.float32(0.5)).astype(np.float32)
    y = rng.uniform(0.8, 1.2, size=24).astype(np.float32)
    contents = np.concatenate([[7.0], y, [-7.0]]).astype(np.float32)
    v = np.concatenate([rng.uniform(5.0, 1500.0, 20000), centres, edges]).astype(np.float32)
    out = orc.get_bin_contents(v, edges, contents, interpolate=True)
    want = np.interp(v.astype(np.float64), centres.astype(np.float64), y.astype(np.float64))
    np.testing.assert_allclose(out, want, rtol=0, atol=4e-7 * 1.2)


# ---------------------------------------------------------------------------
# jet-pt scale variation: one binary32 product, round to nearest even
# ---------------------------------------------------------------------------

def test_scale_binary32_products_by_hand(orc):
    # exact products and hand-rounded ones (ulp of [1, 2) is 2^-23):
    #  3 * 0.5 = 1.5 exactly;
    #  (1 + 2^-12)^2 = 1 + 2^-11 + 2^-24: half an ulp above 1 + 2^-11, a tie,
    #    to even: 1 + 2^-11 (its last mantissa bit is 0);
    #  (1 + 3 2^-12)^2 = 1 + 3 2^-11 + 4.5 2^-23: a tie between 4 and 5 ulps
    #    above 1 + 3 2^-11, to even: + 4 ulps = + 2^-21;
    #  (1 + 2^-23) * 1.75 = 1.75 + 1.75 2^-23: 1.75 ulps, to nearest: + 2 ulps;
    #  2^127 * 2 overflows to +inf; -0 * 2 = -0; inf * 2 = inf; NaN stays NaN.
    x = np.array([3.0, 1 + 2 ** -12, 1 + 3 * 2 ** -12, 1 + 2 ** -23, 2.0 ** 127, -0.0, np.inf, np.nan],
                 dtype=np.float32)
    s = [0.5, 1 + 2 ** -12, 1 + 3 * 2 ** -12, 1.75, 2.0, 2.0, 2.0, 2.0]
    want = [1.5, 1 + 2 ** -11, 1 + 3 * 2 ** -11 + 2 ** -21, 1.75 + 2 ** -22, np.inf, -0.0, np.inf, np.nan]
    for xi, si, wi in zip(x, s, want):
        got = orc.scale(np.array([xi], dtype=np.float32), float(si))[0]
        if np.isnan(wi):
            assert np.isnan(got)
        else:
            assert got == np.float32(wi), (xi, si, got, wi)
            assert np.signbit(got) == np.signbit(np.float32(wi))


def test_scale_half_inputs_widen_exactly(orc):
    # binary16 0x3E00 = 1.5 and bfloat16 0x3FC0 = 1.5 (the upper half of the
    # binary32 pattern 0x3FC00000); 1.5 * 2 = 3 and 1.5 * 3 = 4.5 exactly
    f16 = np.array([0x3E00, 0x3C00, 0x7C00], dtype=np.uint16)   # 1.5, 1.0, +inf
    got = orc.scale(f16, 2.0, fmt="f16")
    assert got[0] == 3.0 and got[1] == 2.0 and np.isinf(got[2])
    bf = np.array([0x3FC0, 0xBF80], dtype=np.uint16)             # 1.5, -1.0
    got = orc.scale(bf, 3.0, fmt="bf16")
    assert got[0] == 4.5 and got[1] == -3.0
    # element by element: the i-th output comes from the i-th input only
    x = np.arange(1, 8, dtype=np.float32)
    np.testing.assert_array_equal(orc.scale(x, 2.0), 2.0 * np.arange(1, 8))


# ---------------------------------------------------------------------------
# pair mass: local indices inside sliced events, NaN outside
# ---------------------------------------------------------------------------

def test_pair_mass_local_indices_and_sliced_offsets(orc):
    # content starts with 5 elements that belong to no event (offsets[0] = 5,
    # a slice of a larger batch); events: [0] two massless objects back to
    # back (m = 2 pt = 80), [1] three objects, pair (2, 0) massless at right
    # angles (m^2 = 2 pt1 pt2 (1 - cos 90deg) = 1800), [2] one object, index 1
    # is its count: NaN, [3] index -1: NaN, [4] an object paired with itself
    # (twice its mass: 10)
    junk = [999.0] * 5
    pt = np.array(junk + [40, 40, 30, 7, 30, 12, 13, 10], dtype=np.float32)
    eta = np.array(junk + [0, 0, 0, 2, 0, 0, 0, 0.3], dtype=np.float32)
    phi = np.array(junk + [0, math.pi, 0, 1, math.pi / 2, 0, 0, 1.0], dtype=np.float32)
    m = np.array(junk + [0, 0, 0, 3, 0, 1, 1, 5], dtype=np.float32)
    off = np.array([5, 7, 10, 11, 12, 13], dtype=np.int64)
    ia = [0, 2, 1, -1, 0]
    ib = [1, 0, 0, 0, 0]
    got = orc.pair_mass(pt, eta, phi, m, off, ia, ib)
    assert abs(got[0] - 80.0) <= 1e-9 * 80
    assert abs(got[1] - math.sqrt(1800.0)) <= 1e-6 * math.sqrt(1800.0)
    assert np.isnan(got[2]) and np.isnan(got[3])
    assert abs(got[4] - 10.0) <= 1e-9 * 10
    # int32 offsets give the same
    got32 = orc.pair_mass(pt, eta, phi, m, off.astype(np.int32), ia, ib)
    np.testing.assert_array_equal(np.isnan(got32), np.isnan(got))
    ok = ~np.isnan(got)
    np.testing.assert_array_equal(got32[ok], got[ok])
    # rows with mask_rows unset keep their value (NaN here)
    masked = orc.pair_mass(pt, eta, phi, m, off, ia, ib, mask_rows=np.array([0, 1, 1, 1, 1], dtype=np.uint8))
    assert np.isnan(masked[0]) and masked[1] == got[1]


# ---------------------------------------------------------------------------
# jet-energy corrections by table lookup (Section IV), linear in pt
# ---------------------------------------------------------------------------

def test_jec_constant_tables_equal_the_scales(orc):
    # a table whose every entry is float32(1 + 0.01 k) corrects every jet by
    # exactly that factor, so variation k is the scale variation k
    b = synth.generate(20_011, 12)
    shifts = [0, 3, -3]
    eta_e = np.array([-2.5, -1.0, 0.0, 1.0, 2.5], dtype=F32)
    pt_e = np.array([20, 30, 50, 80, 150, 400], dtype=F32)
    contents = np.stack([np.full((len(eta_e) + 1, len(pt_e) + 1), F32(1.0 + 0.01 * k), dtype=F32) for k in shifts])
    jec = dict(eta_edges=eta_e, pt_edges=pt_e, contents=contents)
    a = orc.run_chain(b, synth.CUTS, synth.HIST_SPECS, shifts, jec=jec)
    s = orc.run_chain(b, synth.CUTS, synth.HIST_SPECS, shifts)
    for key in ("pass", "njet", "nb", "idx", "counts", "sumw"):
        np.testing.assert_array_equal(a[key], s[key], err_msg=key)
    np.testing.assert_array_equal(np.isnan(a["vars"]), np.isnan(s["vars"]))
    ok = ~np.isnan(s["vars"])
    np.testing.assert_array_equal(a["vars"][ok], s["vars"][ok])


def test_jec_hand_event(orc):
    # eta rows: [-2.5, 0) -> row 1, [0, 2.5) -> row 2; pt bin centres 30, 50,
    # 70, 100. Variation 0: row 1 = 1.5, 1.25, 1.0, 0.75; row 2 = 2.0, 1.5,
    # 1.0, 0.5 (flow entries 9, never read). Jets, far from the muon in phi:
    #   pt 50  at eta -1.0: centre 50, factor 1.25 -> 62.5
    #   pt 100 at eta  1.0: centre 100, factor 0.5 -> 50
    #   pt 60  at eta -0.5: halfway 50..70, 1.25 + 0.5 (1.0 - 1.25) = 1.125 -> 67.5
    #   pt 25  at eta  0.5: below the first centre, factor 2.0 -> 50
    #   pt 200 at eta -2.0: above the last centre, factor 0.75 -> 150
    # all exact in binary32: 5 jets, HT = 380, leading 150, b-jet the first.
    # Variation 1: every entry 0.5 -> 25, 50, 30, 12.5, 100: two jets above
    # 30 (30 itself fails), the b-jet (25) not selected: no pass, HT = 150.
    ev = {"jet": [{"pt": 50, "eta": -1.0, "phi": 2.0, "mass": 5, "btag": 0.9},
                   {"pt": 100, "eta": 1.0, "phi": 2.5, "mass": 5, "btag": 0.1},
                   {"pt": 60, "eta": -0.5, "phi": 3.0, "mass": 5, "btag": 0.1},
                   {"pt": 25, "eta": 0.5, "phi": -2.0, "mass": 5, "btag": 0.1},
                   {"pt": 200, "eta": -2.0, "phi": -2.5, "mass": 5, "btag": 0.1}],
          "mu": [{"pt": 50, "eta": 0.0, "phi": 0.0, "mass": 0.1, "iso": 0.01, "tight": 1, "charge": 1}],
          "el": [], "weight": 1.0}
    b = synth.hand_batch([ev])
    eta_e = np.array([-2.5, 0.0, 2.5], dtype=F32)
    pt_e = np.array([20, 40, 60, 80, 120], dtype=F32)
    c = np.full((2, 4, 6), 9.0, dtype=F32)
    c[0, 1, 1:5] = [1.5, 1.25, 1.0, 0.75]
    c[0, 2, 1:5] = [2.0, 1.5, 1.0, 0.5]
    c[1, :, :] = 0.5
    o = orc.run_chain(b, synth.CUTS, synth.HIST_SPECS, [0, 1], jec=dict(eta_edges=eta_e, pt_edges=pt_e, contents=c))
    assert o["njet"][0, 0] == 5 and o["nb"][0, 0] == 1 and o["pass"][0, 0] == 1
    assert o["vars"][0, VAR["ht"], 0] == 380.0 and o["vars"][0, VAR["lead_jet_pt"], 0] == 150.0
    assert o["vars"][0, VAR["sublead_jet_pt"], 0] == 67.5
    assert o["njet"][1, 0] == 2 and o["nb"][1, 0] == 0 and o["pass"][1, 0] == 0
    assert o["vars"][1, VAR["ht"], 0] == 150.0
