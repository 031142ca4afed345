"""GPU parity of the per-operation kernels against the oracle, through the
C ABI (Section III kernels). Sizes span many warp tiles with a ragged tail;
edge cases: empty input, empty events, an event too large for the shared-
memory stage (straight-from-global path), sliced offsets (offsets[0] != 0),
int32 and int64 offsets, float32 / bfloat16 / float16 content."""
import math

import numpy as np
import pytest
import torch

from paper_1906_06242_gb300 import synth

pytestmark = pytest.mark.gpu
F32 = np.float32


@pytest.fixture(scope="module")
def H():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1906_06242_gb300 import hepacc
    hepacc.load()
    return hepacc


def dev(a, fmt=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if a.dtype == np.uint16:
        t = t.view(torch.int16).view(torch.bfloat16 if fmt == "bf16" else torch.float16)
    return t.cuda()


def host(t):
    return t.cpu().numpy()


def jagged(rng, n, lam, off_dtype=np.int64, big_row=None, first=0):
    counts = rng.poisson(lam, n)
    if big_row is not None:
        counts[big_row] = 20000
    if n > 10:
        counts[3] = 0
        counts[4] = 0
    off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    return (off + first).astype(off_dtype)


CASES = [
    # (n, lam, offsets dtype, fmt, big row, first offset)
    (70001, 5.0, np.int64, "f32", None, 0),
    (70001, 5.0, np.int32, "bf16", None, 0),
    (33333, 12.0, np.int64, "f16", None, 0),
    (5003, 3.0, np.int64, "f32", 2500, 0),     # one event of 20000 elements
    (4099, 4.0, np.int32, "f32", None, 12345),  # sliced batch: offsets start at 12345
    (1, 7.0, np.int64, "f32", None, 0),
    (37, 0.0, np.int64, "f32", None, 0),        # every event empty
]


def make_case(seed, n, lam, off_dtype, fmt, big, first):
    rng = np.random.default_rng(seed)
    off = jagged(rng, n, lam, off_dtype, big, first)
    m = int(off[-1])
    x32 = rng.normal(50, 30, m).astype(np.float32)
    x32[rng.random(m) < 0.01] = np.nan
    xh = x32 if fmt == "f32" else synth.to_half_bits(x32, fmt)
    mc = (rng.random(m) < 0.7).astype(np.uint8)
    mr = (rng.random(n) < 0.9).astype(np.uint8)
    return off, xh, mc, mr


@pytest.mark.parametrize("case", range(len(CASES)))
def test_sum_max_min_get(H, orc, case):
    n, lam, od, fmt, big, first = CASES[case]
    off, x, mc, mr = make_case(100 + case, n, lam, od, fmt, big, first)
    ofmt = None if fmt == "f32" else fmt
    d_off, d_x, d_mc, d_mr = dev(off), dev(x, ofmt), dev(mc), dev(mr)
    x_nonan = x.copy()
    if fmt == "f32":
        x_nonan[np.isnan(x_nonan)] = 1.0
    # sum: Listing 1 (+= into a preset output, masked rows untouched)
    init = np.linspace(-3, 3, n).astype(np.float32)
    xs = x_nonan if fmt == "f32" else x
    want = orc.sum_in_offsets(xs, off, mr, mc, out=init.copy(), fmt=ofmt)
    got = H.hepacc_sum_in_offsets(dev(xs, ofmt), d_off, d_mr, d_mc, out=dev(init.copy()))
    np.testing.assert_array_equal(host(got), want)
    # counting objects: sum of a uint8 mask
    want_c = orc.sum_in_offsets(mc, off)
    for odt in (torch.int32, torch.int64):
        got_c = H.hepacc_sum_in_offsets(d_mc, d_off, out_dtype=odt)
        np.testing.assert_array_equal(host(got_c).astype(np.int64), want_c)
    # max / min with argmax / argmin
    for is_max in (True, False):
        o0 = np.full(n, 99.0, np.float32)
        a0 = np.full(n, 99, np.int32)
        wv, wa = orc.minmax_in_offsets(x, off, is_max, mr, mc, empty=-1e30 if is_max else 1e30,
                                       out=o0.copy(), arg=a0.copy(), fmt=ofmt)
        fn = H.hepacc_max_in_offsets if is_max else H.hepacc_min_in_offsets
        gv, ga = fn(d_x, d_off, d_mr, d_mc, empty=-1e30 if is_max else 1e30, out=dev(o0.copy()), arg=dev(a0.copy()))
        np.testing.assert_array_equal(host(gv), wv)
        np.testing.assert_array_equal(host(ga), wa)
    # get: per-row n and scalar n
    rng = np.random.default_rng(7)
    nth = rng.integers(-1, 6, n).astype(np.int32)
    wv, wi = orc.get_in_offsets(x, off, nth, mr, mc, default=-5.0, out=np.full(n, 9, np.float32),
                                idx=np.full(n, 9, np.int32), fmt=ofmt)
    gv, gi = H.hepacc_get_in_offsets(d_x, d_off, dev(nth), d_mr, d_mc, default=-5.0,
                                     out=dev(np.full(n, 9, np.float32)), index=dev(np.full(n, 9, np.int32)))
    np.testing.assert_array_equal(host(gv), wv)
    np.testing.assert_array_equal(host(gi), wi)
    wv, wi = orc.get_in_offsets(x, off, 2, None, mc, default=-5.0, fmt=ofmt)
    gv, gi = H.hepacc_get_in_offsets(d_x, d_off, 2, None, d_mc, default=-5.0)
    np.testing.assert_array_equal(host(gv), wv)
    np.testing.assert_array_equal(host(gi), wi)
    assert H.device_error() == 0


def test_empty_input_is_noop(H):
    off = torch.zeros(1, dtype=torch.int64, device="cuda")
    x = torch.zeros(0, dtype=torch.float32, device="cuda")
    out = torch.zeros(0, dtype=torch.float32, device="cuda")
    H.hepacc_sum_in_offsets(x, off, out=out)
    H.hepacc_max_in_offsets(x, off)
    torch.cuda.synchronize()


def test_set_in_offsets(H, orc):
    rng = np.random.default_rng(11)
    off = jagged(rng, 20011, 4.0)
    m = int(off[-1])
    mask = (rng.random(m) < 0.6).astype(np.uint8)
    nth = rng.integers(-1, 4, 20011).astype(np.int32)
    rows = (rng.random(20011) < 0.8).astype(np.uint8)
    want = orc.set_in_offsets(mask.copy(), off, nth, 0, rows, mask)
    d = dev(mask.copy())
    H.hepacc_set_in_offsets(d, dev(off), dev(nth), 0, dev(rows), dev(mask))
    np.testing.assert_array_equal(host(d), want)
    xf = rng.random(m).astype(np.float32)
    want = orc.set_in_offsets(xf.copy(), off, 1, -2.5)
    d = dev(xf.copy())
    H.hepacc_set_in_offsets(d, dev(off), 1, -2.5)
    np.testing.assert_array_equal(host(d), want)


@pytest.mark.parametrize("fmt", ["f32", "bf16", "f16"])
def test_select_and_scale(H, orc, fmt):
    rng = np.random.default_rng(12)
    x = (rng.normal(30, 5, 100003)).astype(np.float32)
    x[:3] = [30.0, np.nextafter(F32(30), F32(99)), np.nan]
    xh = x if fmt == "f32" else synth.to_half_bits(x, fmt)
    ofmt = None if fmt == "f32" else fmt
    mi = (rng.random(len(x)) < 0.5).astype(np.uint8)
    for scale, lo, hi, ab in ((1.0, 30.0, math.inf, False), (0.99, 29.0, 31.0, True), (1.01, -math.inf, 2.5, True)):
        want = orc.select_range(xh, lo, hi, scale, ab, mi, fmt=ofmt)
        got = H.hepacc_select_range(dev(xh, ofmt), lo, hi, scale, ab, dev(mi))
        np.testing.assert_array_equal(host(got), want)
    want = orc.scale(xh, 1.03, fmt=ofmt)
    np.testing.assert_array_equal(host(H.hepacc_scale(dev(xh, ofmt), 1.03)), want)


@pytest.mark.parametrize("dtype", [np.uint8, np.int8, np.int32, np.float32])
@pytest.mark.parametrize("shift", [0, 1, 3])
def test_select_range_vector_and_unaligned(H, orc, dtype, shift):
    # the 16-byte vector path (aligned views, ragged tail) and the element
    # path (views starting off a 16-byte boundary)
    rng = np.random.default_rng(13)
    n = 50_011 + shift
    if dtype == np.float32:
        x = rng.normal(30, 20, n).astype(np.float32)
    else:
        x = rng.integers(-60 if dtype != np.uint8 else 0, 120, n).astype(dtype)
    mi = (rng.random(n) < 0.7).astype(np.uint8)
    want = orc.select_range(np.ascontiguousarray(x[shift:]), 10.0, 60.0, 1.0, False, mi[shift:])
    got = H.hepacc_select_range(dev(x)[shift:], 10.0, 60.0, 1.0, False, dev(mi)[shift:])
    np.testing.assert_array_equal(host(got), want)


@pytest.mark.parametrize("fmt", ["f32", "bf16"])
@pytest.mark.parametrize("shift", [0, 1, 5])
def test_scale_vector_and_unaligned(H, orc, fmt, shift):
    rng = np.random.default_rng(14)
    x = rng.normal(30, 5, 40_007).astype(np.float32)
    xh = x if fmt == "f32" else synth.to_half_bits(x, fmt)
    ofmt = None if fmt == "f32" else fmt
    want = orc.scale(np.ascontiguousarray(xh[shift:]), 0.97, fmt=ofmt)
    np.testing.assert_array_equal(host(H.hepacc_scale(dev(xh, ofmt)[shift:], 0.97)), want)


@pytest.mark.parametrize("fmt,od", [("f32", np.int64), ("bf16", np.int32), ("f16", np.int64)])
def test_mask_deltar(H, orc, fmt, od):
    b = synth.generate(50021, 31, lam_mu=2.0, offset_dtype=od)
    if fmt != "f32":
        b = synth.reduced_precision(b, fmt)
    ofmt = None if fmt == "f32" else fmt
    c = b.cols
    rng = np.random.default_rng(3)
    m1 = (rng.random(len(c["jet_eta"])) < 0.9).astype(np.uint8)
    m2 = (rng.random(len(c["mu_eta"])) < 0.8).astype(np.uint8)
    rows = (rng.random(b.n_events) < 0.95).astype(np.uint8)
    init = np.full(len(c["jet_eta"]), 7, np.uint8)
    want = orc.mask_deltar(c["jet_eta"], c["jet_phi"], b.jet_offsets, c["mu_eta"], c["mu_phi"], b.mu_offsets,
                           rows, m1, m2, 0.16, out=init.copy(), fmt1=ofmt, fmt2=ofmt)
    got = H.hepacc_mask_deltar(dev(c["jet_eta"], ofmt), dev(c["jet_phi"], ofmt), dev(b.jet_offsets),
                               dev(c["mu_eta"], ofmt), dev(c["mu_phi"], ofmt), dev(b.mu_offsets), dev(rows),
                               dev(m1), dev(m2), 0.16, mask1_out=dev(init.copy()))
    np.testing.assert_array_equal(host(got), want)
    # in place (mask1_out == mask1_in), no masks
    want = orc.mask_deltar(c["jet_eta"], c["jet_phi"], b.jet_offsets, c["el_eta"], c["el_phi"], b.el_offsets,
                           None, m1, None, 1.0, out=m1.copy(), fmt1=ofmt, fmt2=ofmt)
    d = dev(m1.copy())
    H.hepacc_mask_deltar(dev(c["jet_eta"], ofmt), dev(c["jet_phi"], ofmt), dev(b.jet_offsets),
                         dev(c["el_eta"], ofmt), dev(c["el_phi"], ofmt), dev(b.el_offsets), None, d, None, 1.0,
                         mask1_out=d)
    np.testing.assert_array_equal(host(d), want)


# 100, 37, 64 bins: exact integer sums; 1000 bins: binary64 shared-memory
# sums; 5000 bins: global memory
@pytest.mark.parametrize("nbins,uniform,dt", [(100, True, "f32"), (37, False, "f32"), (1000, True, "f32"),
                                              (5000, True, "f32"), (100, True, "bf16"), (64, True, "i32")])
def test_fill_histogram(H, orc, nbins, uniform, dt):
    rng = np.random.default_rng(13)
    n = 300007
    x = rng.normal(0.5, 1.0, n).astype(np.float32)
    if uniform:
        edges = orc.hist_edges(-2.0, 3.0, nbins)
    else:
        edges = np.sort(rng.uniform(-2, 3, nbins + 1)).astype(np.float32)
    x[:nbins + 1] = edges          # values exactly on the edges
    x[nbins + 1] = np.nan
    x[nbins + 2] = np.inf
    if dt == "i32":
        x = rng.integers(-5, 70, n).astype(np.int32)
        edges = orc.hist_edges(0, 64, nbins)
    xh = synth.to_half_bits(x, "bf16") if dt == "bf16" else x
    ofmt = "bf16" if dt == "bf16" else None
    w = rng.normal(1, 0.3, n).astype(np.float32)
    mask = (rng.random(n) < 0.85).astype(np.uint8)
    wc, ws, ws2 = orc.fill_histogram(xh, edges, w, mask, fmt=ofmt)
    d_e = dev(edges)
    gc, gs, gs2 = H.hepacc_fill_histogram(dev(xh, ofmt), d_e, weights=dev(w), mask=dev(mask))
    np.testing.assert_array_equal(host(gc).astype(np.uint64), wc)
    np.testing.assert_allclose(host(gs), ws, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(host(gs2), ws2, rtol=1e-9, atol=1e-9)
    # accumulation across two calls, without weights and mask
    gc2, gs2_, _ = H.hepacc_fill_histogram(dev(xh, ofmt), d_e, counts=gc.clone(), sumw=gs.clone(), with_sumw2=False)
    wc2, _, _ = orc.fill_histogram(xh, edges, None, None, fmt=ofmt)
    np.testing.assert_array_equal(host(gc2).astype(np.uint64), wc + wc2)


def test_fill_histogram_weight_edge_cases(H, orc):
    """Weights the integer sums take exactly (normal, zero, negative) and the
    ones they hand to binary64 (subnormal, below 2^-50, at or above 2^63,
    infinite, NaN), each in a bin of its own next to ordinary weights."""
    rng = np.random.default_rng(17)
    n = 200_003
    edges = orc.hist_edges(0.0, 10.0, 10)
    x = rng.uniform(0.0, 10.0, n).astype(np.float32)
    w = rng.normal(1.0, 0.5, n).astype(np.float32)
    special = {0.5: 0.0, 1.5: -0.0, 2.5: 1e-40, 3.5: 3e-16, 4.5: 2.0 ** 63, 5.5: 1e25, 6.5: np.inf,
               7.5: np.nan, 8.5: -3.0e18, 9.5: 2.0 ** -50}
    for k, (xv, wv) in enumerate(special.items()):
        x[k * 7:(k + 1) * 7] = xv
        w[k * 7:(k + 1) * 7] = wv
    wc, ws, ws2 = orc.fill_histogram(x, edges, w)
    gc, gs, gs2 = H.hepacc_fill_histogram(dev(x), dev(edges), weights=dev(w))
    np.testing.assert_array_equal(host(gc).astype(np.uint64), wc)
    np.testing.assert_allclose(host(gs), ws, rtol=1e-9, atol=1e-9, equal_nan=True)
    np.testing.assert_allclose(host(gs2), ws2, rtol=1e-9, atol=1e-9, equal_nan=True)


def test_fill_histogram_sums_are_exact(H):
    """One weight repeated m times in one bin: the integer sums give m w
    exactly (m w fits in binary64); m w^2 is exact per block, then rounded
    once per block and added over the blocks in binary64 (a few hundred
    roundings: relative error below 1e-12)."""
    m = 3_000_017
    x = torch.full((m,), 0.5, device="cuda")
    edges = torch.tensor([0.0, 1.0], device="cuda")
    for wv in (0.1, -7.3e-9, 1234.567):
        w = torch.full((m,), wv, dtype=torch.float32, device="cuda")
        c, s, s2 = H.hepacc_fill_histogram(x, edges, weights=w)
        w32 = float(np.float32(wv))
        assert int(c[1]) == m and float(s[1]) == m * w32
        assert float(s2[1]) == pytest.approx(m * w32 * w32, rel=1e-12)


@pytest.mark.parametrize("fmt,lam", [("f32", 5.0), ("bf16", 5.0), ("f32", 12.0)])
def test_trijet_and_pair_mass(H, orc, fmt, lam):
    b = synth.generate(40009, 41, lam_jet=lam)
    if fmt != "f32":
        b = synth.reduced_precision(b, fmt)
    ofmt = None if fmt == "f32" else fmt
    c = b.cols
    off = b.jet_offsets
    eta32 = orc.scale(c["jet_eta"], 1.0, fmt=ofmt)
    mask = orc.select_range(eta32, -np.inf, 2.5, 1.0, True)
    args = [dev(c[k], ofmt) for k in ("jet_pt", "jet_eta", "jet_phi", "jet_mass")]
    om, opt, oidx, gap = orc.max_pt_trijet(c["jet_pt"], c["jet_eta"], c["jet_phi"], c["jet_mass"], off,
                                           mask_content=mask, fmt=ofmt)
    gm, gpt, gidx = H.hepacc_max_pt_trijet(*args, dev(off), mask_content=dev(mask))
    gm, gpt, gidx = host(gm), host(gpt), host(gidx)
    near = gap < 1e-4
    same = (gidx == oidx).all(axis=1)
    assert (same | near).all()
    ok = same & ~np.isnan(om)
    assert (np.isnan(gm) == np.isnan(om)).all()
    rel = np.abs(gm[ok] - om[ok]) / om[ok]
    assert rel.max() <= 1e-5, rel.max()
    ptsum = orc.sum_in_offsets(orc.scale(c["jet_pt"], 1.0, fmt=ofmt), off, mask_content=mask).astype(np.float64)
    assert (np.abs(gpt[ok] - opt[ok]) <= 1e-5 * ptsum[ok] + 1e-6).all()
    # pair mass of random local index pairs (some out of range)
    rng = np.random.default_rng(5)
    cnt = np.diff(off.astype(np.int64))
    ia = (rng.integers(-1, 8, b.n_events)).astype(np.int32)
    ib = (rng.integers(-1, 8, b.n_events)).astype(np.int32)
    want = orc.pair_mass(c["jet_pt"], c["jet_eta"], c["jet_phi"], c["jet_mass"], off, ia, ib, fmt=ofmt)
    got = host(H.hepacc_pair_mass(*args, dev(off), dev(ia), dev(ib)))
    assert (np.isnan(got) == np.isnan(want)).all()
    ok = ~np.isnan(want)
    rel = np.abs(got[ok] - want[ok]) / np.maximum(want[ok], 1e-6)
    assert rel.max() <= 1e-5, rel.max()
    assert ((ia < 0) | (ia >= cnt) | (ib < 0) | (ib >= cnt))[~ok].all()


def test_pair_mass_closed_form(H):
    # two-body decay M -> (m1, p*) + (massless, p*) back to back, random directions
    rng = np.random.default_rng(6)
    n = 10000
    M = rng.uniform(20, 500, n)
    m1 = rng.uniform(0, 0.45, n) * M
    p = (M * M - m1 * m1) / (2 * M)
    theta = rng.uniform(0.2, math.pi - 0.2, n)
    phi = rng.uniform(-3, 3, n)
    pt = np.stack([p * np.sin(theta)] * 2, 1).ravel().astype(np.float32)
    eta = np.stack([-np.log(np.tan(theta / 2)), np.log(np.tan(theta / 2))], 1).ravel().astype(np.float32)
    ph = np.stack([phi, phi + math.pi], 1).ravel().astype(np.float32)
    mass = np.stack([m1, np.zeros(n)], 1).ravel().astype(np.float32)
    off = np.arange(0, 2 * n + 1, 2, dtype=np.int64)
    zero = torch.zeros(n, dtype=torch.int32, device="cuda")
    got = host(H.hepacc_pair_mass(dev(pt), dev(eta), dev(ph), dev(mass), dev(off), zero, zero + 1))
    # the float32 rounding of the inputs moves M slightly; compare within 1e-5
    assert (np.abs(got - M) / M).max() < 1e-5


def test_validate_offsets(H):
    off = np.array([0, 3, 3, 7, 9, 12], dtype=np.int64)
    assert int(host(H.hepacc_validate_offsets(dev(off), 12))[0]) == -1
    assert int(host(H.hepacc_validate_offsets(dev(off), 11))[0]) == 4
    bad = off.copy()
    bad[3] = 2
    assert int(host(H.hepacc_validate_offsets(dev(bad), 12))[0]) == 2
    neg = off.astype(np.int32).copy()
    neg[0] = -1
    assert int(host(H.hepacc_validate_offsets(dev(neg), 12))[0]) == -2


def test_bounded_wait_reports_timeout(H):
    # a wait that nothing completes gives up, sets the error word, and the
    # context stays usable
    assert H.device_error() == 0
    H.hepacc_selftest_wait_timeout(200_000)
    assert H.device_error() & 1
    assert H.device_error() == 0
    off = torch.tensor([0, 2, 5], dtype=torch.int64, device="cuda")
    x = torch.arange(5, dtype=torch.float32, device="cuda")
    np.testing.assert_array_equal(host(H.hepacc_sum_in_offsets(x, off)), [1.0, 9.0])


def test_invalid_arguments_rejected(H):
    off = torch.tensor([0, 2, 5], dtype=torch.int64, device="cuda")
    x = torch.arange(5, dtype=torch.float32, device="cuda")
    with pytest.raises(H.HepaccError) as ei:
        H.hepacc_sum_in_offsets(x, off, out=torch.zeros(2, dtype=torch.int32, device="cuda"))
    assert ei.value.status == 2
    with pytest.raises(H.HepaccError):
        H.hepacc_fill_histogram(x, torch.zeros(1, dtype=torch.float32, device="cuda"))
    with pytest.raises(H.HepaccError):
        H.hepacc_selftest_wait_timeout(0)
