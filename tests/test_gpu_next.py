"""GPU parity of the next-row kernels against the oracle, through the C ABI:
the top candidate closest to the top mass (Section IV), the opposite-sign
pair selection and the histogram lookup (Section III)."""
import numpy as np
import pytest
import torch

from paper_1906_06242_gb300 import synth

pytestmark = pytest.mark.gpu
TOP = 172.0


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


@pytest.mark.parametrize("n,lam,fmt,off_dtype", [(40_001, 5.0, "f32", np.int64), (20_011, 5.0, "bf16", np.int32),
                                                 (3_001, 14.0, "f32", np.int64), (1, 4.0, "f32", np.int64)])
def test_trijet_closest_mass(H, orc, n, lam, fmt, off_dtype):
    b = synth.generate(n, 21, lam_jet=lam, offset_dtype=off_dtype)
    if fmt != "f32":
        b = synth.reduced_precision(b, fmt)
    c = b.cols
    rng = np.random.default_rng(3)
    mask = (rng.random(len(c["jet_pt"])) < 0.9).astype(np.uint8)
    rows = (rng.random(n) < 0.95).astype(np.uint8)
    f = fmt if fmt != "f32" else None
    om, oidx, gap = orc.trijet_closest_mass(c["jet_pt"], c["jet_eta"], c["jet_phi"], c["jet_mass"], b.jet_offsets,
                                            target=TOP, mask_rows=rows, mask_content=mask, fmt=f)
    gm = torch.full((n,), -7.0, device="cuda")
    gi = torch.full((n, 3), -7, dtype=torch.int32, device="cuda")
    H.hepacc_trijet_closest_mass(dev(c["jet_pt"], f), dev(c["jet_eta"], f), dev(c["jet_phi"], f),
                                 dev(c["jet_mass"], f), dev(b.jet_offsets), target=TOP, mask_rows=dev(rows),
                                 mask_content=dev(mask), out_mass=gm, out_idx3=gi)
    torch.cuda.synchronize()
    gm, gi = gm.cpu().numpy(), gi.cpu().numpy()
    off_rows = rows == 0
    assert (gm[off_rows] == -7.0).all() and (gi[off_rows] == -7).all()   # untouched
    on = ~off_rows
    none = on & np.isnan(om)
    assert np.isnan(gm[none]).all() and (gi[none] == -1).all()
    have = on & ~np.isnan(om)
    # binary32 masses (relative error < 1e-5): the choice is exact unless the
    # runner-up is within the two masses' tolerance of the best
    tol = 1e-5 * (om + TOP)
    clear = have & (gap > 2 * tol)
    np.testing.assert_array_equal(gi[clear], oidx[clear])
    same = have & (gi == oidx).all(axis=1)
    rel = np.abs(gm[same] - om[same]) / om[same]
    assert rel.max(initial=0) < 1e-5
    # where the runner-up may have been picked, it is as close as the best within the tolerance
    amb = have & ~same
    assert (np.abs(np.abs(gm[amb] - TOP) - np.abs(om[amb] - TOP)) <= 2 * tol[amb]).all()
    assert H.device_error() == 0


@pytest.mark.parametrize("off_dtype,first", [(np.int64, 0), (np.int32, 0), (np.int64, 777)])
def test_select_opposite_sign(H, orc, off_dtype, first):
    b = synth.generate(50_003, 22, lam_mu=2.5, offset_dtype=np.int64)
    q = b.cols["mu_charge"].copy()
    rng = np.random.default_rng(4)
    q[rng.random(len(q)) < 0.05] = 0          # a few neutral objects
    mask_in = (rng.random(len(q)) < 0.85).astype(np.uint8)
    rows = (rng.random(b.n_events) < 0.9).astype(np.uint8)
    off = b.mu_offsets
    if first:
        # a slice of a larger batch: offsets start at `first`
        pad = np.zeros(first, np.int8)
        q = np.concatenate([pad, q])
        mask_in = np.concatenate([np.ones(first, np.uint8), mask_in])
        off = off + first
    off = off.astype(off_dtype)
    want = np.full(len(q), 7, np.uint8)
    orc.select_opposite_sign(q, off, mask_rows=rows, mask_in=mask_in, out=want)
    got = torch.full((len(q),), 7, dtype=torch.uint8, device="cuda")
    H.hepacc_select_opposite_sign(dev(q), dev(off), mask_rows=dev(rows), mask_in=dev(mask_in), mask_out=got)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(got.cpu().numpy(), want)
    # every selected event keeps exactly two objects of opposite charge
    g = got.cpu().numpy()
    for e in np.nonzero(rows)[0][:2000]:
        sel = np.nonzero(g[off[e]:off[e + 1]])[0]
        assert len(sel) in (0, 2)
        if len(sel) == 2:
            assert int(q[off[e] + sel[0]]) * int(q[off[e] + sel[1]]) < 0


@pytest.mark.parametrize("fmt", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("interpolate", [False, True])
def test_get_bin_contents(H, orc, fmt, interpolate):
    rng = np.random.default_rng(5)
    edges = np.sort(rng.uniform(-3, 3, 61)).astype(np.float32)
    contents = rng.normal(1.0, 0.2, 62).astype(np.float32)
    centres = ((edges[:-1] + edges[1:]) * np.float32(0.5)).astype(np.float32)
    x = np.concatenate([rng.normal(0, 1.5, 200_000), edges, centres, [np.nan, np.inf, -np.inf, -10, 10]])
    x = x.astype(np.float32)
    f = None
    if fmt != "f32":
        x = synth.to_half_bits(x, fmt)
        f = fmt
    want = orc.get_bin_contents(x, edges, contents, interpolate=interpolate, fmt=f)
    got = H.hepacc_get_bin_contents(dev(x, f), dev(edges), dev(contents), interpolate=interpolate)
    torch.cuda.synchronize()
    g = got.cpu().numpy()
    nan = np.isnan(want)
    assert (np.isnan(g) == nan).all()
    np.testing.assert_array_equal(g[~nan], want[~nan])   # same binary32 operations on both sides


def test_get_bin_contents_one_bin_and_empty(H, orc):
    edges = np.array([0.0, 1.0], np.float32)
    contents = np.array([3.0, 4.0, 5.0], np.float32)
    x = np.array([-1.0, 0.0, 0.5, 1.0, 2.0], np.float32)
    for interp in (False, True):
        want = orc.get_bin_contents(x, edges, contents, interpolate=interp)
        got = H.hepacc_get_bin_contents(dev(x), dev(edges), dev(contents), interpolate=interp).cpu().numpy()
        np.testing.assert_array_equal(got, want)
    empty = torch.empty(0, dtype=torch.float32, device="cuda")
    assert H.hepacc_get_bin_contents(empty, dev(edges), dev(contents)).numel() == 0
