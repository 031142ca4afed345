"""The seeded input generator (host logic, CPU): determinism, the recipe's
ranges and ordering, parallel draws equal to sequential ones, and the
round-to-nearest-even half-precision copies."""
import math

import numpy as np
import pytest

from paper_1906_06242_gb300 import synth


def _same(a, b):
    assert a.n_events == b.n_events
    for k in ("jet", "mu", "el"):
        np.testing.assert_array_equal(a.offsets[k], b.offsets[k])
    assert sorted(a.cols) == sorted(b.cols)
    for k in a.cols:
        np.testing.assert_array_equal(a.cols[k], b.cols[k])
    np.testing.assert_array_equal(a.weight, b.weight)


def test_generate_is_deterministic_and_seeded():
    _same(synth.generate(2_000, 3), synth.generate(2_000, 3))
    a, b = synth.generate(2_000, 3), synth.generate(2_000, 4)
    assert not np.array_equal(a.cols["jet_pt"][:100], b.cols["jet_pt"][:100])


def test_generate_recipe_ranges_and_order():
    b = synth.generate(20_000, 1, lam_jet=5.0, lam_mu=1.0, lam_el=0.8)
    for coll, lam in (("jet", 5.0), ("mu", 1.0), ("el", 0.8)):
        off = b.offsets[coll]
        assert off[0] == 0 and (np.diff(off) >= 0).all() and off[-1] == len(b.cols[f"{coll}_pt"])
        counts = np.diff(off)
        assert abs(counts.mean() - lam) < 5 * math.sqrt(lam / b.n_events)     # Poisson mean
        pt = b.cols[f"{coll}_pt"]
        assert pt.dtype == np.float32 and (pt >= 20.0).all()
        eta, phi = b.cols[f"{coll}_eta"], b.cols[f"{coll}_phi"]
        assert (np.abs(eta) <= np.float32(4.7)).all()
        assert (np.abs(phi) <= np.float32(math.pi)).all()
        # objects sorted by descending pt inside every event
        ev = np.repeat(np.arange(b.n_events), counts)
        same_event = ev[1:] == ev[:-1]
        assert (pt[1:][same_event] <= pt[:-1][same_event]).all()
    assert set(np.unique(b.cols["mu_charge"])) <= {-1, 1}
    assert set(np.unique(b.cols["el_tight"])) <= {0, 1}
    assert abs(float(b.weight.mean()) - 1.0) < 0.01


@pytest.mark.parametrize("offset_dtype", [np.int32, np.int64])
def test_chunked_parallel_equals_sequential(offset_dtype):
    kw = dict(lam_jet=7.0, lam_mu=1.5, offset_dtype=offset_dtype)
    seq = synth.generate_chunked(25_003, 9, chunk=6_000, workers=1, **kw)
    par = synth.generate_chunked(25_003, 9, chunk=6_000, workers=2, **kw)
    _same(seq, par)
    assert seq.jet_offsets.dtype == offset_dtype
    # chunk i is the recipe drawn from the seed sequence [seed, i]
    first = synth.generate(6_000, 0, rng=np.random.default_rng([9, 0]), **kw)
    np.testing.assert_array_equal(seq.cols["jet_pt"][:len(first.cols["jet_pt"])], first.cols["jet_pt"])
    np.testing.assert_array_equal(seq.jet_offsets[:6_001], first.jet_offsets)


def test_batched_samples_parallel_equals_sequential():
    seq = synth.batched_samples(3, size_scale=0.001, workers=1)
    par = synth.batched_samples(3, size_scale=0.001, workers=2)
    assert len(seq) == len(par) == 3
    for a, b in zip(seq, par):
        _same(a, b)
    assert len({s.n_events for s in seq}) == 3          # uneven sizes


def test_half_bits_round_to_nearest_even():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 1.0 + 2 ** -7 + 2 ** -8, -2.5, 0.0], np.float32)
    bits = synth.to_half_bits(x, "bf16")
    back = (bits.astype(np.uint32) << 16).view(np.float32)
    # 1 + 2^-8 is half way between 1 and 1 + 2^-7: ties go to the even 1.0;
    # 1 + 3*2^-9 is above the half way point; 1 + 2^-7 + 2^-8 ties up to 1 + 2^-6
    np.testing.assert_array_equal(back, np.array([1.0, 1.0, 1.0 + 2 ** -7, 1.0 + 2 ** -6, -2.5, 0.0], np.float32))
    h = synth.to_half_bits(np.array([65504.0, 1.0 + 2 ** -11, 1e-8], np.float32), "f16")
    np.testing.assert_array_equal(h.view(np.float16).astype(np.float32),
                                  np.array([65504.0, 1.0, 0.0], np.float32))
