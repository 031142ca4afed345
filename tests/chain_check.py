"""Comparison of GPU chain outputs with the oracle's (test helper).

Tolerances (from the arithmetic of the two sides):
  * masks, counts, indices and every variable the chain computes with
    IEEE binary32 operations in a fixed order (HT, ST, pt_k, sums of masses,
    lepton and leading-jet attributes) must match bit for bit;
  * the pair and trijet masses: the GPU evaluates them in binary32 without
    cancellation, the oracle in binary64 from the definition; relative
    tolerance 1e-5;
  * the trijet |sum pT| can cancel between the three jets; its binary32
    error is bounded relative to the scalar sum of the jets' pt, so the
    tolerance is 1e-5 * HT (HT >= that scalar sum);
  * the trijet choice is an argmax over binary32 (GPU) and binary64 (oracle)
    ranking values |sum pT|^2. The GPU's components ptk cos(phi) carry
    correctly rounded sin/cos (error <= ~1 ulp) and three rounded additions,
    so its ranking value is within ~5e-7 (sum pt / |sum pT|) relative of the
    exact one; when the oracle's best and runner-up differ by less than
    1e-5 relative either is accepted (enough for sum pt / |sum pT| up to
    20), and such near ties must stay rare (at most 1e-4 of the events with
    a triplet, plus two);
  * histogram counts must be equal, except that an event whose mass
    variable lies within the mass tolerance of a bin edge may sit in either
    neighbouring bin (checked as a bound on the net flow across each edge);
    weighted sums agree to 1e-9 relative plus the weights of such events.
"""
import numpy as np

from paper_1906_06242_gb300 import synth

MASS_VARS = (7, 11)
PTJJJ = 12
REL_MASS = 1e-5
NEAR_TIE = 1e-5
NEAR_TIE_MAX_FRACTION = 1e-4


def edges_of(cfg_edges, nbins, h):
    e0 = int(sum(nbins[:h] + 1))
    return cfg_edges[e0:e0 + int(nbins[h]) + 1]


def trijet_free(orc, gpu_idx=None):
    """[n_var, N] bool: near-tie events (the GPU may pick the runner-up)."""
    return orc["gap"] < NEAR_TIE


def compare_per_event(gpu, orc, shifts):
    """gpu: dict of numpy arrays from the per-event outputs."""
    nv = len(shifts)
    np.testing.assert_array_equal(gpu["nlep"], orc["nlep"])
    np.testing.assert_array_equal(gpu["pass"], orc["pass"])
    np.testing.assert_array_equal(gpu["njet"], orc["njet"])
    np.testing.assert_array_equal(gpu["nb"], orc["nb"])
    np.testing.assert_array_equal(gpu["idx"][:, :2], orc["idx"][:, :2])
    free = trijet_free(orc)
    tri_g, tri_o, tri_2 = gpu["idx"][:, 2:], orc["idx"][:, 2:], orc["idx2"]
    same = (tri_g == tri_o).all(axis=1)
    runner = (tri_g == tri_2).all(axis=1)
    bad = ~same & ~(free & runner)
    assert not bad.any(), f"trijet indices differ in {int(bad.sum())} events (first {np.argwhere(bad)[:3].tolist()})"
    with_tri = int((orc["idx"][:, 2] >= 0).sum())
    assert int(free.sum()) <= NEAR_TIE_MAX_FRACTION * with_tri + 2, \
        f"{int(free.sum())} near-tie trijets among {with_tri}: the tie allowance covers too much"
    gv, ov = gpu["vars"], orc["vars"]
    for h in range(synth.N_HIST):
        g = gv[:, h]
        o = ov[:, h]
        assert (np.isnan(g) == np.isnan(o)).all(), f"NaN pattern differs for variable {h}"
        ok = ~np.isnan(o)
        if h in MASS_VARS:
            sel = ok if h == 7 else ok & same
            rel = np.abs(g[sel].astype(np.float64) - o[sel]) / np.maximum(np.abs(o[sel]), 1e-6)
            assert rel.max(initial=0) <= REL_MASS, f"variable {h}: worst relative error {rel.max()}"
        elif h == PTJJJ:
            sel = ok & same
            ht = ov[:, 0][sel]
            err = np.abs(g[sel].astype(np.float64) - o[sel])
            assert (err <= REL_MASS * ht + 1e-6).all(), f"pt_jjj: worst error {err.max()}"
        else:
            np.testing.assert_array_equal(g[ok], o[ok].astype(np.float32), err_msg=f"variable {h}")
    return {"near_ties": int(free.sum()), "runner_up_picked": int((~same & runner).sum())}


def hist_allowance(orc, weight, nbins, edges):
    """The edge-ambiguity allowance of the histogram comparison, from the
    oracle's per-event outputs: per variation k and histogram h, amb[k][h]
    (per edge: events whose mass variable lies within the mass tolerance of
    it), amb_w[k][h] (per bin: their absolute weights, on both sides),
    nfree[k][h] and free_w[k][h] (near-tie trijet events and their weight).
    Additive over event ranges."""
    nv = orc["counts"].shape[0]
    passed = orc["pass"].astype(bool)
    free = trijet_free(orc) & passed
    w = weight.astype(np.float64)
    res = {"amb": {}, "amb_w": {}, "nfree": {}, "free_w": {}}
    for k in range(nv):
        tri_ok = passed[k] & (orc["njet"][k] >= 3)
        for h in range(synth.N_HIST):
            nb = int(nbins[h])
            e = edges_of(edges, nbins, h).astype(np.float64)
            amb = np.zeros(nb + 1, dtype=np.int64)
            amb_w = np.zeros(nb + 2)
            nfree, free_w = 0, 0.0
            if h in MASS_VARS or h == PTJJJ:
                fill = tri_ok if h in (11, 12) else passed[k]
                vals = orc["vars"][k, h][fill]
                ww = np.abs(w[fill])
                if h == PTJJJ:
                    tol = REL_MASS * orc["vars"][k, 0][fill] + 1e-6
                else:
                    tol = REL_MASS * np.maximum(np.abs(vals), 1e-3)
                for j in range(nb + 1):
                    near = np.abs(vals - e[j]) <= tol
                    if near.any():
                        amb[j] += near.sum()
                        amb_w[j] += ww[near].sum()
                        amb_w[j + 1] += ww[near].sum()
                if h in (11, 12):
                    fr = free[k] & tri_ok
                    nfree = int(fr.sum())
                    free_w = float(np.abs(w[fr]).sum())
            res["amb"][k, h] = amb
            res["amb_w"][k, h] = amb_w
            res["nfree"][k, h] = nfree
            res["free_w"][k, h] = free_w
    return res


def add_allowances(a, b):
    """Allowances of two event ranges together."""
    if a is None:
        return b
    return {key: {kh: a[key][kh] + b[key][kh] for kh in a[key]} for key in a}


def check_hists(g_counts, g_sumw, g_sumw2, o_counts, o_sumw, o_sumw2, allow, nbins):
    """GPU histograms against the oracle's with the allowance of
    hist_allowance: counts equal except for the net flow across edges
    within the mass tolerance; weighted sums to 1e-9 relative plus the
    ambiguous weights."""
    nv = o_counts.shape[0]
    boff = np.concatenate([[0], np.cumsum(nbins + 2)[:-1]])
    stats = {"ambiguous": 0}
    for k in range(nv):
        for h in range(synth.N_HIST):
            lo, nb = int(boff[h]), int(nbins[h])
            sl = slice(lo, lo + nb + 2)
            gc = g_counts[k, sl].astype(np.int64)
            oc = o_counts[k, sl].astype(np.int64)
            gw, ow = g_sumw[k, sl], o_sumw[k, sl]
            d = gc - oc
            assert d.sum() == 0, f"k={k} h={h}: total count differs by {d.sum()}"
            amb, amb_w = allow["amb"][k, h], allow["amb_w"][k, h]
            nfree, free_w = allow["nfree"][k, h], allow["free_w"][k, h]
            stats["ambiguous"] += int(amb.sum())
            flow = np.cumsum(d)[:-1]
            assert (np.abs(flow) <= amb + nfree).all(), \
                f"k={k} h={h}: counts differ beyond edge ambiguity: d={np.nonzero(d)[0][:6]} flow={flow[np.abs(flow) > 0][:6]}"
            allow_w = 1e-9 * np.maximum(np.abs(ow), 1.0) + amb_w + free_w
            assert (np.abs(gw - ow) <= allow_w).all(), f"k={k} h={h}: sumw differs: {np.abs(gw - ow).max()}"
            if g_sumw2 is not None:
                gw2, ow2 = g_sumw2[k, sl], o_sumw2[k, sl]
                allow2 = 1e-9 * np.maximum(np.abs(ow2), 1.0) + 4 * (amb_w + free_w)
                assert (np.abs(gw2 - ow2) <= allow2).all(), f"k={k} h={h}: sumw2 differs"
    return stats


def compare_hists(g_counts, g_sumw, g_sumw2, orc, weight, nbins, edges):
    """Histogram check with the edge-ambiguity allowance described above."""
    allow = hist_allowance(orc, weight, nbins, edges)
    return check_hists(g_counts, g_sumw, g_sumw2, orc["counts"], orc["sumw"], orc["sumw2"], allow, nbins)
