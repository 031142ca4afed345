"""Plants plausible mistakes in copies of the oracle source (on the CPU) and
checks that the pins of test_oracle_pins.py catch every one of them."""
import os
import shutil
import tempfile

import pytest

import tests.test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "hepacc_oracle.c")

# (name, text in the source, replacement)
MUTATIONS = [
    ("dphi wrap sign", "dphi = dphi - OR_TWO_PI_F;", "dphi = dphi + OR_TWO_PI_F;"),
    ("dr2 operand", "float a = deta * deta;", "float a = deta * dphi;"),
    ("sum assigns", "acc = acc + get_f(x, xt, i);", "acc = get_f(x, xt, i);"),
    ("sum range cursor not advanced", "        lo = hi;\n", "\n"),
    ("max tie keeps last", "(want_max ? v > best : v < best)", "(want_max ? v >= best : v <= best)"),
    ("pz uses cosh", "v.pz = pt * sinh(eta);", "v.pz = pt * cosh(eta);"),
    ("mass sign", "double m2 = v.e * v.e - (", "double m2 = v.e * v.e + ("),
    ("bin upper edge inside", "if (v < (double)e[b])", "if (v <= (double)e[b])"),
    ("iso cut inclusive", "iso[i] < c->lep_iso_max;", "iso[i] <= c->lep_iso_max;"),
    ("two jets required", "njet >= 2 && nb >= 1", "njet >= 1 && nb >= 1"),
    ("trijet tie keeps last", "if (v > *best_v) {", "if (v >= *best_v) {"),
    ("lepton is the last", "if (!have_lep) {", "if (1) {"),
    ("f16 exponent bias", "e - 25);", "e - 24);"),
    ("get counts from 1", "if (seen == want) {\n                found = i;", "if (seen == want + 1) {\n                found = i;"),
    ("sub-leading may be leading", "if (q == lead_q)\n                    continue;", ""),
    ("chain dR inclusive", "< c->dr2_cut)\n                            sel = 0;", "<= c->dr2_cut)\n                            sel = 0;"),
    ("jet pt unscaled", "pt * jec_factor(c, k, pt, eta) : pt * s;", "pt * jec_factor(c, k, pt, eta) : pt;"),
    ("HT in FP64", "ht += ptk;", "ht = (float)((double)ht + (double)ptk + 1e-7 * ptk);"),
    ("weight squared missing", "o->sumw2[at] += w * w;", "o->sumw2[at] += w;"),
    ("set writes next", "((uint8_t *)x)[i] = (uint8_t)value;", "((uint8_t *)x)[i + 1] = (uint8_t)value;"),
    ("closest mass tie keeps last", "if (d < best_d) {", "if (d <= best_d) {"),
    ("closest mass uses max", "double d = fabs(m - target);", "double d = -fabs(m - target);"),
    ("opposite sign is different", "(int)charge[i] * (int)charge[j] < 0", "charge[i] != charge[j]"),
    ("opposite sign ignores mask", "if (on(mask_in, j) && ", "if ("),
    ("lookup interpolates from the upper bin", "return contents[b] + prod;", "return contents[b + 1] - prod;"),
    ("lookup centre is the lower edge", "float cb = (edges[b - 1] + edges[b]) * 0.5f;", "float cb = edges[b - 1];"),
    ("nd stride drops the flow bins", "cell = cell * (nbins[d] + 2) + b;", "cell = cell * (nbins[d] + 1) + b;"),
    ("nd NaN goes to underflow", "skip = 1;\n                break;", "b = 0;"),
    ("nd cell order reversed", "for (int d = 0; d < ndim; d++) {", "for (int d = ndim - 1; d >= 0; d--) {"),
    ("mass clamp maps NaN to 0", "return sqrt(m2 < 0.0 ? 0.0 : m2);", "return sqrt(m2 > 0.0 ? m2 : 0.0);"),
    ("scale adds", "out[i] = get_f(x, xt, i) * s;", "out[i] = get_f(x, xt, i) + s;"),
    ("scale reads the next element", "out[i] = get_f(x, xt, i) * s;", "out[i] = get_f(x, xt, i + 1 < m ? i + 1 : i) * s;"),
    ("scale rounds toward zero", "out[i] = get_f(x, xt, i) * s;",
     "{ double d = (double)get_f(x, xt, i) * s; float f = (float)d; out[i] = fabs((double)f) > fabs(d) ? "
     "nextafterf(f, 0.0f) : f; }"),
    ("pair index at the count allowed", "a >= i1 - i0 || b >= i1 - i0", "a > i1 - i0 || b > i1 - i0"),
    ("pair index not rebased", "a += i0;\n        b += i0;", "a += 0;\n        b += 0;"),
    ("pair negative index allowed", "if (a < 0 || b < 0 ||", "if ("),
    ("jec row of the eta bin below", "int row = bin_of((double)eta, c->jec_eta_edges, c->jec_neta);",
     "int row = bin_of((double)eta, c->jec_eta_edges, c->jec_neta);\n    row = row > 0 ? row - 1 : row;"),
    ("jec looks up the row at the lower edge", "return lookup_interp(pt, c->jec_pt_edges, c->jec_npt, r);",
     "return r[bin_of((double)pt, c->jec_pt_edges, c->jec_npt)];"),
]

PIN_TESTS = [getattr(pins, n) for n in dir(pins) if n.startswith("test_")]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(orc, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {name}"
    tmp = tempfile.mkdtemp(prefix="oracle_mut_")
    try:
        path = os.path.join(tmp, "mut.c")
        with open(path, "w") as f:
            f.write(src.replace(old, new))
        so = orc.compile_source(path, os.path.join(tmp, "mut.so"))
        orc.use_library(so)
        failed = []
        for t in PIN_TESTS:
            try:
                t(orc)
            except (AssertionError, pytest.skip.Exception) as e:
                if isinstance(e, AssertionError):
                    failed.append(t.__name__)
        assert failed, f"no pin caught the planted mistake '{name}'"
    finally:
        orc.use_library(None)
        shutil.rmtree(tmp, ignore_errors=True)
