/*
 * hepacc oracle: a plain, slow, obviously correct CPU implementation of the
 * jagged-array kernels and of the benchmark analysis chain of
 * "Processing Columnar Collider Data with GPU-Accelerated Kernels"
 * (Pata & Spiropulu, arXiv:1906.06242).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library path may call this code;
 * only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark load it. It shares no source, header, table or helper with the
 * GPU library.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -shared -fPIC
 * (-ffp-contract=off keeps every a*b+c as two rounded operations, which the
 * FP32 cut arithmetic below relies on).
 *
 * Data model (Section II): a collection of N events with M objects in total is
 * an offsets array of N+1 entries plus one flat array of M entries per
 * feature; event i owns elements [off[i], off[i+1]). off[0] need not be 0.
 *
 * Precision: object cuts, Delta R^2 and event sums are FP32, in the element
 * order of the per-event loop (Listing 1 of Section III accumulates with +=
 * element by element). Invariant masses and the trijet ranking are computed
 * in FP64 from their definitions. Histogram weighted sums are FP64.
 *
 * Parity pins: see tests/test_oracle_*.py (hand-made events, closed forms,
 * brute force, invariants, numpy.histogram for the binning).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* dtype codes (the Python wrapper of this file uses the same numbers) */
enum { OR_F32 = 0, OR_F16 = 1, OR_BF16 = 2, OR_I8 = 3, OR_U8 = 4, OR_I32 = 5, OR_I64 = 6 };

/* ---------------------------------------------------------------------------
 * Element access
 * ------------------------------------------------------------------------- */

/* IEEE 754 binary16 -> value, from the format's definition:
 * (-1)^s * 2^(e-15) * (1 + f/1024) for 0 < e < 31, (-1)^s * 2^-14 * f/1024 for
 * e == 0, inf/NaN for e == 31. Every binary16 value is exact in binary32. */
static float f16_value(uint16_t h)
{
    int s = (h >> 15) & 1;
    int e = (h >> 10) & 0x1f;
    int f = h & 0x3ff;
    double v;
    if (e == 0)
        v = ldexp((double)f, -24);
    else if (e == 31)
        v = f ? NAN : INFINITY;
    else
        v = ldexp((double)(1024 + f), e - 25);
    return (float)(s ? -v : v);
}

/* bfloat16 is the upper half of a binary32 bit pattern. */
static float bf16_value(uint16_t h)
{
    uint32_t u = (uint32_t)h << 16;
    float x;
    memcpy(&x, &u, sizeof x);
    return x;
}

static float get_f(const void *p, int t, int64_t i)
{
    switch (t) {
    case OR_F32: return ((const float *)p)[i];
    case OR_F16: return f16_value(((const uint16_t *)p)[i]);
    case OR_BF16: return bf16_value(((const uint16_t *)p)[i]);
    case OR_I8: return (float)((const int8_t *)p)[i];
    case OR_U8: return (float)((const uint8_t *)p)[i];
    case OR_I32: return (float)((const int32_t *)p)[i];
    case OR_I64: return (float)((const int64_t *)p)[i];
    }
    return NAN;
}

static int64_t get_i(const void *p, int t, int64_t i)
{
    switch (t) {
    case OR_I8: return ((const int8_t *)p)[i];
    case OR_U8: return ((const uint8_t *)p)[i];
    case OR_I32: return ((const int32_t *)p)[i];
    case OR_I64: return ((const int64_t *)p)[i];
    }
    return 0;
}

static int64_t get_off(const void *off, int ot, int64_t i)
{
    return ot == OR_I32 ? (int64_t)((const int32_t *)off)[i] : ((const int64_t *)off)[i];
}

static int on(const uint8_t *mask, int64_t i) { return mask == NULL || mask[i] != 0; }

/* ---------------------------------------------------------------------------
 * Generic kernels (Section III)
 * ------------------------------------------------------------------------- */

/* The FP32 sum of the masked-in elements of x in [lo, hi), one addition at
 * a time in element order, starting from acc. */
static float fsum_masked(const void *x, int xt, int64_t lo, int64_t hi, const uint8_t *mask, float acc)
{
    for (int64_t i = lo; i < hi; i++)
        if (on(mask, i))
            acc = acc + get_f(x, xt, i);
    return acc;
}

/* sum_in_offsets over floating content (Section III): event ev owns the
 * elements [off[ev], off[ev+1]); a selected event (mask_rows) adds the FP32
 * sum of its masked-in elements (mask_content), in element order, to the
 * value already in out[ev]; other events keep theirs. One pass over the
 * events, the end of one event's range being the start of the next. */
void oracle_sum_in_offsets_f(const void *x, int xt, const void *off, int ot, int64_t n,
                             const uint8_t *mask_rows, const uint8_t *mask_content, float *out)
{
    int64_t lo = n > 0 ? get_off(off, ot, 0) : 0;
    for (int64_t ev = 0; ev < n; ev++) {
        const int64_t hi = get_off(off, ot, ev + 1);
        if (on(mask_rows, ev))
            out[ev] = fsum_masked(x, xt, lo, hi, mask_content, out[ev]);
        lo = hi;
    }
}

/* sum_in_offsets over integer content (used to count objects by summing
 * masks, Section III); exact in int64. */
void oracle_sum_in_offsets_i(const void *x, int xt, const void *off, int ot, int64_t n,
                             const uint8_t *mask_rows, const uint8_t *mask_content, int64_t *out)
{
    for (int64_t ev = 0; ev < n; ev++) {
        if (!on(mask_rows, ev))
            continue;
        int64_t i0 = get_off(off, ot, ev), i1 = get_off(off, ot, ev + 1);
        for (int64_t i = i0; i < i1; i++)
            if (on(mask_content, i))
                out[ev] += get_i(x, xt, i);
    }
}

/* max_in_offsets / min_in_offsets (Section III). Among the masked-in, non-NaN
 * elements of the event: the largest (smallest) value and the local index
 * (0-based inside the event) of its first occurrence. No such element:
 * out = empty, arg = -1. Events with mask_rows unset are untouched. */
void oracle_minmax_in_offsets(const void *x, int xt, const void *off, int ot, int64_t n,
                              const uint8_t *mask_rows, const uint8_t *mask_content,
                              int want_max, float empty, float *out, int32_t *arg)
{
    for (int64_t ev = 0; ev < n; ev++) {
        if (!on(mask_rows, ev))
            continue;
        int64_t i0 = get_off(off, ot, ev), i1 = get_off(off, ot, ev + 1);
        int64_t best_i = -1;
        float best = empty;
        for (int64_t i = i0; i < i1; i++) {
            if (!on(mask_content, i))
                continue;
            float v = get_f(x, xt, i);
            if (isnan(v))
                continue;
            if (best_i < 0 || (want_max ? v > best : v < best)) {
                best = v;
                best_i = i;
            }
        }
        if (out)
            out[ev] = best_i < 0 ? empty : best;
        if (arg)
            arg[ev] = best_i < 0 ? -1 : (int32_t)(best_i - i0);
    }
}

/* get_in_offsets (Section III): the n-th masked-in element of each event
 * (n counted from 0 among the elements with mask_content set). n comes from
 * nth[ev] if nth is given, else nth_scalar. Missing (n < 0 or too few
 * elements): out = dflt, idx = -1. idx is the element's local index. */
void oracle_get_in_offsets(const void *x, int xt, const void *off, int ot, int64_t n,
                           const int32_t *nth, int32_t nth_scalar,
                           const uint8_t *mask_rows, const uint8_t *mask_content,
                           float dflt, float *out, int32_t *idx)
{
    for (int64_t ev = 0; ev < n; ev++) {
        if (!on(mask_rows, ev))
            continue;
        int64_t want = nth ? nth[ev] : nth_scalar;
        int64_t i0 = get_off(off, ot, ev), i1 = get_off(off, ot, ev + 1);
        int64_t seen = 0, found = -1;
        for (int64_t i = i0; i < i1 && want >= 0; i++) {
            if (!on(mask_content, i))
                continue;
            if (seen == want) {
                found = i;
                break;
            }
            seen++;
        }
        if (out)
            out[ev] = found < 0 ? dflt : get_f(x, xt, found);
        if (idx)
            idx[ev] = found < 0 ? -1 : (int32_t)(found - i0);
    }
}

/* set_in_offsets (Section III): set the n-th masked-in element of each event
 * to value; events without such an element are unchanged. Content is uint8
 * (a mask) or float32, selected by xt. */
void oracle_set_in_offsets(void *x, int xt, const void *off, int ot, int64_t n,
                           const int32_t *nth, int32_t nth_scalar,
                           const uint8_t *mask_rows, const uint8_t *mask_content, double value)
{
    for (int64_t ev = 0; ev < n; ev++) {
        if (!on(mask_rows, ev))
            continue;
        int64_t want = nth ? nth[ev] : nth_scalar;
        int64_t i0 = get_off(off, ot, ev), i1 = get_off(off, ot, ev + 1);
        int64_t seen = 0;
        for (int64_t i = i0; i < i1 && want >= 0; i++) {
            if (!on(mask_content, i))
                continue;
            if (seen == want) {
                if (xt == OR_U8)
                    ((uint8_t *)x)[i] = (uint8_t)value;
                else
                    ((float *)x)[i] = (float)value;
                break;
            }
            seen++;
        }
    }
}

/* Elementwise object selection: out[i] = in[i] && lo < v && v < hi with
 * v = x[i] * scale (one FP32 multiply) or |x[i] * scale| when use_abs. */
void oracle_select_range(const void *x, int xt, int64_t m, float scale, float lo, float hi,
                         int use_abs, const uint8_t *mask_in, uint8_t *mask_out)
{
    for (int64_t i = 0; i < m; i++) {
        float v = get_f(x, xt, i) * scale;
        if (use_abs)
            v = fabsf(v);
        mask_out[i] = (uint8_t)(on(mask_in, i) && v > lo && v < hi);
    }
}

/* Elementwise scaling: out[i] = x[i] * s in FP32 (jet-pt scale variation). */
void oracle_scale(const void *x, int xt, int64_t m, float s, float *out)
{
    for (int64_t i = 0; i < m; i++)
        out[i] = get_f(x, xt, i) * s;
}

/* ---------------------------------------------------------------------------
 * Delta R masking (mask_deltar_first, Section III)
 * ------------------------------------------------------------------------- */

#define OR_PI_F ((float)3.14159265358979)
#define OR_TWO_PI_F ((float)6.28318530717959)

/* Delta R^2 = Delta eta^2 + Delta phi^2 in FP32, Delta phi brought into
 * [-pi, pi] by one shift of 2 pi; two rounded products and one rounded sum. */
static float dr2_f32(float eta1, float phi1, float eta2, float phi2)
{
    float deta = eta1 - eta2;
    float dphi = phi1 - phi2;
    if (dphi > OR_PI_F)
        dphi = dphi - OR_TWO_PI_F;
    else if (dphi < -OR_PI_F)
        dphi = dphi + OR_TWO_PI_F;
    float a = deta * deta;
    float b = dphi * dphi;
    return a + b;
}

float oracle_dr2(float eta1, float phi1, float eta2, float phi2)
{
    return dr2_f32(eta1, phi1, eta2, phi2);
}

/* mask1_out[i] = mask1_in[i] and no masked-in object j of collection 2 in the
 * same event has Delta R^2(i, j) < dr2_cut. Events with mask_rows unset are
 * untouched. */
void oracle_mask_deltar(const void *eta1, const void *phi1, int t1, const void *off1,
                        const void *eta2, const void *phi2, int t2, const void *off2, int ot,
                        int64_t n, const uint8_t *mask_rows, const uint8_t *mask1_in,
                        const uint8_t *mask2, float dr2_cut, uint8_t *mask1_out)
{
    for (int64_t ev = 0; ev < n; ev++) {
        if (!on(mask_rows, ev))
            continue;
        int64_t a0 = get_off(off1, ot, ev), a1 = get_off(off1, ot, ev + 1);
        int64_t b0 = get_off(off2, ot, ev), b1 = get_off(off2, ot, ev + 1);
        for (int64_t i = a0; i < a1; i++) {
            int keep = on(mask1_in, i);
            for (int64_t j = b0; j < b1 && keep; j++) {
                if (!on(mask2, j))
                    continue;
                float d = dr2_f32(get_f(eta1, t1, i), get_f(phi1, t1, i),
                                  get_f(eta2, t2, j), get_f(phi2, t2, j));
                if (d < dr2_cut)
                    keep = 0;
            }
            mask1_out[i] = (uint8_t)keep;
        }
    }
}

/* ---------------------------------------------------------------------------
 * Histograms (fill_histogram, Section III)
 * ------------------------------------------------------------------------- */

/* Bin of v for edges e[0..nbins]: 0 below e[0], nbins+1 at or above
 * e[nbins], else the b with e[b-1] <= v < e[b]. Linear scan. NaN -> -1. */
static int bin_of(double v, const float *e, int nbins)
{
    if (isnan(v))
        return -1;
    if (v < (double)e[0])
        return 0;
    if (v >= (double)e[nbins])
        return nbins + 1;
    for (int b = 1; b <= nbins; b++)
        if (v < (double)e[b])
            return b;
    return nbins + 1;
}

int oracle_bin_of(double v, const float *edges, int nbins) { return bin_of(v, edges, nbins); }

/* counts[b] += 1, sumw[b] += w, sumw2[b] += w*w for every element with mask
 * set and a non-NaN value (w = 1 without weights). Accumulates. */
void oracle_fill_histogram(const void *x, int xt, const float *w, const uint8_t *mask, int64_t m,
                           const float *edges, int nbins, uint64_t *counts, double *sumw,
                           double *sumw2)
{
    for (int64_t i = 0; i < m; i++) {
        if (!on(mask, i))
            continue;
        int b = bin_of((double)get_f(x, xt, i), edges, nbins);
        if (b < 0)
            continue;
        double wi = w ? (double)w[i] : 1.0;
        counts[b] += 1;
        if (sumw)
            sumw[b] += wi;
        if (sumw2)
            sumw2[b] += wi * wi;
    }
}

/* Histogram over several variables (Section III notes that the fill
 * extends to more dimensions). Axis d bins x[d][i] exactly as bin_of does
 * (nbins[d] + 2 bins with under- and overflow); the cell of element i is
 * the row-major index of (b_0, ..., b_{ndim-1}), axis 0 slowest. Elements
 * with mask unset or a NaN on any axis are not filled. Accumulates. */
void oracle_fill_histogram_nd(int ndim, const void *const *x, const int *xt, const float *const *edges,
                              const int *nbins, const float *w, const uint8_t *mask, int64_t m,
                              uint64_t *counts, double *sumw, double *sumw2)
{
    for (int64_t i = 0; i < m; i++) {
        if (!on(mask, i))
            continue;
        int64_t cell = 0;
        int skip = 0;
        for (int d = 0; d < ndim; d++) {
            int b = bin_of((double)get_f(x[d], xt[d], i), edges[d], nbins[d]);
            if (b < 0) {
                skip = 1;
                break;
            }
            cell = cell * (nbins[d] + 2) + b;
        }
        if (skip)
            continue;
        double wi = w ? (double)w[i] : 1.0;
        counts[cell] += 1;
        if (sumw)
            sumw[cell] += wi;
        if (sumw2)
            sumw2[cell] += wi * wi;
    }
}

/* ---------------------------------------------------------------------------
 * Invariant masses (Section IV: pair and triplet candidates), FP64
 * ------------------------------------------------------------------------- */

typedef struct { double px, py, pz, e; } p4_t;

/* Four-momentum from (pt, eta, phi, m): px = pt cos phi, py = pt sin phi,
 * pz = pt sinh eta, E = sqrt(|p|^2 + m^2). */
static p4_t p4_of(double pt, double eta, double phi, double m)
{
    p4_t v;
    v.px = pt * cos(phi);
    v.py = pt * sin(phi);
    v.pz = pt * sinh(eta);
    v.e = sqrt(v.px * v.px + v.py * v.py + v.pz * v.pz + m * m);
    return v;
}

static p4_t p4_add(p4_t a, p4_t b)
{
    p4_t s = {a.px + b.px, a.py + b.py, a.pz + b.pz, a.e + b.e};
    return s;
}

/* m = sqrt(max(0, E^2 - |p|^2)) of a four-momentum. */
static double p4_mass(p4_t v)
{
    double m2 = v.e * v.e - (v.px * v.px + v.py * v.py + v.pz * v.pz);
    return sqrt(m2 < 0.0 ? 0.0 : m2);   /* rounding below 0 clamps; NaN stays NaN */
}

double oracle_mass2(double pt1, double eta1, double phi1, double m1,
                    double pt2, double eta2, double phi2, double m2)
{
    return p4_mass(p4_add(p4_of(pt1, eta1, phi1, m1), p4_of(pt2, eta2, phi2, m2)));
}

double oracle_mass3(const double *pt, const double *eta, const double *phi, const double *m)
{
    p4_t s = p4_of(pt[0], eta[0], phi[0], m[0]);
    s = p4_add(s, p4_of(pt[1], eta[1], phi[1], m[1]));
    s = p4_add(s, p4_of(pt[2], eta[2], phi[2], m[2]));
    return p4_mass(s);
}

/* Pair mass of the objects at local indices ia[ev], ib[ev] of each event;
 * NaN if either index is negative or out of the event. */
void oracle_pair_mass(const void *pt, const void *eta, const void *phi, const void *mass, int t,
                      const void *off, int ot, int64_t n, const int32_t *ia, const int32_t *ib,
                      const uint8_t *mask_rows, double *out)
{
    for (int64_t ev = 0; ev < n; ev++) {
        if (!on(mask_rows, ev))
            continue;
        int64_t i0 = get_off(off, ot, ev), i1 = get_off(off, ot, ev + 1);
        int64_t a = ia[ev], b = ib[ev];
        if (a < 0 || b < 0 || a >= i1 - i0 || b >= i1 - i0) {
            out[ev] = NAN;
            continue;
        }
        a += i0;
        b += i0;
        out[ev] = oracle_mass2(get_f(pt, t, a), get_f(eta, t, a), get_f(phi, t, a), get_f(mass, t, a),
                               get_f(pt, t, b), get_f(eta, t, b), get_f(phi, t, b), get_f(mass, t, b));
    }
}

/* Trijet choice for one event: over all triplets i<j<k of the listed
 * objects, maximise |sum of transverse momentum vectors|^2 (FP64); ties go
 * to the first triplet in lexicographic order. Returns the number of
 * triplets; writes the chosen positions (into the list), the runner-up
 * positions and both ranking values. */
static int64_t trijet_choose(int64_t cnt, const double *pt, const double *phi, int best[3],
                             int second[3], double *best_v, double *second_v)
{
    int64_t ntrip = 0;
    *best_v = -1.0;
    *second_v = -1.0;
    best[0] = best[1] = best[2] = -1;
    second[0] = second[1] = second[2] = -1;
    for (int64_t i = 0; i < cnt; i++)
        for (int64_t j = i + 1; j < cnt; j++)
            for (int64_t k = j + 1; k < cnt; k++) {
                double sx = pt[i] * cos(phi[i]) + pt[j] * cos(phi[j]) + pt[k] * cos(phi[k]);
                double sy = pt[i] * sin(phi[i]) + pt[j] * sin(phi[j]) + pt[k] * sin(phi[k]);
                double v = sx * sx + sy * sy;
                ntrip++;
                if (v > *best_v) {
                    *second_v = *best_v;
                    memcpy(second, best, 3 * sizeof(int));
                    *best_v = v;
                    best[0] = (int)i; best[1] = (int)j; best[2] = (int)k;
                } else if (v > *second_v) {
                    *second_v = v;
                    second[0] = (int)i; second[1] = (int)j; second[2] = (int)k;
                }
            }
    return ntrip;
}

/* Per event: the triplet of masked-in objects with the largest |sum pT|,
 * its mass (FP64), its |sum pT|, the local indices, and the relative gap
 * (best - runner-up) / best of the ranking value (+inf with one triplet).
 * Fewer than three objects: mass = pt = NaN, indices -1. */
void oracle_max_pt_trijet(const void *pt, const void *eta, const void *phi, const void *mass, int t,
                          const void *off, int ot, int64_t n, const uint8_t *mask_rows,
                          const uint8_t *mask_content, double *out_mass, double *out_pt,
                          int32_t *out_idx3, double *out_gap)
{
    for (int64_t ev = 0; ev < n; ev++) {
        if (!on(mask_rows, ev))
            continue;
        int64_t i0 = get_off(off, ot, ev), i1 = get_off(off, ot, ev + 1);
        int64_t cnt = 0;
        for (int64_t i = i0; i < i1; i++)
            cnt += on(mask_content, i);
        double *vpt = malloc((size_t)(cnt + 1) * sizeof(double));
        double *veta = malloc((size_t)(cnt + 1) * sizeof(double));
        double *vphi = malloc((size_t)(cnt + 1) * sizeof(double));
        double *vm = malloc((size_t)(cnt + 1) * sizeof(double));
        int64_t *loc = malloc((size_t)(cnt + 1) * sizeof(int64_t));
        int64_t c = 0;
        for (int64_t i = i0; i < i1; i++) {
            if (!on(mask_content, i))
                continue;
            vpt[c] = get_f(pt, t, i);
            veta[c] = get_f(eta, t, i);
            vphi[c] = get_f(phi, t, i);
            vm[c] = get_f(mass, t, i);
            loc[c] = i - i0;
            c++;
        }
        int best[3], second[3];
        double bv, sv;
        int64_t ntrip = trijet_choose(cnt, vpt, vphi, best, second, &bv, &sv);
        if (ntrip == 0 || best[0] < 0) {   /* no triplet, or none with a comparable (non-NaN) value */
            if (out_mass) out_mass[ev] = NAN;
            if (out_pt) out_pt[ev] = NAN;
            if (out_idx3) out_idx3[3 * ev] = out_idx3[3 * ev + 1] = out_idx3[3 * ev + 2] = -1;
            if (out_gap) out_gap[ev] = INFINITY;
        } else {
            double p3[3] = {vpt[best[0]], vpt[best[1]], vpt[best[2]]};
            double e3[3] = {veta[best[0]], veta[best[1]], veta[best[2]]};
            double f3[3] = {vphi[best[0]], vphi[best[1]], vphi[best[2]]};
            double m3[3] = {vm[best[0]], vm[best[1]], vm[best[2]]};
            if (out_mass) out_mass[ev] = oracle_mass3(p3, e3, f3, m3);
            if (out_pt) out_pt[ev] = sqrt(bv);
            if (out_idx3) {
                out_idx3[3 * ev] = (int32_t)loc[best[0]];
                out_idx3[3 * ev + 1] = (int32_t)loc[best[1]];
                out_idx3[3 * ev + 2] = (int32_t)loc[best[2]];
            }
            if (out_gap) out_gap[ev] = ntrip > 1 ? (bv - sv) / bv : INFINITY;
        }
        free(vpt); free(veta); free(vphi); free(vm); free(loc);
    }
}

/* ---------------------------------------------------------------------------
 * Top-quark candidate (Section IV: the jet triplet with invariant mass
 * closest to the top mass), FP64
 * ------------------------------------------------------------------------- */

/* Per event with mask_rows set: among triplets i<j<k of masked-in objects,
 * the one whose mass (FP64) is closest to target; ties go to the first in
 * lexicographic order. out_mass its mass, out_idx3 the local indices,
 * out_gap = |m_runner_up - target| - |m_best - target| (+inf with one
 * triplet). Fewer than three objects: NaN and -1 -1 -1. */
void oracle_trijet_closest_mass(const void *pt, const void *eta, const void *phi, const void *mass, int t,
                                const void *off, int ot, int64_t n, const uint8_t *mask_rows,
                                const uint8_t *mask_content, double target, double *out_mass,
                                int32_t *out_idx3, double *out_gap)
{
    for (int64_t ev = 0; ev < n; ev++) {
        if (!on(mask_rows, ev))
            continue;
        int64_t i0 = get_off(off, ot, ev), i1 = get_off(off, ot, ev + 1);
        double best_d = INFINITY, second_d = INFINITY, best_m = NAN;
        int64_t bi = -1, bj = -1, bk = -1, ntrip = 0;
        for (int64_t i = i0; i < i1; i++) {
            if (!on(mask_content, i))
                continue;
            for (int64_t j = i + 1; j < i1; j++) {
                if (!on(mask_content, j))
                    continue;
                for (int64_t k = j + 1; k < i1; k++) {
                    if (!on(mask_content, k))
                        continue;
                    double p3[3] = {get_f(pt, t, i), get_f(pt, t, j), get_f(pt, t, k)};
                    double e3[3] = {get_f(eta, t, i), get_f(eta, t, j), get_f(eta, t, k)};
                    double f3[3] = {get_f(phi, t, i), get_f(phi, t, j), get_f(phi, t, k)};
                    double m3[3] = {get_f(mass, t, i), get_f(mass, t, j), get_f(mass, t, k)};
                    double m = oracle_mass3(p3, e3, f3, m3);
                    double d = fabs(m - target);
                    ntrip++;
                    if (d < best_d) {
                        second_d = best_d;
                        best_d = d;
                        best_m = m;
                        bi = i - i0; bj = j - i0; bk = k - i0;
                    } else if (d < second_d) {
                        second_d = d;
                    }
                }
            }
        }
        if (out_mass) out_mass[ev] = ntrip ? best_m : NAN;
        if (out_idx3) {
            out_idx3[3 * ev] = (int32_t)bi;
            out_idx3[3 * ev + 1] = (int32_t)bj;
            out_idx3[3 * ev + 2] = (int32_t)bk;
        }
        if (out_gap) out_gap[ev] = ntrip > 1 ? second_d - best_d : INFINITY;
    }
}

/* ---------------------------------------------------------------------------
 * select_opposite_sign_muons (Section III, specialised kernels)
 * ------------------------------------------------------------------------- */

/* Per event with mask_rows set: over the masked-in objects in stored order
 * (the data's pt order), the first i that has a later masked-in j of
 * opposite charge (charge[i] * charge[j] < 0), with the first such j.
 * mask_out is 1 for those two and 0 for every other object of the event
 * (all 0 without such a pair). Events with mask_rows unset are untouched. */
void oracle_select_opposite_sign(const int8_t *charge, const void *off, int ot, int64_t n,
                                 const uint8_t *mask_rows, const uint8_t *mask_in, uint8_t *mask_out)
{
    for (int64_t ev = 0; ev < n; ev++) {
        if (!on(mask_rows, ev))
            continue;
        int64_t i0 = get_off(off, ot, ev), i1 = get_off(off, ot, ev + 1);
        int64_t a = -1, b = -1;
        for (int64_t i = i0; i < i1 && a < 0; i++) {
            if (!on(mask_in, i))
                continue;
            for (int64_t j = i + 1; j < i1; j++) {
                if (on(mask_in, j) && (int)charge[i] * (int)charge[j] < 0) {
                    a = i;
                    b = j;
                    break;
                }
            }
        }
        for (int64_t i = i0; i < i1; i++)
            mask_out[i] = (uint8_t)(i == a || i == b);
    }
}

/* ---------------------------------------------------------------------------
 * get_bin_contents (Section III kernel list): histogram lookup
 * ------------------------------------------------------------------------- */

/* Linear interpolation of the contents (nbins+2 entries, with under- and
 * overflow) between the centres c_b = (edges[b-1] + edges[b]) / 2 of
 * neighbouring in-range bins, at a non-NaN v: contents[1] below c_1,
 * contents[nbins] at or above c_nbins, else with c_b <= v < c_b+1
 * contents[b] + (v - c_b) / (c_b+1 - c_b) * (contents[b+1] - contents[b]),
 * each operation in binary32 rounded as written. */
static float lookup_interp(float v, const float *edges, int nbins, const float *contents)
{
    float c1 = (edges[0] + edges[1]) * 0.5f;
    float cn = (edges[nbins - 1] + edges[nbins]) * 0.5f;
    if (nbins == 1 || v < c1)
        return contents[1];
    if (v >= cn)
        return contents[nbins];
    for (int b = 1; b < nbins; b++) {
        float cb = (edges[b - 1] + edges[b]) * 0.5f;
        float cb1 = (edges[b] + edges[b + 1]) * 0.5f;
        if (v >= cb && v < cb1) {
            float tt = (v - cb) / (cb1 - cb);
            float d = contents[b + 1] - contents[b];
            float prod = tt * d;
            return contents[b] + prod;
        }
    }
    return contents[nbins];
}

/* out[j] = contents[b] with b the bin of x[j] (bin_of; contents has nbins+2
 * entries, under- and overflow included); NaN for NaN input. With
 * interpolate set: linear interpolation between the contents of
 * neighbouring in-range bins at their centres c_b = (e[b-1] + e[b]) * 0.5,
 * clamped to the first and last in-range bin outside [c_1, c_nbins]. All in
 * binary32, every operation rounded (no contraction): for c_b <= v < c_b+1,
 * t = (v - c_b) / (c_b+1 - c_b) and out = y_b + t * (y_b+1 - y_b). */
void oracle_get_bin_contents(const void *x, int xt, int64_t m, const float *edges, int nbins,
                             const float *contents, int interpolate, float *out)
{
    for (int64_t j = 0; j < m; j++) {
        float v = get_f(x, xt, j);
        if (isnan(v)) {
            out[j] = NAN;
            continue;
        }
        if (!interpolate) {
            out[j] = contents[bin_of((double)v, edges, nbins)];
            continue;
        }
        out[j] = lookup_interp(v, edges, nbins, contents);
    }
}

/* ---------------------------------------------------------------------------
 * The benchmark chain (Section IV), one plain loop per variation and event
 * ------------------------------------------------------------------------- */

#define OR_NVARS 20

typedef struct {
    int64_t n_events;
    int offset_type;
    const void *jet_off, *mu_off, *el_off;
    int kin_type;   /* pt, eta, phi, mass of all collections */
    int btag_type;
    const void *jet_pt, *jet_eta, *jet_phi, *jet_mass, *jet_btag;
    const void *mu_pt, *mu_eta, *mu_phi;
    const float *mu_iso;
    const uint8_t *mu_tight;
    const void *el_pt, *el_eta, *el_phi;
    const float *el_iso;
    const uint8_t *el_tight;
    const float *weight;
} oracle_batch;

typedef struct {
    float lep_pt_min, lep_abseta_max, lep_iso_max;
    float jet_pt_min, jet_abseta_max, dr2_cut, btag_min;
    int n_var;
    const float *scales;     /* [n_var] */
    int n_hist;              /* must be 20 */
    const int32_t *nbins;    /* [n_hist] */
    const float *edges;      /* concatenated, nbins[h] + 1 per histogram */
    /* jet-energy corrections (NULL jec_contents: the scales): per variation
     * a table of (jec_neta + 2) rows, one per eta bin with under- and
     * overflow, of jec_npt + 2 contents over the pt bins */
    int jec_neta, jec_npt;
    const float *jec_eta_edges, *jec_pt_edges;
    const float *jec_contents;   /* [n_var][jec_neta + 2][jec_npt + 2] */
} oracle_config;

/* The jet-energy correction of variation k for a jet (pt, eta) (Section IV:
 * corrections looked up in binned tables, linearly interpolated): the row of
 * the jet's eta bin (bin_of, under- and overflow rows included) read at the
 * jet's pt by lookup_interp; NaN for a NaN pt or eta. */
static float jec_factor(const oracle_config *c, int k, float pt, float eta)
{
    int row = bin_of((double)eta, c->jec_eta_edges, c->jec_neta);
    if (row < 0 || isnan(pt))
        return NAN;
    const float *r = c->jec_contents + ((int64_t)k * (c->jec_neta + 2) + row) * (c->jec_npt + 2);
    return lookup_interp(pt, c->jec_pt_edges, c->jec_npt, r);
}

typedef struct {
    uint64_t *counts;        /* [n_var][total bins] */
    double *sumw, *sumw2;    /* [n_var][total bins]; sumw2 may be NULL */
    uint8_t *ev_pass;        /* [n_var][N] or NULL */
    int32_t *ev_nlep;        /* [N] or NULL */
    int32_t *ev_njet, *ev_nb;/* [n_var][N] or NULL */
    int32_t *ev_idx;         /* [n_var][5][N]: lead, sublead, trijet i, j, k */
    double *ev_vars;         /* [n_var][20][N], NaN where undefined */
    double *ev_gap;          /* [n_var][N] trijet ranking gap */
    int32_t *ev_idx2;        /* [n_var][3][N] runner-up triplet */
} oracle_outputs;

/* The event chain for one event and one jet-pt scale s:
 *  1. leptons (muons, electrons): selected if pt > lep_pt_min, |eta| <
 *     lep_abseta_max, tight, iso < lep_iso_max; n_lep counts both flavours;
 *     "the lepton" is the first selected muon, else the first selected
 *     electron;
 *  2. jets: pt_s = pt * s (FP32); selected if pt_s > jet_pt_min,
 *     |eta| < jet_abseta_max and Delta R^2 >= dr2_cut to every selected
 *     lepton;
 *  3. n_jet, n_b (btag > btag_min) by summing masks; pass if n_lep == 1,
 *     n_jet >= 2, n_b >= 1;
 *  4. HT = FP32 sum of pt_s over selected jets in element order; leading and
 *     sub-leading selected jets by pt_s (first occurrence wins ties); max
 *     btag; sum of selected-jet masses (FP32, element order); ST = HT +
 *     lepton pt (FP32);
 *  5. m_jj of the two leading jets and the max-|sum pT| trijet (FP64);
 *  6. passing events fill the 20 weighted histograms (trijet ones only with
 *     n_jet >= 3). */
void oracle_run_chain(const oracle_batch *b, const oracle_config *c, oracle_outputs *o)
{
    const int64_t n = b->n_events;
    const int kt = b->kin_type, ot = b->offset_type;
    int64_t total_bins = 0;
    int64_t hoff[OR_NVARS];
    const float *hedge[OR_NVARS];
    {
        const float *e = c->edges;
        for (int h = 0; h < c->n_hist && h < OR_NVARS; h++) {
            hoff[h] = total_bins;
            hedge[h] = e;
            total_bins += c->nbins[h] + 2;
            e += c->nbins[h] + 1;
        }
    }
    int64_t jcap = 16;
    double *jpt = malloc(jcap * sizeof(double)), *jphi = malloc(jcap * sizeof(double));
    double *jeta = malloc(jcap * sizeof(double)), *jm = malloc(jcap * sizeof(double));
    int64_t *jloc = malloc(jcap * sizeof(int64_t));

    for (int k = 0; k < c->n_var; k++) {
        const float s = c->scales[k];
        for (int64_t ev = 0; ev < n; ev++) {
            /* 1. leptons */
            int32_t nlep = 0;
            int have_lep = 0;
            float lpt = NAN, leta = NAN, lphi = NAN, liso = NAN;
            for (int flav = 0; flav < 2; flav++) {
                const void *off = flav == 0 ? b->mu_off : b->el_off;
                const void *pt = flav == 0 ? b->mu_pt : b->el_pt;
                const void *eta = flav == 0 ? b->mu_eta : b->el_eta;
                const void *phi = flav == 0 ? b->mu_phi : b->el_phi;
                const float *iso = flav == 0 ? b->mu_iso : b->el_iso;
                const uint8_t *tight = flav == 0 ? b->mu_tight : b->el_tight;
                for (int64_t i = get_off(off, ot, ev); i < get_off(off, ot, ev + 1); i++) {
                    float p = get_f(pt, kt, i), e = get_f(eta, kt, i);
                    int sel = p > c->lep_pt_min && fabsf(e) < c->lep_abseta_max && tight[i] != 0 &&
                              iso[i] < c->lep_iso_max;
                    if (!sel)
                        continue;
                    nlep++;
                    if (!have_lep) {
                        have_lep = 1;
                        lpt = p; leta = e; lphi = get_f(phi, kt, i); liso = iso[i];
                    }
                }
            }
            /* 2. jets */
            const int64_t j0 = get_off(b->jet_off, ot, ev), j1 = get_off(b->jet_off, ot, ev + 1);
            if (j1 - j0 > jcap) {
                jcap = j1 - j0;
                jpt = realloc(jpt, jcap * sizeof(double));
                jphi = realloc(jphi, jcap * sizeof(double));
                jeta = realloc(jeta, jcap * sizeof(double));
                jm = realloc(jm, jcap * sizeof(double));
                jloc = realloc(jloc, jcap * sizeof(int64_t));
            }
            int32_t njet = 0, nb = 0;
            float ht = 0.0f, summ = 0.0f;
            int64_t lead = -1, sub = -1, lead_q = -1;
            float lead_pt = 0.0f, sub_pt = 0.0f, max_bt = 0.0f;
            int have_bt = 0;
            for (int64_t i = j0; i < j1; i++) {
                float eta = get_f(b->jet_eta, kt, i), phi = get_f(b->jet_phi, kt, i);
                float pt = get_f(b->jet_pt, kt, i);
                /* the variation's jet pt: scaled, or corrected by its table */
                float ptk = c->jec_contents ? pt * jec_factor(c, k, pt, eta) : pt * s;
                int sel = ptk > c->jet_pt_min && fabsf(eta) < c->jet_abseta_max;
                for (int flav = 0; flav < 2 && sel; flav++) {
                    const void *off = flav == 0 ? b->mu_off : b->el_off;
                    const void *pt = flav == 0 ? b->mu_pt : b->el_pt;
                    const void *leta_p = flav == 0 ? b->mu_eta : b->el_eta;
                    const void *lphi_p = flav == 0 ? b->mu_phi : b->el_phi;
                    const float *iso = flav == 0 ? b->mu_iso : b->el_iso;
                    const uint8_t *tight = flav == 0 ? b->mu_tight : b->el_tight;
                    for (int64_t l = get_off(off, ot, ev); l < get_off(off, ot, ev + 1); l++) {
                        float p = get_f(pt, kt, l), e = get_f(leta_p, kt, l);
                        int lsel = p > c->lep_pt_min && fabsf(e) < c->lep_abseta_max &&
                                   tight[l] != 0 && iso[l] < c->lep_iso_max;
                        if (lsel && dr2_f32(eta, phi, e, get_f(lphi_p, kt, l)) < c->dr2_cut)
                            sel = 0;
                    }
                }
                if (!sel)
                    continue;
                float bt = get_f(b->jet_btag, b->btag_type, i);
                float m = get_f(b->jet_mass, kt, i);
                jpt[njet] = ptk; jeta[njet] = eta; jphi[njet] = phi; jm[njet] = m;
                jloc[njet] = i - j0;
                if (bt > c->btag_min)
                    nb++;
                ht += ptk;
                summ += m;
                if (lead < 0 || ptk > lead_pt) {
                    lead = i; lead_pt = ptk; lead_q = njet;
                }
                if (!isnan(bt) && (!have_bt || bt > max_bt)) {
                    have_bt = 1; max_bt = bt;
                }
                njet++;
            }
            /* sub-leading: the same scan over the selected jets without the leading one */
            for (int64_t q = 0; q < njet; q++) {
                if (q == lead_q)
                    continue;
                float ptk = (float)jpt[q];
                if (sub < 0 || ptk > sub_pt) {
                    sub = j0 + jloc[q]; sub_pt = ptk;
                }
            }
            const int pass = nlep == 1 && njet >= 2 && nb >= 1;

            /* 5. masses */
            double vars[OR_NVARS];
            for (int h = 0; h < OR_NVARS; h++)
                vars[h] = NAN;
            int tri[3] = {-1, -1, -1}, tri2[3] = {-1, -1, -1};
            double gap = INFINITY;
            vars[0] = ht;
            vars[8] = njet;
            vars[9] = nb;
            vars[18] = summ;
            vars[19] = b->weight[ev];
            if (lead >= 0) {
                vars[1] = lead_pt;
                vars[2] = get_f(b->jet_eta, kt, lead);
                vars[3] = get_f(b->jet_phi, kt, lead);
                vars[4] = get_f(b->jet_mass, kt, lead);
                vars[5] = get_f(b->jet_btag, b->btag_type, lead);
            }
            if (have_bt)
                vars[10] = max_bt;
            if (sub >= 0) {
                vars[6] = sub_pt;
                vars[7] = oracle_mass2(lead_pt, get_f(b->jet_eta, kt, lead), get_f(b->jet_phi, kt, lead),
                                       get_f(b->jet_mass, kt, lead), sub_pt, get_f(b->jet_eta, kt, sub),
                                       get_f(b->jet_phi, kt, sub), get_f(b->jet_mass, kt, sub));
            }
            if (njet >= 3) {
                double bv, sv;
                int64_t ntrip = trijet_choose(njet, jpt, jphi, tri, tri2, &bv, &sv);
                /* a NaN ranking value never wins: with none comparable there
                 * is no trijet (its variables stay NaN and are not filled) */
                if (tri[0] >= 0) {
                    double p3[3], e3[3], f3[3], m3[3];
                    for (int q = 0; q < 3; q++) {
                        p3[q] = jpt[tri[q]]; e3[q] = jeta[tri[q]]; f3[q] = jphi[tri[q]]; m3[q] = jm[tri[q]];
                    }
                    vars[11] = oracle_mass3(p3, e3, f3, m3);
                    vars[12] = sqrt(bv);
                    gap = ntrip > 1 ? (bv - sv) / bv : INFINITY;
                }
            }
            if (have_lep) {
                vars[13] = lpt;
                vars[14] = leta;
                vars[15] = lphi;
                vars[16] = liso;
                vars[17] = ht + lpt;   /* FP32 sum: both operands are float */
            }

            /* outputs */
            if (o->ev_pass) o->ev_pass[(int64_t)k * n + ev] = (uint8_t)pass;
            if (o->ev_nlep && k == 0) o->ev_nlep[ev] = nlep;
            if (o->ev_njet) o->ev_njet[(int64_t)k * n + ev] = njet;
            if (o->ev_nb) o->ev_nb[(int64_t)k * n + ev] = nb;
            if (o->ev_idx) {
                int32_t *ix = o->ev_idx + (int64_t)k * 5 * n;
                ix[0 * n + ev] = lead < 0 ? -1 : (int32_t)(lead - j0);
                ix[1 * n + ev] = sub < 0 ? -1 : (int32_t)(sub - j0);
                for (int q = 0; q < 3; q++)
                    ix[(2 + q) * n + ev] = tri[q] < 0 ? -1 : (int32_t)jloc[tri[q]];
            }
            if (o->ev_idx2) {
                int32_t *ix = o->ev_idx2 + (int64_t)k * 3 * n;
                for (int q = 0; q < 3; q++)
                    ix[q * n + ev] = tri2[q] < 0 ? -1 : (int32_t)jloc[tri2[q]];
            }
            if (o->ev_vars)
                for (int h = 0; h < OR_NVARS; h++)
                    o->ev_vars[((int64_t)k * OR_NVARS + h) * n + ev] = vars[h];
            if (o->ev_gap) o->ev_gap[(int64_t)k * n + ev] = gap;

            /* 6. histograms */
            if (!pass)
                continue;
            const double w = b->weight[ev];
            for (int h = 0; h < OR_NVARS && h < c->n_hist; h++) {
                if ((h == 11 || h == 12) && njet < 3)
                    continue;
                int bin = bin_of(vars[h], hedge[h], c->nbins[h]);
                if (bin < 0)
                    continue;
                int64_t at = (int64_t)k * total_bins + hoff[h] + bin;
                o->counts[at] += 1;
                o->sumw[at] += w;
                if (o->sumw2)
                    o->sumw2[at] += w * w;
            }
        }
    }
    free(jpt); free(jphi); free(jeta); free(jm); free(jloc);
}
