/*
 * hepacc: GPU kernels for columnar (jagged-array) collider event data.
 *
 * Operations from "Processing Columnar Collider Data with GPU-Accelerated
 * Kernels" (Pata & Spiropulu, arXiv:1906.06242), written for NVIDIA GB300
 * (sm_103a).
 *
 * Data model (Section II). N events with M objects of one collection are an
 * offsets array of N+1 entries plus one flat content array of M entries per
 * feature; event i owns elements [offsets[i], offsets[i+1]). offsets[0] may be
 * non-zero (a slice of a larger batch); offsets must be non-decreasing.
 * Event masks (mask_rows, N bytes) and content masks (mask_content, M bytes)
 * are uint8 arrays, non-zero meaning "selected" (Section III); a NULL mask
 * selects everything.
 *
 * Conventions for every call below.
 *  - Pointers to arrays are DEVICE pointers owned by the caller, unless the
 *    call says otherwise; the library keeps no reference after the call
 *    returns and frees nothing. Per-operation calls allocate no memory.
 *  - Calls are asynchronous: they validate their scalar arguments on the
 *    host, enqueue work on `stream` (NULL = the legacy default stream) and
 *    return. A non-OK status means nothing was enqueued, except
 *    HEPACC_ERR_CUDA, returned when a launch failed.
 *  - Content columns are read in whole 16-byte-aligned chunks: up to 15
 *    bytes before the first and after the last element of an event block
 *    may be read (never written, never used). Such a chunk never leaves the
 *    memory page of a valid element.
 *  - Local indices are 0-based inside the event; -1 means "none".
 *  - hepacc_last_error() describes the most recent failing call made on the
 *    calling host thread.
 */
#ifndef HEPACC_H
#define HEPACC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t (the runtime's stream handle type). */
typedef struct CUstream_st *hepacc_stream;

typedef enum {
    HEPACC_OK = 0,
    HEPACC_ERR_INVALID_ARG = 1,   /* NULL required pointer, negative size, bad bins ... */
    HEPACC_ERR_DTYPE = 2,         /* unsupported element type for this call */
    HEPACC_ERR_CUDA = 3,          /* a CUDA runtime call or launch failed */
    HEPACC_ERR_OOM = 4,           /* a plan could not allocate its workspace */
    HEPACC_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up */
    HEPACC_ERR_DEVICE_CHECK = 6   /* device-side validation found bad input */
} hepacc_status;

typedef enum {
    HEPACC_F32 = 0,
    HEPACC_F16 = 1,
    HEPACC_BF16 = 2,
    HEPACC_I8 = 3,
    HEPACC_U8 = 4,
    HEPACC_I32 = 5,
    HEPACC_I64 = 6,
    HEPACC_F64 = 7
} hepacc_dtype;

/* ---------------------------------------------------------------------------
 * Library state and diagnostics
 * ------------------------------------------------------------------------- */

/* Version string of the library; static storage. */
const char *hepacc_version(void);

/* Text of the last failing call on this host thread ("" if none); valid until
 * the next failing call on the same thread. */
const char *hepacc_last_error(void);

/* Name of a status code; static storage. */
const char *hepacc_status_string(hepacc_status s);

/* Reads and clears the device error word of the current device, which
 * kernels set when a bounded wait gives up (bit 0) or a device-side check
 * fails (bit 1). Synchronises the device. *flags receives the word. */
hepacc_status hepacc_device_error(uint32_t *flags);

/* Self-test of the bounded-wait path: launches one thread that waits on an
 * mbarrier nothing ever completes, giving up after about limit_cycles SM
 * clocks (1 <= limit_cycles <= 2^31). The kernel then sets bit 0 of the
 * device error word and returns, leaving the context usable; read it with
 * hepacc_device_error(). Asynchronous. */
hepacc_status hepacc_selftest_wait_timeout(int64_t limit_cycles, hepacc_stream stream);

/* Offsets check (Section II layout): offsets[0] >= 0, non-decreasing, and
 * offsets[n_rows] <= content_len. *first_bad (a DEVICE int64) receives the
 * smallest event index i whose offsets[i+1] breaks a rule (-1 if none; -2 if
 * offsets[0] < 0). offsets_type is HEPACC_I32 or HEPACC_I64. Asynchronous. */
hepacc_status hepacc_validate_offsets(const void *offsets, hepacc_dtype offsets_type, int64_t n_rows,
                                      int64_t content_len, int64_t *first_bad, hepacc_stream stream);

/* ---------------------------------------------------------------------------
 * Generic kernels over jagged arrays (Section III)
 * ------------------------------------------------------------------------- */

/* sum_in_offsets (Section III, Listing 1). For every event i with
 * mask_rows[i] set: out[i] += content[j] for each j in [offsets[i],
 * offsets[i+1]) with mask_content[j] set, one element at a time in element
 * order. Events with mask_rows[i] unset keep their value of out[i]; with
 * out zero-filled the result is the plain sum.
 * content_type F32, F16 or BF16: out_type must be F32 and every addition is
 * an IEEE binary32 addition (half inputs widened exactly).
 * content_type U8, I8, I32: out_type I32 or I64 (counting selected objects by
 * summing masks); I64 content needs out_type I64. */
hepacc_status hepacc_sum_in_offsets(const void *content, hepacc_dtype content_type, const void *offsets,
                                    hepacc_dtype offsets_type, int64_t n_rows, const uint8_t *mask_rows,
                                    const uint8_t *mask_content, void *out, hepacc_dtype out_type,
                                    hepacc_stream stream);

/* max_in_offsets / min_in_offsets (Section III). For every event i with
 * mask_rows[i] set: out[i] = the largest (smallest) masked-in non-NaN value,
 * out_arg[i] = its local index (first occurrence on ties); with no such
 * element out[i] = empty_value and out_arg[i] = -1. content_type F32, F16,
 * BF16, U8, I8 or I32 (compared as float). out or out_arg may be NULL (not
 * both). Events with mask_rows[i] unset are untouched. */
hepacc_status hepacc_max_in_offsets(const void *content, hepacc_dtype content_type, const void *offsets,
                                    hepacc_dtype offsets_type, int64_t n_rows, const uint8_t *mask_rows,
                                    const uint8_t *mask_content, float empty_value, float *out,
                                    int32_t *out_arg, hepacc_stream stream);
hepacc_status hepacc_min_in_offsets(const void *content, hepacc_dtype content_type, const void *offsets,
                                    hepacc_dtype offsets_type, int64_t n_rows, const uint8_t *mask_rows,
                                    const uint8_t *mask_content, float empty_value, float *out,
                                    int32_t *out_arg, hepacc_stream stream);

/* get_in_offsets (Section III). For every event i with mask_rows[i] set:
 * the n-th masked-in element (n counted from 0 over elements with
 * mask_content set), n = nth[i] if nth (DEVICE int32[n_rows]) is non-NULL,
 * else nth_scalar. out[i] = its value as float, out_index[i] = its local
 * index; if n < 0 or the event has too few such elements, out[i] =
 * default_value and out_index[i] = -1. Either output may be NULL (not both).
 * content_type as for max_in_offsets. */
hepacc_status hepacc_get_in_offsets(const void *content, hepacc_dtype content_type, const void *offsets,
                                    hepacc_dtype offsets_type, int64_t n_rows, const int32_t *nth,
                                    int32_t nth_scalar, const uint8_t *mask_rows,
                                    const uint8_t *mask_content, float default_value, float *out,
                                    int32_t *out_index, hepacc_stream stream);

/* set_in_offsets (Section III). For every event i with mask_rows[i] set,
 * the n-th masked-in element (as in get_in_offsets) of content is set to
 * value (converted to the content type); events without such an element are
 * unchanged. content_type U8 (a mask, e.g. keep the first two jets) or F32.
 * content is modified in place. */
hepacc_status hepacc_set_in_offsets(void *content, hepacc_dtype content_type, const void *offsets,
                                    hepacc_dtype offsets_type, int64_t n_rows, const int32_t *nth,
                                    int32_t nth_scalar, const uint8_t *mask_rows,
                                    const uint8_t *mask_content, double value, hepacc_stream stream);

/* Object selection by a cut (Section IV: object selection on pt, eta):
 * mask_out[j] = mask_in[j] && lo < v && v < hi for j < n, with
 * v = content[j] * scale as one binary32 product (|v| when use_abs != 0).
 * NaN never passes. content_type F32, F16, BF16, U8, I8 or I32. mask_in may
 * be NULL and may equal mask_out. */
hepacc_status hepacc_select_range(const void *content, hepacc_dtype content_type, int64_t n, float scale,
                                  float lo, float hi, int use_abs, const uint8_t *mask_in,
                                  uint8_t *mask_out, hepacc_stream stream);

/* out[j] = content[j] * scale (one binary32 product) for j < n: a jet
 * energy-scale variation (Section IV). content_type F32, F16 or BF16. */
hepacc_status hepacc_scale(const void *content, hepacc_dtype content_type, int64_t n, float scale,
                           float *out, hepacc_stream stream);

/* ---------------------------------------------------------------------------
 * Specialised kernels (Section III)
 * ------------------------------------------------------------------------- */

/* mask_deltar_first (Section III): for every event i with mask_rows[i] set
 * and every object j of collection 1 in it, mask1_out[j] = mask1_in[j] and
 * no masked-in object k of collection 2 in the same event has
 * Delta R^2 = Delta eta^2 + Delta phi^2 < dr2_cut, with Delta phi folded into
 * [-pi, pi] by one shift of 2 pi and the sum of two rounded binary32
 * squares (no fused multiply-add). Events with mask_rows[i] unset keep
 * mask1_out. Both collections have n_rows events and offsets of the same
 * type; eta/phi of one collection share one type (F32, F16 or BF16).
 * mask1_in, mask2 may be NULL; mask1_out must not alias mask1_in unless
 * equal. */
hepacc_status hepacc_mask_deltar(const void *eta1, const void *phi1, hepacc_dtype type1, const void *offsets1,
                                 const void *eta2, const void *phi2, hepacc_dtype type2, const void *offsets2,
                                 hepacc_dtype offsets_type, int64_t n_rows, const uint8_t *mask_rows,
                                 const uint8_t *mask1_in, const uint8_t *mask2, float dr2_cut,
                                 uint8_t *mask1_out, hepacc_stream stream);

/* fill_histogram (Section III): for j < n with mask[j] set and data[j] not
 * NaN, bin b of data[j] against the binary32 edges[0..nbins] (increasing):
 * b = 0 if v < edges[0], nbins+1 if v >= edges[nbins], else the b with
 * edges[b-1] <= v < edges[b]. Accumulates counts[b] += 1, sumw[b] += w,
 * sumw2[b] += w*w with w = weights[j] (1 if weights is NULL), sums in
 * binary64. counts, sumw have nbins+2 entries; sumw and sumw2 may be NULL.
 * 1 <= nbins <= 65536. data_type F32, F16, BF16, U8, I8 or I32. Accuracy:
 * up to about 250 bins (with sumw2; 740 without) the weights of a block of
 * at most 2^15 elements are summed exactly in integers (w^2 exactly as the
 * sum of two binary32 values) and each block's sums are added in binary64
 * (relative error ~ blocks x 2^-53); weights of magnitude outside
 * [2^-50, 2^63), infinities and NaNs, and larger histograms, are summed in
 * binary64 directly. The order of the binary64 additions is unspecified. */
hepacc_status hepacc_fill_histogram(const void *data, hepacc_dtype data_type, const float *weights,
                                    const uint8_t *mask, int64_t n, const float *edges, int32_t nbins,
                                    uint64_t *counts, double *sumw, double *sumw2, hepacc_stream stream);

/* Histogram over several variables (Section III: the fill extends to more
 * dimensions). ndim in [1, HEPACC_MAX_HIST_DIMS]. Axis d bins data[d][j]
 * (n elements of type data_types[d]: F32, F16, BF16, U8, I8 or I32) against
 * the increasing binary32 edges[d][0..nbins[d]] exactly as
 * hepacc_fill_histogram does, so axis d has nbins[d] + 2 bins with under-
 * and overflow. The cell of element j is the row-major index of
 * (b_0, ..., b_{ndim-1}), axis 0 slowest: ((b_0 (nbins[1]+2) + b_1)
 * (nbins[2]+2) + b_2) ...; counts, sumw and sumw2 have prod_d (nbins[d]+2)
 * <= 2^24 entries (sumw, sumw2 may be NULL), and counts[c] += 1,
 * sumw[c] += w, sumw2[c] += w*w with the accuracy of the one-dimensional
 * fill (exact per block up to about 250 cells with sumw2, 760 without).
 * Elements with mask[j] unset or a NaN on any axis are not filled. data,
 * data_types, edges and nbins are HOST arrays of ndim entries (data[d] and
 * edges[d] are device pointers), read before the call returns.
 * 1 <= nbins[d] <= 65536. */
#define HEPACC_MAX_HIST_DIMS 4
hepacc_status hepacc_fill_histogram_nd(int32_t ndim, const void *const *data, const hepacc_dtype *data_types,
                                       const float *const *edges, const int32_t *nbins, const float *weights,
                                       const uint8_t *mask, int64_t n, uint64_t *counts, double *sumw,
                                       double *sumw2, hepacc_stream stream);

/* Invariant mass of a pair of objects per event (Section IV: high-level
 * variables). For every event i with mask_rows[i] set: out[i] = mass of the
 * sum of the four-momenta of the objects at local indices idx_a[i] and
 * idx_b[i] (from pt, eta, phi, mass), NaN if an index is negative or outside
 * the event. Computed in binary32 through a form without cancellation
 * (relative error below 1e-5). type F32, F16 or BF16 for all four columns. */
hepacc_status hepacc_pair_mass(const void *pt, const void *eta, const void *phi, const void *mass,
                               hepacc_dtype type, const void *offsets, hepacc_dtype offsets_type,
                               int64_t n_rows, const int32_t *idx_a, const int32_t *idx_b,
                               const uint8_t *mask_rows, float *out, hepacc_stream stream);

/* Trijet candidate (Section IV: top quark candidate from a jet triplet).
 * For every event i with mask_rows[i] set: among triplets a<b<c of masked-in
 * objects, the one with the largest |pT_a + pT_b + pT_c| (transverse
 * vectors; first in lexicographic order on ties); out_mass[i] its invariant
 * mass, out_pt[i] that |sum pT|, out_idx3[3i..3i+2] the local indices. Fewer
 * than three objects: NaN, NaN, -1 -1 -1. Any output may be NULL. */
hepacc_status hepacc_max_pt_trijet(const void *pt, const void *eta, const void *phi, const void *mass,
                                   hepacc_dtype type, const void *offsets, hepacc_dtype offsets_type,
                                   int64_t n_rows, const uint8_t *mask_rows, const uint8_t *mask_content,
                                   float *out_mass, float *out_pt, int32_t *out_idx3,
                                   hepacc_stream stream);

/* Top-quark candidate (Section IV: the jet triplet with invariant mass
 * closest to the top mass). For every event i with mask_rows[i] set: among
 * triplets a<b<c of masked-in objects, the one whose mass (binary32,
 * cancellation-free as in hepacc_pair_mass) is closest to target (first in
 * lexicographic order on ties); out_mass[i] its mass, out_idx3[3i..3i+2]
 * its local indices. Fewer than three objects: NaN and -1 -1 -1. Either
 * output may be NULL (not both). */
hepacc_status hepacc_trijet_closest_mass(const void *pt, const void *eta, const void *phi, const void *mass,
                                         hepacc_dtype type, const void *offsets, hepacc_dtype offsets_type,
                                         int64_t n_rows, const uint8_t *mask_rows, const uint8_t *mask_content,
                                         float target, float *out_mass, int32_t *out_idx3, hepacc_stream stream);

/* select_opposite_sign_muons (Section III, specialised kernels). For every
 * event i with mask_rows[i] set: over the objects with mask_in set, in
 * stored order (the pt order of the data), the first object that has a
 * later one of opposite charge (charge_a * charge_b < 0), and the first such
 * partner; mask_out is 1 for those two and 0 for every other object of the
 * event (all 0 without such a pair). Objects of events with mask_rows unset
 * are untouched. charge is int8 (content size); mask_in may be NULL (all
 * objects); mask_out must not alias mask_in. */
hepacc_status hepacc_select_opposite_sign(const int8_t *charge, const void *offsets, hepacc_dtype offsets_type,
                                          int64_t n_rows, const uint8_t *mask_rows, const uint8_t *mask_in,
                                          uint8_t *mask_out, hepacc_stream stream);

/* get_bin_contents (Section III: lookup histograms for reweighting). For
 * j < n: with interpolate = 0, out[j] = contents[b] for the bin b of
 * data[j] as in hepacc_fill_histogram (contents has nbins+2 entries,
 * under- and overflow included); with interpolate != 0, the linear
 * interpolation between the contents of neighbouring in-range bins at
 * their centres c_b = (edges[b-1] + edges[b]) * 0.5, clamped to
 * contents[1] below c_1 and contents[nbins] at or above c_nbins:
 * t = (v - c_b) / (c_b+1 - c_b), out = contents[b] + t * (contents[b+1] -
 * contents[b]) for c_b <= v < c_b+1, every operation in binary32 rounded as
 * written. NaN data gives NaN. edges (nbins+1, increasing) and contents are
 * DEVICE float32; 1 <= nbins <= 65536; data_type F32, F16 or BF16. */
hepacc_status hepacc_get_bin_contents(const void *data, hepacc_dtype data_type, int64_t n, const float *edges,
                                      int32_t nbins, const float *contents, int32_t interpolate, float *out,
                                      hepacc_stream stream);

/* ---------------------------------------------------------------------------
 * The fused analysis chain (Section IV benchmark analysis), one launch
 * ------------------------------------------------------------------------- */

#define HEPACC_CHAIN_NVARS 20
#define HEPACC_JEC_MAX_BINS 64
#define HEPACC_MAX_VARIATIONS 64
#define HEPACC_CHAIN_MAX_EDGES 4096

/* One sample of events: three collections (jets, muons, electrons) sharing
 * n_events and one offsets type. kin_type (F32, F16, BF16) is the type of
 * pt, eta, phi, mass of all collections; btag_type F32 or F16. Lepton iso is
 * float32 and tight uint8. All pointers DEVICE. */
typedef struct {
    int64_t n_events;
    hepacc_dtype offsets_type;
    const void *jet_offsets, *mu_offsets, *el_offsets;
    hepacc_dtype kin_type;
    hepacc_dtype btag_type;
    const void *jet_pt, *jet_eta, *jet_phi, *jet_mass, *jet_btag;
    const void *mu_pt, *mu_eta, *mu_phi;
    const float *mu_iso;
    const uint8_t *mu_tight;
    const void *el_pt, *el_eta, *el_phi;
    const float *el_iso;
    const uint8_t *el_tight;
    const float *weight;
    /* Mean jets, muons and electrons per event, used only to size the
     * shared-memory staging of each collection; 0 selects 6, 1 and 1. */
    float jets_per_event, muons_per_event, electrons_per_event;
    /* Content lengths of the jet, muon and electron columns (elements, >= 0).
     * The debug checks (HEPACC_DEBUG, HEPACC_PLAN_VALIDATE) reject a batch
     * whose offsets[n_events] exceeds them before anything reads a column. */
    int64_t jet_len, mu_len, el_len;
} hepacc_event_batch;

/* Cuts, jet-pt scale variations and the 20 histograms. HOST memory: the call
 * copies what it needs. Histogram h has nbins[h] bins and nbins[h]+1
 * increasing binary32 edges, stored one histogram after another in edges;
 * its bins (with underflow and overflow, nbins[h]+2 of them) start at
 * sum over h' < h of (nbins[h'] + 2) inside one variation's histogram block
 * of total_bins = sum of (nbins[h] + 2) entries. */
typedef struct {
    float lep_pt_min, lep_abseta_max, lep_iso_max;
    float jet_pt_min, jet_abseta_max, dr2_cut, btag_min;
    int32_t n_var;                         /* 1 .. HEPACC_MAX_VARIATIONS */
    const float *scales;                   /* [n_var] jet-pt scale factors, finite and > 0 */
    int32_t nbins[HEPACC_CHAIN_NVARS];
    const float *edges;                    /* sum (nbins[h]+1) <= HEPACC_CHAIN_MAX_EDGES */
    /* Jet-energy corrections by table lookup (Section IV), optional: with
     * jec_contents non-NULL the variations correct each jet's pt instead of
     * scaling it: variation k takes the row of the jet's eta bin
     * (jec_eta_edges, jec_neta bins, rows for under- and overflow
     * included) of its table and reads it at the jet's pt as
     * hepacc_get_bin_contents interpolates (jec_pt_edges, jec_npt bins):
     * pt_k = pt * factor (binary32); scales are then ignored (but must still
     * be valid). Edges HOST (copied), increasing, 1 <= bins <=
     * HEPACC_JEC_MAX_BINS; contents DEVICE float32
     * [n_var][jec_neta + 2][jec_npt + 2], read by the kernels (valid while
     * calls and plans that use them run). With tables the batch's btag
     * column is F32 for F32 kinematics and F16 for half kinematics
     * (HEPACC_ERR_DTYPE otherwise). */
    int32_t jec_neta, jec_npt;
    const float *jec_eta_edges, *jec_pt_edges;
    const float *jec_contents;
} hepacc_chain_config;

/* Outputs, DEVICE memory. counts, sumw (and sumw2 if non-NULL) are
 * [n_var][total_bins] and accumulate (+=), so batches add up. The per-event
 * arrays are optional (NULL = not written); when any is given, every
 * variable is evaluated for every event:
 *   ev_pass [n_var][N] uint8, ev_nlep [N], ev_njet and ev_nb [n_var][N],
 *   ev_idx [n_var][5][N] local indices (leading, sub-leading, trijet a, b, c),
 *   ev_vars [n_var][20][N] the histogram variables, NaN where undefined. */
typedef struct {
    uint64_t *counts;
    double *sumw;
    double *sumw2;
    uint8_t *ev_pass;
    int32_t *ev_nlep;
    int32_t *ev_njet, *ev_nb;
    int32_t *ev_idx;
    float *ev_vars;
} hepacc_chain_outputs;

/* The Section IV chain for every event and every variation k (scale s_k):
 *  1. leptons (muons and electrons) selected by pt > lep_pt_min,
 *     |eta| < lep_abseta_max, tight != 0, iso < lep_iso_max; n_lep counts
 *     both; "the lepton" is the first selected muon, else electron;
 *  2. jets: pt_k = pt * s_k (binary32; with correction tables pt * the
 *     variation's table factor, see hepacc_chain_config); selected if pt_k > jet_pt_min,
 *     |eta| < jet_abseta_max and Delta R^2 >= dr2_cut (as in
 *     hepacc_mask_deltar) to every selected lepton;
 *  3. n_jet, n_b (btag > btag_min); pass = n_lep == 1, n_jet >= 2, n_b >= 1;
 *  4. the 20 variables, in order: HT (binary32 sum of pt_k in element
 *     order), leading-jet pt_k, eta, phi, mass, btag, sub-leading pt_k,
 *     dijet mass of the two leading jets, n_jet, n_b, max btag, trijet mass
 *     and |sum pT| (max-|sum pT| triplet, n_jet >= 3), lepton pt, eta, phi,
 *     iso, ST = HT + lepton pt, sum of selected-jet masses, event weight;
 *  5. every passing event adds its weight to one bin of each histogram
 *     (the trijet ones only when n_jet >= 3).
 * One kernel launch; each input column is read once.
 * Debug checks: with the environment variable HEPACC_DEBUG set (and not 0)
 * the three offsets arrays are first checked on the device (offsets[0] >= 0,
 * non-decreasing, offsets[n_events] <= the collection's content length; the
 * call waits for the check); a failure returns HEPACC_ERR_DEVICE_CHECK
 * before the chain is launched.
 * Shared memory: the call lays out blocks of 128 threads for three, two or
 * one resident block per SM (the most whose pair buffer holds half a
 * tile's jets), using up to the device's per-block opt-in limit. */
hepacc_status hepacc_run_chain(const hepacc_event_batch *batch, const hepacc_chain_config *config,
                               const hepacc_chain_outputs *out, hepacc_stream stream);

/* ---------------------------------------------------------------------------
 * Batched chain plans (Section IV: the benchmark runs the chain over many
 * samples of uneven size, each with its jet-pt variations)
 * ------------------------------------------------------------------------- */

/* Opaque plan: samples, their outputs, the kernel configuration chosen for
 * them and (optionally) a CUDA graph of the launches. */
typedef struct hepacc_plan hepacc_plan;

#define HEPACC_PLAN_AUTOTUNE 1          /* time the candidate configurations on the samples, keep the fastest */
#define HEPACC_PLAN_GRAPH 2             /* capture the launches once; runs replay the graph */
/* Candidate histogram placements (none of these flags = all of them). */
#define HEPACC_PLAN_HIST_BLOCK 4        /* block-private shared memory */
#define HEPACC_PLAN_HIST_CLUSTER8 8     /* shared memory of a cluster of 8 blocks */
#define HEPACC_PLAN_HIST_CLUSTER16 16   /* shared memory of a cluster of 16 blocks */
#define HEPACC_PLAN_HIST_GLOBAL 32      /* global memory */
#define HEPACC_PLAN_VALIDATE 64         /* check every sample's offsets on the device at creation */

/* Builds a plan that runs the chain of hepacc_run_chain over samples[0..n)
 * with one configuration, up to sixteen samples per persistent launch. With
 * global histograms the samples' tiles form one range that the blocks share
 * (no block waits at a sample boundary; the kernel of hepacc_run_chain,
 * with a choice of stage counts); with shared-memory histograms every block
 * walks through the samples in turn and adds its histograms to a sample's
 * outputs when done with it. Sample i adds to outputs[i]
 * (counts, sumw, sumw2 as in
 * hepacc_run_chain; per-event arrays must be NULL). All samples use I64
 * offsets and the same kin_type and btag_type (F32 with F32, F16 with F16
 * or BF16). Histogram placement is a kernel configuration: block-private
 * shared memory, shared memory spread over a cluster of 8 or 16 blocks
 * (updated through distributed shared memory), or global memory. The
 * candidates: the kernel of hepacc_run_chain with blocks of 64, 128 and
 * 256 threads x blocks per SM x 2-4 stages (every layout that fits), then
 * the walking kernel with each allowed shared-memory placement. Without
 * HEPACC_PLAN_AUTOTUNE the first candidate is taken; with it, every
 * candidate is run three times on the samples (DEVICE pointers given
 * here must be valid), the fastest kept, and the outputs cleared to zero
 * afterwards, on `stream`, which the call synchronises. The choice is
 * remembered for the life of the process, keyed by the GPU's name, the
 * configuration's values, the column types, the allowed placements, the
 * samples per launch, the objects per event (to 0.1) and the events (to a
 * power of two); a later plan with the same key takes it without timing
 * (hepacc_plan_describe then reports "tuned_from_cache": true). config is HOST
 * memory and copied; the sample and output structs are copied; the device
 * buffers they point to must stay valid while runs use them. With
 * HEPACC_PLAN_VALIDATE (or HEPACC_DEBUG set, as for hepacc_run_chain) every
 * sample's offsets are checked first; a failure returns
 * HEPACC_ERR_DEVICE_CHECK and nothing runs. *plan is NULL on error. */
hepacc_status hepacc_plan_create(const hepacc_chain_config *config, int32_t n_samples,
                                 const hepacc_event_batch *samples, const hepacc_chain_outputs *outputs,
                                 int32_t flags, hepacc_stream stream, hepacc_plan **plan);

/* Runs the plan once on `stream` (outputs accumulate). With samples and
 * outputs NULL it runs the samples and outputs the plan was created with.
 * Otherwise it runs the same chain, configuration and (with
 * HEPACC_PLAN_GRAPH) captured graph over another batch of n_samples
 * samples and their outputs (Section II: the cache is processed in
 * batches): n_samples must equal the plan's, the column types must match;
 * event counts may differ (the graph's kernel nodes are given the new
 * samples' descriptors before the replay). The structs are read before the
 * call returns; the device buffers must stay valid until the run is done.
 * Not thread-safe on one plan; two runs of one plan on different streams
 * race on their outputs if they share them. */
hepacc_status hepacc_plan_run(hepacc_plan *plan, int32_t n_samples, const hepacc_event_batch *samples,
                              const hepacc_chain_outputs *outputs, hepacc_stream stream);

/* Writes a one-line JSON description of the chosen configuration and of
 * every candidate the autotuner timed into buf[0..len) (NUL-terminated,
 * truncated to fit). */
hepacc_status hepacc_plan_describe(const hepacc_plan *plan, char *buf, int32_t len);

/* Frees the plan (NULL is allowed); outputs and inputs are not touched. */
void hepacc_plan_destroy(hepacc_plan *plan);

#ifdef __cplusplus
}
#endif

#endif /* HEPACC_H */
