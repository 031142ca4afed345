// Host side of the fused chain: validates calls, prepares the kernel
// parameters (cuts, scales, histogram edges), chooses the shared-memory
// layout and launches the compacting kernel (fused_kernel.cuh) for the column
// types; batched plans (many samples per launch, autotuned over block
// layouts and histogram placements, replayed as a CUDA graph, reusable over
// new batches of the same shape).
#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <new>
#include <vector>

#include "fused_kernel.cuh"

namespace hepacc {

namespace chain {
namespace {

hepacc_status make_params(const hepacc_chain_config* cfg, ChainParams& P) {
    if (cfg->n_var < 1 || cfg->n_var > HEPACC_MAX_VARIATIONS) return fail(HEPACC_ERR_INVALID_ARG, "n_var out of range");
    if (!cfg->scales || !cfg->edges) return fail(HEPACC_ERR_INVALID_ARG, "config scales and edges are required");
    std::memset(&P, 0, sizeof P);
    P.lep_pt_min = cfg->lep_pt_min;
    P.lep_abseta_max = cfg->lep_abseta_max;
    P.lep_iso_max = cfg->lep_iso_max;
    P.jet_pt_min = cfg->jet_pt_min;
    P.jet_abseta_max = cfg->jet_abseta_max;
    P.dr2_cut = cfg->dr2_cut;
    P.btag_min = cfg->btag_min;
    P.n_var = cfg->n_var;
    for (int k = 0; k < cfg->n_var; ++k) {
        // the kernel decides the jet counts through thresholds, exact for
        // positive finite scales only
        if (!(cfg->scales[k] > 0.0f) || !std::isfinite(cfg->scales[k]))
            return fail(HEPACC_ERR_INVALID_ARG, "scale %d is not a positive finite number", k);
        P.scales[k] = cfg->scales[k];
    }
    int ne = 0, nbt = 0;
    for (int h = 0; h < kNV; ++h) {
        const int nb = cfg->nbins[h];
        if (nb < 1) return fail(HEPACC_ERR_INVALID_ARG, "histogram %d has no bins", h);
        if (ne + nb + 1 > HEPACC_CHAIN_MAX_EDGES) return fail(HEPACC_ERR_INVALID_ARG, "too many histogram edges");
        P.nbins[h] = nb;
        P.eoff[h] = ne;
        P.boff[h] = nbt;
        for (int i = 0; i <= nb; ++i) {
            P.edges[ne + i] = cfg->edges[ne + i];
            if (i > 0 && !(cfg->edges[ne + i] >= cfg->edges[ne + i - 1]))
                return fail(HEPACC_ERR_INVALID_ARG, "edges of histogram %d are not increasing", h);
        }
        const float span = cfg->edges[ne + nb] - cfg->edges[ne];
        P.invw[h] = span > 0.0f ? static_cast<float>(nb) / span : 0.0f;
        P.e_lo[h] = cfg->edges[ne];
        P.e_hi[h] = cfg->edges[ne + nb];
        ne += nb + 1;
        nbt += nb + 2;
    }
    P.n_edges = ne;
    P.total_bins = nbt;
    if (cfg->jec_contents) {
        const int na = cfg->jec_neta, np = cfg->jec_npt;
        if (na < 1 || na > HEPACC_JEC_MAX_BINS || np < 1 || np > HEPACC_JEC_MAX_BINS)
            return fail(HEPACC_ERR_INVALID_ARG, "correction tables need 1 to %d bins per axis", HEPACC_JEC_MAX_BINS);
        if (!cfg->jec_eta_edges || !cfg->jec_pt_edges) return fail(HEPACC_ERR_INVALID_ARG, "correction table edges are required");
        for (int i = 0; i <= na; ++i) {
            if (i > 0 && !(cfg->jec_eta_edges[i] > cfg->jec_eta_edges[i - 1]))
                return fail(HEPACC_ERR_INVALID_ARG, "correction eta edges are not increasing");
            P.jec_edges[i] = cfg->jec_eta_edges[i];
        }
        for (int i = 0; i <= np; ++i) {
            if (i > 0 && !(cfg->jec_pt_edges[i] > cfg->jec_pt_edges[i - 1]))
                return fail(HEPACC_ERR_INVALID_ARG, "correction pt edges are not increasing");
            P.jec_edges[na + 1 + i] = cfg->jec_pt_edges[i];
        }
        P.jec_neta = na;
        P.jec_npt = np;
        P.jec_contents = cfg->jec_contents;
        P.jec_eta_invw = static_cast<float>(na) / (cfg->jec_eta_edges[na] - cfg->jec_eta_edges[0]);
    }
    return HEPACC_OK;
}

hepacc_status check_batch(const hepacc_event_batch* b) {
    if (b->n_events < 0) return fail(HEPACC_ERR_INVALID_ARG, "n_events < 0");
    if (b->n_events >= (int64_t(1) << 31)) return fail(HEPACC_ERR_INVALID_ARG, "at most 2^31 - 1 events per sample");
    if (!is_offsets_type(b->offsets_type)) return fail(HEPACC_ERR_DTYPE, "offsets must be I32 or I64");
    if (!is_float_type(b->kin_type)) return fail(HEPACC_ERR_DTYPE, "kin_type must be F32, F16 or BF16");
    if (b->btag_type != HEPACC_F32 && b->btag_type != HEPACC_F16) return fail(HEPACC_ERR_DTYPE, "btag_type must be F32 or F16");
    if (b->jet_len < 0 || b->mu_len < 0 || b->el_len < 0) return fail(HEPACC_ERR_INVALID_ARG, "negative content length");
    if (b->n_events > 0 &&
        (!b->jet_offsets || !b->mu_offsets || !b->el_offsets || !b->weight || !b->jet_pt || !b->jet_eta ||
         !b->jet_phi || !b->jet_mass || !b->jet_btag || !b->mu_pt || !b->mu_eta || !b->mu_phi || !b->mu_iso ||
         !b->mu_tight || !b->el_pt || !b->el_eta || !b->el_phi || !b->el_iso || !b->el_tight))
        return fail(HEPACC_ERR_INVALID_ARG, "a batch column is NULL");
    return HEPACC_OK;
}

// The three offsets arrays of a batch checked on the device against their
// content lengths (debug checks).
hepacc_status check_batch_offsets(const hepacc_event_batch* b, cudaStream_t s) {
    const void* offs[3] = {b->jet_offsets, b->mu_offsets, b->el_offsets};
    const int64_t lens[3] = {b->jet_len, b->mu_len, b->el_len};
    for (int c = 0; c < 3; ++c) {
        const hepacc_status st = check_offsets(offs[c], b->offsets_type, b->n_events, lens[c], s);
        if (st != HEPACC_OK) return st;
    }
    return HEPACC_OK;
}

bool has_per_event(const hepacc_chain_outputs* o) {
    return o->ev_pass || o->ev_nlep || o->ev_njet || o->ev_nb || o->ev_idx || o->ev_vars;
}

void make_sample(const hepacc_event_batch* b, const hepacc_chain_outputs* out, SampleDesc& d) {
    std::memset(&d, 0, sizeof d);
    d.col[J_PT] = b->jet_pt;
    d.col[J_ETA] = b->jet_eta;
    d.col[J_PHI] = b->jet_phi;
    d.col[J_MASS] = b->jet_mass;
    d.col[J_BTAG] = b->jet_btag;
    d.col[M_PT] = b->mu_pt;
    d.col[M_ETA] = b->mu_eta;
    d.col[M_PHI] = b->mu_phi;
    d.col[M_ISO] = b->mu_iso;
    d.col[M_TIGHT] = b->mu_tight;
    d.col[E_PT] = b->el_pt;
    d.col[E_ETA] = b->el_eta;
    d.col[E_PHI] = b->el_phi;
    d.col[E_ISO] = b->el_iso;
    d.col[E_TIGHT] = b->el_tight;
    d.weight = b->weight;
    d.off[0] = b->jet_offsets;
    d.off[1] = b->mu_offsets;
    d.off[2] = b->el_offsets;
    d.n = b->n_events;
    d.out.counts = reinterpret_cast<unsigned long long*>(out->counts);
    d.out.sumw = out->sumw;
    d.out.sumw2 = out->sumw2;
    d.out.ev_pass = out->ev_pass;
    d.out.ev_nlep = out->ev_nlep;
    d.out.ev_njet = out->ev_njet;
    d.out.ev_nb = out->ev_nb;
    d.out.ev_idx = out->ev_idx;
    d.out.ev_vars = out->ev_vars;
}

// Shared-memory layout for blocks of E threads (tiles of E events): stage
// capacities from the mean objects per event (tiles that do not fit are read
// from global memory), two stages, a 32-slot record queue, jet acceptance
// flags, a 64-entry pair list and the event summaries per warp, and the
// histograms of the placement (all of them in H_SMEM, a
// 1/cluster slice in H_CLUSTER, none in H_GLOBAL). Returns whether it fits.
bool layout_for(int E, int hmode, int cluster, double lam_j, double lam_m, double lam_e, size_t kes, size_t bes,
                int blocks_per_sm, const ChainParams& P, Layout& L) {
    std::memset(&L, 0, sizeof L);
    auto cap_of = [&](double lam) {
        const double m = E * lam;
        return static_cast<uint32_t>(((static_cast<size_t>(m + 4.0 * std::sqrt(m) + 64.0)) + 31) & ~size_t(31));
    };
    const uint32_t cj = cap_of(lam_j), cm = cap_of(lam_m), ce = cap_of(lam_e);
    uint32_t off = 0;
    auto add = [&](int c, size_t es, int coll, uint32_t cap) {
        ColSpec& cs = L.col[c];
        cs.base = nullptr;
        cs.es = static_cast<uint32_t>(es);
        cs.coll = static_cast<uint32_t>(coll);
        cs.cap = static_cast<uint32_t>((cap * es + 32 + 15) & ~size_t(15));
        cs.soff = off;
        off += cs.cap;
    };
    add(J_PT, kes, 0, cj);
    add(J_ETA, kes, 0, cj);
    add(J_PHI, kes, 0, cj);
    add(J_MASS, kes, 0, cj);
    add(J_BTAG, bes, 0, cj);
    add(M_PT, kes, 1, cm);
    add(M_ETA, kes, 1, cm);
    add(M_PHI, kes, 1, cm);
    add(M_ISO, 4, 1, cm);
    add(M_TIGHT, 1, 1, cm);
    add(E_PT, kes, 2, ce);
    add(E_ETA, kes, 2, ce);
    add(E_PHI, kes, 2, ce);
    add(E_ISO, 4, 2, ce);
    add(E_TIGHT, 1, 2, ce);
    auto up = [](size_t x) { return static_cast<uint32_t>((x + 127) & ~size_t(127)); };
    // every region starts on a 16-byte boundary (8-byte fields live in
    // several of them)
    auto region = [](size_t& at, size_t bytes) {
        at = (at + 15) & ~size_t(15);
        const uint32_t start = static_cast<uint32_t>(at);
        at += bytes;
        return start;
    };
    L.stage_bytes = up(kHdr + off);
    size_t at = 0;
    region(at, 2 * static_cast<size_t>(L.stage_bytes));
    L.bars = region(at, 32 + 48 + 48 + 16);   // four mbarriers, spans of two tiles
    L.edges = region(at, static_cast<size_t>((P.n_edges + 3) & ~3) * 4);
    L.queue = region(at, static_cast<size_t>(E) * R_WORDS * 4);
    L.acc_words = static_cast<int>(cj / 32 + 2);
    L.acc = region(at, static_cast<size_t>(E / 32) * L.acc_words * 4);
    L.pairs = region(at, static_cast<size_t>(E / 32) * 64 * 2);
    L.evs = region(at, static_cast<size_t>(E / 32) * kEvWords * 32 * 4);
    L.sample = region(at, sizeof(SampleDesc));
    L.tri = region(at, 256);
    L.hist = region(at, 0);
    const size_t nbins = static_cast<size_t>(P.n_var) * P.total_bins;
    if (hmode == H_SMEM) at += nbins * (8 + 8 + 4);
    if (hmode == H_CLUSTER) {
        L.hist_slice = static_cast<int>((nbins + cluster - 1) / cluster);
        at += static_cast<size_t>(L.hist_slice) * (8 + 8 + 4);
    }
    L.total = static_cast<uint32_t>((at + 15) & ~size_t(15));
    const DeviceInfo di = device_info();
    const size_t per_block = static_cast<size_t>(di.smem_per_sm / blocks_per_sm - di.smem_reserved);
    return L.total <= std::min(per_block, static_cast<size_t>(di.smem_optin));
}

// Shared-memory layout of the compacting kernel for blocks (and tiles) of NT
// threads with S stages: stage capacities from the mean objects per event
// (a tile that does not fit is read from global memory), the edges, scales
// and (flat launches) sample descriptors, then the buffer of passing events
// and their jets in what is left of the block's shared memory (at most
// 2 NT events). Returns whether it fits with room for at least 4 x 32 jets.
bool fused_layout(int NT, int S, double lam_j, double lam_m, double lam_e, size_t kes, size_t bes, const ChainParams& P,
                  int flat_samples, int blocks_per_sm, fused::FLayout& L) {
    std::memset(&L, 0, sizeof L);
    if (S < 2 || S > fused::kMaxStages) return false;
    // a tile's objects of a collection: mean m = NT lambda, Poisson spread
    // sqrt(m); the stage holds m + 3 sqrt(m) + 16 (a tile beyond it, about
    // one in a thousand, is read from global memory)
    auto cap_of = [&](double lam) {
        const double m = NT * lam;
        return static_cast<uint32_t>(((static_cast<size_t>(m + 3.0 * std::sqrt(m) + 16.0)) + 31) & ~size_t(31));
    };
    const uint32_t cj = cap_of(lam_j), cm = cap_of(lam_m), ce = cap_of(lam_e);
    uint32_t off = 0;
    auto add = [&](int c, size_t es, int coll, uint32_t cap) {
        ColSpec& cs = L.col[c];
        cs.base = nullptr;
        cs.es = static_cast<uint32_t>(es);
        cs.coll = static_cast<uint32_t>(coll);
        cs.cap = static_cast<uint32_t>((cap * es + 32 + 15) & ~size_t(15));
        cs.soff = off;
        off += cs.cap;
    };
    add(J_PT, kes, 0, cj);
    add(J_ETA, kes, 0, cj);
    add(J_PHI, kes, 0, cj);
    add(J_MASS, kes, 0, cj);
    add(J_BTAG, bes, 0, cj);
    add(M_PT, kes, 1, cm);
    add(M_ETA, kes, 1, cm);
    add(M_PHI, kes, 1, cm);
    add(M_ISO, 4, 1, cm);
    add(M_TIGHT, 1, 1, cm);
    add(E_PT, kes, 2, ce);
    add(E_ETA, kes, 2, ce);
    add(E_PHI, kes, 2, ce);
    add(E_ISO, 4, 2, ce);
    add(E_TIGHT, 1, 2, ce);
    auto region = [](size_t& at, size_t bytes) {
        at = (at + 15) & ~size_t(15);
        const uint32_t start = static_cast<uint32_t>(at);
        at += bytes;
        return start;
    };
    L.stages = S;
    L.stage_bytes = static_cast<uint32_t>((fused::kHdrBytes + off + 127) & ~size_t(127));
    size_t at = 0;
    region(at, static_cast<size_t>(S) * L.stage_bytes);
    L.bars = region(at, 8 * fused::kMaxStages + 6 * 8);
    L.edges = region(at, static_cast<size_t>(P.n_edges) * 4);
    L.scales = region(at, static_cast<size_t>(P.n_var) * 4);
    L.jec = region(at, static_cast<size_t>(P.jec_contents ? P.jec_neta + P.jec_npt + 2 : 1) * 4);
    L.samples = region(at, static_cast<size_t>(std::max(flat_samples, 1)) * sizeof(SampleDesc));
    L.misc = region(at, fused::kMiscWords * 4 + sizeof(L.col));   // counter, warp totals, column specs
    const DeviceInfo di = device_info();
    const size_t limit =
        std::min(static_cast<size_t>(di.smem_per_sm / blocks_per_sm - di.smem_reserved), static_cast<size_t>(di.smem_optin));
    const bool jec = P.jec_contents != nullptr;
    const size_t slack = 16 * (jec ? 26 : 24);   // alignment of the buffer's regions
    if (at + slack >= limit) return false;
    const size_t avail = limit - at - slack;
    // per buffered jet: 7 floats and the acceptance byte, with correction
    // tables also its table position (int32 offset, float weight)
    const size_t per_ev = 11 * 4 + 2 * 8, per_j = 7 * 4 + 1 + (jec ? 8 : 0);
    // events and jets in the proportion a passing event brings (its summary
    // and lambda_j jets, plus one), so that neither side fills first;
    // between 32 and 2 NT events
    const double per_pass = static_cast<double>(per_ev) + (lam_j + 1.0) * static_cast<double>(per_j);
    int cap_ev = static_cast<int>(std::min<double>(2.0 * NT, static_cast<double>(avail) / per_pass)) & ~31;
    cap_ev = std::max(cap_ev, 32);
    if (static_cast<size_t>(cap_ev) * per_ev + 4 * 32 * per_j > avail) return false;
    const int cap_j = static_cast<int>(std::min<size_t>((avail - cap_ev * per_ev) / per_j, 65535));
    L.cap_ev = cap_ev;
    L.cap_j = cap_j;
    const size_t ne = static_cast<size_t>(cap_ev), nj = static_cast<size_t>(cap_j);
    L.b_q = region(at, ne * 8);
    L.b_p = region(at, ne * 8);
    L.b_e = region(at, ne * 4);
    L.b_s = region(at, ne * 4);
    L.b_w = region(at, ne * 4);
    L.b_lpt = region(at, ne * 4);
    L.b_leta = region(at, ne * 4);
    L.b_lphi = region(at, ne * 4);
    L.b_liso = region(at, ne * 4);
    L.b_nlep = region(at, ne * 4);
    L.b_j0 = region(at, ne * 4);
    L.b_nj = region(at, ne * 4);
    L.b_ps = region(at, ne * 4);
    L.j_pt = region(at, nj * 4);
    L.j_eta = region(at, nj * 4);
    L.j_phi = region(at, nj * 4);
    L.j_m = region(at, nj * 4);
    L.j_bt = region(at, nj * 4);
    L.j_c = region(at, nj * 4);
    L.j_s = region(at, nj * 4);
    L.j_acc = region(at, nj);
    if (jec) {
        L.j_jo = region(at, nj * 4);
        L.j_ju = region(at, nj * 4);
    }
    L.total = static_cast<uint32_t>((at + 15) & ~size_t(15));
    return L.total <= limit;
}

// The configuration of single-sample launches (hepacc_run_chain): blocks of
// kDebugBlock threads with two stages, laid out for the most blocks per SM
// (three, then two) whose pair buffer holds at least half a tile's jets
// (smaller buffers drain so often that the extra warps do not pay: as plan
// candidates on GB300, 10M-event FP32 set, a 305-jet buffer at three
// blocks per SM ran 4.3 ms against 2.7 ms at two); else one block per SM.
bool single_config(double lam_j, double lam_m, double lam_e, size_t kes, size_t bes, const ChainParams& P,
                   fused::FLayout& L, int& NT) {
    NT = fused::kDebugBlock;
    // objects per event so dense that no stage fits: smaller stages (the
    // tiles that do not fit one are read from global memory)
    for (double f = 1.0; f >= 1.0 / 64; f *= 0.5) {
        for (int bps = fused::min_blocks_for(NT); bps >= 2; --bps)
            if (fused_layout(NT, 2, lam_j * f, lam_m * f, lam_e * f, kes, bes, P, 0, bps, L) &&
                L.cap_j >= 0.5 * NT * lam_j)
                return true;
        if (fused_layout(NT, 2, lam_j * f, lam_m * f, lam_e * f, kes, bes, P, 0, 1, L)) return true;
    }
    return fused_layout(NT, 2, 1.0, 0.25, 0.25, kes, bes, P, 0, 1, L);
}

hepacc_status dispatch_fused(hepacc_dtype kin, const fused::FusedArgs& a) {
    switch (kin) {
        case HEPACC_F32: return fused::run_fused_f32(a);
        case HEPACC_F16: return fused::run_fused_f16(a);
        default: return fused::run_fused_bf16(a);
    }
}

hepacc_status dispatch_walking(hepacc_dtype kin, const LaunchArgs& a) {
    switch (kin) {
        case HEPACC_F32: return run_batched_f32(a);
        case HEPACC_F16: return run_batched_f16(a);
        default: return run_batched_bf16(a);
    }
}

}  // namespace
}  // namespace chain
}  // namespace hepacc

using namespace hepacc;
using namespace hepacc::chain;

extern "C" hepacc_status hepacc_run_chain(const hepacc_event_batch* b, const hepacc_chain_config* cfg,
                                          const hepacc_chain_outputs* out, hepacc_stream stream) {
    if (!b || !cfg || !out) return fail(HEPACC_ERR_INVALID_ARG, "batch, config and outputs are required");
    ChainParams P;
    hepacc_status st = make_params(cfg, P);
    if (st != HEPACC_OK) return st;
    if (!out->counts || !out->sumw) return fail(HEPACC_ERR_INVALID_ARG, "counts and sumw are required");
    st = check_batch(b);
    if (st != HEPACC_OK) return st;
    if (b->n_events == 0) return HEPACC_OK;
    if (debug_checks()) {
        st = check_batch_offsets(b, reinterpret_cast<cudaStream_t>(stream));
        if (st != HEPACC_OK) return st;
    }
    BatchDesc B;
    std::memset(&B, 0, sizeof B);
    B.n_samples = 1;
    make_sample(b, out, B.s[0]);

    const double lam_j = b->jets_per_event > 0 ? b->jets_per_event : 6.0;
    const double lam_m = b->muons_per_event > 0 ? b->muons_per_event : 1.0;
    const double lam_e = b->electrons_per_event > 0 ? b->electrons_per_event : 1.0;
    const size_t kes = dtype_size(b->kin_type), bes = dtype_size(b->btag_type);
    fused::FLayout L;
    int NT = 0;
    if (!single_config(lam_j, lam_m, lam_e, kes, bes, P, L, NT))
        return fail(HEPACC_ERR_INVALID_ARG, "chain stage buffers do not fit in shared memory");

    fused::FusedArgs a;
    a.layout = L;
    a.P = &P;
    a.B = &B;
    a.offsets_type = b->offsets_type;
    a.btag_type = b->btag_type;
    a.debug = has_per_event(out);
    a.flat = false;
    a.jec = P.jec_contents != nullptr;
    a.block = NT;
    a.grid = 0;
    a.cap_grid = true;
    a.ntiles = (b->n_events + NT - 1) / NT;
    a.stream = reinterpret_cast<cudaStream_t>(stream);
    return dispatch_fused(b->kin_type, a);
}

// ---------------------------------------------------------------------------
// Batched plans
// ---------------------------------------------------------------------------

namespace {

// A kernel configuration of a plan: the compacting kernel over the samples'
// tiles as one flat range (global histograms; block layout with S stages),
// or the walking kernel with shared-memory histograms in one block or spread
// over a cluster.
struct Candidate {
    bool compacting;
    int hmode, cluster, block, blocks_per_sm, stages;
    Layout L;            // walking kernel
    fused::FLayout FL;   // compacting kernel
};

}  // namespace

struct hepacc_plan {
    ChainParams P;
    int n_samples;
    std::vector<hepacc_chain_outputs> outs;
    std::vector<hepacc_event_batch> samples;
    hepacc_dtype kin, btag;
    Candidate c;         // the chosen configuration
    float tuned_ms;
    bool tuned_from_cache;   // the choice came from the autotune cache
    int n_candidates;
    std::vector<std::string> tried;   // candidate descriptions and times (JSON fragments)
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    std::vector<cudaGraphNode_t> nodes;   // the graph's kernel nodes, one per launch, in launch order
};

namespace {

// The launches of a set of samples: up to kMaxSamples per launch.
std::vector<BatchDesc> make_launches(int n, const hepacc_event_batch* samples, const hepacc_chain_outputs* outs,
                                     int block) {
    std::vector<BatchDesc> v;
    for (int i0 = 0; i0 < n; i0 += kMaxSamples) {
        BatchDesc B;
        std::memset(&B, 0, sizeof B);
        B.n_samples = std::min(kMaxSamples, n - i0);
        for (int j = 0; j < B.n_samples; ++j) make_sample(&samples[i0 + j], &outs[i0 + j], B.s[j]);
        // flat launches: the first tile of every sample for this block size
        B.tile_start[0] = 0;
        for (int i = 0; i < B.n_samples; ++i) B.tile_start[i + 1] = B.tile_start[i] + (B.s[i].n + block - 1) / block;
        v.push_back(B);
    }
    return v;
}

// Launches one BatchDesc with the plan's configuration. The grid is the
// full persistent grid whatever the sizes, so that a captured launch can be
// pointed at other samples.
hepacc_status launch_one(const hepacc_plan* p, const Candidate& c, const BatchDesc& B, cudaStream_t s) {
    if (c.compacting) {
        fused::FusedArgs a;
        a.layout = c.FL;
        a.P = &p->P;
        a.B = &B;
        a.offsets_type = HEPACC_I64;
        a.btag_type = p->btag;
        a.debug = false;
        a.flat = true;
        a.jec = p->P.jec_contents != nullptr;
        a.block = c.block;
        a.grid = 0;
        a.cap_grid = false;
        a.ntiles = B.tile_start[B.n_samples];
        a.stream = s;
        return dispatch_fused(p->kin, a);
    }
    LaunchArgs a;
    a.layout = c.L;
    a.P = &p->P;
    a.B = &B;
    a.offsets_type = HEPACC_I64;
    a.btag_type = p->btag;
    a.debug = false;
    a.hmode = c.hmode;
    a.block = c.block;
    a.cluster = c.cluster;
    a.grid = 0;
    a.max_tiles = int64_t(1) << 40;
    a.stream = s;
    return dispatch_walking(p->kin, a);
}

hepacc_status plan_launch(const hepacc_plan* p, const Candidate& c, const std::vector<BatchDesc>& launches,
                          cudaStream_t s) {
    for (const BatchDesc& B : launches) {
        const hepacc_status st = launch_one(p, c, B, s);
        if (st != HEPACC_OK) return st;
    }
    return HEPACC_OK;
}

hepacc_status zero_outputs(const hepacc_plan* p, cudaStream_t s) {
    const size_t nb = static_cast<size_t>(p->P.n_var) * p->P.total_bins;
    for (const hepacc_chain_outputs& o : p->outs) {
        cudaError_t e = cudaMemsetAsync(o.counts, 0, nb * sizeof(uint64_t), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(o.sumw, 0, nb * sizeof(double), s);
        if (e == cudaSuccess && o.sumw2) e = cudaMemsetAsync(o.sumw2, 0, nb * sizeof(double), s);
        if (e != cudaSuccess) return cuda_fail(e, "clearing plan outputs");
    }
    return HEPACC_OK;
}

std::string describe(const Candidate& c) {
    char buf[160];
    if (c.compacting)
        snprintf(buf, sizeof buf, "{\"kernel\": \"compacting\", \"histograms\": \"global\", \"block\": %d, "
                 "\"blocks_per_sm\": %d, \"stages\": %d, \"buffer_events\": %d, \"buffer_jets\": %d", c.block,
                 c.blocks_per_sm, c.stages, c.FL.cap_ev, c.FL.cap_j);
    else
        snprintf(buf, sizeof buf, "{\"kernel\": \"walking\", \"histograms\": \"%s\", \"cluster\": %d, \"block\": %d",
                 c.hmode == H_SMEM ? "block" : "cluster", c.cluster, c.block);
    return buf;
}

// The autotune cache of this process: the configuration an earlier plan of
// the same shape chose, keyed by the GPU's name, the configuration's
// values (cuts, edges, scales, tables: a hash), the column types, the
// allowed placements, the launch's sample count, the objects per event
// (to 0.1) and the events (to a power of two).
struct TuneChoice {
    bool compacting;
    int hmode, cluster, block, blocks_per_sm, stages;
    float ms;
};
std::mutex& tune_mu() {
    static std::mutex m;
    return m;
}
std::map<std::string, TuneChoice>& tune_cache() {
    static std::map<std::string, TuneChoice> c;
    return c;
}
std::string tune_key(const ChainParams& P, hepacc_dtype kin, hepacc_dtype btag, uint32_t allowed, int flat_samples,
                     double lam_j, double lam_m, double lam_e, double events) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    std::memset(&prop, 0, sizeof prop);
    cudaGetDeviceProperties(&prop, dev);
    // FNV-1a over the configuration's bytes (ChainParams is zeroed before it
    // is filled, so its padding hashes the same every time)
    uint64_t h = 1469598103934665603ull;
    const unsigned char* b = reinterpret_cast<const unsigned char*>(&P);
    for (size_t i = 0; i < sizeof P; ++i) h = (h ^ b[i]) * 1099511628211ull;
    char buf[512];
    snprintf(buf, sizeof buf, "%s|%016llx|%d|%d|%u|%d|%ld|%ld|%ld|%d", prop.name, static_cast<unsigned long long>(h),
             static_cast<int>(kin), static_cast<int>(btag), allowed, flat_samples, std::lround(lam_j * 10),
             std::lround(lam_m * 10), std::lround(lam_e * 10), events > 1 ? static_cast<int>(std::log2(events)) : 0);
    return buf;
}
bool same_choice(const Candidate& c, const TuneChoice& t) {
    return c.compacting == t.compacting && c.hmode == t.hmode && c.cluster == t.cluster && c.block == t.block &&
           c.blocks_per_sm == t.blocks_per_sm && c.stages == t.stages;
}

// Times every candidate (one warm-up run, two timed) on the plan's samples
// and returns the index of the fastest, -1 if none ran.
int autotune(hepacc_plan* p, const std::vector<Candidate>& cands, cudaStream_t s, float& best_ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return -1;
    }
    int pick = -1;
    best_ms = -1.0f;
    for (size_t i = 0; i < cands.size(); ++i) {
        const auto launches = make_launches(p->n_samples, p->samples.data(), p->outs.data(), cands[i].block);
        std::string d = describe(cands[i]);
        if (plan_launch(p, cands[i], launches, s) != HEPACC_OK) {
            cudaGetLastError();
            p->tried.push_back(d + ", \"ms\": null}");
            continue;
        }
        cudaEventRecord(e0, s);
        const bool ok = plan_launch(p, cands[i], launches, s) == HEPACC_OK && plan_launch(p, cands[i], launches, s) == HEPACC_OK;
        cudaEventRecord(e1, s);
        float ms = 0.0f;
        if (cudaEventSynchronize(e1) == cudaSuccess && ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
            ms *= 0.5f;
            char t[48];
            snprintf(t, sizeof t, ", \"ms\": %.4f}", static_cast<double>(ms));
            p->tried.push_back(d + t);
            if (best_ms < 0.0f || ms < best_ms) {
                best_ms = ms;
                pick = static_cast<int>(i);
            }
        } else {
            cudaGetLastError();
            p->tried.push_back(d + ", \"ms\": null}");
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return pick;
}

// Captures the plan's launches into a graph and records its kernel nodes in
// launch order (the capture of one stream is a chain).
hepacc_status capture(hepacc_plan* p) {
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "capture stream");
    hepacc_status st = HEPACC_OK;
    const auto launches = make_launches(p->n_samples, p->samples.data(), p->outs.data(), p->c.block);
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        st = plan_launch(p, p->c, launches, cs);
        const cudaError_t e2 = cudaStreamEndCapture(cs, &p->graph);
        if (st == HEPACC_OK && e2 != cudaSuccess) st = cuda_fail(e2, "graph capture");
    } else {
        st = cuda_fail(e, "begin capture");
    }
    cudaStreamDestroy(cs);
    if (st != HEPACC_OK) return st;
    size_t nroots = 1;
    cudaGraphNode_t node = nullptr;
    e = cudaGraphGetRootNodes(p->graph, &node, &nroots);
    if (e != cudaSuccess) return cuda_fail(e, "graph roots");
    while (node) {
        cudaGraphNodeType t;
        e = cudaGraphNodeGetType(node, &t);
        if (e != cudaSuccess) return cuda_fail(e, "graph node type");
        if (t == cudaGraphNodeTypeKernel) p->nodes.push_back(node);
        size_t nd = 0;
        e = cudaGraphNodeGetDependentNodes(node, nullptr, nullptr, &nd);
        if (e != cudaSuccess) return cuda_fail(e, "graph node dependents");
        if (nd > 1) return fail(HEPACC_ERR_CUDA, "plan graph is not a chain");
        cudaGraphNode_t nx = nullptr;
        if (nd == 1) {
            e = cudaGraphNodeGetDependentNodes(node, &nx, nullptr, &nd);
            if (e != cudaSuccess) return cuda_fail(e, "graph node dependents");
        }
        node = nx;
    }
    if (p->nodes.size() != launches.size()) return fail(HEPACC_ERR_CUDA, "plan graph has %zu kernel nodes for %zu launches",
                                                        p->nodes.size(), launches.size());
    e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    return HEPACC_OK;
}

// Checks a set of samples against a plan's: count, types; outputs given.
hepacc_status check_plan_samples(int n_samples, const hepacc_event_batch* samples, const hepacc_chain_outputs* outputs,
                                 hepacc_dtype kin, hepacc_dtype btag) {
    for (int i = 0; i < n_samples; ++i) {
        const hepacc_event_batch& b = samples[i];
        const hepacc_chain_outputs& o = outputs[i];
        hepacc_status st = check_batch(&b);
        if (st != HEPACC_OK) return st;
        if (!o.counts || !o.sumw) return fail(HEPACC_ERR_INVALID_ARG, "sample %d: counts and sumw are required", i);
        if (has_per_event(&o)) return fail(HEPACC_ERR_INVALID_ARG, "plans write no per-event outputs");
        if (b.offsets_type != HEPACC_I64) return fail(HEPACC_ERR_DTYPE, "plans need I64 offsets");
        if (b.kin_type != kin || b.btag_type != btag)
            return fail(HEPACC_ERR_DTYPE, "all samples of a plan share their column types");
        if ((b.kin_type == HEPACC_F32) != (b.btag_type == HEPACC_F32))
            return fail(HEPACC_ERR_DTYPE, "plans take F32 btag with F32 kinematics, F16 btag with half kinematics");
    }
    return HEPACC_OK;
}

}  // namespace

extern "C" {

hepacc_status hepacc_plan_create(const hepacc_chain_config* cfg, int32_t n_samples, const hepacc_event_batch* samples,
                                 const hepacc_chain_outputs* outputs, int32_t flags, hepacc_stream stream,
                                 hepacc_plan** plan) {
    if (!plan) return fail(HEPACC_ERR_INVALID_ARG, "plan is required");
    *plan = nullptr;
    if (!cfg) return fail(HEPACC_ERR_INVALID_ARG, "config is required");
    if (n_samples < 1 || !samples || !outputs) return fail(HEPACC_ERR_INVALID_ARG, "need at least one sample and its outputs");
    const int hist_flags = HEPACC_PLAN_HIST_BLOCK | HEPACC_PLAN_HIST_CLUSTER8 | HEPACC_PLAN_HIST_CLUSTER16 |
                           HEPACC_PLAN_HIST_GLOBAL;
    if (flags & ~(HEPACC_PLAN_AUTOTUNE | HEPACC_PLAN_GRAPH | HEPACC_PLAN_VALIDATE | hist_flags))
        return fail(HEPACC_ERR_INVALID_ARG, "unknown plan flags");
    const int allowed = (flags & hist_flags) ? (flags & hist_flags) : hist_flags;
    hepacc_plan* p = new (std::nothrow) hepacc_plan();
    if (!p) return fail(HEPACC_ERR_OOM, "plan allocation");
    auto drop = [&](hepacc_status st) {
        if (p->exec) cudaGraphExecDestroy(p->exec);
        if (p->graph) cudaGraphDestroy(p->graph);
        delete p;
        return st;
    };
    hepacc_status st = make_params(cfg, p->P);
    if (st != HEPACC_OK) return drop(st);
    st = check_plan_samples(n_samples, samples, outputs, samples[0].kin_type, samples[0].btag_type);
    if (st != HEPACC_OK) return drop(st);
    double jets = 0, mus = 0, els = 0, events = 0;
    for (int i = 0; i < n_samples; ++i) {
        const hepacc_event_batch& b = samples[i];
        const double n = static_cast<double>(b.n_events);
        jets += (b.jets_per_event > 0 ? b.jets_per_event : 6.0) * n;
        mus += (b.muons_per_event > 0 ? b.muons_per_event : 1.0) * n;
        els += (b.electrons_per_event > 0 ? b.electrons_per_event : 1.0) * n;
        events += n;
    }
    if ((flags & HEPACC_PLAN_VALIDATE) || debug_checks()) {
        for (int i = 0; i < n_samples; ++i) {
            st = check_batch_offsets(&samples[i], reinterpret_cast<cudaStream_t>(stream));
            if (st != HEPACC_OK) return drop(fail(st, "sample %d: %s", i, hepacc_last_error()));
        }
    }
    p->n_samples = n_samples;
    p->kin = samples[0].kin_type;
    p->btag = samples[0].btag_type;
    const double lam_j0 = events > 0 ? jets / events : 6.0;
    const double lam_m0 = events > 0 ? mus / events : 1.0;
    const double lam_e0 = events > 0 ? els / events : 1.0;
    p->outs.assign(outputs, outputs + n_samples);
    p->samples.assign(samples, samples + n_samples);
    const int flat_samples = std::min(n_samples, kMaxSamples);

    // candidates: the compacting kernel (global histograms) with every stage
    // count that fits, then the walking kernel with histograms in block
    // shared memory or spread over clusters of 8 or 16 blocks
    const size_t kes = dtype_size(p->kin), bes = dtype_size(p->btag);
    std::vector<Candidate> cands;
    // objects per event so dense that nothing fits: smaller stages (tiles
    // that do not fit one are read from global memory)
    for (double f = 1.0; cands.empty() && f >= 1.0 / 64; f *= 0.5) {
        const double lam_j = lam_j0 * f, lam_m = lam_m0 * f, lam_e = lam_e0 * f;
        if (allowed & HEPACC_PLAN_HIST_GLOBAL) {
            // block size x blocks per SM (the share of the SM's shared memory
            // each block is laid out for) x stages
            // (correction tables: blocks of kDebugBlock threads only)
            for (int nt : fused::kBlocks)
                for (int bps = 1; bps <= fused::min_blocks_for(nt) && (!p->P.jec_contents || nt == fused::kDebugBlock);
                     ++bps)
                    for (int S = 2; S <= fused::kMaxStages; ++S) {
                        Candidate c{};
                        // (a buffer for a quarter of a tile's jets: only passing
                        // events append theirs)
                        if (fused_layout(nt, S, lam_j, lam_m, lam_e, kes, bes, p->P, flat_samples, bps, c.FL) &&
                            c.FL.cap_j >= nt * lam_j / 4) {
                            c.compacting = true;
                            c.hmode = H_GLOBAL;
                            c.cluster = 1;
                            c.block = nt;
                            c.blocks_per_sm = bps;
                            c.stages = S;
                            cands.push_back(c);
                        }
                    }
        }
        const int modes[3][3] = {{H_SMEM, 1, HEPACC_PLAN_HIST_BLOCK},
                                 {H_CLUSTER, 8, HEPACC_PLAN_HIST_CLUSTER8},
                                 {H_CLUSTER, 16, HEPACC_PLAN_HIST_CLUSTER16}};
        // (the walking kernel applies scales only: plans with correction
        // tables run the compacting kernel)
        for (const auto& m : modes) {
            for (int e = kMaxThreadsBatched; e >= 64 && (allowed & m[2]) && !p->P.jec_contents; e -= 32) {
                Candidate c{};
                if (layout_for(e, m[0], m[1], lam_j, lam_m, lam_e, kes, bes, kMinBlocksBatched, p->P, c.L)) {
                    c.compacting = false;
                    c.hmode = m[0];
                    c.cluster = m[1];
                    c.block = e;
                    c.blocks_per_sm = kMinBlocksBatched;
                    c.stages = 2;
                    cands.push_back(c);
                    break;
                }
            }
        }
    }
    if (cands.empty()) return drop(fail(HEPACC_ERR_INVALID_ARG, "no chain layout fits in shared memory"));
    p->n_candidates = static_cast<int>(cands.size());
    p->tuned_ms = -1.0f;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int pick = 0;
    p->tuned_from_cache = false;
    const std::string key = tune_key(p->P, p->kin, p->btag, allowed, flat_samples, lam_j0, lam_m0, lam_e0, events);
    if (flags & HEPACC_PLAN_AUTOTUNE) {
        std::lock_guard<std::mutex> g(tune_mu());
        auto it = tune_cache().find(key);
        if (it != tune_cache().end())
            for (size_t i = 0; i < cands.size(); ++i)
                if (same_choice(cands[i], it->second)) {
                    pick = static_cast<int>(i);
                    p->tuned_ms = it->second.ms;
                    p->tuned_from_cache = true;
                    break;
                }
    }
    if ((flags & HEPACC_PLAN_AUTOTUNE) && !p->tuned_from_cache) {
        pick = autotune(p, cands, s, p->tuned_ms);
        cudaGetLastError();   // failures of rejected candidates
        if (pick < 0) return drop(fail(HEPACC_ERR_CUDA, "no candidate chain configuration ran"));
        {
            const Candidate& c = cands[pick];
            std::lock_guard<std::mutex> g(tune_mu());
            tune_cache()[key] =
                TuneChoice{c.compacting, c.hmode, c.cluster, c.block, c.blocks_per_sm, c.stages, p->tuned_ms};
        }
        st = zero_outputs(p, s);
        if (st == HEPACC_OK) {
            const cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) st = cuda_fail(e, "autotune");
        }
        if (st != HEPACC_OK) return drop(st);
    }
    p->c = cands[pick];
    if (flags & HEPACC_PLAN_GRAPH) {
        st = capture(p);
        if (st != HEPACC_OK) return drop(st);
    }
    *plan = p;
    return HEPACC_OK;
}

hepacc_status hepacc_plan_run(hepacc_plan* p, int32_t n_samples, const hepacc_event_batch* samples,
                              const hepacc_chain_outputs* outputs, hepacc_stream stream) {
    if (!p) return fail(HEPACC_ERR_INVALID_ARG, "plan is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!samples && !outputs) {
        if (p->exec) {
            const cudaError_t e = cudaGraphLaunch(p->exec, s);
            if (e != cudaSuccess) return cuda_fail(e, "graph launch");
            return HEPACC_OK;
        }
        return plan_launch(p, p->c, make_launches(p->n_samples, p->samples.data(), p->outs.data(), p->c.block), s);
    }
    if (!samples || !outputs) return fail(HEPACC_ERR_INVALID_ARG, "samples and outputs go together");
    if (n_samples != p->n_samples) return fail(HEPACC_ERR_INVALID_ARG, "the plan runs %d samples, not %d", p->n_samples, n_samples);
    hepacc_status st = check_plan_samples(n_samples, samples, outputs, p->kin, p->btag);
    if (st != HEPACC_OK) return st;
    if (debug_checks()) {
        for (int i = 0; i < n_samples; ++i) {
            st = check_batch_offsets(&samples[i], s);
            if (st != HEPACC_OK) return fail(st, "sample %d: %s", i, hepacc_last_error());
        }
    }
    const auto launches = make_launches(n_samples, samples, outputs, p->c.block);
    if (!p->exec) return plan_launch(p, p->c, launches, s);
    // the captured graph, each kernel node pointed at the new descriptors
    for (size_t i = 0; i < launches.size(); ++i) {
        cudaKernelNodeParams kp;
        cudaError_t e = cudaGraphKernelNodeGetParams(p->nodes[i], &kp);
        if (e != cudaSuccess) return cuda_fail(e, "kernel node parameters");
        const void* args[3] = {p->c.compacting ? static_cast<const void*>(&p->c.FL) : static_cast<const void*>(&p->c.L),
                               &p->P, &launches[i]};
        kp.kernelParams = const_cast<void**>(args);
        kp.extra = nullptr;
        e = cudaGraphExecKernelNodeSetParams(p->exec, p->nodes[i], &kp);
        if (e != cudaSuccess) return cuda_fail(e, "rebinding the plan's graph");
    }
    const cudaError_t e = cudaGraphLaunch(p->exec, s);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    return HEPACC_OK;
}

hepacc_status hepacc_plan_describe(const hepacc_plan* p, char* buf, int32_t len) {
    if (!p || !buf || len < 1) return fail(HEPACC_ERR_INVALID_ARG, "plan and buffer are required");
    std::string tried;
    for (size_t i = 0; i < p->tried.size(); ++i) tried += (i ? ", " : "") + p->tried[i];
    const size_t nl = (p->n_samples + kMaxSamples - 1) / kMaxSamples;
    const unsigned smem = p->c.compacting ? p->c.FL.total : p->c.L.total;
    snprintf(buf, static_cast<size_t>(len),
             "{\"chosen\": %s, \"smem_bytes\": %u}, \"launches\": %zu, \"graph\": %s, \"candidates\": %d, "
             "\"tuned_ms\": %.4f, \"tuned_from_cache\": %s, \"tried\": [%s]}",
             describe(p->c).c_str(), smem, nl, p->exec ? "true" : "false", p->n_candidates,
             static_cast<double>(p->tuned_ms), p->tuned_from_cache ? "true" : "false", tried.c_str());
    return HEPACC_OK;
}

void hepacc_plan_destroy(hepacc_plan* p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    delete p;
}

}  // extern "C"
