// Host entry point of the fused chain: validates the call, prepares the
// kernel parameters (cuts, scales, histogram edges, stage layout) and picks
// the shared-memory layout, then launches the kernel for the column types.
#include <cmath>

#include "chain_kernel.cuh"

namespace hepacc {

unsigned int tu_error_chain(bool clear) {
    return chain::tu_error_f32(clear) | chain::tu_error_bf16(clear) | chain::tu_error_f16(clear);
}

namespace chain {

// Tunables of the chain launch (set by the autotuner; 0 = default).
struct ChainTuning {
    int jet_cap;     // stage capacity for jets, elements per warp tile
    int lep_cap;     // stage capacity per lepton collection
    int grid;        // blocks (0 = resident blocks x SMs)
    int warps;       // upper bound of warps per block (0 = 16)
};
ChainTuning g_tuning = {0, 0, 0, 0};


}  // namespace chain
}  // namespace hepacc

using namespace hepacc;
using namespace hepacc::chain;

extern "C" hepacc_status hepacc_run_chain(const hepacc_event_batch* b, const hepacc_chain_config* cfg,
                                          const hepacc_chain_outputs* out, hepacc_stream stream) {
    if (!b || !cfg || !out) return fail(HEPACC_ERR_INVALID_ARG, "batch, config and outputs are required");
    if (b->n_events < 0) return fail(HEPACC_ERR_INVALID_ARG, "n_events < 0");
    if (cfg->n_var < 1 || cfg->n_var > HEPACC_MAX_VARIATIONS) return fail(HEPACC_ERR_INVALID_ARG, "n_var out of range");
    if (!cfg->scales || !cfg->edges) return fail(HEPACC_ERR_INVALID_ARG, "config scales and edges are required");
    if (!out->counts || !out->sumw) return fail(HEPACC_ERR_INVALID_ARG, "counts and sumw are required");
    if (!is_offsets_type(b->offsets_type)) return fail(HEPACC_ERR_DTYPE, "offsets must be I32 or I64");
    if (!is_float_type(b->kin_type)) return fail(HEPACC_ERR_DTYPE, "kin_type must be F32, F16 or BF16");
    if (b->btag_type != HEPACC_F32 && b->btag_type != HEPACC_F16) return fail(HEPACC_ERR_DTYPE, "btag_type must be F32 or F16");
    ChainParams P;
    std::memset(&P, 0, sizeof P);
    P.lep_pt_min = cfg->lep_pt_min;
    P.lep_abseta_max = cfg->lep_abseta_max;
    P.lep_iso_max = cfg->lep_iso_max;
    P.jet_pt_min = cfg->jet_pt_min;
    P.jet_abseta_max = cfg->jet_abseta_max;
    P.dr2_cut = cfg->dr2_cut;
    P.btag_min = cfg->btag_min;
    P.n_var = cfg->n_var;
    for (int k = 0; k < cfg->n_var; ++k) P.scales[k] = cfg->scales[k];
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
        ne += nb + 1;
        nbt += nb + 2;
    }
    P.n_edges = ne;
    P.total_bins = nbt;
    const int64_t n = b->n_events;
    if (n == 0) return HEPACC_OK;
    const bool debug = out->ev_pass || out->ev_nlep || out->ev_njet || out->ev_nb || out->ev_idx || out->ev_vars;
    if (!b->jet_offsets || !b->mu_offsets || !b->el_offsets || !b->weight || !b->jet_pt || !b->jet_eta ||
        !b->jet_phi || !b->jet_mass || !b->jet_btag || !b->mu_pt || !b->mu_eta || !b->mu_phi || !b->mu_iso ||
        !b->mu_tight || !b->el_pt || !b->el_eta || !b->el_phi || !b->el_iso || !b->el_tight)
        return fail(HEPACC_ERR_INVALID_ARG, "a batch column is NULL");

    ChainOut o;
    o.counts = reinterpret_cast<unsigned long long*>(out->counts);
    o.sumw = out->sumw;
    o.sumw2 = out->sumw2;
    o.ev_pass = out->ev_pass;
    o.ev_nlep = out->ev_nlep;
    o.ev_njet = out->ev_njet;
    o.ev_nb = out->ev_nb;
    o.ev_idx = out->ev_idx;
    o.ev_vars = out->ev_vars;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    if (n >= (int64_t(1) << 31)) return fail(HEPACC_ERR_INVALID_ARG, "at most 2^31 - 1 events per call");
    ChainCols C;
    C.jet_pt = b->jet_pt; C.jet_eta = b->jet_eta; C.jet_phi = b->jet_phi; C.jet_mass = b->jet_mass;
    C.jet_btag = b->jet_btag;
    C.mu_pt = b->mu_pt; C.mu_eta = b->mu_eta; C.mu_phi = b->mu_phi; C.mu_iso = b->mu_iso; C.mu_tight = b->mu_tight;
    C.el_pt = b->el_pt; C.el_eta = b->el_eta; C.el_phi = b->el_phi; C.el_iso = b->el_iso; C.el_tight = b->el_tight;
    C.weight = b->weight;

    // Shared-memory layout for tiles of E events: stage capacities from the
    // mean objects per event (tiles that do not fit are read from global
    // memory), two stages, a 32-slot queue per warp and, when they fit, the
    // block-private histograms; the largest E (multiple of 32, <= 384) that
    // fits wins, preferring shared-memory histograms.
    const double lam_j = b->jets_per_event > 0 ? b->jets_per_event : 6.0;
    const double lam_l = b->leptons_per_event > 0 ? b->leptons_per_event : 1.5;
    const size_t kes = dtype_size(b->kin_type), bes = dtype_size(b->btag_type);
    const DeviceInfo di = device_info();
    auto layout_for = [&](int E, bool with_hist, Layout& L) -> bool {
        std::memset(&L, 0, sizeof L);
        auto cap_of = [&](double lam) {
            const double m = E * lam;
            return static_cast<uint32_t>(((static_cast<size_t>(m + 4.0 * std::sqrt(m) + 64.0)) + 31) & ~size_t(31));
        };
        const uint32_t cj = cap_of(lam_j), cl = cap_of(lam_l);
        uint32_t off = 0;
        auto add = [&](int c, const void* base, size_t es, int coll, uint32_t cap) {
            ColSpec& cs = L.col[c];
            cs.base = static_cast<const unsigned char*>(base);
            cs.es = static_cast<uint32_t>(es);
            cs.coll = static_cast<uint32_t>(coll);
            cs.cap = static_cast<uint32_t>((cap * es + 32 + 15) & ~size_t(15));
            cs.soff = off;
            off += cs.cap;
        };
        add(J_PT, b->jet_pt, kes, 0, cj);
        add(J_ETA, b->jet_eta, kes, 0, cj);
        add(J_PHI, b->jet_phi, kes, 0, cj);
        add(J_MASS, b->jet_mass, kes, 0, cj);
        add(J_BTAG, b->jet_btag, bes, 0, cj);
        add(M_PT, b->mu_pt, kes, 1, cl);
        add(M_ETA, b->mu_eta, kes, 1, cl);
        add(M_PHI, b->mu_phi, kes, 1, cl);
        add(M_ISO, b->mu_iso, 4, 1, cl);
        add(M_TIGHT, b->mu_tight, 1, 1, cl);
        add(E_PT, b->el_pt, kes, 2, cl);
        add(E_ETA, b->el_eta, kes, 2, cl);
        add(E_PHI, b->el_phi, kes, 2, cl);
        add(E_ISO, b->el_iso, 4, 2, cl);
        add(E_TIGHT, b->el_tight, 1, 2, cl);
        auto up = [](size_t x) { return static_cast<uint32_t>((x + 127) & ~size_t(127)); };
        L.stage_bytes = up(kHdr + off);
        size_t at = 2 * static_cast<size_t>(L.stage_bytes);
        L.bars = static_cast<uint32_t>(at);
        at += 32 + 48 + 16;   // four mbarriers, spans of the next tile
        L.edges = static_cast<uint32_t>(at);
        at += static_cast<size_t>((P.n_edges + 3) & ~3) * 4;
        L.queue = static_cast<uint32_t>(at);
        at += static_cast<size_t>(E) * R_WORDS * 4;
        L.acc_words = static_cast<int>(cj / 32 + 2);
        L.acc = static_cast<uint32_t>(at);
        at += static_cast<size_t>(E / 32) * L.acc_words * 4;
        L.tri = static_cast<uint32_t>(at);
        at += 256;
        at = (at + 15) & ~size_t(15);
        L.hist = static_cast<uint32_t>(at);
        if (with_hist) at += static_cast<size_t>(P.n_var) * P.total_bins * (8 + 8 + 4);
        L.total = static_cast<uint32_t>((at + 15) & ~size_t(15));
        return L.total <= static_cast<size_t>(di.smem_optin);
    };
    const int max_e = std::min(kMaxThreads, g_tuning.warps > 0 ? 32 * g_tuning.warps : kMaxThreads);
    Layout L;
    int E = 0;
    bool smem_hist = false;
    for (int e = max_e; e >= 128 && E == 0; e -= 32)
        if (layout_for(e, true, L)) {
            E = e;
            smem_hist = true;
        }
    for (int e = max_e; e >= 32 && E == 0; e -= 32)
        if (layout_for(e, false, L)) E = e;
    if (E == 0) return fail(HEPACC_ERR_INVALID_ARG, "chain stage buffers do not fit in shared memory");
    if (!smem_hist) layout_for(E, false, L);
    else layout_for(E, true, L);

    LaunchArgs a;
    a.layout = L;
    a.P = &P;
    a.C = C;
    a.joff = b->jet_offsets;
    a.moff = b->mu_offsets;
    a.eoff = b->el_offsets;
    a.offsets_type = b->offsets_type;
    a.btag_type = b->btag_type;
    a.n = n;
    a.out = o;
    a.debug = debug;
    a.smem_hist = smem_hist;
    a.block = E;
    a.grid = g_tuning.grid;
    a.stream = s;
    switch (b->kin_type) {
        case HEPACC_F32: return run_f32(a);
        case HEPACC_F16: return run_f16(a);
        default: return run_bf16(a);
    }
}
