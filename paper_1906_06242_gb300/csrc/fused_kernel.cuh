// The fused benchmark chain of Section IV of arXiv:1906.06242, compacting
// form (kernel k_fused; the host side is in chain.cu, the typed launchers in
// fused_<type>.cu).
//
// Persistent blocks of NT threads work on tiles of NT consecutive events:
//  * staging: a tile's span of every column the chain reads (15 columns) is
//    copied into one of S shared-memory stages by bulk asynchronous copies
//    (cp.async.bulk, the TMA engine), one copy per column issued by one lane
//    each, completion on the stage's mbarrier; S - 1 tiles are in flight
//    while one is processed. A tile whose spans do not fit the stage is read
//    from global memory instead (same code, another accessor).
//  * selection (one warp per 32 events of the tile, thread = event): lepton
//    selection with lanes over the warp's leptons and ballots; then each
//    event with exactly one selected lepton walks its jets once (|eta|,
//    Delta R) and keeps two thresholds, the second-largest accepted jet pt
//    p2 and the largest accepted b-tagged jet pt pb, which decide every
//    jet-pt variation s_k: fl(p2 s_k) > cut and fl(pb s_k) > cut (x ->
//    fl(x s) is non-decreasing for s > 0). With jet-energy correction
//    tables (a factor per jet and variation) there is no common order: each
//    accepted jet's table position is found once and every variation counts
//    its selected jets and b-jets directly (as bit masks over variations).
//  * compaction: an event that passes any variation appends its summary and
//    all its jets (lanes over the warp's queued jets) to a block-wide buffer
//    in shared memory; a warp reserves its space with one atomic.
//  * pairs: when the buffer is nearly full (and at the end), the whole block
//    drains it with one thread per (event, variation) pair: jet counts, HT
//    and the mass sum in element order, the leading pair, the max-|sum pT|
//    triplet, the invariant masses, the 20 variables and their histogram
//    fills (global atomics). With per-event outputs every event is queued
//    and writes its outputs here. The drain first computes, once per
//    buffered accepted jet, sin and cos of phi and (with tables) the jet's
//    table position, which every variation of the event then reuses.
// A warp whose reservation does not fit processes its events' pairs itself
// (thread = event) from the stage; so does a tile that is not staged.
#pragma once

#include <type_traits>

#include "chain_kernel.cuh"

namespace hepacc {
namespace fused {

using chain::BatchDesc;
using chain::ChainOut;
using chain::ChainParams;
using chain::kNV;
using chain::NC;
using chain::qnan;
using chain::SampleDesc;
using namespace chain;   // column indices J_PT ... E_TIGHT

constexpr int kMaxStages = 4;
constexpr int kHdrBytes = 96;   // stage header: spans (3 x int64), column offsets (15 x u32), staged flag
constexpr int kMiscWords = 36;  // misc region: counter word, three spare words, 32 warp totals; the
                                // column specifications follow

// Shared-memory layout of a block (byte offsets into dynamic shared memory).
struct FLayout {
    ColSpec col[NC];        // soff: offset of the column's region inside a stage, after the header
    uint32_t stage_bytes;   // one stage
    int stages;             // S
    uint32_t bars;          // full[S] mbarriers
    uint32_t edges;         // histogram edges (n_edges floats)
    uint32_t scales;        // n_var floats
    uint32_t jec;           // jet-energy correction edges: eta, then pt
    uint32_t samples;       // flat launches: the samples' descriptors
    int cap_ev, cap_j;      // buffer capacity: events, jets
    // buffered events
    uint32_t b_e, b_s, b_w, b_lpt, b_leta, b_lphi, b_liso, b_nlep, b_j0, b_nj, b_ps;   // 4 bytes each
    uint32_t b_q, b_p;      // 8 bytes each: variations to process, variations that pass
    // buffered jets
    uint32_t j_pt, j_eta, j_phi, j_m, j_bt, j_c, j_s;   // float
    uint32_t j_acc;         // uint8
    uint32_t j_jo, j_ju;    // int32, float: correction-table positions (tables only)
    uint32_t misc;          // counter word (events << 16 | jets), warp scan scratch, column specifications
    uint32_t total;
};

// The result of one (event, variation) pair: the 20 variables and the
// indices (local to the event; -1 = none).
struct PairRes {
    float v[kNV];
    int njet, nb, lead, sub, ta, tb, tc;
};

__device__ __forceinline__ int popc64(uint64_t x) { return __popcll(x); }

// Position of the r-th (0-based) set bit of x (x has more than r set bits).
__device__ __forceinline__ int nth_bit64(uint64_t x, int r) {
    const uint32_t lo = static_cast<uint32_t>(x);
    const int nlo = __popc(lo);
    if (r < nlo) return static_cast<int>(__fns(lo, 0, r + 1));
    return 32 + static_cast<int>(__fns(static_cast<uint32_t>(x >> 32), 0, r - nlo + 1));
}

// Column accessors of a tile: staged (shared-memory offsets of each
// column's first element of the tile) or direct (global addresses).
struct SCols {
    uint32_t off[NC];
    template <typename T>
    __device__ __forceinline__ T ld(int c, int r) const {
        return *reinterpret_cast<const T*>(g_dyn_smem + off[c] + r * static_cast<int>(sizeof(T)));
    }
};
struct DCols {
    const unsigned char* p[NC];
    template <typename T>
    __device__ __forceinline__ T ld(int c, int r) const {
        return reinterpret_cast<const T*>(p[c])[r];
    }
};

// Lepton selection of element i of the muons (c0 = M_PT) or electrons (E_PT).
template <typename KT, class A>
__device__ __forceinline__ bool lep_sel(const A& T, const ChainParams& P, int c0, int i) {
    return Elem<KT>::f(T.template ld<KT>(c0, i)) > P.lep_pt_min &&
           fabsf(Elem<KT>::f(T.template ld<KT>(c0 + 1, i))) < P.lep_abseta_max && T.template ld<uint8_t>(c0 + 4, i) != 0 &&
           T.template ld<float>(c0 + 3, i) < P.lep_iso_max;
}

// Jet acceptance (everything but the pt cut): |eta| below the cut and Delta
// R^2 not below the cut to every selected lepton of the event. The event's
// selected leptons: none, exactly one (leta, lphi), or several (recounted
// from its lepton ranges [m0, m1), [e0, e1)).
template <typename KT, class A>
__device__ __forceinline__ bool jet_acc(const A& T, const ChainParams& P, int i, int nlep, float leta, float lphi,
                                        int m0, int m1, int e0, int e1) {
    const float eta = Elem<KT>::f(T.template ld<KT>(J_ETA, i));
    if (!(fabsf(eta) < P.jet_abseta_max)) return false;
    if (nlep == 0) return true;
    const float phi = Elem<KT>::f(T.template ld<KT>(J_PHI, i));
    if (nlep == 1) return !(dr2_f32(eta, phi, leta, lphi) < P.dr2_cut);
    for (int l = m0; l < m1; ++l)
        if (lep_sel<KT>(T, P, M_PT, l) &&
            dr2_f32(eta, phi, Elem<KT>::f(T.template ld<KT>(M_ETA, l)), Elem<KT>::f(T.template ld<KT>(M_PHI, l))) <
                P.dr2_cut)
            return false;
    for (int l = e0; l < e1; ++l)
        if (lep_sel<KT>(T, P, E_PT, l) &&
            dr2_f32(eta, phi, Elem<KT>::f(T.template ld<KT>(E_ETA, l)), Elem<KT>::f(T.template ld<KT>(E_PHI, l))) <
                P.dr2_cut)
            return false;
    return true;
}

// Jet-energy correction tables in shared memory (edges) and global memory
// (contents, [n_var][neta + 2][npt + 2]).
struct JecTab {
    const float* eta_e;   // neta + 1 edges
    const float* pt_e;    // npt + 1 edges
    const float* contents;
    int neta, npt;
    float eta_invw;       // eta bins per unit (first guess of the bin search)
};

// Where a jet (pt, eta) reads every variation's table: the offset, inside
// one variation's [neta + 2][npt + 2] table, of the pt bin b of its eta row
// (under- and overflow rows included) and the interpolation weight u, such
// that the correction of variation k is y_b + u (y_{b+1} - y_b) with y the
// row of table k. Between the centres c_b = (e[b-1] + e[b]) / 2 of the pt
// bins u = (pt - c_b) / (c_{b+1} - c_b); below the first centre b = 1 and
// above the last b = npt, both with u = 0 (clamped, so y_b exactly); every
// operation binary32 rounded as written (the lookup of
// hepacc_get_bin_contents). A NaN pt or eta gives u = NaN (a NaN factor).
struct JecPos {
    int off;
    float u;
};
__device__ __forceinline__ JecPos jec_pos(const JecTab& t, float pt, float eta) {
    const int row = find_bin(eta, t.eta_e, t.neta, t.eta_invw);
    if (row < 0 || pt != pt) return JecPos{0, qnan()};
    const int rb = row * (t.npt + 2);
    const int nb = t.npt;
    auto centre = [&](int b) { return __fmul_rn(__fadd_rn(t.pt_e[b - 1], t.pt_e[b]), 0.5f); };
    if (nb == 1 || pt < centre(1)) return JecPos{rb + 1, 0.0f};
    if (pt >= centre(nb)) return JecPos{rb + nb, 0.0f};
    int lo = 1, hi = nb - 1;   // the smallest b with pt < c_{b+1} (then c_b <= pt)
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (pt < centre(mid + 1))
            hi = mid;
        else
            lo = mid + 1;
    }
    const float cb = centre(lo), cb1 = centre(lo + 1);
    return JecPos{rb + lo, __fdiv_rn(__fsub_rn(pt, cb), __fsub_rn(cb1, cb))};
}

// The correction of variation k at a jet's position (y_b + 0 = y_b at the
// clamped ends: the tables hold finite values).
__device__ __forceinline__ float jec_factor(const JecTab& t, int k, JecPos q) {
    const float* r = t.contents + static_cast<int64_t>(k) * ((t.neta + 2) * (t.npt + 2)) + q.off;
    const float yb = __ldg(r), yb1 = __ldg(r + 1);
    return __fadd_rn(yb, __fmul_rn(q.u, __fsub_rn(yb1, yb)));
}

// Jets of one event in the shared-memory buffer (binary32, widened).
struct BufJets {
    const float *pt_, *eta_, *phi_, *m_, *bt_, *c_, *s_;
    const uint8_t* acc_;
    const int* jo_;     // correction-table positions of the accepted jets (with tables)
    const float* ju_;
    int n;
    template <class TB>
    __device__ __forceinline__ JecPos jpos(int i, const TB&) const { return JecPos{jo_[i], ju_[i]}; }
    __device__ __forceinline__ bool acc(int i) const { return acc_[i] != 0; }
    __device__ __forceinline__ float pt(int i) const { return pt_[i]; }
    __device__ __forceinline__ float eta(int i) const { return eta_[i]; }
    __device__ __forceinline__ float phi(int i) const { return phi_[i]; }
    __device__ __forceinline__ float mass(int i) const { return m_[i]; }
    __device__ __forceinline__ float btag(int i) const { return bt_[i]; }
    __device__ __forceinline__ void cs(int i, float& c, float& s) const {
        c = c_[i];
        s = s_[i];
    }
};

// Jets of one event read from a tile accessor (stage or global memory),
// acceptance evaluated on the way.
template <typename KT, typename BT, class A>
struct ColJets {
    A T;   // held by value: an accessor whose address is taken would live in local memory
    const ChainParams* P;
    int j0, n;
    int nlep;
    float leta, lphi;
    int m0, m1, e0, e1;
    __device__ __forceinline__ bool acc(int i) const {
        return jet_acc<KT>(T, *P, j0 + i, nlep, leta, lphi, m0, m1, e0, e1);
    }
    __device__ __forceinline__ float pt(int i) const { return Elem<KT>::f(T.template ld<KT>(J_PT, j0 + i)); }
    __device__ __forceinline__ float eta(int i) const { return Elem<KT>::f(T.template ld<KT>(J_ETA, j0 + i)); }
    __device__ __forceinline__ float phi(int i) const { return Elem<KT>::f(T.template ld<KT>(J_PHI, j0 + i)); }
    __device__ __forceinline__ float mass(int i) const { return Elem<KT>::f(T.template ld<KT>(J_MASS, j0 + i)); }
    __device__ __forceinline__ float btag(int i) const { return Elem<BT>::f(T.template ld<BT>(J_BTAG, j0 + i)); }
    __device__ __forceinline__ void cs(int i, float& c, float& s) const { sincosf(phi(i), &s, &c); }
    template <class TB>
    __device__ __forceinline__ JecPos jpos(int i, const TB& t) const { return jec_pos(t, pt(i), eta(i)); }
};

// A variation's jet pt: pt scaled by s, or (JEC) corrected by the
// variation's table at the jet's position (JS::jpos).
template <bool JEC>
struct VarPt {
    float s;
    int k;
    JecTab t;
    template <class JS>
    __device__ __forceinline__ float operator()(const JS& J, int i) const {
        if constexpr (JEC)
            return __fmul_rn(J.pt(i), jec_factor(t, k, J.jpos(i, t)));
        else
            return __fmul_rn(J.pt(i), s);
    }
};

// One (event, variation): the jets selected under the variation (accepted
// and pt_k > cut, pt_k = ptk_of(pt, eta)), their counts, HT and mass sum in element order, the
// leading and sub-leading jet (first occurrence on ties), the max btag,
// the triplet with the largest |sum pT| (first in lexicographic order on
// ties; ranked in binary32 from sin/cos of phi), the dijet and trijet
// masses. Fills v[0..12], v[18] and the counts and indices.
template <class JS, class VP>
__device__ __forceinline__ void process_pair(const JS& J, const VP& ptk_of, const ChainParams& P, PairRes& R) {
    auto ptk_at = [&](int i) { return ptk_of(J, i); };
    const int n = J.n;
    float ht = 0.0f, summ = 0.0f, maxbt = qnan(), lead_pt = 0.0f, sub_pt = 0.0f;
    int lead = -1, sub = -1, nsel = 0, nbj = 0;
    uint64_t selm = 0;   // selected jets among the first 64
    for (int i = 0; i < n; ++i) {
        if (!J.acc(i)) continue;
        const float ptk = ptk_at(i);
        if (!(ptk > P.jet_pt_min)) continue;
        const float bt = J.btag(i);
        nbj += bt > P.btag_min ? 1 : 0;
        ht = __fadd_rn(ht, ptk);
        summ = __fadd_rn(summ, J.mass(i));
        if (lead < 0 || ptk > lead_pt) {
            sub = lead;
            sub_pt = lead_pt;
            lead = i;
            lead_pt = ptk;
        } else if (sub < 0 || ptk > sub_pt) {
            sub = i;
            sub_pt = ptk;
        }
        if (!(bt != bt) && (maxbt != maxbt || bt > maxbt)) maxbt = bt;
        if (i < 64) selm |= 1ull << i;
        ++nsel;
    }
#pragma unroll
    for (int h = 0; h < kNV; ++h) R.v[h] = qnan();
    R.v[0] = ht;
    R.v[8] = static_cast<float>(nsel);
    R.v[9] = static_cast<float>(nbj);
    R.v[10] = maxbt;
    R.v[18] = summ;
    R.njet = nsel;
    R.nb = nbj;
    R.lead = lead;
    R.sub = sub;
    R.ta = R.tb = R.tc = -1;
    // max |sum pT| triplet
    float best = -1.0f;
    int ta = -1, tb = -1, tc = -1;
    if (nsel >= 3) {
        if (n <= 64) {
            for (uint64_t ma = selm; ma; ma &= ma - 1) {
                const int a = __ffsll(static_cast<long long>(ma)) - 1;
                float ca, sa;
                J.cs(a, ca, sa);
                const float pa = ptk_at(a);
                const float ax = pa * ca, ay = pa * sa;
                for (uint64_t mb = ma & (ma - 1); mb; mb &= mb - 1) {
                    const int b = __ffsll(static_cast<long long>(mb)) - 1;
                    float cb, sb;
                    J.cs(b, cb, sb);
                    const float pb = ptk_at(b);
                    const float bx = ax + pb * cb, by = ay + pb * sb;
                    for (uint64_t mc = mb & (mb - 1); mc; mc &= mc - 1) {
                        const int c = __ffsll(static_cast<long long>(mc)) - 1;
                        float cc, sc;
                        J.cs(c, cc, sc);
                        const float pc = ptk_at(c);
                        const float tx = bx + pc * cc, ty = by + pc * sc;
                        const float val = tx * tx + ty * ty;
                        if (val > best) {
                            best = val;
                            ta = a;
                            tb = b;
                            tc = c;
                        }
                    }
                }
            }
        } else {
            auto sel = [&](int i) { return J.acc(i) && ptk_at(i) > P.jet_pt_min; };
            for (int a = 0; a < n; ++a) {
                if (!sel(a)) continue;
                float ca, sa;
                J.cs(a, ca, sa);
                const float pa = ptk_at(a);
                const float ax = pa * ca, ay = pa * sa;
                for (int b = a + 1; b < n; ++b) {
                    if (!sel(b)) continue;
                    float cb, sb;
                    J.cs(b, cb, sb);
                    const float pb = ptk_at(b);
                    const float bx = ax + pb * cb, by = ay + pb * sb;
                    for (int c = b + 1; c < n; ++c) {
                        if (!sel(c)) continue;
                        float cc, sc;
                        J.cs(c, cc, sc);
                        const float pc = ptk_at(c);
                        const float tx = bx + pc * cc, ty = by + pc * sc;
                        const float val = tx * tx + ty * ty;
                        if (val > best) {
                            best = val;
                            ta = a;
                            tb = b;
                            tc = c;
                        }
                    }
                }
            }
        }
    }
    MassObj ol, os;
    float p_ls = 0.0f;   // E_lead E_sub - p_lead . p_sub, shared with the triplet
    if (lead >= 0) {
        R.v[1] = lead_pt;
        R.v[2] = J.eta(lead);
        R.v[3] = J.phi(lead);
        R.v[4] = J.mass(lead);
        R.v[5] = J.btag(lead);
        ol = mass_obj(R.v[1], R.v[2], R.v[3], R.v[4]);
    }
    if (sub >= 0) {
        R.v[6] = sub_pt;
        os = mass_obj(sub_pt, J.eta(sub), J.phi(sub), J.mass(sub));
        p_ls = pair_dot(ol, os);
        R.v[7] = sqrtf(ol.m * ol.m + os.m * os.m + 2.0f * p_ls);
    }
    if (nsel >= 3 && ta >= 0) {
        auto obj = [&](int i) {
            if (i == lead) return ol;
            if (i == sub) return os;
            return mass_obj(ptk_at(i), J.eta(i), J.phi(i), J.mass(i));
        };
        const MassObj oa = obj(ta), ob = obj(tb), oc = obj(tc);
        auto pd = [&](int i, const MassObj& x, int j, const MassObj& y) {
            if ((i == lead && j == sub) || (i == sub && j == lead)) return p_ls;
            return pair_dot(x, y);
        };
        const float msum = oa.m * oa.m + ob.m * ob.m + oc.m * oc.m;
        R.v[11] = sqrtf(msum + 2.0f * (pd(ta, oa, tb, ob) + pd(ta, oa, tc, oc) + pd(tb, ob, tc, oc)));
        R.v[12] = sqrtf(best);
        R.ta = ta;
        R.tb = tb;
        R.tc = tc;
    }
}

// Per-event outputs (optional) and the histogram fill of one pair: event e
// of a sample with n events, variation k; only passing pairs fill.
template <bool DEBUG>
__device__ __forceinline__ void emit(const ChainParams& P, const float* s_edges, const ChainOut& out, int64_t n,
                                     int64_t e, int k, bool pass, const PairRes& R) {
    if (DEBUG) {
        const int64_t kn = static_cast<int64_t>(k) * n;
        if (out.ev_pass) out.ev_pass[kn + e] = pass ? 1 : 0;
        if (out.ev_njet) out.ev_njet[kn + e] = R.njet;
        if (out.ev_nb) out.ev_nb[kn + e] = R.nb;
        if (out.ev_idx) {
            int32_t* ix = out.ev_idx + static_cast<int64_t>(k) * 5 * n;
            ix[e] = R.lead;
            ix[n + e] = R.sub;
            ix[2 * n + e] = R.njet >= 3 ? R.ta : -1;
            ix[3 * n + e] = R.njet >= 3 ? R.tb : -1;
            ix[4 * n + e] = R.njet >= 3 ? R.tc : -1;
        }
        if (out.ev_vars) {
            float* vv = out.ev_vars + static_cast<int64_t>(k) * kNV * n;
#pragma unroll
            for (int h = 0; h < kNV; ++h) vv[h * n + e] = R.v[h];
        }
    }
    if (!pass) return;
    const double wd = static_cast<double>(R.v[19]);
    const int base = k * P.total_bins;
#pragma unroll
    for (int h = 0; h < kNV; ++h) {
        const int bin = find_bin_lim(R.v[h], s_edges + P.eoff[h], P.e_lo[h], P.e_hi[h], P.nbins[h], P.invw[h]);
        if (bin < 0) continue;
        const int at = base + P.boff[h] + bin;
        atomicAdd(&out.counts[at], 1ull);
        atomicAdd(&out.sumw[at], wd);
        if (out.sumw2) atomicAdd(&out.sumw2[at], wd * wd);
    }
}

// Blocks per SM the register allocation is sized for: 128-thread blocks at
// three per SM (168 registers, the pair work without spills), the others as
// many as their shared-memory layouts allow (64: four, 256: one).
constexpr int min_blocks_for(int nt) { return nt == 128 ? 3 : nt == 64 ? 4 : 1; }

template <typename KT, typename BT, typename OffT, bool DEBUG, bool FLAT, int NT, bool JEC>
__global__ void __launch_bounds__(NT, min_blocks_for(NT))
    k_fused(const __grid_constant__ FLayout L, const __grid_constant__ ChainParams P,
            const __grid_constant__ BatchDesc B) {
    static_assert(NT % 32 == 0 && NT <= 1024, "block of whole warps");
    unsigned char* smem = g_dyn_smem;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int S = L.stages;
    float* s_edges = reinterpret_cast<float*>(smem + L.edges);
    float* s_scales = reinterpret_cast<float*>(smem + L.scales);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bars);
    uint32_t* s_cnt = reinterpret_cast<uint32_t*>(smem + L.misc);
    uint32_t* s_ws = s_cnt + 4;   // warp totals of a block scan
    const uint32_t smem0 = smem_addr(smem);
    SampleDesc* s_samples = reinterpret_cast<SampleDesc*>(smem + L.samples);
    ColSpec* s_cols = reinterpret_cast<ColSpec*>(smem + L.misc + kMiscWords * 4);

    // buffer arrays
    int32_t* b_e = reinterpret_cast<int32_t*>(smem + L.b_e);
    int32_t* b_s = reinterpret_cast<int32_t*>(smem + L.b_s);
    float* b_w = reinterpret_cast<float*>(smem + L.b_w);
    float* b_lpt = reinterpret_cast<float*>(smem + L.b_lpt);
    float* b_leta = reinterpret_cast<float*>(smem + L.b_leta);
    float* b_lphi = reinterpret_cast<float*>(smem + L.b_lphi);
    float* b_liso = reinterpret_cast<float*>(smem + L.b_liso);
    int32_t* b_nlep = reinterpret_cast<int32_t*>(smem + L.b_nlep);
    int32_t* b_j0 = reinterpret_cast<int32_t*>(smem + L.b_j0);
    int32_t* b_nj = reinterpret_cast<int32_t*>(smem + L.b_nj);
    int32_t* b_ps = reinterpret_cast<int32_t*>(smem + L.b_ps);
    uint64_t* b_q = reinterpret_cast<uint64_t*>(smem + L.b_q);
    uint64_t* b_p = reinterpret_cast<uint64_t*>(smem + L.b_p);
    float* j_pt = reinterpret_cast<float*>(smem + L.j_pt);
    float* j_eta = reinterpret_cast<float*>(smem + L.j_eta);
    float* j_phi = reinterpret_cast<float*>(smem + L.j_phi);
    float* j_m = reinterpret_cast<float*>(smem + L.j_m);
    float* j_bt = reinterpret_cast<float*>(smem + L.j_bt);
    float* j_c = reinterpret_cast<float*>(smem + L.j_c);
    float* j_s = reinterpret_cast<float*>(smem + L.j_s);
    uint8_t* j_acc = reinterpret_cast<uint8_t*>(smem + L.j_acc);
    int32_t* j_jo = reinterpret_cast<int32_t*>(smem + L.j_jo);
    float* j_ju = reinterpret_cast<float*>(smem + L.j_ju);

    for (int i = tid; i < P.n_edges; i += NT) s_edges[i] = P.edges[i];
    for (int i = tid; i < P.n_var; i += NT) s_scales[i] = P.scales[i];
    float* s_jec = reinterpret_cast<float*>(smem + L.jec);
    if constexpr (JEC)
        for (int i = tid; i < P.jec_neta + P.jec_npt + 2; i += NT) s_jec[i] = P.jec_edges[i];
    const JecTab jt{s_jec, s_jec + P.jec_neta + 1, P.jec_contents, P.jec_neta, P.jec_npt, P.jec_eta_invw};
    // the samples' descriptors and the column specifications in shared
    // memory: lanes read them at different indices, which the constant bank
    // holding kernel parameters would serialise
    {
        const int words = (FLAT ? B.n_samples : 1) * static_cast<int>(sizeof(SampleDesc) / 8);
        for (int i = tid; i < words; i += NT)
            reinterpret_cast<uint64_t*>(s_samples)[i] = reinterpret_cast<const uint64_t*>(&B.s[0])[i];
        for (int i = tid; i < static_cast<int>(sizeof(L.col) / 8); i += NT)
            reinterpret_cast<uint64_t*>(s_cols)[i] = reinterpret_cast<const uint64_t*>(&L.col[0])[i];
    }
    if (tid == 0) {
        for (int b = 0; b < S; ++b) mbar_init(smem_addr(bars + b), 1);
        fence_mbar_init();
        *s_cnt = 0u;
    }
    __syncthreads();

    // a sample's descriptor: kernel parameters, which lanes read at one
    // index per tile or per pair (the copy issue reads the column bases at
    // a per-lane index from the shared copy instead)
    auto SD = [&](int s) -> const SampleDesc& {
        if constexpr (FLAT)
            return B.s[s];
        else
            return B.s[0];
    };
    const int64_t ntiles = FLAT ? B.tile_start[B.n_samples] : (B.s[0].n + NT - 1) / NT;
    const int64_t G = gridDim.x;
    // sample and tile within the sample of launch tile t
    auto where = [&](int64_t t, int& ts, int64_t& lt) {
        if constexpr (FLAT) {
            int k = 0;
            for (int j = 1; j < B.n_samples; ++j) k = B.tile_start[j] <= t ? j : k;
            ts = k;
            lt = t - B.tile_start[k];
        } else {
            ts = 0;
            lt = t;
        }
    };
    // warp 0: the first and last element of every collection in tile tt,
    // lane c < 6 loads element c of (first jet, muon, electron, last + 1
    // jet, muon, electron); kept in a register until the tile is issued, an
    // iteration later, so that the load latency overlaps a tile's work
    auto load_span = [&](int64_t tt) -> int64_t {
        int64_t v = 0;
        if (lane < 6) {
            int ts;
            int64_t lt;
            where(tt, ts, lt);
            const int64_t ns = SD(ts).n;
            const int64_t a = lt * NT;
            const int64_t z = a + NT < ns ? a + NT : ns;
            v = ldoff(static_cast<const OffT*>(SD(ts).off[lane % 3]), lane < 3 ? a : z);
        }
        return v;
    };
    // warp 0: header of stage b and the bulk copies of tile tt's spans (sp
    // as load_span returned it), column c by lane c (whole 16-byte chunks);
    // a tile that does not fit is marked unstaged and its barrier completes
    // without bytes
    auto issue = [&](int b, int64_t tt, int64_t sp) {
        int ts;
        int64_t lt;
        where(tt, ts, lt);
        const SampleDesc& sd = SD(ts);
        unsigned char* st = smem + b * L.stage_bytes;
        int64_t* hdr = reinterpret_cast<int64_t*>(st);
        uint32_t* hoff = reinterpret_cast<uint32_t*>(st + 32);
        uint32_t bytes = 0;
        uintptr_t a16 = 0;
        bool fits_c = true;
        const int coll = lane < NC ? static_cast<int>(s_cols[lane].coll) : 0;
        const int64_t S0 = __shfl_sync(0xffffffffu, sp, coll);
        const int64_t T0 = __shfl_sync(0xffffffffu, sp, 3 + coll);
        if (lane < NC) {
            const ColSpec& cs = s_cols[lane];
            const uintptr_t cb = reinterpret_cast<uintptr_t>(s_samples[ts].col[lane]);
            const uintptr_t a = cb + static_cast<uintptr_t>(S0) * cs.es;
            const uintptr_t z = cb + static_cast<uintptr_t>(T0) * cs.es;
            a16 = a & ~uintptr_t(15);
            bytes = T0 > S0 ? static_cast<uint32_t>(((z + 15) & ~uintptr_t(15)) - a16) : 0u;
            fits_c = T0 - S0 <= static_cast<int64_t>(cs.cap) && bytes <= cs.cap;
            hoff[lane] = b * L.stage_bytes + kHdrBytes + cs.soff + static_cast<uint32_t>(a & 15u);
        }
        const bool fits = __all_sync(0xffffffffu, fits_c);
        uint32_t total = bytes;
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) total += __shfl_xor_sync(0xffffffffu, total, d);
        if (lane < 3) hdr[lane] = sp;
        if (lane == 0) hoff[NC] = fits ? 1u : 0u;
        // one proxy fence for the warp: the stage's earlier generic reads
        // are ordered before the copies that overwrite it
        __syncwarp();
        fence_proxy_async_smem();
        const uint32_t bar = smem_addr(bars + b);
        if (lane == 0) mbar_arrive_expect_tx(bar, fits ? total : 0u);
        __syncwarp();
        if (fits && lane < NC && bytes > 0)
            bulk_g2s(smem0 + b * L.stage_bytes + kHdrBytes + s_cols[lane].soff, reinterpret_cast<const void*>(a16),
                     bytes, bar);
    };
    // this thread's offsets and weight in tile t
    auto own_offsets = [&](int64_t t, int64_t (&os)[3], int64_t (&ot)[3], float& w) {
        int ts;
        int64_t lt;
        where(t, ts, lt);
        const SampleDesc& sd = SD(ts);
        const int64_t ns = sd.n;
        const int64_t e = lt * NT + tid;
        const int64_t elo = e < ns ? e : ns, ehi = e + 1 < ns ? e + 1 : ns;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            os[c] = ldoff(static_cast<const OffT*>(sd.off[c]), elo);
            ot[c] = ldoff(static_cast<const OffT*>(sd.off[c]), ehi);
        }
        w = e < ns ? sd.weight[e] : 0.0f;
    };

    // Drains the buffer: all threads, one (event, variation) pair per thread
    // at a time. Ends with a barrier after which the buffer is empty.
    auto drain = [&]() {
        const uint32_t cnt = *s_cnt;
        const int nev = static_cast<int>(cnt >> 16);
        const int nj = static_cast<int>(cnt & 0xffffu);
        // sin and cos of the accepted jets' phi, once for every variation
        // (and their correction-table positions)
        for (int j = tid; j < nj; j += NT)
            if (j_acc[j]) {
                sincosf(j_phi[j], &j_s[j], &j_c[j]);
                if constexpr (JEC) {
                    const JecPos jp = jec_pos(jt, j_pt[j], j_eta[j]);
                    j_jo[j] = jp.off;
                    j_ju[j] = jp.u;
                }
            }
        // first pair of every event: block-wide exclusive scan of its variation count
        const int ept = (nev + NT - 1) / NT;
        const int lo = min(tid * ept, nev), hi = min(lo + ept, nev);
        int local = 0;
        for (int i = lo; i < hi; ++i) local += popc64(b_q[i]);
        int x = local;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        if (lane == 31) s_ws[warp] = static_cast<uint32_t>(x);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < NT / 32; ++w) {
            const int v = static_cast<int>(s_ws[w]);
            before += w < warp ? v : 0;
            total += v;
        }
        int run = before + x - local;
        for (int i = lo; i < hi; ++i) {
            b_ps[i] = run;
            run += popc64(b_q[i]);
        }
        if (tid == 0) *s_cnt = 0u;   // read by everyone above; appends resume after the closing barrier
        __syncthreads();
        for (int i = tid; i < total; i += NT) {
            // the event: the last one whose first pair is at or before i
            int a = 0, z = nev - 1;
            while (a < z) {
                const int m = (a + z + 1) >> 1;
                if (b_ps[m] <= i)
                    a = m;
                else
                    z = m - 1;
            }
            const int ev = a;
            const int k = nth_bit64(b_q[ev], i - b_ps[ev]);
            const int j0 = b_j0[ev];
            BufJets J{j_pt + j0, j_eta + j0, j_phi + j0, j_m + j0, j_bt + j0, j_c + j0, j_s + j0, j_acc + j0,
                      j_jo + j0, j_ju + j0, b_nj[ev]};
            PairRes R;
            process_pair(J, VarPt<JEC>{s_scales[k], k, jt}, P, R);
            if (b_nlep[ev] >= 1) {
                R.v[13] = b_lpt[ev];
                R.v[14] = b_leta[ev];
                R.v[15] = b_lphi[ev];
                R.v[16] = b_liso[ev];
                R.v[17] = __fadd_rn(R.v[0], R.v[13]);
            }
            R.v[19] = b_w[ev];
            const SampleDesc& sd = SD(b_s[ev]);
            emit<DEBUG>(P, s_edges, sd.out, sd.n, b_e[ev], k, ((b_p[ev] >> k) & 1ull) != 0, R);
        }
        __syncthreads();
    };

    int64_t cs_[3] = {0, 0, 0}, ct_[3] = {0, 0, 0};
    float cw_ = 0.0f;
    const int64_t t0 = blockIdx.x;
    // prologue: the first S - 1 tiles of this block in flight
    int64_t sp_next = 0;   // warp 0: spans of the next tile to issue
    if (warp == 0) {
        for (int j = 0; j < S - 1; ++j) {
            const int64_t tj = t0 + j * G;
            if (tj >= ntiles) break;
            issue(j, tj, load_span(tj));
        }
        const int64_t tn = t0 + (S - 1) * G;
        if (tn < ntiles) sp_next = load_span(tn);
    }
    if (t0 < ntiles) own_offsets(t0, cs_, ct_, cw_);
    bool stop = false;
    int maxj = 0, maxe = 0;   // most jets / events one tile appended so far (same in every thread)
    uint32_t last_cnt = 0;
    int64_t it = 0;
    // the tile's stage, the stage refilled at its start (the previous
    // tile's), and the phase parity of each stage's barrier: advanced once
    // per tile, so that the loop does no integer division
    int b = 0, bprev = S - 1;
    uint32_t parbits = 0u;
    for (int64_t tile = t0; tile < ntiles; tile += G, ++it) {
        const int64_t next = tile + G;
        int64_t ns_[3] = {0, 0, 0}, nt_[3] = {0, 0, 0};
        float nw_ = 0.0f;
        if (next < ntiles) own_offsets(next, ns_, nt_, nw_);
        const bool ok = mbar_wait_bounded(smem_addr(bars + b), (parbits >> b) & 1u);
        parbits ^= 1u << b;
        // every thread is done with the previous tile: its stage is free and
        // the buffer counter is settled
        if (!__syncthreads_and(ok)) {
            stop = true;
            break;
        }
        {
            const uint32_t cnt = *s_cnt;
            const int dj = static_cast<int>(cnt & 0xffffu) - static_cast<int>(last_cnt & 0xffffu);
            const int de = static_cast<int>(cnt >> 16) - static_cast<int>(last_cnt >> 16);
            maxj = max(maxj, dj);
            maxe = max(maxe, de);
            // refill the stage of the previous tile
            if (warp == 0) {
                const int64_t tn = tile + (S - 1) * G;
                if (tn < ntiles) {
                    issue(bprev, tn, sp_next);
                    if (tn + G < ntiles) sp_next = load_span(tn + G);
                }
            }
            // drain when the next tile might not fit
            if (static_cast<int>(cnt & 0xffffu) + maxj > L.cap_j || static_cast<int>(cnt >> 16) + maxe > L.cap_ev) {
                drain();
                last_cnt = 0;
            } else {
                last_cnt = cnt;
            }
        }

        const unsigned char* st = smem + b * L.stage_bytes;
        const int64_t* hdr = reinterpret_cast<const int64_t*>(st);
        const uint32_t* hoff = reinterpret_cast<const uint32_t*>(st + 32);
        int cur_s;
        int64_t ltile;
        where(tile, cur_s, ltile);
        const SampleDesc& sd = SD(cur_s);
        const int64_t n = sd.n;
        const int64_t e = ltile * NT + tid;
        const bool valid = e < n;
        int rs[3], rt[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            rs[c] = static_cast<int>(cs_[c] - hdr[c]);
            rt[c] = static_cast<int>(ct_[c] - hdr[c]);
        }
        int W0[3], W1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            W0[c] = __shfl_sync(0xffffffffu, rs[c], 0);
            W1[c] = __shfl_sync(0xffffffffu, rt[c], 31);
        }

        auto body = [&](const auto& T) {
            // bits of [lo, hi) inside the 32-element window starting at base
            auto range_mask = [](int lo, int hi, int base) -> unsigned {
                const int a = lo - base > 0 ? lo - base : 0;
                const int z = hi - base < 32 ? hi - base : 32;
                if (z <= a) return 0u;
                const unsigned top = z >= 32 ? 0xffffffffu : ((1u << z) - 1u);
                return top & ~((1u << a) - 1u);
            };
            // leptons, lanes over the warp's muons then electrons
            int nlep = 0, lfirst = -1, lflav = 0;
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                const int c0 = f == 0 ? M_PT : E_PT;
                const int coll = 1 + f;
                for (int base = W0[coll]; base < W1[coll]; base += 32) {
                    const int p = base + lane;
                    const bool sel = p < W1[coll] && lep_sel<KT>(T, P, c0, p);
                    const unsigned hit = __ballot_sync(0xffffffffu, sel) & range_mask(rs[coll], rt[coll], base);
                    nlep += __popc(hit);
                    if (lfirst < 0 && hit) {
                        lfirst = base + __ffs(hit) - 1;
                        lflav = f;
                    }
                }
            }
            if (!valid) nlep = 0;
            float lpt = qnan(), leta = qnan(), lphi = qnan(), liso = qnan();
            // (constant column indices: an accessor indexed at run time would live in local memory)
            if (valid && lfirst >= 0 && lflav == 0) {
                lpt = Elem<KT>::f(T.template ld<KT>(M_PT, lfirst));
                leta = Elem<KT>::f(T.template ld<KT>(M_ETA, lfirst));
                lphi = Elem<KT>::f(T.template ld<KT>(M_PHI, lfirst));
                liso = T.template ld<float>(M_ISO, lfirst);
            } else if (valid && lfirst >= 0) {
                lpt = Elem<KT>::f(T.template ld<KT>(E_PT, lfirst));
                leta = Elem<KT>::f(T.template ld<KT>(E_ETA, lfirst));
                lphi = Elem<KT>::f(T.template ld<KT>(E_PHI, lfirst));
                liso = T.template ld<float>(E_ISO, lfirst);
            }
            if (DEBUG && valid && sd.out.ev_nlep) sd.out.ev_nlep[e] = nlep;
            // only events with exactly one lepton can pass; with per-event
            // outputs every event is evaluated
            const bool active = valid && (DEBUG || nlep == 1);
            // thresholds: second-largest accepted jet pt, largest accepted b-tagged pt
            float p1 = -INFINITY, p2 = -INFINITY, pb = -INFINITY;
            if (!JEC && active && nlep == 1) {
                for (int i = rs[0]; i < rt[0]; ++i) {
                    if (!jet_acc<KT>(T, P, i, 1, leta, lphi, 0, 0, 0, 0)) continue;
                    const float pt = Elem<KT>::f(T.template ld<KT>(J_PT, i));
                    if (pt > p1) {
                        p2 = p1;
                        p1 = pt;
                    } else if (pt > p2) {
                        p2 = pt;
                    }
                    if (pt > pb && Elem<BT>::f(T.template ld<BT>(J_BTAG, i)) > P.btag_min) pb = pt;
                }
            }
            uint64_t pm = 0;
            if (!JEC && active && nlep == 1) {
                for (int k = 0; k < P.n_var; ++k) {
                    const float s = s_scales[k];
                    if (__fmul_rn(p2, s) > P.jet_pt_min && __fmul_rn(pb, s) > P.jet_pt_min) pm |= 1ull << k;
                }
            }
            if (JEC && active && nlep == 1) {
                // corrected jets need no common order: each accepted jet's
                // table position is found once, then the variations that
                // select it form a mask; per variation the masks record one
                // selected jet, two or more, and a selected b-jet
                uint64_t one = 0, two = 0, bsel = 0;
                for (int i = rs[0]; i < rt[0]; ++i) {
                    if (!jet_acc<KT>(T, P, i, 1, leta, lphi, 0, 0, 0, 0)) continue;
                    const float pt = Elem<KT>::f(T.template ld<KT>(J_PT, i));
                    const JecPos jp = jec_pos(jt, pt, Elem<KT>::f(T.template ld<KT>(J_ETA, i)));
                    uint64_t sel = 0;
                    for (int k = 0; k < P.n_var; ++k)
                        if (__fmul_rn(pt, jec_factor(jt, k, jp)) > P.jet_pt_min) sel |= 1ull << k;
                    two |= one & sel;
                    one |= sel;
                    if (Elem<BT>::f(T.template ld<BT>(J_BTAG, i)) > P.btag_min) bsel |= sel;
                }
                pm = two & bsel;
            }
            const uint64_t qm = DEBUG ? (valid ? (P.n_var >= 64 ? ~0ull : ((1ull << P.n_var) - 1ull)) : 0ull) : pm;
            const bool q = qm != 0ull;
            const unsigned bal = __ballot_sync(0xffffffffu, q);
            if (bal == 0u) return;
            // append: events and all their jets; lanes over the warp's queued jets
            const int njev = q ? rt[0] - rs[0] : 0;
            int xs = njev;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, xs, d);
                if (lane >= d) xs += y;
            }
            const int totj = __shfl_sync(0xffffffffu, xs, 31);
            const int jpre = xs - njev;
            const int nq = __popc(bal);
            int base_ev = -1, base_j = 0;
            if (lane == 0) {
                uint32_t old = *reinterpret_cast<volatile uint32_t*>(s_cnt);
                while (true) {
                    const int ce = static_cast<int>(old >> 16), cj = static_cast<int>(old & 0xffffu);
                    if (ce + nq > L.cap_ev || cj + totj > L.cap_j) break;
                    const uint32_t nw = (static_cast<uint32_t>(ce + nq) << 16) | static_cast<uint32_t>(cj + totj);
                    const uint32_t got = atomicCAS(s_cnt, old, nw);
                    if (got == old) {
                        base_ev = ce;
                        base_j = cj;
                        break;
                    }
                    old = got;
                }
            }
            base_ev = __shfl_sync(0xffffffffu, base_ev, 0);
            base_j = __shfl_sync(0xffffffffu, base_j, 0);
            if (base_ev >= 0) {
                if (q) {
                    const int slot = base_ev + __popc(bal & lt_mask);
                    b_e[slot] = static_cast<int32_t>(e);
                    b_s[slot] = cur_s;
                    b_w[slot] = cw_;
                    b_lpt[slot] = lpt;
                    b_leta[slot] = leta;
                    b_lphi[slot] = lphi;
                    b_liso[slot] = liso;
                    b_nlep[slot] = nlep;
                    b_j0[slot] = base_j + jpre;
                    b_nj[slot] = njev;
                    b_q[slot] = qm;
                    b_p[slot] = pm;
                }
                for (int f0 = 0; f0 < totj; f0 += 32) {
                    const int f = f0 + lane;
                    // owner: the last lane whose queued jets start at or before f
                    int own = 0;
#pragma unroll
                    for (int step = 16; step >= 1; step >>= 1) {
                        const int v = __shfl_sync(0xffffffffu, jpre, own + step);
                        if (v <= f) own += step;
                    }
                    const int o_rs = __shfl_sync(0xffffffffu, rs[0], own);
                    const int o_jp = __shfl_sync(0xffffffffu, jpre, own);
                    const int o_nl = __shfl_sync(0xffffffffu, nlep, own);
                    const float o_le = __shfl_sync(0xffffffffu, leta, own);
                    const float o_lp = __shfl_sync(0xffffffffu, lphi, own);
                    const int o_m0 = __shfl_sync(0xffffffffu, rs[1], own), o_m1 = __shfl_sync(0xffffffffu, rt[1], own);
                    const int o_e0 = __shfl_sync(0xffffffffu, rs[2], own), o_e1 = __shfl_sync(0xffffffffu, rt[2], own);
                    if (f < totj) {
                        const int i = o_rs + (f - o_jp);
                        const int d = base_j + f;
                        j_pt[d] = Elem<KT>::f(T.template ld<KT>(J_PT, i));
                        j_eta[d] = Elem<KT>::f(T.template ld<KT>(J_ETA, i));
                        j_phi[d] = Elem<KT>::f(T.template ld<KT>(J_PHI, i));
                        j_m[d] = Elem<KT>::f(T.template ld<KT>(J_MASS, i));
                        j_bt[d] = Elem<BT>::f(T.template ld<BT>(J_BTAG, i));
                        j_acc[d] = jet_acc<KT>(T, P, i, o_nl, o_le, o_lp, o_m0, o_m1, o_e0, o_e1) ? 1 : 0;
                    }
                }
            } else if (q) {
                // the buffer is full: this thread's event, every queued variation, from the tile
                using A = typename std::decay<decltype(T)>::type;
                ColJets<KT, BT, A> J{T, &P, rs[0], rt[0] - rs[0], nlep, leta, lphi, rs[1], rt[1], rs[2], rt[2]};
                for (uint64_t m = qm; m; m &= m - 1) {
                    const int k = __ffsll(static_cast<long long>(m)) - 1;
                    PairRes R;
                    process_pair(J, VarPt<JEC>{s_scales[k], k, jt}, P, R);
                    if (nlep >= 1) {
                        R.v[13] = lpt;
                        R.v[14] = leta;
                        R.v[15] = lphi;
                        R.v[16] = liso;
                        R.v[17] = __fadd_rn(R.v[0], lpt);
                    }
                    R.v[19] = cw_;
                    emit<DEBUG>(P, s_edges, sd.out, n, e, k, ((pm >> k) & 1ull) != 0, R);
                }
            }
        };
        if (hoff[NC] != 0u) {
            SCols sc;
#pragma unroll
            for (int c = 0; c < NC; ++c) sc.off[c] = hoff[c];
            body(sc);
        } else {
            DCols dc;
#pragma unroll
            for (int c = 0; c < NC; ++c)
                dc.p[c] = reinterpret_cast<const unsigned char*>(sd.col[c]) +
                          static_cast<uintptr_t>(hdr[L.col[c].coll]) * L.col[c].es;
            body(dc);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            cs_[c] = ns_[c];
            ct_[c] = nt_[c];
        }
        cw_ = nw_;
        bprev = b;
        b = b + 1 == S ? 0 : b + 1;
    }
    if (stop) {
        // a bounded wait gave up (error word set): let the copies already
        // issued land before the block exits, then leave the rest undone
        // (the failed tile's parity bit was already flipped)
        for (int j = 0; j < S - 1; ++j) {
            const int64_t tj = t0 + (it + j) * G;
            if (tj >= ntiles) break;
            const int sb = b + j < S ? b + j : b + j - S;
            const uint32_t par = ((parbits >> sb) & 1u) ^ (j == 0 ? 1u : 0u);
            if (tid == 0) mbar_wait_bounded(smem_addr(bars + sb), par);
        }
        return;
    }
    __syncthreads();
    if (*s_cnt != 0u) drain();
}

// Launch parameters prepared by the host entry points.
struct FusedArgs {
    FLayout layout;
    const ChainParams* P;
    const BatchDesc* B;
    hepacc_dtype offsets_type, btag_type;
    bool debug;
    bool flat;
    bool jec;           // correction tables (built for blocks of kDebugBlock threads only)
    int block;          // threads per block (a built block size)
    int grid;           // 0 = as many resident blocks as fit (one per SM)
    bool cap_grid;      // no more blocks than tiles (plans keep the full grid to stay reusable)
    int64_t ntiles;     // tiles of the launch
    cudaStream_t stream;
};

// Block sizes the kernel is built for (threads = events per tile); per-event
// outputs run in one of them.
constexpr int kBlocks[3] = {64, 128, 256};
constexpr int kDebugBlock = 128;

struct FCache {
    std::mutex mu;
    std::unordered_map<const void*, int> smem_set;
};
inline FCache& fcache() {
    static FCache c;
    return c;
}

template <typename K>
hepacc_status launch_fused(K kernel, const FusedArgs& a) {
    const DeviceInfo di = device_info();
    const size_t smem = a.layout.total;
    if (smem > static_cast<size_t>(di.smem_optin)) return fail(HEPACC_ERR_INVALID_ARG, "fused chain shared memory too large");
    {
        std::lock_guard<std::mutex> g(fcache().mu);
        auto it = fcache().smem_set.find(reinterpret_cast<const void*>(kernel));
        if (it == fcache().smem_set.end() || it->second < static_cast<int>(smem)) {
            const cudaError_t e =
                cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
            if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
            fcache().smem_set[reinterpret_cast<const void*>(kernel)] = static_cast<int>(smem);
        }
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, a.block, smem);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    if (per_sm < 1) return fail(HEPACC_ERR_INVALID_ARG, "fused chain kernel does not fit on an SM");
    int64_t grid = static_cast<int64_t>(per_sm) * di.sms;
    if (a.grid > 0) grid = a.grid;
    if (a.cap_grid) grid = std::max<int64_t>(1, std::min<int64_t>(grid, a.ntiles));
    kernel<<<static_cast<unsigned>(grid), a.block, smem, a.stream>>>(a.layout, *a.P, *a.B);
    HEPACC_CHECK_LAUNCH("fused chain launch");
    return HEPACC_OK;
}

template <typename KT, int NT>
hepacc_status run_fused_nt(const FusedArgs& a) {
    // the btag type of flat launches and of correction tables: F32 with F32
    // kinematics, F16 with half kinematics
    using HB = typename std::conditional<std::is_same<KT, float>::value, float, __half>::type;
    if (a.jec) {
        // correction tables: blocks of kDebugBlock threads only
        if constexpr (NT == kDebugBlock) {
            if (a.btag_type != (std::is_same<KT, float>::value ? HEPACC_F32 : HEPACC_F16))
                return fail(HEPACC_ERR_DTYPE, "with correction tables btag must be F32 with F32 kinematics, F16 with half");
            if (a.flat) {
                if (a.offsets_type != HEPACC_I64) return fail(HEPACC_ERR_DTYPE, "batched launches need I64 offsets");
                return launch_fused(k_fused<KT, HB, int64_t, false, true, NT, true>, a);
            }
            if (a.offsets_type == HEPACC_I32)
                return a.debug ? launch_fused(k_fused<KT, HB, int32_t, true, false, NT, true>, a)
                               : launch_fused(k_fused<KT, HB, int32_t, false, false, NT, true>, a);
            return a.debug ? launch_fused(k_fused<KT, HB, int64_t, true, false, NT, true>, a)
                           : launch_fused(k_fused<KT, HB, int64_t, false, false, NT, true>, a);
        } else {
            return fail(HEPACC_ERR_INVALID_ARG, "correction tables run in blocks of %d threads", kDebugBlock);
        }
    }
    if (a.flat) {
        // flat launches: int64 offsets, btag F32 with F32 kinematics, F16 with half
        if (a.offsets_type != HEPACC_I64) return fail(HEPACC_ERR_DTYPE, "batched launches need I64 offsets");
        return launch_fused(k_fused<KT, HB, int64_t, false, true, NT, false>, a);
    }
    auto go = [&](auto bt, auto ot) -> hepacc_status {
        using BT = typename decltype(bt)::type;
        using O = typename decltype(ot)::type;
        if constexpr (NT == kDebugBlock) {
            if (a.debug) return launch_fused(k_fused<KT, BT, O, true, false, NT, false>, a);
        } else {
            if (a.debug) return fail(HEPACC_ERR_INVALID_ARG, "per-event outputs run in blocks of %d threads", kDebugBlock);
        }
        return launch_fused(k_fused<KT, BT, O, false, false, NT, false>, a);
    };
    auto with_o = [&](auto bt) -> hepacc_status {
        if (a.offsets_type == HEPACC_I32) return go(bt, chain::Tag<int32_t>{});
        return go(bt, chain::Tag<int64_t>{});
    };
    if (a.btag_type == HEPACC_F32) return with_o(chain::Tag<float>{});
    return with_o(chain::Tag<__half>{});
}

template <typename KT>
hepacc_status run_fused_typed(const FusedArgs& a) {
    switch (a.block) {
        case 64: return run_fused_nt<KT, 64>(a);
        case 128: return run_fused_nt<KT, 128>(a);
        case 256: return run_fused_nt<KT, 256>(a);
    }
    return fail(HEPACC_ERR_INVALID_ARG, "fused chain: no kernel built for blocks of %d threads", a.block);
}

hepacc_status run_fused_f32(const FusedArgs& a);
hepacc_status run_fused_bf16(const FusedArgs& a);
hepacc_status run_fused_f16(const FusedArgs& a);

}  // namespace fused
}  // namespace hepacc
