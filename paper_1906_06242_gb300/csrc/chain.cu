// The fused benchmark chain of Section IV of arXiv:1906.06242 in one kernel:
// lepton selection -> jet selection with jet-lepton Delta R masking ->
// per-variation jet-pt scale, counts, HT, leading jets, pair and trijet
// masses -> 20 weighted histograms. Each input column is read once, staged
// per warp tile through the bulk-copy pipeline; histograms are accumulated
// in a block-private shared-memory copy (or straight into global memory
// when n_var copies do not fit) and added to the output at block exit.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "hepacc_host.h"
#include "hepacc_tiles.cuh"

namespace hepacc {

unsigned int tu_error_chain(bool clear) {
    unsigned int v = 0;
    cudaMemcpyFromSymbol(&v, g_device_error, sizeof v);
    if (clear && v) {
        unsigned int z = 0;
        cudaMemcpyToSymbol(g_device_error, &z, sizeof z);
    }
    return v;
}

namespace {

constexpr int NC = 15;   // jets: pt eta phi mass btag | mu: pt eta phi iso tight | el: pt eta phi iso tight
constexpr int kNV = HEPACC_CHAIN_NVARS;
constexpr int kQ = kNV + 1;   // queue entry: 20 variables + weight
constexpr int kTriLocal = 24;
using Spec = StageSpec<NC>;

enum : int { J_PT = 0, J_ETA, J_PHI, J_MASS, J_BTAG, M_PT, M_ETA, M_PHI, M_ISO, M_TIGHT, E_PT, E_ETA, E_PHI, E_ISO, E_TIGHT };

struct ChainParams {
    float lep_pt_min, lep_abseta_max, lep_iso_max;
    float jet_pt_min, jet_abseta_max, dr2_cut, btag_min;
    int n_var;
    int total_bins;
    int n_edges;
    float scales[HEPACC_MAX_VARIATIONS];
    int nbins[kNV];
    int eoff[kNV];      // first edge of histogram h
    int boff[kNV];      // first bin of histogram h inside a variation block
    float edges[HEPACC_CHAIN_MAX_EDGES];
};

struct ChainOut {
    unsigned long long* counts;
    double* sumw;
    double* sumw2;
    uint8_t* ev_pass;
    int32_t* ev_nlep;
    int32_t* ev_njet;
    int32_t* ev_nb;
    int32_t* ev_idx;
    float* ev_vars;
};

__device__ __forceinline__ float qnan() { return __int_as_float(0x7fc00000); }

struct ChainCols {
    const void *jet_pt, *jet_eta, *jet_phi, *jet_mass, *jet_btag;
    const void *mu_pt, *mu_eta, *mu_phi;
    const float *mu_iso;
    const uint8_t *mu_tight;
    const void *el_pt, *el_eta, *el_phi;
    const float *el_iso;
    const uint8_t *el_tight;
    const float *weight;
};

// One queued (event, variation) after the selection phase: words of a
// shared-memory slot of kQ words.
enum : int { R_E = 0, R_K, R_NJ, R_LEAD, R_SUB, R_HT, R_SUMM, R_MAXBT, R_OKLO, R_OKHI, R_LPT, R_LETA, R_LPHI, R_LISO };

template <typename T>
__device__ __forceinline__ float gload(const void* p, int64_t i) {
    return Elem<T>::f(static_cast<const T*>(p)[i]);
}

// Jet acceptance straight from global memory (|eta| and Delta R to every
// selected lepton of event e); used for jets past the 64 cached flags.
template <typename KT, typename OffT>
__device__ bool jet_ok_global(const ChainParams& P, const ChainCols& C, const OffT* moff, const OffT* eoff,
                              int64_t e, int64_t i) {
    const float eta = gload<KT>(C.jet_eta, i);
    if (!(fabsf(eta) < P.jet_abseta_max)) return false;
    const float phi = gload<KT>(C.jet_phi, i);
    for (int f = 0; f < 2; ++f) {
        const OffT* off = f == 0 ? moff : eoff;
        const void* pt = f == 0 ? C.mu_pt : C.el_pt;
        const void* le = f == 0 ? C.mu_eta : C.el_eta;
        const void* lp = f == 0 ? C.mu_phi : C.el_phi;
        const float* iso = f == 0 ? C.mu_iso : C.el_iso;
        const uint8_t* tight = f == 0 ? C.mu_tight : C.el_tight;
        for (int64_t l = ldoff(off, e); l < ldoff(off, e + 1); ++l) {
            const float p = gload<KT>(pt, l), x = gload<KT>(le, l);
            const bool sel = p > P.lep_pt_min && fabsf(x) < P.lep_abseta_max && tight[l] != 0 && iso[l] < P.lep_iso_max;
            if (sel && dr2_f32(eta, phi, x, gload<KT>(lp, l)) < P.dr2_cut) return false;
        }
    }
    return true;
}

// The second phase for one queued (event, variation): the 20 variables,
// including the pair and trijet masses, reading the event's jets from
// global memory (recently staged, so mostly L2 hits).
template <typename KT, typename BT, typename OffT>
__device__ void finish_event(const ChainParams& P, const ChainCols& C, const OffT* joff, const OffT* moff,
                             const OffT* eoff, const uint32_t* rec, float (&var)[kNV], int32_t (&tri)[3],
                             int& lead_o, int& sub_o) {
    const int64_t e = static_cast<int64_t>(rec[R_E]);
    const int k = rec[R_K] & 0xff;
    const int nlep = rec[R_K] >> 16;
    const int njet = rec[R_NJ] & 0xffff, nb = rec[R_NJ] >> 16;
    const int lead = static_cast<int32_t>(rec[R_LEAD]), sub = static_cast<int32_t>(rec[R_SUB]);
    const float s = P.scales[k];
    const float ht = __uint_as_float(rec[R_HT]);
    const uint64_t okbits = (static_cast<uint64_t>(rec[R_OKHI]) << 32) | rec[R_OKLO];
    const int64_t j0 = ldoff(joff, e), j1 = ldoff(joff, e + 1);
#pragma unroll
    for (int h = 0; h < kNV; ++h) var[h] = qnan();
    var[0] = ht;
    var[8] = static_cast<float>(njet);
    var[9] = static_cast<float>(nb);
    var[10] = __uint_as_float(rec[R_MAXBT]);
    var[18] = __uint_as_float(rec[R_SUMM]);
    var[19] = C.weight[e];
    if (nlep >= 1) {
        const float lpt = __uint_as_float(rec[R_LPT]);
        var[13] = lpt;
        var[14] = __uint_as_float(rec[R_LETA]);
        var[15] = __uint_as_float(rec[R_LPHI]);
        var[16] = __uint_as_float(rec[R_LISO]);
        var[17] = __fadd_rn(ht, lpt);
    }
    lead_o = lead;
    sub_o = sub;
    tri[0] = tri[1] = tri[2] = -1;
    MassObj ol;
    if (lead >= 0) {
        const int64_t i = j0 + lead;
        var[1] = __fmul_rn(gload<KT>(C.jet_pt, i), s);
        var[2] = gload<KT>(C.jet_eta, i);
        var[3] = gload<KT>(C.jet_phi, i);
        var[4] = gload<KT>(C.jet_mass, i);
        var[5] = gload<BT>(C.jet_btag, i);
        ol = mass_obj(var[1], var[2], var[3], var[4]);
    }
    if (sub >= 0) {
        const int64_t i = j0 + sub;
        var[6] = __fmul_rn(gload<KT>(C.jet_pt, i), s);
        const MassObj os = mass_obj(var[6], gload<KT>(C.jet_eta, i), gload<KT>(C.jet_phi, i), gload<KT>(C.jet_mass, i));
        var[7] = mass2obj(ol, os);
    }
    if (njet < 3) return;
    auto sel = [&](int64_t i, float& ptk) -> bool {
        const bool ok = (i - j0) < 64 ? ((okbits >> (i - j0)) & 1ull) != 0 : jet_ok_global<KT>(P, C, moff, eoff, e, i);
        if (!ok) return false;
        ptk = __fmul_rn(gload<KT>(C.jet_pt, i), s);
        return ptk > P.jet_pt_min;
    };
    float best = -1.0f;
    if (njet <= kTriLocal) {
        float px[kTriLocal], py[kTriLocal];
        int32_t li[kTriLocal];
        int cnt = 0;
        for (int64_t i = j0; i < j1 && cnt < kTriLocal; ++i) {
            float ptk;
            if (!sel(i, ptk)) continue;
            float sn, cs;
            sincosf(gload<KT>(C.jet_phi, i), &sn, &cs);
            px[cnt] = ptk * cs;
            py[cnt] = ptk * sn;
            li[cnt] = static_cast<int32_t>(i - j0);
            ++cnt;
        }
        for (int a = 0; a < cnt; ++a)
            for (int b = a + 1; b < cnt; ++b) {
                const float sx = px[a] + px[b], sy = py[a] + py[b];
                for (int c = b + 1; c < cnt; ++c) {
                    const float tx = sx + px[c], ty = sy + py[c];
                    const float val = tx * tx + ty * ty;
                    if (val > best) {
                        best = val;
                        tri[0] = li[a];
                        tri[1] = li[b];
                        tri[2] = li[c];
                    }
                }
            }
    } else {
        // more selected jets than the local buffers: enumerate directly
        for (int64_t a = j0; a < j1; ++a) {
            float pa;
            if (!sel(a, pa)) continue;
            float sa, ca;
            sincosf(gload<KT>(C.jet_phi, a), &sa, &ca);
            for (int64_t b = a + 1; b < j1; ++b) {
                float pb;
                if (!sel(b, pb)) continue;
                float sb, cb;
                sincosf(gload<KT>(C.jet_phi, b), &sb, &cb);
                const float sx = pa * ca + pb * cb, sy = pa * sa + pb * sb;
                for (int64_t c = b + 1; c < j1; ++c) {
                    float pc;
                    if (!sel(c, pc)) continue;
                    float sc, cc;
                    sincosf(gload<KT>(C.jet_phi, c), &sc, &cc);
                    const float tx = sx + pc * cc, ty = sy + pc * sc;
                    const float val = tx * tx + ty * ty;
                    if (val > best) {
                        best = val;
                        tri[0] = static_cast<int32_t>(a - j0);
                        tri[1] = static_cast<int32_t>(b - j0);
                        tri[2] = static_cast<int32_t>(c - j0);
                    }
                }
            }
        }
    }
    MassObj o3[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int64_t i = j0 + tri[q];
        o3[q] = mass_obj(__fmul_rn(gload<KT>(C.jet_pt, i), s), gload<KT>(C.jet_eta, i), gload<KT>(C.jet_phi, i),
                         gload<KT>(C.jet_mass, i));
    }
    var[11] = mass3obj(o3[0], o3[1], o3[2]);
    var[12] = sqrtf(best);
}

template <typename KT, typename BT, typename OffT, bool DEBUG, bool SMEM_HIST>
__global__ void __launch_bounds__(512, 1) k_chain(Spec spec, const __grid_constant__ ChainParams P, ChainCols C,
                                                  const OffT* joff, const OffT* moff, const OffT* eoff, int64_t n,
                                                  ChainOut out) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int nwarp = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    // shared memory after the pipeline's stage buffers: edges, per-warp
    // queues, block-private histograms
    unsigned char* tail = smem + static_cast<size_t>(nwarp) * stage_bytes_per_warp(spec);
    float* s_edges = reinterpret_cast<float*>(tail);
    uint32_t* s_queue = reinterpret_cast<uint32_t*>(s_edges + ((P.n_edges + 3) & ~3));   // [nwarp][32][kQ]
    unsigned char* hist_base = reinterpret_cast<unsigned char*>(s_queue + nwarp * 32 * kQ);
    hist_base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(hist_base) + 15) & ~uintptr_t(15));
    const int hist_n = P.n_var * P.total_bins;
    double* s_w = reinterpret_cast<double*>(hist_base);
    double* s_w2 = s_w + (SMEM_HIST ? hist_n : 0);
    unsigned int* s_c = reinterpret_cast<unsigned int*>(s_w2 + (SMEM_HIST ? hist_n : 0));

    for (int i = threadIdx.x; i < P.n_edges; i += blockDim.x) s_edges[i] = P.edges[i];
    if (SMEM_HIST) {
        for (int i = threadIdx.x; i < hist_n; i += blockDim.x) {
            s_w[i] = 0.0;
            s_w2[i] = 0.0;
            s_c[i] = 0u;
        }
    }
    __syncthreads();
    uint32_t* my_q = s_queue + warp * 32 * kQ;
    int qcount = 0;

    // Phase 2 for the queued records [0, m): every lane finishes one record,
    // passing ones are staged (20 variables + weight) in the same slots and
    // lane h < 20 then fills histogram h for each of them.
    auto flush = [&](int m) {
        uint32_t rec[kQ];
        const bool have = lane < m;
        if (have) {
#pragma unroll
            for (int w = 0; w <= R_LISO; ++w) rec[w] = my_q[lane * kQ + w];
        }
        __syncwarp();
        float var[kNV];
        int32_t tri[3];
        int lead = -1, sub = -1;
        bool pass = false;
        int k = 0;
        if (have) {
            finish_event<KT, BT, OffT>(P, C, joff, moff, eoff, rec, var, tri, lead, sub);
            pass = ((rec[R_K] >> 8) & 1u) != 0;
            k = rec[R_K] & 0xff;
            if (DEBUG) {
                const int64_t e = rec[R_E];
                const int64_t kn = static_cast<int64_t>(k) * n;
                if (out.ev_pass) out.ev_pass[kn + e] = pass ? 1 : 0;
                if (out.ev_njet) out.ev_njet[kn + e] = rec[R_NJ] & 0xffff;
                if (out.ev_nb) out.ev_nb[kn + e] = rec[R_NJ] >> 16;
                if (out.ev_idx) {
                    int32_t* ix = out.ev_idx + static_cast<int64_t>(k) * 5 * n;
                    ix[e] = lead;
                    ix[n + e] = sub;
                    ix[2 * n + e] = tri[0];
                    ix[3 * n + e] = tri[1];
                    ix[4 * n + e] = tri[2];
                }
                if (out.ev_vars) {
                    float* vv = out.ev_vars + static_cast<int64_t>(k) * kNV * n;
#pragma unroll
                    for (int h = 0; h < kNV; ++h) vv[h * n + e] = var[h];
                }
            }
        }
        const unsigned pmask = __ballot_sync(0xffffffffu, pass);
        if (pass) {
            uint32_t* q = my_q + __popc(pmask & lt_mask) * kQ;
#pragma unroll
            for (int h = 0; h < kNV; ++h) q[h] = __float_as_uint(var[h]);
            q[kNV] = static_cast<uint32_t>(k);
        }
        __syncwarp();
        const int np = __popc(pmask);
        if (lane < kNV && np > 0) {
            const int h = lane;
            const float* eh = s_edges + P.eoff[h];
            const int nb_h = P.nbins[h];
            const float span = eh[nb_h] - eh[0];
            const float invw = span > 0.0f ? static_cast<float>(nb_h) / span : 0.0f;
            for (int j = 0; j < np; ++j) {
                const uint32_t* q = my_q + j * kQ;
                const int b = find_bin(__uint_as_float(q[h]), eh, nb_h, invw);
                if (b < 0) continue;
                const double wd = static_cast<double>(__uint_as_float(q[19]));
                const int at = static_cast<int>(q[kNV]) * P.total_bins + P.boff[h] + b;
                if (SMEM_HIST) {
                    atomicAdd(&s_c[at], 1u);
                    atomicAdd(&s_w[at], wd);
                    if (out.sumw2) atomicAdd(&s_w2[at], wd * wd);
                } else {
                    atomicAdd(&out.counts[at], 1ull);
                    atomicAdd(&out.sumw[at], wd);
                    if (out.sumw2) atomicAdd(&out.sumw2[at], wd * wd);
                }
            }
        }
        __syncwarp();
    };

    const OffT* const offs[3] = {joff, moff, eoff};
    tile_loop<OffT, 3, NC>(spec, offs, n, [&](const TileView<3, NC>& v) {
        const bool valid = v.valid;
        // phase 1a: leptons
        int nlep = 0;
        float lpt = qnan(), leta = qnan(), lphi = qnan(), liso = qnan();
        if (valid) {
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                const int c0 = f == 0 ? M_PT : E_PT;
                const int coll = 1 + f;
                for (int64_t i = v.s[coll]; i < v.t[coll]; ++i) {
                    const float p = Elem<KT>::f(v.template at<KT>(c0, coll, i));
                    const float x = Elem<KT>::f(v.template at<KT>(c0 + 1, coll, i));
                    const float iso = v.template at<float>(c0 + 3, coll, i);
                    const bool sel = p > P.lep_pt_min && fabsf(x) < P.lep_abseta_max &&
                                     v.template at<uint8_t>(c0 + 4, coll, i) != 0 && iso < P.lep_iso_max;
                    if (!sel) continue;
                    if (nlep == 0) {
                        lpt = p;
                        leta = x;
                        lphi = Elem<KT>::f(v.template at<KT>(c0 + 2, coll, i));
                        liso = iso;
                    }
                    ++nlep;
                }
            }
        }
        if (DEBUG && valid && out.ev_nlep) out.ev_nlep[v.e] = nlep;
        // without per-event outputs only single-lepton events can pass
        const bool active = valid && (DEBUG || nlep == 1);

        // phase 1b: variation-independent jet acceptance (|eta|, Delta R)
        auto jet_ok = [&](int64_t i) -> bool {
            const float eta = Elem<KT>::f(v.template at<KT>(J_ETA, 0, i));
            if (!(fabsf(eta) < P.jet_abseta_max)) return false;
            const float phi = Elem<KT>::f(v.template at<KT>(J_PHI, 0, i));
            if (nlep == 1) return !(dr2_f32(eta, phi, leta, lphi) < P.dr2_cut);
            if (nlep == 0) return true;
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                const int c0 = f == 0 ? M_PT : E_PT;
                const int coll = 1 + f;
                for (int64_t l = v.s[coll]; l < v.t[coll]; ++l) {
                    const float p = Elem<KT>::f(v.template at<KT>(c0, coll, l));
                    const float x = Elem<KT>::f(v.template at<KT>(c0 + 1, coll, l));
                    const bool sel = p > P.lep_pt_min && fabsf(x) < P.lep_abseta_max &&
                                     v.template at<uint8_t>(c0 + 4, coll, l) != 0 &&
                                     v.template at<float>(c0 + 3, coll, l) < P.lep_iso_max;
                    if (sel && dr2_f32(eta, phi, x, Elem<KT>::f(v.template at<KT>(c0 + 2, coll, l))) < P.dr2_cut)
                        return false;
                }
            }
            return true;
        };
        uint64_t okbits = 0;
        const int64_t j0 = v.s[0], j1 = v.t[0];
        if (active) {
            const int64_t jlim = j1 < j0 + 64 ? j1 : j0 + 64;
            for (int64_t i = j0; i < jlim; ++i)
                if (jet_ok(i)) okbits |= 1ull << (i - j0);
        }

        // phase 1c: per variation, counts and sums over the selected jets
        for (int k = 0; k < P.n_var; ++k) {
            const float s = P.scales[k];
            int njet = 0, nb = 0;
            float ht = 0.0f, summ = 0.0f, maxbt = qnan();
            int64_t lead = -1, sub = -1;
            float lead_pt = 0.0f, sub_pt = 0.0f;
            if (active) {
                for (int64_t i = j0; i < j1; ++i) {
                    const bool ok = (i - j0) < 64 ? ((okbits >> (i - j0)) & 1ull) != 0 : jet_ok(i);
                    if (!ok) continue;
                    const float ptk = __fmul_rn(Elem<KT>::f(v.template at<KT>(J_PT, 0, i)), s);
                    if (!(ptk > P.jet_pt_min)) continue;
                    ++njet;
                    const float bt = Elem<BT>::f(v.template at<BT>(J_BTAG, 0, i));
                    nb += bt > P.btag_min ? 1 : 0;
                    ht = __fadd_rn(ht, ptk);
                    summ = __fadd_rn(summ, Elem<KT>::f(v.template at<KT>(J_MASS, 0, i)));
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
                }
            }
            const bool pass = active && nlep == 1 && njet >= 2 && nb >= 1;
            const bool enq = DEBUG ? valid : pass;
            const unsigned emask = __ballot_sync(0xffffffffu, enq);
            const int m = __popc(emask);
            if (m == 0) continue;
            if (qcount + m > 32) {
                flush(qcount);
                qcount = 0;
            }
            if (enq) {
                uint32_t* r = my_q + (qcount + __popc(emask & lt_mask)) * kQ;
                r[R_E] = static_cast<uint32_t>(v.e);
                r[R_K] = static_cast<uint32_t>(k) | (pass ? 0x100u : 0u) | (static_cast<uint32_t>(min(nlep, 0xffff)) << 16);
                r[R_NJ] = static_cast<uint32_t>(min(njet, 0xffff)) | (static_cast<uint32_t>(min(nb, 0xffff)) << 16);
                r[R_LEAD] = static_cast<uint32_t>(lead < 0 ? -1 : static_cast<int32_t>(lead - j0));
                r[R_SUB] = static_cast<uint32_t>(sub < 0 ? -1 : static_cast<int32_t>(sub - j0));
                r[R_HT] = __float_as_uint(ht);
                r[R_SUMM] = __float_as_uint(summ);
                r[R_MAXBT] = __float_as_uint(maxbt);
                r[R_OKLO] = static_cast<uint32_t>(okbits);
                r[R_OKHI] = static_cast<uint32_t>(okbits >> 32);
                r[R_LPT] = __float_as_uint(lpt);
                r[R_LETA] = __float_as_uint(leta);
                r[R_LPHI] = __float_as_uint(lphi);
                r[R_LISO] = __float_as_uint(liso);
            }
            __syncwarp();
            qcount += m;
        }
    });
    if (qcount > 0) flush(qcount);

    if (SMEM_HIST) {
        __syncthreads();
        for (int i = threadIdx.x; i < hist_n; i += blockDim.x) {
            const unsigned c = s_c[i];
            if (c == 0u) continue;
            atomicAdd(&out.counts[i], static_cast<unsigned long long>(c));
            atomicAdd(&out.sumw[i], s_w[i]);
            if (out.sumw2) atomicAdd(&out.sumw2[i], s_w2[i]);
        }
    }
}

template <typename T> struct Tag { using type = T; };

struct Cache {
    std::mutex mu;
    std::unordered_map<const void*, int> smem_set;
};
Cache& cache() {
    static Cache c;
    return c;
}

template <typename K, typename... A>
hepacc_status launch_chain(K kernel, int block, size_t smem, int64_t n, cudaStream_t stream, int grid_override,
                           A... args) {
    const DeviceInfo di = device_info();
    if (smem > static_cast<size_t>(di.smem_optin)) return fail(HEPACC_ERR_INVALID_ARG, "chain shared memory too large");
    {
        std::lock_guard<std::mutex> g(cache().mu);
        auto it = cache().smem_set.find(reinterpret_cast<const void*>(kernel));
        if (it == cache().smem_set.end() || it->second < static_cast<int>(smem)) {
            cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
            if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
            cache().smem_set[reinterpret_cast<const void*>(kernel)] = static_cast<int>(smem);
        }
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    if (per_sm < 1) return fail(HEPACC_ERR_INVALID_ARG, "chain kernel does not fit on an SM");
    const int64_t ntiles = (n + kTile - 1) / kTile;
    const int64_t want = (ntiles + (block / 32) - 1) / (block / 32);
    int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(want, static_cast<int64_t>(per_sm) * di.sms)));
    if (grid_override > 0) grid = grid_override;
    kernel<<<grid, block, smem, stream>>>(args...);
    HEPACC_CHECK_LAUNCH("chain launch");
    return HEPACC_OK;
}

}  // namespace

// Tunables of the chain launch (set by the autotuner; 0 = default).
struct ChainTuning {
    int jet_cap;     // stage capacity for jets, elements per warp tile
    int lep_cap;     // stage capacity per lepton collection
    int grid;        // blocks (0 = resident blocks x SMs)
    int warps;       // upper bound of warps per block (0 = 16)
};
static ChainTuning g_tuning = {0, 0, 0, 0};

}  // namespace hepacc

using namespace hepacc;

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

    const size_t kes = dtype_size(b->kin_type), bes = dtype_size(b->btag_type);
    const int jcap = g_tuning.jet_cap > 0 ? g_tuning.jet_cap : 192;
    const int lcap = g_tuning.lep_cap > 0 ? g_tuning.lep_cap : 64;
    Spec spec{};
    uint32_t off = 0;
    auto add = [&](int c, const void* base, size_t es, int coll, int cap) {
        ColSpec& cs = spec.col[c];
        cs.base = static_cast<const unsigned char*>(base);
        cs.es = static_cast<uint32_t>(es);
        cs.coll = static_cast<uint32_t>(coll);
        cs.cap = static_cast<uint32_t>((cap * es + 32 + 15) & ~size_t(15));
        cs.soff = off;
        off += cs.cap;
    };
    add(J_PT, b->jet_pt, kes, 0, jcap);
    add(J_ETA, b->jet_eta, kes, 0, jcap);
    add(J_PHI, b->jet_phi, kes, 0, jcap);
    add(J_MASS, b->jet_mass, kes, 0, jcap);
    add(J_BTAG, b->jet_btag, bes, 0, jcap);
    add(M_PT, b->mu_pt, kes, 1, lcap);
    add(M_ETA, b->mu_eta, kes, 1, lcap);
    add(M_PHI, b->mu_phi, kes, 1, lcap);
    add(M_ISO, b->mu_iso, 4, 1, lcap);
    add(M_TIGHT, b->mu_tight, 1, 1, lcap);
    add(E_PT, b->el_pt, kes, 2, lcap);
    add(E_ETA, b->el_eta, kes, 2, lcap);
    add(E_PHI, b->el_phi, kes, 2, lcap);
    add(E_ISO, b->el_iso, 4, 2, lcap);
    add(E_TIGHT, b->el_tight, 1, 2, lcap);
    spec.ncol = NC;
    spec.buf_bytes = (off + 127) & ~uint32_t(127);

    if (n >= (int64_t(1) << 31)) return fail(HEPACC_ERR_INVALID_ARG, "at most 2^31 - 1 events per call");
    ChainCols C;
    C.jet_pt = b->jet_pt; C.jet_eta = b->jet_eta; C.jet_phi = b->jet_phi; C.jet_mass = b->jet_mass;
    C.jet_btag = b->jet_btag;
    C.mu_pt = b->mu_pt; C.mu_eta = b->mu_eta; C.mu_phi = b->mu_phi; C.mu_iso = b->mu_iso; C.mu_tight = b->mu_tight;
    C.el_pt = b->el_pt; C.el_eta = b->el_eta; C.el_phi = b->el_phi; C.el_iso = b->el_iso; C.el_tight = b->el_tight;
    C.weight = b->weight;

    // warps per block from the shared-memory budget: per warp two stage
    // buffers and a 32-slot queue; per block the edges and (if they fit) the
    // block-private histograms of every variation
    const DeviceInfo di = device_info();
    const size_t per_warp = stage_bytes_per_warp(spec) + 32 * kQ * 4;
    const size_t edges_b = static_cast<size_t>((P.n_edges + 3) & ~3) * 4 + 16;
    const size_t hist = static_cast<size_t>(P.n_var) * P.total_bins * (8 + 8 + 4);
    const int max_warps = g_tuning.warps > 0 ? g_tuning.warps : 16;
    auto warps_for = [&](size_t fixed) -> int {
        if (fixed >= static_cast<size_t>(di.smem_optin)) return 0;
        return static_cast<int>(std::min<size_t>(max_warps, (di.smem_optin - fixed) / per_warp));
    };
    bool smem_hist = warps_for(edges_b + hist) >= 4;
    const int nwarp = smem_hist ? warps_for(edges_b + hist) : warps_for(edges_b);
    if (nwarp < 1) return fail(HEPACC_ERR_INVALID_ARG, "chain stage buffers do not fit in shared memory");
    const size_t smem = per_warp * nwarp + edges_b + (smem_hist ? hist : 0);
    const int block = 32 * nwarp;

    auto go = [&](auto kt, auto bt, auto ot) -> hepacc_status {
        using KT = typename decltype(kt)::type;
        using BT = typename decltype(bt)::type;
        using O = typename decltype(ot)::type;
        const O* jo = static_cast<const O*>(b->jet_offsets);
        const O* mo = static_cast<const O*>(b->mu_offsets);
        const O* eo = static_cast<const O*>(b->el_offsets);
        const int g = g_tuning.grid;
        if (debug) {
            if (smem_hist)
                return launch_chain(k_chain<KT, BT, O, true, true>, block, smem, n, s, g, spec, P, C, jo, mo, eo, n, o);
            return launch_chain(k_chain<KT, BT, O, true, false>, block, smem, n, s, g, spec, P, C, jo, mo, eo, n, o);
        }
        if (smem_hist)
            return launch_chain(k_chain<KT, BT, O, false, true>, block, smem, n, s, g, spec, P, C, jo, mo, eo, n, o);
        return launch_chain(k_chain<KT, BT, O, false, false>, block, smem, n, s, g, spec, P, C, jo, mo, eo, n, o);
    };
    auto with_o = [&](auto kt, auto bt) -> hepacc_status {
        if (b->offsets_type == HEPACC_I32) return go(kt, bt, Tag<int32_t>{});
        return go(kt, bt, Tag<int64_t>{});
    };
    auto with_b = [&](auto kt) -> hepacc_status {
        if (b->btag_type == HEPACC_F32) return with_o(kt, Tag<float>{});
        return with_o(kt, Tag<__half>{});
    };
    switch (b->kin_type) {
        case HEPACC_F32: return with_b(Tag<float>{});
        case HEPACC_F16: return with_b(Tag<__half>{});
        default: return with_b(Tag<__nv_bfloat16>{});
    }
}
