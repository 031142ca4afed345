// The fused benchmark chain of Section IV of arXiv:1906.06242: kernel
// templates shared by the per-type translation units (chain_<type>.cu for
// single-sample launches, chain_batched_<type>.cu for many samples per
// launch) and the host side (chain.cu).
//
// One kernel, persistent blocks; a block works on tiles of E = blockDim.x
// consecutive events (thread = event):
//  * staging: warp 0 copies every needed column's span of the tile (one
//    lane per column) into one of two shared-memory stage buffers with bulk
//    asynchronous copies
//    (cp.async.bulk, the TMA engine; whole 16-byte chunks), completion on a
//    "full" mbarrier; warps release a stage on an "empty" mbarrier, so they
//    run independently (up to one tile apart) without block barriers; the
//    tile spans are read two tiles ahead;
//  * selection (thread = event, staged data): lepton selection, jet
//    acceptance (|eta|, Delta R to the selected leptons, lanes over jets),
//    and per event the two pt thresholds that decide every jet-pt variation
//    (second-largest accepted jet pt, largest accepted b-tagged jet pt);
//  * pairs (thread = passing (event, variation), 32 at a time per warp):
//    the pair's lane gathers the jet counts, HT, the mass sum, the leading
//    jets and the max-|sum pT| triplet from shared memory and writes a
//    self-contained record (with the jets' four-momenta) to a per-warp queue;
//  * masses (thread = queued pair, 32 at a time per warp): pair and triplet
//    invariant masses and the 20 variables, pure arithmetic;
//  * fill: lane h bins variable h of every queued entry (no two lanes of a
//    warp touch one bin) into the histograms of the placement: block-private
//    shared memory, shared memory spread over a thread-block cluster
//    (distributed shared memory reductions into the block that owns the
//    bin) or global memory; shared-memory histograms go to the outputs when
//    the block is done with a sample.
// Batched launches walk through up to kMaxSamples samples in turn, each with
// its own columns and outputs, without a grid-wide barrier between them.
#pragma once

#include <algorithm>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "hepacc_host.h"
#include "hepacc_tiles.cuh"

namespace hepacc {
namespace chain {

constexpr int NC = 15;            // staged columns
constexpr int kNV = HEPACC_CHAIN_NVARS;
constexpr int kScratch = 10;      // selected jets ranked from a queue slot (2 x 10 words of it)
// Block shape of each launch form: threads per block (the largest tile) and
// blocks per SM, measured best on GB300. Register allocation rounds blocks
// up (160 threads count like 192, 320 like 384), so two blocks of 160 cap a
// thread at 168 registers (some spilling) and one block of 256 at 255.
// Single-sample launches run two independent 160-thread blocks per SM (a
// stalled stage refill in one leaves the other running); batched launches,
// with their loop over samples, run spill-free in one 256-thread block.
constexpr int kMaxThreads = 160;
constexpr int kMinBlocks = 2;
constexpr int kMaxThreadsBatched = 256;
constexpr int kMinBlocksBatched = 1;
constexpr int kHdr = 96;          // stage header: spans, staged flag, column offsets
constexpr int kEvWords = 12;      // event summary handed to the pairs

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
    float invw[kNV];    // bins per unit of histogram h (first guess of the bin search)
    float e_lo[kNV], e_hi[kNV];   // first and last edge of histogram h
    // jet-energy correction tables (jec_contents null: the scales)
    int jec_neta, jec_npt;
    const float* jec_contents;    // DEVICE [n_var][jec_neta + 2][jec_npt + 2]
    float jec_eta_invw;
    float jec_edges[2 * (HEPACC_JEC_MAX_BINS + 1)];   // eta edges, then pt edges
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

// One sample of a launch: column bases (staged-column order), offsets,
// weights and its outputs.
constexpr int kMaxSamples = 16;
struct SampleDesc {
    const void* col[NC];
    const float* weight;
    const void* off[3];
    int64_t n;
    ChainOut out;
};
struct BatchDesc {
    int n_samples;
    SampleDesc s[kMaxSamples];
    int64_t tile_start[kMaxSamples + 1];   // F_FLAT: first flat tile of each sample (and the total)
};

// Launch forms: one sample; several samples walked in turn by every block
// (histograms in block or cluster shared memory, flushed per sample); or
// several samples as one flat sequence of tiles (global histograms: every
// tile finds its sample, every record carries it).
enum : int { F_SINGLE = 0, F_SAMPLES = 1, F_FLAT = 2 };

// Histogram placement: block-private shared memory, global memory, or
// spread over the shared memory of a thread-block cluster (each block owns
// a contiguous slice of the bins, updated through distributed shared memory).
enum : int { H_SMEM = 0, H_GLOBAL = 1, H_CLUSTER = 2 };

__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t map_to_rank(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ void red_cluster_u32(uint32_t addr, uint32_t v) {
    asm volatile("red.shared::cluster.add.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void red_cluster_f64(uint32_t addr, double v) {
    asm volatile("red.shared::cluster.add.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Shared-memory layout of a block (byte offsets into dynamic shared memory).
struct Layout {
    ColSpec col[NC];       // soff relative to the stage's column area
    uint32_t stage_bytes;  // one stage: kHdr header + column regions
    uint32_t bars;         // four mbarriers: full[2], empty[2]
    uint32_t edges;        // n_edges floats
    uint32_t queue;        // per warp 32 slots of R_WORDS words
    uint32_t acc;          // per warp acc_words words of jet acceptance flags
    uint32_t pairs;        // per warp 64 queued (event lane, variation) pairs, uint16
    uint32_t evs;          // per warp kEvWords x 32 words: the events' summaries
    uint32_t sample;       // batched launches: the current sample's descriptor
    int acc_words;
    uint32_t tri;          // triplet table (uint16 per triplet, colex order)
    uint32_t hist;         // histograms (H_SMEM: all bins, H_CLUSTER: this block's slice)
    int hist_slice;        // H_CLUSTER: bins per block
    uint32_t total;
};

// A queued (event, variation): words of a per-warp queue slot. Jets are
// (pt_k, eta, phi, mass); the leading one also carries btag. The slot
// stride is odd so that lanes reading one word of their slots hit distinct
// shared-memory banks.
enum : int {
    R_E = 0, R_K, R_NJ, R_IDX, R_TAB, R_TC, R_HT, R_SUMM, R_MAXBT, R_BEST, R_W,
    R_LPT, R_LETA, R_LPHI, R_LISO,
    R_J1 = 15, R_J2 = 20, R_T1 = 24, R_T2 = 28, R_T3 = 32, R_WORDS = 37
};

__device__ __forceinline__ float qnan() { return __int_as_float(0x7fc00000); }


// Column access for the selection phase.
struct StagedCols {
    uint32_t off[NC];      // byte offset of the tile's first element of each column in shared memory
    template <typename T>
    __device__ __forceinline__ T ld(int c, int r) const {
        return *reinterpret_cast<const T*>(g_dyn_smem + off[c] + r * static_cast<int>(sizeof(T)));
    }
};
struct DirectCols {
    const Layout* L;       // column element sizes and collections
    const void* const* base;   // column bases of the sample
    int64_t S[3];          // the tile's first element per collection
    template <typename T>
    __device__ __forceinline__ T ld(int c, int r) const {
        return reinterpret_cast<const T*>(base[c])[S[L->col[c].coll] + r];
    }
};

__device__ __forceinline__ void put4(uint32_t* q, float a, float b, float c, float d) {
    q[0] = __float_as_uint(a);
    q[1] = __float_as_uint(b);
    q[2] = __float_as_uint(c);
    q[3] = __float_as_uint(d);
}

template <typename KT, typename BT, typename OffT, bool DEBUG, int HMODE, int FORM>
__global__ void __launch_bounds__(FORM == F_SAMPLES ? kMaxThreadsBatched : kMaxThreads,
                                  FORM == F_SAMPLES ? kMinBlocksBatched : kMinBlocks) k_chain(const __grid_constant__ Layout L,
                                                          const __grid_constant__ ChainParams P,
                                                          const __grid_constant__ BatchDesc B) {
    constexpr bool MULTI = FORM == F_SAMPLES;
    constexpr bool FLAT = FORM == F_FLAT;
    static_assert(!FLAT || HMODE == H_GLOBAL, "flat batched launches fill global histograms");
    unsigned char* smem = g_dyn_smem;
    const int tid = threadIdx.x;
    const int E = blockDim.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int nwarp = E >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    float* s_edges = reinterpret_cast<float*>(smem + L.edges);
    uint32_t* my_q = reinterpret_cast<uint32_t*>(smem + L.queue) + warp * 32 * R_WORDS;
    const int hist_n = P.n_var * P.total_bins;
    const int hist_local = HMODE == H_SMEM ? hist_n : (HMODE == H_CLUSTER ? L.hist_slice : 0);
    double* s_w = reinterpret_cast<double*>(smem + L.hist);
    double* s_w2 = s_w + hist_local;
    unsigned int* s_c = reinterpret_cast<unsigned int*>(s_w2 + hist_local);
    const uint32_t my_rank = HMODE == H_CLUSTER ? cluster_ctarank() : 0u;
    uint16_t* s_tri = reinterpret_cast<uint16_t*>(smem + L.tri);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bars);
    const uint32_t full[2] = {smem_addr(bars), smem_addr(bars + 1)};
    const uint32_t empty[2] = {smem_addr(bars + 2), smem_addr(bars + 3)};
    const uint32_t smem0 = smem_addr(smem);

    for (int i = tid; i < P.n_edges; i += E) s_edges[i] = P.edges[i];
    // all triplets a<b<c<kScratch in colex order (c, then b, then a): the
    // first C(n,3) are those among n jets
    if (tid == 0) {
        int t = 0;
        for (int c = 2; c < kScratch; ++c)
            for (int b2 = 1; b2 < c; ++b2)
                for (int a = 0; a < b2; ++a) s_tri[t++] = static_cast<uint16_t>(a | (b2 << 4) | (c << 8));
    }
    for (int i = tid; i < hist_local; i += E) {
        s_w[i] = 0.0;
        s_w2[i] = 0.0;
        s_c[i] = 0u;
    }
    if (tid == 0) {
        mbar_init(full[0], 1);
        mbar_init(full[1], 1);
        mbar_init(empty[0], nwarp);
        mbar_init(empty[1], nwarp);
        fence_mbar_init();
    }
    __syncthreads();
    if (HMODE == H_CLUSTER) cluster_sync_all();

    // The sample being processed: single-sample launches read its
    // descriptor from the kernel parameters; batched ones copy the current
    // sample's descriptor to shared memory at the top of the sample loop
    // (its fields are then read where they are used instead of occupying
    // registers for the whole sample).
    // Flat launches read the descriptor of each tile's own sample.
    SampleDesc* cur = reinterpret_cast<SampleDesc*>(smem + L.sample);
    auto SDs = [&](int s) -> const SampleDesc& {
        if constexpr (MULTI)
            return *cur;
        else if constexpr (FLAT)
            return B.s[s];
        else
            return B.s[0];
    };
    int64_t n = 0;
    int64_t ntiles = 0;
    const int64_t grid = gridDim.x;
    // sample and tile within the sample of launch tile t (flat launches:
    // the last sample whose first tile is at or before t)
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

    // Warp 0 stages the tiles. load_span: the first and last element of
    // every collection in tile tt, span[0..2] and span[3..5] (shared
    // memory), one lane each.
    auto load_span = [&](int64_t tt, int64_t* span) {
        __syncwarp();   // earlier readers of span are done
        if (lane < 6) {
            int ts;
            int64_t lt;
            where(tt, ts, lt);
            const int64_t ns = SDs(ts).n;
            const int64_t a = lt * E;
            const int64_t z = a + E < ns ? a + E : ns;
            span[lane] = ldoff(static_cast<const OffT*>(SDs(ts).off[lane % 3]), lane < 3 ? a : z);
        }
        __syncwarp();
    };
    // issue: header of stage b and the bulk copies of the spans of tile tt
    // (sample ts), column c by lane c; the copies are issued after lane 0
    // registered their total on the stage's "full" mbarrier
    auto issue = [&](int b, int ts, const int64_t* span) {
        const SampleDesc& sd = SDs(ts);
        unsigned char* st = smem + b * L.stage_bytes;
        int64_t* hdr = reinterpret_cast<int64_t*>(st);
        uint32_t* hoff = reinterpret_cast<uint32_t*>(st + 32);
        uint32_t bytes = 0;
        uintptr_t a16 = 0;
        bool fits_c = true;
        if (lane < NC) {
            const ColSpec& cs = L.col[lane];
            const int64_t S = span[cs.coll], T = span[3 + cs.coll];
            const uintptr_t cb = reinterpret_cast<uintptr_t>(sd.col[lane]);
            const uintptr_t a = cb + static_cast<uintptr_t>(S) * cs.es;
            const uintptr_t z = cb + static_cast<uintptr_t>(T) * cs.es;
            a16 = a & ~uintptr_t(15);
            bytes = T > S ? static_cast<uint32_t>(((z + 15) & ~uintptr_t(15)) - a16) : 0u;
            fits_c = bytes <= cs.cap;
            hoff[lane] = b * L.stage_bytes + kHdr + cs.soff + static_cast<uint32_t>(a & 15u);
        }
        const bool fits = __all_sync(0xffffffffu, fits_c);
        uint32_t total = bytes;
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) total += __shfl_xor_sync(0xffffffffu, total, d);
        if (lane < 3) hdr[lane] = span[lane];
        if (lane == 0) hoff[NC] = fits ? 1u : 0u;
        __syncwarp();
        if (lane == 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(full[b], fits ? total : 0u);
        }
        __syncwarp();
        if (fits && lane < NC && bytes > 0) {
            fence_proxy_async_smem();
            bulk_g2s(smem0 + b * L.stage_bytes + kHdr + L.col[lane].soff, reinterpret_cast<const void*>(a16), bytes,
                     full[b]);
        }
    };

    // Masses and fill for this warp's queued records [0, m) (warp-uniform).
    auto flush = [&](int m) {
        const uint32_t* r = my_q + lane * R_WORDS;   // this lane's record
        const bool have = lane < m;
        const ChainOut& out = SDs(have ? static_cast<int>((r[R_K] >> 9) & 0x7fu) : 0).out;
        float var[kNV];
        int k = 0;
        bool pass = false;
        if (have) {
            k = r[R_K] & 0xff;
            pass = ((r[R_K] >> 8) & 1u) != 0;
            const int nlep = r[R_K] >> 16;
            const int njet = r[R_NJ] & 0xffff;
            const int lead = static_cast<int16_t>(r[R_IDX] & 0xffff), sub = static_cast<int16_t>(r[R_IDX] >> 16);
            const int ta = static_cast<int16_t>(r[R_TAB] & 0xffff), tb = static_cast<int16_t>(r[R_TAB] >> 16);
            const int tc = static_cast<int32_t>(r[R_TC]);
            auto f = [&](int w) { return __uint_as_float(r[w]); };
#pragma unroll
            for (int h = 0; h < kNV; ++h) var[h] = qnan();
            var[0] = f(R_HT);
            var[8] = static_cast<float>(njet);
            var[9] = static_cast<float>(r[R_NJ] >> 16);
            var[10] = f(R_MAXBT);
            var[18] = f(R_SUMM);
            var[19] = f(R_W);
            if (nlep >= 1) {
                var[13] = f(R_LPT);
                var[14] = f(R_LETA);
                var[15] = f(R_LPHI);
                var[16] = f(R_LISO);
                var[17] = __fadd_rn(var[0], var[13]);
            }
            MassObj ol, os;
            float p_ls = 0.0f;   // E_lead E_sub - p_lead . p_sub, shared with the triplet
            if (lead >= 0) {
                var[1] = f(R_J1);
                var[2] = f(R_J1 + 1);
                var[3] = f(R_J1 + 2);
                var[4] = f(R_J1 + 3);
                var[5] = f(R_J1 + 4);
                ol = mass_obj(var[1], var[2], var[3], var[4]);
            }
            if (sub >= 0) {
                var[6] = f(R_J2);
                os = mass_obj(var[6], f(R_J2 + 1), f(R_J2 + 2), f(R_J2 + 3));
                p_ls = pair_dot(ol, os);
                var[7] = sqrtf(ol.m * ol.m + os.m * os.m + 2.0f * p_ls);
            }
            if (njet >= 3 && ta >= 0) {
                // the triplet's four-momenta; jets shared with the leading pair reuse its terms
                auto obj = [&](int idx, int w) {
                    if (idx == lead) return ol;
                    if (idx == sub) return os;
                    return mass_obj(f(w), f(w + 1), f(w + 2), f(w + 3));
                };
                const MassObj oa = obj(ta, R_T1), ob = obj(tb, R_T2), oc = obj(tc, R_T3);
                auto pd = [&](int i, const MassObj& x, int j, const MassObj& y) {
                    if ((i == lead && j == sub) || (i == sub && j == lead)) return p_ls;
                    return pair_dot(x, y);
                };
                const float msum = oa.m * oa.m + ob.m * ob.m + oc.m * oc.m;
                var[11] = sqrtf(msum + 2.0f * (pd(ta, oa, tb, ob) + pd(ta, oa, tc, oc) + pd(tb, ob, tc, oc)));
                var[12] = sqrtf(f(R_BEST));
            }
            if (DEBUG) {
                const int64_t e = r[R_E];
                const int64_t kn = static_cast<int64_t>(k) * n;
                if (out.ev_pass) out.ev_pass[kn + e] = pass ? 1 : 0;
                if (out.ev_njet) out.ev_njet[kn + e] = njet;
                if (out.ev_nb) out.ev_nb[kn + e] = static_cast<int32_t>(r[R_NJ] >> 16);
                if (out.ev_idx) {
                    int32_t* ix = out.ev_idx + static_cast<int64_t>(k) * 5 * n;
                    ix[e] = lead;
                    ix[n + e] = sub;
                    ix[2 * n + e] = njet >= 3 ? ta : -1;
                    ix[3 * n + e] = njet >= 3 ? tb : -1;
                    ix[4 * n + e] = njet >= 3 ? tc : -1;
                }
                if (out.ev_vars) {
                    float* vv = out.ev_vars + static_cast<int64_t>(k) * kNV * n;
#pragma unroll
                    for (int h = 0; h < kNV; ++h) vv[h * n + e] = var[h];
                }
            }
        }
        __syncwarp();
        // fill entries overwrite the records: 20 variables and the variation
        // (0xffffffff: nothing to fill)
        if (have) {
            uint32_t* q = my_q + lane * R_WORDS;
#pragma unroll
            for (int h = 0; h < kNV; ++h) q[h] = __float_as_uint(var[h]);
            q[kNV] = pass ? static_cast<uint32_t>(k) : 0xffffffffu;
        }
        __syncwarp();
        if (HMODE == H_GLOBAL) {
            // global histograms: lane j fills every histogram of entry j
            // (lanes that meet on a bin are serialised by the L2 atomics)
            if (lane < m) {
                const uint32_t* q = my_q + lane * R_WORDS;
                const uint32_t kk = q[kNV];
                const double wd = static_cast<double>(__uint_as_float(q[19]));
                if (kk != 0xffffffffu) {
                    for (int h = 0; h < kNV; ++h) {
                        const float* eh = s_edges + P.eoff[h];
                        const int nb_h = P.nbins[h];
                        const int bin = find_bin_lim(__uint_as_float(q[h]), eh, P.e_lo[h], P.e_hi[h], nb_h, P.invw[h]);
                        if (bin < 0) continue;
                        const int at = static_cast<int>(kk) * P.total_bins + P.boff[h] + bin;
                        atomicAdd(&out.counts[at], 1ull);
                        atomicAdd(&out.sumw[at], wd);
                        if (out.sumw2) atomicAdd(&out.sumw2[at], wd * wd);
                    }
                }
            }
            __syncwarp();
            return;
        }
        // shared-memory histograms: lane h fills histogram h for every
        // queued entry (no two lanes of the warp touch the same bin)
        if (lane < kNV) {
            const int h = lane;
            const float* eh = s_edges + P.eoff[h];
            const int nb_h = P.nbins[h];
            const float invw = P.invw[h];
            const int boff = P.boff[h];
            for (int j = 0; j < m; ++j) {
                const uint32_t* q = my_q + j * R_WORDS;
                const uint32_t kk = q[kNV];
                if (kk == 0xffffffffu) continue;
                const int bin = find_bin(__uint_as_float(q[h]), eh, nb_h, invw);
                if (bin < 0) continue;
                const int at = static_cast<int>(kk) * P.total_bins + boff + bin;
                const double wd = static_cast<double>(__uint_as_float(q[19]));
                if (HMODE == H_SMEM) {
                    atomicAdd(&s_c[at], 1u);
                    atomicAdd(&s_w[at], wd);
                    if (out.sumw2) atomicAdd(&s_w2[at], wd * wd);
                } else {
                    const uint32_t rk = static_cast<uint32_t>(at) / static_cast<uint32_t>(L.hist_slice);
                    const int loc = at - static_cast<int>(rk) * L.hist_slice;
                    red_cluster_u32(map_to_rank(smem_addr(s_c + loc), rk), 1u);
                    red_cluster_f64(map_to_rank(smem_addr(s_w + loc), rk), wd);
                    if (out.sumw2) red_cluster_f64(map_to_rank(smem_addr(s_w2 + loc), rk), wd * wd);
                }
            }
        }
        __syncwarp();
    };

    int qcount = 0;
    int64_t* span1 = reinterpret_cast<int64_t*>(smem + L.bars + 32);   // warp 0: spans of the tile after next
    int64_t* span0 = reinterpret_cast<int64_t*>(smem + L.bars + 80);   // warp 0: spans of a sample's first tile
    uint32_t fpar[2] = {0u, 0u};
    uint32_t uses[2] = {0u, 0u};   // warp 0: copies issued into each stage
    int b = 0;
    bool stop = false;   // a bounded wait gave up: skip the remaining work, keep the barriers
    // this thread's offsets and weight of tile t (loaded a tile ahead)
    auto own_offsets = [&](int64_t t, int64_t (&os)[3], int64_t (&ot)[3], float& w) {
        int ts;
        int64_t lt;
        where(t, ts, lt);
        const SampleDesc& sd = SDs(ts);
        const int64_t ns = sd.n;
        const int64_t e = lt * E + tid;
        const int64_t elo = e < ns ? e : ns, ehi = e + 1 < ns ? e + 1 : ns;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            os[c] = ldoff(static_cast<const OffT*>(sd.off[c]), elo);
            ot[c] = ldoff(static_cast<const OffT*>(sd.off[c]), ehi);
        }
        w = e < ns ? sd.weight[e] : 0.0f;
    };
    for (int sl = 0; sl < (MULTI ? B.n_samples : 1); ++sl) {
    if constexpr (MULTI) {
        __syncthreads();   // every warp is done with the previous descriptor
        for (int i = tid; i < static_cast<int>(sizeof(SampleDesc) / 8); i += E)
            reinterpret_cast<uint64_t*>(cur)[i] = reinterpret_cast<const uint64_t*>(&B.s[sl])[i];
        __syncthreads();
    }
    if constexpr (FLAT) {
        ntiles = B.tile_start[B.n_samples];
    } else {
        n = SDs(0).n;
        ntiles = (n + E - 1) / E;
    }
    int64_t tile = stop ? ntiles : blockIdx.x;
    int64_t cs_[3] = {0, 0, 0}, ct_[3] = {0, 0, 0};
    float cw_ = 0.0f;   // this thread's event weight, loaded a tile ahead like its offsets
    if (tile < ntiles) {
        if (warp == 0) {
            load_span(tile, span0);
            // the stage is free once every warp released its last use
            bool ok = true;
            if (uses[b] > 0) ok = mbar_wait_bounded(empty[b], (uses[b] - 1) & 1u);
            if (__all_sync(0xffffffffu, ok)) {
                int ts;
                int64_t lt;
                where(tile, ts, lt);
                issue(b, ts, span0);
                ++uses[b];
            }
            if (tile + grid < ntiles) load_span(tile + grid, span1);
        }
        own_offsets(tile, cs_, ct_, cw_);
    }
    for (; tile < ntiles; tile += grid) {
        const int64_t next = tile + grid;
        if (warp == 0 && next < ntiles) {
            // the other stage is free once every warp released its previous tile
            bool ok = true;
            if (uses[b ^ 1] > 0) ok = mbar_wait_bounded(empty[b ^ 1], (uses[b ^ 1] - 1) & 1u);
            if (__all_sync(0xffffffffu, ok)) {
                int ts;
                int64_t lt;
                where(next, ts, lt);
                issue(b ^ 1, ts, span1);
                ++uses[b ^ 1];
                if (next + grid < ntiles) load_span(next + grid, span1);
            }
        }
        __syncwarp();
        int64_t ns_[3] = {0, 0, 0}, nt_[3] = {0, 0, 0};
        float nw_ = 0.0f;
        if (next < ntiles) own_offsets(next, ns_, nt_, nw_);
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(full[b], fpar[b]))) {   // error word set; this warp stops
            stop = true;
            break;
        }
        fpar[b] ^= 1u;

        const unsigned char* st = smem + b * L.stage_bytes;
        const int64_t* hdr = reinterpret_cast<const int64_t*>(st);
        const uint32_t* hoff = reinterpret_cast<const uint32_t*>(st + 32);
        // this tile's sample and its first event within the sample
        int cur_s;
        int64_t ltile;
        where(tile, cur_s, ltile);
        if constexpr (FLAT) n = SDs(cur_s).n;
        const int64_t e = ltile * E + tid;
        const bool valid = e < n;
        int rs[3], rt[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            rs[c] = static_cast<int>(cs_[c] - hdr[c]);
            rt[c] = static_cast<int>(ct_[c] - hdr[c]);
        }
        const bool staged = hoff[NC] != 0;
        StagedCols sc;
        DirectCols dc;
        dc.L = &L;
        dc.base = SDs(cur_s).col;
#pragma unroll
        for (int c = 0; c < 3; ++c) dc.S[c] = hdr[c];
        if (staged) {
#pragma unroll
            for (int c = 0; c < NC; ++c) sc.off[c] = hoff[c];
        }

        // this warp's spans per collection (tile-relative)
        int W0[3], W1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            W0[c] = __shfl_sync(0xffffffffu, rs[c], 0);
            W1[c] = __shfl_sync(0xffffffffu, rt[c], 31);
        }
        // bits of [lo, hi) inside the 32-element window starting at base
        auto range_mask = [](int lo, int hi, int base) -> unsigned {
            const int a = lo - base > 0 ? lo - base : 0;
            const int z = hi - base < 32 ? hi - base : 32;
            if (z <= a) return 0u;
            const unsigned top = z >= 32 ? 0xffffffffu : ((1u << z) - 1u);
            return top & ~((1u << a) - 1u);
        };
        auto lep_sel = [&](const auto& T, int c0, int i) -> bool {
            return Elem<KT>::f(T.template ld<KT>(c0, i)) > P.lep_pt_min &&
                   fabsf(Elem<KT>::f(T.template ld<KT>(c0 + 1, i))) < P.lep_abseta_max &&
                   T.template ld<uint8_t>(c0 + 4, i) != 0 && T.template ld<float>(c0 + 3, i) < P.lep_iso_max;
        };

        // selection, lanes over objects: leptons (muons first, then
        // electrons); per event the count and the first selected one
        int nlep = 0, lfirst = -1, lflav = 0;
        auto leptons = [&](const auto& T) {
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                const int c0 = f == 0 ? M_PT : E_PT;
                const int coll = 1 + f;
                for (int base = W0[coll]; base < W1[coll]; base += 32) {
                    const int p = base + lane;
                    const bool sel = p < W1[coll] && lep_sel(T, c0, p);
                    const unsigned hit = __ballot_sync(0xffffffffu, sel) & range_mask(rs[coll], rt[coll], base);
                    nlep += __popc(hit);
                    if (lfirst < 0 && hit) {
                        lfirst = base + __ffs(hit) - 1;
                        lflav = f;
                    }
                }
            }
        };
        if (staged)
            leptons(sc);
        else
            leptons(dc);
        if (!valid) nlep = 0;
        float lpt = qnan(), leta = qnan(), lphi = qnan(), liso = qnan();
        auto lep_vals = [&](const auto& T) {
            if (lfirst < 0) return;
            if (lflav == 0) {
                lpt = Elem<KT>::f(T.template ld<KT>(M_PT, lfirst));
                leta = Elem<KT>::f(T.template ld<KT>(M_ETA, lfirst));
                lphi = Elem<KT>::f(T.template ld<KT>(M_PHI, lfirst));
                liso = T.template ld<float>(M_ISO, lfirst);
            } else {
                lpt = Elem<KT>::f(T.template ld<KT>(E_PT, lfirst));
                leta = Elem<KT>::f(T.template ld<KT>(E_ETA, lfirst));
                lphi = Elem<KT>::f(T.template ld<KT>(E_PHI, lfirst));
                liso = T.template ld<float>(E_ISO, lfirst);
            }
        };
        if (valid) {
            if (staged)
                lep_vals(sc);
            else
                lep_vals(dc);
        }
        if (DEBUG && valid && SDs(0).out.ev_nlep) SDs(0).out.ev_nlep[e] = nlep;
        // without per-event outputs only single-lepton events can pass
        const bool active = valid && (DEBUG || nlep == 1);
        const unsigned amask = __ballot_sync(0xffffffffu, active);

        // jet acceptance (|eta|, Delta R >= cut to every selected lepton of
        // the jet's event), lanes over jets; one word of flags per 32 jets
        const int nround = (W1[0] - W0[0] + 31) >> 5;
        uint32_t* accw = reinterpret_cast<uint32_t*>(smem + L.acc) + warp * L.acc_words;
        // Delta R test of jet (eta, phi) against every selected lepton of the
        // event whose lepton ranges are given (events with several leptons)
        auto far_from_all = [&](const auto& T, float eta, float phi, int m0, int m1, int e0, int e1) -> bool {
            for (int l = m0; l < m1; ++l)
                if (lep_sel(T, M_PT, l) && dr2_f32(eta, phi, Elem<KT>::f(T.template ld<KT>(M_ETA, l)),
                                                   Elem<KT>::f(T.template ld<KT>(M_PHI, l))) < P.dr2_cut)
                    return false;
            for (int l = e0; l < e1; ++l)
                if (lep_sel(T, E_PT, l) && dr2_f32(eta, phi, Elem<KT>::f(T.template ld<KT>(E_ETA, l)),
                                                   Elem<KT>::f(T.template ld<KT>(E_PHI, l))) < P.dr2_cut)
                    return false;
            return true;
        };
        auto accept = [&](const auto& T) {
            for (int r = 0; r < nround && r < L.acc_words; ++r) {
                const int base = W0[0] + 32 * r;
                const int p = base + lane;
                // owner of jet p: the last lane whose jets start at or before p
                int own = 0;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    const int v = __shfl_sync(0xffffffffu, rs[0], own + step);
                    if (v <= p) own += step;
                }
                const int kind = __shfl_sync(0xffffffffu, nlep, own);
                const float le = __shfl_sync(0xffffffffu, leta, own);
                const float lp = __shfl_sync(0xffffffffu, lphi, own);
                const int m0 = __shfl_sync(0xffffffffu, rs[1], own), m1 = __shfl_sync(0xffffffffu, rt[1], own);
                const int e0 = __shfl_sync(0xffffffffu, rs[2], own), e1 = __shfl_sync(0xffffffffu, rt[2], own);
                bool ok = false;
                if (p < W1[0] && ((amask >> own) & 1u)) {
                    const float eta = Elem<KT>::f(T.template ld<KT>(J_ETA, p));
                    if (fabsf(eta) < P.jet_abseta_max) {
                        const float phi = Elem<KT>::f(T.template ld<KT>(J_PHI, p));
                        if (kind == 1)
                            ok = !(dr2_f32(eta, phi, le, lp) < P.dr2_cut);
                        else if (kind == 0)
                            ok = true;
                        else
                            ok = far_from_all(T, eta, phi, m0, m1, e0, e1);
                    }
                }
                const unsigned m = __ballot_sync(0xffffffffu, ok);
                if (lane == 0) accw[r] = m;
            }
        };
        if (amask) {
            if (staged)
                accept(sc);
            else
                accept(dc);
        }
        __syncwarp();
        // An event as the jet selection sees it: its jets, leptons and the
        // selected-lepton summary (taken from the event's own lane).
        struct Ev {
            int j0, j1, m0, m1, e0, e1, nlep;
            float leta, lphi;
        };
        // acceptance of jet i of event ev (flags, or recomputed past them)
        auto acc_of = [&](const auto& T, const Ev& ev, int i) -> bool {
            const int q = i - W0[0];
            if ((q >> 5) < L.acc_words) return ((accw[q >> 5] >> (q & 31)) & 1u) != 0;
            const float eta = Elem<KT>::f(T.template ld<KT>(J_ETA, i));
            if (!(fabsf(eta) < P.jet_abseta_max)) return false;
            const float phi = Elem<KT>::f(T.template ld<KT>(J_PHI, i));
            if (ev.nlep == 1) return !(dr2_f32(eta, phi, ev.leta, ev.lphi) < P.dr2_cut);
            if (ev.nlep == 0) return true;
            return far_from_all(T, eta, phi, ev.m0, ev.m1, ev.e0, ev.e1);
        };
        auto jet_sel = [&](const auto& T, const Ev& ev, int i, float s, float& ptk) -> bool {
            if (!acc_of(T, ev, i)) return false;
            ptk = __fmul_rn(Elem<KT>::f(T.template ld<KT>(J_PT, i)), s);
            return ptk > P.jet_pt_min;
        };
        const Ev own = {rs[0], rt[0], rs[1], rt[1], rs[2], rt[2], nlep, leta, lphi};
        // The jet counts decide the event through two thresholds: x -> fl(x * s)
        // is non-decreasing for s > 0, so at least two selected jets (pt_k >
        // cut) exist iff the second-largest accepted pt p2 has fl(p2 * s) >
        // cut, and a selected b-jet exists iff the largest accepted b-tagged
        // pt pb has fl(pb * s) > cut. p2 and pb do not depend on the
        // variation: one pass over the event's jets, by its own lane.
        float p1 = -INFINITY, p2 = -INFINITY, pb = -INFINITY;
        auto thresholds = [&](const auto& T) {
            for (int i = rs[0]; i < rt[0]; ++i) {
                if (!acc_of(T, own, i)) continue;
                const float pt = Elem<KT>::f(T.template ld<KT>(J_PT, i));
                if (pt > p1) {
                    p2 = p1;
                    p1 = pt;
                } else if (pt > p2) {
                    p2 = pt;
                }
                if (pt > pb && Elem<BT>::f(T.template ld<BT>(J_BTAG, i)) > P.btag_min) pb = pt;
            }
        };
        if (active) {
            if (staged)
                thresholds(sc);
            else
                thresholds(dc);
        }
        // a queued (event, variation): jet and b-jet counts, HT and the mass
        // sum (element order), leading pair, max btag; the transverse momenta
        // and tile indices of the first kScratch selected jets go to the slot
        // (its jet area and first words are free until the record is written)
        auto sums = [&](const auto& T, const Ev& ev, float s, uint32_t* r, int& nsel, int& nbj, int& lead,
                        int& sub) {
            float ht = 0.0f, summ = 0.0f, maxbt = qnan(), lead_pt = 0.0f, sub_pt = 0.0f;
            lead = -1;
            sub = -1;
            float* sx = reinterpret_cast<float*>(r + R_J1);
            float* sy = sx + kScratch;
            int16_t* li = reinterpret_cast<int16_t*>(r);
            nsel = 0;
            nbj = 0;
            for (int i = ev.j0; i < ev.j1; ++i) {
                float ptk;
                if (!jet_sel(T, ev, i, s, ptk)) continue;
                const float bt = Elem<BT>::f(T.template ld<BT>(J_BTAG, i));
                nbj += bt > P.btag_min ? 1 : 0;
                ht = __fadd_rn(ht, ptk);
                summ = __fadd_rn(summ, Elem<KT>::f(T.template ld<KT>(J_MASS, i)));
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
                if (nsel < kScratch) {
                    float sn, cs;
                    __sincosf(Elem<KT>::f(T.template ld<KT>(J_PHI, i)), &sn, &cs);
                    sx[nsel] = ptk * cs;
                    sy[nsel] = ptk * sn;
                    li[nsel] = static_cast<int16_t>(i);
                }
                ++nsel;
            }
            r[R_HT] = __float_as_uint(ht);
            r[R_SUMM] = __float_as_uint(summ);
            r[R_MAXBT] = __float_as_uint(maxbt);
        };
        // max |sum pT| triplet among the first n <= kScratch selected jets of
        // a slot: all C(n,3) triplets (colex table), largest value wins, ties
        // go to the smallest (a, b, c), i.e. the first in lexicographic order
        auto triplet = [&](const uint32_t* r, int n, float& best, int& key) {
            const float* qx = reinterpret_cast<const float*>(r + R_J1);
            const float* qy = qx + kScratch;
            const int ntri = n * (n - 1) * (n - 2) / 6;
            best = -1.0f;
            key = 0xfff;
            for (int t = 0; t < ntri; ++t) {
                const int abc = s_tri[t];
                const int a = abc & 15, b2 = (abc >> 4) & 15, c = abc >> 8;
                const float tx = (qx[a] + qx[b2]) + qx[c], ty = (qy[a] + qy[b2]) + qy[c];
                const float val = tx * tx + ty * ty;
                const int kk = (a << 8) | (b2 << 4) | c;
                if (val > best || (val == best && kk < key)) {
                    best = val;
                    key = kk;
                }
            }
        };
        // more selected jets than the scratch holds: all triplets from the tile
        auto slow_triplet = [&](const auto& T, const Ev& ev, float s, float& best, int& ta, int& tb, int& tc) {
            for (int a = ev.j0; a < ev.j1; ++a) {
                float pa;
                if (!jet_sel(T, ev, a, s, pa)) continue;
                float sa, ca;
                __sincosf(Elem<KT>::f(T.template ld<KT>(J_PHI, a)), &sa, &ca);
                for (int bq = a + 1; bq < ev.j1; ++bq) {
                    float pb2;
                    if (!jet_sel(T, ev, bq, s, pb2)) continue;
                    float sb, cb;
                    __sincosf(Elem<KT>::f(T.template ld<KT>(J_PHI, bq)), &sb, &cb);
                    const float bx = pa * ca + pb2 * cb, by = pa * sa + pb2 * sb;
                    for (int c = bq + 1; c < ev.j1; ++c) {
                        float pc;
                        if (!jet_sel(T, ev, c, s, pc)) continue;
                        float sc2, cc;
                        __sincosf(Elem<KT>::f(T.template ld<KT>(J_PHI, c)), &sc2, &cc);
                        const float tx = bx + pc * cc, ty = by + pc * sc2;
                        const float val = tx * tx + ty * ty;
                        if (val > best) {
                            best = val;
                            ta = a;
                            tb = bq;
                            tc = c;
                        }
                    }
                }
            }
        };
        auto jet4 = [&](const auto& T, float s, int i, uint32_t* q) {
            put4(q, __fmul_rn(Elem<KT>::f(T.template ld<KT>(J_PT, i)), s), Elem<KT>::f(T.template ld<KT>(J_ETA, i)),
                 Elem<KT>::f(T.template ld<KT>(J_PHI, i)), Elem<KT>::f(T.template ld<KT>(J_MASS, i)));
        };

        // The (event, variation) pairs to queue, 32 at a time with one lane
        // per pair: the event's lane hands over its summary, the pair's lane
        // builds the record (jet sums, triplet, four-momenta) from the stage.
        // each event's summary goes to shared memory (field-major, lane
        // minor), where the pairs read it
        uint16_t* my_pairs = reinterpret_cast<uint16_t*>(smem + L.pairs) + warp * 64;
        uint32_t* my_evs = reinterpret_cast<uint32_t*>(smem + L.evs) + warp * (kEvWords * 32);
        my_evs[0 * 32 + lane] = static_cast<uint32_t>(rs[0]);
        my_evs[1 * 32 + lane] = static_cast<uint32_t>(rt[0]);
        my_evs[2 * 32 + lane] = static_cast<uint32_t>(rs[1]);
        my_evs[3 * 32 + lane] = static_cast<uint32_t>(rt[1]);
        my_evs[4 * 32 + lane] = static_cast<uint32_t>(rs[2]);
        my_evs[5 * 32 + lane] = static_cast<uint32_t>(rt[2]);
        my_evs[6 * 32 + lane] = static_cast<uint32_t>(nlep);
        my_evs[7 * 32 + lane] = __float_as_uint(leta);
        my_evs[8 * 32 + lane] = __float_as_uint(lphi);
        my_evs[9 * 32 + lane] = __float_as_uint(cw_);
        my_evs[10 * 32 + lane] = __float_as_uint(lpt);
        my_evs[11 * 32 + lane] = __float_as_uint(liso);
        __syncwarp();
        auto process = [&](int m) {
            if (qcount + m > 32) {
                flush(qcount);
                qcount = 0;
            }
            const bool mine = lane < m;
            const int pk = my_pairs[mine ? lane : 0];
            const int el = pk & 31;
            Ev ev;
            ev.j0 = static_cast<int>(my_evs[0 * 32 + el]);
            ev.j1 = static_cast<int>(my_evs[1 * 32 + el]);
            ev.m0 = static_cast<int>(my_evs[2 * 32 + el]);
            ev.m1 = static_cast<int>(my_evs[3 * 32 + el]);
            ev.e0 = static_cast<int>(my_evs[4 * 32 + el]);
            ev.e1 = static_cast<int>(my_evs[5 * 32 + el]);
            ev.nlep = static_cast<int>(my_evs[6 * 32 + el]);
            ev.leta = __uint_as_float(my_evs[7 * 32 + el]);
            ev.lphi = __uint_as_float(my_evs[8 * 32 + el]);
            uint32_t* r = my_q + (qcount + (mine ? lane : 0)) * R_WORDS;
            const int k = (pk >> 5) & 63;
            const bool pass = (pk & 0x800) != 0;
            const float s = P.scales[k];
            int nsel = 0, nbj = 0, lead = -1, sub = -1;
            if (mine) {
                if (staged)
                    sums(sc, ev, s, r, nsel, nbj, lead, sub);
                else
                    sums(dc, ev, s, r, nsel, nbj, lead, sub);
            }
            __syncwarp();
            float best = -1.0f;
            int key = 0xfff;
            if (mine && nsel >= 3 && nsel <= kScratch) triplet(r, nsel, best, key);
            if (mine) {
                int ta = -1, tb = -1, tc = -1;
                if (nsel >= 3 && nsel <= kScratch) {
                    // key 0xfff: every triplet's value was NaN (a NaN phi), no triplet
                    if (key != 0xfff) {
                        const int16_t* li = reinterpret_cast<const int16_t*>(r);
                        ta = li[key >> 8];
                        tb = li[(key >> 4) & 15];
                        tc = li[key & 15];
                    }
                } else if (nsel > kScratch) {
                    if (staged)
                        slow_triplet(sc, ev, s, best, ta, tb, tc);
                    else
                        slow_triplet(dc, ev, s, best, ta, tb, tc);
                }
                r[R_BEST] = __float_as_uint(best);
                const int l16 = lead < 0 ? 0xffff : (lead - ev.j0) & 0xffff;
                const int s16 = sub < 0 ? 0xffff : (sub - ev.j0) & 0xffff;
                r[R_IDX] = static_cast<uint32_t>(l16) | (static_cast<uint32_t>(s16) << 16);
                const int a16 = ta < 0 ? 0xffff : (ta - ev.j0) & 0xffff;
                const int b16 = tb < 0 ? 0xffff : (tb - ev.j0) & 0xffff;
                r[R_TAB] = static_cast<uint32_t>(a16) | (static_cast<uint32_t>(b16) << 16);
                r[R_TC] = static_cast<uint32_t>(tc < 0 ? -1 : tc - ev.j0);
                auto write4 = [&](const auto& T) {
                    if (lead >= 0) {
                        jet4(T, s, lead, r + R_J1);
                        r[R_J1 + 4] = __float_as_uint(Elem<BT>::f(T.template ld<BT>(J_BTAG, lead)));
                    }
                    if (sub >= 0) jet4(T, s, sub, r + R_J2);
                    if (ta >= 0) {
                        jet4(T, s, ta, r + R_T1);
                        jet4(T, s, tb, r + R_T2);
                        jet4(T, s, tc, r + R_T3);
                    }
                };
                if (staged)
                    write4(sc);
                else
                    write4(dc);
                r[R_E] = static_cast<uint32_t>(ltile * E + warp * 32 + el);
                r[R_K] = static_cast<uint32_t>(k) | (pass ? 0x100u : 0u) | (static_cast<uint32_t>(cur_s) << 9) |
                         (static_cast<uint32_t>(min(ev.nlep, 0xffff)) << 16);
                r[R_NJ] = static_cast<uint32_t>(min(nsel, 0xffff)) | (static_cast<uint32_t>(min(nbj, 0xffff)) << 16);
                r[R_W] = my_evs[9 * 32 + el];
                r[R_LPT] = my_evs[10 * 32 + el];
                r[R_LETA] = __float_as_uint(ev.leta);
                r[R_LPHI] = __float_as_uint(ev.lphi);
                r[R_LISO] = my_evs[11 * 32 + el];
            }
            __syncwarp();
            qcount += m;
        };
        int npairs = 0;
        for (int k = 0; k < P.n_var; ++k) {
            const float s = P.scales[k];
            const bool pass = active && nlep == 1 && __fmul_rn(p2, s) > P.jet_pt_min &&
                              __fmul_rn(pb, s) > P.jet_pt_min;
            const bool enq = DEBUG ? valid : pass;
            const unsigned emask = __ballot_sync(0xffffffffu, enq);
            if (emask == 0u) continue;
            if (enq) my_pairs[npairs + __popc(emask & lt_mask)] = static_cast<uint16_t>(lane | (k << 5) | (pass ? 0x800 : 0));
            npairs += __popc(emask);
            __syncwarp();
            if (npairs >= 32) {
                process(32);
                // the rest (fewer than 32) moves to the front
                const int rest = npairs - 32;
                const uint16_t v = lane < rest ? my_pairs[32 + lane] : 0;
                __syncwarp();
                if (lane < rest) my_pairs[lane] = v;
                __syncwarp();
                npairs = rest;
            }
        }
        if (npairs > 0) process(npairs);
        // this warp is done with the stage
        __syncwarp();
        if (lane == 0) mbar_arrive(empty[b]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            cs_[c] = ns_[c];
            ct_[c] = nt_[c];
        }
        cw_ = nw_;
        b ^= 1;
    }
    if (qcount > 0) flush(qcount);
    qcount = 0;

    // the sample's histograms: block-private or cluster-slice copies go to
    // the sample's outputs and are cleared for the next sample
    if (HMODE != H_GLOBAL) {
        const ChainOut& out = SDs(0).out;
        if (HMODE == H_CLUSTER)
            cluster_sync_all();
        else
            __syncthreads();
        const int first = HMODE == H_CLUSTER ? static_cast<int>(my_rank) * L.hist_slice : 0;
        for (int i = tid; i < hist_local; i += E) {
            const int g = first + i;
            const unsigned c = s_c[i];
            if (c != 0u && g < hist_n) {
                atomicAdd(&out.counts[g], static_cast<unsigned long long>(c));
                atomicAdd(&out.sumw[g], s_w[i]);
                if (out.sumw2) atomicAdd(&out.sumw2[g], s_w2[i]);
            }
            s_c[i] = 0u;
            s_w[i] = 0.0;
            s_w2[i] = 0.0;
        }
        if (HMODE == H_CLUSTER)
            cluster_sync_all();
        else
            __syncthreads();
    }
    }
}

// Launch parameters prepared by the host entry points for the typed launchers.
struct LaunchArgs {
    Layout layout;
    const ChainParams* P;
    const BatchDesc* B;
    hepacc_dtype offsets_type, btag_type;
    bool debug;
    int hmode;
    int block;
    int cluster;         // blocks per cluster (H_CLUSTER)
    int grid;            // 0 = as many resident blocks (clusters) as fit
    int64_t max_tiles;   // most tiles of any sample (caps the grid)
    cudaStream_t stream;
};

template <typename T> struct Tag { using type = T; };

struct Cache {
    std::mutex mu;
    std::unordered_map<const void*, int> smem_set;
};
inline Cache& cache() {
    static Cache c;
    return c;
}

template <typename K>
hepacc_status launch_chain(K kernel, const LaunchArgs& a) {
    const DeviceInfo di = device_info();
    const size_t smem = a.layout.total;
    if (smem > static_cast<size_t>(di.smem_optin)) return fail(HEPACC_ERR_INVALID_ARG, "chain shared memory too large");
    {
        std::lock_guard<std::mutex> g(cache().mu);
        auto it = cache().smem_set.find(reinterpret_cast<const void*>(kernel));
        if (it == cache().smem_set.end() || it->second < static_cast<int>(smem)) {
            cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
            if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
            if (a.hmode == H_CLUSTER) {
                e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
                if (e != cudaSuccess) return cuda_fail(e, "cluster size attribute");
            }
            cache().smem_set[reinterpret_cast<const void*>(kernel)] = static_cast<int>(smem);
        }
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.blockDim = dim3(a.block, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = a.stream;
    int grid = 0;
    if (a.hmode == H_CLUSTER) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = a.cluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cfg.gridDim = dim3(a.cluster * di.sms, 1, 1);
        int nclusters = 0;
        cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, kernel, &cfg);
        if (e != cudaSuccess) return cuda_fail(e, "cluster occupancy query");
        if (nclusters < 1) return fail(HEPACC_ERR_INVALID_ARG, "chain clusters of %d blocks do not fit", a.cluster);
        grid = nclusters * a.cluster;
        if (a.grid > 0) grid = std::min(grid, (a.grid / a.cluster) * a.cluster);
        if (grid < a.cluster) grid = a.cluster;
    } else {
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, a.block, smem);
        if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
        if (per_sm < 1) return fail(HEPACC_ERR_INVALID_ARG, "chain kernel does not fit on an SM");
        grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(a.max_tiles, static_cast<int64_t>(per_sm) * di.sms)));
        if (a.grid > 0) grid = a.grid;
    }
    cfg.gridDim = dim3(grid, 1, 1);
    cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, a.layout, *a.P, *a.B);
    if (e != cudaSuccess) return cuda_fail(e, "chain launch");
    HEPACC_CHECK_LAUNCH("chain launch");
    return HEPACC_OK;
}

// Many samples in one launch with shared-memory histograms (int64 offsets;
// btag float32 with float32 kinematics, float16 with half kinematics):
// every block walks the samples in turn. Plans with global histograms run
// the compacting kernel (fused_kernel.cuh) instead.
template <typename KT, typename BT>
hepacc_status run_batched_typed(const LaunchArgs& a) {
    if (a.offsets_type != HEPACC_I64) return fail(HEPACC_ERR_DTYPE, "batched launches need I64 offsets");
    if (a.hmode == H_CLUSTER) return launch_chain(k_chain<KT, BT, int64_t, false, H_CLUSTER, F_SAMPLES>, a);
    if (a.hmode == H_SMEM) return launch_chain(k_chain<KT, BT, int64_t, false, H_SMEM, F_SAMPLES>, a);
    return fail(HEPACC_ERR_INVALID_ARG, "walking launches keep their histograms in shared memory");
}

hepacc_status run_batched_f32(const LaunchArgs& a);
hepacc_status run_batched_bf16(const LaunchArgs& a);
hepacc_status run_batched_f16(const LaunchArgs& a);

}  // namespace chain
}  // namespace hepacc
