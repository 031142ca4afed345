// Per-operation kernels (Section III of arXiv:1906.06242): segmented sum,
// max/min, get/set within offsets, Delta R masking, trijet and pair masses,
// object selection, scaling and weighted histogram filling, with their C-ABI
// entry points.
#include <algorithm>
#include <cstdlib>
#include <mutex>
#include <unordered_map>

#include "hepacc_host.h"
#include "hepacc_tiles.cuh"

namespace hepacc {

// Debug checks of the offsets before a chain launch: on when the
// environment variable HEPACC_DEBUG is set to a value other than 0, or when
// the caller asks (plans).
bool debug_checks() {
    static const bool on = [] {
        const char* v = std::getenv("HEPACC_DEBUG");
        return v != nullptr && v[0] != '\0' && !(v[0] == '0' && v[1] == '\0');
    }();
    return on;
}


namespace {

constexpr int kBlock = 256;             // 8 warps
constexpr int NC = 6;                   // columns per stage at most
using Spec = StageSpec<NC>;

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

template <typename T> struct Acc { using type = float; };
template <> struct Acc<uint8_t> { using type = int64_t; };
template <> struct Acc<int8_t> { using type = int64_t; };
template <> struct Acc<int32_t> { using type = int64_t; };
template <> struct Acc<int64_t> { using type = int64_t; };

template <typename AccT, typename T>
__device__ __forceinline__ AccT acc_add(AccT a, T x) { return a + static_cast<AccT>(x); }
template <>
__device__ __forceinline__ float acc_add<float, float>(float a, float x) { return __fadd_rn(a, x); }
template <>
__device__ __forceinline__ float acc_add<float, __half>(float a, __half x) { return __fadd_rn(a, __half2float(x)); }
template <>
__device__ __forceinline__ float acc_add<float, __nv_bfloat16>(float a, __nv_bfloat16 x) {
    return __fadd_rn(a, __bfloat162float(x));
}

// sum_in_offsets (Listing 1): out[e] += masked elements in element order.
// Columns: 0 = content, 1 = mask_content. Lane = event, no staging.
template <typename T, typename OffT, typename OutT>
__global__ void __launch_bounds__(kBlock) k_sum(Spec spec, const OffT* off, int64_t n,
                                                const uint8_t* __restrict__ mask_rows, OutT* __restrict__ out) {
    const OffT* const offs[1] = {off};
    const bool hm = spec.col[1].base != nullptr;
    event_loop<OffT, 1, NC>(spec, offs, n, [&](const auto& C, const TileRanges<1>& r) {
        if (!r.valid || (mask_rows && !mask_rows[r.e])) return;
        using A = typename Acc<T>::type;
        A acc = static_cast<A>(out[r.e]);
        for (int i = r.rs[0]; i < r.rt[0]; ++i) {
            if (hm && !C.template ld<uint8_t>(1, i)) continue;
            acc = acc_add<A, T>(acc, C.template ld<T>(0, i));
        }
        out[r.e] = static_cast<OutT>(acc);
    });
}

// max/min_in_offsets: first occurrence of the extreme non-NaN masked value.
// Lane = event, no staging.
template <typename T, typename OffT, bool MAX>
__global__ void __launch_bounds__(kBlock) k_minmax(Spec spec, const OffT* off, int64_t n,
                                                   const uint8_t* __restrict__ mask_rows, float empty,
                                                   float* __restrict__ out, int32_t* __restrict__ arg) {
    const OffT* const offs[1] = {off};
    const bool hm = spec.col[1].base != nullptr;
    event_loop<OffT, 1, NC>(spec, offs, n, [&](const auto& C, const TileRanges<1>& r) {
        if (!r.valid || (mask_rows && !mask_rows[r.e])) return;
        int bi = -1;
        float best = empty;
        for (int i = r.rs[0]; i < r.rt[0]; ++i) {
            if (hm && !C.template ld<uint8_t>(1, i)) continue;
            const float x = Elem<T>::f(C.template ld<T>(0, i));
            if (x != x) continue;
            if (bi < 0 || (MAX ? x > best : x < best)) {
                best = x;
                bi = i;
            }
        }
        if (out) out[r.e] = bi < 0 ? empty : best;
        if (arg) arg[r.e] = bi < 0 ? -1 : bi - r.rs[0];
    });
}

// get_in_offsets: the n-th masked-in element. Lane = event, no staging.
template <typename T, typename OffT>
__global__ void __launch_bounds__(kBlock) k_get(Spec spec, const OffT* off, int64_t n,
                                                const int32_t* __restrict__ nth, int32_t nth_scalar,
                                                const uint8_t* __restrict__ mask_rows, float dflt,
                                                float* __restrict__ out, int32_t* __restrict__ oidx) {
    const OffT* const offs[1] = {off};
    const bool hm = spec.col[1].base != nullptr;
    event_loop<OffT, 1, NC>(spec, offs, n, [&](const auto& C, const TileRanges<1>& r) {
        if (!r.valid || (mask_rows && !mask_rows[r.e])) return;
        const int64_t want = nth ? nth[r.e] : nth_scalar;
        int64_t seen = 0;
        int found = -1;
        if (want >= 0) {
            for (int i = r.rs[0]; i < r.rt[0]; ++i) {
                if (hm && !C.template ld<uint8_t>(1, i)) continue;
                if (seen == want) {
                    found = i;
                    break;
                }
                ++seen;
            }
        }
        if (out) out[r.e] = found < 0 ? dflt : Elem<T>::f(C.template ld<T>(0, found));
        if (oidx) oidx[r.e] = found < 0 ? -1 : found - r.rs[0];
    });
}

// mask_deltar_first. Columns: 0 eta1, 1 phi1, 2 mask1_in (collection 0);
// 3 eta2, 4 phi2, 5 mask2 (collection 1). Lane = event, no staging.
template <typename T1, typename T2, typename OffT>
__global__ void __launch_bounds__(kBlock) k_deltar(Spec spec, const OffT* off1, const OffT* off2, int64_t n,
                                                   const uint8_t* __restrict__ mask_rows, float cut,
                                                   uint8_t* __restrict__ mask_out) {
    const OffT* const offs[2] = {off1, off2};
    const bool h1 = spec.col[2].base != nullptr, h2 = spec.col[5].base != nullptr;
    event_loop<OffT, 2, NC>(spec, offs, n, [&](const auto& C, const TileRanges<2>& r) {
        if (!r.valid || (mask_rows && !mask_rows[r.e])) return;
        for (int i = r.rs[0]; i < r.rt[0]; ++i) {
            bool keep = h1 ? C.template ld<uint8_t>(2, i) != 0 : true;
            if (keep) {
                const float e1 = Elem<T1>::f(C.template ld<T1>(0, i));
                const float p1 = Elem<T1>::f(C.template ld<T1>(1, i));
                for (int j = r.rs[1]; j < r.rt[1]; ++j) {
                    if (h2 && !C.template ld<uint8_t>(5, j)) continue;
                    const float d = dr2_f32(e1, p1, Elem<T2>::f(C.template ld<T2>(3, j)),
                                            Elem<T2>::f(C.template ld<T2>(4, j)));
                    if (d < cut) {
                        keep = false;
                        break;
                    }
                }
            }
            mask_out[r.S[0] + i] = keep ? 1 : 0;
        }
    });
}

// Trijet: max |sum pT| over triplets of masked-in objects, its mass.
// Columns: 0 pt, 1 eta, 2 phi, 3 mass, 4 mask. Lane = event, no staging.
constexpr int kTriLocal = 24;

template <typename T, typename OffT>
__global__ void __launch_bounds__(kBlock) k_trijet(Spec spec, const OffT* off, int64_t n,
                                                   const uint8_t* __restrict__ mask_rows, float* __restrict__ om,
                                                   float* __restrict__ opt, int32_t* __restrict__ oidx) {
    const OffT* const offs[1] = {off};
    const bool hm = spec.col[4].base != nullptr;
    event_loop<OffT, 1, NC>(spec, offs, n, [&](const auto& C, const TileRanges<1>& r) {
        if (!r.valid || (mask_rows && !mask_rows[r.e])) return;
        auto pt_of = [&](int i) { return Elem<T>::f(C.template ld<T>(0, i)); };
        auto phi_of = [&](int i) { return Elem<T>::f(C.template ld<T>(2, i)); };
        auto on = [&](int i) { return !hm || C.template ld<uint8_t>(4, i) != 0; };
        float px[kTriLocal], py[kTriLocal];
        int32_t li[kTriLocal];
        int cnt = 0;
        for (int i = r.rs[0]; i < r.rt[0]; ++i) {
            if (!on(i)) continue;
            if (cnt < kTriLocal) {
                float sn, cs;
                const float pt = pt_of(i);
                sincosf(phi_of(i), &sn, &cs);
                px[cnt] = pt * cs;
                py[cnt] = pt * sn;
                li[cnt] = i - r.rs[0];
            }
            ++cnt;
        }
        int32_t ba = -1, bb = -1, bc = -1;
        float best = -1.0f;
        if (cnt >= 3 && cnt <= kTriLocal) {
            for (int a = 0; a < cnt; ++a)
                for (int b = a + 1; b < cnt; ++b) {
                    const float sx = px[a] + px[b], sy = py[a] + py[b];
                    for (int c = b + 1; c < cnt; ++c) {
                        const float tx = sx + px[c], ty = sy + py[c];
                        const float val = tx * tx + ty * ty;
                        if (val > best) {
                            best = val;
                            ba = li[a];
                            bb = li[b];
                            bc = li[c];
                        }
                    }
                }
        } else if (cnt > kTriLocal) {
            // many objects: enumerate the masked-in elements directly
            for (int a = r.rs[0]; a < r.rt[0]; ++a) {
                if (!on(a)) continue;
                float sa, ca;
                sincosf(phi_of(a), &sa, &ca);
                const float pa = pt_of(a);
                for (int b = a + 1; b < r.rt[0]; ++b) {
                    if (!on(b)) continue;
                    float sb, cb;
                    sincosf(phi_of(b), &sb, &cb);
                    const float pb = pt_of(b);
                    const float sx = pa * ca + pb * cb, sy = pa * sa + pb * sb;
                    for (int c = b + 1; c < r.rt[0]; ++c) {
                        if (!on(c)) continue;
                        float sc, cc;
                        sincosf(phi_of(c), &sc, &cc);
                        const float pc = pt_of(c);
                        const float tx = sx + pc * cc, ty = sy + pc * sc;
                        const float val = tx * tx + ty * ty;
                        if (val > best) {
                            best = val;
                            ba = a - r.rs[0];
                            bb = b - r.rs[0];
                            bc = c - r.rs[0];
                        }
                    }
                }
            }
        }
        float m = __int_as_float(0x7fc00000), ptj = m;
        if (ba >= 0) {
            MassObj o[3];
            const int32_t ix[3] = {ba, bb, bc};
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int i = r.rs[0] + ix[q];
                o[q] = mass_obj(pt_of(i), Elem<T>::f(C.template ld<T>(1, i)), phi_of(i),
                                Elem<T>::f(C.template ld<T>(3, i)));
            }
            m = mass3obj(o[0], o[1], o[2]);
            ptj = sqrtf(best);
        }
        if (om) om[r.e] = m;
        if (opt) opt[r.e] = ptj;
        if (oidx) {
            oidx[3 * r.e] = ba;
            oidx[3 * r.e + 1] = bb;
            oidx[3 * r.e + 2] = bc;
        }
    });
}

template <typename T, typename OffT>
__global__ void __launch_bounds__(kBlock) k_pair_mass(const T* pt, const T* eta, const T* phi, const T* mass,
                                                      const OffT* off, int64_t n, const int32_t* ia,
                                                      const int32_t* ib, const uint8_t* mask_rows, float* out) {
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (mask_rows && !mask_rows[e]) continue;
        const int64_t i0 = ldoff(off, e), cnt = ldoff(off, e + 1) - i0;
        const int64_t a = ia[e], b = ib[e];
        if (a < 0 || b < 0 || a >= cnt || b >= cnt) {
            out[e] = __int_as_float(0x7fc00000);
            continue;
        }
        const MassObj oa = mass_obj(ldf(pt, i0 + a), ldf(eta, i0 + a), ldf(phi, i0 + a), ldf(mass, i0 + a));
        const MassObj ob = mass_obj(ldf(pt, i0 + b), ldf(eta, i0 + b), ldf(phi, i0 + b), ldf(mass, i0 + b));
        out[e] = mass2obj(oa, ob);
    }
}

// Top candidate (Section IV): the triplet of masked-in objects whose mass
// is closest to the target; ties keep the first triplet in lexicographic
// order. Per-event form (one thread, the event's objects in a loop): the
// objects' mass terms are prepared once per event (up to kCloseLocal of
// them; beyond that they are recomputed per triplet).
constexpr int kCloseLocal = 12;

struct Closest {
    float m;
    int32_t a, b, c;
};

template <typename T>
__device__ Closest closest_loop(const T* pt, const T* eta, const T* phi, const T* mass, int64_t i0, int64_t i1,
                                const uint8_t* mask_content, float target) {
    auto on = [&](int64_t i) { return mask_content == nullptr || mask_content[i] != 0; };
    auto obj = [&](int64_t i) { return mass_obj(ldf(pt, i), ldf(eta, i), ldf(phi, i), ldf(mass, i)); };
    MassObj o[kCloseLocal];
    int32_t li[kCloseLocal];
    int cnt = 0;
    for (int64_t i = i0; i < i1; ++i) {
        if (!on(i)) continue;
        if (cnt < kCloseLocal) {
            o[cnt] = obj(i);
            li[cnt] = static_cast<int32_t>(i - i0);
        }
        ++cnt;
    }
    float best_d = INFINITY;
    Closest r{__int_as_float(0x7fc00000), -1, -1, -1};
    if (cnt >= 3 && cnt <= kCloseLocal) {
        for (int a = 0; a < cnt; ++a)
            for (int b = a + 1; b < cnt; ++b)
                for (int c = b + 1; c < cnt; ++c) {
                    const float m = mass3obj(o[a], o[b], o[c]);
                    const float d = fabsf(m - target);
                    if (d < best_d) {
                        best_d = d;
                        r = Closest{m, li[a], li[b], li[c]};
                    }
                }
    } else if (cnt > kCloseLocal) {
        for (int64_t a = i0; a < i1; ++a) {
            if (!on(a)) continue;
            const MassObj oa = obj(a);
            for (int64_t b = a + 1; b < i1; ++b) {
                if (!on(b)) continue;
                const MassObj ob = obj(b);
                for (int64_t c = b + 1; c < i1; ++c) {
                    if (!on(c)) continue;
                    const float m = mass3obj(oa, ob, obj(c));
                    const float d = fabsf(m - target);
                    if (d < best_d) {
                        best_d = d;
                        r = Closest{m, static_cast<int32_t>(a - i0), static_cast<int32_t>(b - i0),
                                    static_cast<int32_t>(c - i0)};
                    }
                }
            }
        }
    }
    return r;
}

// Warp-cooperative form. A warp takes 32 consecutive events (lane l owns
// event l). Events with 3..kCoopMax masked-in objects are admitted in lane
// order while the warp's objects and pairs fit its shared-memory slots; the
// others (more objects, or past the capacity) take closest_loop. For the
// admitted events: (A) each owner lists its masked-in objects; (B) their
// mass terms are computed lane-parallel over the warp's objects; (C) every
// pair term E_aE_b - p_a.p_b is computed once, lane-parallel over the warp's
// pairs (pair (x < y) of an event in slot C(y,2) + x, colex order);
// (D) the triplets of all admitted events are ranked lane-parallel, 32 at a
// time (triplet (a < b < c) is rank C(c,3) + C(b,2) + a of its event), each
// mass from three pair terms in the same order as mass3obj, with the key
// (|m - target| bits, a << 8 | b << 4 | c) so that the minimum key is the
// closest triplet
// and, on ties, the first in lexicographic order; a segmented minimum over
// the lanes holding one event's triplets goes to the owner lane. NaN
// distances never win (their keys exceed the initial one).
constexpr int kCoopMax = 16;      // objects per admitted event (4 bits per index in the key)
constexpr int kCoopObj = 256;     // object slots per warp
constexpr int kCoopPair = 1024;   // pair slots per warp
constexpr int kCoopTri = 560;     // C(16, 3)
constexpr int kCoopPairs16 = 120; // C(16, 2)

struct CoopWarp {
    MassObj obj[kCoopObj];
    float pd[kCoopPair];
    int32_t li[kCoopObj];   // local index of the object in its event
    uint8_t ev[kCoopObj];   // owner lane of the object
    int64_t i0[32];
    int32_t cnt[32], obase[32], pincl[32], tincl[32];
};

inline size_t coop_smem() {
    return static_cast<size_t>(kBlock / 32) * sizeof(CoopWarp) + kCoopTri * 2 + kCoopPairs16 * 2;
}

__device__ __forceinline__ int choose2(int k) { return k * (k - 1) / 2; }
__device__ __forceinline__ int choose3(int k) { return k * (k - 1) * (k - 2) / 6; }

__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// smallest lane l with incl[l] > q (q below incl[31])
__device__ __forceinline__ int owner_of(const int32_t* incl, int q) {
    int lo = 0, hi = 31;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (incl[mid] > q) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

template <typename T, typename OffT>
__global__ void __launch_bounds__(kBlock) k_trijet_closest(const T* pt, const T* eta, const T* phi, const T* mass,
                                                           const OffT* off, int64_t n, const uint8_t* mask_rows,
                                                           const uint8_t* mask_content, float target,
                                                           float* out_mass, int32_t* out_idx3) {
    extern __shared__ __align__(16) unsigned char smem[];
    CoopWarp* warps = reinterpret_cast<CoopWarp*>(smem);
    uint16_t* tri_tab = reinterpret_cast<uint16_t*>(smem + (kBlock / 32) * sizeof(CoopWarp));
    uint16_t* pair_tab = tri_tab + kCoopTri;
    // colex tables: rank -> (a, b, c) as a | b << 4 | c << 8, rank -> (x, y) as x | y << 4
    for (int r = threadIdx.x; r < kCoopTri; r += blockDim.x) {
        int c = 2;
        while (choose3(c + 1) <= r) ++c;
        const int rem = r - choose3(c);
        int b = 1;
        while (choose2(b + 1) <= rem) ++b;
        tri_tab[r] = static_cast<uint16_t>((rem - choose2(b)) | (b << 4) | (c << 8));
    }
    for (int q = threadIdx.x; q < kCoopPairs16; q += blockDim.x) {
        int y = 1;
        while (choose2(y + 1) <= q) ++y;
        pair_tab[q] = static_cast<uint16_t>((q - choose2(y)) | (y << 4));
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    CoopWarp& W = warps[threadIdx.x >> 5];
    auto on = [&](int64_t i) { return mask_content == nullptr || mask_content[i] != 0; };
    const int64_t nwb = (n + 31) / 32;
    for (int64_t wb = static_cast<int64_t>(blockIdx.x) * (kBlock / 32) + (threadIdx.x >> 5); wb < nwb;
         wb += static_cast<int64_t>(gridDim.x) * (kBlock / 32)) {
        const int64_t e = wb * 32 + lane;
        const bool valid = e < n && (!mask_rows || mask_rows[e]);
        int64_t i0 = 0, i1 = 0;
        int cnt = 0;
        if (valid) {
            i0 = ldoff(off, e);
            i1 = ldoff(off, e + 1);
            for (int64_t i = i0; i < i1 && cnt <= kCoopMax; ++i) cnt += on(i) ? 1 : 0;
        }
        const bool cand = valid && cnt >= 3 && cnt <= kCoopMax;
        // admission: candidates in lane order while objects and pairs fit
        const int oi = warp_incl_scan(cand ? cnt : 0, lane);
        const int pi = warp_incl_scan(cand ? choose2(cnt) : 0, lane);
        const bool admit = cand && oi <= kCoopObj && pi <= kCoopPair;
        const int ocnt = admit ? cnt : 0;
        const int oincl = warp_incl_scan(ocnt, lane);
        const int pincl = warp_incl_scan(admit ? choose2(cnt) : 0, lane);
        const int tincl = warp_incl_scan(admit ? choose3(cnt) : 0, lane);
        const int obase = oincl - ocnt;
        W.i0[lane] = i0;
        W.cnt[lane] = ocnt;
        W.obase[lane] = obase;
        W.pincl[lane] = pincl;
        W.tincl[lane] = tincl;
        // (A) the admitted events' masked-in objects
        if (admit) {
            int k = 0;
            for (int64_t i = i0; i < i1 && k < cnt; ++i) {
                if (!on(i)) continue;
                W.li[obase + k] = static_cast<int32_t>(i - i0);
                W.ev[obase + k] = static_cast<uint8_t>(lane);
                ++k;
            }
        }
        __syncwarp();
        const int n_obj = W.obase[31] + W.cnt[31];
        const int n_pair = W.pincl[31];
        const int n_tri = W.tincl[31];
        // (B) mass terms, lane-parallel over the objects
        for (int sidx = lane; sidx < n_obj; sidx += 32) {
            const int64_t gi = W.i0[W.ev[sidx]] + W.li[sidx];
            W.obj[sidx] = mass_obj(ldf(pt, gi), ldf(eta, gi), ldf(phi, gi), ldf(mass, gi));
        }
        __syncwarp();
        // (C) pair terms, lane-parallel over the pairs
        for (int q = lane; q < n_pair; q += 32) {
            const int ow = owner_of(W.pincl, q);
            const int local = q - (W.pincl[ow] - choose2(W.cnt[ow]));
            const int xy = pair_tab[local];
            const int ob = W.obase[ow];
            W.pd[q] = pair_dot(W.obj[ob + (xy & 15)], W.obj[ob + (xy >> 4)]);
        }
        __syncwarp();
        // (D) triplets, 32 at a time
        const unsigned long long kInit = static_cast<unsigned long long>(0x7f800000u) << 32;
        unsigned long long best = kInit;
        const int my_texcl = tincl - (admit ? choose3(cnt) : 0);
        for (int chunk = 0; chunk < n_tri; chunk += 32) {
            const int t = chunk + lane;
            int ow = 32;
            unsigned long long key = ~0ull;
            if (t < n_tri) {
                ow = owner_of(W.tincl, t);
                const int r = t - (W.tincl[ow] - choose3(W.cnt[ow]));
                const int abc = tri_tab[r];
                const int a = abc & 15, b = (abc >> 4) & 15, c = abc >> 8;
                const int ob = W.obase[ow];
                const float* pd = W.pd + (W.pincl[ow] - choose2(W.cnt[ow]));
                const float pab = pd[choose2(b) + a], pac = pd[choose2(c) + a], pbc = pd[choose2(c) + b];
                const float ma = W.obj[ob + a].m, mb = W.obj[ob + b].m, mc = W.obj[ob + c].m;
                const float s3 = ma * ma + mb * mb + mc * mc;
                const float m = sqrtf(s3 + 2.0f * (pab + pac + pbc));
                const float d = fabsf(m - target);
                key = (static_cast<unsigned long long>(__float_as_uint(d)) << 32) |
                      static_cast<unsigned long long>((a << 8) | (b << 4) | c);
            }
            // segmented suffix minimum over lanes of the same event
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long other = __shfl_down_sync(0xffffffffu, key, o);
                const int other_ow = __shfl_down_sync(0xffffffffu, ow, o);
                if (lane + o < 32 && other_ow == ow && other < key) key = other;
            }
            // the owner takes the value of its first lane in this chunk
            const bool mine = admit && my_texcl < chunk + 32 && tincl > chunk;
            const int src = mine ? (my_texcl > chunk ? my_texcl - chunk : 0) : lane;
            const unsigned long long v = __shfl_sync(0xffffffffu, key, src);
            if (mine && v < best) best = v;
        }
        // outputs
        if (valid) {
            Closest res{__int_as_float(0x7fc00000), -1, -1, -1};
            if (admit) {
                if (best < kInit) {
                    const int a = static_cast<int>((best >> 8) & 15), b = static_cast<int>((best >> 4) & 15),
                              c = static_cast<int>(best & 15);
                    const float* pd = W.pd + (pincl - choose2(cnt));
                    const float pab = pd[choose2(b) + a], pac = pd[choose2(c) + a], pbc = pd[choose2(c) + b];
                    const float ma = W.obj[obase + a].m, mb = W.obj[obase + b].m, mc = W.obj[obase + c].m;
                    const float s3 = ma * ma + mb * mb + mc * mc;
                    res = Closest{sqrtf(s3 + 2.0f * (pab + pac + pbc)), W.li[obase + a], W.li[obase + b],
                                  W.li[obase + c]};
                }
            } else if (cnt >= 3) {
                res = closest_loop(pt, eta, phi, mass, i0, i1, mask_content, target);
            }
            if (out_mass) out_mass[e] = res.m;
            if (out_idx3) {
                out_idx3[3 * e] = res.a;
                out_idx3[3 * e + 1] = res.b;
                out_idx3[3 * e + 2] = res.c;
            }
        }
        __syncwarp();
    }
}

// select_opposite_sign_muons (Section III), lane = event: over masked-in
// objects in stored order, the first i with a later masked-in j of opposite
// charge, and the first such j; those two are kept, every other object of
// the event is masked out.
template <typename OffT>
__global__ void __launch_bounds__(kBlock) k_opposite_sign(const int8_t* charge, const OffT* off, int64_t n,
                                                          const uint8_t* mask_rows, const uint8_t* mask_in,
                                                          uint8_t* mask_out) {
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (mask_rows && !mask_rows[e]) continue;
        const int64_t i0 = ldoff(off, e), i1 = ldoff(off, e + 1);
        auto on = [&](int64_t i) { return mask_in == nullptr || mask_in[i] != 0; };
        int64_t a = -1, b = -1;
        for (int64_t i = i0; i < i1 && a < 0; ++i) {
            if (!on(i)) continue;
            const int qi = charge[i];
            for (int64_t j = i + 1; j < i1; ++j) {
                if (on(j) && qi * static_cast<int>(charge[j]) < 0) {
                    a = i;
                    b = j;
                    break;
                }
            }
        }
        for (int64_t i = i0; i < i1; ++i) mask_out[i] = (i == a || i == b) ? 1 : 0;
    }
}

// get_bin_contents (Section III), lane = element: the content of the value's
// bin, or the binary32 linear interpolation between the contents of the two
// neighbouring in-range bin centres c_b = (e[b-1] + e[b]) * 0.5 (clamped to
// the first and last centre), every operation rounded as written.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_bin_contents(const T* x, int64_t n, const float* __restrict__ edges,
                                                         int nb, const float* __restrict__ contents,
                                                         int interpolate, float* out) {
    const float e0 = __ldg(edges), en = __ldg(edges + nb);
    const float span = en - e0;
    const float invw = span > 0.0f ? static_cast<float>(nb) / span : 0.0f;
    auto centre = [&](int b) { return __fmul_rn(__fadd_rn(__ldg(edges + b - 1), __ldg(edges + b)), 0.5f); };
    for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < n;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float v = ldf(x, j);
        if (v != v) {
            out[j] = __int_as_float(0x7fc00000);
            continue;
        }
        if (!interpolate) {
            out[j] = __ldg(contents + find_bin(v, edges, nb, invw));
            continue;
        }
        if (nb == 1 || v < centre(1)) {
            out[j] = __ldg(contents + 1);
            continue;
        }
        if (v >= centre(nb)) {
            out[j] = __ldg(contents + nb);
            continue;
        }
        // the smallest b in [1, nb-1] with v < c_{b+1} (then c_b <= v)
        int lo = 1, hi = nb - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (v < centre(mid + 1))
                hi = mid;
            else
                lo = mid + 1;
        }
        const float cb = centre(lo), cb1 = centre(lo + 1);
        const float yb = __ldg(contents + lo), yb1 = __ldg(contents + lo + 1);
        const float t = __fdiv_rn(__fsub_rn(v, cb), __fsub_rn(cb1, cb));
        out[j] = __fadd_rn(yb, __fmul_rn(t, __fsub_rn(yb1, yb)));
    }
}

template <typename T, typename OffT>
__global__ void __launch_bounds__(kBlock) k_set(T* x, const OffT* off, int64_t n, const int32_t* nth, int32_t nth_scalar,
                                                const uint8_t* mask_rows, const uint8_t* mask_content, T value) {
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (mask_rows && !mask_rows[e]) continue;
        const int64_t want = nth ? nth[e] : nth_scalar;
        if (want < 0) continue;
        int64_t seen = 0;
        for (int64_t i = ldoff(off, e); i < ldoff(off, e + 1); ++i) {
            if (mask_content && !mask_content[i]) continue;
            if (seen == want) {
                x[i] = value;
                break;
            }
            ++seen;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_select(const T* x, int64_t n, float scale, float lo, float hi, int use_abs,
                                                   const uint8_t* min, uint8_t* mout) {
    for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < n;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        float v = __fmul_rn(ldf(x, j), scale);
        if (use_abs) v = fabsf(v);
        const bool in = min ? min[j] != 0 : true;
        mout[j] = (in && v > lo && v < hi) ? 1 : 0;
    }
}

// Vector forms of the elementwise kernels: each thread takes whole 16-byte
// chunks of the content (V = 16 / sizeof(T) elements) and the matching V
// bytes of the masks or 4 V bytes of the output, so that every load and
// store is as wide as the data allows; the last n % V elements go one by
// one. The host takes them when every pointer is aligned to its access.
template <int V> struct VBytes;
template <> struct VBytes<4> { using type = uint32_t; };
template <> struct VBytes<8> { using type = uint2; };
template <> struct VBytes<16> { using type = uint4; };

template <typename T>
__global__ void __launch_bounds__(kBlock) k_select_vec(const T* x, int64_t n, float scale, float lo, float hi,
                                                       int use_abs, const uint8_t* min, uint8_t* mout) {
    constexpr int V = 16 / static_cast<int>(sizeof(T));
    using MV = typename VBytes<V>::type;
    const int64_t nv = n / V;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t t0 = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    for (int64_t c = t0; c < nv; c += stride) {
        const uint4 raw = __ldg(reinterpret_cast<const uint4*>(x) + c);
        const T* v = reinterpret_cast<const T*>(&raw);
        MV inm;
        if (min) inm = __ldg(reinterpret_cast<const MV*>(min) + c);
        const uint8_t* in = reinterpret_cast<const uint8_t*>(&inm);
        MV o;
        uint8_t* ob = reinterpret_cast<uint8_t*>(&o);
#pragma unroll
        for (int i = 0; i < V; ++i) {
            float f = __fmul_rn(Elem<T>::f(v[i]), scale);
            if (use_abs) f = fabsf(f);
            ob[i] = ((!min || in[i] != 0) && f > lo && f < hi) ? 1 : 0;
        }
        reinterpret_cast<MV*>(mout)[c] = o;
    }
    for (int64_t j = nv * V + t0; j < n; j += stride) {
        float f = __fmul_rn(ldf(x, j), scale);
        if (use_abs) f = fabsf(f);
        mout[j] = ((!min || min[j] != 0) && f > lo && f < hi) ? 1 : 0;
    }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_scale_vec(const T* x, int64_t n, float s, float* out) {
    constexpr int V = 16 / static_cast<int>(sizeof(T));
    const int64_t nv = n / V;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t t0 = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    for (int64_t c = t0; c < nv; c += stride) {
        const uint4 raw = __ldg(reinterpret_cast<const uint4*>(x) + c);
        const T* v = reinterpret_cast<const T*>(&raw);
        float4* o = reinterpret_cast<float4*>(out + c * V);
#pragma unroll
        for (int q = 0; q < V / 4; ++q)
            o[q] = make_float4(__fmul_rn(Elem<T>::f(v[4 * q]), s), __fmul_rn(Elem<T>::f(v[4 * q + 1]), s),
                               __fmul_rn(Elem<T>::f(v[4 * q + 2]), s), __fmul_rn(Elem<T>::f(v[4 * q + 3]), s));
    }
    for (int64_t j = nv * V + t0; j < n; j += stride) out[j] = __fmul_rn(ldf(x, j), s);
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_scale(const T* x, int64_t n, float s, float* out) {
    for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < n;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x)
        out[j] = __fmul_rn(ldf(x, j), s);
}

// ---------------------------------------------------------------------------
// Exact weighted sums with integer arithmetic. A finite binary32 value is
// m 2^(e-150) (e its biased exponent, m its 24-bit significand; e = 1 and no
// implicit bit for subnormals), i.e. x 2^(8 (e >> 3) - 150) with the integer
// x = m << (e & 7) < 2^31. The accumulator of exponent group e >> 3 adds the
// low 16 bits and the high 15 bits of +-x in two int32 words (shared-memory
// int32 atomics are fast, int64 ones are not); a launch gives each block at
// most 2^15 elements, so neither word can overflow and the block's sums are
// exact until each group is converted to binary64 once, at the end. The
// binary64 pipe (narrow on this part) does no per-element work. w^2 enters
// exactly as p + q with p = fl(w w) and q = w w - p from a fused
// multiply-add. Weights outside [2^-50, 2^63) in magnitude (where p or q
// could leave the binary32 range), infinities and NaNs go to the global
// binary64 sums directly.
// ---------------------------------------------------------------------------
constexpr int kWG = 15;      // groups of w: |w| in [2^-50, 2^63) has e in [77, 189], groups 9..23
constexpr int kWG0 = 9;
constexpr int kW2G = 32;     // groups of p and q: every finite binary32 value
// words per bin: odd, so that lanes on different bins and the same group
// fall in different shared-memory banks
constexpr int kWS = 2 * kWG + 1;
constexpr int kW2S = 2 * kW2G + 1;
constexpr int64_t kExactPerBlock = int64_t(1) << 15;
constexpr size_t kExactSmemMax = 96 * 1024;   // two blocks per SM

__device__ __forceinline__ bool exact_weight(float w) {
    const uint32_t e = (__float_as_uint(w) >> 23) & 0xffu;
    return w == 0.0f || (e >= 77u && e <= 189u);
}

// adds the finite binary32 value v to the int32 word pairs acc (group 0 of
// acc is exponent group g0)
__device__ __forceinline__ void exact_put(float v, int* acc, int g0) {
    const uint32_t bits = __float_as_uint(v);
    uint32_t e = (bits >> 23) & 0xffu;
    uint32_t m = bits & 0x7fffffu;
    if (e) m |= 0x800000u;
    else e = 1u;
    const uint32_t x = m << (e & 7u);
    int lo = static_cast<int>(x & 0xffffu), hi = static_cast<int>(x >> 16);
    if (bits >> 31) {
        lo = -lo;
        hi = -hi;
    }
    int* a = acc + 2 * (static_cast<int>(e >> 3) - g0);
    atomicAdd(a, lo);
    atomicAdd(a + 1, hi);
}

// Adds weight w of one element of bin/cell c to the block's accumulators (or
// to the global sums when w is outside the exact range).
__device__ __forceinline__ void exact_add(int c, float w, int* s_w, int* s_w2, double* sumw, double* sumw2) {
    if (!exact_weight(w)) {
        const double wd = static_cast<double>(w);
        if (sumw) atomicAdd(&sumw[c], wd);
        if (sumw2) atomicAdd(&sumw2[c], wd * wd);
        return;
    }
    if (w == 0.0f) return;
    if (s_w) exact_put(w, s_w + kWS * c, kWG0);
    if (s_w2) {
        const float p = __fmul_rn(w, w);
        const float q = __fmaf_rn(w, w, -p);
        exact_put(p, s_w2 + kW2S * c, 0);
        if (q != 0.0f) exact_put(q, s_w2 + kW2S * c, 0);
    }
}

// binary64 value of one bin's groups (first group g0, ng groups)
__device__ __forceinline__ double exact_value(const int* acc, int g0, int ng) {
    double s = 0.0;
    for (int g = 0; g < ng; ++g) {
        const long long a = static_cast<long long>(acc[2 * g]) + (static_cast<long long>(acc[2 * g + 1]) << 16);
        if (a == 0) continue;
        const double unit = __longlong_as_double(static_cast<long long>(1023 + 8 * (g0 + g) - 150) << 52);
        s += __ll2double_rn(a) * unit;
    }
    return s;
}

// Shared memory of the exact-sum kernels: int32 word pairs of w and w^2 per
// bin and group (kWS, kW2S words per bin), then u32 counts (then the edges for the one-variable kernel).
inline size_t exact_smem(int64_t nbin, bool with_w, bool with_w2) {
    return static_cast<size_t>(nbin) * ((with_w ? kWS * 4 : 0) + (with_w2 ? kW2S * 4 : 0) + 4);
}

__device__ __forceinline__ void exact_layout(unsigned char* smem, int nbin, bool with_w, bool with_w2, int*& s_w,
                                             int*& s_w2, unsigned int*& s_c) {
    int* p = reinterpret_cast<int*>(smem);
    s_w2 = with_w2 ? p : nullptr;
    p += with_w2 ? static_cast<size_t>(nbin) * kW2S : 0;
    s_w = with_w ? p : nullptr;
    p += with_w ? static_cast<size_t>(nbin) * kWS : 0;
    s_c = reinterpret_cast<unsigned int*>(p);
}

__device__ __forceinline__ void exact_zero(int nbin, int* s_w, int* s_w2, unsigned int* s_c) {
    for (int i = threadIdx.x; i < nbin; i += blockDim.x) s_c[i] = 0u;
    if (s_w)
        for (int i = threadIdx.x; i < nbin * kWS; i += blockDim.x) s_w[i] = 0;
    if (s_w2)
        for (int i = threadIdx.x; i < nbin * kW2S; i += blockDim.x) s_w2[i] = 0;
}

__device__ __forceinline__ void exact_merge(int nbin, const int* s_w, const int* s_w2, const unsigned int* s_c,
                                            unsigned long long* counts, double* sumw, double* sumw2) {
    for (int i = threadIdx.x; i < nbin; i += blockDim.x) {
        if (s_c[i] == 0u) continue;
        atomicAdd(&counts[i], static_cast<unsigned long long>(s_c[i]));
        if (s_w) atomicAdd(&sumw[i], exact_value(s_w + kWS * i, kWG0, kWG));
        if (s_w2) atomicAdd(&sumw2[i], exact_value(s_w2 + kW2S * i, 0, kW2G));
    }
}

// fill_histogram with a block-private histogram in shared memory and exact
// integer weighted sums (see above); lanes add their own element.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_hist_exact(const T* x, const float* w, const uint8_t* mask, int64_t n,
                                                       const float* edges, int nb, unsigned long long* counts,
                                                       double* sumw, double* sumw2) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int nbin = nb + 2;
    int *s_w, *s_w2;
    unsigned int* s_c;
    exact_layout(smem, nbin, sumw != nullptr, sumw2 != nullptr, s_w, s_w2, s_c);
    float* s_e = reinterpret_cast<float*>(s_c + nbin);
    exact_zero(nbin, s_w, s_w2, s_c);
    for (int i = threadIdx.x; i <= nb; i += blockDim.x) s_e[i] = edges[i];
    __syncthreads();
    const float span = s_e[nb] - s_e[0];
    const float inv_width = span > 0.0f ? static_cast<float>(nb) / span : 0.0f;
    for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < n;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (mask && !mask[j]) continue;
        const int b = find_bin(ldf(x, j), s_e, nb, inv_width);
        if (b < 0) continue;
        atomicAdd(&s_c[b], 1u);
        exact_add(b, w ? w[j] : 1.0f, s_w, s_w2, sumw, sumw2);
    }
    __syncthreads();
    exact_merge(nbin, s_w, s_w2, s_c, counts, sumw, sumw2);
}

// fill_histogram with a block-private copy of the histogram in shared memory:
// edges, u32 counts, f64 sums. Lanes that hit the same bin are merged first
// (__match_any_sync) so one lane per bin does the shared-memory atomics; the
// block adds its histogram to global memory at the end.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_hist_smem(const T* x, const float* w, const uint8_t* mask, int64_t n,
                                                      const float* edges, int nb,
                                                      unsigned long long* counts, double* sumw, double* sumw2) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int nbin = nb + 2;
    double* s_w = reinterpret_cast<double*>(smem);
    double* s_w2 = s_w + nbin;
    double* s_lane = s_w2 + nbin;
    unsigned int* s_c = reinterpret_cast<unsigned int*>(s_lane + blockDim.x);
    float* s_e = reinterpret_cast<float*>(s_c + nbin);
    for (int i = threadIdx.x; i < nbin; i += blockDim.x) {
        s_w[i] = 0.0;
        s_w2[i] = 0.0;
        s_c[i] = 0u;
    }
    for (int i = threadIdx.x; i <= nb; i += blockDim.x) s_e[i] = edges[i];
    __syncthreads();
    const float span = s_e[nb] - s_e[0];
    const float inv_width = span > 0.0f ? static_cast<float>(nb) / span : 0.0f;
    const int lane = threadIdx.x & 31;
    double* my = s_lane + (threadIdx.x & ~31);
    const int64_t step = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t base = static_cast<int64_t>(blockIdx.x) * blockDim.x + (threadIdx.x & ~31); base < n; base += step) {
        const int64_t j = base + lane;
        int b = -1;
        double ww = 0.0;
        if (j < n && (!mask || mask[j])) {
            b = find_bin(ldf(x, j), s_e, nb, inv_width);
            ww = w ? static_cast<double>(w[j]) : 1.0;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        my[lane] = ww;
        __syncwarp();
        if (b >= 0 && lane == __ffs(peers) - 1) {
            double sw = 0.0, sw2 = 0.0;
            for (unsigned m = peers; m; m &= m - 1) {
                const double q = my[__ffs(m) - 1];
                sw += q;
                sw2 += q * q;
            }
            atomicAdd(&s_c[b], static_cast<unsigned>(__popc(peers)));
            if (sumw) atomicAdd(&s_w[b], sw);
            if (sumw2) atomicAdd(&s_w2[b], sw2);
        }
        __syncwarp();
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nbin; i += blockDim.x) {
        if (s_c[i] == 0u) continue;
        atomicAdd(&counts[i], static_cast<unsigned long long>(s_c[i]));
        if (sumw) atomicAdd(&sumw[i], s_w[i]);
        if (sumw2) atomicAdd(&sumw2[i], s_w2[i]);
    }
}

// fill_histogram straight into global memory (histograms too large for
// shared memory).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_hist_global(const T* x, const float* w, const uint8_t* mask, int64_t n,
                                                        const float* edges, int nb,
                                                        unsigned long long* counts, double* sumw, double* sumw2) {
    const float span = edges[nb] - edges[0];
    const float inv_width = span > 0.0f ? static_cast<float>(nb) / span : 0.0f;
    for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < n;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (mask && !mask[j]) continue;
        const int b = find_bin(ldf(x, j), edges, nb, inv_width);
        if (b < 0) continue;
        const double ww = w ? static_cast<double>(w[j]) : 1.0;
        atomicAdd(&counts[b], 1ull);
        if (sumw) atomicAdd(&sumw[b], ww);
        if (sumw2) atomicAdd(&sumw2[b], ww * ww);
    }
}

// Several variables: the axes' columns, edges and sizes (HEPACC_MAX_HIST_DIMS
// at most), passed by value.
struct HistAxes {
    const void* x[HEPACC_MAX_HIST_DIMS];
    const float* e[HEPACC_MAX_HIST_DIMS];
    int dt[HEPACC_MAX_HIST_DIMS];
    int nb[HEPACC_MAX_HIST_DIMS];
    int ndim;
};

// Element j of a column whose type is known only at run time.
__device__ __forceinline__ float ld_any(const void* p, int dt, int64_t j) {
    switch (dt) {
        case HEPACC_F32: return __ldg(static_cast<const float*>(p) + j);
        case HEPACC_F16: return __half2float(static_cast<const __half*>(p)[j]);
        case HEPACC_BF16: return __bfloat162float(static_cast<const __nv_bfloat16*>(p)[j]);
        case HEPACC_U8: return static_cast<float>(static_cast<const uint8_t*>(p)[j]);
        case HEPACC_I8: return static_cast<float>(static_cast<const int8_t*>(p)[j]);
        default: return static_cast<float>(__ldg(static_cast<const int32_t*>(p) + j));
    }
}

// Row-major cell of element j over the axes (axis 0 slowest), -1 for a NaN
// on any axis.
__device__ __forceinline__ int64_t cell_of(const HistAxes& a, const float (&inv_w)[HEPACC_MAX_HIST_DIMS], int64_t j) {
    int64_t at = 0;
#pragma unroll
    for (int d = 0; d < HEPACC_MAX_HIST_DIMS; ++d) {
        if (d >= a.ndim) break;
        const int b = find_bin(ld_any(a.x[d], a.dt[d], j), a.e[d], a.nb[d], inv_w[d]);
        if (b < 0) return -1;
        at = at * (a.nb[d] + 2) + b;
    }
    return at;
}

__device__ __forceinline__ void axis_widths(const HistAxes& a, float (&inv_w)[HEPACC_MAX_HIST_DIMS]) {
#pragma unroll
    for (int d = 0; d < HEPACC_MAX_HIST_DIMS; ++d) {
        inv_w[d] = 0.0f;
        if (d < a.ndim) {
            const float span = __ldg(a.e[d] + a.nb[d]) - __ldg(a.e[d]);
            inv_w[d] = span > 0.0f ? static_cast<float>(a.nb[d]) / span : 0.0f;
        }
    }
}

// fill_histogram_nd with a block-private histogram in shared memory (u32
// counts, f64 sums; edges read through the read-only cache). Lanes of a warp
// that hit the same cell are merged first, as in k_hist_smem.
__global__ void __launch_bounds__(kBlock) k_hist_nd_smem(const __grid_constant__ HistAxes a, const float* w,
                                                         const uint8_t* mask, int64_t n, int ncell,
                                                         unsigned long long* counts, double* sumw, double* sumw2) {
    extern __shared__ __align__(16) unsigned char smem[];
    double* s_w = reinterpret_cast<double*>(smem);
    double* s_w2 = s_w + ncell;
    double* s_lane = s_w2 + ncell;
    unsigned int* s_c = reinterpret_cast<unsigned int*>(s_lane + blockDim.x);
    for (int i = threadIdx.x; i < ncell; i += blockDim.x) {
        s_w[i] = 0.0;
        s_w2[i] = 0.0;
        s_c[i] = 0u;
    }
    float inv_w[HEPACC_MAX_HIST_DIMS];
    axis_widths(a, inv_w);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    double* my = s_lane + (threadIdx.x & ~31);
    const int64_t step = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t base = static_cast<int64_t>(blockIdx.x) * blockDim.x + (threadIdx.x & ~31); base < n; base += step) {
        const int64_t j = base + lane;
        int c = -1;
        double ww = 0.0;
        if (j < n && (!mask || mask[j])) {
            c = static_cast<int>(cell_of(a, inv_w, j));
            ww = w ? static_cast<double>(w[j]) : 1.0;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, c);
        my[lane] = ww;
        __syncwarp();
        if (c >= 0 && lane == __ffs(peers) - 1) {
            double sw = 0.0, sw2 = 0.0;
            for (unsigned m = peers; m; m &= m - 1) {
                const double q = my[__ffs(m) - 1];
                sw += q;
                sw2 += q * q;
            }
            atomicAdd(&s_c[c], static_cast<unsigned>(__popc(peers)));
            if (sumw) atomicAdd(&s_w[c], sw);
            if (sumw2) atomicAdd(&s_w2[c], sw2);
        }
        __syncwarp();
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ncell; i += blockDim.x) {
        if (s_c[i] == 0u) continue;
        atomicAdd(&counts[i], static_cast<unsigned long long>(s_c[i]));
        if (sumw) atomicAdd(&sumw[i], s_w[i]);
        if (sumw2) atomicAdd(&sumw2[i], s_w2[i]);
    }
}

// fill_histogram_nd straight into global memory (more cells than fit in
// shared memory).
__global__ void __launch_bounds__(kBlock) k_hist_nd_global(const __grid_constant__ HistAxes a, const float* w,
                                                           const uint8_t* mask, int64_t n, unsigned long long* counts,
                                                           double* sumw, double* sumw2) {
    float inv_w[HEPACC_MAX_HIST_DIMS];
    axis_widths(a, inv_w);
    for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < n;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (mask && !mask[j]) continue;
        const int64_t c = cell_of(a, inv_w, j);
        if (c < 0) continue;
        const double ww = w ? static_cast<double>(w[j]) : 1.0;
        atomicAdd(&counts[c], 1ull);
        if (sumw) atomicAdd(&sumw[c], ww);
        if (sumw2) atomicAdd(&sumw2[c], ww * ww);
    }
}

// fill_histogram_nd with a block-private histogram and exact integer sums.
__global__ void __launch_bounds__(kBlock) k_hist_nd_exact(const __grid_constant__ HistAxes a, const float* w,
                                                          const uint8_t* mask, int64_t n, int ncell,
                                                          unsigned long long* counts, double* sumw, double* sumw2) {
    extern __shared__ __align__(16) unsigned char smem[];
    int *s_w, *s_w2;
    unsigned int* s_c;
    exact_layout(smem, ncell, sumw != nullptr, sumw2 != nullptr, s_w, s_w2, s_c);
    exact_zero(ncell, s_w, s_w2, s_c);
    float inv_w[HEPACC_MAX_HIST_DIMS];
    axis_widths(a, inv_w);
    __syncthreads();
    for (int64_t j = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; j < n;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (mask && !mask[j]) continue;
        const int c = static_cast<int>(cell_of(a, inv_w, j));
        if (c < 0) continue;
        atomicAdd(&s_c[c], 1u);
        exact_add(c, w ? w[j] : 1.0f, s_w, s_w2, sumw, sumw2);
    }
    __syncthreads();
    exact_merge(ncell, s_w, s_w2, s_c, counts, sumw, sumw2);
}

template <typename OffT>
__global__ void k_validate(const OffT* off, int64_t n, int64_t m, unsigned long long* first_bad) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t a = ldoff(off, i), b = ldoff(off, i + 1);
        if (b < a || (i + 1 == n && b > m)) atomicMin(first_bad, static_cast<unsigned long long>(i));
    }
}

// Offsets check that reports through the device error word: bit 1 when
// offsets[0] < 0, the offsets decrease anywhere, or offsets[n] > m (the
// content length).
template <typename OffT>
__global__ void k_check_offsets(const OffT* off, int64_t n, int64_t m) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t a = ldoff(off, i), b = ldoff(off, i + 1);
        if (b < a || (i == 0 && a < 0) || (i + 1 == n && b > m)) atomicOr(&g_device_error, kErrCheck);
    }
}

// One thread waits on an mbarrier that is never completed (bounded wait).
__global__ void k_wait_timeout(long long limit_cycles) {
    __shared__ uint64_t bar;
    const uint32_t b = smem_addr(&bar);
    mbar_init(b, 1);
    fence_mbar_init();
    mbar_wait_bounded(b, 0, limit_cycles);
}

__global__ void k_validate_init(const void* off, int ot64, unsigned long long* first_bad) {
    *first_bad = ~0ull;
    const int64_t o0 = ot64 ? *static_cast<const int64_t*>(off) : *static_cast<const int32_t*>(off);
    if (o0 < 0) *first_bad = ~0ull - 1;
}

__global__ void k_validate_fini(unsigned long long* first_bad) {
    const unsigned long long v = *first_bad;
    long long r;
    if (v == ~0ull) r = -1;
    else if (v == ~0ull - 1) r = -2;
    else r = static_cast<long long>(v);
    *reinterpret_cast<long long*>(first_bad) = r;
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------

struct LaunchCache {
    std::mutex mu;
    std::unordered_map<const void*, int> smem_set;   // kernel -> dynamic smem attribute set
};
LaunchCache& cache() {
    static LaunchCache c;
    return c;
}

// Sets the kernel's dynamic shared memory limit once and returns the grid
// size for `work` warp tiles (persistent: at most resident blocks x SMs).
template <typename K>
hepacc_status tile_grid(K kernel, size_t smem, int64_t ntiles, int* grid) {
    const DeviceInfo di = device_info();
    if (smem > static_cast<size_t>(di.smem_optin)) return fail(HEPACC_ERR_INVALID_ARG, "stage buffers exceed shared memory");
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
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, smem);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
    if (per_sm < 1) per_sm = 1;
    const int64_t want = (ntiles + (kBlock / 32) - 1) / (kBlock / 32);
    *grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(want, static_cast<int64_t>(per_sm) * di.sms)));
    return HEPACC_OK;
}

inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

inline int flat_grid(int64_t n) {
    const DeviceInfo di = device_info();
    const int64_t want = (n + kBlock - 1) / kBlock;
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(want, static_cast<int64_t>(di.sms) * 8)));
}

struct SpecBuilder {
    Spec s{};
    uint32_t off = 0;
    SpecBuilder() { s.ncol = 0; }
    void add(const void* base, size_t es, int coll, int cap_elems = 0) {
        ColSpec& c = s.col[s.ncol++];
        c.base = static_cast<const unsigned char*>(base);
        c.es = static_cast<uint32_t>(es);
        c.coll = static_cast<uint32_t>(coll);
        c.cap = base ? static_cast<uint32_t>((cap_elems * es + 32 + 15) & ~size_t(15)) : 0u;
        c.soff = off;
        off += c.cap;
    }
    Spec done() {
        s.buf_bytes = (off + 127) & ~uint32_t(127);
        if (s.buf_bytes == 0) s.buf_bytes = 128;
        return s;
    }
};

#define HEPACC_CHECK(cond, ...) \
    do {                        \
        if (!(cond)) return fail(HEPACC_ERR_INVALID_ARG, __VA_ARGS__); \
    } while (0)

// Calls f(tag) with tag's ::type set to the C++ type of dtype t.
template <typename T> struct Tag { using type = T; };

template <typename F>
hepacc_status with_float_type(hepacc_dtype t, F&& f) {
    switch (t) {
        case HEPACC_F32: return f(Tag<float>{});
        case HEPACC_F16: return f(Tag<__half>{});
        case HEPACC_BF16: return f(Tag<__nv_bfloat16>{});
        default: return fail(HEPACC_ERR_DTYPE, "expected a floating content type (F32, F16, BF16)");
    }
}

template <typename F>
hepacc_status with_value_type(hepacc_dtype t, F&& f) {
    switch (t) {
        case HEPACC_F32: return f(Tag<float>{});
        case HEPACC_F16: return f(Tag<__half>{});
        case HEPACC_BF16: return f(Tag<__nv_bfloat16>{});
        case HEPACC_U8: return f(Tag<uint8_t>{});
        case HEPACC_I8: return f(Tag<int8_t>{});
        case HEPACC_I32: return f(Tag<int32_t>{});
        default: return fail(HEPACC_ERR_DTYPE, "unsupported content type");
    }
}

template <typename F>
hepacc_status with_offsets_type(hepacc_dtype t, F&& f) {
    switch (t) {
        case HEPACC_I32: return f(Tag<int32_t>{});
        case HEPACC_I64: return f(Tag<int64_t>{});
        default: return fail(HEPACC_ERR_DTYPE, "offsets must be I32 or I64");
    }
}

// Kernels on event_loop: no shared memory, one thread per event at a time.
template <typename K, typename... Args>
hepacc_status launch_flat(K kernel, const Spec& spec, int64_t n, cudaStream_t stream, Args... args) {
    kernel<<<flat_grid(n), kBlock, 0, stream>>>(spec, args...);
    HEPACC_CHECK_LAUNCH("kernel launch");
    return HEPACC_OK;
}


}  // namespace
}  // namespace hepacc

using namespace hepacc;

extern "C" {

hepacc_status hepacc_sum_in_offsets(const void* content, hepacc_dtype ct, const void* offsets, hepacc_dtype ot,
                                    int64_t n, const uint8_t* mask_rows, const uint8_t* mask_content, void* out,
                                    hepacc_dtype out_t, hepacc_stream stream) {
    HEPACC_CHECK(n >= 0, "n_rows < 0");
    if (n == 0) return HEPACC_OK;
    HEPACC_CHECK(content && offsets && out, "content, offsets and out are required");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    return with_offsets_type(ot, [&](auto ot_tag) -> hepacc_status {
        using O = typename decltype(ot_tag)::type;
        const O* off = static_cast<const O*>(offsets);
        SpecBuilder b;
        if (is_float_type(ct)) {
            if (out_t != HEPACC_F32) return fail(HEPACC_ERR_DTYPE, "floating content sums into F32");
            return with_float_type(ct, [&](auto t) -> hepacc_status {
                using T = typename decltype(t)::type;
                b.add(content, sizeof(T), 0);
                b.add(mask_content, 1, 0);
                return launch_flat(k_sum<T, O, float>, b.done(), n, s, off, n, mask_rows, static_cast<float*>(out));
            });
        }
        auto run_int = [&](auto t) -> hepacc_status {
            using T = typename decltype(t)::type;
            b.add(content, sizeof(T), 0);
            b.add(mask_content, 1, 0);
            if (out_t == HEPACC_I64)
                return launch_flat(k_sum<T, O, int64_t>, b.done(), n, s, off, n, mask_rows, static_cast<int64_t*>(out));
            if (out_t == HEPACC_I32 && ct != HEPACC_I64)
                return launch_flat(k_sum<T, O, int32_t>, b.done(), n, s, off, n, mask_rows, static_cast<int32_t*>(out));
            return fail(HEPACC_ERR_DTYPE, "integer content sums into I32 or I64 (I64 content: I64)");
        };
        switch (ct) {
            case HEPACC_U8: return run_int(Tag<uint8_t>{});
            case HEPACC_I8: return run_int(Tag<int8_t>{});
            case HEPACC_I32: return run_int(Tag<int32_t>{});
            case HEPACC_I64: return run_int(Tag<int64_t>{});
            default: return fail(HEPACC_ERR_DTYPE, "unsupported content type");
        }
    });
}

static hepacc_status minmax_impl(bool is_max, const void* content, hepacc_dtype ct, const void* offsets,
                                 hepacc_dtype ot, int64_t n, const uint8_t* mask_rows, const uint8_t* mask_content,
                                 float empty, float* out, int32_t* arg, hepacc_stream stream) {
    HEPACC_CHECK(n >= 0, "n_rows < 0");
    if (n == 0) return HEPACC_OK;
    HEPACC_CHECK(content && offsets && (out || arg), "content, offsets and an output are required");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    return with_offsets_type(ot, [&](auto ot_tag) -> hepacc_status {
        using O = typename decltype(ot_tag)::type;
        return with_value_type(ct, [&](auto t) -> hepacc_status {
            using T = typename decltype(t)::type;
            SpecBuilder b;
            b.add(content, sizeof(T), 0);
            b.add(mask_content, 1, 0);
            if (is_max)
                return launch_flat(k_minmax<T, O, true>, b.done(), n, s, static_cast<const O*>(offsets), n, mask_rows,
                                    empty, out, arg);
            return launch_flat(k_minmax<T, O, false>, b.done(), n, s, static_cast<const O*>(offsets), n, mask_rows,
                                empty, out, arg);
        });
    });
}

hepacc_status hepacc_max_in_offsets(const void* content, hepacc_dtype ct, const void* offsets, hepacc_dtype ot,
                                    int64_t n, const uint8_t* mask_rows, const uint8_t* mask_content, float empty,
                                    float* out, int32_t* arg, hepacc_stream stream) {
    return minmax_impl(true, content, ct, offsets, ot, n, mask_rows, mask_content, empty, out, arg, stream);
}

hepacc_status hepacc_min_in_offsets(const void* content, hepacc_dtype ct, const void* offsets, hepacc_dtype ot,
                                    int64_t n, const uint8_t* mask_rows, const uint8_t* mask_content, float empty,
                                    float* out, int32_t* arg, hepacc_stream stream) {
    return minmax_impl(false, content, ct, offsets, ot, n, mask_rows, mask_content, empty, out, arg, stream);
}

hepacc_status hepacc_get_in_offsets(const void* content, hepacc_dtype ct, const void* offsets, hepacc_dtype ot,
                                    int64_t n, const int32_t* nth, int32_t nth_scalar, const uint8_t* mask_rows,
                                    const uint8_t* mask_content, float dflt, float* out, int32_t* oidx,
                                    hepacc_stream stream) {
    HEPACC_CHECK(n >= 0, "n_rows < 0");
    if (n == 0) return HEPACC_OK;
    HEPACC_CHECK(content && offsets && (out || oidx), "content, offsets and an output are required");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    return with_offsets_type(ot, [&](auto ot_tag) -> hepacc_status {
        using O = typename decltype(ot_tag)::type;
        return with_value_type(ct, [&](auto t) -> hepacc_status {
            using T = typename decltype(t)::type;
            SpecBuilder b;
            b.add(content, sizeof(T), 0);
            b.add(mask_content, 1, 0);
            return launch_flat(k_get<T, O>, b.done(), n, s, static_cast<const O*>(offsets), n, nth, nth_scalar,
                                mask_rows, dflt, out, oidx);
        });
    });
}

hepacc_status hepacc_set_in_offsets(void* content, hepacc_dtype ct, const void* offsets, hepacc_dtype ot, int64_t n,
                                    const int32_t* nth, int32_t nth_scalar, const uint8_t* mask_rows,
                                    const uint8_t* mask_content, double value, hepacc_stream stream) {
    HEPACC_CHECK(n >= 0, "n_rows < 0");
    if (n == 0) return HEPACC_OK;
    HEPACC_CHECK(content && offsets, "content and offsets are required");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    return with_offsets_type(ot, [&](auto ot_tag) -> hepacc_status {
        using O = typename decltype(ot_tag)::type;
        const O* off = static_cast<const O*>(offsets);
        if (ct == HEPACC_U8) {
            k_set<uint8_t, O><<<flat_grid(n), kBlock, 0, s>>>(static_cast<uint8_t*>(content), off, n, nth, nth_scalar,
                                                              mask_rows, mask_content, static_cast<uint8_t>(value));
        } else if (ct == HEPACC_F32) {
            k_set<float, O><<<flat_grid(n), kBlock, 0, s>>>(static_cast<float*>(content), off, n, nth, nth_scalar,
                                                            mask_rows, mask_content, static_cast<float>(value));
        } else {
            return fail(HEPACC_ERR_DTYPE, "set_in_offsets content must be U8 or F32");
        }
        HEPACC_CHECK_LAUNCH("set_in_offsets launch");
        return HEPACC_OK;
    });
}

hepacc_status hepacc_select_range(const void* content, hepacc_dtype ct, int64_t n, float scale, float lo, float hi,
                                  int use_abs, const uint8_t* mask_in, uint8_t* mask_out, hepacc_stream stream) {
    HEPACC_CHECK(n >= 0, "n < 0");
    if (n == 0) return HEPACC_OK;
    HEPACC_CHECK(content && mask_out, "content and mask_out are required");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    return with_value_type(ct, [&](auto t) -> hepacc_status {
        using T = typename decltype(t)::type;
        constexpr int V = 16 / static_cast<int>(sizeof(T));
        const bool vec = aligned(content, 16) && aligned(mask_out, V) && (!mask_in || aligned(mask_in, V));
        if (vec)
            k_select_vec<T><<<flat_grid((n + V - 1) / V), kBlock, 0, s>>>(static_cast<const T*>(content), n, scale, lo,
                                                                          hi, use_abs, mask_in, mask_out);
        else
            k_select<T><<<flat_grid(n), kBlock, 0, s>>>(static_cast<const T*>(content), n, scale, lo, hi, use_abs,
                                                        mask_in, mask_out);
        HEPACC_CHECK_LAUNCH("select_range launch");
        return HEPACC_OK;
    });
}

hepacc_status hepacc_scale(const void* content, hepacc_dtype ct, int64_t n, float scale, float* out,
                           hepacc_stream stream) {
    HEPACC_CHECK(n >= 0, "n < 0");
    if (n == 0) return HEPACC_OK;
    HEPACC_CHECK(content && out, "content and out are required");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    return with_float_type(ct, [&](auto t) -> hepacc_status {
        using T = typename decltype(t)::type;
        constexpr int V = 16 / static_cast<int>(sizeof(T));
        if (aligned(content, 16) && aligned(out, 16))
            k_scale_vec<T><<<flat_grid((n + V - 1) / V), kBlock, 0, s>>>(static_cast<const T*>(content), n, scale, out);
        else
            k_scale<T><<<flat_grid(n), kBlock, 0, s>>>(static_cast<const T*>(content), n, scale, out);
        HEPACC_CHECK_LAUNCH("scale launch");
        return HEPACC_OK;
    });
}

hepacc_status hepacc_mask_deltar(const void* eta1, const void* phi1, hepacc_dtype t1, const void* off1,
                                 const void* eta2, const void* phi2, hepacc_dtype t2, const void* off2,
                                 hepacc_dtype ot, int64_t n, const uint8_t* mask_rows, const uint8_t* mask1_in,
                                 const uint8_t* mask2, float dr2_cut, uint8_t* mask1_out, hepacc_stream stream) {
    HEPACC_CHECK(n >= 0, "n_rows < 0");
    if (n == 0) return HEPACC_OK;
    HEPACC_CHECK(eta1 && phi1 && off1 && eta2 && phi2 && off2 && mask1_out, "missing required pointer");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    return with_offsets_type(ot, [&](auto ot_tag) -> hepacc_status {
        using O = typename decltype(ot_tag)::type;
        return with_float_type(t1, [&](auto a) -> hepacc_status {
            using T1 = typename decltype(a)::type;
            return with_float_type(t2, [&](auto b2) -> hepacc_status {
                using T2 = typename decltype(b2)::type;
                SpecBuilder b;
                b.add(eta1, sizeof(T1), 0);
                b.add(phi1, sizeof(T1), 0);
                b.add(mask1_in, 1, 0);
                b.add(eta2, sizeof(T2), 1, 256);
                b.add(phi2, sizeof(T2), 1, 256);
                b.add(mask2, 1, 1, 256);
                return launch_flat(k_deltar<T1, T2, O>, b.done(), n, s, static_cast<const O*>(off1),
                                    static_cast<const O*>(off2), n, mask_rows, dr2_cut, mask1_out);
            });
        });
    });
}

hepacc_status hepacc_pair_mass(const void* pt, const void* eta, const void* phi, const void* mass, hepacc_dtype t,
                               const void* offsets, hepacc_dtype ot, int64_t n, const int32_t* ia, const int32_t* ib,
                               const uint8_t* mask_rows, float* out, hepacc_stream stream) {
    HEPACC_CHECK(n >= 0, "n_rows < 0");
    if (n == 0) return HEPACC_OK;
    HEPACC_CHECK(pt && eta && phi && mass && offsets && ia && ib && out, "missing required pointer");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    return with_offsets_type(ot, [&](auto ot_tag) -> hepacc_status {
        using O = typename decltype(ot_tag)::type;
        return with_float_type(t, [&](auto tt) -> hepacc_status {
            using T = typename decltype(tt)::type;
            k_pair_mass<T, O><<<flat_grid(n), kBlock, 0, s>>>(
                static_cast<const T*>(pt), static_cast<const T*>(eta), static_cast<const T*>(phi),
                static_cast<const T*>(mass), static_cast<const O*>(offsets), n, ia, ib, mask_rows, out);
            HEPACC_CHECK_LAUNCH("pair_mass launch");
            return HEPACC_OK;
        });
    });
}

hepacc_status hepacc_max_pt_trijet(const void* pt, const void* eta, const void* phi, const void* mass,
                                   hepacc_dtype t, const void* offsets, hepacc_dtype ot, int64_t n,
                                   const uint8_t* mask_rows, const uint8_t* mask_content, float* out_mass,
                                   float* out_pt, int32_t* out_idx3, hepacc_stream stream) {
    HEPACC_CHECK(n >= 0, "n_rows < 0");
    if (n == 0) return HEPACC_OK;
    HEPACC_CHECK(pt && eta && phi && mass && offsets, "missing required pointer");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    return with_offsets_type(ot, [&](auto ot_tag) -> hepacc_status {
        using O = typename decltype(ot_tag)::type;
        return with_float_type(t, [&](auto tt) -> hepacc_status {
            using T = typename decltype(tt)::type;
            SpecBuilder b;
            b.add(pt, sizeof(T), 0);
            b.add(eta, sizeof(T), 0);
            b.add(phi, sizeof(T), 0);
            b.add(mass, sizeof(T), 0);
            b.add(mask_content, 1, 0);
            return launch_flat(k_trijet<T, O>, b.done(), n, s, static_cast<const O*>(offsets), n, mask_rows, out_mass,
                                out_pt, out_idx3);
        });
    });
}

hepacc_status hepacc_trijet_closest_mass(const void* pt, const void* eta, const void* phi, const void* mass,
                                         hepacc_dtype t, const void* offsets, hepacc_dtype ot, int64_t n,
                                         const uint8_t* mask_rows, const uint8_t* mask_content, float target,
                                         float* out_mass, int32_t* out_idx3, hepacc_stream stream) {
    HEPACC_CHECK(n >= 0, "n_rows < 0");
    if (n == 0) return HEPACC_OK;
    HEPACC_CHECK(pt && eta && phi && mass && offsets, "missing required pointer");
    HEPACC_CHECK(out_mass || out_idx3, "no output requested");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    return with_offsets_type(ot, [&](auto ot_tag) -> hepacc_status {
        using O = typename decltype(ot_tag)::type;
        return with_float_type(t, [&](auto tt) -> hepacc_status {
            using T = typename decltype(tt)::type;
            const size_t smem = coop_smem();
            int grid = 0;
            hepacc_status st = tile_grid(k_trijet_closest<T, O>, smem, (n + 31) / 32, &grid);
            if (st != HEPACC_OK) return st;
            k_trijet_closest<T, O><<<grid, kBlock, smem, s>>>(
                static_cast<const T*>(pt), static_cast<const T*>(eta), static_cast<const T*>(phi),
                static_cast<const T*>(mass), static_cast<const O*>(offsets), n, mask_rows, mask_content, target,
                out_mass, out_idx3);
            HEPACC_CHECK_LAUNCH("trijet_closest_mass launch");
            return HEPACC_OK;
        });
    });
}

hepacc_status hepacc_select_opposite_sign(const int8_t* charge, const void* offsets, hepacc_dtype ot, int64_t n,
                                          const uint8_t* mask_rows, const uint8_t* mask_in, uint8_t* mask_out,
                                          hepacc_stream stream) {
    HEPACC_CHECK(n >= 0, "n_rows < 0");
    if (n == 0) return HEPACC_OK;
    HEPACC_CHECK(charge && offsets && mask_out, "charge, offsets and mask_out are required");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    return with_offsets_type(ot, [&](auto ot_tag) -> hepacc_status {
        using O = typename decltype(ot_tag)::type;
        k_opposite_sign<O><<<flat_grid(n), kBlock, 0, s>>>(charge, static_cast<const O*>(offsets), n, mask_rows,
                                                            mask_in, mask_out);
        HEPACC_CHECK_LAUNCH("select_opposite_sign launch");
        return HEPACC_OK;
    });
}

hepacc_status hepacc_get_bin_contents(const void* data, hepacc_dtype dt, int64_t n, const float* edges, int32_t nbins,
                                      const float* contents, int32_t interpolate, float* out, hepacc_stream stream) {
    HEPACC_CHECK(n >= 0, "n < 0");
    HEPACC_CHECK(nbins >= 1 && nbins <= 65536, "nbins must be in [1, 65536]");
    if (n == 0) return HEPACC_OK;
    HEPACC_CHECK(data && edges && contents && out, "data, edges, contents and out are required");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    return with_float_type(dt, [&](auto tt) -> hepacc_status {
        using T = typename decltype(tt)::type;
        k_bin_contents<T><<<flat_grid(n), kBlock, 0, s>>>(static_cast<const T*>(data), n, edges, nbins, contents,
                                                          interpolate ? 1 : 0, out);
        HEPACC_CHECK_LAUNCH("get_bin_contents launch");
        return HEPACC_OK;
    });
}

hepacc_status hepacc_fill_histogram(const void* data, hepacc_dtype dt, const float* weights, const uint8_t* mask,
                                    int64_t n, const float* edges, int32_t nbins, uint64_t* counts, double* sumw,
                                    double* sumw2, hepacc_stream stream) {
    HEPACC_CHECK(n >= 0, "n < 0");
    HEPACC_CHECK(nbins >= 1 && nbins <= 65536, "nbins must be in [1, 65536]");
    if (n == 0) return HEPACC_OK;
    HEPACC_CHECK(data && edges && counts, "data, edges and counts are required");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned long long* c = reinterpret_cast<unsigned long long*>(counts);
    return with_value_type(dt, [&](auto t) -> hepacc_status {
        using T = typename decltype(t)::type;
        const int nbin = nbins + 2;
        const size_t ex_smem = exact_smem(nbin, sumw != nullptr, sumw2 != nullptr) + static_cast<size_t>(nbins + 1) * 4;
        if (ex_smem <= kExactSmemMax) {
            int grid = 0;
            hepacc_status st = tile_grid(k_hist_exact<T>, ex_smem, (n + 31) / 32, &grid);
            if (st != HEPACC_OK) return st;
            // no block adds more than kExactPerBlock elements in one launch
            const int64_t chunk = static_cast<int64_t>(grid) * kExactPerBlock;
            const T* xt = static_cast<const T*>(data);
            for (int64_t off = 0; off < n; off += chunk) {
                k_hist_exact<T><<<grid, kBlock, ex_smem, s>>>(xt + off, weights ? weights + off : nullptr,
                                                              mask ? mask + off : nullptr, std::min(chunk, n - off),
                                                              edges, nbins, c, sumw, sumw2);
                HEPACC_CHECK_LAUNCH("fill_histogram launch");
            }
            return HEPACC_OK;
        }
        const size_t smem = static_cast<size_t>(nbin) * (8 + 8 + 4) + static_cast<size_t>(nbins + 1) * 4 + kBlock * 8;
        if (nbin <= 4096) {
            int grid = 0;
            hepacc_status st = tile_grid(k_hist_smem<T>, smem, (n + 31) / 32, &grid);
            if (st != HEPACC_OK) return st;
            k_hist_smem<T><<<grid, kBlock, smem, s>>>(static_cast<const T*>(data), weights, mask, n, edges, nbins,
                                                      c, sumw, sumw2);
        } else {
            k_hist_global<T><<<flat_grid(n), kBlock, 0, s>>>(static_cast<const T*>(data), weights, mask, n, edges,
                                                             nbins, c, sumw, sumw2);
        }
        HEPACC_CHECK_LAUNCH("fill_histogram launch");
        return HEPACC_OK;
    });
}

hepacc_status hepacc_fill_histogram_nd(int32_t ndim, const void* const* data, const hepacc_dtype* data_types,
                                       const float* const* edges, const int32_t* nbins, const float* weights,
                                       const uint8_t* mask, int64_t n, uint64_t* counts, double* sumw,
                                       double* sumw2, hepacc_stream stream) {
    HEPACC_CHECK(ndim >= 1 && ndim <= HEPACC_MAX_HIST_DIMS, "ndim must be in [1, %d]", HEPACC_MAX_HIST_DIMS);
    HEPACC_CHECK(data && data_types && edges && nbins, "data, data_types, edges and nbins are required");
    HEPACC_CHECK(n >= 0, "n < 0");
    HistAxes a{};
    a.ndim = ndim;
    int64_t ncell = 1;
    for (int d = 0; d < ndim; ++d) {
        HEPACC_CHECK(nbins[d] >= 1 && nbins[d] <= 65536, "nbins[%d] must be in [1, 65536]", d);
        switch (data_types[d]) {
            case HEPACC_F32: case HEPACC_F16: case HEPACC_BF16: case HEPACC_U8: case HEPACC_I8: case HEPACC_I32:
                break;
            default: return fail(HEPACC_ERR_DTYPE, "unsupported data type on axis %d", d);
        }
        a.x[d] = data[d];
        a.e[d] = edges[d];
        a.dt[d] = static_cast<int>(data_types[d]);
        a.nb[d] = nbins[d];
        ncell *= nbins[d] + 2;
        HEPACC_CHECK(ncell <= (int64_t(1) << 24), "more than 2^24 cells");
        HEPACC_CHECK(n == 0 || (data[d] && edges[d]), "data[%d] and edges[%d] are required", d, d);
    }
    if (n == 0) return HEPACC_OK;
    HEPACC_CHECK(counts, "counts is required");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned long long* c = reinterpret_cast<unsigned long long*>(counts);
    const size_t ex_smem = exact_smem(ncell, sumw != nullptr, sumw2 != nullptr);
    if (ex_smem <= kExactSmemMax) {
        int grid = 0;
        hepacc_status st = tile_grid(k_hist_nd_exact, ex_smem, (n + 31) / 32, &grid);
        if (st != HEPACC_OK) return st;
        const int64_t chunk = static_cast<int64_t>(grid) * kExactPerBlock;
        for (int64_t off = 0; off < n; off += chunk) {
            HistAxes ac = a;
            for (int d = 0; d < ndim; ++d)
                ac.x[d] = static_cast<const unsigned char*>(a.x[d]) + off * dtype_size(data_types[d]);
            k_hist_nd_exact<<<grid, kBlock, ex_smem, s>>>(ac, weights ? weights + off : nullptr,
                                                          mask ? mask + off : nullptr, std::min(chunk, n - off),
                                                          static_cast<int>(ncell), c, sumw, sumw2);
            HEPACC_CHECK_LAUNCH("fill_histogram_nd launch");
        }
        return HEPACC_OK;
    }
    if (ncell <= 4096) {
        const size_t smem = static_cast<size_t>(ncell) * (8 + 8 + 4) + kBlock * 8;
        int grid = 0;
        hepacc_status st = tile_grid(k_hist_nd_smem, smem, (n + 31) / 32, &grid);
        if (st != HEPACC_OK) return st;
        k_hist_nd_smem<<<grid, kBlock, smem, s>>>(a, weights, mask, n, static_cast<int>(ncell), c, sumw, sumw2);
    } else {
        k_hist_nd_global<<<flat_grid(n), kBlock, 0, s>>>(a, weights, mask, n, c, sumw, sumw2);
    }
    HEPACC_CHECK_LAUNCH("fill_histogram_nd launch");
    return HEPACC_OK;
}

hepacc_status hepacc_selftest_wait_timeout(int64_t limit_cycles, hepacc_stream stream) {
    HEPACC_CHECK(limit_cycles >= 1 && limit_cycles <= (int64_t(1) << 31), "limit_cycles must be in [1, 2^31]");
    k_wait_timeout<<<1, 1, 0, reinterpret_cast<cudaStream_t>(stream)>>>(static_cast<long long>(limit_cycles));
    HEPACC_CHECK_LAUNCH("selftest launch");
    return HEPACC_OK;
}

}  // extern "C"

namespace hepacc {

// Launches the offsets check, waits for it and reads (and clears) the check
// bit of this translation unit's error word: HEPACC_ERR_DEVICE_CHECK if the
// offsets are negative at the start or decrease.
hepacc_status check_offsets(const void* offsets, hepacc_dtype ot, int64_t n, int64_t content_len, cudaStream_t s) {
    if (n <= 0) return HEPACC_OK;
    if (!offsets) return fail(HEPACC_ERR_INVALID_ARG, "offsets are required");
    hepacc_status st = with_offsets_type(ot, [&](auto ot_tag) -> hepacc_status {
        using O = typename decltype(ot_tag)::type;
        k_check_offsets<O><<<flat_grid(n), kBlock, 0, s>>>(static_cast<const O*>(offsets), n, content_len);
        HEPACC_CHECK_LAUNCH("offsets check launch");
        return HEPACC_OK;
    });
    if (st != HEPACC_OK) return st;
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "offsets check");
    unsigned int v = 0;
    cudaMemcpyFromSymbol(&v, g_device_error, sizeof v);
    if (v & kErrCheck) {
        const unsigned int keep = v & ~kErrCheck;
        cudaMemcpyToSymbol(g_device_error, &keep, sizeof keep);
        return fail(HEPACC_ERR_DEVICE_CHECK, "offsets are negative at the start, decrease, or end past the content");
    }
    return HEPACC_OK;
}

}  // namespace hepacc

extern "C" {

hepacc_status hepacc_validate_offsets(const void* offsets, hepacc_dtype ot, int64_t n, int64_t content_len,
                                      int64_t* first_bad, hepacc_stream stream) {
    HEPACC_CHECK(n >= 0 && content_len >= 0, "negative size");
    HEPACC_CHECK(offsets && first_bad, "offsets and first_bad are required");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned long long* fb = reinterpret_cast<unsigned long long*>(first_bad);
    return with_offsets_type(ot, [&](auto ot_tag) -> hepacc_status {
        using O = typename decltype(ot_tag)::type;
        k_validate_init<<<1, 1, 0, s>>>(offsets, ot == HEPACC_I64, fb);
        if (n > 0) k_validate<O><<<flat_grid(n), kBlock, 0, s>>>(static_cast<const O*>(offsets), n, content_len, fb);
        k_validate_fini<<<1, 1, 0, s>>>(fb);
        HEPACC_CHECK_LAUNCH("validate_offsets launch");
        return HEPACC_OK;
    });
}

}  // extern "C"
