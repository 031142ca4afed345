// Device-side building blocks shared by the hepacc kernels (sm_103a):
// bulk asynchronous copies (TMA, cp.async.bulk) into shared memory tracked by
// mbarriers, bounded waits that report a timeout instead of hanging, element
// widening to binary32, the Delta R^2 of Section III and the invariant mass
// in a cancellation-free binary32 form.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace hepacc {

constexpr int kWarp = 32;
constexpr int kTile = 32;   // events per warp tile (one per lane)

// Device error word of this translation unit: bit 0 = a bounded wait gave
// up, bit 1 = a device-side input check failed. Each translation unit has its
// own copy, and registers a reader for it when the library is loaded, so
// hepacc_device_error() reads and clears every copy without a list to keep.
static __device__ unsigned int g_device_error;

using ErrorWordReader = unsigned int (*)(bool clear);
void register_error_word(ErrorWordReader reader);   // library state (api.cu)

namespace {
unsigned int read_error_word_of_unit(bool clear) {
    unsigned int v = 0;
    cudaMemcpyFromSymbol(&v, g_device_error, sizeof v);
    if (clear && v) {
        const unsigned int z = 0;
        cudaMemcpyToSymbol(g_device_error, &z, sizeof z);
    }
    return v;
}
const bool g_error_word_registered = (register_error_word(&read_error_word_of_unit), true);
}  // namespace

constexpr unsigned int kErrTimeout = 1u;
constexpr unsigned int kErrCheck = 2u;

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Bulk copy global -> shared (TMA engine, no tensor map); src, dst and bytes
// are multiples of 16. Completion is signalled on the mbarrier as bytes.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the mbarrier phase with the given parity, giving up after about
// `limit_cycles` SM clocks. Returns false on timeout (after setting the
// device error word).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  long long limit_cycles = (1ll << 31)) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > limit_cycles) {
            atomicOr(&g_device_error, kErrTimeout);
            return false;
        }
    }
}

// ---------------------------------------------------------------------------
// Element access
// ---------------------------------------------------------------------------

template <typename T> struct Elem;
template <> struct Elem<float> {
    static __device__ __forceinline__ float f(float v) { return v; }
};
template <> struct Elem<__half> {
    static __device__ __forceinline__ float f(__half v) { return __half2float(v); }
};
template <> struct Elem<__nv_bfloat16> {
    static __device__ __forceinline__ float f(__nv_bfloat16 v) { return __bfloat162float(v); }
};
template <> struct Elem<uint8_t> {
    static __device__ __forceinline__ float f(uint8_t v) { return static_cast<float>(v); }
};
template <> struct Elem<int8_t> {
    static __device__ __forceinline__ float f(int8_t v) { return static_cast<float>(v); }
};
template <> struct Elem<int32_t> {
    static __device__ __forceinline__ float f(int32_t v) { return static_cast<float>(v); }
};

template <typename T>
__device__ __forceinline__ float ldf(const T* p, int64_t i) {
    return Elem<T>::f(p[i]);
}

// Event offsets as int64 regardless of storage type.
template <typename OffT>
__device__ __forceinline__ int64_t ldoff(const OffT* off, int64_t i) {
    return static_cast<int64_t>(off[i]);
}

// ---------------------------------------------------------------------------
// Delta R^2 (Section III): Delta phi folded into [-pi, pi] by one shift of
// 2 pi, two rounded binary32 squares and one rounded sum (no contraction).
// ---------------------------------------------------------------------------

__device__ __forceinline__ float dr2_f32(float eta1, float phi1, float eta2, float phi2) {
    const float kPi = 3.14159265358979f;
    const float kTwoPi = 6.28318530717959f;
    const float deta = __fsub_rn(eta1, eta2);
    float dphi = __fsub_rn(phi1, phi2);
    if (dphi > kPi)
        dphi = __fsub_rn(dphi, kTwoPi);
    else if (dphi < -kPi)
        dphi = __fadd_rn(dphi, kTwoPi);
    return __fadd_rn(__fmul_rn(deta, deta), __fmul_rn(dphi, dphi));
}

// ---------------------------------------------------------------------------
// Invariant masses in binary32 without cancellation.
//
// For objects i, j with transverse momentum pt, pseudorapidity eta, azimuth
// phi and mass m: E_i E_j - p_i.p_j = A_ij + 2 mT_i mT_j sinh^2(dy/2)
// + 2 pt_i pt_j sin^2(dphi/2), with mT = sqrt(pt^2 + m^2), y the rapidity and
// A_ij = mT_i mT_j - pt_i pt_j = (pt_i^2 m_j^2 + m_i^2 pt_j^2 + m_i^2 m_j^2)
//        / (mT_i mT_j + pt_i pt_j).
// Every term is non-negative, so the sum m^2 = sum m_i^2 + 2 sum_{i<j}(...)
// loses nothing to cancellation. The rapidity difference is
// dy = (eta_i - eta_j) + (c_i - c_j) with the small correction c = y - eta
// = (log1p(u e^-eta) - log1p(u e^eta)) / 2, u = (E - p) / pt and
// E - p = m^2 / (E + p), which follows from y = ln((E+pz)/(E-pz))/2 and
// eta = ln((p+pz)/(p-pz))/2 with p + pz = pt e^eta, p - pz = pt e^-eta.
// ---------------------------------------------------------------------------

struct MassObj {
    float pt, eta, phi, m;
    float mt;   // sqrt(pt^2 + m^2)
    float c;    // rapidity minus pseudorapidity
    float e;    // energy
};

__device__ __forceinline__ MassObj mass_obj(float pt, float eta, float phi, float m) {
    MassObj o;
    o.pt = pt;
    o.eta = eta;
    o.phi = phi;
    o.m = m;
    const float m2 = m * m;
    o.mt = sqrtf(pt * pt + m2);
    // e^eta and e^-eta to a few 1e-7 relative (the approximate exponential):
    // they enter the energy and the small rapidity correction c only; their
    // difference in c loses relative accuracy near eta = 0, where c (of
    // order u eta) is negligible against the rapidity difference it corrects
    const float ex = __expf(eta);
    const float emx = __expf(-eta);
    const float p = pt * 0.5f * (ex + emx);   // pt cosh(eta)
    o.e = sqrtf(p * p + m2);
    if (pt > 0.0f) {
        // c = (log1p(u e^-eta) - log1p(u e^eta)) / 2 as one logarithm:
        // log1p(-u (e^eta - e^-eta) / (1 + u e^eta)) / 2
        const float u = __fdividef(__fdividef(m2, o.e + p), pt);
        o.c = 0.5f * log1pf(-__fdividef(u * (ex - emx), 1.0f + u * ex));
    } else {
        o.c = 0.0f;
    }
    return o;
}

// E_i E_j - p_i . p_j, non-negative.
__device__ __forceinline__ float pair_dot(const MassObj& a, const MassObj& b) {
    if (a.pt == 0.0f) return a.m * b.e;
    if (b.pt == 0.0f) return b.m * a.e;
    const float a_ij = __fdividef(a.pt * a.pt * b.m * b.m + a.m * a.m * b.pt * b.pt + a.m * a.m * b.m * b.m,
                                  a.mt * b.mt + a.pt * b.pt);
    const float hy = 0.5f * ((a.eta - b.eta) + (a.c - b.c));
    const float sh = sinhf(hy);
    // sin(dphi / 2) as sinpi(dphi / (2 pi)): exact argument reduction, so
    // small angles keep their relative accuracy
    const float sp = sinpif((a.phi - b.phi) * 0.159154943f);
    return a_ij + 2.0f * a.mt * b.mt * sh * sh + 2.0f * a.pt * b.pt * sp * sp;
}

__device__ __forceinline__ float mass2obj(const MassObj& a, const MassObj& b) {
    return sqrtf(a.m * a.m + b.m * b.m + 2.0f * pair_dot(a, b));
}

__device__ __forceinline__ float mass3obj(const MassObj& a, const MassObj& b, const MassObj& c) {
    const float s = a.m * a.m + b.m * b.m + c.m * c.m;
    return sqrtf(s + 2.0f * (pair_dot(a, b) + pair_dot(a, c) + pair_dot(b, c)));
}

// ---------------------------------------------------------------------------
// Histogram bin of v against increasing binary32 edges e[0..nb]: 0 below
// e[0], nb+1 at or above e[nb], else b with e[b-1] <= v < e[b]; -1 for NaN.
// The first guess assumes uniform spacing; the explicit comparisons that
// follow make the result exact for any increasing edges.
// ---------------------------------------------------------------------------

// The same with the first and last edge given (e0 = e[0], en = e[nb]).
__device__ __forceinline__ int find_bin_lim(float v, const float* e, float e0, float en, int nb, float inv_width) {
    if (v != v) return -1;
    if (v < e0) return 0;
    if (v >= en) return nb + 1;
    int b = static_cast<int>((v - e0) * inv_width) + 1;
    b = b < 1 ? 1 : (b > nb ? nb : b);
    while (b > 1 && v < e[b - 1]) --b;
    while (b < nb && v >= e[b]) ++b;
    return b;
}

__device__ __forceinline__ int find_bin(float v, const float* e, int nb, float inv_width) {
    if (v != v) return -1;
    if (v < e[0]) return 0;
    if (v >= e[nb]) return nb + 1;
    int b = static_cast<int>((v - e[0]) * inv_width) + 1;
    b = b < 1 ? 1 : (b > nb ? nb : b);
    while (b > 1 && v < e[b - 1]) --b;
    while (b < nb && v >= e[b]) ++b;
    return b;
}

}  // namespace hepacc
