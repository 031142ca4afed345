// Warp-tile pipeline over jagged arrays (Section II layout).
//
// A warp owns tiles of 32 consecutive events (lane = event). For a tile it
// reads the events' offsets, and one elected lane copies every needed content
// column's contiguous span [off[e0], off[e0+32]) into the warp's shared-memory
// stage buffer with bulk asynchronous copies (cp.async.bulk, the TMA engine),
// covering whole 16-byte-aligned chunks, completion tracked by an mbarrier.
// Two stage buffers per warp: the copies of the next tile are in flight while
// the lanes work on the current one. A tile whose span does not fit the
// stage capacity is processed straight from global memory instead.
#pragma once

#include "hepacc_device.cuh"

namespace hepacc {

struct ColSpec {
    const unsigned char* base;   // global column base (nullptr = column unused)
    uint32_t es;                 // element size in bytes
    uint32_t coll;               // index of the offsets array it follows
    uint32_t soff;               // byte offset of its region in a stage buffer
    uint32_t cap;                // region size in bytes (multiple of 16)
};

template <int NC>
struct StageSpec {
    ColSpec col[NC];
    int ncol;
    uint32_t buf_bytes;          // one stage buffer, multiple of 128
};

// Shared memory the pipeline needs per warp (two stage buffers and two
// mbarriers); the pipeline uses the first warps * this bytes of dynamic
// shared memory.
template <int NC>
__host__ __device__ inline uint32_t stage_bytes_per_warp(const StageSpec<NC>& s) { return 2 * s.buf_bytes + 16; }

template <int NCOLL, int kMaxCols>
struct TileView {
    int64_t e;                   // this lane's event
    bool valid;                  // e < n
    int64_t s[NCOLL], t[NCOLL];  // this lane's element range per collection
    int64_t S[NCOLL];            // first element of the tile per collection
    const unsigned char* colp[kMaxCols];   // element i of column c at colp[c] + (i - S[coll]) * es
    bool staged;

    template <typename T>
    __device__ __forceinline__ T at(int c, int coll, int64_t i) const {
        return reinterpret_cast<const T*>(colp[c])[i - S[coll]];
    }
};

// Runs body(TileView&) for every tile this warp owns. Kernels that use it
// need stage_bytes_per_warp(spec) * warps bytes of dynamic shared memory.
template <typename OffT, int NCOLL, int kMaxCols, typename Body>
__device__ __forceinline__ void tile_loop(const StageSpec<kMaxCols>& spec, const OffT* const (&offs)[NCOLL],
                                          int64_t n, Body&& body) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarp = blockDim.x >> 5;
    unsigned char* wbuf = smem + static_cast<size_t>(warp) * 2 * spec.buf_bytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + static_cast<size_t>(nwarp) * 2 * spec.buf_bytes) + 2 * warp;
    const uint32_t bar[2] = {smem_addr(bars), smem_addr(bars + 1)};
    if (lane == 0) {
        mbar_init(bar[0], 1);
        mbar_init(bar[1], 1);
        fence_mbar_init();
    }
    __syncwarp();

    const int64_t ntiles = (n + kTile - 1) / kTile;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * nwarp;
    int64_t tile = static_cast<int64_t>(blockIdx.x) * nwarp + warp;
    uint32_t parity[2] = {0u, 0u};

    // Loads the offsets of `tt` and starts its copies into stage `b`.
    auto issue = [&](int64_t tt, int b, int64_t (&s)[NCOLL], int64_t (&t)[NCOLL], bool& staged) {
        const int64_t e = tt * kTile + lane;
        const int64_t e_lo = e < n ? e : n;
        const int64_t e_hi = e + 1 < n ? e + 1 : n;
        int64_t S[NCOLL], T[NCOLL];
#pragma unroll
        for (int c = 0; c < NCOLL; ++c) {
            s[c] = ldoff(offs[c], e_lo);
            t[c] = ldoff(offs[c], e_hi);
            S[c] = __shfl_sync(0xffffffffu, s[c], 0);
            T[c] = __shfl_sync(0xffffffffu, t[c], 31);
        }
        bool fits = true;
        uint32_t total = 0;
#pragma unroll
        for (int c = 0; c < kMaxCols; ++c) {
            if (c >= spec.ncol || spec.col[c].base == nullptr) continue;
            const ColSpec& cs = spec.col[c];
            const uintptr_t a = reinterpret_cast<uintptr_t>(cs.base) + static_cast<uintptr_t>(S[cs.coll]) * cs.es;
            const uintptr_t z = reinterpret_cast<uintptr_t>(cs.base) + static_cast<uintptr_t>(T[cs.coll]) * cs.es;
            const uintptr_t bytes = T[cs.coll] > S[cs.coll] ? ((z + 15) & ~uintptr_t(15)) - (a & ~uintptr_t(15)) : 0;
            if (bytes > cs.cap) fits = false;
            total += static_cast<uint32_t>(bytes);
        }
        staged = fits;
        if (lane == 0) {
            if (fits) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(bar[b], total);
#pragma unroll
                for (int c = 0; c < kMaxCols; ++c) {
                    if (c >= spec.ncol || spec.col[c].base == nullptr) continue;
                    const ColSpec& cs = spec.col[c];
                    if (T[cs.coll] <= S[cs.coll]) continue;
                    const uintptr_t a = reinterpret_cast<uintptr_t>(cs.base) + static_cast<uintptr_t>(S[cs.coll]) * cs.es;
                    const uintptr_t z = reinterpret_cast<uintptr_t>(cs.base) + static_cast<uintptr_t>(T[cs.coll]) * cs.es;
                    const uintptr_t a16 = a & ~uintptr_t(15);
                    const uint32_t bytes = static_cast<uint32_t>(((z + 15) & ~uintptr_t(15)) - a16);
                    bulk_g2s(smem_addr(wbuf + b * spec.buf_bytes + cs.soff), reinterpret_cast<const void*>(a16),
                             bytes, bar[b]);
                }
            } else {
                mbar_arrive_expect_tx(bar[b], 0);
            }
        }
    };

    int64_t cs_[NCOLL], ct_[NCOLL], ns_[NCOLL], nt_[NCOLL];
    bool cstaged = false, nstaged = false;
    int b = 0;
    if (tile < ntiles) issue(tile, 0, cs_, ct_, cstaged);
    for (; tile < ntiles; tile += stride) {
        const int64_t next = tile + stride;
        if (next < ntiles) issue(next, b ^ 1, ns_, nt_, nstaged);
        if (!mbar_wait_bounded(bar[b], parity[b])) {
            // give the copies still in flight a bounded chance to land, then stop
            mbar_wait_bounded(bar[b ^ 1], parity[b ^ 1]);
            return;
        }
        parity[b] ^= 1u;

        TileView<NCOLL, kMaxCols> v;
        v.e = tile * kTile + lane;
        v.valid = v.e < n;
        v.staged = cstaged;
#pragma unroll
        for (int c = 0; c < NCOLL; ++c) {
            v.s[c] = cs_[c];
            v.t[c] = ct_[c];
            v.S[c] = __shfl_sync(0xffffffffu, cs_[c], 0);
        }
#pragma unroll
        for (int c = 0; c < kMaxCols; ++c) {
            if (c >= spec.ncol || spec.col[c].base == nullptr) {
                v.colp[c] = nullptr;
                continue;
            }
            const ColSpec& cs = spec.col[c];
            const uintptr_t a = reinterpret_cast<uintptr_t>(cs.base) + static_cast<uintptr_t>(v.S[cs.coll]) * cs.es;
            v.colp[c] = cstaged ? wbuf + b * spec.buf_bytes + cs.soff + (a & 15u)
                                : reinterpret_cast<const unsigned char*>(a);
        }
        body(v);
        __syncwarp();
#pragma unroll
        for (int c = 0; c < NCOLL; ++c) {
            cs_[c] = ns_[c];
            ct_[c] = nt_[c];
        }
        cstaged = nstaged;
        b ^= 1;
    }
}

}  // namespace hepacc
