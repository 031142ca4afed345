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
//
// Inside a tile every element index is 32-bit and relative to the tile's
// first element of its collection.
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

extern __shared__ __align__(128) unsigned char g_dyn_smem[];

// This lane's event and element ranges inside the current tile.
template <int NCOLL>
struct TileRanges {
    int64_t e;                   // event index
    bool valid;                  // e < n
    int rs[NCOLL], rt[NCOLL];    // [rs, rt): the event's elements, relative to S
    int64_t S[NCOLL];            // absolute index of the tile's first element
};

// Column access for a staged tile: element r of column c is in shared memory.
template <int NC>
struct SmemCols {
    uint32_t off[NC];            // byte offset of element 0 (relative to S) in dynamic shared memory
    template <typename T>
    __device__ __forceinline__ T ld(int c, int r) const {
        return *reinterpret_cast<const T*>(g_dyn_smem + off[c] + r * static_cast<int>(sizeof(T)));
    }
};

// Column access straight from global memory (tiles too large to stage).
template <int NC>
struct GlobCols {
    const unsigned char* p[NC];  // address of element 0 (relative to S)
    template <typename T>
    __device__ __forceinline__ T ld(int c, int r) const {
        return reinterpret_cast<const T*>(p[c])[r];
    }
};

// Runs body(cols, ranges) for every tile this warp owns, with cols a
// SmemCols (staged) or GlobCols. Kernels that use it need
// stage_bytes_per_warp(spec) * warps bytes at the start of dynamic shared
// memory.
template <typename OffT, int NCOLL, int NC, typename Body>
__device__ __forceinline__ void tile_loop(const StageSpec<NC>& spec, const OffT* const (&offs)[NCOLL], int64_t n,
                                          Body&& body) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarp = blockDim.x >> 5;
    const uint32_t wbuf = static_cast<uint32_t>(warp) * 2u * spec.buf_bytes;     // offset in dynamic smem
    uint64_t* bars = reinterpret_cast<uint64_t*>(g_dyn_smem + static_cast<size_t>(nwarp) * 2 * spec.buf_bytes) + 2 * warp;
    const uint32_t bar[2] = {smem_addr(bars), smem_addr(bars + 1)};
    const uint32_t smem0 = smem_addr(g_dyn_smem);
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
        for (int c = 0; c < NC; ++c) {
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
                for (int c = 0; c < NC; ++c) {
                    if (c >= spec.ncol || spec.col[c].base == nullptr) continue;
                    const ColSpec& cs = spec.col[c];
                    if (T[cs.coll] <= S[cs.coll]) continue;
                    const uintptr_t a = reinterpret_cast<uintptr_t>(cs.base) + static_cast<uintptr_t>(S[cs.coll]) * cs.es;
                    const uintptr_t z = reinterpret_cast<uintptr_t>(cs.base) + static_cast<uintptr_t>(T[cs.coll]) * cs.es;
                    const uintptr_t a16 = a & ~uintptr_t(15);
                    const uint32_t bytes = static_cast<uint32_t>(((z + 15) & ~uintptr_t(15)) - a16);
                    bulk_g2s(smem0 + wbuf + b * spec.buf_bytes + cs.soff, reinterpret_cast<const void*>(a16), bytes,
                             bar[b]);
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

        TileRanges<NCOLL> r;
        r.e = tile * kTile + lane;
        r.valid = r.e < n;
#pragma unroll
        for (int c = 0; c < NCOLL; ++c) {
            r.S[c] = __shfl_sync(0xffffffffu, cs_[c], 0);
            r.rs[c] = static_cast<int>(cs_[c] - r.S[c]);
            r.rt[c] = static_cast<int>(ct_[c] - r.S[c]);
        }
        if (cstaged) {
            SmemCols<NC> sc;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                sc.off[c] = 0;
                if (c >= spec.ncol || spec.col[c].base == nullptr) continue;
                const ColSpec& col = spec.col[c];
                const uintptr_t a = reinterpret_cast<uintptr_t>(col.base) + static_cast<uintptr_t>(r.S[col.coll]) * col.es;
                sc.off[c] = wbuf + b * spec.buf_bytes + col.soff + static_cast<uint32_t>(a & 15u);
            }
            body(sc, r);
        } else {
            GlobCols<NC> gc;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                gc.p[c] = nullptr;
                if (c >= spec.ncol || spec.col[c].base == nullptr) continue;
                const ColSpec& col = spec.col[c];
                gc.p[c] = col.base + static_cast<uintptr_t>(r.S[col.coll]) * col.es;
            }
            body(gc, r);
        }
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

// Lane = event over [0, n) with a grid-stride loop and no staging: each
// event's elements are read straight from global memory through the cache
// (the events of a warp are adjacent, so its loads share cache lines). For
// kernels whose per-event work is a short scan this costs fewer instructions
// per event than the staged tiles. body(cols, ranges) as for tile_loop, with
// a GlobCols and the ranges of one event (rs = 0).
template <typename OffT, int NCOLL, int NC, typename Body>
__device__ __forceinline__ void event_loop(const StageSpec<NC>& spec, const OffT* const (&offs)[NCOLL], int64_t n,
                                           Body&& body) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n; e += stride) {
        TileRanges<NCOLL> r;
        r.e = e;
        r.valid = true;
#pragma unroll
        for (int c = 0; c < NCOLL; ++c) {
            const int64_t a = ldoff(offs[c], e);
            r.S[c] = a;
            r.rs[c] = 0;
            r.rt[c] = static_cast<int>(ldoff(offs[c], e + 1) - a);
        }
        GlobCols<NC> gc;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            gc.p[c] = nullptr;
            if (c >= spec.ncol || spec.col[c].base == nullptr) continue;
            const ColSpec& col = spec.col[c];
            gc.p[c] = col.base + static_cast<uintptr_t>(r.S[col.coll]) * col.es;
        }
        body(gc, r);
    }
}

}  // namespace hepacc
