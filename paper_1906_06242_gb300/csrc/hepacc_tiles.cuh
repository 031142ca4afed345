// Column specifications and the event loop of the per-operation kernels
// over jagged arrays (Section II layout): one thread per event over the
// whole range, each event's elements read straight from global memory
// (columns described by a StageSpec: base, element size, collection). The
// fused chain stages its tiles itself (chain_kernel.cuh); the dynamic
// shared-memory symbol declared here is shared by both.
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

extern __shared__ __align__(128) unsigned char g_dyn_smem[];

// This thread's event and its element ranges.
template <int NCOLL>
struct TileRanges {
    int64_t e;                   // event index
    bool valid;                  // e < n
    int rs[NCOLL], rt[NCOLL];    // [rs, rt): the event's elements, relative to S
    int64_t S[NCOLL];            // absolute index of the event's first element
};

// Column access straight from global memory.
template <int NC>
struct GlobCols {
    const unsigned char* p[NC];  // address of element 0 (relative to S)
    template <typename T>
    __device__ __forceinline__ T ld(int c, int r) const {
        return reinterpret_cast<const T*>(p[c])[r];
    }
};

// Lane = event over [0, n) with a grid-stride loop and no staging: each
// event's elements are read straight from global memory through the cache
// (the events of a warp are adjacent, so its loads share cache lines); for
// kernels whose per-event work is a short scan this costs far fewer
// instructions per event than staged warp tiles. Calls body(cols, ranges)
// with a GlobCols and the ranges of one event (rs = 0).
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
