// Host-side helpers shared by the hepacc translation units: error recording,
// argument checks, device properties and launch sizing.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <string>

#include "hepacc.h"

namespace hepacc {

hepacc_status fail(hepacc_status s, const char* fmt, ...);
hepacc_status cuda_fail(cudaError_t e, const char* what);

// Number of SMs and the opt-in shared memory limit of the current device
// (cached per device).
struct DeviceInfo {
    int sms;
    int smem_optin;
    int max_threads_per_sm;
    int smem_per_sm;      // shared memory of one SM
    int smem_reserved;    // shared memory the runtime reserves per block
};
DeviceInfo device_info();

// Debug checks before chain launches (environment variable HEPACC_DEBUG set
// and not 0), and the offsets check they run: a kernel over the offsets,
// then a wait for it; HEPACC_ERR_DEVICE_CHECK when offsets[0] < 0, the
// offsets decrease, or offsets[n] > content_len.
bool debug_checks();

// Readers of the device error words: every translation unit that includes
// the device header registers one (hepacc_device.cuh); hepacc_device_error()
// calls them all.
using ErrorWordReader = unsigned int (*)(bool clear);
void register_error_word(ErrorWordReader reader);
hepacc_status check_offsets(const void* offsets, hepacc_dtype ot, int64_t n, int64_t content_len, cudaStream_t s);

inline bool is_float_type(hepacc_dtype t) { return t == HEPACC_F32 || t == HEPACC_F16 || t == HEPACC_BF16; }
inline bool is_offsets_type(hepacc_dtype t) { return t == HEPACC_I32 || t == HEPACC_I64; }
inline size_t dtype_size(hepacc_dtype t) {
    switch (t) {
        case HEPACC_F32: case HEPACC_I32: return 4;
        case HEPACC_F16: case HEPACC_BF16: return 2;
        case HEPACC_I8: case HEPACC_U8: return 1;
        case HEPACC_I64: case HEPACC_F64: return 8;
    }
    return 0;
}

}  // namespace hepacc

#define HEPACC_CHECK_LAUNCH(what)                                  \
    do {                                                           \
        cudaError_t e_ = cudaGetLastError();                       \
        if (e_ != cudaSuccess) return ::hepacc::cuda_fail(e_, what); \
    } while (0)
