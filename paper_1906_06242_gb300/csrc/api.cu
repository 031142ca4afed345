// Library state of the hepacc C ABI: error text, status names, device
// properties and the device error words.
#include <mutex>
#include <vector>

#include "hepacc_host.h"

namespace hepacc {

namespace {
thread_local std::string t_last_error;

struct ErrorWords {
    std::mutex mu;
    std::vector<ErrorWordReader> readers;
};
ErrorWords& error_words() {
    static ErrorWords w;
    return w;
}
}  // namespace

void register_error_word(ErrorWordReader reader) {
    ErrorWords& w = error_words();
    std::lock_guard<std::mutex> g(w.mu);
    w.readers.push_back(reader);
}

hepacc_status fail(hepacc_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_last_error = buf;
    return s;
}

hepacc_status cuda_fail(cudaError_t e, const char* what) {
    return fail(HEPACC_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

DeviceInfo device_info() {
    static std::mutex mu;
    static std::vector<DeviceInfo> cache;
    static std::vector<bool> have;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(mu);
    if (dev >= static_cast<int>(cache.size())) {
        cache.resize(dev + 1);
        have.resize(dev + 1, false);
    }
    if (!have[dev]) {
        DeviceInfo d{};
        cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaDeviceGetAttribute(&d.max_threads_per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
        cudaDeviceGetAttribute(&d.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&d.smem_reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
        if (d.sms <= 0) d.sms = 1;
        if (d.smem_optin <= 0) d.smem_optin = 48 * 1024;
        if (d.smem_per_sm <= 0) d.smem_per_sm = d.smem_optin;
        if (d.smem_reserved < 0) d.smem_reserved = 0;
        cache[dev] = d;
        have[dev] = true;
    }
    return cache[dev];
}

}  // namespace hepacc

using namespace hepacc;

extern "C" {

const char* hepacc_version(void) { return "hepacc 0.1.0 (sm_103a)"; }

const char* hepacc_last_error(void) { return t_last_error.c_str(); }

const char* hepacc_status_string(hepacc_status s) {
    switch (s) {
        case HEPACC_OK: return "HEPACC_OK";
        case HEPACC_ERR_INVALID_ARG: return "HEPACC_ERR_INVALID_ARG";
        case HEPACC_ERR_DTYPE: return "HEPACC_ERR_DTYPE";
        case HEPACC_ERR_CUDA: return "HEPACC_ERR_CUDA";
        case HEPACC_ERR_OOM: return "HEPACC_ERR_OOM";
        case HEPACC_ERR_TIMEOUT: return "HEPACC_ERR_TIMEOUT";
        case HEPACC_ERR_DEVICE_CHECK: return "HEPACC_ERR_DEVICE_CHECK";
    }
    return "HEPACC_UNKNOWN_STATUS";
}

hepacc_status hepacc_device_error(uint32_t* flags) {
    if (!flags) return fail(HEPACC_ERR_INVALID_ARG, "flags is NULL");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    unsigned int v = 0;
    {
        ErrorWords& w = error_words();
        std::lock_guard<std::mutex> g(w.mu);
        for (ErrorWordReader r : w.readers) v |= r(true);
    }
    *flags = v;
    return HEPACC_OK;
}

}  // extern "C"
