// noalloc.cu -- bh_sort_keys_static: the stable radix sort of sort.cu over
// caller buffers, with its scratch (per-tile digit histograms and scan block
// sums) in one fixed array in device global memory instead of memory from
// cudaMalloc.  Nothing in this file allocates.
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "bh_internal.cuh"

namespace bh {
namespace {

// Largest n this entry point accepts, and the scratch that n needs:
// 256 digit counts per 4096-key tile plus the scan's block sums (1 MiB).
constexpr int64_t kStaticSortMaxN = BH_SORT_STATIC_MAX_N;
constexpr int64_t kStaticWords = 256 * (kStaticSortMaxN / 4096) + (256 * (kStaticSortMaxN / 4096) + 2047) / 2048;

static __device__ __align__(256) uint32_t g_sort_scratch[kStaticWords];

constexpr int kMaxDevices = 64;

struct DeviceSlot {
    bool ready = false;
    uint32_t* scratch = nullptr;
};

std::mutex g_setup_mu;
DeviceSlot g_slots[kMaxDevices];

int report(char* err, size_t err_len, int code, const char* fmt, ...) {
    if (err && err_len > 0) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(err, err_len, fmt, ap);
        va_end(ap);
    }
    return code;
}

// Per-device set-up, done once with the caller's device current: look up the
// address of g_sort_scratch on that device and raise the downsweep kernel's
// shared-memory limit there.  A failure is reported and retried next call.
// The cached address belongs to the device's primary context: it is not valid
// after that context is destroyed (cudaDeviceReset), after which this entry
// point must not be called again in the process.
int device_scratch(uint32_t** out, char* err, size_t err_len) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return report(err, err_len, BH_E_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return report(err, err_len, BH_E_INVAL, "device ordinal %d outside the supported 0..%d", dev,
                      kMaxDevices - 1);
    std::lock_guard<std::mutex> lock(g_setup_mu);
    DeviceSlot& s = g_slots[dev];
    if (!s.ready) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sort_scratch);
        if (e != cudaSuccess)
            return report(err, err_len, BH_E_CUDA, "cudaGetSymbolAddress(sort scratch) on device %d: %s", dev,
                          cudaGetErrorString(e));
        e = sort_setup_device();
        if (e != cudaSuccess)
            return report(err, err_len, BH_E_CUDA, "setting the sort kernel's shared-memory limit on device %d: %s",
                          dev, cudaGetErrorString(e));
        s.scratch = static_cast<uint32_t*>(p);
        s.ready = true;
    }
    *out = s.scratch;
    return BH_OK;
}

}  // namespace
}  // namespace bh

extern "C" int bh_sort_keys_static(uint64_t* keys, uint32_t* idx, uint64_t* keys_tmp, uint32_t* idx_tmp, int64_t n,
                                   void* stream, char* err, size_t err_len) {
    using namespace bh;
    if (err && err_len > 0) err[0] = '\0';
    if (n < 0 || n > kStaticSortMaxN)
        return report(err, err_len, BH_E_INVAL,
                      "n = %lld is outside 0..%lld, the largest sort the fixed scratch array holds",
                      (long long)n, (long long)kStaticSortMaxN);
    if (n == 0) return BH_OK;
    if (!keys || !idx || !keys_tmp || !idx_tmp)
        return report(err, err_len, BH_E_INVAL, "null buffer pointer");
    {  // the four buffers must be pairwise disjoint byte ranges
        const uintptr_t lo[4] = {(uintptr_t)keys, (uintptr_t)idx, (uintptr_t)keys_tmp, (uintptr_t)idx_tmp};
        const uintptr_t len[4] = {(uintptr_t)n * 8u, (uintptr_t)n * 4u, (uintptr_t)n * 8u, (uintptr_t)n * 4u};
        static const char* const name[4] = {"keys", "idx", "keys_tmp", "idx_tmp"};
        for (int a = 0; a < 4; ++a)
            for (int b = a + 1; b < 4; ++b)
                if (lo[a] < lo[b] + len[b] && lo[b] < lo[a] + len[a])
                    return report(err, err_len, BH_E_INVAL, "%s and %s overlap (the four buffers must be disjoint)",
                                  name[a], name[b]);
    }
    if (sort_scratch_words(n) > kStaticWords)
        return report(err, err_len, BH_E_INVAL, "sort of n = %lld needs %lld scratch words, %lld available",
                      (long long)n, (long long)sort_scratch_words(n), (long long)kStaticWords);
    uint32_t* scratch = nullptr;
    int rc = device_scratch(&scratch, err, err_len);
    if (rc != BH_OK) return rc;
    // The histograms are fully written by every upsweep and the block sums by
    // every reduce before they are read, so no part of the scratch has to
    // start at zero.
    cudaError_t e = sort_pairs_with((cudaStream_t)stream, keys, idx, keys_tmp, idx_tmp, n, scratch);
    if (e != cudaSuccess) return report(err, err_len, BH_E_CUDA, "sort launch: %s", cudaGetErrorString(e));
    return BH_OK;
}
