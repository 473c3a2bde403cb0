// lodge_sort_pairs_noalloc: the onesweep pair sort with its scratch in a
// fixed, statically allocated device array instead of context-owned buffers
// grown with cudaMallocAsync.
//
// It serves callers that cannot allocate device memory at the point of the
// call: code embedded in a host application that owns every device
// allocation itself (an engine or plugin host with its own allocator and
// budget), and latency-critical loops where an allocation, which may
// synchronise the device or fail under memory pressure, is not acceptable.
// They pass their own key and value buffers; the library touches no other
// memory than the array below.
#include <cstdio>
#include <mutex>

#include "common.cuh"

namespace lodge {

namespace {

// Largest input, in (key, value) pairs.
constexpr int64_t kStaticSortMaxPairs = 1ll << 20;
// Layout of the array: alternate keys | alternate values | status word
// (padded to 256 B) | onesweep scratch (digit offsets, tile counters and
// look-back words for up to four 8-bit passes).
constexpr size_t kAltBytes = sizeof(uint32_t) * (size_t)kStaticSortMaxPairs;
constexpr size_t kErrOffset = 2 * kAltBytes;
constexpr size_t kScratchOffset = kErrOffset + 256;
// The look-back words grow with the number of tiles, which is largest with
// small tiles: size for the worst case over every n up to the limit.
constexpr int64_t kWorstTiles = (kStaticSortMaxPairs + kSortTileSmall - 1) / kSortTileSmall;
static_assert(kWorstTiles * kSortTileSmall >= kStaticSortMaxPairs, "tile count");
static_assert(sort_scratch_words(kStaticSortMaxPairs, 4) <= 4 * 256 + 32 + 4 * kWorstTiles * 256,
              "scratch bound");
constexpr size_t kScratchBytes = sizeof(uint32_t) * (size_t)(4 * 256 + 32 + 4 * kWorstTiles * 256);
constexpr size_t kStaticBytes = kScratchOffset + kScratchBytes;  // about 12.6 MB

// One copy per device that loads the library, held until process exit.
__device__ __align__(256) unsigned char g_sort_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
void* g_addr[kMaxDevices] = {};

// Device address of g_sort_scratch on the current device.  The host-side
// name is only a stand-in for the symbol, so the address is looked up once
// per device with that device current.
lodge_status scratch_address(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return set_error(LODGE_E_INVALID, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
        if (e != cudaSuccess || p == nullptr) {
            char msg[256];
            snprintf(msg, sizeof msg, "cudaGetSymbolAddress of the static sort scratch failed: %s",
                     cudaGetErrorString(e));
            cudaGetLastError();
            return set_error(LODGE_E_CUDA, msg);
        }
        g_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_addr[dev]);
    return LODGE_OK;
}

}  // namespace

}  // namespace lodge

extern "C" lodge_status lodge_sort_pairs_noalloc(uint32_t* d_keys, uint32_t* d_vals, int64_t n,
                                                 int32_t key_bits, void* stream) {
    using namespace lodge;
    if (n < 0 || key_bits < 0 || key_bits > 32) return set_error(LODGE_E_INVALID, "bad argument");
    if (n > kStaticSortMaxPairs) {
        char msg[160];
        snprintf(msg, sizeof msg, "n = %lld exceeds the static scratch limit of %lld pairs",
                 (long long)n, (long long)kStaticSortMaxPairs);
        return set_error(LODGE_E_INVALID, msg);
    }
    if (n > 0 && (!d_keys || !d_vals)) return set_error(LODGE_E_INVALID, "NULL key or value array");
    if (n <= 1 || key_bits == 0) return LODGE_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(LODGE_E_CUDA, cudaGetErrorString(e));
    unsigned char* base = nullptr;
    lodge_status st = scratch_address(dev, &base);
    if (st != LODGE_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t* alt_keys = reinterpret_cast<uint32_t*>(base);
    uint32_t* alt_vals = reinterpret_cast<uint32_t*>(base + kAltBytes);
    uint32_t* err = reinterpret_cast<uint32_t*>(base + kErrOffset);
    void* scratch = base + kScratchOffset;
    // the array keeps the previous call's contents: clear the status word
    // (launch_onesweep clears its own offsets, counters and look-back words)
    e = cudaMemsetAsync(err, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return set_error(LODGE_E_CUDA, cudaGetErrorString(e));
    int w = launch_onesweep(d_keys, d_vals, alt_keys, alt_vals, n, key_bits, scratch, err, s);
    if (w) {
        cudaMemcpyAsync(d_keys, alt_keys, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(d_vals, alt_vals, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s);
    }
    uint32_t h_err = 0;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_error(LODGE_E_CUDA, cudaGetErrorString(e));
    if (h_err & kErrTimeout) return set_error(LODGE_E_TIMEOUT, "a device-side wait of the sort timed out");
    if (h_err) return set_error(LODGE_E_OVERFLOW, "the sort reported an internal capacity error");
    return LODGE_OK;
}
