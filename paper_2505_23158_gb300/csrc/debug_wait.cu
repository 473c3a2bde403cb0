// lodge_debug_lookback: the library's bounded decoupled look-back run alone,
// with one tile that never publishes, to show that the waits give up and the
// host sees LODGE_E_TIMEOUT instead of a hung GPU.
#include <cstdio>

#include "common.cuh"

namespace lodge {

namespace {

// One warp per tile.  Tile b publishes its aggregate (b + 1) unless it is
// the missing one, walks back over its predecessors with the bounded wait and
// publishes its inclusive prefix.
__global__ void lookback_probe_kernel(uint32_t* status, int32_t n_tiles, int32_t missing,
                                      uint32_t limit, uint32_t* err, uint32_t* prefix_out) {
    const uint32_t tile = blockIdx.x;
    if ((int32_t)tile >= n_tiles || (int32_t)tile == missing) return;
    const uint32_t agg = tile + 1;
    if (threadIdx.x == 0) {
        st_volatile(status + tile, (tile == 0 ? kStInc : kStAgg) | agg);
        __threadfence();
    }
    __syncwarp();
    uint32_t prefix = tile == 0 ? 0u : warp_lookback(status, tile, err, limit);
    if (threadIdx.x == 0) {
        prefix_out[tile] = prefix;
        __threadfence();
        st_volatile(status + tile, kStInc | ((prefix + agg) & kStVal));
    }
}

}  // namespace

}  // namespace lodge

extern "C" lodge_status lodge_debug_lookback(int32_t n_tiles, int32_t missing, uint32_t spin_limit,
                                             uint32_t* h_prefix, void* stream) {
    using namespace lodge;
    if (n_tiles < 1 || n_tiles > 1024) return set_error(LODGE_E_INVALID, "n_tiles must be 1..1024");
    if (spin_limit < 1 || spin_limit > kSpinLimit) return set_error(LODGE_E_INVALID, "spin_limit must be 1..2^22");
    if (!h_prefix) return set_error(LODGE_E_INVALID, "NULL prefix output");
    if (missing >= n_tiles) return set_error(LODGE_E_INVALID, "missing tile out of range");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // words: status[n_tiles] | err | prefix[n_tiles]
    uint32_t* d = nullptr;
    size_t words = 2 * (size_t)n_tiles + 1;
    cudaError_t e = cudaMalloc(&d, sizeof(uint32_t) * words);
    if (e != cudaSuccess) return set_error(LODGE_E_CUDA, cudaGetErrorString(e));
    uint32_t* status = d;
    uint32_t* err = d + n_tiles;
    uint32_t* prefix = d + n_tiles + 1;
    uint32_t h_err = 0;
    e = cudaMemsetAsync(d, 0, sizeof(uint32_t) * words, s);
    if (e == cudaSuccess) {
        lookback_probe_kernel<<<n_tiles, 32, 0, s>>>(status, n_tiles, missing, spin_limit, err, prefix);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h_prefix, prefix, sizeof(uint32_t) * (size_t)n_tiles, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) return set_error(LODGE_E_CUDA, cudaGetErrorString(e));
    if (h_err & kErrTimeout) {
        char msg[160];
        snprintf(msg, sizeof msg, "a look-back wait gave up after %u polls (tile %d never published)",
                 spin_limit, missing);
        return set_error(LODGE_E_TIMEOUT, msg);
    }
    return LODGE_OK;
}
