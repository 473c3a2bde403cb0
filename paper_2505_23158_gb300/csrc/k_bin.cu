// K4: tile binning.  Walks the visible records in depth order and emits one
// (tile id, record) pair per tile that the record's rect covers (Sec. 3
// "Preliminaries: 3DGS": each 2D Gaussian is assigned to every 16x16 tile it
// overlaps).  Offsets come from a block scan plus decoupled look-back; each
// block then writes its pairs cooperatively (load-balanced: thread s finds
// its record by binary search over the block's prefix sums), so the writes
// are coalesced however unequal the rect sizes are.
//
// K6: per-tile [begin, end) ranges of the tile-sorted pairs.
#include "common.cuh"

namespace lodge {

namespace {

__global__ void __launch_bounds__(kEmitThreads)
emit_kernel(const uint32_t* __restrict__ sorted_rec, int64_t n_vis,
            const uint2* __restrict__ rec_rect, int32_t tiles_x, uint32_t* __restrict__ tile_key,
            uint32_t* __restrict__ tile_val, int64_t cap, uint32_t* __restrict__ status,
            uint32_t* __restrict__ counter, uint32_t* __restrict__ err) {
    __shared__ uint32_t s_pref[kEmitThreads + 1];
    __shared__ uint2 s_rect[kEmitThreads];
    __shared__ uint32_t s_rec[kEmitThreads];
    __shared__ uint32_t s_scan[33];
    __shared__ uint32_t s_tile, s_prefix;
    if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const int64_t i = (int64_t)tile * kEmitThreads + threadIdx.x;
    uint32_t cnt = 0, rec = 0;
    uint2 r = make_uint2(0, 0);
    if (i < n_vis) {
        rec = sorted_rec[i];
        if ((int64_t)rec >= n_vis) { atomicOr(err, kErrBadIndex); rec = 0; }
        r = rec_rect[rec];
        uint32_t w = (r.y & 0xffffu) - (r.x & 0xffffu) + 1u;
        uint32_t h = (r.y >> 16) - (r.x >> 16) + 1u;
        cnt = w * h;
    }
    uint32_t total;
    uint32_t excl = block_exclusive_scan(cnt, s_scan, &total);
    if (threadIdx.x < 32) {
        uint32_t prefix = 0;
        if (tile == 0) {
            if (threadIdx.x == 0) st_volatile(status, kStInc | total);
        } else {
            if (threadIdx.x == 0) st_volatile(status + tile, kStAgg | total);
            prefix = warp_lookback(status, tile, err);
            if (threadIdx.x == 0) st_volatile(status + tile, kStInc | (prefix + total));
        }
        if (threadIdx.x == 0) s_prefix = prefix;
    }
    s_pref[threadIdx.x] = excl;
    s_rect[threadIdx.x] = r;
    s_rec[threadIdx.x] = rec;
    if (threadIdx.x == 0) s_pref[kEmitThreads] = total;
    __syncthreads();
    const int64_t base = s_prefix;
    for (uint32_t s = threadIdx.x; s < total; s += kEmitThreads) {
        int lo = 0, hi = kEmitThreads;
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (s_pref[mid] <= s) lo = mid; else hi = mid;
        }
        uint32_t k = s - s_pref[lo];
        uint2 rr = s_rect[lo];
        uint32_t tx0 = rr.x & 0xffffu, ty0 = rr.x >> 16, tx1 = rr.y & 0xffffu;
        uint32_t w = tx1 - tx0 + 1u;
        uint32_t ty = ty0 + k / w, tx = tx0 + k % w;
        int64_t out = base + s;
        if (out < cap) {
            tile_key[out] = ty * (uint32_t)tiles_x + tx;
            tile_val[out] = s_rec[lo];
        } else {
            atomicOr(err, kErrOverflow);
        }
    }
}

__global__ void ranges_kernel(const uint32_t* __restrict__ key, int64_t n, uint2* __restrict__ ranges,
                              uint32_t ntiles) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t t = key[i];
    if (t >= ntiles) return;
    if (i == 0 || key[i - 1] != t) ranges[t].x = (uint32_t)i;
    if (i == n - 1 || key[i + 1] != t) ranges[t].y = (uint32_t)(i + 1);
}

}  // namespace

void launch_emit(const uint32_t* sorted_rec, int64_t n_vis, const uint2* rec_rect,
                 int32_t tiles_x, uint32_t* tile_key, uint32_t* tile_val, int64_t cap,
                 uint32_t* status, uint32_t* tile_counter, uint32_t* err, cudaStream_t s) {
    int64_t nb = (n_vis + kEmitThreads - 1) / kEmitThreads;
    if (nb == 0) return;
    emit_kernel<<<(unsigned)nb, kEmitThreads, 0, s>>>(sorted_rec, n_vis, rec_rect, tiles_x, tile_key,
                                                      tile_val, cap, status, tile_counter, err);
}

void launch_ranges(const uint32_t* tile_key, int64_t n_keys, uint2* ranges, int64_t ntiles,
                   cudaStream_t s) {
    if (n_keys == 0) return;
    ranges_kernel<<<(unsigned)((n_keys + 255) / 256), 256, 0, s>>>(tile_key, n_keys, ranges,
                                                                 (uint32_t)ntiles);
}

}  // namespace lodge
