// K4: tile binning.  Walks the visible records in depth order and emits one
// (bin id, record) pair per bin that the record's tile rect touches (Sec. 3
// "Preliminaries: 3DGS": each 2D Gaussian is assigned to every 16x16 tile it
// overlaps).  A bin is the tile itself or a square of 2^bin_log2 tiles; the
// compositing then drops, per tile, the records of its bin that miss the
// tile.  Two passes: key offsets by block scan plus decoupled look-back, then
// emission, key-balanced for small records, one warp per record for large
// ones.
//
// K6: per-bin [begin, end) ranges of the bin-sorted keys.
#include "common.cuh"

namespace lodge {

namespace {

// Pass 1: per depth-sorted visible record, its bin count; block scan plus
// decoupled look-back give the exclusive key offset koff[i] (koff[n_vis] =
// total).  The record id and rect are gathered into depth order (srec,
// srect, in bins) so that pass 2 reads them contiguously.
__global__ void __launch_bounds__(kEmitThreads)
emit_offsets_kernel(const uint32_t* __restrict__ sorted_rec, int64_t n_vis,
                    const uint2* __restrict__ rec_rect, uint32_t* __restrict__ koff,
                    uint32_t* __restrict__ srec, uint2* __restrict__ srect,
                    int bin_log2, uint32_t* __restrict__ status, uint32_t* __restrict__ counter,
                    uint32_t* __restrict__ err) {
    __shared__ uint32_t s_scan[33];
    __shared__ uint32_t s_tile, s_prefix;
    if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint32_t ntiles = (uint32_t)((n_vis + kEmitThreads - 1) / kEmitThreads);
    const int64_t i = (int64_t)tile * kEmitThreads + threadIdx.x;
    uint32_t cnt = 0;
    if (i < n_vis) {
        uint32_t rec = sorted_rec[i];
        if ((int64_t)rec >= n_vis) { atomicOr(err, kErrBadIndex); rec = 0; }
        const uint2 p = rec_rect[rec];   // pixel range -> tile range -> bin range
        const uint2 r = make_uint2((((p.x & 0xffffu) / kTile) >> bin_log2) |
                                       ((((p.x >> 16) / kTile) >> bin_log2) << 16),
                                   (((p.y & 0xffffu) / kTile) >> bin_log2) |
                                       ((((p.y >> 16) / kTile) >> bin_log2) << 16));
        uint32_t w = (r.y & 0xffffu) - (r.x & 0xffffu) + 1u;
        uint32_t h = (r.y >> 16) - (r.x >> 16) + 1u;
        cnt = w * h;
        srec[i] = rec;
        srect[i] = r;
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
        if (threadIdx.x == 0) {
            s_prefix = prefix;
            if (tile == ntiles - 1) koff[n_vis] = prefix + total;
        }
    }
    __syncthreads();
    if (i < n_vis) koff[i] = s_prefix + excl;
}

// Pass 2, many small records: the key list is cut into slices of kEmitKeysPerCta keys; a CTA
// writes whole slices (grid-stride).  The (at most kEmitKeysPerCta) records
// that own a slice are located by one warp-parallel search in koff, staged in
// shared memory, and each key finds its record by binary search there, so
// every slice costs the same however large single rects are.  The CTA also
// counts the tile sort's digits (shared-memory histograms flushed once).
__device__ __forceinline__ int64_t warp_upper_bound(const uint32_t* __restrict__ a, int64_t n,
                                                    uint32_t v) {
    // last index g in [0, n) with a[g] <= v (a ascending, a[0] <= v)
    const int lane = threadIdx.x & 31;
    int64_t lo = 0, hi = n;
    while (hi - lo > 32) {
        const int64_t step = (hi - lo + 31) / 32;
        const int64_t p = lo + (int64_t)lane * step;
        const bool ok = p < hi && a[p] <= v;
        const uint32_t m = __ballot_sync(0xffffffffu, ok);
        const int last = 31 - __clz(m);   // lane 0 always qualifies
        const int64_t nlo = lo + (int64_t)last * step;
        hi = min(hi, nlo + step);
        lo = nlo;
    }
    const int64_t p = lo + lane;
    const bool ok = p < hi && a[p] <= v;
    const uint32_t m = __ballot_sync(0xffffffffu, ok);
    return lo + (31 - __clz(m));
}

__global__ void __launch_bounds__(kEmitThreads)
emit_keys_sliced_kernel(const uint32_t* __restrict__ koff, const uint32_t* __restrict__ srec,
                 const uint2* __restrict__ srect, int64_t n_vis, int64_t n_keys, int32_t tiles_x,
                 uint32_t* __restrict__ tile_key, uint32_t* __restrict__ tile_val, int rbits,
                 int passes, uint32_t last_mask, uint32_t* __restrict__ digit_hist,
                 uint32_t* __restrict__ err) {
    __shared__ uint32_t s_off[kEmitKeysPerCta + 1];
    __shared__ uint2 s_rect[kEmitKeysPerCta];
    __shared__ uint32_t s_rec[kEmitKeysPerCta];
    __shared__ uint32_t s_hist[3][256];
    __shared__ int64_t s_g0;
    __shared__ int s_m;
    for (int i = threadIdx.x; i < 3 * 256; i += kEmitThreads) (&s_hist[0][0])[i] = 0;
    const int64_t nslices = (n_keys + kEmitKeysPerCta - 1) / kEmitKeysPerCta;
    for (int64_t sl = blockIdx.x; sl < nslices; sl += gridDim.x) {
        const int64_t k0 = sl * kEmitKeysPerCta;
        const int64_t k1 = min(k0 + (int64_t)kEmitKeysPerCta, n_keys);
        __syncthreads();
        if (threadIdx.x < 32) {
            const int64_t g0 = warp_upper_bound(koff, n_vis, (uint32_t)k0);
            const int64_t g1 = warp_upper_bound(koff + g0, n_vis - g0, (uint32_t)(k1 - 1)) + g0;
            if (threadIdx.x == 0) {
                int64_t m = g1 - g0 + 1;
                if (m > kEmitKeysPerCta) { atomicOr(err, kErrOverflow); m = kEmitKeysPerCta; }
                s_g0 = g0;
                s_m = (int)m;
            }
        }
        __syncthreads();
        const int64_t g0 = s_g0;
        const int m = s_m;
        for (int j = threadIdx.x; j < m; j += kEmitThreads) {
            s_off[j] = koff[g0 + j];
            s_rect[j] = srect[g0 + j];
            s_rec[j] = srec[g0 + j];
        }
        __syncthreads();
        for (int64_t key = k0 + threadIdx.x; key < k1; key += kEmitThreads) {
            int lo = 0, hi = m;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (s_off[mid] <= (uint32_t)key) lo = mid; else hi = mid;
            }
            const uint32_t k = (uint32_t)key - s_off[lo];
            const uint2 rr = s_rect[lo];
            const uint32_t tx0 = rr.x & 0xffffu, ty0 = rr.x >> 16, tx1 = rr.y & 0xffffu;
            const uint32_t w = tx1 - tx0 + 1u;
            const uint32_t q = k / w;
            const uint32_t tile = (ty0 + q) * (uint32_t)tiles_x + tx0 + (k - q * w);
            if (rbits) {
                tile_key[key] = (tile << rbits) | s_rec[lo];
            } else {
                tile_key[key] = tile;
                tile_val[key] = s_rec[lo];
            }
            for (int p = 0; p < passes; ++p)
                atomicAdd(&s_hist[p][(tile >> (8 * p)) & (p == passes - 1 ? last_mask : 0xffu)], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += kEmitThreads) {
        const uint32_t c = (&s_hist[0][0])[i];
        if (c) atomicAdd(digit_hist + i, c);
    }
}

// Pass 2, large records: one warp per depth-sorted record writes the record's keys,
// koff[i] .. koff[i+1]-1, its rect row-major, the lanes striding over them
// (warps of a CTA take consecutive records, CTAs stride over the list).  The
// CTA also counts the tile sort's digits in shared-memory histograms flushed
// once: the lowest digit per key (consecutive tiles fall in different bins),
// the higher digits per rect row, whose tile ids are one contiguous range
// that crosses a digit boundary at most once per 256 tiles.
__global__ void __launch_bounds__(kEmitThreads)
emit_keys_rect_kernel(const uint32_t* __restrict__ koff, const uint32_t* __restrict__ srec,
                 const uint2* __restrict__ srect, int64_t n_vis, int32_t tiles_x,
                 uint32_t* __restrict__ tile_key, uint32_t* __restrict__ tile_val, int rbits,
                 int passes, uint32_t last_mask, uint32_t* __restrict__ digit_hist) {
    __shared__ uint32_t s_hist[3][256];
    for (int i = threadIdx.x; i < 3 * 256; i += kEmitThreads) (&s_hist[0][0])[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t wstride = (int64_t)gridDim.x * (kEmitThreads / 32);
    for (int64_t i = (int64_t)blockIdx.x * (kEmitThreads / 32) + (threadIdx.x >> 5); i < n_vis;
         i += wstride) {
        const uint32_t k0 = koff[i];
        const uint32_t cnt = koff[i + 1] - k0;
        const uint2 rr = srect[i];
        const uint32_t rec = srec[i];
        const uint32_t tx0 = rr.x & 0xffffu, ty0 = rr.x >> 16;
        const uint32_t w = (rr.y & 0xffffu) - tx0 + 1u, h = (rr.y >> 16) - ty0 + 1u;
        // key k = lane + 32 j sits at row k / w, column k % w (stepped)
        uint32_t row = lane / w, col = lane - row * w;
        const uint32_t drow = 32u / w, dcol = 32u - drow * w;
        for (uint32_t k = lane; k < cnt; k += 32) {
            const uint32_t tile = (ty0 + row) * (uint32_t)tiles_x + tx0 + col;
            if (rbits) {
                tile_key[k0 + k] = (tile << rbits) | rec;
            } else {
                tile_key[k0 + k] = tile;
                tile_val[k0 + k] = rec;
            }
            atomicAdd(&s_hist[0][tile & (passes == 1 ? last_mask : 0xffu)], 1u);
            row += drow;
            col += dcol;
            if (col >= w) { col -= w; ++row; }
        }
        for (int p = 1; p < passes; ++p) {
            const uint32_t mask = p == passes - 1 ? last_mask : 0xffu;
            const int sh = 8 * p;
            for (uint32_t r = lane; r < h; r += 32) {
                uint32_t a = (ty0 + r) * (uint32_t)tiles_x + tx0;
                const uint32_t b = a + w - 1u;
                while (a <= b) {   // split [a, b] where digit p changes
                    const uint32_t end = min(b, ((a >> sh) + 1u << sh) - 1u);
                    atomicAdd(&s_hist[p][(a >> sh) & mask], end - a + 1u);
                    a = end + 1u;
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += kEmitThreads) {
        const uint32_t c = (&s_hist[0][0])[i];
        if (c) atomicAdd(digit_hist + i, c);
    }
}

// Coarse bins (a few keys per record): offsets and emission in one pass.
// A CTA takes 256 depth-sorted records, scans their bin counts and finds
// its key offset by decoupled look-back.  A record of at most 32 keys is
// written by its own thread; larger ones (the nearest records, which all
// fall in the first CTAs) go to a shared list that the CTA's warps take one
// record at a time, the lanes striding over the record's keys.  The bin
// sort's digit counts are kept in shared memory and flushed once.
constexpr uint32_t kFusedThreadKeys = 32;
__global__ void __launch_bounds__(kEmitThreads)
emit_fused_kernel(const uint32_t* __restrict__ sorted_rec, int64_t n_vis,
                  const uint2* __restrict__ rec_rect, int bin_log2, int32_t bins_x, int64_t n_keys,
                  uint32_t* __restrict__ tile_key, uint32_t* __restrict__ tile_val, int rbits,
                  int passes, uint32_t last_mask, uint32_t* __restrict__ digit_hist,
                  uint32_t* __restrict__ status, uint32_t* __restrict__ counter,
                  uint32_t* __restrict__ err, const unsigned long long* __restrict__ d_nvis,
                  const unsigned long long* __restrict__ d_nkeys) {
    // with device counts, n_vis and n_keys are capacities: the counts decide
    // which CTAs work and the keys must fit n_keys
    if (d_nvis) {
        const unsigned long long c = *d_nvis;
        if (c < (unsigned long long)n_vis) n_vis = (int64_t)c;
    }
    const int64_t key_cap = n_keys;
    if (d_nkeys) n_keys = (int64_t)*d_nkeys;
    __shared__ uint32_t s_scan[33];
    __shared__ uint32_t s_tile, s_prefix, s_nbig;
    __shared__ uint32_t s_big[kEmitThreads];
    __shared__ uint32_t s_off[kEmitThreads];
    __shared__ uint32_t s_cnt[kEmitThreads];
    __shared__ uint2 s_rect[kEmitThreads];
    __shared__ uint32_t s_rec[kEmitThreads];
    __shared__ uint32_t s_hist[3][256];
    for (int i = threadIdx.x; i < 3 * 256; i += kEmitThreads) (&s_hist[0][0])[i] = 0;
    if (threadIdx.x == 0) { s_tile = atomicAdd(counter, 1u); s_nbig = 0; }
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint32_t ntiles = (uint32_t)((n_vis + kEmitThreads - 1) / kEmitThreads);
    if (tile >= ntiles) return;   // past the device count (later tiles too)
    const int64_t i = (int64_t)tile * kEmitThreads + threadIdx.x;
    uint32_t cnt = 0, rec = 0, x0 = 0, y0 = 0, w = 1;
    if (i < n_vis) {
        rec = sorted_rec[i];
        if ((int64_t)rec >= n_vis) { atomicOr(err, kErrBadIndex); rec = 0; }
        const uint2 p = rec_rect[rec];   // pixel range -> tile range -> bin range
        x0 = ((p.x & 0xffffu) / kTile) >> bin_log2;
        y0 = ((p.x >> 16) / kTile) >> bin_log2;
        const uint32_t x1 = ((p.y & 0xffffu) / kTile) >> bin_log2, y1 = ((p.y >> 16) / kTile) >> bin_log2;
        w = x1 - x0 + 1u;
        cnt = w * (y1 - y0 + 1u);
    }
    uint32_t total;
    const uint32_t excl = block_exclusive_scan(cnt, s_scan, &total);
    if (cnt > kFusedThreadKeys) {
        const uint32_t slot = atomicAdd(&s_nbig, 1u);
        s_big[slot] = threadIdx.x;
        s_off[threadIdx.x] = excl;
        s_cnt[threadIdx.x] = cnt;
        s_rect[threadIdx.x] = make_uint2(x0 | (y0 << 16), w);   // bin coordinates < 2^12
        s_rec[threadIdx.x] = rec;
    }
    if (threadIdx.x < 32) {
        uint32_t prefix = 0;
        if (tile == 0) {
            if (threadIdx.x == 0) st_volatile(status, kStInc | total);
        } else {
            if (threadIdx.x == 0) st_volatile(status + tile, kStAgg | total);
            prefix = warp_lookback(status, tile, err);
            if (threadIdx.x == 0) st_volatile(status + tile, kStInc | (prefix + total));
        }
        if (threadIdx.x == 0) {
            s_prefix = prefix;
            if (tile == ntiles - 1 && (int64_t)prefix + total != n_keys) atomicOr(err, kErrOverflow);
        }
    }
    __syncthreads();
    const int64_t base = s_prefix;
    if ((int64_t)base + total > n_keys || (int64_t)base + total > key_cap) {
        // more keys than counted (never for consistent counts) or than fit
        if (threadIdx.x == 0) atomicOr(err, kErrOverflow);
        return;
    }
    // small records: the owning thread
    if (cnt <= kFusedThreadKeys) {
        uint32_t row = 0, col = 0;
        for (uint32_t k = 0; k < cnt; ++k) {
            const uint32_t bin = (y0 + row) * (uint32_t)bins_x + x0 + col;
            const int64_t at = base + excl + k;
            if (rbits) {
                tile_key[at] = (bin << rbits) | rec;
            } else {
                tile_key[at] = bin;
                tile_val[at] = rec;
            }
            for (int p = 0; p < passes; ++p)
                atomicAdd(&s_hist[p][(bin >> (8 * p)) & (p == passes - 1 ? last_mask : 0xffu)], 1u);
            if (++col == w) { col = 0; ++row; }
        }
    }
    // large records: one warp each
    const int lane = threadIdx.x & 31;
    const uint32_t nbig = s_nbig;
    for (uint32_t b = threadIdx.x >> 5; b < nbig; b += kEmitThreads / 32) {
        const uint32_t t = s_big[b];
        const uint2 rr = s_rect[t];
        const uint32_t bx0 = rr.x & 0xffffu, by0 = rr.x >> 16, bw = rr.y, bc = s_cnt[t];
        const uint32_t brec = s_rec[t];
        const int64_t at0 = base + s_off[t];
        uint32_t row = lane / bw, col = lane - row * bw;
        const uint32_t drow = 32u / bw, dcol = 32u - drow * bw;
        for (uint32_t k = lane; k < bc; k += 32) {
            const uint32_t bin = (by0 + row) * (uint32_t)bins_x + bx0 + col;
            if (rbits) {
                tile_key[at0 + k] = (bin << rbits) | brec;
            } else {
                tile_key[at0 + k] = bin;
                tile_val[at0 + k] = brec;
            }
            for (int p = 0; p < passes; ++p)
                atomicAdd(&s_hist[p][(bin >> (8 * p)) & (p == passes - 1 ? last_mask : 0xffu)], 1u);
            row += drow;
            col += dcol;
            if (col >= bw) { col -= bw; ++row; }
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < passes * 256; j += kEmitThreads) {
        const uint32_t c = (&s_hist[0][0])[j];
        if (c) atomicAdd(digit_hist + j, c);
    }
}

// Emission for large frames in three launches without look-back: count the
// bin keys of each tile of 1024 depth-sorted records, scan the tile counts
// in one CTA, then write each tile's keys at its offset.  With thousands of
// tiles in flight the fused kernel's CTAs spend most of their time at the
// barrier behind their look-back; here every CTA works independently and
// the records' rects are read twice instead.
constexpr int64_t kEmitSplitMin = 1ll << 21;                 // record capacity above which it is used

__device__ __forceinline__ uint32_t rec_bin_rect(const uint2* __restrict__ rec_rect, uint32_t rec,
                                                 int bin_log2, uint32_t& x0, uint32_t& y0, uint32_t& w) {
    const uint2 p = rec_rect[rec];   // pixel range -> tile range -> bin range
    x0 = ((p.x & 0xffffu) / kTile) >> bin_log2;
    y0 = ((p.x >> 16) / kTile) >> bin_log2;
    const uint32_t x1 = ((p.y & 0xffffu) / kTile) >> bin_log2, y1 = ((p.y >> 16) / kTile) >> bin_log2;
    w = x1 - x0 + 1u;
    return w * (y1 - y0 + 1u);
}

__device__ __forceinline__ int64_t device_count(int64_t cap, const unsigned long long* d) {
    if (!d) return cap;
    const unsigned long long c = *d;
    return c < (unsigned long long)cap ? (int64_t)c : cap;
}

template <int kEmitRecs>
__global__ void __launch_bounds__(kEmitThreads)
emit_count_kernel(const uint32_t* __restrict__ sorted_rec, int64_t n_vis_cap,
                  const unsigned long long* __restrict__ d_nvis, const uint2* __restrict__ rec_rect,
                  int bin_log2, uint32_t* __restrict__ tile_sum, uint32_t* __restrict__ err) {
    constexpr int kEmitTileRecs = kEmitThreads * kEmitRecs;
    __shared__ uint32_t s_part[kEmitThreads / 32];
    const int64_t n_vis = device_count(n_vis_cap, d_nvis);
    const int64_t t0 = (int64_t)blockIdx.x * kEmitTileRecs;
    if (t0 >= n_vis) return;   // past the device count (later tiles too)
    uint32_t sum = 0;
#pragma unroll
    for (int j = 0; j < kEmitRecs; ++j) {
        const int64_t i = t0 + (int64_t)j * kEmitThreads + threadIdx.x;
        if (i < n_vis) {
            uint32_t rec = sorted_rec[i];
            if ((int64_t)rec >= n_vis) { atomicOr(err, kErrBadIndex); rec = 0; }
            uint32_t x0, y0, w;
            sum += rec_bin_rect(rec_rect, rec, bin_log2, x0, y0, w);
        }
    }
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t tot = 0;
        for (int w = 0; w < kEmitThreads / 32; ++w) tot += s_part[w];
        tile_sum[blockIdx.x] = tot;
    }
}

// One CTA of 1024 threads: the tile counts become exclusive offsets in place;
// their total must equal the keys the projection counted and fit key_cap.
__global__ void __launch_bounds__(1024)
emit_scan_kernel(int tile_recs, uint32_t* __restrict__ tile_sum, int64_t n_vis_cap, const unsigned long long* __restrict__ d_nvis,
                 int64_t key_cap, const unsigned long long* __restrict__ d_nkeys, uint32_t* __restrict__ err) {
    __shared__ uint32_t s_scan[33];
    const int64_t n_vis = device_count(n_vis_cap, d_nvis);
    const int64_t ntiles = (n_vis + tile_recs - 1) / tile_recs;
    uint64_t carry = 0;
    for (int64_t base = 0; base < ntiles; base += 1024) {
        const int64_t t = base + threadIdx.x;
        const uint32_t v = t < ntiles ? tile_sum[t] : 0u;
        uint32_t total;
        const uint32_t e = block_exclusive_scan(v, s_scan, &total);
        if (t < ntiles) tile_sum[t] = (uint32_t)(carry + e);
        carry += total;
    }
    if (threadIdx.x == 0) {
        const int64_t n_keys = d_nkeys ? (int64_t)*d_nkeys : key_cap;
        if ((int64_t)carry != n_keys || (int64_t)carry > key_cap) atomicOr(err, kErrOverflow);
    }
}

template <int kEmitRecs>
__global__ void __launch_bounds__(kEmitThreads)
emit_write_kernel(const uint32_t* __restrict__ sorted_rec, int64_t n_vis_cap,
                  const unsigned long long* __restrict__ d_nvis, const uint2* __restrict__ rec_rect,
                  int bin_log2, int32_t bins_x, int64_t key_cap, const uint32_t* __restrict__ tile_off,
                  uint32_t* __restrict__ tile_key, uint32_t* __restrict__ tile_val, int rbits, int passes,
                  uint32_t last_mask, uint32_t* __restrict__ digit_hist, uint32_t* __restrict__ err) {
    constexpr int kEmitTileRecs = kEmitThreads * kEmitRecs;
    __shared__ uint32_t s_scan[33];
    __shared__ uint32_t s_nbig;
    __shared__ uint32_t s_big[kEmitTileRecs];     // (thread << 2 | j) of records with many keys
    __shared__ uint32_t s_off[kEmitTileRecs];
    __shared__ uint32_t s_hist[3][256];
    const int64_t n_vis = device_count(n_vis_cap, d_nvis);
    const int64_t t0 = (int64_t)blockIdx.x * kEmitTileRecs;
    if (t0 >= n_vis) return;
    for (int i = threadIdx.x; i < 3 * 256; i += kEmitThreads) (&s_hist[0][0])[i] = 0;
    if (threadIdx.x == 0) s_nbig = 0;
    // a thread's records are j * kEmitThreads + thread, so that the loads
    // are coalesced; the keys follow record order, which the scan below
    // gives as (j, thread) order
    uint32_t rec[kEmitRecs], cnt[kEmitRecs], bx[kEmitRecs], by[kEmitRecs], bw[kEmitRecs];
#pragma unroll
    for (int j = 0; j < kEmitRecs; ++j) {
        const int64_t i = t0 + (int64_t)j * kEmitThreads + threadIdx.x;
        rec[j] = 0; cnt[j] = 0; bx[j] = 0; by[j] = 0; bw[j] = 1;
        if (i < n_vis) {
            rec[j] = sorted_rec[i];
            if ((int64_t)rec[j] >= n_vis) rec[j] = 0;   // flagged by the count kernel
            cnt[j] = rec_bin_rect(rec_rect, rec[j], bin_log2, bx[j], by[j], bw[j]);
        }
    }
    const int64_t tbase = tile_off[blockIdx.x];
    uint32_t run = 0;   // keys of the record groups before group j in this tile
    __syncthreads();   // s_hist and s_nbig are set
#pragma unroll
    for (int j = 0; j < kEmitRecs; ++j) {
        uint32_t total;
        const uint32_t excl = block_exclusive_scan(cnt[j], s_scan, &total);
        const int64_t at0 = tbase + run + excl;
        if (at0 + cnt[j] > key_cap) {
            if (cnt[j]) atomicOr(err, kErrOverflow);
        } else if (cnt[j] > kFusedThreadKeys) {
            const uint32_t slot = atomicAdd(&s_nbig, 1u);
            s_big[slot] = (threadIdx.x << 2) | (uint32_t)j;
            s_off[slot] = run + excl;
        } else {
            uint32_t row = 0, col = 0;
            for (uint32_t k = 0; k < cnt[j]; ++k) {
                const uint32_t bin = (by[j] + row) * (uint32_t)bins_x + bx[j] + col;
                const int64_t at = at0 + k;
                if (rbits) {
                    tile_key[at] = (bin << rbits) | rec[j];
                } else {
                    tile_key[at] = bin;
                    tile_val[at] = rec[j];
                }
                for (int p = 0; p < passes; ++p)
                    atomicAdd(&s_hist[p][(bin >> (8 * p)) & (p == passes - 1 ? last_mask : 0xffu)], 1u);
                if (++col == bw[j]) { col = 0; ++row; }
            }
        }
        // the next record group's keys follow this group's
        run += total;
    }
    __syncthreads();
    // records with many keys: one warp each; their rects are read again
    const int lane = threadIdx.x & 31;
    const uint32_t nbig = s_nbig;
    for (uint32_t b = threadIdx.x >> 5; b < nbig; b += kEmitThreads / 32) {
        const uint32_t tj = s_big[b];
        const int64_t i = t0 + (int64_t)(tj & 3u) * kEmitThreads + (tj >> 2);
        uint32_t r = sorted_rec[i];
        if ((int64_t)r >= n_vis) r = 0;
        uint32_t x0, y0, w;
        const uint32_t c = rec_bin_rect(rec_rect, r, bin_log2, x0, y0, w);
        const int64_t at0 = tbase + s_off[b];
        uint32_t row = lane / w, col = lane - row * w;
        const uint32_t drow = 32u / w, dcol = 32u - drow * w;
        for (uint32_t k = lane; k < c; k += 32) {
            const uint32_t bin = (y0 + row) * (uint32_t)bins_x + x0 + col;
            if (rbits) {
                tile_key[at0 + k] = (bin << rbits) | r;
            } else {
                tile_key[at0 + k] = bin;
                tile_val[at0 + k] = r;
            }
            for (int p = 0; p < passes; ++p)
                atomicAdd(&s_hist[p][(bin >> (8 * p)) & (p == passes - 1 ? last_mask : 0xffu)], 1u);
            row += drow;
            col += dcol;
            if (col >= w) { col -= w; ++row; }
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < passes * 256; j += kEmitThreads) {
        const uint32_t c = (&s_hist[0][0])[j];
        if (c) atomicAdd(digit_hist + j, c);
    }
}

// exclusive scan of each pass's 256-bin digit histogram, in place
__global__ void digit_scan_kernel(uint32_t* hist) {
    __shared__ uint32_t s_scan[33];
    uint32_t* h = hist + blockIdx.x * 256;
    uint32_t v = h[threadIdx.x], total;
    h[threadIdx.x] = block_exclusive_scan(v, s_scan, &total);
}

// K6: per tile [begin, end) of the tile-sorted keys (tile = key >> shift);
// 4 keys per thread.
__global__ void ranges_kernel(const uint32_t* __restrict__ key, int64_t n, uint2* __restrict__ ranges,
                              uint32_t ntiles, int shift) {
    const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (i0 >= n) return;
    uint32_t prev = i0 > 0 ? key[i0 - 1] >> shift : 0xffffffffu;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int64_t i = i0 + j;
        if (i >= n) break;
        const uint32_t t = key[i] >> shift;
        const uint32_t next = i + 1 < n ? key[i + 1] >> shift : 0xffffffffu;
        if (t < ntiles) {
            if (t != prev) ranges[t].x = (uint32_t)i;
            if (t != next) ranges[t].y = (uint32_t)(i + 1);
        }
        prev = t;
    }
}

}  // namespace

void launch_emit(const uint32_t* sorted_rec, int64_t n_vis, const uint2* rec_rect,
                 int32_t bins_x, int bin_log2, uint32_t* koff, uint32_t* srec, uint2* srect,
                 int64_t n_keys, uint32_t* tile_key, uint32_t* tile_val, int rbits, int key_bits,
                 uint32_t* digit_hist, uint32_t* status, uint32_t* tile_counter, uint32_t* err,
                 cudaStream_t s) {
    const int32_t tiles_x = bins_x;   // the emit kernels index bins as tiles
    int64_t nb = (n_vis + kEmitThreads - 1) / kEmitThreads;
    if (nb == 0) return;
    const int P = (key_bits + 7) / 8;
    const int last_bits = key_bits - 8 * (P - 1);
    const uint32_t last_mask = last_bits >= 8 ? 0xffu : ((1u << last_bits) - 1u);
    if (n_keys > 0 && n_keys < kEmitWarpMinKeys * n_vis && bin_log2 > 0) {
        // coarse bins: a few keys per record, one fused pass
        emit_fused_kernel<<<(unsigned)nb, kEmitThreads, 0, s>>>(sorted_rec, n_vis, rec_rect, bin_log2, bins_x,
                                                                n_keys, tile_key, tile_val, rbits, P, last_mask,
                                                                digit_hist, status, tile_counter, err, nullptr,
                                                                nullptr);
        digit_scan_kernel<<<P, 256, 0, s>>>(digit_hist);
        return;
    }
    emit_offsets_kernel<<<(unsigned)nb, kEmitThreads, 0, s>>>(sorted_rec, n_vis, rec_rect, koff, srec,
                                                              srect, bin_log2, status, tile_counter, err);
    if (n_keys == 0) return;
    if (n_keys >= kEmitWarpMinKeys * n_vis) {
        // records average a warp's worth of keys or more: one warp per record
        const unsigned grid = (unsigned)std::min<int64_t>((n_vis + kEmitThreads / 32 - 1) / (kEmitThreads / 32),
                                                          (int64_t)device_sms() * 8);
        emit_keys_rect_kernel<<<grid, kEmitThreads, 0, s>>>(koff, srec, srect, n_vis, tiles_x, tile_key,
                                                            tile_val, rbits, P, last_mask, digit_hist);
    } else {
        const int64_t nslices = (n_keys + kEmitKeysPerCta - 1) / kEmitKeysPerCta;
        const unsigned grid = (unsigned)std::min<int64_t>(nslices, (int64_t)device_sms() * 4);
        emit_keys_sliced_kernel<<<grid, kEmitThreads, 0, s>>>(koff, srec, srect, n_vis, n_keys, tiles_x,
                                                              tile_key, tile_val, rbits, P, last_mask,
                                                              digit_hist, err);
    }
    digit_scan_kernel<<<P, 256, 0, s>>>(digit_hist);
}

int launch_emit_counted(const uint32_t* sorted_rec, int64_t n_vis_cap, const unsigned long long* d_nvis,
                        const uint2* rec_rect, int32_t bins_x, int bin_log2, int64_t key_cap,
                        const unsigned long long* d_nkeys, uint32_t* tile_key, uint32_t* tile_val,
                        int rbits, int key_bits, uint32_t* digit_hist, uint32_t* status,
                        uint32_t* tile_counter, uint32_t* err, cudaStream_t s) {
    const int64_t nb = (n_vis_cap + kEmitThreads - 1) / kEmitThreads;
    if (nb == 0) return 0;
    const int P = (key_bits + 7) / 8;
    const int last_bits = key_bits - 8 * (P - 1);
    const uint32_t last_mask = last_bits >= 8 ? 0xffu : ((1u << last_bits) - 1u);
    if (n_vis_cap > kEmitSplitMin) {
        // count, scan, write (the tile counts and offsets live in `status`,
        // which holds one word per 256 records)
        const unsigned nt = (unsigned)((n_vis_cap + 4 * kEmitThreads - 1) / (4 * kEmitThreads));
        emit_count_kernel<4><<<nt, kEmitThreads, 0, s>>>(sorted_rec, n_vis_cap, d_nvis, rec_rect, bin_log2,
                                                         status, err);
        emit_scan_kernel<<<1, 1024, 0, s>>>(4 * kEmitThreads, status, n_vis_cap, d_nvis, key_cap, d_nkeys, err);
        emit_write_kernel<4><<<nt, kEmitThreads, 0, s>>>(sorted_rec, n_vis_cap, d_nvis, rec_rect, bin_log2, bins_x,
                                                         key_cap, status, tile_key, tile_val, rbits, P, last_mask,
                                                         digit_hist, err);
        return 3;
    }
    emit_fused_kernel<<<(unsigned)nb, kEmitThreads, 0, s>>>(sorted_rec, n_vis_cap, rec_rect, bin_log2, bins_x,
                                                            key_cap, tile_key, tile_val, rbits, P, last_mask,
                                                            digit_hist, status, tile_counter, err, d_nvis,
                                                            d_nkeys);
    return 1;
}

void launch_digit_scan(uint32_t* hist, int passes, cudaStream_t s) {
    if (passes > 0) digit_scan_kernel<<<passes, 256, 0, s>>>(hist);
}

int emit_launches(int64_t n_vis, int64_t n_keys, int bin_log2) {
    if (n_vis == 0) return 0;
    if (n_keys > 0 && n_keys < kEmitWarpMinKeys * n_vis && bin_log2 > 0) return 2;
    return n_keys > 0 ? 3 : 1;
}

void launch_ranges(const uint32_t* tile_key, int64_t n_keys, uint2* ranges, int64_t ntiles,
                   int shift, cudaStream_t s) {
    if (n_keys == 0) return;
    const int64_t nt = (n_keys + 3) / 4;
    ranges_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(tile_key, n_keys, ranges,
                                                             (uint32_t)ntiles, shift);
}

}  // namespace lodge
