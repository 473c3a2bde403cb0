// K1 (Eq. 2 active-set selection) and K2 (union of two chunk sets with the
// Eq. 4 membership flags): order-preserving stream compaction over the
// level-concatenated scene, one pass, decoupled look-back.
//
// Eq. 2 (Sec. 3 "LOD representation"): Gaussian g of level l is active at
// centre c iff d_l <= |mu_g - c| < d_{l+1}, d_0 = 0, d_L = inf.  The test is
// evaluated on squared distances in FP32 with every operation rounded
// (D = (dx*dx + dy*dy) + dz*dz, thresholds rounded once from FP64), so the
// selected set is reproducible bit for bit.
#include "common.cuh"

namespace lodge {

namespace {

struct SelectParams {
    const float* mx;
    const float* my;
    const float* mz;
    int64_t n;
    int32_t num_levels;
    int64_t level_off[kMaxLevels + 1];
    float thr_lo[kMaxLevels];
    float thr_hi[kMaxLevels];
    float c[3];
};

// Loads kSelectIPT consecutive items starting at `first` (a multiple of 16;
// planes are padded to a multiple of 64 elements) and returns the predicate
// bits; out_val[j] receives the value to emit for item j.
struct LodSelectF {
    SelectParams p;
    __device__ __forceinline__ uint32_t operator()(int64_t first, uint32_t* out_val) const {
        float x[kSelectIPT], y[kSelectIPT], z[kSelectIPT];
        const float4* px = reinterpret_cast<const float4*>(p.mx + first);
        const float4* py = reinterpret_cast<const float4*>(p.my + first);
        const float4* pz = reinterpret_cast<const float4*>(p.mz + first);
        if (first < p.n) {
#pragma unroll
            for (int q = 0; q < kSelectIPT / 4; ++q) {
                float4 a = __ldcs(px + q), b = __ldcs(py + q), c = __ldcs(pz + q);
                x[4 * q] = a.x; x[4 * q + 1] = a.y; x[4 * q + 2] = a.z; x[4 * q + 3] = a.w;
                y[4 * q] = b.x; y[4 * q + 1] = b.y; y[4 * q + 2] = b.z; y[4 * q + 3] = b.w;
                z[4 * q] = c.x; z[4 * q + 1] = c.y; z[4 * q + 2] = c.z; z[4 * q + 3] = c.w;
            }
        }
        int l = 0;
        while (l + 1 < p.num_levels && first >= p.level_off[l + 1]) ++l;
        uint32_t bits = 0;
#pragma unroll
        for (int j = 0; j < kSelectIPT; ++j) {
            int64_t g = first + j;
            while (l + 1 < p.num_levels && g >= p.level_off[l + 1]) ++l;
            float dx = __fsub_rn(x[j], p.c[0]);
            float dy = __fsub_rn(y[j], p.c[1]);
            float dz = __fsub_rn(z[j], p.c[2]);
            float D = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
            bool in = (g < p.n) && (p.thr_lo[l] <= D) && (D < p.thr_hi[l]);
            bits |= (uint32_t)in << j;
            out_val[j] = (uint32_t)g;
        }
        return bits;
    }
};

// Visibility filtering (Sec. 3): keep the entries of a chunk's gid list
// whose importance score reaches the threshold, in list order.
struct ScoreKeepF {
    const uint32_t* list;
    const float* score;
    float thr;
    int64_t n, n_total;
    __device__ __forceinline__ uint32_t operator()(int64_t first, uint32_t* out_val) const {
        uint32_t bits = 0;
#pragma unroll
        for (int j = 0; j < kSelectIPT; ++j) {
            const int64_t i = first + j;
            uint32_t g = 0;
            bool keep = false;
            if (i < n) {
                g = __ldg(list + i);
                keep = (int64_t)g < n_total && __ldg(score + g) >= thr;
            }
            bits |= (uint32_t)keep << j;
            out_val[j] = g;
        }
        return bits;
    }
};

struct UnionF {
    const uint8_t* marks;
    int64_t n;
    __device__ __forceinline__ uint32_t operator()(int64_t first, uint32_t* out_val) const {
        uint4 m = make_uint4(0, 0, 0, 0);
        if (first < n) m = __ldcs(reinterpret_cast<const uint4*>(marks + first));
        uint32_t w[4] = {m.x, m.y, m.z, m.w};
        uint32_t bits = 0;
#pragma unroll
        for (int j = 0; j < kSelectIPT; ++j) {
            uint32_t b = (w[j >> 2] >> (8 * (j & 3))) & 0xffu;
            int64_t g = first + j;
            bool in = (g < n) && b;
            bits |= (uint32_t)in << j;
            out_val[j] = (uint32_t)g | ((b & 1u) ? kFlagA : 0u) | ((b & 2u) ? kFlagB : 0u);
        }
        return bits;
    }
};

template <class F>
__global__ void __launch_bounds__(kSelectThreads)
compact_kernel(F f, int64_t n, uint32_t* __restrict__ out, uint32_t* __restrict__ d_count,
               uint32_t* __restrict__ status, uint32_t* __restrict__ tile_counter,
               uint32_t* __restrict__ err) {
    __shared__ uint32_t s_tile, s_prefix;
    __shared__ uint32_t s_scan[33];
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint32_t ntiles = (uint32_t)((n + kSelectTile - 1) / kSelectTile);
    const int64_t first = (int64_t)tile * kSelectTile + (int64_t)threadIdx.x * kSelectIPT;
    uint32_t vals[kSelectIPT];
    uint32_t bits = f(first, vals);
    uint32_t cnt = __popc(bits), total;
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
            if (tile == ntiles - 1) *d_count = prefix + total;
        }
    }
    __syncthreads();
    uint32_t pos = s_prefix + excl;
#pragma unroll
    for (int j = 0; j < kSelectIPT; ++j)
        if (bits >> j & 1u) out[pos++] = vals[j];
}

__global__ void mark_kernel(const uint32_t* __restrict__ list, int64_t n, uint8_t* marks,
                            uint8_t bit, int64_t n_total, uint32_t* err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t g = list[i] & kGidMask;
    if ((int64_t)g >= n_total) { atomicOr(err, kErrBadIndex); return; }
    marks[g] = (uint8_t)(marks[g] | bit);
}

}  // namespace

void launch_lod_select(const DevScene& sc, const float c32[3], const float* thr_lo,
                       const float* thr_hi, uint32_t* out, uint32_t* d_count, uint32_t* status,
                       uint32_t* tile_counter, uint32_t* err, cudaStream_t s) {
    SelectParams p;
    p.mx = sc.mx; p.my = sc.my; p.mz = sc.mz;
    p.n = sc.n_total;
    p.num_levels = sc.num_levels;
    for (int l = 0; l <= kMaxLevels; ++l) p.level_off[l] = sc.level_off[l];
    for (int l = 0; l < kMaxLevels; ++l) { p.thr_lo[l] = thr_lo[l]; p.thr_hi[l] = thr_hi[l]; }
    for (int k = 0; k < 3; ++k) p.c[k] = c32[k];
    int64_t ntiles = (sc.n_total + kSelectTile - 1) / kSelectTile;
    if (ntiles == 0) { cudaMemsetAsync(d_count, 0, 4, s); return; }
    compact_kernel<LodSelectF><<<(unsigned)ntiles, kSelectThreads, 0, s>>>(
        LodSelectF{p}, sc.n_total, out, d_count, status, tile_counter, err);
}

void launch_chunk_union(const uint32_t* a, int64_t na, const uint32_t* b, int64_t nb,
                        int64_t n_total, uint8_t* marks, uint32_t* out, uint32_t* d_count,
                        uint32_t* status, uint32_t* tile_counter, uint32_t* err, cudaStream_t s) {
    int64_t padded = (n_total + 63) / 64 * 64;
    cudaMemsetAsync(marks, 0, (size_t)padded, s);
    if (na) mark_kernel<<<(unsigned)((na + 255) / 256), 256, 0, s>>>(a, na, marks, 1, n_total, err);
    if (nb) mark_kernel<<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(b, nb, marks, 2, n_total, err);
    int64_t ntiles = (n_total + kSelectTile - 1) / kSelectTile;
    if (ntiles == 0) { cudaMemsetAsync(d_count, 0, 4, s); return; }
    compact_kernel<UnionF><<<(unsigned)ntiles, kSelectThreads, 0, s>>>(
        UnionF{marks, n_total}, n_total, out, d_count, status, tile_counter, err);
}

void launch_score_filter(const uint32_t* list, int64_t n, const float* score, float thr,
                         int64_t n_total, uint32_t* out, uint32_t* d_count, uint32_t* status,
                         uint32_t* tile_counter, uint32_t* err, cudaStream_t s) {
    const int64_t ntiles = (n + kSelectTile - 1) / kSelectTile;
    if (ntiles == 0) { cudaMemsetAsync(d_count, 0, 4, s); return; }
    compact_kernel<ScoreKeepF><<<(unsigned)ntiles, kSelectThreads, 0, s>>>(
        ScoreKeepF{list, score, thr, n, n_total}, n, out, d_count, status, tile_counter, err);
}

}  // namespace lodge
