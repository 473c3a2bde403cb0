// Internal declarations shared by the library's translation units.
#pragma once

#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/lodge.h"

namespace lodge {

constexpr int kTile = 16;             // 16x16 pixel tiles (Sec. 3, Preliminaries)
constexpr int kMaxLevels = 8;
constexpr uint32_t kFlagA = 1u << 31; // active-list entry belongs to chunk A
constexpr uint32_t kFlagB = 1u << 30; // ... to chunk B
constexpr uint32_t kGidMask = (1u << 30) - 1u;

// device status word bits (set with atomicOr, read by the host after a sync)
constexpr uint32_t kErrTimeout = 1u << 0;   // a bounded spin gave up
constexpr uint32_t kErrOverflow = 1u << 1;  // an output capacity was exceeded
constexpr uint32_t kErrBadIndex = 1u << 2;  // an index was out of range

constexpr uint32_t kSpinLimit = 1u << 22;   // iterations before a wait gives up
constexpr uint32_t kSpinFast = 64;          // polls before a wait starts to sleep between polls

// ---------------------------------------------------------------------------
// decoupled look-back over 32-bit status words: flag in bits 31..30, value in
// bits 29..0 (so per-tile counts must stay below 2^30).
// ---------------------------------------------------------------------------
constexpr uint32_t kStAgg = 1u << 30;
constexpr uint32_t kStInc = 2u << 30;
constexpr uint32_t kStVal = (1u << 30) - 1u;

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) {
    return *reinterpret_cast<const volatile uint32_t*>(p);
}
__device__ __forceinline__ void st_volatile(uint32_t* p, uint32_t v) {
    *reinterpret_cast<volatile uint32_t*>(p) = v;
}

// Warp-cooperative exclusive look-back for one counter (called by a full
// warp).  status[tile] must have been published as AGG by this tile already
// (except tile 0, which needs no look-back).  Returns the exclusive prefix in
// every lane.  A predecessor that stays unpublished for `limit` polls sets
// kErrTimeout in *err and is counted as 0, so the kernel always terminates.
__device__ __forceinline__ uint32_t warp_lookback(const uint32_t* status, uint32_t tile,
                                                  uint32_t* err, uint32_t limit = kSpinLimit) {
    const int lane = threadIdx.x & 31;
    uint32_t prefix = 0;
    int64_t pos = (int64_t)tile - 1;
    while (pos >= 0) {
        int64_t idx = pos - lane;
        uint32_t v = kStInc;  // lanes before tile 0 act as an inclusive zero
        if (idx >= 0) {
            uint32_t spins = 0;
            v = ld_volatile(status + idx);
            while ((v & ~kStVal) == 0u) {
                if (++spins > limit) { atomicOr(err, kErrTimeout); v = kStInc; break; }
                // the predecessor is usually about to publish: poll at once a
                // few times before backing off with a sleep
                if (spins > kSpinFast) __nanosleep(32);
                v = ld_volatile(status + idx);
            }
        }
        uint32_t inc_mask = __ballot_sync(0xffffffffu, (v & ~kStVal) == kStInc);
        int stop = inc_mask ? (__ffs(inc_mask) - 1) : 31;
        uint32_t mine = (lane <= stop) ? (v & kStVal) : 0u;
        for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
        prefix += mine;
        if (inc_mask) break;
        pos -= 32;
    }
    return prefix;
}

// Block-wide exclusive scan of one uint32 per thread (blockDim.x multiple of
// 32, at most 1024).  `scratch` holds >= 33 words of shared memory.  Returns
// the exclusive prefix; *total receives the block sum (all threads).
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* scratch,
                                                         uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) scratch[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = (lane < nwarps) ? scratch[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nwarps) scratch[lane] = w;  // inclusive per-warp totals
        if (lane == 31) scratch[32] = w;
    }
    __syncthreads();
    uint32_t warp_prefix = warp ? scratch[warp - 1] : 0u;
    *total = scratch[32];
    uint32_t r = warp_prefix + x - v;
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// device-side scene (structure of arrays, levels concatenated)
// ---------------------------------------------------------------------------
struct DevScene {
    int64_t n_total = 0;
    int32_t num_levels = 0;
    int32_t sh_degree = 3;
    int32_t filter2d = 0;   // 1: opacity-compensated 2D filter
    int64_t level_off[kMaxLevels + 1] = {0};
    float filter_var[kMaxLevels] = {0};
    const float* mx = nullptr;   // means, one plane per axis
    const float* my = nullptr;
    const float* mz = nullptr;
    const float4* scale_op = nullptr;  // (s0, s1, s2, opacity), activated
    const float4* quat = nullptr;      // unit (w, x, y, z)
    const float4* sh = nullptr;        // 12 planes of n_total float4 (48 coeffs)
};

// camera as seen by kernels
struct DevCamera {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int32_t width, height;
    float znear;
    // lateral limits of the EWA Jacobian's evaluation point: x/z and y/z are
    // clamped to +-1.3 tan(fov/2), tan(fovx/2) = W / (2 fx) (the 3DGS
    // rasteriser's clamp), formed in FP64 and rounded to FP32
    float limx, limy;
    // camera-relative evaluation: p = R (mu - chat) + tp, with chat = (float)
    // centre and tp = t + R chat formed in FP64; clo = centre - chat
    float chat[3];
    float tp[3];
    float clo[3];
    int32_t tiles_x, tiles_y;
};

// ---------------------------------------------------------------------------
// kernel launchers (defined in the .cu files)
// ---------------------------------------------------------------------------
struct SortScratch;

// K1: Eq. 2 stream compaction.  thr_lo/thr_hi: per level squared distance
// bounds in FP32.  Writes selected gids (ascending) to out, count to
// *d_count.  status must hold ceil(n / kSelectTile) words, zeroed, plus one
// tile counter at status_counter (zeroed).
constexpr int kSelectThreads = 256;
constexpr int kSelectIPT = 16;
constexpr int kSelectTile = kSelectThreads * kSelectIPT;
void launch_lod_select(const DevScene& sc, const float c32[3], const float* thr_lo,
                       const float* thr_hi, uint32_t* out, uint32_t* d_count, uint32_t* status,
                       uint32_t* tile_counter, uint32_t* err, cudaStream_t s);


// Visibility filtering: entries of list (n, gid ascending) whose score[gid]
// (n_total floats) is >= thr, compacted in order into out; *d_count = kept.
void launch_score_filter(const uint32_t* list, int64_t n, const float* score, float thr,
                         int64_t n_total, uint32_t* out, uint32_t* d_count, uint32_t* status,
                         uint32_t* tile_counter, uint32_t* err, cudaStream_t s);

// K2: union of two gid-ascending lists with membership flags (bit 31 = A,
// bit 30 = B).  marks: n_total bytes of scratch.
void launch_chunk_union(const uint32_t* a, int64_t na, const uint32_t* b, int64_t nb,
                        int64_t n_total, uint8_t* marks, uint32_t* out, uint32_t* d_count,
                        uint32_t* status, uint32_t* tile_counter, uint32_t* err, cudaStream_t s);

// K3: projection + SH + visibility compaction.
struct ProjectOut {
    float4* rec_a;      // (mean'x, mean'y, u00, u01)
    float4* rec_b;      // (u11, log2 opacity', r, g)
    float* rec_c;       // b
    uint2* rec_rect;    // pixel range (x0 | y0 << 16, x1 | y1 << 16), inclusive
    uint32_t* rec_gid;  // gid of the record
    uint32_t* depth_key;  // FP32 depth bits (sort key), index = record
    uint32_t* depth_val;  // record index
    uint32_t* counts;     // 8-byte aligned: [0] = visible (u32), [2..3] = tile keys (u64),
                          // [4..5] = bin keys (u64, only when bin_log2 > 0)
    int32_t bin_log2 = 0; // bins of 2^bin_log2 x 2^bin_log2 tiles (see launch_emit)
    uint32_t* depth_hist = nullptr;  // null, or 4 x 256 zeroed words: += the digit counts
                                     // of the visible records' depth keys (the depth sort's)
};
constexpr int kProjThreads = 256;
// look-back status words of the projection: one per CTA of kProjThreads entries
inline int64_t proj_status_words(int64_t n_active) {
    return std::max<int64_t>((n_active + kProjThreads - 1) / kProjThreads, 1);
}
// Attribute sources for streamed scenes: list entries index into chunk block
// A (bit 31) or B, whose gid lists give the Gaussians' gids.
struct ProjSources {
    DevScene a, b;
    const uint32_t* gid_a = nullptr;
    const uint32_t* gid_b = nullptr;
    int64_t n_a = 0, n_b = 0, npad_a = 0, npad_b = 0;
};
void launch_project(const DevScene& sc, const DevCamera& cam, const uint32_t* list,
                    int64_t n_active, float tA, float tB, const ProjectOut& o, uint32_t* status,
                    uint32_t* tile_counter, uint32_t* err, cudaStream_t s,
                    const ProjSources* src = nullptr);
// copy the extent table to this device's constant memory (once per device)
cudaError_t upload_qtable(const float* q65);

// K10: per-candidate tile-key counts of the greedy depth-threshold search for
// one view over the Gaussians of levels 0..lvl (n = level_off[lvl + 1]).
// lo/hi: squared Eq. 2 bands of the fixed levels (lo also for level lvl - 1);
// c: camera centre rounded to FP32; d_thr: K ascending squared candidates
// (device); acc: 2K + 2 zeroed counters (bucket layout in k_project.cu).
struct ThreshBands {
    float lo[kMaxLevels];
    float hi[kMaxLevels];
    float c[3];
};
constexpr int kMaxThreshCandidates = 1024;
size_t threshold_cost_smem(int K);
void launch_threshold_cost(const DevScene& sc, const DevCamera& cam, int64_t n, int lvl,
                           const ThreshBands& b, const float* d_thr, int K, unsigned long long* acc,
                           cudaStream_t s);

// onesweep LSD radix sort of u32 keys (and u32 values if vals != null) on
// key bits [shift0, shift0 + key_bits).  Result lands in (keys, vals) or
// (keys_alt, vals_alt): the return value says which (0 = keys/vals).
constexpr int kSortThreads = 256;
constexpr int kSortIPT = 15;
constexpr int kSortTile = kSortThreads * kSortIPT;
// inputs of at most kSortSmallMax pairs use tiles of kSortTileSmall pairs
constexpr int kSortTileSmall = kSortThreads * 4;
constexpr int64_t kSortSmallMax = 1ll << 20;
constexpr int64_t sort_tile_for(int64_t n) { return n <= kSortSmallMax ? kSortTileSmall : kSortTile; }
// scratch words: 4 x 256 digit offsets, 32 tile counters, look-back words
constexpr int64_t sort_scratch_words(int64_t n, int passes) {
    return 4 * 256 + 32 + (int64_t)passes * ((n + sort_tile_for(n) - 1) / sort_tile_for(n)) * 256;
}
// digit_offsets: optional exclusive per-pass digit offsets (passes x 256)
// that replace the upfront histogram; final_keys = false skips writing the
// keys in the last pass (only the values are wanted).  ranges: for a sort by
// tile (tile = key >> shift0), the last pass also records each tile's
// [begin, end) in the output for tiles < range_tiles; .x must start at
// 0xffffffff and .y at 0 (a tile without keys keeps begin > end).  Not
// written if n <= 1.  d_count: optional device word (u64) holding the number
// of pairs, at most n; n is then a capacity that sizes the grid and the
// scratch, tiles past the count exit at once, and digit_offsets must be
// given (the sort then runs for any count, 0 and 1 included).
// scratch_cleared: the caller has zeroed the scratch (no memset here).
// digit_counts: digit_offsets holds the per-pass digit counts instead, which
// each pass scans itself (no separate scan launch).
size_t sort_scratch_bytes(int64_t n, int key_bits);
int launch_onesweep(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                    int64_t n, int key_bits, void* scratch, uint32_t* err, cudaStream_t s,
                    const uint32_t* digit_offsets = nullptr, bool final_keys = true, int shift0 = 0,
                    uint2* ranges = nullptr, uint32_t range_tiles = 0,
                    const unsigned long long* d_count = nullptr, bool scratch_cleared = false,
                    bool digit_counts = false);
int onesweep_launches(int64_t n, int key_bits, bool offsets_supplied);

// K4: emit (bin, record) pairs in depth order.  A bin is a square of
// 2^bin_log2 x 2^bin_log2 tiles (bin_log2 = 0: the 16x16 tile itself), bins_x
// per image row; a record goes to every bin its tile rect touches.  koff:
// n_vis + 1 words; srec / srect: n_vis gathered record ids and bin rects;
// n_keys (bin keys) from the projection's count.  digit_hist (zeroed,
// 4 x 256 words) receives the exclusive digit offsets of the bin sort on
// key_bits bin bits.  rbits > 0: one packed word per pair,
// bin << rbits | record (tile_val unused); rbits = 0: bin in tile_key,
// record in tile_val.
constexpr int kEmitThreads = 256;
constexpr int kEmitKeysPerCta = 2048;   // slice of the key list (small records)
constexpr int64_t kEmitWarpMinKeys = 32;  // mean keys per record for one warp per record
void launch_emit(const uint32_t* sorted_rec, int64_t n_vis, const uint2* rec_rect,
                 int32_t bins_x, int bin_log2, uint32_t* koff, uint32_t* srec, uint2* srect,
                 int64_t n_keys, uint32_t* tile_key, uint32_t* tile_val, int rbits, int key_bits,
                 uint32_t* digit_hist, uint32_t* status, uint32_t* tile_counter, uint32_t* err,
                 cudaStream_t s);
// The same emission with the counts on the device (one fused launch, or
// count / scan / write above a 2^21-record capacity; bins of any size,
// per-tile lists included): n_vis_cap and key_cap are capacities
// (key_tile/tile_val hold key_cap words); d_nvis and d_nkeys (u64) the
// frame's visible records and bin keys.  digit_hist receives the bin sort's
// digit counts, not scanned (launch_onesweep with digit_counts scans them).
// A frame whose keys exceed key_cap writes none and sets kErrOverflow.
// Returns the launches.
int launch_emit_counted(const uint32_t* sorted_rec, int64_t n_vis_cap, const unsigned long long* d_nvis,
                         const uint2* rec_rect, int32_t bins_x, int bin_log2, int64_t key_cap,
                         const unsigned long long* d_nkeys, uint32_t* tile_key, uint32_t* tile_val,
                         int rbits, int key_bits, uint32_t* digit_hist, uint32_t* status,
                         uint32_t* tile_counter, uint32_t* err, cudaStream_t s);

int emit_launches(int64_t n_vis, int64_t n_keys, int bin_log2);
// exclusive scan, in place, of `passes` 256-bin digit histograms (one launch)
void launch_digit_scan(uint32_t* hist, int passes, cudaStream_t s);

// K6: per tile [begin, end) of the sorted keys (tile = key >> shift);
// ranges zeroed by the caller.
void launch_ranges(const uint32_t* tile_key, int64_t n_keys, uint2* ranges, int64_t ntiles,
                   int shift, cudaStream_t s);

// Alpha of a projection record at a pixel (Eq. 1 with the record's
// Cholesky form): alpha = min(0.99, 2^(log2 o' - (u00 dx + u01 dy)^2 -
// (u11 dy)^2)), a = (mean', u00, u01), b = (u11, log2 o', ...).  The
// compositing thread owns the pixels of rows y and y + 4 of an 8-row block
// and forms the second row's t and w from the first's by the row step (one
// FMA each), so a pixel whose row within its tile has bit 2 set takes that
// form here too: every walk (compositing, adjoint, importance) then decides
// skip and stop on the same FP32 values.  t and w are returned for the
// adjoint.
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float alpha_of(float4 b, float t, float w) {
    return fminf(0.99f, ex2_approx(fmaf(-t, t, fmaf(-w, w, b.y))));
}
// t and w at row py0 (a pixel-centre y) and at py0 + 4
__device__ __forceinline__ void row_pair_tw(float4 a, float4 b, float dx, float py0, float& t0, float& w0,
                                            float& t1, float& w1) {
    const float dy = py0 - a.y;
    t0 = fmaf(a.z, dx, a.w * dy);
    w0 = b.x * dy;
    t1 = fmaf(4.f, a.w, t0);
    w1 = fmaf(4.f, b.x, w0);
}
// t and w at pixel row y (image row; tiles start at multiples of 16, so bit
// 2 of y is bit 2 of the row within the tile)
__device__ __forceinline__ void pixel_tw(float4 a, float4 b, float dx, int y, float& t, float& w) {
    float t0, w0, t1, w1;
    if (y & 4) {
        row_pair_tw(a, b, dx, (float)(y - 4) + 0.5f, t0, w0, t1, w1);
        t = t1;
        w = w1;
    } else {
        row_pair_tw(a, b, dx, (float)y + 0.5f, t0, w0, t1, w1);
        t = t0;
        w = w0;
    }
}

// K7: per tile front-to-back compositing.
struct BlendOut {
    float* rgb;        // H x W x 3
    float* T_final;    // H x W (may be null)
    uint32_t* last;    // H x W (may be null): keys processed up to the last blended one
};
// tile_val[i] & vmask is the record of sorted pair i (vmask = all ones for
// separate values, the low rbits for packed keys).
// bin_log2 > 0: ranges and keys are per bin of 2^bin_log2 x 2^bin_log2
// tiles (launch_emit); a tile walks its bin's list and skips the records
// whose tile rect (from rec_rect) misses it, which leaves exactly the
// tile's own list, in the same order.
void launch_blend(const DevCamera& cam, const uint2* ranges, const uint32_t* tile_val, uint32_t vmask,
                  int64_t n_keys, const float4* rec_a, const float4* rec_b, const float* rec_c,
                  int64_t n_rec, const BlendOut& o, cudaStream_t s, int bin_log2 = 0,
                  const uint2* rec_rect = nullptr, unsigned long long* pairs = nullptr,
                  uint32_t* tile_ctr = nullptr);
// tile_ctr (a zeroed device word) makes the compositing a grid of
// kBlendCtasPerSM CTAs per SM that take tiles from the counter, so that
// other streams' kernels keep room on every SM while it runs (used when
// frames of other slots run at the same time; a lone frame takes one CTA
// per tile and the whole GPU).  Measured with 1080p chunk
// frames on four streams: 2 / 3 / 4 / 6 / 8 / 12 CTAs per SM gave 5790 /
// 5936 / 5894 / 5775 / 5706 / 5729 frames/s; the single-frame compositing
// time grows from 0.081 ms at 8 to 0.090 ms at 4).
constexpr int kBlendCtasPerSM = 4;
// Everything one frame's compositing reads and writes; a batch of frames is
// composited by one launch over all their tiles (at most kMaxBlendBatch);
// frames of a batch write images only (no T_final, no last).
struct BlendFrame {
    int32_t width, height, tiles_x, ntiles;
    uint32_t tile_base;        // first tile of this frame in a batch launch
    uint32_t vmask, n_keys, n_rec;
    int32_t bin_log2, bins_x;  // key lists per bin of 2^bin_log2 tiles square
    const uint2* ranges;       // per bin
    const uint32_t* tile_val;
    const uint2* rec_rect;     // pixel ranges (read when bin_log2 > 0)
    unsigned long long* pairs; // null, or [0] += pairs evaluated, [1] += pairs composited
    const float4* rec_a;
    const float4* rec_b;
    const float* rec_c;
    float* rgb;
    float* T_final;
    uint32_t* last;
};
constexpr int kMaxBlendBatch = 64;
struct BlendBatch {
    int32_t n;
    BlendFrame f[kMaxBlendBatch];
};
BlendFrame blend_frame(const DevCamera& cam, const uint2* ranges, const uint32_t* tile_val, uint32_t vmask,
                       int64_t n_keys, const float4* rec_a, const float4* rec_b, const float* rec_c,
                       int64_t n_rec, const BlendOut& o, int bin_log2 = 0, const uint2* rec_rect = nullptr);
// One launch composites every frame's tiles.  With tile_ctr (a zeroed device
// word) the launch is persistent: a grid of a few CTAs per SM takes (frame,
// tile) items from the counter until all are done; without it, one CTA per
// tile.
void launch_blend_batch(const BlendFrame* frames, int n, cudaStream_t s, uint32_t* tile_ctr = nullptr);

// K12: importance score: the blend's walk, and per record the largest
// weight T * alpha it receives (rec_score, n_rec words, zeroed, FP32 bits),
// then score[gid] (n_total floats, non-negative) raised to it.  rgb as in
// launch_blend.
void launch_importance(const DevCamera& cam, const uint2* ranges, const uint32_t* tile_val,
                       uint32_t vmask, int64_t n_keys, const float4* rec_a, const float4* rec_b,
                       const float* rec_c, int64_t n_rec, const uint32_t* rec_gid, float* rgb,
                       uint32_t* rec_score, int64_t n_total, float* score, cudaStream_t s);

// K8 / K9: adjoint of compositing and projection (fine-tuning path).
// grec: 9 x n_rec doubles, zeroed: d(mean'x, mean'y, u00, u01, u11, o', r, g, b).
void launch_blend_bwd(const DevCamera& cam, const uint2* ranges, const uint32_t* tile_val,
                      uint32_t vmask, int64_t n_keys, const float4* rec_a, const float4* rec_b, const float* rec_c,
                      int64_t n_rec, const float* T_final, const uint32_t* last,
                      const float* dL_drgb, double* grec, cudaStream_t s);
// Levels of a parameter frame as the adjoint sees them: the Eq. 3 filter
// variance of each level (gid ranges level_off) and the trained level's gid
// range [train_lo, train_hi).  Records outside it get no gradient; the raw
// parameter and gradient arrays hold the trained level only and are indexed
// by gid - train_lo (the activated arrays by gid).
struct BwdLevels {
    int32_t num_levels = 1;
    int64_t level_off[kMaxLevels + 1] = {0};
    float filter_var[kMaxLevels] = {0};
    int64_t train_lo = 0, train_hi = 0;
};
void launch_project_bwd(const DevCamera& cam, int64_t n_rec, const uint32_t* rec_gid,
                        const double* grec, const float* means, const float4* act_so,
                        const float4* act_q, const float* quats, const float* sh, int sh_degree,
                        const BwdLevels& lv, float* g_means, float* g_log_scales, float* g_quats,
                        float* g_logits, float* g_sh, cudaStream_t s);

// SM count of the current device (queried once per device; 152 on GB300),
// for grids sized as a multiple of the SMs
int device_sms();

// records msg as the calling thread's lodge_last_error message; returns s
lodge_status set_error(lodge_status s, const char* msg);

// Q table for the opacity-aware extent (65 entries), host-computed.
void fill_qtable(float* q65);

}  // namespace lodge
