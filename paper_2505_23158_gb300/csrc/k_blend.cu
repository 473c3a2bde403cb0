// K7: per-tile front-to-back alpha compositing (Eq. 1; Sec. 3
// "Preliminaries: 3DGS").  One CTA of 128 threads per 16x16 tile, two pixels
// per thread (one column, 4 rows apart), so each record read from shared
// memory serves two pixels; each warp covers an 8x8 block so that its
// pixels terminate together.  The tile's Gaussians arrive in batches of 128
// records, gathered from the projection records into shared memory with
// cp.async and double-buffered (batch b+1 is in flight while batch b is
// composited).  A pixel stops at the first Gaussian that would take its
// transmittance below 1e-4; a warp whose 64 pixels have all stopped skips
// the batch, and the CTA leaves as soon as all 256 have stopped.
//
// Frames that keep neither the final transmittance nor list positions take
// the filtered walk: each batch also stages the records' pixel rects, and
// every warp ballots which of the 128 records have a pixel rect meeting its
// own 8x8 block and an ellipse reaching one of its pixel centres
// (splat_meets_block), and visits only those, in list order.  A record
// failing either test would be skipped by every pixel of the block (alpha <
// 1/255 there), so the image is the unfiltered walk's bit for bit.
// With coarse bins (squares of 2^bin_log2 tiles) the tile walks its bin's
// key list the same way (a record meeting the block has a tile rect holding
// the tile, so it is on the tile's own list).  This walk is branch-free: a
// pixel that stops gets T = 0, which makes every later step a no-op.
//
// Per pixel and Gaussian (record = mean', upper-triangular U with
// U^T U = (1/2) log2(e) Sigma'^-1, log2 o', colour):
//   q = (u00 dx + u01 dy)^2 + (u11 dy)^2,  alpha = min(0.99, 2^(log2 o' - q))
//   (= o' 2^-q; the exponent is formed by two FMAs and the product is saved)
//   skip if alpha < 1/255; T' = T (1 - alpha); stop if T' < 1e-4;
//   C += T alpha rgb; T = T'.
#include "common.cuh"

namespace lodge {

namespace {

constexpr int kBatch = 256;        // importance kernel: records per batch
constexpr int kBlendThreads = 128; // blend: two pixels per thread
constexpr int kBlendBatch = 128;   // blend: records per batch (one per thread)


__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }

// one record of the batch against one pixel (Eq. 1); kCount: count the
// evaluation and, if the pixel composites it, the composited pair
template <bool kCount, bool kLast>
__device__ __forceinline__ void blend_px(const float alpha, const float4 bb, const float cz, float& T,
                                         float& C0, float& C1, float& C2, bool& done, uint32_t& last,
                                         uint32_t pos, uint32_t& n_eval, uint32_t& n_used) {
    if (kCount) ++n_eval;
    if (alpha >= (1.0f / 255.0f)) {
        const float Tn = T * (1.f - alpha);
        if (Tn < 1e-4f) {
            done = true;
        } else {
            const float wgt = T * alpha;
            C0 = fmaf(wgt, bb.z, C0);
            C1 = fmaf(wgt, bb.w, C1);
            C2 = fmaf(wgt, cz, C2);
            T = Tn;
            if (kLast) last = pos;
            if (kCount) ++n_used;
        }
    }
}

// The same step without branches, for walks that need neither the final
// transmittance nor list positions: a pixel that stops gets T = 0, after
// which every step leaves it unchanged (its weight is 0 and T stays 0).
// While T > 0 the arithmetic and decisions are blend_px's.
template <bool kCount>
__device__ __forceinline__ void blend_px_flat(const float alpha, const float4 bb, const float cz, float& T,
                                              float& C0, float& C1, float& C2, uint32_t& n_eval,
                                              uint32_t& n_used) {
    const float Tn = T * (1.f - alpha);
    const bool ok = alpha >= (1.0f / 255.0f);
    const bool go = ok && !(Tn < 1e-4f);
    const float wgt = go ? T * alpha : 0.f;
    C0 = fmaf(wgt, bb.z, C0);
    C1 = fmaf(wgt, bb.w, C1);
    C2 = fmaf(wgt, cz, C2);
    if (kCount) {
        n_eval += T > 0.f ? 1u : 0u;
        n_used += go ? 1u : 0u;
    }
    T = go ? Tn : (ok ? 0.f : T);
}

// Whether a splat can reach alpha >= 1/255 at some pixel centre of an 8x8
// block whose first pixel centre is (bx, by).  With d = p - mean' and
// q(d) = (u00 dx + u01 dy)^2 + (u11 dy)^2 (the exponent's quadratic, a convex
// function with its minimum 0 at d = 0), the least q over the centres' box
// [bx, bx + 7] x [by, by + 7] lies on the line dx = xc or on dy = yc, where
// xc, yc are the box coordinates nearest the mean (0 where the box spans it):
// along each line q is a one-dimensional quadratic whose minimiser is
// clamped to the box.  A pixel centre can pass the 1/255 skip only if
// q <= log2 o' + log2 255; the test adds a margin of 0.01 (in log2 units)
// for the rounding of q, so it never drops a record that some pixel of the
// block would composite, and the walk's result is the unfiltered walk's.
__device__ __forceinline__ bool splat_meets_block(const float4 a, const float4 b, float bx, float by) {
    constexpr float kLog2_255 = 7.99435343f;
    const float X0 = bx - a.x, X1 = X0 + 7.f, Y0 = by - a.y, Y1 = Y0 + 7.f;
    const float xc = fminf(fmaxf(0.f, X0), X1), yc = fminf(fmaxf(0.f, Y0), Y1);
    const float u00 = a.z, u01 = a.w, u11 = b.x;
    // on dx = xc the minimiser is dy = -u00 u01 xc / (u01^2 + u11^2)
    const float dy = fminf(fmaxf(__fdividef(-u00 * u01 * xc, fmaf(u01, u01, u11 * u11)), Y0), Y1);
    const float t1 = fmaf(u00, xc, u01 * dy), w1 = u11 * dy;
    // on dy = yc it is dx = -u01 yc / u00
    const float dx = fminf(fmaxf(__fdividef(-u01 * yc, u00), X0), X1);
    const float t2 = fmaf(u00, dx, u01 * yc), w2 = u11 * yc;
    const float q = fminf(fmaf(t1, t1, w1 * w1), fmaf(t2, t2, w2 * w2));
    return q <= b.y + (kLog2_255 + 0.01f);
}

template <bool kBins, bool kCount = false>
__device__ __forceinline__ void blend_tile(const BlendFrame& f, int tile) {
    __shared__ float4 sa[2][kBlendBatch];
    __shared__ float4 sb[2][kBlendBatch];
    __shared__ float sc[2][kBlendBatch];
    __shared__ uint2 sr[2][kBins ? kBlendBatch : 1];
    const int32_t width = f.width, height = f.height, tiles_x = f.tiles_x;
    const uint2* __restrict__ ranges = f.ranges;
    const uint32_t* __restrict__ tile_val = f.tile_val;
    const uint32_t vmask = f.vmask, n_keys = f.n_keys, n_rec = f.n_rec;
    const float4* __restrict__ rec_a = f.rec_a;
    const float4* __restrict__ rec_b = f.rec_b;
    const float* __restrict__ rec_c = f.rec_c;
    float* __restrict__ out_rgb = f.rgb;
    float* __restrict__ out_T = f.T_final;
    uint32_t* __restrict__ out_last = f.last;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // warp w covers the 8x8 block (w & 1, w >> 1) of the tile; a lane owns
    // two pixels of one column, 4 rows apart
    const int x = tx * kTile + (warp & 1) * 8 + (lane & 7);
    const int y0 = ty * kTile + (warp >> 1) * 8 + (lane >> 3), y1 = y0 + 4;
    const bool in0 = x < width && y0 < height, in1 = x < width && y1 < height;
    const float pxf = (float)x + 0.5f, py0 = (float)y0 + 0.5f;
    const uint32_t wx0 = tx * kTile + (warp & 1) * 8, wx1 = wx0 + 7;   // the warp's 8x8 block
    const uint32_t wy0 = ty * kTile + (warp >> 1) * 8, wy1 = wy0 + 7;
    const float bxf = (float)wx0 + 0.5f, byf = (float)wy0 + 0.5f;   // the block's first pixel centre
    const uint2* __restrict__ rec_rect = f.rec_rect;
    // the rect test needs the records' pixel rects (frames that keep the
    // final transmittance or positions have none); a frame of a filtered
    // batch launch may still have per-tile lists without rects
    const bool binned = kBins && rec_rect != nullptr;
    const int bin = (binned && f.bin_log2 > 0) ? (ty >> f.bin_log2) * f.bins_x + (tx >> f.bin_log2) : tile;
    uint2 rg = ranges[bin];
    if (rg.y > n_keys || rg.x > rg.y) rg = make_uint2(0, 0);  // never for a consistent sort
    const int n = (int)(rg.y - rg.x);
    const int nb = (n + kBlendBatch - 1) / kBlendBatch;

    // the binned walk marks a pixel outside the image or stopped by T = 0
    float T0 = (kBins && !in0) ? 0.f : 1.f, C00 = 0.f, C01 = 0.f, C02 = 0.f;
    float T1 = (kBins && !in1) ? 0.f : 1.f, C10 = 0.f, C11 = 0.f, C12 = 0.f;
    bool done0 = !in0, done1 = !in1;
    uint32_t last0 = 0, last1 = 0;
    uint32_t n_eval = 0, n_used = 0;   // counting mode only
    // per-pixel list positions are wanted only by the adjoint, whose frames
    // always have per-tile lists
    constexpr bool kLast = !kBins;

    if (nb > 0) {
        if (tid < n) {
            uint32_t j = min(tile_val[rg.x + tid] & vmask, n_rec - 1u);
            cp_async16(&sa[0][tid], rec_a + j);
            cp_async16(&sb[0][tid], rec_b + j);
            cp_async4(&sc[0][tid], rec_c + j);
            if (binned) cp_async8(&sr[0][tid], rec_rect + j);
        }
        cp_async_commit();
    }
    for (int b = 0; b < nb; ++b) {
        const int buf = b & 1;
        if (b + 1 < nb) {
            int k = (b + 1) * kBlendBatch + tid;
            if (k < n) {
                uint32_t j = min(tile_val[rg.x + k] & vmask, n_rec - 1u);
                cp_async16(&sa[buf ^ 1][tid], rec_a + j);
                cp_async16(&sb[buf ^ 1][tid], rec_b + j);
                cp_async4(&sc[buf ^ 1][tid], rec_c + j);
                if (binned) cp_async8(&sr[buf ^ 1][tid], rec_rect + j);
            }
        }
        cp_async_commit();
        cp_async_wait1();
        __syncthreads();
        const int cnt = min(kBlendBatch, n - b * kBlendBatch);
        if (kBins) {
            // which records of the batch can reach this warp's block: 4
            // ballots per warp
            uint32_t m[kBlendBatch / 32];
#pragma unroll
            for (int w = 0; w < kBlendBatch / 32; ++w) {
                const int k = w * 32 + lane;
                bool hit = k < cnt;
                if (hit && binned) {
                    // the record's pixel rect meets this warp's 8x8 block (so
                    // its tile rect holds the tile); outside the rect every
                    // pixel would skip it (alpha < 1/255), so no result changes
                    const uint2 r = sr[buf][k];
                    hit = (r.x & 0xffffu) <= wx1 && (r.y & 0xffffu) >= wx0 && (r.x >> 16) <= wy1 &&
                          (r.y >> 16) >= wy0;
                }
                // and its ellipse reaches a pixel centre of the block
                if (hit) hit = splat_meets_block(sa[buf][k], sb[buf][k], bxf, byf);
                m[w] = __ballot_sync(0xffffffffu, hit);
            }
            // flat walk over the hits, 8 batch positions at a time, the warp
            // leaving once all its pixels have stopped (T = 0)
            if (!__all_sync(0xffffffffu, T0 == 0.f && T1 == 0.f)) {
                // the hits in batch order, taken bit by bit from the masks
                // (a warp visits a quarter or less of a staged batch; a scan
                // over all 128 positions with a test each cost more)
                bool open = true;
#pragma unroll
                for (int w = 0; w < kBlendBatch / 32; ++w) {
                    uint32_t mw = open ? m[w] : 0u;
                    uint32_t cnt8 = 0;
                    while (mw) {
                        const int k = w * 32 + __ffs(mw) - 1;
                        mw &= mw - 1u;
                        const float4 a = sa[buf][k];
                        const float4 bb = sb[buf][k];
                        const float cz = sc[buf][k];
                        float t0, w0, t1, w1;
                        row_pair_tw(a, bb, pxf - a.x, py0, t0, w0, t1, w1);
                        blend_px_flat<kCount>(alpha_of(bb, t0, w0), bb, cz, T0, C00, C01, C02, n_eval, n_used);
                        blend_px_flat<kCount>(alpha_of(bb, t1, w1), bb, cz, T1, C10, C11, C12, n_eval, n_used);
                        if ((++cnt8 & 7u) == 0u && __all_sync(0xffffffffu, T0 == 0.f && T1 == 0.f)) {
                            open = false;
                            break;
                        }
                    }
                }
            }
        } else if (!__all_sync(0xffffffffu, done0 && done1)) {
            for (int k = 0; k < cnt && !(done0 && done1); ++k) {
                const float4 a = sa[buf][k];
                const float4 bb = sb[buf][k];
                const float cz = sc[buf][k];
                const uint32_t pos = (uint32_t)(b * kBlendBatch + k + 1);
                float t0, w0, t1, w1;
                row_pair_tw(a, bb, pxf - a.x, py0, t0, w0, t1, w1);
                if (!done0)
                    blend_px<kCount, kLast>(alpha_of(bb, t0, w0), bb, cz, T0, C00, C01, C02, done0, last0, pos,
                                            n_eval, n_used);
                if (!done1)
                    blend_px<kCount, kLast>(alpha_of(bb, t1, w1), bb, cz, T1, C10, C11, C12, done1, last1, pos,
                                            n_eval, n_used);
            }
        }
        if (kBins) {
            if (__syncthreads_count(T0 == 0.f && T1 == 0.f) == kBlendThreads) break;
        } else if (__syncthreads_count(done0 && done1) == kBlendThreads) {
            break;
        }
    }
    cp_async_wait0();
    if (kCount) {
        for (int off = 16; off > 0; off >>= 1) {
            n_eval += __shfl_xor_sync(0xffffffffu, n_eval, off);
            n_used += __shfl_xor_sync(0xffffffffu, n_used, off);
        }
        if (lane == 0 && f.pairs) {
            atomicAdd(f.pairs, (unsigned long long)n_eval);
            atomicAdd(f.pairs + 1, (unsigned long long)n_used);
        }
    }
    if (in0) {
        const int64_t pix = (int64_t)y0 * width + x;
        out_rgb[3 * pix + 0] = C00;
        out_rgb[3 * pix + 1] = C01;
        out_rgb[3 * pix + 2] = C02;
        if (!kBins && out_T) out_T[pix] = T0;
        if (kLast && out_last) out_last[pix] = last0;
    }
    if (in1) {
        const int64_t pix = (int64_t)y1 * width + x;
        out_rgb[3 * pix + 0] = C10;
        out_rgb[3 * pix + 1] = C11;
        out_rgb[3 * pix + 2] = C12;
        if (!kBins && out_T) out_T[pix] = T1;
        if (kLast && out_last) out_last[pix] = last1;
    }
}

template <bool kBins, bool kCount>
__global__ void __launch_bounds__(kBlendThreads) blend_kernel(BlendFrame f) {
    blend_tile<kBins, kCount>(f, blockIdx.x);
}

// fewer CTAs than tiles: each takes the next tile from the counter
template <bool kBins, bool kCount>
__global__ void __launch_bounds__(kBlendThreads) blend_loop_kernel(BlendFrame f, uint32_t* __restrict__ tile_ctr) {
    __shared__ int s_t;
    for (;;) {
        if (threadIdx.x == 0) s_t = (int)atomicAdd(tile_ctr, 1u);
        __syncthreads();
        const int t = s_t;
        __syncthreads();   // s_t is rewritten for the next tile
        if (t >= f.ntiles) break;
        blend_tile<kBins, kCount>(f, t);
    }
}

// One launch for the tiles of several frames (a serving step): CTA b
// composites tile b - tile_base of the last frame whose tile_base <= b.
template <bool kBins>
__global__ void __launch_bounds__(kBlendThreads) blend_batch_kernel(BlendBatch bb) {
    const uint32_t b = blockIdx.x;
    int lo = 0, hi = bb.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bb.f[mid].tile_base <= b) lo = mid; else hi = mid - 1;
    }
    blend_tile<kBins>(bb.f[lo], (int)(b - bb.f[lo].tile_base));
}

// The same as a persistent grid: each CTA takes the next (frame, tile) item
// of the step from the counter until all `total` are done.
template <bool kBins>
__global__ void __launch_bounds__(kBlendThreads) blend_batch_loop_kernel(BlendBatch bb, uint32_t total,
                                                                         uint32_t* __restrict__ tile_ctr) {
    __shared__ uint32_t s_t;
    for (;;) {
        if (threadIdx.x == 0) s_t = atomicAdd(tile_ctr, 1u);
        __syncthreads();
        const uint32_t b = s_t;
        __syncthreads();   // s_t is rewritten for the next item
        if (b >= total) break;
        int lo = 0, hi = bb.n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (bb.f[mid].tile_base <= b) lo = mid; else hi = mid - 1;
        }
        blend_tile<kBins>(bb.f[lo], (int)(b - bb.f[lo].tile_base));
    }
}


// K12: importance score (Sec. 3 "Importance pruning" / "Visibility
// filtering", after RadSplat): the same per-pixel walk as blend_kernel (same
// decisions, same arithmetic), and for every composited (pixel, record)
// pair the blending weight T * alpha; each warp takes the maximum over its
// 32 pixels and raises rec_score[record] (FP32 bits, non-negative, so the
// unsigned maximum is the float maximum).  The image is written as well.
// Lanes stay converged over the batch so the warp maximum can be taken per
// record; a warp leaves the batch once all its pixels have stopped.
__global__ void __launch_bounds__(256)
importance_kernel(int32_t width, int32_t height, int32_t tiles_x, const uint2* __restrict__ ranges,
                  const uint32_t* __restrict__ tile_val, uint32_t vmask, uint32_t n_keys,
                  uint32_t n_rec, const float4* __restrict__ rec_a, const float4* __restrict__ rec_b,
                  const float* __restrict__ rec_c, float* __restrict__ out_rgb,
                  uint32_t* __restrict__ rec_score) {
    __shared__ float4 sa[kBatch];
    __shared__ float4 sb[kBatch];
    __shared__ float sc[kBatch];
    __shared__ uint32_t sr[kBatch];
    const int tile = blockIdx.x;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x = tx * kTile + (warp & 1) * 8 + (lane & 7);
    const int y = ty * kTile + (warp >> 1) * 4 + (lane >> 3);
    const bool inside = x < width && y < height;
    const float pxf = (float)x + 0.5f;
    uint2 rg = ranges[tile];
    if (rg.y > n_keys || rg.x > rg.y) rg = make_uint2(0, 0);
    const int n = (int)(rg.y - rg.x);
    const int nb = (n + kBatch - 1) / kBatch;
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    bool done = !inside;
    for (int b = 0; b < nb; ++b) {
        __syncthreads();
        const int k0 = b * kBatch + tid;
        if (k0 < n) {
            const uint32_t j = min(tile_val[rg.x + k0] & vmask, n_rec - 1u);
            sr[tid] = j;
            sa[tid] = rec_a[j];
            sb[tid] = rec_b[j];
            sc[tid] = rec_c[j];
        }
        __syncthreads();
        const int cnt = min(kBatch, n - b * kBatch);
        for (int k = 0; k < cnt; ++k) {
            if (__all_sync(0xffffffffu, done)) break;
            float w = 0.f;
            if (!done) {
                const float4 a = sa[k];
                const float4 bb = sb[k];
                float t, wq;
                pixel_tw(a, bb, pxf - a.x, y, t, wq);
                const float alpha = alpha_of(bb, t, wq);
                if (alpha >= (1.0f / 255.0f)) {
                    const float Tn = T * (1.f - alpha);
                    if (Tn < 1e-4f) {
                        done = true;
                    } else {
                        w = T * alpha;
                        C0 = fmaf(w, bb.z, C0);
                        C1 = fmaf(w, bb.w, C1);
                        C2 = fmaf(w, sc[k], C2);
                        T = Tn;
                    }
                }
            }
            const uint32_t wmax = __reduce_max_sync(0xffffffffu, __float_as_uint(w));
            if (lane == 0 && wmax) atomicMax(rec_score + sr[k], wmax);
        }
        if (__syncthreads_count(done) == 256) break;
    }
    if (inside) {
        const int64_t pix = (int64_t)y * width + x;
        out_rgb[3 * pix + 0] = C0;
        out_rgb[3 * pix + 1] = C1;
        out_rgb[3 * pix + 2] = C2;
    }
}

// raise score[gid] to each record's score
__global__ void record_score_to_gid_kernel(const uint32_t* __restrict__ rec_score,
                                           const uint32_t* __restrict__ rec_gid, int64_t n_rec,
                                           int64_t n_total, uint32_t* __restrict__ score) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rec) return;
    const uint32_t v = rec_score[r];
    const uint32_t g = rec_gid[r];
    if (v && (int64_t)g < n_total) atomicMax(score + g, v);
}
}  // namespace

BlendFrame blend_frame(const DevCamera& cam, const uint2* ranges, const uint32_t* tile_val, uint32_t vmask,
                       int64_t n_keys, const float4* rec_a, const float4* rec_b, const float* rec_c,
                       int64_t n_rec, const BlendOut& o, int bin_log2, const uint2* rec_rect) {
    BlendFrame f;
    f.width = cam.width;
    f.height = cam.height;
    f.tiles_x = cam.tiles_x;
    f.ntiles = cam.tiles_x * cam.tiles_y;
    f.tile_base = 0;
    f.vmask = vmask;
    f.n_keys = (uint32_t)n_keys;
    f.n_rec = (uint32_t)std::max<int64_t>(n_rec, 1);
    // the filtered walk keeps neither the final transmittance nor positions
    const bool filt = rec_rect && !o.T_final && !o.last;
    f.bin_log2 = filt ? bin_log2 : 0;
    f.bins_x = (cam.tiles_x + (1 << f.bin_log2) - 1) >> f.bin_log2;
    f.ranges = ranges;
    f.tile_val = tile_val;
    f.rec_rect = filt ? rec_rect : nullptr;
    f.pairs = nullptr;
    f.rec_a = rec_a;
    f.rec_b = rec_b;
    f.rec_c = rec_c;
    f.rgb = o.rgb;
    f.T_final = o.T_final;
    f.last = o.last;
    return f;
}

void launch_blend(const DevCamera& cam, const uint2* ranges, const uint32_t* tile_val, uint32_t vmask,
                  int64_t n_keys, const float4* rec_a, const float4* rec_b, const float* rec_c,
                  int64_t n_rec, const BlendOut& o, cudaStream_t s, int bin_log2, const uint2* rec_rect,
                  unsigned long long* pairs, uint32_t* tile_ctr) {
    BlendFrame f = blend_frame(cam, ranges, tile_val, vmask, n_keys, rec_a, rec_b, rec_c, n_rec, o,
                               bin_log2, rec_rect);
    if (f.ntiles == 0) return;
    f.pairs = pairs;
    unsigned grid = (unsigned)f.ntiles;
    if (tile_ctr) {
        grid = (unsigned)std::min<int64_t>(f.ntiles, (int64_t)device_sms() * kBlendCtasPerSM);
    }
    const bool filt = f.rec_rect != nullptr;
    if (tile_ctr) {
        if (pairs) {   // counting variant (profiling), same walk
            if (filt)
                blend_loop_kernel<true, true><<<grid, kBlendThreads, 0, s>>>(f, tile_ctr);
            else
                blend_loop_kernel<false, true><<<grid, kBlendThreads, 0, s>>>(f, tile_ctr);
        } else if (filt) {
            blend_loop_kernel<true, false><<<grid, kBlendThreads, 0, s>>>(f, tile_ctr);
        } else {
            blend_loop_kernel<false, false><<<grid, kBlendThreads, 0, s>>>(f, tile_ctr);
        }
    } else if (pairs) {
        if (filt)
            blend_kernel<true, true><<<grid, kBlendThreads, 0, s>>>(f);
        else
            blend_kernel<false, true><<<grid, kBlendThreads, 0, s>>>(f);
    } else if (filt) {
        blend_kernel<true, false><<<grid, kBlendThreads, 0, s>>>(f);
    } else {
        blend_kernel<false, false><<<grid, kBlendThreads, 0, s>>>(f);
    }
}

void launch_blend_batch(const BlendFrame* frames, int n, cudaStream_t s, uint32_t* tile_ctr) {
    BlendBatch bb;
    uint32_t base = 0;
    bb.n = 0;
    bool bins = false;   // the filtered walk also serves frames without rects
    for (int i = 0; i < n && i < kMaxBlendBatch; ++i) {
        if (frames[i].ntiles == 0) continue;
        bb.f[bb.n] = frames[i];
        bb.f[bb.n].tile_base = base;
        base += (uint32_t)frames[i].ntiles;
        bins = bins || frames[i].rec_rect != nullptr;
        ++bb.n;
    }
    if (bb.n == 0) return;
    if (tile_ctr) {
        // as many CTAs as fit on the device at once (the step's compositing
        // runs after every frame's earlier stages)
        int per_sm = 1;
        const int nsm = device_sms();
        if (bins)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, blend_batch_loop_kernel<true>, kBlendThreads, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, blend_batch_loop_kernel<false>, kBlendThreads, 0);
        const unsigned grid = (unsigned)std::min<int64_t>((int64_t)base, (int64_t)nsm * std::max(per_sm, 1));
        if (bins)
            blend_batch_loop_kernel<true><<<grid, kBlendThreads, 0, s>>>(bb, base, tile_ctr);
        else
            blend_batch_loop_kernel<false><<<grid, kBlendThreads, 0, s>>>(bb, base, tile_ctr);
        return;
    }
    if (bins)
        blend_batch_kernel<true><<<base, kBlendThreads, 0, s>>>(bb);
    else
        blend_batch_kernel<false><<<base, kBlendThreads, 0, s>>>(bb);
}

void launch_importance(const DevCamera& cam, const uint2* ranges, const uint32_t* tile_val,
                       uint32_t vmask, int64_t n_keys, const float4* rec_a, const float4* rec_b,
                       const float* rec_c, int64_t n_rec, const uint32_t* rec_gid, float* rgb,
                       uint32_t* rec_score, int64_t n_total, float* score, cudaStream_t s) {
    const int ntiles = cam.tiles_x * cam.tiles_y;
    if (ntiles == 0) return;
    importance_kernel<<<ntiles, 256, 0, s>>>(cam.width, cam.height, cam.tiles_x, ranges, tile_val, vmask,
                                             (uint32_t)n_keys, (uint32_t)std::max<int64_t>(n_rec, 1),
                                             rec_a, rec_b, rec_c, rgb, rec_score);
    if (n_rec > 0)
        record_score_to_gid_kernel<<<(unsigned)((n_rec + 255) / 256), 256, 0, s>>>(
            rec_score, rec_gid, n_rec, n_total, reinterpret_cast<uint32_t*>(score));
}

}  // namespace lodge
