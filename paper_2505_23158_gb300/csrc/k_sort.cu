// K5: stable LSD radix sort of u32 keys, with or without u32 values,
// "onesweep" style: the digit histograms are known before the first pass (one
// upfront histogram pass, or supplied by the caller), then each 8-bit digit
// is scattered in a single pass in which a tile of pairs (3840, or 1024 for
// inputs up to 2^20 so that small sorts still fill the SMs) learns its global
// offsets by decoupled look-back over its predecessors' per-digit counts.
//
// Used twice per frame: by FP32 depth (4 digits) over the visible records,
// then by tile id over the emitted (tile, record) pairs, which yields the
// per-tile front-to-back order of Sec. 3 ("Preliminaries: 3DGS": Gaussians
// are sorted by depth per tile) with ties broken by record (= gid) order.
//
// Ranking inside a tile is warp-private and stable: each warp ranks its IPT x
// 32 keys in input order with __match_any_sync and a per-warp digit
// histogram; warps are combined by a per-digit exclusive scan.  Keys are held
// in registers, ranks packed two per register, values are read only when they
// are scattered, which keeps the pass at four 256-thread CTAs per SM.
#include "common.cuh"

namespace lodge {

namespace {

constexpr int kRadix = 256;
constexpr int kWarps = kSortThreads / 32;
constexpr int kMaxPasses = 4;
constexpr int kLookback = 8;    // predecessors read per look-back step

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__global__ void __launch_bounds__(256)
hist_kernel(const uint32_t* __restrict__ keys, int64_t n, int passes, uint32_t last_mask,
            uint32_t* __restrict__ hist, int shift0) {
    __shared__ uint32_t sh[kMaxPasses][kRadix];
    for (int i = threadIdx.x; i < kMaxPasses * kRadix; i += blockDim.x) (&sh[0][0])[i] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        uint32_t k = __ldg(keys + i);
        for (int p = 0; p < passes; ++p)
            atomicAdd(&sh[p][(k >> (shift0 + 8 * p)) & (p == passes - 1 ? last_mask : 0xffu)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * kRadix; i += blockDim.x) {
        uint32_t c = (&sh[0][0])[i];
        if (c) atomicAdd(hist + i, c);
    }
}

// exclusive scan of each pass's 256-bin histogram, in place (one block per pass)
__global__ void hist_scan_kernel(uint32_t* hist) {
    __shared__ uint32_t s_scan[33];
    uint32_t* h = hist + blockIdx.x * kRadix;
    uint32_t v = h[threadIdx.x], total;
    uint32_t e = block_exclusive_scan(v, s_scan, &total);
    h[threadIdx.x] = e;
}

template <int kIPT, bool kWriteKeys, bool kValues>
__global__ void __launch_bounds__(kSortThreads, 4)
onesweep_pass(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
              uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n, int shift,
              uint32_t dmask, const uint32_t* __restrict__ offsets, uint32_t* __restrict__ status,
              uint32_t* __restrict__ counter, uint32_t* __restrict__ err, uint2* __restrict__ ranges,
              int range_shift, uint32_t range_tiles, const unsigned long long* __restrict__ d_count,
              bool raw_counts) {
    constexpr int kTileN = kSortThreads * kIPT;
    __shared__ uint32_t s_whist[kWarps][kRadix];
    __shared__ uint32_t s_keys[kTileN];
    __shared__ uint32_t s_vals[kValues ? kTileN : 1];
    __shared__ uint32_t s_dstart[kRadix];
    __shared__ uint32_t s_gbase[kRadix];
    __shared__ uint32_t s_scan[33];
    __shared__ uint32_t s_tile;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < kWarps * kRadix; i += kSortThreads) (&s_whist[0][0])[i] = 0;
    if (tid == 0) s_tile = atomicAdd(counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (d_count) {   // n is a capacity; the device count (<= n) decides
        const unsigned long long c = *d_count;
        if (c < (unsigned long long)n) n = (int64_t)c;
        if ((int64_t)tile * kTileN >= n) return;   // all later tiles are empty too
    }
    // the pass's digit offsets: given, or the exclusive scan of its digit
    // counts taken here (every CTA the same)
    uint32_t dbase = offsets[tid];
    if (raw_counts) {
        uint32_t dtotal;
        dbase = block_exclusive_scan(dbase, s_scan, &dtotal);
    }
    const int64_t seg = (int64_t)tile * kTileN + (int64_t)warp * 32 * kIPT;
    const int64_t base = seg + lane;
    const int64_t nvalid = n - seg;   // items of this warp's segment that exist (may be <= 0)

    uint32_t k[kIPT];
#pragma unroll
    for (int j = 0; j < kIPT; ++j) k[j] = (j * 32 + lane < nvalid) ? __ldcs(kin + base + j * 32) : 0u;

    // warp-private stable ranking in (j, lane) order = input order; ranks
    // (< 2^16) packed two per register.  The lanes holding the same digit
    // are found either with match.any or with one ballot per digit bit; the
    // first lane of each group adds the group's size to the warp's count
    // with a shared atomic and hands the previous count to the group by a
    // shuffle (no warp barriers in the loop).
    const uint32_t lt = lanemask_lt();
    uint32_t rk[(kIPT + 1) / 2];
#pragma unroll
    for (int j = 0; j < kIPT; ++j) {
        const bool valid = j * 32 + lane < nvalid;
        const uint32_t d = valid ? (k[j] >> shift) & dmask : 0u;
        uint32_t peers;
        if (j % 3 == 0) {
            // every third key through match.any (the ADU pipe), the others
            // through ballots (the ALU pipe), so that both pipes share the work
            peers = __match_any_sync(0xffffffffu, valid ? d : 0x100u);
        } else {
            peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
            for (int bit = 0; bit < 8; ++bit) {   // bits above a short last digit are 0: no-ops
                const bool on = (d >> bit) & 1u;
                const uint32_t m = __ballot_sync(0xffffffffu, on);
                peers &= on ? m : ~m;
            }
        }
        if (!valid) peers = 1u << lane;
        const int leader = __ffs(peers) - 1;
        uint32_t before = 0;
        if (valid && lane == leader) before = atomicAdd(&s_whist[warp][d], (uint32_t)__popc(peers));
        before = __shfl_sync(0xffffffffu, before, leader);
        const uint32_t r = before + __popc(peers & lt);
        if (j & 1) rk[j >> 1] |= r << 16; else rk[j >> 1] = r;
    }
    __syncthreads();

    // per digit (thread d): warp offsets inside the tile, tile count
    const uint32_t d = tid;
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        uint32_t c = s_whist[w][d];
        s_whist[w][d] = run;
        run += c;
    }
    // decoupled look-back for this digit (bounded waits).  The status words
    // of kLookback predecessors are loaded together and then consumed in
    // order, so a walk over tiles that have only published their counts
    // costs one memory round trip per kLookback tiles instead of per tile.
    uint32_t excl = 0;
    uint32_t* st = status + (size_t)tile * kRadix + d;
    if (tile == 0) {
        st_volatile(st, kStInc | run);
    } else {
        st_volatile(st, kStAgg | run);
        int64_t t = (int64_t)tile - 1;
        bool found = false;
        while (!found) {
            uint32_t x[kLookback];
#pragma unroll
            for (int j = 0; j < kLookback; ++j)
                x[j] = t - j >= 0 ? ld_volatile(status + (size_t)(t - j) * kRadix + d) : kStInc;
#pragma unroll
            for (int j = 0; j < kLookback; ++j) {
                if (found) break;
                uint32_t v = x[j], spins = 0;
                while ((v & ~kStVal) == 0u) {   // only for t - j >= 0: x[j] = kStInc below 0
                    if (++spins > kSpinLimit) { atomicOr(err, kErrTimeout); v = kStInc; break; }
                    if (spins > kSpinFast) __nanosleep(20);
                    v = ld_volatile(status + (size_t)(t - j) * kRadix + d);
                }
                excl += v & kStVal;
                found = (v & ~kStVal) == kStInc;
            }
            t -= kLookback;
        }
        st_volatile(st, kStInc | (excl + run));
    }
    s_gbase[d] = dbase + excl;
    uint32_t total;
    s_dstart[d] = block_exclusive_scan(run, s_scan, &total);
    __syncthreads();

    // scatter keys and values into shared memory in digit order
#pragma unroll
    for (int j = 0; j < kIPT; ++j) {
        if (j * 32 + lane < nvalid) {
            const uint32_t dd = (k[j] >> shift) & dmask;
            const uint32_t r = (j & 1) ? (rk[j >> 1] >> 16) : (rk[j >> 1] & 0xffffu);
            const uint32_t pos = s_dstart[dd] + s_whist[warp][dd] + r;
            s_keys[pos] = k[j];
            if (kValues) s_vals[pos] = __ldcs(vin + base + j * 32);
        }
    }
    __syncthreads();
    for (uint32_t i = tid; i < total; i += kSortThreads) {
        const uint32_t key = s_keys[i];
        const uint32_t dd = (key >> shift) & dmask;
        const uint32_t out = s_gbase[dd] + (i - s_dstart[dd]);
        if ((int64_t)out < n) {
            if (kWriteKeys) kout[out] = key;
            if (kValues) vout[out] = s_vals[i];
            if (ranges) {
                // last pass of a sort by tile: the keys of one tile are one
                // run here and one run in the output; the first and last
                // key of each run of this tile bound the tile's range
                const uint32_t t = key >> range_shift;
                if (t < range_tiles) {
                    if (i == 0 || (s_keys[i - 1] >> range_shift) != t) atomicMin(&ranges[t].x, out);
                    if (i + 1 == total || (s_keys[i + 1] >> range_shift) != t)
                        atomicMax(&ranges[t].y, out + 1u);
                } else {
                    atomicOr(err, kErrBadIndex);
                }
            }
        } else {
            atomicOr(err, kErrOverflow);  // only after a look-back gave up
        }
    }
}

int passes_for(int key_bits) { return key_bits <= 0 ? 0 : (key_bits + 7) / 8; }

uint32_t last_mask_for(int key_bits) {
    const int P = passes_for(key_bits);
    const int last_bits = key_bits - 8 * (P - 1);
    return last_bits >= 8 ? 0xffu : ((1u << last_bits) - 1u);
}

constexpr int kSmallIPT = kSortTileSmall / kSortThreads;
static_assert(kSmallIPT * kSortThreads == kSortTileSmall, "small tile must be whole items per thread");

template <bool kWK, bool kV>
void launch_pass(bool small, int64_t ntiles, const uint32_t* ki, const uint32_t* vi, uint32_t* ko,
                 uint32_t* vo, int64_t n, int shift, uint32_t dm, const uint32_t* off, uint32_t* st,
                 uint32_t* ctr, uint32_t* err, uint2* ranges, int range_shift, uint32_t range_tiles,
                 const unsigned long long* d_count, bool raw, cudaStream_t s) {
    if (small)
        onesweep_pass<kSmallIPT, kWK, kV><<<(unsigned)ntiles, kSortThreads, 0, s>>>(
            ki, vi, ko, vo, n, shift, dm, off, st, ctr, err, ranges, range_shift, range_tiles, d_count, raw);
    else
        onesweep_pass<kSortIPT, kWK, kV><<<(unsigned)ntiles, kSortThreads, 0, s>>>(
            ki, vi, ko, vo, n, shift, dm, off, st, ctr, err, ranges, range_shift, range_tiles, d_count, raw);
}

}  // namespace

size_t sort_scratch_bytes(int64_t n, int key_bits) {
    return sizeof(uint32_t) * (size_t)sort_scratch_words(n, passes_for(key_bits));
}

int launch_onesweep(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                    int64_t n, int key_bits, void* scratch, uint32_t* err, cudaStream_t s,
                    const uint32_t* digit_offsets, bool final_keys, int shift0, uint2* ranges,
                    uint32_t range_tiles, const unsigned long long* d_count, bool scratch_cleared,
                    bool digit_counts) {
    const int P = passes_for(key_bits);
    if (P == 0 || (d_count ? n < 1 : n <= 1)) return 0;
    if (d_count && !digit_offsets) return 0;   // device counts need supplied digit offsets
    const bool small = sort_tile_for(n) == kSortTileSmall;
    const int64_t ntiles = (n + sort_tile_for(n) - 1) / sort_tile_for(n);
    const bool values = vals != nullptr;
    uint32_t* hist = static_cast<uint32_t*>(scratch);
    uint32_t* counters = hist + kMaxPasses * kRadix;
    uint32_t* status = counters + 32;
    const uint32_t last_mask = last_mask_for(key_bits);
    const uint32_t* offs = hist;
    // supplied digit counts are scanned by the passes themselves
    const bool raw = digit_offsets && digit_counts;
    if (digit_offsets) {
        // exclusive digit offsets supplied: clear only counters and look-back words
        if (!scratch_cleared)
            cudaMemsetAsync(counters, 0,
                            sort_scratch_bytes(n, key_bits) - sizeof(uint32_t) * kMaxPasses * kRadix, s);
        offs = digit_offsets;
    } else {
        cudaMemsetAsync(scratch, 0, sort_scratch_bytes(n, key_bits), s);
        int hist_blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)device_sms() * 4);
        hist_kernel<<<hist_blocks, 256, 0, s>>>(keys, n, P, last_mask, hist, shift0);
        hist_scan_kernel<<<P, kRadix, 0, s>>>(hist);
    }
    uint32_t *ki = keys, *vi = vals, *ko = keys_alt, *vo = vals_alt;
    for (int p = 0; p < P; ++p) {
        const uint32_t dm = p == P - 1 ? last_mask : 0xffu;
        uint32_t* stp = status + (size_t)p * ntiles * kRadix;
        const bool wk = !(p == P - 1 && !final_keys);
        const int sh = shift0 + 8 * p;
        uint2* rg = p == P - 1 ? ranges : nullptr;
        if (values) {
            if (wk) launch_pass<true, true>(small, ntiles, ki, vi, ko, vo, n, sh, dm, offs + p * kRadix, stp, counters + p, err, rg, shift0, range_tiles, d_count, raw, s);
            else launch_pass<false, true>(small, ntiles, ki, vi, ko, vo, n, sh, dm, offs + p * kRadix, stp, counters + p, err, rg, shift0, range_tiles, d_count, raw, s);
        } else {
            launch_pass<true, false>(small, ntiles, ki, vi, ko, vo, n, sh, dm, offs + p * kRadix, stp, counters + p, err, rg, shift0, range_tiles, d_count, raw, s);
        }
        std::swap(ki, ko);
        std::swap(vi, vo);
    }
    return (P & 1) ? 1 : 0;
}

int onesweep_launches(int64_t n, int key_bits, bool offsets_supplied) {
    const int P = passes_for(key_bits);
    if (n <= 1 || P == 0) return 0;
    return P + (offsets_supplied ? 0 : 2);
}

}  // namespace lodge
