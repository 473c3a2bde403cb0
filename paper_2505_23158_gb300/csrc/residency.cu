// Streamed residency: chunk blocks in HBM, loaded from a pinned host store.
//
// Sec. 3 ("Chunk-based rendering", "Opacity blending"): only the active
// Gaussians of the chunks in use need to be in GPU memory, and chunk sets are
// (re)loaded in the background as the camera moves.  For a streamed scene the
// activated store lives in pinned, mapped host memory; a chunk block is that
// chunk's active set gathered into HBM (structure-of-arrays planes plus its
// sorted gid list).  On GB300 the gather kernel reads the host store directly
// over NVLink-C2C on a side stream, so no per-chunk copy is materialised on
// the host.  Blocks are cached under the context's HBM budget and evicted
// least-recently-used first when unreferenced; a frame holds the blocks it
// reads (reference count) until its stream has finished.
#include <cstring>

#include "internal.cuh"

namespace lodge {

namespace {

__global__ void gather_block_kernel(int64_t n, const uint32_t* __restrict__ gid, DevScene src,
                                    int64_t src_npad, float* mx, float* my, float* mz,
                                    float4* so, float4* q, float4* sh, int64_t dst_npad,
                                    int nplanes) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t g = gid[i];
    mx[i] = src.mx[g];
    my[i] = src.my[g];
    mz[i] = src.mz[g];
    so[i] = src.scale_op[g];
    q[i] = src.quat[g];
    for (int j = 0; j < nplanes; ++j) sh[(int64_t)j * dst_npad + i] = src.sh[(int64_t)j * src_npad + g];
}

__device__ __forceinline__ bool bsearch_u32(const uint32_t* a, int64_t n, uint32_t v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const uint32_t x = a[mid];
        if (x == v) return true;
        if (x < v) lo = mid + 1; else hi = mid;
    }
    return false;
}

// number of entries of sorted a (length n) below v
__device__ __forceinline__ int64_t lower_bound_u32(const uint32_t* a, int64_t n, uint32_t v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// B-only gids (not in A), in B order, by flag + order-preserving compaction
__global__ void b_only_flags_kernel(const uint32_t* __restrict__ A, int64_t na,
                                    const uint32_t* __restrict__ B, int64_t nb,
                                    uint32_t* __restrict__ flag) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < nb) flag[j] = bsearch_u32(A, na, B[j]) ? 0u : 1u;
}

// A entries: union position i + #(B-only gids < A[i]); flag B if also in B
__global__ void merge_a_kernel(const uint32_t* __restrict__ A, int64_t na,
                               const uint32_t* __restrict__ B, int64_t nb,
                               const uint32_t* __restrict__ bo_gid, int64_t nbo,
                               uint32_t* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= na) return;
    const uint32_t a = A[i];
    const int64_t pos = i + lower_bound_u32(bo_gid, nbo, a);
    out[pos] = (uint32_t)i | kFlagA | (bsearch_u32(B, nb, a) ? kFlagB : 0u);
}

// B-only entries: union position r + #(A gids < gid)
__global__ void merge_b_kernel(const uint32_t* __restrict__ A, int64_t na,
                               const uint32_t* __restrict__ B, const uint32_t* __restrict__ bo_idx,
                               int64_t nbo, uint32_t* __restrict__ bo_gid_out,
                               uint32_t* __restrict__ out) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nbo) return;
    const uint32_t j = bo_idx[r];
    const uint32_t g = B[j];
    out[r + lower_bound_u32(A, na, g)] = j | kFlagB;
    (void)bo_gid_out;
}

__global__ void bo_gather_kernel(const uint32_t* __restrict__ B, const uint32_t* __restrict__ bo_idx,
                                 int64_t nbo, uint32_t* __restrict__ bo_gid) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < nbo) bo_gid[r] = B[bo_idx[r]];
}

__global__ void flag_iota_kernel(uint32_t* out, int64_t n, uint32_t flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (uint32_t)i | flag;
}

// order-preserving compaction of indices j with flag[j] != 0 (single block
// per 256-item tile, decoupled look-back): out[r] = j
__global__ void __launch_bounds__(256)
compact_idx_kernel(const uint32_t* __restrict__ flag, int64_t n, uint32_t* __restrict__ out,
                   uint32_t* __restrict__ d_count, uint32_t* __restrict__ status,
                   uint32_t* __restrict__ counter, uint32_t* __restrict__ err) {
    __shared__ uint32_t s_tile, s_prefix;
    __shared__ uint32_t s_scan[33];
    if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint32_t ntiles = (uint32_t)((n + 255) / 256);
    const int64_t j = (int64_t)tile * 256 + threadIdx.x;
    const uint32_t f = (j < n && flag[j]) ? 1u : 0u;
    uint32_t total;
    const uint32_t excl = block_exclusive_scan(f, s_scan, &total);
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
    if (f) out[s_prefix + excl] = (uint32_t)j;
}

void block_view(Block& b, const DevScene& scene_dev) {
    b.view = scene_dev;   // level information, SH degree
    b.view.n_total = b.n;
    char* base = static_cast<char*>(b.mem);
    b.gid = reinterpret_cast<uint32_t*>(base);
    float* f = reinterpret_cast<float*>(base + sizeof(uint32_t) * b.n_pad);
    b.view.mx = f;
    b.view.my = f + b.n_pad;
    b.view.mz = f + 2 * b.n_pad;
    float4* f4 = reinterpret_cast<float4*>(f + 3 * b.n_pad);
    b.view.scale_op = f4;
    b.view.quat = f4 + b.n_pad;
    b.view.sh = f4 + 2 * b.n_pad;
}

}  // namespace

lodge_status acquire_block(lodge_ctx* ctx, Slot& sl, Scene* sc, int chunk, cudaStream_t s,
                           Block** out) {
    if (chunk < 0 || chunk >= (int)sc->chunks.size())
        return fail(LODGE_E_INVALID, "chunk %d out of range", chunk);
    cudaEvent_t ready = nullptr;
    {
        std::lock_guard<std::recursive_mutex> lk(ctx->mu);
        const auto key = std::make_pair(sc->id, chunk);
        auto it = ctx->blocks.find(key);
        if (it != ctx->blocks.end()) {
            Block* b = it->second.get();
            b->refs += 1;
            b->last_use = ++ctx->tick;
            ctx->res.hits += 1;
            ready = b->ready;
            *out = b;
        } else {
            if (ctx->fail_next_uploads > 0) {
                ctx->fail_next_uploads -= 1;
                ctx->res.failed_uploads += 1;
                return fail(LODGE_E_CUDA, "chunk %d of scene %d: upload failed (injected)", chunk, sc->id);
            }
            std::unique_ptr<Block> b(new Block());
            b->scene = sc->id;
            b->chunk = chunk;
            b->n = sc->chunks[chunk].n;
            b->n_pad = std::max<int64_t>((b->n + 63) / 64 * 64, 64);
            b->bytes = (size_t)b->n_pad * (sizeof(uint32_t) + 3 * sizeof(float) + 14 * sizeof(float4));
            if (!make_room(ctx, b->bytes))
                return fail(LODGE_E_BUDGET, "chunk %d of scene %d (%zu bytes) does not fit the HBM budget "
                            "(%zu of %zu in use, the rest held by frames in flight)",
                            chunk, sc->id, b->bytes, ctx->used, ctx->budget);
            cudaError_t e = cudaMallocAsync(&b->mem, b->bytes, ctx->upload_stream);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(LODGE_E_OOM, "chunk block of %zu bytes: %s", b->bytes, cudaGetErrorString(e));
            }
            ctx->used += b->bytes;
            block_view(*b, sc->dev);
            if (b->n) {
                cudaMemcpyAsync(b->gid, sc->chunks[chunk].list, sizeof(uint32_t) * b->n,
                                cudaMemcpyHostToDevice, ctx->upload_stream);
                const int nplanes = (3 * (sc->dev.sh_degree + 1) * (sc->dev.sh_degree + 1) + 3) / 4;
                gather_block_kernel<<<(unsigned)((b->n + 255) / 256), 256, 0, ctx->upload_stream>>>(
                    b->n, b->gid, sc->dev, sc->n_pad, const_cast<float*>(b->view.mx),
                    const_cast<float*>(b->view.my), const_cast<float*>(b->view.mz),
                    const_cast<float4*>(b->view.scale_op), const_cast<float4*>(b->view.quat),
                    const_cast<float4*>(b->view.sh), b->n_pad, nplanes);
            }
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ready, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventRecord(b->ready, ctx->upload_stream);
            if (e != cudaSuccess) {
                cudaFreeAsync(b->mem, ctx->upload_stream);
                ctx->used -= b->bytes;
                return fail(LODGE_E_CUDA, "chunk upload: %s", cudaGetErrorString(e));
            }
            b->refs = 1;
            b->last_use = ++ctx->tick;
            ctx->res.uploads += 1;
            sl.uploads += 1;
            ctx->res.upload_bytes += (int64_t)b->n * (sizeof(uint32_t) + 3 * sizeof(float) + 2 * sizeof(float4) +
                                                      16 * ((3 * (sc->dev.sh_degree + 1) * (sc->dev.sh_degree + 1) + 3) / 4));
            ready = b->ready;
            *out = b.get();
            ctx->blocks[key] = std::move(b);
        }
    }
    cudaError_t e = cudaStreamWaitEvent(s, ready, 0);
    if (e != cudaSuccess) return fail(LODGE_E_CUDA, "cudaStreamWaitEvent: %s", cudaGetErrorString(e));
    return LODGE_OK;
}

void release_blocks(lodge_ctx* ctx, Slot& sl) {
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    for (int k = 0; k < 2; ++k) {
        if (sl.held[k]) sl.held[k]->refs -= 1;
        sl.held[k] = nullptr;
    }
    ctx->freed.notify_all();
}

void free_scene_blocks(lodge_ctx* ctx, int scene) {
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    for (auto it = ctx->blocks.begin(); it != ctx->blocks.end();) {
        if (it->first.first == scene) {
            Block* b = it->second.get();
            cudaFreeAsync(b->mem, ctx->upload_stream);
            if (b->ready) cudaEventDestroy(b->ready);
            ctx->used -= b->bytes;
            it = ctx->blocks.erase(it);
        } else {
            ++it;
        }
    }
    ctx->freed.notify_all();
}

lodge_status block_union(lodge_ctx* ctx, Slot& sl, const Block* a, const Block* b, cudaStream_t s,
                         int64_t* n_out) {
    Workspace& ws = sl.ws;
    const int64_t na = a->n, nb = b ? b->n : 0;
    lodge_status r0 = ensure(ctx, sl.ulist, sizeof(uint32_t) * (size_t)std::max<int64_t>(na + nb, 1), s);
    if (r0 != LODGE_OK) return r0;
    if (!b) {
        if (na) flag_iota_kernel<<<(unsigned)((na + 255) / 256), 256, 0, s>>>(sl.ulist.as<uint32_t>(), na, kFlagA);
        *n_out = na;
        return cudaGetLastError() == cudaSuccess ? LODGE_OK : fail(LODGE_E_CUDA, "union kernel launch");
    }
    // bonly holds: flags (nb) | B-only indices (nb) | B-only gids (nb)
    const size_t nb1 = (size_t)std::max<int64_t>(nb, 1);
    lodge_status r = ensure(ctx, ws.bonly, sizeof(uint32_t) * 3 * nb1, s);
    if (r != LODGE_OK) return r;
    const int64_t ntiles = std::max<int64_t>((nb + 255) / 256, 1);
    r = ensure(ctx, ws.status, sizeof(uint32_t) * (size_t)ntiles, s);
    if (r != LODGE_OK) return r;
    uint32_t* flag = ws.bonly.as<uint32_t>();
    uint32_t* bo_idx = flag + nb1;
    uint32_t* bo_gid = bo_idx + nb1;
    cudaMemsetAsync(ws.status.p, 0, sizeof(uint32_t) * (size_t)ntiles, s);
    cudaMemsetAsync(sl.d_small, 0, sizeof(uint32_t) * kSmWords, s);
    if (nb) {
        b_only_flags_kernel<<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(a->gid, na, b->gid, nb, flag);
        compact_idx_kernel<<<(unsigned)ntiles, 256, 0, s>>>(flag, nb, bo_idx, sl.d_small + kSmListCount,
                                                            ws.status.as<uint32_t>(), sl.d_small + kSmCtrUnion,
                                                            sl.d_small + kSmErr);
    }
    if (cudaGetLastError() != cudaSuccess) return fail(LODGE_E_CUDA, "union kernel launch");
    r = sync_slot(ctx, sl, s);
    if (r != LODGE_OK) return r;
    const int64_t nbo = nb ? sl.h_small[kSmListCount] : 0;
    if (nbo) bo_gather_kernel<<<(unsigned)((nbo + 255) / 256), 256, 0, s>>>(b->gid, bo_idx, nbo, bo_gid);
    if (na) merge_a_kernel<<<(unsigned)((na + 255) / 256), 256, 0, s>>>(a->gid, na, b->gid, nb, bo_gid, nbo,
                                                                         sl.ulist.as<uint32_t>());
    if (nbo) merge_b_kernel<<<(unsigned)((nbo + 255) / 256), 256, 0, s>>>(a->gid, na, b->gid, bo_idx, nbo,
                                                                           bo_gid, sl.ulist.as<uint32_t>());
    if (cudaGetLastError() != cudaSuccess) return fail(LODGE_E_CUDA, "union kernel launch");
    *n_out = na + nbo;
    return LODGE_OK;
}

}  // namespace lodge
