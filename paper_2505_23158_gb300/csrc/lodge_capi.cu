// C ABI of the LODGE frame renderer: context and scene management, chunk
// choice (Eq. 4), per-chunk active-set precompute (Eq. 2 at chunk centres,
// Sec. 3 "Chunk-based rendering") and the per-frame orchestration of the
// kernels K1..K7 on the caller's stream.
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <thread>

#include "internal.cuh"

namespace lodge {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

lodge_status fail(lodge_status s, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

int device_sms() {
    constexpr int kMaxDev = 64;
    static int cache[kMaxDev] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) { cudaGetLastError(); return 152; }
    if (!cache[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            return 152;
        }
        cache[dev] = n;
    }
    return cache[dev];
}

lodge_status set_error(lodge_status s, const char* msg) {
    g_err = msg;
    return s;
}

const char* last_error() { return g_err.c_str(); }

#define CUDA_TRY(x)                                                                          \
    do {                                                                                     \
        cudaError_t e_ = (x);                                                                \
        if (e_ != cudaSuccess)                                                               \
            return fail(LODGE_E_CUDA, "%s failed: %s (%s:%d)", #x, cudaGetErrorString(e_),   \
                        __FILE__, __LINE__);                                                 \
    } while (0)

#define TRY(x)                                   \
    do {                                         \
        lodge_status s_ = (x);                   \
        if (s_ != LODGE_OK) return s_;           \
    } while (0)

// ---------------------------------------------------------------------------
// device memory with budget accounting
// ---------------------------------------------------------------------------
bool make_room(lodge_ctx* ctx, size_t bytes) {
    if (!ctx->budget) return true;
    while (ctx->used + bytes > ctx->budget) {
        Block* victim = nullptr;
        std::pair<int, int> key;
        for (auto& kv : ctx->blocks) {
            Block* b = kv.second.get();
            if (b->refs == 0 && (!victim || b->last_use < victim->last_use)) {
                victim = b;
                key = kv.first;
            }
        }
        if (!victim) return false;
        // the block is unreferenced: every frame that read it has completed
        cudaFreeAsync(victim->mem, ctx->upload_stream);
        if (victim->ready) cudaEventDestroy(victim->ready);
        ctx->used -= victim->bytes;
        ctx->res.evictions += 1;
        ctx->blocks.erase(key);
    }
    return true;
}

lodge_status dmalloc(lodge_ctx* ctx, void** p, size_t bytes) {
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    if (!make_room(ctx, bytes))
        return fail(LODGE_E_BUDGET, "HBM budget exceeded: %zu in use + %zu requested > %zu",
                    ctx->used, bytes, ctx->budget);
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(LODGE_E_OOM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    ctx->used += bytes;
    return LODGE_OK;
}

void dfree(lodge_ctx* ctx, void* p, size_t bytes) {
    if (!p) return;
    cudaFree(p);
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    ctx->used -= bytes;
    ctx->freed.notify_all();
}

// grow-only, stream-ordered
lodge_status ensure(lodge_ctx* ctx, DBuf& b, size_t bytes, cudaStream_t s) {
    if (bytes <= b.cap && b.p) return LODGE_OK;
    size_t ncap = std::max<size_t>(bytes + bytes / 4, 4096);
    ncap = (ncap + 255) / 256 * 256;
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    const size_t freed = b.p ? b.cap : 0;
    if (ctx->budget && ctx->used - freed + ncap > ctx->budget) {
        if (!make_room(ctx, ncap > freed ? ncap - freed : 0)) {
            ncap = (bytes + 255) / 256 * 256;
            if (!make_room(ctx, ncap > freed ? ncap - freed : 0))
                return fail(LODGE_E_BUDGET, "HBM budget exceeded growing scratch to %zu bytes", ncap);
        }
    }
    if (b.p) {
        cudaFreeAsync(b.p, s);
        ctx->used -= b.cap;
        b.p = nullptr;
        b.cap = 0;
    }
    cudaError_t e = cudaMallocAsync(&b.p, ncap, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return fail(LODGE_E_OOM, "cudaMallocAsync(%zu) failed: %s", ncap, cudaGetErrorString(e));
    }
    b.cap = ncap;
    ctx->used += ncap;
    return LODGE_OK;
}

void release(lodge_ctx* ctx, DBuf& b, cudaStream_t s) {
    if (b.p) {
        cudaFreeAsync(b.p, s);
        std::lock_guard<std::recursive_mutex> lk(ctx->mu);
        ctx->used -= b.cap;
        ctx->freed.notify_all();
    }
    b.p = nullptr;
    b.cap = 0;
}

// stage profiling: events around each stage, read after the next sync
static void prof_begin(Slot& sl, int stage, cudaStream_t s) {
    if (sl.prof_on && !sl.ev_pending[stage]) cudaEventRecord(sl.ev_beg[stage], s);
}
static void prof_end(Slot& sl, int stage, cudaStream_t s, int launches) {
    sl.prof.launches[stage] += launches;
    if (sl.prof_on && !sl.ev_pending[stage]) {
        cudaEventRecord(sl.ev_end[stage], s);
        sl.ev_pending[stage] = true;
    }
}
static void prof_collect(Slot& sl) {
    for (int k = 0; k < LODGE_NUM_STAGES; ++k) {
        if (!sl.ev_pending[k]) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, sl.ev_beg[k], sl.ev_end[k]) == cudaSuccess) sl.prof.ms[k] += ms;
        else cudaGetLastError();
        sl.ev_pending[k] = false;
    }
}

// Slot k >= 1 with its own stream and fence event (created on first use;
// the request loop and batches reuse slot 1 as their first slot).
lodge_status stream_slot(lodge_ctx* ctx, int k, Slot** out) {
    while ((int)ctx->slots.size() < k + 1) {
        Slot* sl = nullptr;
        TRY(create_slot(ctx, &sl));
    }
    Slot* sl = ctx->slots[k].get();
    if (!sl->own) CUDA_TRY(cudaStreamCreateWithFlags(&sl->own, cudaStreamNonBlocking));
    if (!sl->fence) CUDA_TRY(cudaEventCreateWithFlags(&sl->fence, cudaEventDisableTiming));
    sl->prof_on = ctx->slots[0]->prof_on;
    sl->prof_count = ctx->slots[0]->prof_count;
    *out = sl;
    return LODGE_OK;
}

lodge_status create_slot(lodge_ctx* ctx, Slot** out) {
    std::unique_ptr<Slot> sl(new Slot());
    {
        std::lock_guard<std::recursive_mutex> lk(ctx->mu);
        sl->index = (int)ctx->slots.size();
    }
    TRY(dmalloc(ctx, (void**)&sl->d_small, sizeof(uint32_t) * kSmWords));
    CUDA_TRY(cudaMemset(sl->d_small, 0, sizeof(uint32_t) * kSmWords));
    CUDA_TRY(cudaMallocHost((void**)&sl->h_small, sizeof(uint32_t) * kSmWords));
    CUDA_TRY(cudaMallocHost((void**)&sl->h_tail, sizeof(uint32_t) * kSmWords));
    CUDA_TRY(cudaMallocHost((void**)&sl->h_ring, sizeof(uint32_t) * kSmWords * Slot::kRing));
    for (int k = 0; k < Slot::kRing; ++k) CUDA_TRY(cudaEventCreateWithFlags(&sl->ring_ev[k], cudaEventDisableTiming));
    for (int k = 0; k < LODGE_NUM_STAGES; ++k) {
        CUDA_TRY(cudaEventCreate(&sl->ev_beg[k]));
        CUDA_TRY(cudaEventCreate(&sl->ev_end[k]));
    }
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    *out = sl.get();
    ctx->slots.emplace_back(std::move(sl));
    return LODGE_OK;
}

static void destroy_slot(lodge_ctx* ctx, Slot& sl) {
    for (DBuf* b : sl.ws.all())
        if (b->p) cudaFree(b->p);
    if (sl.ulist.p) cudaFree(sl.ulist.p);
    for (auto& u : sl.ucache)
        if (u.list.p) cudaFree(u.list.p);
    if (sl.d_small) cudaFree(sl.d_small);
    if (sl.h_small) cudaFreeHost(sl.h_small);
    if (sl.h_tail) cudaFreeHost(sl.h_tail);
    if (sl.h_ring) cudaFreeHost(sl.h_ring);
    for (int k = 0; k < Slot::kRing; ++k)
        if (sl.ring_ev[k]) cudaEventDestroy(sl.ring_ev[k]);
    for (int k = 0; k < LODGE_NUM_STAGES; ++k) {
        if (sl.ev_beg[k]) cudaEventDestroy(sl.ev_beg[k]);
        if (sl.ev_end[k]) cudaEventDestroy(sl.ev_end[k]);
    }
    if (sl.own) cudaStreamDestroy(sl.own);
    if (sl.fence) cudaEventDestroy(sl.fence);
    if (sl.copy) cudaStreamDestroy(sl.copy);
    if (sl.copy_ev) cudaEventDestroy(sl.copy_ev);
    (void)ctx;
}

// ---------------------------------------------------------------------------
// host helpers (FP64, no contraction: the library is built with
// -ffp-contract=off so these round exactly as written)
// ---------------------------------------------------------------------------
template <class F>
static void parallel_for(int64_t n, F f) {
    unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    if (n < 65536 || nt == 1) { f(0, n); return; }
    std::vector<std::thread> th;
    int64_t step = (n + nt - 1) / nt;
    for (unsigned t = 0; t < nt; ++t) {
        int64_t a = t * step, b = std::min<int64_t>(n, a + step);
        if (a >= b) break;
        th.emplace_back([=] { f(a, b); });
    }
    for (auto& t : th) t.join();
}

static double dist2(const double* a, const double* b) {
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return (dx * dx + dy * dy) + dz * dz;
}

// Two nearest chunk centres (ties to the lower index) and Eq. 4 weights.
static void chunk_pick(const std::vector<double>& centers, const double* c, int* A, int* B,
                       double* tA, double* tB) {
    int K = (int)(centers.size() / 3), a = -1, b = -1;
    double da = INFINITY, db = INFINITY;
    for (int k = 0; k < K; ++k) {
        double d = dist2(c, &centers[3 * k]);
        if (d < da) { b = a; db = da; a = k; da = d; }
        else if (d < db) { b = k; db = d; }
    }
    *A = a; *B = b;
    if (b < 0) { *tA = 1.0; *tB = 1.0; return; }
    const double* mA = &centers[3 * a];
    const double* mB = &centers[3 * b];
    double ab[3] = {mA[0] - mB[0], mA[1] - mB[1], mA[2] - mB[2]};
    double n2 = (ab[0] * ab[0] + ab[1] * ab[1]) + ab[2] * ab[2];
    double cB[3] = {c[0] - mB[0], c[1] - mB[1], c[2] - mB[2]};
    double cA[3] = {c[0] - mA[0], c[1] - mA[1], c[2] - mA[2]};
    double ta = ((cB[0] * ab[0] + cB[1] * ab[1]) + cB[2] * ab[2]) / n2;
    double tb = ((cA[0] * -ab[0] + cA[1] * -ab[1]) + cA[2] * -ab[2]) / n2;
    *tA = std::fmin(1.0, std::fmax(0.0, ta));
    *tB = std::fmin(1.0, std::fmax(0.0, tb));
}

// squared Eq. 2 bands in FP32 for inner thresholds d (L - 1 values)
static void bands(int L, const double* d, float* lo, float* hi) {
    for (int l = 0; l < kMaxLevels; ++l) { lo[l] = 0.f; hi[l] = INFINITY; }
    for (int l = 0; l < L; ++l) {
        double a = (l == 0) ? 0.0 : d[l - 1];
        lo[l] = (float)(a * a);
        if (l + 1 < L) hi[l] = (float)(d[l] * d[l]);
    }
}

// Extent table: Q_b = 2 ln(255 o_hi) * 1.001 with o_hi the upper end of the
// opacity bucket b (FP32 exponent and 3 leading mantissa bits, from 2^-8).
static void fill_qtable_host(float* q) {
    for (uint32_t b = 0; b < 65; ++b) {
        uint32_t u = (b + (119u << 3) + 1u) << 20;
        float hi;
        std::memcpy(&hi, &u, 4);
        q[b] = (float)(2.0 * std::log(255.0 * (double)hi) * 1.001);
    }
}

static DevCamera make_cam(const lodge_camera& c) {
    DevCamera d{};
    for (int i = 0; i < 9; ++i) d.R[i] = c.R[i];
    for (int i = 0; i < 3; ++i) d.t[i] = c.t[i];
    d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy;
    d.width = c.width; d.height = c.height;
    d.znear = c.znear;
    d.limx = (float)(1.3 * ((double)c.width / (2.0 * (double)c.fx)));
    d.limy = (float)(1.3 * ((double)c.height / (2.0 * (double)c.fy)));
    for (int i = 0; i < 3; ++i) d.chat[i] = (float)c.center[i];
    for (int i = 0; i < 3; ++i)
        d.tp[i] = (float)((double)c.t[i] + (((double)c.R[3 * i] * (double)d.chat[0] +
                                             (double)c.R[3 * i + 1] * (double)d.chat[1]) +
                                            (double)c.R[3 * i + 2] * (double)d.chat[2]));
    for (int i = 0; i < 3; ++i) d.clo[i] = (float)(c.center[i] - (double)d.chat[i]);
    d.tiles_x = (c.width + kTile - 1) / kTile;
    d.tiles_y = (c.height + kTile - 1) / kTile;
    return d;
}

static lodge_status check_cam(const lodge_camera& c) {
    if (c.width <= 0 || c.height <= 0)
        return fail(LODGE_E_INVALID, "camera size %dx%d must be positive", c.width, c.height);
    if ((c.width + kTile - 1) / kTile > 65535 || (c.height + kTile - 1) / kTile > 65535)
        return fail(LODGE_E_INVALID, "camera %dx%d exceeds 65535 tiles per side", c.width, c.height);
    if ((int64_t)((c.width + kTile - 1) / kTile) * ((c.height + kTile - 1) / kTile) >= (1ll << 31))
        return fail(LODGE_E_INVALID, "too many tiles");
    return LODGE_OK;
}

static int bits_for(uint32_t v) {
    int b = 0;
    while (b < 32 && (v >> b)) ++b;
    return std::max(b, 1);
}

static Scene* get_scene(lodge_ctx* ctx, int32_t id) {
    if (id < 0 || id >= (int32_t)ctx->scenes.size()) return nullptr;
    return ctx->scenes[id].get();
}

lodge_status sync_slot(lodge_ctx* ctx, Slot& sl, cudaStream_t s) {
    (void)ctx;
    CUDA_TRY(cudaMemcpyAsync(sl.h_small, sl.d_small, sizeof(uint32_t) * kSmWords,
                             cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    prof_collect(sl);
    uint32_t err = sl.h_small[kSmErr];
    if (sl.tail_pending) {
        err |= sl.h_tail[kSmErr];
        sl.tail_pending = false;
    }
    if (err & kErrTimeout) return fail(LODGE_E_TIMEOUT, "a device-side wait timed out (status 0x%x)", err);
    if (err & kErrOverflow) return fail(LODGE_E_OVERFLOW, "device output capacity exceeded (status 0x%x)", err);
    if (err & kErrBadIndex) return fail(LODGE_E_INVALID, "out-of-range index in an active list (status 0x%x)", err);
    return LODGE_OK;
}

// ---------------------------------------------------------------------------
// selection
// ---------------------------------------------------------------------------
// Eq. 2 at centre c with inner thresholds d over the device store `dev` into
// the slot's list; returns count.
static lodge_status run_lod_select(lodge_ctx* ctx, Slot& sl, const DevScene& dev, const double* c,
                                   const double* d, cudaStream_t s, int64_t* n_out) {
    Workspace& ws = sl.ws;
    float lo[kMaxLevels], hi[kMaxLevels];
    bands(dev.num_levels, d, lo, hi);
    float c32[3] = {(float)c[0], (float)c[1], (float)c[2]};
    int64_t ntiles = (dev.n_total + kSelectTile - 1) / kSelectTile;
    TRY(ensure(ctx, ws.list, sizeof(uint32_t) * (size_t)std::max<int64_t>(dev.n_total, 1), s));
    TRY(ensure(ctx, ws.status, sizeof(uint32_t) * (size_t)std::max<int64_t>(ntiles, 1), s));
    CUDA_TRY(cudaMemsetAsync(ws.status.p, 0, sizeof(uint32_t) * (size_t)std::max<int64_t>(ntiles, 1), s));
    CUDA_TRY(cudaMemsetAsync(sl.d_small, 0, sizeof(uint32_t) * kSmWords, s));
    prof_begin(sl, LODGE_STAGE_SELECT, s);
    launch_lod_select(dev, c32, lo, hi, ws.list.as<uint32_t>(), sl.d_small + kSmListCount,
                      ws.status.as<uint32_t>(), sl.d_small + kSmCtrSelect, sl.d_small + kSmErr, s);
    prof_end(sl, LODGE_STAGE_SELECT, s, ntiles > 0 ? 1 : 0);
    CUDA_TRY(cudaGetLastError());
    TRY(sync_slot(ctx, sl, s));
    *n_out = sl.h_small[kSmListCount];
    return LODGE_OK;
}

struct Active {
    const uint32_t* list = nullptr;
    int64_t n = 0;
    int A = -1, B = -1;
    double tA = 1.0, tB = 1.0;
    bool blocks = false;       // entries index into chunk blocks (streamed scenes)
    ProjSources src;
};

static lodge_status select_streamed(lodge_ctx* ctx, Slot& sl, Scene* sc, lodge_mode mode,
                                    cudaStream_t s, Active* act) {
    const bool single = (mode == LODGE_CHUNK || act->B < 0);
    if (single) { act->B = -1; if (mode == LODGE_CHUNK) act->tA = act->tB = 1.0; }
    Block* a = nullptr;
    Block* b = nullptr;
    TRY(acquire_block(ctx, sl, sc, act->A, s, &a));
    sl.held[0] = a;
    if (!single) {
        TRY(acquire_block(ctx, sl, sc, act->B, s, &b));
        sl.held[1] = b;
    }
    if (sl.u_scene != sc->id || sl.ua != act->A || sl.ub != act->B) {
        int64_t n;
        sl.u_scene = -1;
        prof_begin(sl, LODGE_STAGE_UNION, s);
        TRY(block_union(ctx, sl, a, b, s, &n));
        prof_end(sl, LODGE_STAGE_UNION, s, b ? 5 : 1);
        sl.un = n;
        sl.u_scene = sc->id;
        sl.ua = act->A;
        sl.ub = act->B;
    }
    act->list = sl.ulist.as<uint32_t>();
    act->n = sl.un;
    act->blocks = true;
    act->src.a = a->view;
    act->src.gid_a = a->gid;
    act->src.n_a = a->n;
    act->src.npad_a = a->n_pad;
    const Block* bb = b ? b : a;
    act->src.b = bb->view;
    act->src.gid_b = bb->gid;
    act->src.n_b = bb->n;
    act->src.npad_b = bb->n_pad;
    return LODGE_OK;
}

// Union of chunk sets A and B of a resident scene into `out` (gid
// ascending, bit 31 / 30 = member of A / B); waits for the count.  The union
// is complete on the device when this returns.
static lodge_status compute_union(lodge_ctx* ctx, Slot& sl, Scene* sc, int A, int B, cudaStream_t s,
                                  DBuf& out, int64_t* n) {
    const Chunk& a = sc->chunks[A];
    const Chunk& b = sc->chunks[B];
    Workspace& ws = sl.ws;
    int64_t ntiles = (sc->dev.n_total + kSelectTile - 1) / kSelectTile;
    TRY(ensure(ctx, out, sizeof(uint32_t) * (size_t)std::max<int64_t>(a.n + b.n, 1), s));
    TRY(ensure(ctx, ws.marks, (size_t)((sc->dev.n_total + 63) / 64 * 64), s));
    TRY(ensure(ctx, ws.status, sizeof(uint32_t) * (size_t)std::max<int64_t>(ntiles, 1), s));
    CUDA_TRY(cudaMemsetAsync(ws.status.p, 0, sizeof(uint32_t) * (size_t)std::max<int64_t>(ntiles, 1), s));
    CUDA_TRY(cudaMemsetAsync(sl.d_small, 0, sizeof(uint32_t) * kSmWords, s));
    prof_begin(sl, LODGE_STAGE_UNION, s);
    launch_chunk_union(a.list, a.n, b.list, b.n, sc->dev.n_total, ws.marks.as<uint8_t>(),
                       out.as<uint32_t>(), sl.d_small + kSmListCount, ws.status.as<uint32_t>(),
                       sl.d_small + kSmCtrUnion, sl.d_small + kSmErr, s);
    prof_end(sl, LODGE_STAGE_UNION, s, (a.n > 0) + (b.n > 0) + (ntiles > 0));
    CUDA_TRY(cudaGetLastError());
    TRY(sync_slot(ctx, sl, s));
    *n = sl.h_small[kSmListCount];
    return LODGE_OK;
}

static lodge_status select_active(lodge_ctx* ctx, Slot& sl, Scene* sc, lodge_mode mode,
                                  const lodge_camera& cam, cudaStream_t s, Active* act) {
    *act = Active{};
    if (mode != LODGE_FULL && mode != LODGE_LOD && mode != LODGE_CHUNK && mode != LODGE_CHUNK_BLEND)
        return fail(LODGE_E_INVALID, "unknown render mode %d", (int)mode);
    if (sc->residency == kStreamed && (mode == LODGE_FULL || mode == LODGE_LOD))
        return fail(LODGE_E_NOT_RESIDENT,
                    "scene %d is streamed by chunk: only CHUNK and CHUNK_BLEND can render it", sc->id);
    if (mode == LODGE_FULL) {
        act->n = sc->dev.level_off[1];
        return LODGE_OK;
    }
    if (mode == LODGE_LOD) {
        int64_t n;
        TRY(run_lod_select(ctx, sl, sc->dev, cam.center, sc->d_inner.data(), s, &n));
        act->list = sl.ws.list.as<uint32_t>();
        act->n = n;
        return LODGE_OK;
    }
    if (sc->chunks.empty()) return fail(LODGE_E_INVALID, "scene has no chunks");
    chunk_pick(sc->centers, cam.center, &act->A, &act->B, &act->tA, &act->tB);
    if (sc->residency == kStreamed) return select_streamed(ctx, sl, sc, mode, s, act);
    if (mode == LODGE_CHUNK || act->B < 0) {
        act->list = sc->chunks[act->A].list;
        act->n = sc->chunks[act->A].n;
        if (mode == LODGE_CHUNK) { act->B = -1; act->tA = act->tB = 1.0; }
        return LODGE_OK;
    }
    // the pair's union: shared by all slots once computed, else this slot's cache
    const uint64_t key = ((uint64_t)(uint32_t)act->A << 32) | (uint32_t)act->B;
    {
        std::lock_guard<std::recursive_mutex> lk(ctx->mu);
        auto it = sc->unions.find(key);
        if (it == sc->unions.end() && sc->unions.size() < kMaxPairUnions) {
            Scene::PairUnion pu;
            lodge_status r = compute_union(ctx, sl, sc, act->A, act->B, s, pu.list, &pu.n);
            if (r == LODGE_OK) {
                it = sc->unions.emplace(key, pu).first;
            } else {
                release(ctx, pu.list, s);
                if (r != LODGE_E_BUDGET) return r;   // out of budget: a slot's cache below
            }
        }
        if (it != sc->unions.end()) {
            act->list = it->second.list.as<uint32_t>();
            act->n = it->second.n;
            return LODGE_OK;
        }
    }
    Slot::UnionEntry* ue = nullptr;
    for (auto& u : sl.ucache)
        if (u.scene == sc->id && u.a == act->A && u.b == act->B) ue = &u;
    if (!ue) {
        ue = &sl.ucache[0];
        for (auto& u : sl.ucache)
            if (u.used < ue->used) ue = &u;
        ue->scene = -1;
        TRY(compute_union(ctx, sl, sc, act->A, act->B, s, ue->list, &ue->n));
        ue->scene = sc->id;
        ue->a = act->A;
        ue->b = act->B;
    }
    ue->used = ++sl.utick;
    act->list = ue->list.as<uint32_t>();
    act->n = ue->n;
    return LODGE_OK;
}

// ---------------------------------------------------------------------------
// one frame
// ---------------------------------------------------------------------------
static void take(DBuf& dst, DBuf& src) { dst = src; src = DBuf{}; }

// end_sync = false leaves the frame's last kernels running when it returns
// (the next frame on the same stream queues behind them); their status words
// are checked at the slot's next sync.
// importance != null: composite with K12 instead of K7 and raise
// importance[gid] (n_total floats) to each Gaussian's largest weight.
// job != null: stop before compositing and describe it in *job (the caller
// composites a batch of frames with one launch and then syncs their slots).
// The scratch words a frame starts from, set by one launch: segment k of
// n[k] words gets v0[k] at even and v1[k] at odd word indices.
struct FillPlan {
    static constexpr int kMax = 8;
    uint32_t* p[kMax];
    int64_t n[kMax];
    uint32_t v0[kMax], v1[kMax];
    int count = 0;
    void add(uint32_t* ptr, int64_t words, uint32_t a = 0u, uint32_t b = 0u) {
        if (count < kMax && ptr && words > 0) {
            p[count] = ptr; n[count] = words; v0[count] = a; v1[count] = b; ++count;
        }
    }
};
__global__ void fill_kernel(FillPlan f) {
    const int k = blockIdx.y;
    uint32_t* __restrict__ p = f.p[k];
    const int64_t n = f.n[k];
    const uint32_t a = f.v0[k], b = f.v1[k];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (i & 1) ? b : a;
}

// pend != null allows the frame to run without its mid-frame sync (counts
// left on the device, scratch sized by capacities; see Slot::Pending): it
// then sets pend->used, appends *pend to the slot's pending list, and its
// stats and profile counts are taken when the slot is harvested.
// default bin size: per-tile lists from this active-set size up
constexpr int64_t kPerTileActiveMin = 1ll << 21;

static lodge_status render_frame(lodge_ctx* ctx, Slot& sl, const DevScene& dsc, const Active& act,
                                 const lodge_camera& c, float* d_rgb, cudaStream_t s, Saved* save,
                                 lodge_frame_stats* st, bool end_sync, float* importance = nullptr,
                                 BlendFrame* job = nullptr, Slot::Pending* pend = nullptr) {
    Workspace& ws = sl.ws;
    TRY(check_cam(c));
    DevCamera cam = make_cam(c);
    const int64_t ntiles_img = (int64_t)cam.tiles_x * cam.tiles_y;
    const int64_t na = act.n;
    const size_t na1 = (size_t)std::max<int64_t>(na, 1);
    if (na >= (1ll << 30)) return fail(LODGE_E_INVALID, "active set too large");

    // ---- K3 projection
    TRY(ensure(ctx, ws.rec_a, sizeof(float4) * na1, s));
    TRY(ensure(ctx, ws.rec_b, sizeof(float4) * na1, s));
    TRY(ensure(ctx, ws.rec_c, sizeof(float) * na1, s));
    TRY(ensure(ctx, ws.rec_rect, sizeof(uint2) * na1, s));
    TRY(ensure(ctx, ws.rec_gid, sizeof(uint32_t) * na1, s));
    TRY(ensure(ctx, ws.dkey, sizeof(uint32_t) * na1, s));
    TRY(ensure(ctx, ws.dval, sizeof(uint32_t) * na1, s));
    const int64_t ptiles = proj_status_words(na);
    TRY(ensure(ctx, ws.status, sizeof(uint32_t) * (size_t)ptiles, s));
    TRY(ensure(ctx, ws.doffs, sizeof(uint32_t) * 8 * 256, s));
    // frames kept for the adjoint and the importance walk use per-tile lists
    // (their per-pixel positions index the tile's own list); otherwise the
    // context's bin size, or by default per-tile lists for active sets of
    // kPerTileActiveMin Gaussians or more (many small splats, whose bin
    // lists are long against their tiles' lists) and bins of 2x2 tiles below
    const int bl = (save || importance) ? 0
                   : ctx->bin_log2 >= 0 ? ctx->bin_log2
                   : (na >= kPerTileActiveMin ? 0 : 1);
    // the key capacity is learned per bin size
    if (!save && !importance && sl.key_cap_bl != bl) {
        sl.key_cap = 0;
        sl.key_cap_bl = bl;
    }
    // no mid-frame sync: plain frames once the slot knows a key capacity
    const bool deferred = pend && !save && !importance && !sl.prof_count &&
                          sl.key_cap > 0 && na > 0 && (int)sl.pending.size() < Slot::kRing;
    if (pend) pend->used = false;
    const int32_t bins_x = (cam.tiles_x + (1 << bl) - 1) >> bl;
    const int32_t bins_y = (cam.tiles_y + (1 << bl) - 1) >> bl;
    const int64_t nbins = (int64_t)bins_x * bins_y;
    const int tbits = bits_for((uint32_t)std::max<int64_t>(nbins - 1, 0));
    if (deferred) {
        // every scratch word the frame starts from, sized by capacities and
        // set by one launch: look-back words of the projection and the
        // emission, the slot's small words, both digit histograms, both sorts'
        // counters and look-back words, the bin ranges (begin ~0, end 0)
        const int64_t etiles = std::max<int64_t>((na + kEmitThreads - 1) / kEmitThreads, 1);
        TRY(ensure(ctx, ws.status2, sizeof(uint32_t) * (size_t)etiles, s));
        TRY(ensure(ctx, ws.sort, sort_scratch_bytes(na, 32), s));
        TRY(ensure(ctx, ws.sort2, sort_scratch_bytes(sl.key_cap, tbits), s));
        TRY(ensure(ctx, ws.ranges, sizeof(uint2) * (size_t)std::max<int64_t>(nbins, 1), s));
        FillPlan fp;
        fp.add(ws.status.as<uint32_t>(), ptiles);
        fp.add(sl.d_small, kSmWords);
        fp.add(ws.doffs.as<uint32_t>(), 8 * 256);
        fp.add(ws.status2.as<uint32_t>(), etiles);
        fp.add(ws.sort.as<uint32_t>(), (int64_t)(sort_scratch_bytes(na, 32) / sizeof(uint32_t)));
        fp.add(ws.sort2.as<uint32_t>(), (int64_t)(sort_scratch_bytes(sl.key_cap, tbits) / sizeof(uint32_t)));
        fp.add(reinterpret_cast<uint32_t*>(ws.ranges.p), 2 * nbins, 0xffffffffu, 0u);
        int64_t most = 0;
        for (int k = 0; k < fp.count; ++k) most = std::max(most, fp.n[k]);
        const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((most + 255) / 256, 512));
        fill_kernel<<<dim3(gx, (unsigned)fp.count), 256, 0, s>>>(fp);
    } else {
        CUDA_TRY(cudaMemsetAsync(ws.status.p, 0, sizeof(uint32_t) * (size_t)ptiles, s));
        CUDA_TRY(cudaMemsetAsync(sl.d_small, 0, sizeof(uint32_t) * kSmWords, s));
        CUDA_TRY(cudaMemsetAsync(ws.doffs.p, 0, sizeof(uint32_t) * 8 * 256, s));
    }
    ProjectOut po;
    po.rec_a = ws.rec_a.as<float4>();
    po.rec_b = ws.rec_b.as<float4>();
    po.rec_c = ws.rec_c.as<float>();
    po.rec_rect = ws.rec_rect.as<uint2>();
    po.rec_gid = ws.rec_gid.as<uint32_t>();
    po.depth_key = ws.dkey.as<uint32_t>();
    po.depth_val = ws.dval.as<uint32_t>();
    po.counts = sl.d_small + kSmProj;
    // digit counts: [0, 1024) the bin sort's (from K4), [1024, 2048) the
    // depth sort's (from K3)
    po.depth_hist = ws.doffs.as<uint32_t>() + 4 * 256;
    po.bin_log2 = bl;
    prof_begin(sl, LODGE_STAGE_PROJECT, s);
    launch_project(dsc, cam, act.list, na, (float)act.tA, (float)act.tB, po,
                   ws.status.as<uint32_t>(), sl.d_small + kSmCtrProj, sl.d_small + kSmErr, s,
                   act.blocks ? &act.src : nullptr);
    // (the launch count of the projection stage includes the frame's fill)
    prof_end(sl, LODGE_STAGE_PROJECT, s, (na > 0 ? 1 : 0) + (deferred ? 1 : 0));
    CUDA_TRY(cudaGetLastError());
    int64_t n_vis = 0, n_keys = 0, n_bkeys = 0;
    // device counts (u64 words: the visible count's high word stays 0)
    const unsigned long long* d_nvis = nullptr;
    const unsigned long long* d_nbk = nullptr;
    if (deferred) {
        n_vis = na;              // capacities
        n_bkeys = sl.key_cap;
        d_nvis = reinterpret_cast<const unsigned long long*>(sl.d_small + kSmProj);
        d_nbk = reinterpret_cast<const unsigned long long*>(sl.d_small + kSmProj + (bl > 0 ? 4 : 2));
    } else {
        TRY(sync_slot(ctx, sl, s));
        n_vis = sl.h_small[kSmProj];
        uint64_t nk64;
        std::memcpy(&nk64, sl.h_small + kSmProj + 2, 8);
        n_keys = (int64_t)nk64;
        if (n_keys >= (1ll << 30)) return fail(LODGE_E_OVERFLOW, "%lld tile keys exceed 2^30", (long long)n_keys);
        // key lists per bin: the tile itself (bl = 0) or a square of 2^bl tiles
        n_bkeys = n_keys;
        if (bl > 0) {
            std::memcpy(&nk64, sl.h_small + kSmProj + 4, 8);
            n_bkeys = (int64_t)nk64;
        }
        // capacity for later frames of this slot that skip the sync
        if (!save && !importance)
            sl.key_cap = std::max<int64_t>(sl.key_cap, n_bkeys + n_bkeys / 2 + 65536);
    }
    const size_t nv1 = (size_t)std::max<int64_t>(n_vis, 1), nk1 = (size_t)std::max<int64_t>(n_bkeys, 1);

    // ---- K5 depth sort of the visible records
    TRY(ensure(ctx, ws.dkey2, sizeof(uint32_t) * nv1, s));
    TRY(ensure(ctx, ws.dval2, sizeof(uint32_t) * nv1, s));
    if (!deferred)   // (frames without a sync set up their own sort scratch above)
        TRY(ensure(ctx, ws.sort, std::max(sort_scratch_bytes(n_vis, 32), sort_scratch_bytes(n_bkeys, tbits)), s));
    prof_begin(sl, LODGE_STAGE_DEPTH_SORT, s);
    // (the passes scan the projection's digit counts themselves)
    int w1 = launch_onesweep(ws.dkey.as<uint32_t>(), ws.dval.as<uint32_t>(), ws.dkey2.as<uint32_t>(),
                             ws.dval2.as<uint32_t>(), n_vis, 32, ws.sort.p, sl.d_small + kSmErr, s,
                             po.depth_hist, true, 0, nullptr, 0, d_nvis, deferred, true);
    prof_end(sl, LODGE_STAGE_DEPTH_SORT, s, onesweep_launches(n_vis, 32, true));
    DBuf& zs = w1 ? ws.dkey2 : ws.dkey;
    DBuf& rs = w1 ? ws.dval2 : ws.dval;

    // ---- K4 emit (bin, record) in depth order, with the bin sort's digit
    // counts.  When bin and record index fit in one word together, each pair
    // is one packed key (bin << rbits | record) and the bin sort moves keys
    // only; otherwise bin and record are sorted as a (key, value) pair.
    const int rbits_need = bits_for((uint32_t)std::max<int64_t>(n_vis - 1, 0));
    const int rbits = tbits + rbits_need <= 32 ? rbits_need : 0;
    TRY(ensure(ctx, ws.tkey, sizeof(uint32_t) * nk1, s));
    TRY(ensure(ctx, ws.tkey2, sizeof(uint32_t) * nk1, s));
    if (!rbits) {
        TRY(ensure(ctx, ws.tval, sizeof(uint32_t) * nk1, s));
        TRY(ensure(ctx, ws.tval2, sizeof(uint32_t) * nk1, s));
    }
    TRY(ensure(ctx, ws.koff, sizeof(uint32_t) * (nv1 + 1), s));
    TRY(ensure(ctx, ws.srec, sizeof(uint32_t) * nv1, s));
    TRY(ensure(ctx, ws.srect, sizeof(uint2) * nv1, s));
    if (!deferred) {
        int64_t etiles = std::max<int64_t>((n_vis + kEmitThreads - 1) / kEmitThreads, 1);
        TRY(ensure(ctx, ws.status, sizeof(uint32_t) * (size_t)etiles, s));
        CUDA_TRY(cudaMemsetAsync(ws.status.p, 0, sizeof(uint32_t) * (size_t)etiles, s));
    }
    prof_begin(sl, LODGE_STAGE_EMIT, s);
    int emit_n = 0;
    if (deferred) {
        emit_n = launch_emit_counted(rs.as<uint32_t>(), n_vis, d_nvis, ws.rec_rect.as<uint2>(), bins_x, bl, n_bkeys,
                            d_nbk, ws.tkey.as<uint32_t>(), ws.tval.as<uint32_t>(), rbits, tbits,
                            ws.doffs.as<uint32_t>(), ws.status2.as<uint32_t>(), sl.d_small + kSmCtrEmit,
                            sl.d_small + kSmErr, s);
    } else {
        launch_emit(rs.as<uint32_t>(), n_vis, ws.rec_rect.as<uint2>(), bins_x, bl,
                    ws.koff.as<uint32_t>(), ws.srec.as<uint32_t>(), ws.srect.as<uint2>(), n_bkeys,
                    ws.tkey.as<uint32_t>(), ws.tval.as<uint32_t>(), rbits, tbits, ws.doffs.as<uint32_t>(),
                    ws.status.as<uint32_t>(), sl.d_small + kSmCtrEmit, sl.d_small + kSmErr, s);
    }
    prof_end(sl, LODGE_STAGE_EMIT, s, deferred ? emit_n : emit_launches(n_vis, n_bkeys, bl));

    // ---- K6 bin ranges: recorded by the bin sort's last pass (begin by
    // atomic minimum from 0xffffffff, end by atomic maximum from 0); with at
    // most one key the sort does not run and K6 scans the key list instead
    const bool fused_ranges = deferred || n_bkeys > 1;
    if (!deferred) {   // (set up by the frame's fill when deferred)
        TRY(ensure(ctx, ws.ranges, sizeof(uint2) * (size_t)std::max<int64_t>(nbins, 1), s));
        CUDA_TRY(cudaMemsetAsync(ws.ranges.p, 0, sizeof(uint2) * (size_t)nbins, s));
        if (fused_ranges && nbins)
            CUDA_TRY(cudaMemset2DAsync(ws.ranges.p, sizeof(uint2), 0xff, sizeof(uint32_t), (size_t)nbins, s));
    }

    // ---- K5 bin sort (stable: keeps depth order within a bin)
    prof_begin(sl, LODGE_STAGE_TILE_SORT, s);
    int w2 = launch_onesweep(ws.tkey.as<uint32_t>(), rbits ? nullptr : ws.tval.as<uint32_t>(),
                             ws.tkey2.as<uint32_t>(), rbits ? nullptr : ws.tval2.as<uint32_t>(), n_bkeys,
                             tbits, deferred ? ws.sort2.p : ws.sort.p, sl.d_small + kSmErr, s,
                             ws.doffs.as<uint32_t>(), true, rbits,
                             fused_ranges ? ws.ranges.as<uint2>() : nullptr, (uint32_t)nbins, d_nbk, deferred,
                             deferred);   // deferred frames' emission leaves its digit counts unscanned
    prof_end(sl, LODGE_STAGE_TILE_SORT, s, onesweep_launches(n_bkeys, tbits, true));
    DBuf& ks = w2 ? ws.tkey2 : ws.tkey;
    DBuf& vs = w2 ? ws.tval2 : ws.tval;
    const uint32_t* rec_of_pair = rbits ? ks.as<uint32_t>() : vs.as<uint32_t>();
    const uint32_t vmask = rbits ? (1u << rbits) - 1u : 0xffffffffu;
    if (!fused_ranges) {
        prof_begin(sl, LODGE_STAGE_RANGES, s);
        launch_ranges(ks.as<uint32_t>(), n_bkeys, ws.ranges.as<uint2>(), nbins, rbits, s);
        prof_end(sl, LODGE_STAGE_RANGES, s, n_bkeys > 0 ? 1 : 0);
    }

    // ---- K7 blend
    BlendOut bo{d_rgb, nullptr, nullptr};
    if (save) {
        const size_t npix = (size_t)c.width * c.height;
        TRY(ensure(ctx, ws.T, sizeof(float) * npix, s));
        TRY(ensure(ctx, ws.last, sizeof(uint32_t) * npix, s));
        bo.T_final = ws.T.as<float>();
        bo.last = ws.last.as<uint32_t>();
    }
    if (job) {
        *job = blend_frame(cam, ws.ranges.as<uint2>(), rec_of_pair, vmask, n_bkeys, ws.rec_a.as<float4>(),
                           ws.rec_b.as<float4>(), ws.rec_c.as<float>(), n_vis, bo, bl,
                           ws.rec_rect.as<uint2>());
        end_sync = false;
    }
    prof_begin(sl, LODGE_STAGE_BLEND, s);
    if (job) {
        // composited later by the batch launch
    } else if (importance) {
        TRY(ensure(ctx, ws.iscore, sizeof(uint32_t) * nv1, s));
        CUDA_TRY(cudaMemsetAsync(ws.iscore.p, 0, sizeof(uint32_t) * nv1, s));
        launch_importance(cam, ws.ranges.as<uint2>(), rec_of_pair, vmask, n_keys, ws.rec_a.as<float4>(),
                          ws.rec_b.as<float4>(), ws.rec_c.as<float>(), n_vis, ws.rec_gid.as<uint32_t>(),
                          d_rgb, ws.iscore.as<uint32_t>(), dsc.n_total, importance, s);
    } else {
        launch_blend(cam, ws.ranges.as<uint2>(), rec_of_pair, vmask, n_bkeys, ws.rec_a.as<float4>(),
                     ws.rec_b.as<float4>(), ws.rec_c.as<float>(), n_vis, bo, s, bl, ws.rec_rect.as<uint2>(),
                     sl.prof_count ? reinterpret_cast<unsigned long long*>(sl.d_small + kSmPairs) : nullptr,
                     sl.share_sms ? sl.d_small + kSmCtrBlend : nullptr);
        if (sl.prof_count) end_sync = true;   // the counts are read back with the frame
    }
    prof_end(sl, LODGE_STAGE_BLEND, s, job ? 0 : ntiles_img > 0 ? (importance ? 1 + (n_vis > 0) : 1) : 0);
    CUDA_TRY(cudaGetLastError());
    if (deferred) {
        // status words and counts into the slot's ring; read at its harvest
        const int ring = sl.ring_next;
        sl.ring_next = (sl.ring_next + 1) % Slot::kRing;
        CUDA_TRY(cudaMemcpyAsync(sl.h_ring + (size_t)ring * kSmWords, sl.d_small, sizeof(uint32_t) * kSmWords,
                                 cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaEventRecord(sl.ring_ev[ring], s));
        pend->ring = ring;
        pend->used = true;
        pend->st = st;
        pend->n_active = na;
        pend->n_tiles = ntiles_img;
        pend->A = act.A;
        pend->B = act.B;
        pend->tA = act.tA;
        pend->tB = act.tB;
        pend->packed = rbits != 0;
        pend->sort_passes = (tbits + 7) / 8;
        pend->bin_log2 = bl;
        sl.pending.push_back(*pend);
        return LODGE_OK;
    }
    if (job) {
        // the caller syncs after the batch launch
    } else if (end_sync || save) {
        TRY(sync_slot(ctx, sl, s));
    } else {
        CUDA_TRY(cudaMemcpyAsync(sl.h_tail, sl.d_small, sizeof(uint32_t) * kSmWords,
                                 cudaMemcpyDeviceToHost, s));
        sl.tail_pending = true;
    }

    sl.prof.frames += 1;
    sl.prof.keys += n_keys;
    sl.prof.bin_keys += n_bkeys;
    if (rbits) sl.prof.packed_keys += n_bkeys;
    sl.prof.bin_sort_passes += n_bkeys > 1 ? (tbits + 7) / 8 : 0;
    if (sl.prof_count && !job && !importance) {
        uint64_t pe, pu;
        std::memcpy(&pe, sl.h_small + kSmPairs, 8);
        std::memcpy(&pu, sl.h_small + kSmPairs + 2, 8);
        sl.prof.blend_pairs += (int64_t)pe;
        sl.prof.blend_pairs_used += (int64_t)pu;
    }
    sl.prof.visible += n_vis;
    sl.prof.active += na;
    if (st) {
        st->n_active = na;
        st->n_visible = n_vis;
        st->n_keys = n_keys;
        st->n_tiles = ntiles_img;
        st->chunk_a = act.A;
        st->chunk_b = act.B;
        st->t_a = act.tA;
        st->t_b = act.tB;
    }
    if (save) {
        save->cam = cam;
        save->n_vis = n_vis;
        save->n_keys = n_keys;
        save->rbits = rbits;
        take(save->rec_a, ws.rec_a);
        take(save->rec_b, ws.rec_b);
        take(save->rec_c, ws.rec_c);
        take(save->rec_rect, ws.rec_rect);
        take(save->rec_gid, ws.rec_gid);
        take(save->zsorted, zs);
        take(save->rsorted, rs);
        take(save->tkey, ks);
        if (!rbits) take(save->tval, vs);
        take(save->ranges, ws.ranges);
        take(save->T, ws.T);
        take(save->last, ws.last);
    }
    return LODGE_OK;
}

// Wait for a slot's stream and take the status words and counts of its
// deferred frames (stats, profile).  A frame whose bin keys outgrew the
// slot's capacity wrote no keys: the capacity grows and the frame's index is
// appended to *redo, to be rendered again with its mid-frame sync.
static void take_pending(Slot& sl, const Slot::Pending& p, std::vector<int>* redo, lodge_status* r);

static lodge_status harvest(lodge_ctx* ctx, Slot& sl, cudaStream_t s, std::vector<int>* redo) {
    (void)ctx;
    if (sl.pending.empty()) return LODGE_OK;
    CUDA_TRY(cudaStreamSynchronize(s));
    prof_collect(sl);
    lodge_status r = LODGE_OK;
    for (const Slot::Pending& p : sl.pending) take_pending(sl, p, redo, &r);
    sl.pending.clear();
    return r;
}

// The oldest deferred frames of a slot, until `keep` remain: each waits for
// its own ring entry only, so the slot's later frames keep running while the
// host goes on enqueuing (a full harvest would drain the slot's stream).
static lodge_status harvest_front(Slot& sl, size_t keep, std::vector<int>* redo) {
    lodge_status r = LODGE_OK;
    size_t k = 0;
    for (; k + keep < sl.pending.size(); ++k) {
        const Slot::Pending& p = sl.pending[k];
        CUDA_TRY(cudaEventSynchronize(sl.ring_ev[p.ring]));
        take_pending(sl, p, redo, &r);
    }
    sl.pending.erase(sl.pending.begin(), sl.pending.begin() + (ptrdiff_t)k);
    return r;
}

// one deferred frame's status words and counts: stats, profile counters,
// capacity, errors; a frame that overflowed its key capacity is listed for
// rendering again
static void take_pending(Slot& sl, const Slot::Pending& p, std::vector<int>* redo, lodge_status* rp) {
    lodge_status& r = *rp;
    const uint32_t* w = sl.h_ring + (size_t)p.ring * kSmWords;
    const uint32_t err = w[kSmErr];
    uint64_t nk, nb;
    std::memcpy(&nk, w + kSmProj + 2, 8);
    std::memcpy(&nb, w + kSmProj + (p.bin_log2 > 0 ? 4 : 2), 8);
    const int64_t n_vis = w[kSmProj];
    // keep the capacity half a frame ahead of the largest seen
    sl.key_cap = std::max<int64_t>(sl.key_cap, (int64_t)(nb + nb / 2 + 65536));
    if (err & kErrOverflow) {
        sl.prof.redone += 1;
        if (redo) redo->push_back(p.frame);
        return;
    }
    if (r == LODGE_OK && (err & kErrTimeout))
        r = fail(LODGE_E_TIMEOUT, "a device-side wait timed out (status 0x%x)", err);
    if (r == LODGE_OK && (err & kErrBadIndex))
        r = fail(LODGE_E_INVALID, "out-of-range index in an active list (status 0x%x)", err);
    sl.prof.frames += 1;
    sl.prof.keys += (int64_t)nk;
    sl.prof.bin_keys += (int64_t)nb;
    if (p.packed) sl.prof.packed_keys += (int64_t)nb;
    sl.prof.bin_sort_passes += nb > 1 ? p.sort_passes : 0;
    sl.prof.visible += n_vis;
    sl.prof.active += p.n_active;
    if (p.st) {
        p.st->n_active = p.n_active;
        p.st->n_visible = n_vis;
        p.st->n_keys = (int64_t)nk;
        p.st->n_tiles = p.n_tiles;
        p.st->chunk_a = p.A;
        p.st->chunk_b = p.B;
        p.st->t_a = p.tA;
        p.st->t_b = p.tB;
    }
}

// Select and render one camera of a scene on a slot; blocks of streamed
// scenes are held for the frame and released after it.  pend: see
// render_frame (resident scenes only).
lodge_status render_one(lodge_ctx* ctx, Slot& sl, Scene* sc, lodge_mode mode,
                        const lodge_camera& cam, float* d_rgb, cudaStream_t s, Saved* save,
                        lodge_frame_stats* st, bool end_sync, float* importance, Slot::Pending* pend) {
    Active act;
    lodge_status r = select_active(ctx, sl, sc, mode, cam, s, &act);
    // blocks of a streamed scene are released after the frame: wait for it
    if (sc->residency == kStreamed) {
        end_sync = true;
        pend = nullptr;
    }
    if (pend) pend->used = false;
    if (r == LODGE_OK)
        r = render_frame(ctx, sl, sc->dev, act, cam, d_rgb, s, save, st, end_sync, importance, nullptr, pend);
    if (sc->residency == kStreamed) {
        if (r != LODGE_OK) cudaStreamSynchronize(s);
        release_blocks(ctx, sl);
    }
    return r;
}

// A batch of frames (any scenes, modes and sizes) on slots first .. first+n-1
// of one stream: each frame runs its own stages up to the tile ranges on its
// slot's scratch, then one launch composites the tiles of all of them.
// items[k].status receives each frame's outcome.
lodge_status render_batch(lodge_ctx* ctx, BatchItem* items, int n, int first, cudaStream_t s) {
    if (n < 1 || n > kMaxBlendBatch) return fail(LODGE_E_INVALID, "batch of %d frames (1..%d)", n, kMaxBlendBatch);
    std::vector<Slot*> q((size_t)n);
    for (int k = 0; k < n; ++k) TRY(stream_slot(ctx, first + k, &q[k]));
    std::vector<BlendFrame> jobs;
    std::vector<int> ok;
    std::vector<Slot::Pending> pd((size_t)n);
    // every frame's stages up to the tile ranges on its own slot and stream,
    // started after the work already queued on s; a slot that has rendered a
    // frame before skips the mid-frame sync (counts stay on the device)
    for (int k = 0; k < n; ++k) {
        BatchItem& it = items[k];
        Slot& sl = *q[k];
        sl.share_sms = true;
        CUDA_TRY(cudaEventRecord(sl.fence, s));
        CUDA_TRY(cudaStreamWaitEvent(sl.own, sl.fence, 0));
        Active act;
        BlendFrame job;
        pd[k].frame = k;
        lodge_status r = select_active(ctx, sl, it.sc, it.mode, it.cam, sl.own, &act);
        if (r == LODGE_OK)
            r = render_frame(ctx, sl, it.sc->dev, act, it.cam, it.d_rgb, sl.own, nullptr, it.st, false, nullptr,
                             &job, &pd[k]);
        it.status = r;
        if (r == LODGE_OK) {
            jobs.push_back(job);
            ok.push_back(k);
        } else {
            cudaStreamSynchronize(sl.own);
            sl.pending.clear();
            if (it.sc->residency == kStreamed) release_blocks(ctx, sl);
        }
    }
    for (int k = 0; k < n; ++k) {   // s continues after every frame's stages
        CUDA_TRY(cudaEventRecord(q[k]->fence, q[k]->own));
        CUDA_TRY(cudaStreamWaitEvent(s, q[k]->fence, 0));
    }
    // one persistent launch composites the tiles of every frame of the step
    if (!jobs.empty()) {
        uint32_t* ctr = q[0]->d_small + kSmCtrBlend;
        CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(uint32_t), s));
        launch_blend_batch(jobs.data(), (int)jobs.size(), s, ctr);
    }
    const cudaError_t e = cudaGetLastError();
    std::vector<int> redo;
    for (int k : ok) {
        Slot& sl = *q[k];
        lodge_status r;
        if (e != cudaSuccess) {
            r = fail(LODGE_E_CUDA, "%s", cudaGetErrorString(e));
        } else if (pd[k].used) {
            std::vector<int> rk;
            r = harvest(ctx, sl, s, &rk);
            if (r == LODGE_OK && !rk.empty()) redo.push_back(k);   // keys outgrew the slot's capacity
        } else {
            r = sync_slot(ctx, sl, s);
        }
        items[k].status = r;
    }
    for (int k : ok) {
        if (items[k].sc->residency == kStreamed) release_blocks(ctx, *q[k]);
        q[k]->share_sms = false;
    }
    // frames whose keys outgrew their slot's capacity: rendered again alone,
    // with their sync (the capacity has grown for the next step)
    for (int k : redo) {
        BatchItem& it = items[k];
        it.status = render_one(ctx, *q[k], it.sc, it.mode, it.cam, it.d_rgb, s, nullptr, it.st, true, nullptr,
                               nullptr);
    }
    return LODGE_OK;
}

// ---------------------------------------------------------------------------
// small kernels of the host API
// ---------------------------------------------------------------------------
// Image i of a call back to the host, on the frame's stream.  (A copy kernel
// writing through the host buffer's device alias measured slower than the
// copy engine: 3751 vs 5190 frames/s end to end at 1080p.)
static lodge_status copy_back(float* h_dst, const float* d_src, size_t nfloat, cudaStream_t s) {
    if (nfloat) CUDA_TRY(cudaMemcpyAsync(h_dst, d_src, sizeof(float) * nfloat, cudaMemcpyDeviceToHost, s));
    return LODGE_OK;
}

__global__ void iota_kernel(uint32_t* out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (uint32_t)i;
}

// gids of block-indexed union entries, flags kept
__global__ void block_gid_kernel(const uint32_t* list, int64_t n, const uint32_t* gid_a,
                                 const uint32_t* gid_b, uint32_t flag_mask, uint32_t* out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t e = list[i];
    const uint32_t g = ((e & kFlagA) ? gid_a : gid_b)[e & kGidMask];
    out[i] = g | (e & flag_mask);
}

__global__ void zrec_kernel(const uint32_t* zsorted, const uint32_t* rsorted, int64_t n, uint32_t* zrec) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && (int64_t)rsorted[i] < n) zrec[rsorted[i]] = zsorted[i];
}

__global__ void debug_keys_kernel(const uint32_t* tkey, const uint32_t* tval, int rbits, int64_t n,
                                  int64_t n_rec, const uint32_t* zrec, const uint32_t* gid,
                                  uint64_t* keys, uint32_t* gids) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t k = tkey[i];
    uint32_t r = rbits ? k & ((1u << rbits) - 1u) : tval[i];
    const uint32_t tile = rbits ? k >> rbits : k;
    if ((int64_t)r >= n_rec) r = 0;
    if (keys) keys[i] = ((uint64_t)tile << 32) | zrec[r];
    if (gids) gids[i] = gid[r];
}

__global__ void debug_records_kernel(int64_t n, const float4* ra, const float4* rb, const float* rc,
                                     const uint2* rect, const uint32_t* gid_in, const uint32_t* zrec,
                                     uint32_t* gid, float* depth, int32_t* r4, float* mean2,
                                     float* conic, float* opac, float* rgb) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 a = ra[i], b = rb[i];
    if (gid) gid[i] = gid_in[i];
    if (depth) depth[i] = __uint_as_float(zrec[i]);
    if (r4) {
        uint2 r = rect[i];   // pixel range; reported in tiles
        r4[4 * i + 0] = (int32_t)((r.x & 0xffffu) / kTile);
        r4[4 * i + 1] = (int32_t)((r.x >> 16) / kTile);
        r4[4 * i + 2] = (int32_t)((r.y & 0xffffu) / kTile);
        r4[4 * i + 3] = (int32_t)((r.y >> 16) / kTile);
    }
    if (mean2) { mean2[2 * i] = a.x; mean2[2 * i + 1] = a.y; }
    if (conic) {
        const float s = 0.7213475204444817f;
        float u00 = a.z, u01 = a.w, u11 = b.x;
        conic[3 * i + 0] = u00 * u00 / s;
        conic[3 * i + 1] = u00 * u01 / s;
        conic[3 * i + 2] = (u01 * u01 + u11 * u11) / s;
    }
    if (opac) opac[i] = exp2f(b.y);   // records hold log2 of the opacity
    if (rgb) { rgb[3 * i] = b.z; rgb[3 * i + 1] = b.w; rgb[3 * i + 2] = rc[i]; }
}

// FP32 device activation for the raw-parameter path.
__global__ void activate_kernel(int64_t n, const float* ls, const float* q, const float* lg,
                                float4* so, float4* qo) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s0 = expf(ls[3 * i]), s1 = expf(ls[3 * i + 1]), s2 = expf(ls[3 * i + 2]);
    float o = 1.f / (1.f + expf(-lg[i]));
    so[i] = make_float4(s0, s1, s2, o);
    float w = q[4 * i], x = q[4 * i + 1], y = q[4 * i + 2], z = q[4 * i + 3];
    float r = rsqrtf(w * w + x * x + y * y + z * z);
    qo[i] = make_float4(w * r, x * r, y * r, z * r);
}

// N x 48 SH coefficients -> 12 planes of float4 with stride np
__global__ void sh_planes_kernel(int64_t n, const float* sh, float4* planes, int64_t np) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4* src = reinterpret_cast<const float4*>(sh + 48 * i);
#pragma unroll
    for (int j = 0; j < 12; ++j) planes[(size_t)j * np + i] = src[j];
}

__global__ void planes_kernel(int64_t n, const float* means, float* mx, float* my, float* mz) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    mx[i] = means[3 * i]; my[i] = means[3 * i + 1]; mz[i] = means[3 * i + 2];
}

static void free_saved(lodge_ctx* ctx, Saved& v, bool sync_free) {
    for (DBuf* b : {&v.rec_a, &v.rec_b, &v.rec_c, &v.rec_rect, &v.rec_gid, &v.zsorted, &v.rsorted,
                    &v.tkey, &v.tval, &v.ranges, &v.T, &v.last, &v.act_so, &v.act_q}) {
        if (sync_free) { if (b->p) cudaFree(b->p); *b = DBuf{}; }
        else release(ctx, *b, 0);
    }
}

// Fill the structure-of-arrays store of a scene (activated in FP64, rounded
// once) at `dst` (device or pinned host), plane stride NP.
static lodge_status fill_store(const lodge_scene_desc* desc, const DevScene& d, int64_t NP,
                               float* dst, bool dst_is_host) {
    const int L = desc->num_levels;
    auto put = [&](void* to, const void* from, size_t bytes) -> cudaError_t {
        if (dst_is_host) { std::memcpy(to, from, bytes); return cudaSuccess; }
        return cudaMemcpy(to, from, bytes, cudaMemcpyHostToDevice);
    };
    std::vector<float> plane;
    std::vector<float4> plane4;
    if (!dst_is_host) {
        plane.assign((size_t)NP, 0.f);
        plane4.assign((size_t)NP, make_float4(0, 0, 0, 0));
    }
    for (int axis = 0; axis < 3; ++axis) {
        float* out = dst_is_host ? dst + axis * NP : plane.data();
        for (int l = 0; l < L; ++l) {
            const lodge_level_desc& lv = desc->levels[l];
            const int64_t o = d.level_off[l];
            parallel_for(lv.n, [&](int64_t a, int64_t b) {
                for (int64_t i = a; i < b; ++i) out[o + i] = lv.means[3 * i + axis];
            });
        }
        if (!dst_is_host) CUDA_TRY(put(dst + axis * NP, plane.data(), sizeof(float) * NP));
    }
    float4* f4 = reinterpret_cast<float4*>(dst + 3 * NP);
    float4* out4 = dst_is_host ? f4 : plane4.data();
    for (int l = 0; l < L; ++l) {
        const lodge_level_desc& lv = desc->levels[l];
        const int64_t o = d.level_off[l];
        parallel_for(lv.n, [&](int64_t a, int64_t b) {
            for (int64_t i = a; i < b; ++i) {
                float s0 = (float)std::exp((double)lv.log_scales[3 * i]);
                float s1 = (float)std::exp((double)lv.log_scales[3 * i + 1]);
                float s2 = (float)std::exp((double)lv.log_scales[3 * i + 2]);
                float op = (float)(1.0 / (1.0 + std::exp(-(double)lv.opacity_logits[i])));
                out4[o + i] = make_float4(s0, s1, s2, op);
            }
        });
    }
    if (!dst_is_host) CUDA_TRY(put(f4, plane4.data(), sizeof(float4) * NP));
    out4 = dst_is_host ? f4 + NP : plane4.data();
    for (int l = 0; l < L; ++l) {
        const lodge_level_desc& lv = desc->levels[l];
        const int64_t o = d.level_off[l];
        parallel_for(lv.n, [&](int64_t a, int64_t b) {
            for (int64_t i = a; i < b; ++i) {
                double w = lv.quats[4 * i], x = lv.quats[4 * i + 1], y = lv.quats[4 * i + 2], z = lv.quats[4 * i + 3];
                double nrm = std::sqrt(((w * w + x * x) + y * y) + z * z);
                out4[o + i] = make_float4((float)(w / nrm), (float)(x / nrm), (float)(y / nrm), (float)(z / nrm));
            }
        });
    }
    if (!dst_is_host) CUDA_TRY(put(f4 + NP, plane4.data(), sizeof(float4) * NP));
    for (int j = 0; j < 12; ++j) {
        out4 = dst_is_host ? f4 + (size_t)(2 + j) * NP : plane4.data();
        for (int l = 0; l < L; ++l) {
            const lodge_level_desc& lv = desc->levels[l];
            const int64_t o = d.level_off[l];
            parallel_for(lv.n, [&](int64_t a, int64_t b) {
                for (int64_t i = a; i < b; ++i) {
                    const float* p = lv.sh + 48 * i + 4 * j;
                    out4[o + i] = make_float4(p[0], p[1], p[2], p[3]);
                }
            });
        }
        if (!dst_is_host) CUDA_TRY(put(f4 + (size_t)(2 + j) * NP, plane4.data(), sizeof(float4) * NP));
    }
    return LODGE_OK;
}

static void point_store(DevScene& d, float* base, int64_t NP) {
    d.mx = base;
    d.my = base + NP;
    d.mz = base + 2 * NP;
    float4* f4 = reinterpret_cast<float4*>(base + 3 * NP);
    d.scale_op = f4;
    d.quat = f4 + NP;
    d.sh = f4 + 2 * NP;
}

// (callers have synchronised the device: no frame still reads the lists)
static void free_pair_unions(lodge_ctx* ctx, Scene& sc) {
    for (auto& kv : sc.unions) release(ctx, kv.second.list, 0);
    sc.unions.clear();
}

static void free_scene(lodge_ctx* ctx, Scene& sc) {
    free_scene_blocks(ctx, sc.id);
    if (sc.block) dfree(ctx, sc.block, sc.block_bytes);
    sc.block = nullptr;
    if (sc.host_store) cudaFreeHost(sc.host_store);
    sc.host_store = nullptr;
    if (sc.host_lists) cudaFreeHost(sc.host_lists);
    sc.host_lists = nullptr;
    if (sc.residency == kResident)
        for (auto& ch : sc.chunks)
            if (ch.list) dfree(ctx, ch.list, sizeof(uint32_t) * (size_t)std::max<int64_t>(ch.n, 1));
    sc.chunks.clear();
    free_pair_unions(ctx, sc);
}

}  // namespace lodge

using namespace lodge;

// ===========================================================================
// extern "C"
// ===========================================================================
extern "C" {

const char* lodge_last_error(void) { return lodge::last_error(); }

lodge_status lodge_create(int device, size_t hbm_budget_bytes, lodge_ctx** out) {
    if (!out) return fail(LODGE_E_INVALID, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(LODGE_E_INVALID, "device %d not present (%d devices)", device, ndev);
    CUDA_TRY(cudaSetDevice(device));
    std::unique_ptr<lodge_ctx> ctx(new lodge_ctx());
    ctx->device = device;
    ctx->budget = hbm_budget_bytes;
    float q[65];
    fill_qtable_host(q);
    CUDA_TRY(upload_qtable(q));
    CUDA_TRY(cudaStreamCreateWithFlags(&ctx->upload_stream, cudaStreamNonBlocking));
    Slot* s0 = nullptr;
    TRY(create_slot(ctx.get(), &s0));
    *out = ctx.release();
    return LODGE_OK;
}

lodge_status lodge_destroy(lodge_ctx* ctx) {
    if (!ctx) return LODGE_OK;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (auto& kv : ctx->saved) free_saved(ctx, *kv.second, true);
    ctx->saved.clear();
    for (auto& sp : ctx->scenes)
        if (sp) free_scene(ctx, *sp);
    for (auto& sl : ctx->slots) destroy_slot(ctx, *sl);
    if (ctx->upload_stream) cudaStreamDestroy(ctx->upload_stream);
    cudaDeviceSynchronize();
    delete ctx;
    return LODGE_OK;
}

lodge_status lodge_load_scene(lodge_ctx* ctx, const lodge_scene_desc* desc, int32_t* scene_id) {
    if (!ctx || !desc || !scene_id) return fail(LODGE_E_INVALID, "NULL argument");
    const int L = desc->num_levels;
    if (L < 1 || L > kMaxLevels) return fail(LODGE_E_INVALID, "num_levels %d outside 1..%d", L, kMaxLevels);
    if (desc->sh_degree < 0 || desc->sh_degree > 3) return fail(LODGE_E_INVALID, "sh_degree %d outside 0..3", desc->sh_degree);
    if (!desc->levels) return fail(LODGE_E_INVALID, "levels is NULL");
    if (L > 1 && !desc->d_thresholds) return fail(LODGE_E_INVALID, "d_thresholds is NULL");
    for (int l = 0; l + 2 < L; ++l)
        if (!(desc->d_thresholds[l] <= desc->d_thresholds[l + 1]))
            return fail(LODGE_E_INVALID, "d_thresholds must be ascending");
    if (desc->num_chunks < 0 || (desc->num_chunks > 0 && !desc->chunk_centers))
        return fail(LODGE_E_INVALID, "bad chunk centres");
    if (desc->residency != kResident && desc->residency != kStreamed)
        return fail(LODGE_E_INVALID, "unknown residency %d", desc->residency);
    if (desc->filter2d != 0 && desc->filter2d != 1)
        return fail(LODGE_E_INVALID, "filter2d must be 0 or 1");
    if (desc->residency == kStreamed && desc->num_chunks < 1)
        return fail(LODGE_E_INVALID, "a streamed scene needs chunk centres");
    CUDA_TRY(cudaSetDevice(ctx->device));
    std::unique_ptr<Scene> sc(new Scene());
    sc->residency = desc->residency;
    DevScene& d = sc->dev;
    d.num_levels = L;
    d.sh_degree = desc->sh_degree;
    d.filter2d = desc->filter2d;
    d.level_off[0] = 0;
    for (int l = 0; l < L; ++l) {
        const lodge_level_desc& lv = desc->levels[l];
        if (lv.n < 0) return fail(LODGE_E_INVALID, "level %d has negative size", l);
        if (lv.n > 0 && (!lv.means || !lv.log_scales || !lv.quats || !lv.opacity_logits || !lv.sh))
            return fail(LODGE_E_INVALID, "level %d has a NULL array", l);
        d.level_off[l + 1] = d.level_off[l] + lv.n;
        d.filter_var[l] = lv.filter_var;
    }
    for (int l = L; l < kMaxLevels; ++l) d.level_off[l + 1] = d.level_off[L];
    const int64_t N = d.level_off[L];
    if (N >= (1ll << 30)) return fail(LODGE_E_INVALID, "scene has %lld Gaussians, limit 2^30", (long long)N);
    d.n_total = N;
    const int64_t NP = std::max<int64_t>((N + 63) / 64 * 64, 64);
    sc->n_pad = NP;
    // store: 3 mean planes, scale_op, quat, 12 SH planes
    const size_t bytes = sizeof(float) * 3 * NP + sizeof(float4) * (2 + 12) * NP;
    Slot& sl = *ctx->slots[0];
    cudaStream_t s = 0;
    void* means_tmp = nullptr;   // streamed: device copy of the mean planes for the precompute
    size_t means_tmp_bytes = 0;
    if (sc->residency == kResident) {
        TRY(dmalloc(ctx, &sc->block, bytes));
        sc->block_bytes = bytes;
        point_store(d, static_cast<float*>(sc->block), NP);
        lodge_status r = fill_store(desc, d, NP, static_cast<float*>(sc->block), false);
        if (r != LODGE_OK) { dfree(ctx, sc->block, bytes); return r; }
    } else {
        cudaError_t e = cudaHostAlloc(&sc->host_store, bytes, cudaHostAllocMapped | cudaHostAllocPortable);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(LODGE_E_OOM, "pinned host store of %zu bytes: %s", bytes, cudaGetErrorString(e));
        }
        sc->host_bytes = bytes;
        lodge_status r = fill_store(desc, d, NP, static_cast<float*>(sc->host_store), true);
        if (r != LODGE_OK) { cudaFreeHost(sc->host_store); return r; }
        void* dview = nullptr;
        CUDA_TRY(cudaHostGetDevicePointer(&dview, sc->host_store, 0));
        point_store(d, static_cast<float*>(dview), NP);
        means_tmp_bytes = sizeof(float) * 3 * NP;
        TRY(dmalloc(ctx, &means_tmp, means_tmp_bytes));
        CUDA_TRY(cudaMemcpy(means_tmp, sc->host_store, means_tmp_bytes, cudaMemcpyHostToDevice));
    }
    sc->d_inner.assign(desc->d_thresholds, desc->d_thresholds + std::max(L - 1, 0));
    const int K = desc->num_chunks;
    sc->centers.assign(desc->chunk_centers, desc->chunk_centers + 3 * K);
    sc->radius.assign(K, 0.0);
    for (int k = 0; k < K; ++k) {
        double best = INFINITY;
        for (int j = 0; j < K; ++j) {
            if (j == k) continue;
            double dd = std::sqrt(dist2(&sc->centers[3 * k], &sc->centers[3 * j]));
            if (dd < best) best = dd;
        }
        sc->radius[k] = K > 1 ? best : 0.0;
    }
    // per-chunk active sets: Eq. 2 at m_k with thresholds d_l + r_k
    DevScene dsel = d;
    if (means_tmp) {
        float* mp = static_cast<float*>(means_tmp);
        dsel.mx = mp; dsel.my = mp + NP; dsel.mz = mp + 2 * NP;
    }
    sc->chunks.assign(K, Chunk{});
    std::vector<double> dd(std::max(L - 1, 1));
    std::vector<std::vector<uint32_t>> host_lists;
    if (sc->residency == kStreamed) host_lists.resize(K);
    lodge_status r = LODGE_OK;
    for (int k = 0; k < K && r == LODGE_OK; ++k) {
        for (int l = 0; l + 1 < L; ++l) dd[l] = sc->d_inner[l] + sc->radius[k];
        int64_t n;
        r = run_lod_select(ctx, sl, dsel, &sc->centers[3 * k], dd.data(), s, &n);
        if (r != LODGE_OK) break;
        sc->chunks[k].n = n;
        if (sc->residency == kResident) {
            void* p = nullptr;
            r = dmalloc(ctx, &p, sizeof(uint32_t) * (size_t)std::max<int64_t>(n, 1));
            if (r != LODGE_OK) break;
            if (n) cudaMemcpy(p, sl.ws.list.p, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice);
            sc->chunks[k].list = static_cast<uint32_t*>(p);
            sc->chunk_bytes += sizeof(uint32_t) * (size_t)std::max<int64_t>(n, 1);
        } else {
            host_lists[k].resize((size_t)n);
            if (n) cudaMemcpy(host_lists[k].data(), sl.ws.list.p, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost);
        }
    }
    if (means_tmp) dfree(ctx, means_tmp, means_tmp_bytes);
    if (r == LODGE_OK && sc->residency == kStreamed) {
        size_t total = 0;
        for (auto& v : host_lists) total += v.size();
        cudaError_t e = cudaHostAlloc((void**)&sc->host_lists, sizeof(uint32_t) * std::max<size_t>(total, 1),
                                      cudaHostAllocPortable);
        if (e != cudaSuccess) {
            cudaGetLastError();
            r = fail(LODGE_E_OOM, "pinned chunk lists: %s", cudaGetErrorString(e));
        } else {
            size_t off = 0;
            for (int k = 0; k < K; ++k) {
                std::memcpy(sc->host_lists + off, host_lists[k].data(), sizeof(uint32_t) * host_lists[k].size());
                sc->chunks[k].list = sc->host_lists + off;
                off += host_lists[k].size();
            }
        }
    }
    if (r != LODGE_OK) {
        free_scene(ctx, *sc);
        return r;
    }
    CUDA_TRY(cudaDeviceSynchronize());
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    sc->id = (int)ctx->scenes.size();
    *scene_id = sc->id;
    ctx->scenes.emplace_back(std::move(sc));
    return LODGE_OK;
}

lodge_status lodge_unload_scene(lodge_ctx* ctx, int32_t scene_id) {
    if (!ctx) return fail(LODGE_E_INVALID, "NULL context");
    Scene* sc = get_scene(ctx, scene_id);
    if (!sc) return fail(LODGE_E_INVALID, "no scene %d", scene_id);
    CUDA_TRY(cudaSetDevice(ctx->device));
    CUDA_TRY(cudaDeviceSynchronize());
    free_scene(ctx, *sc);
    for (auto& sl : ctx->slots) {
        if (sl->u_scene == scene_id) sl->u_scene = -1;
        for (auto& u : sl->ucache)
            if (u.scene == scene_id) u.scene = -1;
    }
    CUDA_TRY(cudaDeviceSynchronize());
    ctx->scenes[scene_id].reset();
    return LODGE_OK;
}

lodge_status lodge_upload_chunks(lodge_ctx* ctx, int32_t scene_id, const int32_t* chunk_ids,
                                 int32_t n, int blocking) {
    if (!ctx) return fail(LODGE_E_INVALID, "NULL context");
    Scene* sc = get_scene(ctx, scene_id);
    if (!sc) return fail(LODGE_E_INVALID, "no scene %d", scene_id);
    if (n > 0 && !chunk_ids) return fail(LODGE_E_INVALID, "chunk_ids is NULL");
    for (int i = 0; i < n; ++i)
        if (chunk_ids[i] < 0 || chunk_ids[i] >= (int32_t)sc->chunks.size())
            return fail(LODGE_E_INVALID, "chunk id %d out of range", chunk_ids[i]);
    if (sc->residency == kResident) return LODGE_OK;  // every chunk set is resident
    CUDA_TRY(cudaSetDevice(ctx->device));
    Slot& sl = *ctx->slots[0];
    for (int i = 0; i < n; ++i) {
        Block* b = nullptr;
        lodge_status r = acquire_block(ctx, sl, sc, chunk_ids[i], ctx->upload_stream, &b);
        if (r != LODGE_OK) { release_blocks(ctx, sl); return r; }
        sl.held[0] = b;
        release_blocks(ctx, sl);   // uploaded and cached, not pinned by a frame
    }
    if (blocking) CUDA_TRY(cudaStreamSynchronize(ctx->upload_stream));
    return LODGE_OK;
}

// Greedy depth-threshold search (Sec. 3, "Selecting depth thresholds"): for
// l = 1 .. L-1 in turn, d_l is the candidate above d_{l-1} that minimises the
// tile keys summed over the views, with d_1 .. d_{l-1} fixed and levels above
// l unused; ties go to the smaller candidate.  The keys of every candidate
// come from one K10 pass per view and step.
lodge_status lodge_select_thresholds(lodge_ctx* ctx, int32_t scene_id, const lodge_camera* views,
                                     int32_t n_views, const double* candidates, int32_t n_candidates,
                                     double* d_out, int64_t* keys_out, void* stream) {
    if (!ctx || !views || !candidates || !d_out || n_views < 1 || n_candidates < 1)
        return fail(LODGE_E_INVALID, "bad argument");
    if (n_candidates > kMaxThreshCandidates)
        return fail(LODGE_E_INVALID, "more than %d candidates", kMaxThreshCandidates);
    for (int k = 0; k < n_candidates; ++k) {
        if (!(std::isfinite(candidates[k]) && candidates[k] > 0.0))
            return fail(LODGE_E_INVALID, "candidate %d is not a positive finite distance", k);
        if (k && !(candidates[k] > candidates[k - 1]))
            return fail(LODGE_E_INVALID, "candidates must be strictly ascending");
    }
    Scene* sc = get_scene(ctx, scene_id);
    if (!sc) return fail(LODGE_E_INVALID, "no scene %d", scene_id);
    for (int v = 0; v < n_views; ++v) TRY(check_cam(views[v]));
    const int L = sc->dev.num_levels;
    const int K = n_candidates;
    CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<float> thr(K);
    for (int k = 0; k < K; ++k) thr[k] = (float)(candidates[k] * candidates[k]);
    DBuf d_thr, d_acc;
    TRY(ensure(ctx, d_thr, sizeof(float) * K, s));
    TRY(ensure(ctx, d_acc, sizeof(unsigned long long) * (2 * K + 2), s));
    lodge_status r = LODGE_OK;
    std::vector<unsigned long long> acc(2 * K + 2);
    std::vector<double> d;  // thresholds chosen so far
    cudaError_t e = cudaMemcpyAsync(d_thr.p, thr.data(), sizeof(float) * K, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) r = fail(LODGE_E_CUDA, "%s", cudaGetErrorString(e));
    for (int l = 1; l < L && r == LODGE_OK; ++l) {
        const double prev = d.empty() ? 0.0 : d.back();
        int64_t* row = keys_out ? keys_out + (size_t)(l - 1) * K : nullptr;
        if (!std::isfinite(prev)) {  // no candidate was left for an earlier level
            d.push_back(INFINITY);
            if (row) for (int k = 0; k < K; ++k) row[k] = -1;
            continue;
        }
        // Eq. 2 bands of the fixed levels 0 .. l-2 and the lower edge of level l-1
        ThreshBands b;
        for (int j = 0; j < kMaxLevels; ++j) { b.lo[j] = 0.f; b.hi[j] = INFINITY; }
        for (int j = 0; j < l; ++j) {
            const double a = j == 0 ? 0.0 : d[j - 1];
            b.lo[j] = (float)(a * a);
            if (j + 1 < l) b.hi[j] = (float)(d[j] * d[j]);
        }
        e = cudaMemsetAsync(d_acc.p, 0, sizeof(unsigned long long) * (2 * K + 2), s);
        for (int v = 0; v < n_views && e == cudaSuccess; ++v) {
            const DevCamera cam = make_cam(views[v]);
            for (int c = 0; c < 3; ++c) b.c[c] = (float)views[v].center[c];
            launch_threshold_cost(sc->dev, cam, sc->dev.level_off[l + 1], l, b, d_thr.as<float>(), K,
                                  d_acc.as<unsigned long long>(), s);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(acc.data(), d_acc.p, sizeof(unsigned long long) * (2 * K + 2),
                                cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { r = fail(LODGE_E_CUDA, "%s", cudaGetErrorString(e)); break; }
        // per-candidate totals: fixed part + level l-1 entering + level l leaving
        unsigned long long lower = 0, upper = 0;
        for (int m = 1; m <= K; ++m) upper += acc[K + 1 + m];
        int best = -1;
        unsigned long long best_keys = 0;
        for (int k = 0; k < K; ++k) {
            lower += acc[1 + k];
            upper -= acc[K + 1 + k];   // bucket m = k no longer counts for candidate k
            const unsigned long long keys = acc[0] + lower + upper;
            const bool valid = candidates[k] > prev;
            if (row) row[k] = valid ? (int64_t)keys : -1;
            if (valid && (best < 0 || keys < best_keys)) { best = k; best_keys = keys; }
        }
        d.push_back(best < 0 ? INFINITY : candidates[best]);
    }
    release(ctx, d_thr, s);
    release(ctx, d_acc, s);
    if (r != LODGE_OK) return r;
    for (int l = 1; l < L; ++l) d_out[l - 1] = d[l - 1];
    return LODGE_OK;
}

lodge_status lodge_select_lod(lodge_ctx* ctx, int32_t scene_id, lodge_mode mode, const lodge_camera* cams,
                              int32_t n_cams, lodge_selection* out, uint32_t* d_gids,
                              int64_t gids_capacity, void* stream) {
    if (!ctx || !cams || !out || n_cams < 0) return fail(LODGE_E_INVALID, "bad argument");
    Scene* sc = get_scene(ctx, scene_id);
    if (!sc) return fail(LODGE_E_INVALID, "no scene %d", scene_id);
    CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Slot& sl = *ctx->slots[0];
    for (int i = 0; i < n_cams; ++i) {
        Active act;
        lodge_status r = select_active(ctx, sl, sc, mode, cams[i], s, &act);
        if (r == LODGE_OK) {
            out[i].chunk_a = act.A;
            out[i].chunk_b = act.B;
            out[i].t_a = act.tA;
            out[i].t_b = act.tB;
            out[i].n_active = act.n;
            if (d_gids && n_cams == 1) {
                if (act.n > gids_capacity) {
                    r = fail(LODGE_E_OVERFLOW, "active set %lld > capacity %lld", (long long)act.n,
                             (long long)gids_capacity);
                } else if (act.n && act.blocks) {
                    // membership flags are reported only when two chunks are blended
                    block_gid_kernel<<<(unsigned)((act.n + 255) / 256), 256, 0, s>>>(
                        act.list, act.n, act.src.gid_a, act.src.gid_b,
                        act.B >= 0 ? (kFlagA | kFlagB) : 0u, d_gids);
                } else if (act.n && act.list) {
                    cudaMemcpyAsync(d_gids, act.list, sizeof(uint32_t) * act.n, cudaMemcpyDeviceToDevice, s);
                } else if (act.n) {
                    iota_kernel<<<(unsigned)((act.n + 255) / 256), 256, 0, s>>>(d_gids, act.n);
                }
                if (r == LODGE_OK) {
                    cudaError_t e = cudaGetLastError();
                    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                    if (e != cudaSuccess) r = fail(LODGE_E_CUDA, "%s", cudaGetErrorString(e));
                }
            }
        }
        if (sc->residency == kStreamed) {
            cudaStreamSynchronize(s);
            release_blocks(ctx, sl);
        }
        if (r != LODGE_OK) return r;
    }
    return LODGE_OK;
}

// A frame's image back to the host on its slot's copy stream, after the
// frame's work on its render stream `si`: the render stream goes on with the
// slot's next frame while the copy runs.
static lodge_status copy_back_async(Slot& sl, float* h_dst, const float* d_src, size_t nfloat, cudaStream_t si) {
    if (!sl.copy) CUDA_TRY(cudaStreamCreateWithFlags(&sl.copy, cudaStreamNonBlocking));
    if (!sl.copy_ev) CUDA_TRY(cudaEventCreateWithFlags(&sl.copy_ev, cudaEventDisableTiming));
    CUDA_TRY(cudaEventRecord(sl.copy_ev, si));
    CUDA_TRY(cudaStreamWaitEvent(sl.copy, sl.copy_ev, 0));
    return copy_back(h_dst, d_src, nfloat, sl.copy);
}

// The body of lodge_render; h_rgb != null also copies each frame's image to
// h_rgb (same layout as d_rgb) on its slot's copy stream right after the frame,
// so the copies of earlier frames overlap the rendering of later ones.
static lodge_status render_cams(lodge_ctx* ctx, int32_t scene_id, lodge_mode mode, const lodge_camera* cams,
                                int32_t n_cams, float* d_rgb, void* stream, int32_t save_for_backward,
                                int64_t* handle_out, lodge_frame_stats* stats, float* h_rgb) {
    if (!ctx || !cams || !d_rgb || n_cams < 0) return fail(LODGE_E_INVALID, "bad argument");
    if (save_for_backward && (n_cams != 1 || !handle_out))
        return fail(LODGE_E_INVALID, "save_for_backward needs n_cams == 1 and handle_out");
    const auto t_call = std::chrono::steady_clock::now();
    Scene* sc = get_scene(ctx, scene_id);
    if (!sc) return fail(LODGE_E_INVALID, "no scene %d", scene_id);
    CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Slot& sl0 = *ctx->slots[0];
    // Several frames of a resident scene take turns on kRenderStreams slots,
    // slot 0 on the caller's stream and the others on their own: the device
    // runs the stages of several frames at once.  The other streams start
    // after the work already queued on the caller's stream and the caller's
    // stream ends after all of it.
    std::vector<Slot*> rsl{&sl0};
    std::vector<cudaStream_t> rst{s};
    if (n_cams > 1 && !save_for_backward && sc->residency == kResident) {
        const int m = std::min<int>(mode == LODGE_FULL ? kRenderStreamsFull : kRenderStreams, n_cams);
        for (int k = 1; k < m; ++k) {
            Slot* q = nullptr;
            TRY(stream_slot(ctx, k, &q));
            CUDA_TRY(cudaEventRecord(q->fence, s));
            CUDA_TRY(cudaStreamWaitEvent(q->own, q->fence, 0));
            rsl.push_back(q);
            rst.push_back(q->own);
        }
    }
    const int m = (int)rsl.size();
    for (Slot* q : rsl) q->share_sms = m > 1;
    // Frames of a resident scene that are not kept for the adjoint run
    // without their mid-frame sync once their slot knows a key capacity:
    // their counts stay on the device and are read when the slot is
    // harvested (when its ring is full and at the end of the call).
    const bool defer = !save_for_backward && sc->residency == kResident;
    std::vector<size_t> offs((size_t)n_cams + 1, 0);
    for (int i = 0; i < n_cams; ++i) offs[i + 1] = offs[i] + (size_t)cams[i].width * cams[i].height * 3;
    std::vector<int> redo;

    auto drain = [&]() {   // after a failure: nothing of this call stays in flight
        for (int k = 0; k < m; ++k) {
            Slot* q = rsl[k];
            if (q->tail_pending || !q->pending.empty()) cudaStreamSynchronize(rst[k]);
            if (h_rgb && q->copy) cudaStreamSynchronize(q->copy);
            q->tail_pending = false;
            q->pending.clear();
            q->share_sms = false;
        }
    };
    for (int i = 0; i < n_cams; ++i) {
        std::unique_ptr<Saved> sv;
        if (save_for_backward) sv.reset(new Saved());
        Slot& sl = *rsl[i % m];
        cudaStream_t si = rst[i % m];
        // consecutive frames of one call are not waited for one by one: the
        // host prepares the next frames while earlier ones run
        const bool last = i + m >= n_cams;
        Slot::Pending pd;
        pd.frame = i;
        lodge_status r = LODGE_OK;
        if (defer && (int)sl.pending.size() >= Slot::kRing) r = harvest_front(sl, Slot::kRing / 2, &redo);
        if (r == LODGE_OK)
            r = render_one(ctx, sl, sc, mode, cams[i], d_rgb + offs[i], si, sv.get(),
                           stats ? stats + i : nullptr, last, nullptr, defer ? &pd : nullptr);
        if (r != LODGE_OK) {
            drain();
            return r;
        }
        if (h_rgb) r = copy_back_async(sl, h_rgb + offs[i], d_rgb + offs[i], offs[i + 1] - offs[i], si);
        if (r != LODGE_OK) {
            drain();
            return r;
        }
        if (sv) {
            std::lock_guard<std::recursive_mutex> lk(ctx->mu);
            int64_t h = ctx->next_handle++;
            ctx->saved[h] = std::move(sv);
            *handle_out = h;
        }
    }
    // host time spent enqueuing the call's frames (before waiting for them)
    ctx->slots[0]->prof.host_ms +=
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_call).count();
    // counts of the deferred frames; frames whose keys outgrew their slot's
    // capacity are rendered again, one by one with their sync
    lodge_status r = LODGE_OK;
    for (int k = 0; k < m && r == LODGE_OK; ++k) r = harvest(ctx, *rsl[k], rst[k], &redo);
    if (r != LODGE_OK) {
        drain();
        return r;
    }
    for (int k = 1; k < m; ++k) {   // the caller's stream ends after the other streams' frames
        CUDA_TRY(cudaEventRecord(rsl[k]->fence, rst[k]));
        CUDA_TRY(cudaStreamWaitEvent(s, rsl[k]->fence, 0));
    }
    if (h_rgb) {   // ... and after the images' copies (before any frame is rendered again)
        for (int k = 0; k < m; ++k) {
            Slot* q = rsl[k];
            if (!q->copy) continue;
            CUDA_TRY(cudaEventRecord(q->copy_ev, q->copy));
            CUDA_TRY(cudaStreamWaitEvent(s, q->copy_ev, 0));
        }
    }
    for (Slot* q : rsl) q->share_sms = false;   // frames rendered again below run alone
    for (int i : redo) {
        r = render_one(ctx, sl0, sc, mode, cams[i], d_rgb + offs[i], s, nullptr, stats ? stats + i : nullptr,
                       true, nullptr, nullptr);
        if (r != LODGE_OK) {
            drain();
            return r;
        }
        if (h_rgb) TRY(copy_back(h_rgb + offs[i], d_rgb + offs[i], offs[i + 1] - offs[i], s));
    }
    return LODGE_OK;
}

lodge_status lodge_render(lodge_ctx* ctx, int32_t scene_id, lodge_mode mode, const lodge_camera* cams,
                          int32_t n_cams, float* d_rgb, void* stream, int32_t save_for_backward,
                          int64_t* handle_out, lodge_frame_stats* stats) {
    return render_cams(ctx, scene_id, mode, cams, n_cams, d_rgb, stream, save_for_backward, handle_out, stats,
                       nullptr);
}

lodge_status lodge_render_batch(lodge_ctx* ctx, int32_t n, const int32_t* scene_ids, const int32_t* modes,
                                const lodge_camera* cams, float* const* d_rgb, void* stream,
                                lodge_frame_stats* stats, int32_t* statuses) {
    if (!ctx || n < 1 || !scene_ids || !modes || !cams || !d_rgb) return fail(LODGE_E_INVALID, "bad argument");
    if (n > kMaxBlendBatch) return fail(LODGE_E_INVALID, "at most %d frames per batch", kMaxBlendBatch);
    std::vector<BatchItem> items((size_t)n);
    for (int k = 0; k < n; ++k) {
        Scene* sc = get_scene(ctx, scene_ids[k]);
        if (!sc) return fail(LODGE_E_INVALID, "frame %d names no scene", k);
        if (!d_rgb[k]) return fail(LODGE_E_INVALID, "frame %d has no image buffer", k);
        items[k].sc = sc;
        items[k].mode = (lodge_mode)modes[k];
        items[k].cam = cams[k];
        items[k].d_rgb = d_rgb[k];
        items[k].st = stats ? stats + k : nullptr;
    }
    CUDA_TRY(cudaSetDevice(ctx->device));
    // batch frames use slots 1..n (slot 0 serves the single-frame calls)
    TRY(render_batch(ctx, items.data(), n, 1, static_cast<cudaStream_t>(stream)));
    int failed = 0;
    for (int k = 0; k < n; ++k) {
        if (statuses) statuses[k] = items[k].status;
        failed += items[k].status != LODGE_OK;
    }
    if (failed) return fail(LODGE_E_INVALID, "%d of %d frames failed (see their status)", failed, n);
    return LODGE_OK;
}

lodge_status lodge_render_host(lodge_ctx* ctx, int32_t scene_id, lodge_mode mode, const lodge_camera* cams,
                               int32_t n_cams, float* h_rgb, void* stream, lodge_frame_stats* stats) {
    if (!ctx || !cams || !h_rgb || n_cams < 0) return fail(LODGE_E_INVALID, "bad argument");
    CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    size_t total = 0;
    for (int i = 0; i < n_cams; ++i) {
        TRY(check_cam(cams[i]));
        total += (size_t)cams[i].width * cams[i].height * 3;
    }
    Slot& sl = *ctx->slots[0];
    TRY(ensure(ctx, sl.ws.img, sizeof(float) * std::max<size_t>(total, 1), s));
    // each frame's image is copied back as soon as it is done
    TRY(render_cams(ctx, scene_id, mode, cams, n_cams, sl.ws.img.as<float>(), stream, 0, nullptr, stats, h_rgb));
    CUDA_TRY(cudaStreamSynchronize(s));
    return LODGE_OK;
}

// LOD rendering with per-camera thresholds (supplementary "LOD structure
// optimization steps": the build loop renders with d_l drawn from
// U(0.7 d_l, 1.3 d_l) per step; the caller draws them).
lodge_status lodge_render_lod(lodge_ctx* ctx, int32_t scene_id, const lodge_camera* cams,
                              int32_t n_cams, const double* d_inner, float* d_rgb, void* stream,
                              lodge_frame_stats* stats) {
    if (!ctx || !cams || !d_rgb || n_cams < 0) return fail(LODGE_E_INVALID, "bad argument");
    Scene* sc = get_scene(ctx, scene_id);
    if (!sc) return fail(LODGE_E_INVALID, "no scene %d", scene_id);
    if (sc->residency != kResident)
        return fail(LODGE_E_NOT_RESIDENT, "scene %d is streamed by chunk: LOD rendering needs it resident",
                    scene_id);
    const int L = sc->dev.num_levels;
    if (L > 1 && !d_inner) return fail(LODGE_E_INVALID, "d_inner is NULL");
    for (int i = 0; i < n_cams; ++i)
        for (int l = 0; l + 1 < L; ++l) {
            const double v = d_inner[(size_t)i * (L - 1) + l];
            if (!(v >= 0.0) || (l && !(v >= d_inner[(size_t)i * (L - 1) + l - 1])))
                return fail(LODGE_E_INVALID, "camera %d: thresholds must be non-negative and ascending", i);
        }
    CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Slot& sl = *ctx->slots[0];
    size_t off = 0;
    for (int i = 0; i < n_cams; ++i) {
        TRY(check_cam(cams[i]));
        Active act;
        int64_t n = 0;
        TRY(run_lod_select(ctx, sl, sc->dev, cams[i].center, L > 1 ? d_inner + (size_t)i * (L - 1) : nullptr,
                           s, &n));
        act.list = sl.ws.list.as<uint32_t>();
        act.n = n;
        TRY(render_frame(ctx, sl, sc->dev, act, cams[i], d_rgb + off, s, nullptr,
                         stats ? stats + i : nullptr, true));
        off += (size_t)cams[i].width * cams[i].height * 3;
    }
    return LODGE_OK;
}

// Importance score (Sec. 3 "Importance pruning", "Visibility filtering"):
// render each camera with K12 and raise d_score[gid] to the largest weight.
lodge_status lodge_importance(lodge_ctx* ctx, int32_t scene_id, lodge_mode mode, int32_t chunk,
                              const lodge_camera* cams, int32_t n_cams, float* d_score, void* stream) {
    if (!ctx || !cams || !d_score || n_cams < 0) return fail(LODGE_E_INVALID, "bad argument");
    Scene* sc = get_scene(ctx, scene_id);
    if (!sc) return fail(LODGE_E_INVALID, "no scene %d", scene_id);
    if (chunk >= 0) {
        if (chunk >= (int32_t)sc->chunks.size()) return fail(LODGE_E_INVALID, "chunk %d out of range", chunk);
        if (sc->residency != kResident)
            return fail(LODGE_E_NOT_RESIDENT, "a chunk's own set is scored on resident scenes only");
    }
    CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Slot& sl = *ctx->slots[0];
    for (int i = 0; i < n_cams; ++i) {
        TRY(check_cam(cams[i]));
        TRY(ensure(ctx, sl.ws.img, sizeof(float) * 3 * (size_t)cams[i].width * cams[i].height, s));
        if (chunk >= 0) {
            Active act;
            act.list = sc->chunks[chunk].list;
            act.n = sc->chunks[chunk].n;
            act.A = chunk;
            TRY(render_frame(ctx, sl, sc->dev, act, cams[i], sl.ws.img.as<float>(), s, nullptr, nullptr,
                             true, d_score));
        } else {
            TRY(render_one(ctx, sl, sc, mode, cams[i], sl.ws.img.as<float>(), s, nullptr, nullptr, true,
                           d_score));
        }
    }
    return LODGE_OK;
}

// Visibility filtering (Sec. 3): keep the Gaussians of chunk `chunk` whose
// score reaches the threshold.
lodge_status lodge_filter_chunk(lodge_ctx* ctx, int32_t scene_id, int32_t chunk, const float* d_score,
                                float threshold, int64_t* n_kept, void* stream) {
    if (!ctx || !d_score) return fail(LODGE_E_INVALID, "bad argument");
    Scene* sc = get_scene(ctx, scene_id);
    if (!sc) return fail(LODGE_E_INVALID, "no scene %d", scene_id);
    if (chunk < 0 || chunk >= (int32_t)sc->chunks.size()) return fail(LODGE_E_INVALID, "chunk %d out of range", chunk);
    if (sc->residency != kResident)
        return fail(LODGE_E_NOT_RESIDENT, "visibility filtering edits resident chunk sets only");
    if (!std::isfinite(threshold)) return fail(LODGE_E_INVALID, "threshold must be finite");
    CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Slot& sl = *ctx->slots[0];
    Chunk& ch = sc->chunks[chunk];
    const int64_t n = ch.n;
    const int64_t ntiles = std::max<int64_t>((n + kSelectTile - 1) / kSelectTile, 1);
    TRY(ensure(ctx, sl.ws.list, sizeof(uint32_t) * (size_t)std::max<int64_t>(n, 1), s));
    TRY(ensure(ctx, sl.ws.status, sizeof(uint32_t) * (size_t)ntiles, s));
    CUDA_TRY(cudaMemsetAsync(sl.ws.status.p, 0, sizeof(uint32_t) * (size_t)ntiles, s));
    CUDA_TRY(cudaMemsetAsync(sl.d_small, 0, sizeof(uint32_t) * kSmWords, s));
    launch_score_filter(ch.list, n, d_score, threshold, sc->dev.n_total, sl.ws.list.as<uint32_t>(),
                        sl.d_small + kSmListCount, sl.ws.status.as<uint32_t>(), sl.d_small + kSmCtrSelect,
                        sl.d_small + kSmErr, s);
    CUDA_TRY(cudaGetLastError());
    TRY(sync_slot(ctx, sl, s));
    const int64_t kept = sl.h_small[kSmListCount];
    void* p = nullptr;
    TRY(dmalloc(ctx, &p, sizeof(uint32_t) * (size_t)std::max<int64_t>(kept, 1)));
    if (kept) CUDA_TRY(cudaMemcpyAsync(p, sl.ws.list.p, sizeof(uint32_t) * (size_t)kept,
                                       cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    dfree(ctx, ch.list, sizeof(uint32_t) * (size_t)std::max<int64_t>(n, 1));
    sc->chunk_bytes -= sizeof(uint32_t) * (size_t)std::max<int64_t>(n, 1);
    sc->chunk_bytes += sizeof(uint32_t) * (size_t)std::max<int64_t>(kept, 1);
    ch.list = static_cast<uint32_t*>(p);
    ch.n = kept;
    // cached unions may hold the old set
    CUDA_TRY(cudaDeviceSynchronize());
    free_pair_unions(ctx, *sc);
    for (auto& slp : ctx->slots) {
        slp->u_scene = -1;
        for (auto& u : slp->ucache)
            if (u.scene == scene_id) u.scene = -1;
    }
    if (n_kept) *n_kept = kept;
    return LODGE_OK;
}

lodge_status lodge_render_params(lodge_ctx* ctx, int64_t n, const float* d_means, const float* d_log_scales,
                                 const float* d_quats, const float* d_opacity_logits, const float* d_sh,
                                 int32_t sh_degree, float filter_var, const lodge_camera* cam, float* d_rgb,
                                 void* stream, int32_t save_for_backward, int64_t* handle_out,
                                 lodge_frame_stats* stats) {
    if (!ctx || !cam || !d_rgb || n < 0) return fail(LODGE_E_INVALID, "bad argument");
    if (n >= (1ll << 30)) return fail(LODGE_E_INVALID, "too many Gaussians");
    if (n > 0 && (!d_means || !d_log_scales || !d_quats || !d_opacity_logits || !d_sh))
        return fail(LODGE_E_INVALID, "NULL parameter array");
    if (sh_degree < 0 || sh_degree > 3) return fail(LODGE_E_INVALID, "sh_degree outside 0..3");
    if ((uintptr_t)d_sh % 16 != 0) return fail(LODGE_E_INVALID, "d_sh must be 16-byte aligned");
    if (save_for_backward && !handle_out) return fail(LODGE_E_INVALID, "handle_out is NULL");
    CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Slot& sl = *ctx->slots[0];
    Workspace& ws = sl.ws;
    const size_t n1 = (size_t)std::max<int64_t>(n, 1);
    const int64_t NP = std::max<int64_t>((n + 63) / 64 * 64, 64);
    TRY(ensure(ctx, ws.act_so, sizeof(float4) * n1, s));
    TRY(ensure(ctx, ws.act_q, sizeof(float4) * n1, s));
    TRY(ensure(ctx, ws.mtmp, sizeof(float) * 3 * (size_t)NP + sizeof(float4) * 12 * (size_t)NP, s));
    float* mp = ws.mtmp.as<float>();
    float4* shp = reinterpret_cast<float4*>(mp + 3 * NP);
    if (n) {
        unsigned nb = (unsigned)((n + 255) / 256);
        activate_kernel<<<nb, 256, 0, s>>>(n, d_log_scales, d_quats, d_opacity_logits, ws.act_so.as<float4>(), ws.act_q.as<float4>());
        planes_kernel<<<nb, 256, 0, s>>>(n, d_means, mp, mp + NP, mp + 2 * NP);
        sh_planes_kernel<<<nb, 256, 0, s>>>(n, d_sh, shp, NP);
        CUDA_TRY(cudaGetLastError());
    }
    DevScene d;
    d.n_total = n;
    d.num_levels = 1;
    d.sh_degree = sh_degree;
    d.level_off[0] = 0;
    for (int l = 1; l <= kMaxLevels; ++l) d.level_off[l] = n;
    d.filter_var[0] = filter_var;
    d.mx = mp; d.my = mp + NP; d.mz = mp + 2 * NP;
    d.scale_op = ws.act_so.as<float4>();
    d.quat = ws.act_q.as<float4>();
    d.sh = shp;
    Active act;
    act.n = n;
    std::unique_ptr<Saved> sv;
    if (save_for_backward) sv.reset(new Saved());
    TRY(render_frame(ctx, sl, d, act, *cam, d_rgb, s, sv.get(), stats, true));
    if (sv) {
        sv->params = true;
        sv->n = n;
        sv->means = d_means; sv->log_scales = d_log_scales; sv->quats = d_quats;
        sv->logits = d_opacity_logits; sv->sh = d_sh;
        sv->sh_degree = sh_degree;
        sv->lv.num_levels = 1;
        for (int l = 1; l <= kMaxLevels; ++l) sv->lv.level_off[l] = n;
        sv->lv.filter_var[0] = filter_var;
        sv->lv.train_lo = 0;
        sv->lv.train_hi = n;
        take(sv->act_so, ws.act_so);
        take(sv->act_q, ws.act_q);
        std::lock_guard<std::recursive_mutex> lk(ctx->mu);
        int64_t h = ctx->next_handle++;
        ctx->saved[h] = std::move(sv);
        *handle_out = h;
    }
    return LODGE_OK;
}

// LOD rendering of levels given as raw device parameters (supplementary
// "LOD structure optimization steps": the build of level l fine-tunes G_l
// with LOD rendering of the levels up to l, d_l drawn per step).  The levels
// are activated into one gid-ordered store (finest first), Eq. 2 selects
// each level's band at the camera centre with this frame's thresholds, and
// the frame is rendered as any LOD frame.  With d_score it raises the
// importance scores instead (K12); with save_for_backward the adjoint will
// give gradients of level train_level only.
lodge_status lodge_render_params_lod(lodge_ctx* ctx, int32_t num_levels, const int64_t* level_n,
                                     const float* const* d_means, const float* const* d_log_scales,
                                     const float* const* d_quats, const float* const* d_opacity_logits,
                                     const float* const* d_sh, int32_t sh_degree, const float* filter_var,
                                     const double* d_inner, const lodge_camera* cam, float* d_rgb,
                                     float* d_score, int32_t train_level, void* stream,
                                     int32_t save_for_backward, int64_t* handle_out,
                                     lodge_frame_stats* stats) {
    if (!ctx || !cam || !d_rgb || !level_n || !filter_var) return fail(LODGE_E_INVALID, "bad argument");
    if (num_levels < 1 || num_levels > kMaxLevels) return fail(LODGE_E_INVALID, "num_levels outside 1..%d", kMaxLevels);
    if (num_levels > 1 && !d_inner) return fail(LODGE_E_INVALID, "d_inner is NULL");
    if (!d_means || !d_log_scales || !d_quats || !d_opacity_logits || !d_sh)
        return fail(LODGE_E_INVALID, "NULL parameter pointer table");
    if (sh_degree < 0 || sh_degree > 3) return fail(LODGE_E_INVALID, "sh_degree outside 0..3");
    if (save_for_backward && (!handle_out || d_score))
        return fail(LODGE_E_INVALID, "save_for_backward needs handle_out and no d_score");
    if (save_for_backward && (train_level < 0 || train_level >= num_levels))
        return fail(LODGE_E_INVALID, "train_level outside 0..num_levels-1");
    int64_t off[kMaxLevels + 1] = {0};
    for (int l = 0; l < num_levels; ++l) {
        if (level_n[l] < 0) return fail(LODGE_E_INVALID, "level %d: negative size", l);
        if (level_n[l] > 0 && (!d_means[l] || !d_log_scales[l] || !d_quats[l] || !d_opacity_logits[l] || !d_sh[l]))
            return fail(LODGE_E_INVALID, "level %d: NULL parameter array", l);
        if (level_n[l] > 0 && (uintptr_t)d_sh[l] % 16 != 0)
            return fail(LODGE_E_INVALID, "level %d: SH array must be 16-byte aligned", l);
        if (!(filter_var[l] >= 0.f) || !std::isfinite(filter_var[l]))
            return fail(LODGE_E_INVALID, "level %d: filter variance must be finite and >= 0", l);
        off[l + 1] = off[l] + level_n[l];
    }
    for (int l = num_levels + 1; l <= kMaxLevels; ++l) off[l] = off[num_levels];
    const int64_t n = off[num_levels];
    if (n >= (1ll << 30)) return fail(LODGE_E_INVALID, "too many Gaussians");
    for (int l = 0; l + 1 < num_levels; ++l)
        if (!(d_inner[l] >= 0.0) || (l && !(d_inner[l] >= d_inner[l - 1])))
            return fail(LODGE_E_INVALID, "thresholds must be non-negative and ascending");
    CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Slot& sl = *ctx->slots[0];
    Workspace& ws = sl.ws;
    const size_t n1 = (size_t)std::max<int64_t>(n, 1);
    const int64_t NP = std::max<int64_t>((n + 63) / 64 * 64, 64);
    TRY(ensure(ctx, ws.act_so, sizeof(float4) * n1, s));
    TRY(ensure(ctx, ws.act_q, sizeof(float4) * n1, s));
    TRY(ensure(ctx, ws.mtmp, sizeof(float) * 3 * (size_t)NP + sizeof(float4) * 12 * (size_t)NP, s));
    float* mp = ws.mtmp.as<float>();
    float4* shp = reinterpret_cast<float4*>(mp + 3 * NP);
    for (int l = 0; l < num_levels; ++l) {
        const int64_t nl = level_n[l], o = off[l];
        if (!nl) continue;
        unsigned nb = (unsigned)((nl + 255) / 256);
        activate_kernel<<<nb, 256, 0, s>>>(nl, d_log_scales[l], d_quats[l], d_opacity_logits[l],
                                           ws.act_so.as<float4>() + o, ws.act_q.as<float4>() + o);
        planes_kernel<<<nb, 256, 0, s>>>(nl, d_means[l], mp + o, mp + NP + o, mp + 2 * NP + o);
        sh_planes_kernel<<<nb, 256, 0, s>>>(nl, d_sh[l], shp + o, NP);
        CUDA_TRY(cudaGetLastError());
    }
    DevScene d;
    d.n_total = n;
    d.num_levels = num_levels;
    d.sh_degree = sh_degree;
    for (int l = 0; l <= kMaxLevels; ++l) d.level_off[l] = off[l];
    for (int l = 0; l < num_levels; ++l) d.filter_var[l] = filter_var[l];
    d.mx = mp; d.my = mp + NP; d.mz = mp + 2 * NP;
    d.scale_op = ws.act_so.as<float4>();
    d.quat = ws.act_q.as<float4>();
    d.sh = shp;
    Active act;
    if (num_levels > 1) {
        int64_t na = 0;
        TRY(run_lod_select(ctx, sl, d, cam->center, d_inner, s, &na));
        act.list = ws.list.as<uint32_t>();
        act.n = na;
    } else {
        act.n = n;
    }
    std::unique_ptr<Saved> sv;
    if (save_for_backward) sv.reset(new Saved());
    TRY(render_frame(ctx, sl, d, act, *cam, d_rgb, s, sv.get(), stats, true, d_score));
    if (sv) {
        const int tl = train_level;
        sv->params = true;
        sv->n = n;
        sv->means = d_means[tl]; sv->log_scales = d_log_scales[tl]; sv->quats = d_quats[tl];
        sv->logits = d_opacity_logits[tl]; sv->sh = d_sh[tl];
        sv->sh_degree = sh_degree;
        sv->lv.num_levels = num_levels;
        for (int l = 0; l <= kMaxLevels; ++l) sv->lv.level_off[l] = off[l];
        for (int l = 0; l < num_levels; ++l) sv->lv.filter_var[l] = filter_var[l];
        sv->lv.train_lo = off[tl];
        sv->lv.train_hi = off[tl + 1];
        take(sv->act_so, ws.act_so);
        take(sv->act_q, ws.act_q);
        std::lock_guard<std::recursive_mutex> lk(ctx->mu);
        int64_t h = ctx->next_handle++;
        ctx->saved[h] = std::move(sv);
        *handle_out = h;
    }
    return LODGE_OK;
}

lodge_status lodge_render_backward(lodge_ctx* ctx, int64_t handle, const float* d_dL_drgb, float* d_g_means,
                                   float* d_g_log_scales, float* d_g_quats, float* d_g_opacity_logits,
                                   float* d_g_sh, void* stream) {
    if (!ctx || !d_dL_drgb) return fail(LODGE_E_INVALID, "bad argument");
    auto it = ctx->saved.find(handle);
    if (it == ctx->saved.end()) return fail(LODGE_E_INVALID, "no saved frame %lld", (long long)handle);
    Saved& v = *it->second;
    if (!v.params) return fail(LODGE_E_INVALID, "frame %lld was not rendered from parameters", (long long)handle);
    CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Slot& sl = *ctx->slots[0];
    Workspace& ws = sl.ws;
    const size_t n9 = 9 * (size_t)std::max<int64_t>(v.n_vis, 1);
    TRY(ensure(ctx, ws.grec, sizeof(double) * n9, s));
    CUDA_TRY(cudaMemsetAsync(ws.grec.p, 0, sizeof(double) * n9, s));
    CUDA_TRY(cudaMemsetAsync(sl.d_small, 0, sizeof(uint32_t) * kSmWords, s));
    launch_blend_bwd(v.cam, v.ranges.as<uint2>(), v.rbits ? v.tkey.as<uint32_t>() : v.tval.as<uint32_t>(),
                     v.rbits ? (1u << v.rbits) - 1u : 0xffffffffu, v.n_keys, v.rec_a.as<float4>(),
                     v.rec_b.as<float4>(), v.rec_c.as<float>(), v.n_vis, v.T.as<float>(),
                     v.last.as<uint32_t>(), d_dL_drgb, ws.grec.as<double>(), s);
    launch_project_bwd(v.cam, v.n_vis, v.rec_gid.as<uint32_t>(), ws.grec.as<double>(), v.means,
                       v.act_so.as<float4>(), v.act_q.as<float4>(), v.quats, v.sh, v.sh_degree,
                       v.lv, d_g_means, d_g_log_scales, d_g_quats, d_g_opacity_logits, d_g_sh, s);
    CUDA_TRY(cudaGetLastError());
    return sync_slot(ctx, sl, s);
}

lodge_status lodge_release(lodge_ctx* ctx, int64_t handle) {
    if (!ctx) return fail(LODGE_E_INVALID, "NULL context");
    std::unique_ptr<Saved> v;
    {
        std::lock_guard<std::recursive_mutex> lk(ctx->mu);
        auto it = ctx->saved.find(handle);
        if (it == ctx->saved.end()) return fail(LODGE_E_INVALID, "no saved frame %lld", (long long)handle);
        v = std::move(it->second);
        ctx->saved.erase(it);
    }
    CUDA_TRY(cudaSetDevice(ctx->device));
    free_saved(ctx, *v, false);
    return LODGE_OK;
}

lodge_status lodge_debug_keys(lodge_ctx* ctx, int64_t handle, uint64_t* d_keys, uint32_t* d_gids, int64_t cap,
                              int64_t* n_keys, void* stream) {
    if (!ctx || !n_keys) return fail(LODGE_E_INVALID, "bad argument");
    auto it = ctx->saved.find(handle);
    if (it == ctx->saved.end()) return fail(LODGE_E_INVALID, "no saved frame %lld", (long long)handle);
    CUDA_TRY(cudaSetDevice(ctx->device));
    Saved& v = *it->second;
    *n_keys = v.n_keys;
    if (v.n_keys > cap) return fail(LODGE_E_OVERFLOW, "%lld keys > capacity %lld", (long long)v.n_keys, (long long)cap);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DBuf zrec;
    TRY(ensure(ctx, zrec, sizeof(uint32_t) * (size_t)std::max<int64_t>(v.n_vis, 1), s));
    if (v.n_vis) zrec_kernel<<<(unsigned)((v.n_vis + 255) / 256), 256, 0, s>>>(v.zsorted.as<uint32_t>(), v.rsorted.as<uint32_t>(), v.n_vis, zrec.as<uint32_t>());
    if (v.n_keys) debug_keys_kernel<<<(unsigned)((v.n_keys + 255) / 256), 256, 0, s>>>(v.tkey.as<uint32_t>(), v.tval.as<uint32_t>(), v.rbits, v.n_keys, std::max<int64_t>(v.n_vis, 1), zrec.as<uint32_t>(), v.rec_gid.as<uint32_t>(), d_keys, d_gids);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(s));
    release(ctx, zrec, s);
    return LODGE_OK;
}

lodge_status lodge_debug_records(lodge_ctx* ctx, int64_t handle, uint32_t* d_gid, float* d_depth, int32_t* d_rect,
                                 float* d_mean2, float* d_conic, float* d_opacity, float* d_rgb, int64_t cap,
                                 int64_t* n_visible, void* stream) {
    if (!ctx || !n_visible) return fail(LODGE_E_INVALID, "bad argument");
    auto it = ctx->saved.find(handle);
    if (it == ctx->saved.end()) return fail(LODGE_E_INVALID, "no saved frame %lld", (long long)handle);
    CUDA_TRY(cudaSetDevice(ctx->device));
    Saved& v = *it->second;
    *n_visible = v.n_vis;
    if (v.n_vis > cap) return fail(LODGE_E_OVERFLOW, "%lld records > capacity %lld", (long long)v.n_vis, (long long)cap);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DBuf zrec;
    TRY(ensure(ctx, zrec, sizeof(uint32_t) * (size_t)std::max<int64_t>(v.n_vis, 1), s));
    if (v.n_vis) {
        unsigned nb = (unsigned)((v.n_vis + 255) / 256);
        zrec_kernel<<<nb, 256, 0, s>>>(v.zsorted.as<uint32_t>(), v.rsorted.as<uint32_t>(), v.n_vis, zrec.as<uint32_t>());
        debug_records_kernel<<<nb, 256, 0, s>>>(v.n_vis, v.rec_a.as<float4>(), v.rec_b.as<float4>(), v.rec_c.as<float>(),
                                               v.rec_rect.as<uint2>(), v.rec_gid.as<uint32_t>(), zrec.as<uint32_t>(),
                                               d_gid, d_depth, d_rect, d_mean2, d_conic, d_opacity, d_rgb);
    }
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(s));
    release(ctx, zrec, s);
    return LODGE_OK;
}

lodge_status lodge_sort_pairs(lodge_ctx* ctx, uint32_t* d_keys, uint32_t* d_vals, int64_t n, int32_t key_bits,
                              void* stream) {
    if (!ctx || n < 0 || key_bits < 0 || key_bits > 32) return fail(LODGE_E_INVALID, "bad argument");
    if (n >= (1ll << 30)) return fail(LODGE_E_INVALID, "n must be below 2^30");
    if (n > 0 && (!d_keys || !d_vals)) return fail(LODGE_E_INVALID, "NULL key or value array");
    CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Slot& sl = *ctx->slots[0];
    Workspace& ws = sl.ws;
    const size_t n1 = (size_t)std::max<int64_t>(n, 1);
    TRY(ensure(ctx, ws.tkey2, sizeof(uint32_t) * n1, s));
    TRY(ensure(ctx, ws.tval2, sizeof(uint32_t) * n1, s));
    TRY(ensure(ctx, ws.sort, sort_scratch_bytes(n, key_bits), s));
    CUDA_TRY(cudaMemsetAsync(sl.d_small, 0, sizeof(uint32_t) * kSmWords, s));
    int w = launch_onesweep(d_keys, d_vals, ws.tkey2.as<uint32_t>(), ws.tval2.as<uint32_t>(), n, key_bits,
                            ws.sort.p, sl.d_small + kSmErr, s);
    if (w) {
        CUDA_TRY(cudaMemcpyAsync(d_keys, ws.tkey2.p, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(d_vals, ws.tval2.p, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
    }
    CUDA_TRY(cudaGetLastError());
    return sync_slot(ctx, sl, s);
}

lodge_status lodge_profile_enable(lodge_ctx* ctx, int enable) {
    if (!ctx) return fail(LODGE_E_INVALID, "NULL context");
    for (auto& slp : ctx->slots) {
        Slot& sl = *slp;
        sl.prof = lodge_profile{};
        for (int k = 0; k < LODGE_NUM_STAGES; ++k) sl.ev_pending[k] = false;
        sl.prof_on = enable != 0;
        sl.prof_count = enable == 2;
    }
    return LODGE_OK;
}

// the sum over the context's slots (frames of one call may alternate
// between two)
lodge_status lodge_profile_read(lodge_ctx* ctx, lodge_profile* out) {
    if (!ctx || !out) return fail(LODGE_E_INVALID, "bad argument");
    lodge_profile p{};
    for (auto& slp : ctx->slots) {
        const lodge_profile& q = slp->prof;
        for (int k = 0; k < LODGE_NUM_STAGES; ++k) {
            p.ms[k] += q.ms[k];
            p.launches[k] += q.launches[k];
        }
        p.frames += q.frames;
        p.keys += q.keys;
        p.visible += q.visible;
        p.active += q.active;
        p.packed_keys += q.packed_keys;
        p.bin_keys += q.bin_keys;
        p.bin_sort_passes += q.bin_sort_passes;
        p.blend_pairs += q.blend_pairs;
        p.blend_pairs_used += q.blend_pairs_used;
        p.redone += q.redone;
        p.host_ms += q.host_ms;
    }
    *out = p;
    return LODGE_OK;
}

lodge_status lodge_residency_stats(lodge_ctx* ctx, lodge_residency* out) {
    if (!ctx || !out) return fail(LODGE_E_INVALID, "bad argument");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    out->resident_blocks = (int64_t)ctx->blocks.size();
    out->block_hits = ctx->res.hits;
    out->block_uploads = ctx->res.uploads;
    out->block_evictions = ctx->res.evictions;
    out->upload_bytes = ctx->res.upload_bytes;
    out->failed_uploads = ctx->res.failed_uploads;
    out->hbm_used = (int64_t)ctx->used;
    out->hbm_budget = (int64_t)ctx->budget;
    return LODGE_OK;
}

lodge_status lodge_set_bin_size(lodge_ctx* ctx, int32_t log2_tiles) {
    if (!ctx || log2_tiles < -1 || log2_tiles > 3) return fail(LODGE_E_INVALID, "bad argument");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    ctx->bin_log2 = log2_tiles;
    return LODGE_OK;
}

lodge_status lodge_inject_upload_failures(lodge_ctx* ctx, int32_t n) {
    if (!ctx || n < 0) return fail(LODGE_E_INVALID, "bad argument");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    ctx->fail_next_uploads = n;
    return LODGE_OK;
}

}  // extern "C"
