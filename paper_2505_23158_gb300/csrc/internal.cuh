// Host-side state of a context, shared by lodge_capi.cu (API, scenes, frame
// orchestration), residency.cu (streamed chunk blocks) and serve.cu (the
// request loop).
#pragma once

#include <condition_variable>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <utility>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace lodge {

struct DBuf {
    void* p = nullptr;
    size_t cap = 0;
    template <class T> T* as() const { return static_cast<T*>(p); }
};

struct Chunk {
    uint32_t* list = nullptr;  // resident: device list; streamed: pinned host list
    int64_t n = 0;
};

// One chunk's active set resident in HBM (streamed scenes): the sorted gid
// list and the attributes of its Gaussians as structure-of-arrays planes.
struct Block {
    int scene = -1, chunk = -1;
    int64_t n = 0;
    void* mem = nullptr;
    size_t bytes = 0;
    uint32_t* gid = nullptr;
    DevScene view;                 // planes with stride n_pad, scene level info
    int64_t n_pad = 0;
    int refs = 0;
    uint64_t last_use = 0;
    cudaEvent_t ready = nullptr;   // recorded on the upload stream after the gather
};

enum : int { kResident = 0, kStreamed = 1 };

struct Scene {
    int id = -1;
    int residency = kResident;
    DevScene dev;          // resident: device store; streamed: device-visible view of the host store
    void* block = nullptr; // resident device store
    size_t block_bytes = 0;
    void* host_store = nullptr;  // streamed: pinned, mapped host store
    size_t host_bytes = 0;
    uint32_t* host_lists = nullptr;  // streamed: pinned chunk lists, back to back
    int64_t n_pad = 0;
    std::vector<double> d_inner;
    std::vector<double> centers;
    std::vector<double> radius;
    std::vector<Chunk> chunks;
    size_t chunk_bytes = 0;
    // resident scenes: unions of chunk pairs met so far, shared by every slot
    // (computed once and kept while the chunk sets stay as they are)
    struct PairUnion {
        DBuf list;
        int64_t n = 0;
    };
    std::unordered_map<uint64_t, PairUnion> unions;
};
constexpr size_t kMaxPairUnions = 1024;   // per scene; beyond, slots cache their own

struct Saved {
    DevCamera cam{};
    int64_t n_vis = 0, n_keys = 0;
    int rbits = 0;  // > 0: tkey holds packed tile << rbits | record, tval unused
    DBuf rec_a, rec_b, rec_c, rec_rect, rec_gid, zsorted, rsorted, tkey, tval, ranges, T, last;
    bool params = false;
    int64_t n = 0;
    const float *means = nullptr, *log_scales = nullptr, *quats = nullptr, *logits = nullptr,
                *sh = nullptr;
    int sh_degree = 3;
    BwdLevels lv;            // levels, filter variances and the trained level's gid range
    DBuf act_so, act_q;
};

struct Workspace {
    DBuf list, marks, status, rec_a, rec_b, rec_c, rec_rect, rec_gid, dkey, dval, dkey2, dval2,
        tkey, tval, tkey2, tval2, ranges, sort, T, last, img, act_so, act_q, mtmp, koff, srec,
        srect, doffs, grec, bonly, iscore,
        status2, sort2;   // frames without a mid-frame sync: emission and bin-sort scratch of their own
    std::vector<DBuf*> all() {
        return {&list, &marks, &status, &rec_a, &rec_b, &rec_c, &rec_rect, &rec_gid, &dkey, &dval,
                &dkey2, &dval2, &tkey, &tval, &tkey2, &tval2, &ranges, &sort, &T, &last, &img,
                &act_so, &act_q, &mtmp, &koff, &srec, &srect, &doffs, &grec, &bonly, &iscore,
                &status2, &sort2};
    }
};

// small device/host words of a slot
enum : int {
    kSmErr = 0,
    kSmListCount = 1,
    kSmProj = 2,        // [2] visible, [4..5] keys (u64)
    kSmCtrSelect = 8,
    kSmCtrUnion = 9,
    kSmCtrProj = 10,
    kSmCtrEmit = 11,
    kSmPairs = 12,      // [12..13] pairs evaluated, [14..15] composited (u64, counting mode)
    kSmCtrBlend = 16,   // next tile of the compositing CTAs
    kSmWords = 64
};

// Render state of one in-flight frame: scratch, status words, stage profile
// and the union of the last chunk pair.  Slot 0 serves the single-threaded
// API; the request loop adds one slot per concurrent request.
struct Slot {
    int index = 0;
    cudaStream_t own = nullptr;   // stream created for this slot (request loop)
    cudaEvent_t fence = nullptr;  // orders slot 1's stream against the caller's
    cudaStream_t copy = nullptr;   // host-buffer calls: the images' copies back to the host
    cudaEvent_t copy_ev = nullptr; // a frame's end on its render stream, for its copy
    Workspace ws;
    uint32_t* d_small = nullptr;
    uint32_t* h_small = nullptr;  // pinned
    // status words of a frame whose end was not waited for: copied on the
    // stream after its last kernel, checked at the slot's next sync
    uint32_t* h_tail = nullptr;   // pinned
    bool tail_pending = false;
    // Frames rendered with their counts left on the device (no mid-frame
    // sync): scratch is sized by capacities, the bin keys by key_cap (grown
    // from the frames that did sync).  Each such frame copies its status
    // words into a pinned ring entry; the slot's harvest reads them.
    int64_t key_cap = 0;
    int key_cap_bl = -1;          // the bin size key_cap was learned for
    static constexpr int kRing = 32;
    uint32_t* h_ring = nullptr;   // pinned, kRing x kSmWords
    cudaEvent_t ring_ev[kRing] = {};   // each entry's copy done (on the frame's stream)
    int ring_next = 0;
    struct Pending {
        int ring = 0;                   // ring entry
        int frame = 0;                  // index in the caller's list (set by the caller)
        bool used = false;              // the frame took this path
        lodge_frame_stats* st = nullptr;
        int64_t n_active = 0, n_tiles = 0;
        int A = -1, B = -1;
        double tA = 1.0, tB = 1.0;
        bool packed = false;            // bin keys packed with the record
        int sort_passes = 0;
        int bin_log2 = 0;               // 0: per-tile lists (bin keys = tile keys)
    };
    std::vector<Pending> pending;
    bool prof_on = false;
    bool prof_count = false;   // compositing counts its (pixel, Gaussian) pairs
    // other slots' frames run at the same time (several render streams, the
    // request loop): compositing then leaves room on every SM for them
    bool share_sms = false;
    int64_t uploads = 0;       // chunk blocks this slot's frames have gathered
    lodge_profile prof{};
    cudaEvent_t ev_beg[LODGE_NUM_STAGES] = {};
    cudaEvent_t ev_end[LODGE_NUM_STAGES] = {};
    bool ev_pending[LODGE_NUM_STAGES] = {};
    int u_scene = -1, ua = -2, ub = -2;
    int64_t un = 0;
    DBuf ulist;
    Block* held[2] = {nullptr, nullptr};
    // unions of recent chunk pairs of resident scenes, least recently used
    // replaced first (a camera moving inside a cell alternates between a few
    // pairs)
    struct UnionEntry {
        int scene = -1, a = -1, b = -1;
        int64_t n = 0;
        uint64_t used = 0;
        DBuf list;
    };
    static constexpr int kUnionCache = 16;
    UnionEntry ucache[kUnionCache];
    uint64_t utick = 0;
};

struct ResidencyStats {
    int64_t hits = 0, uploads = 0, evictions = 0, upload_bytes = 0, failed_uploads = 0;
};

}  // namespace lodge

struct lodge_ctx {
    int device = 0;
    size_t budget = 0;
    size_t used = 0;                 // device bytes held; guarded by mu
    std::recursive_mutex mu;         // budget, blocks, saved frames, slot list
    std::condition_variable_any freed;  // signalled when device memory is released
    std::vector<std::unique_ptr<lodge::Scene>> scenes;
    std::vector<std::unique_ptr<lodge::Slot>> slots;
    std::map<int64_t, std::unique_ptr<lodge::Saved>> saved;
    int64_t next_handle = 1;
    // streamed residency
    std::map<std::pair<int, int>, std::unique_ptr<lodge::Block>> blocks;
    uint64_t tick = 0;
    cudaStream_t upload_stream = nullptr;
    lodge::ResidencyStats res;
    int fail_next_uploads = 0;       // host-side fault injection
    int bin_log2 = -1;               // key lists per bin of 2^bin_log2 x 2^bin_log2 tiles (-1: by frame)
};

namespace lodge {

// errors (thread-local message)
lodge_status fail(lodge_status s, const char* fmt, ...);

// device memory with budget accounting (thread-safe)
lodge_status dmalloc(lodge_ctx* ctx, void** p, size_t bytes);
void dfree(lodge_ctx* ctx, void* p, size_t bytes);
lodge_status ensure(lodge_ctx* ctx, DBuf& b, size_t bytes, cudaStream_t s);
void release(lodge_ctx* ctx, DBuf& b, cudaStream_t s);
// evict unreferenced blocks (least recently used first) until `bytes` more
// fit in the budget; caller holds ctx->mu; returns false if they cannot
bool make_room(lodge_ctx* ctx, size_t bytes);

lodge_status sync_slot(lodge_ctx* ctx, Slot& sl, cudaStream_t s);
const char* last_error();
lodge_status create_slot(lodge_ctx* ctx, Slot** out);
// slot k >= 1 with its own stream (created on first use)
lodge_status stream_slot(lodge_ctx* ctx, int k, Slot** out);
// streams the frames of one multi-camera render call take turns on: eight
// for chunk frames, three for full-detail frames, whose working set (the
// whole finest level) is far larger than L2 (measured at 1080p: chunk frames
// 5519 / 5718 / 5803 frames/s with 4 / 6 / 8 streams; full-detail frames
// 596 / 705 with 2 / 3, their long compositing tails filled by the next
// frame's stages)
constexpr int kRenderStreams = 8;
constexpr int kRenderStreamsFull = 3;

// a batch of frames composited by one launch (lodge_capi.cu)
struct BatchItem {
    Scene* sc = nullptr;
    lodge_mode mode = LODGE_FULL;
    lodge_camera cam{};
    float* d_rgb = nullptr;
    lodge_frame_stats* st = nullptr;
    lodge_status status = LODGE_OK;
};
lodge_status render_batch(lodge_ctx* ctx, BatchItem* items, int n, int first, cudaStream_t s);
// select and render one camera on a slot (lodge_capi.cu); pend != null lets
// a frame of a resident scene skip its mid-frame sync (Slot::Pending)
lodge_status render_one(lodge_ctx* ctx, Slot& sl, Scene* sc, lodge_mode mode, const lodge_camera& cam,
                        float* d_rgb, cudaStream_t s, Saved* save, lodge_frame_stats* st, bool end_sync,
                        float* importance, Slot::Pending* pend = nullptr);

// residency (residency.cu)
lodge_status acquire_block(lodge_ctx* ctx, Slot& sl, Scene* sc, int chunk, cudaStream_t s,
                           Block** out);
void release_blocks(lodge_ctx* ctx, Slot& sl);
void free_scene_blocks(lodge_ctx* ctx, int scene);
// union of two blocks' sorted gid lists into sl.ulist: entries are the index
// into block A (bit 31 set) or block B (bit 30 only); bit 30 is also set on
// A entries present in B.  b may be null (single block).
lodge_status block_union(lodge_ctx* ctx, Slot& sl, const Block* a, const Block* b,
                         cudaStream_t s, int64_t* n_out);

}  // namespace lodge
