/*
 * lodge.h - C ABI of the GB300 (sm_103a) LODGE frame renderer.
 *
 * The library renders a level-of-detail, chunked 3D Gaussian Splatting
 * scene (arXiv 2505.23158, "LODGE") on one GPU.  Per camera it
 *   1. picks the two nearest chunk centres and the Eq. 4 blend weights
 *      (Sec. 3 "Opacity blending"),
 *   2. takes the active Gaussian set: Eq. 2 at the camera (LOD mode), the
 *      precomputed set of the nearest chunk (CHUNK), or the union of the two
 *      nearest chunks with Eq. 4 opacity modulation (CHUNK_BLEND)
 *      (Sec. 3 "LOD representation", "Chunk-based rendering"),
 *   3. projects the active Gaussians with EWA covariance, the per-level 3D
 *      filter of Eq. 3 and degree-3 SH colour (Sec. 3 "Preliminaries: 3DGS"),
 *   4. bins them to 16x16 tiles, sorts (tile, depth) keys and composites each
 *      tile front to back with Eq. 1 alpha (Sec. 3 "Preliminaries: 3DGS").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Errors: every call returns a lodge_status; LODGE_OK is 0.  No call aborts
 *   or throws across the ABI.  lodge_last_error() returns a message for the
 *   last failing call on the calling thread (valid until the next call on
 *   that thread).
 * Pointers: parameters named d_* are DEVICE pointers on the context's
 *   device; every other pointer is a HOST pointer.  All pointers are
 *   borrowed for the duration of the call only, except where stated.
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Device work of a call is ordered on that stream; host outputs
 *   are valid when the call returns (the call synchronises the stream where
 *   it returns host data).
 * Layouts: images are row-major H x W x 3 float32 (HWC), pixel (i, j) has
 *   its centre at (i + 0.5, j + 0.5).  Cameras map world to camera as
 *   p_c = R p_w + t with OpenCV axes (x right, y down, z forward).
 * Sizes: a scene holds at most 2^30 Gaussians in total; an image at most
 *   65535 tiles per side.
 */
#ifndef LODGE_H
#define LODGE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lodge_ctx lodge_ctx; /* opaque, owned by the library */

typedef enum {
    LODGE_OK = 0,
    LODGE_E_INVALID = 1,      /* bad argument (message says which) */
    LODGE_E_OOM = 2,          /* device or pinned host allocation failed */
    LODGE_E_CUDA = 3,         /* a CUDA runtime call failed */
    LODGE_E_NOT_RESIDENT = 4, /* chunk data not on the device (streaming mode) */
    LODGE_E_TIMEOUT = 5,      /* a bounded device-side wait gave up */
    LODGE_E_BUDGET = 6,       /* the context's HBM budget would be exceeded */
    LODGE_E_OVERFLOW = 7      /* an internal capacity was exceeded */
} lodge_status;

typedef enum {
    LODGE_FULL = 0,        /* every Gaussian of level 0 (full detail) */
    LODGE_LOD = 1,         /* Eq. 2 evaluated at the camera centre */
    LODGE_CHUNK = 2,       /* precomputed set of the nearest chunk */
    LODGE_CHUNK_BLEND = 3  /* union of the two nearest chunks, Eq. 4 */
} lodge_mode;

/* One LOD level G^(l), raw (un-activated) parameters, host memory,
 * caller-owned, copied by lodge_load_scene.  Activation at load, in FP64
 * rounded once to FP32: scale = exp(log_scale), opacity = sigmoid(logit),
 * quaternion divided by its norm. */
typedef struct {
    int64_t n;                    /* number of Gaussians in this level */
    const float* means;           /* n x 3 world positions */
    const float* log_scales;      /* n x 3 */
    const float* quats;           /* n x 4 (w, x, y, z), nonzero norm */
    const float* opacity_logits;  /* n */
    const float* sh;              /* n x 16 x 3 SH coefficients, coefficient-
                                     major, real basis order (l, m=-l..l) */
    float filter_var;             /* variance of the Eq. 3 3D smoothing filter
                                     for this level (0 = none) */
    float pad_;
} lodge_level_desc;

/* Where a scene's Gaussians live (Sec. 3 "Chunk-based rendering": only the
 * active sets of the chunks in use need GPU memory). */
typedef enum {
    LODGE_RESIDENT = 0,  /* every level in HBM; all four render modes */
    LODGE_STREAMED = 1   /* levels in pinned host memory; each chunk's active
                            set is gathered into an HBM block on first use and
                            cached under the context's budget (LRU eviction);
                            CHUNK and CHUNK_BLEND only */
} lodge_residency_mode;

typedef struct {
    int32_t num_levels;              /* L >= 1, at most 8 */
    int32_t sh_degree;               /* 0..3 */
    const lodge_level_desc* levels;  /* L levels, finest first (G^(0)) */
    const double* d_thresholds;      /* L - 1 ascending distances d_1..d_{L-1}
                                        (Eq. 2; d_0 = 0, d_L = inf) */
    int32_t num_chunks;              /* K >= 0 chunk centres (0: FULL/LOD only) */
    int32_t residency;               /* lodge_residency_mode */
    const double* chunk_centers;     /* K x 3 */
    int32_t filter2d;                /* 0: Sigma' = Sigma2D + 0.3 I (3DGS dilation);
                                        1: the same, and the opacity scaled by
                                        sqrt(det Sigma2D / det Sigma') (Mip-Splatting's
                                        2D filter, supplementary "Details on training
                                        the full representation") */
    int32_t pad_;
} lodge_scene_desc;

typedef struct {
    float R[9];        /* world -> camera rotation, row-major */
    float t[3];        /* world -> camera translation */
    float fx, fy;      /* focal lengths, pixels */
    float cx, cy;      /* principal point, pixels */
    int32_t width, height;
    float znear;       /* Gaussians with camera depth <= znear are culled */
    float pad_;
    double center[3];  /* camera position in world coordinates (FP64) */
} lodge_camera;

/* Per-camera outcome of the selection step (Eq. 2 / Eq. 4). */
typedef struct {
    int32_t chunk_a;   /* nearest chunk, -1 in FULL and LOD modes */
    int32_t chunk_b;   /* second nearest, -1 if none or not blending */
    double t_a, t_b;   /* Eq. 4 weights of A-only / B-only Gaussians */
    int64_t n_active;  /* size of the active set */
} lodge_selection;

/* Per-frame counters of a render (the paper's #G, #Vis. G and tile cost). */
typedef struct {
    int64_t n_active;    /* Gaussians selected (loaded for this frame) */
    int64_t n_visible;   /* Gaussians binned to at least one tile */
    int64_t n_keys;      /* (tile, Gaussian) pairs */
    int64_t n_tiles;     /* tiles in the image */
    int32_t chunk_a, chunk_b;
    double t_a, t_b;
} lodge_frame_stats;

/* ---------------------------------------------------------------- setup */

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the
 * device memory the context may hold (scenes + scratch); 0 = no cap.
 * *out receives the context; destroy it with lodge_destroy. */
lodge_status lodge_create(int device, size_t hbm_budget_bytes, lodge_ctx** out);

/* Free every device and host resource of the context.  NULL is a no-op. */
lodge_status lodge_destroy(lodge_ctx* ctx);

/* Message of the last failing call on this thread ("" if none). */
const char* lodge_last_error(void);

/* Copy a scene to the device (activated, structure-of-arrays, levels
 * concatenated in order, so a Gaussian's gid = its index in the
 * concatenation) and precompute every chunk's active set: Eq. 2 at the
 * chunk centre m_k with thresholds d_l + r_k, r_k = distance to the nearest
 * other chunk centre (Sec. 3 "Chunk-based rendering").  *scene_id receives
 * the scene handle.  Synchronous. */
lodge_status lodge_load_scene(lodge_ctx* ctx, const lodge_scene_desc* desc, int32_t* scene_id);

/* Release a scene's device memory. */
lodge_status lodge_unload_scene(lodge_ctx* ctx, int32_t scene_id);

/* Ensure the listed chunks' active sets are resident (Sec. 3 "Opacity
 * blending": sets are loaded in the background).  Resident scenes: nothing to
 * do.  Streamed scenes: each missing chunk block is gathered into HBM on the
 * context's side stream (evicting unreferenced blocks if the budget requires);
 * blocking != 0 waits for the uploads.  Errors: LODGE_E_BUDGET if a block
 * cannot fit, LODGE_E_CUDA on a failed upload. */
lodge_status lodge_upload_chunks(lodge_ctx* ctx, int32_t scene_id, const int32_t* chunk_ids,
                                 int32_t n, int blocking);

/* Selection only: for each of n_cams cameras fill out[i] (host).  If d_gids
 * is not NULL and n_cams == 1, the active gids (ascending, bit 31 = member
 * of chunk A, bit 30 = member of chunk B in CHUNK_BLEND mode, else 0) are
 * written to d_gids (device, capacity gids_capacity entries); LODGE_E_OVERFLOW
 * if it does not fit (out[0].n_active still reports the size). */
lodge_status lodge_select_lod(lodge_ctx* ctx, int32_t scene_id, lodge_mode mode,
                              const lodge_camera* cams, int32_t n_cams, lodge_selection* out,
                              uint32_t* d_gids, int64_t gids_capacity, void* stream);

/* Greedy choice of the depth thresholds d_1 .. d_{L-1} (Sec. 3, "Selecting
 * depth thresholds"): the cost of a threshold set is the number of (tile,
 * Gaussian) keys that LOD rendering (Eq. 2 at each camera centre) produces,
 * summed over the n_views views (host array) -- the mean number of Gaussians
 * per 16x16 tile up to a constant factor.  d_1 is chosen first with only
 * levels 0 and 1 in use, then each next d_l with the earlier ones fixed and
 * levels above l unused, among the candidates (host, n_candidates <= 1024
 * positive distances in metres, strictly ascending) larger than d_{l-1};
 * ties go to the smaller candidate.  d_out (host, num_levels - 1 doubles)
 * receives the chosen thresholds, +inf for a level for which no candidate
 * was left.  keys_out (host, optional, (num_levels - 1) x n_candidates) receives
 * the key total of every candidate at every step, -1 where a candidate was
 * not eligible.  The scene's own thresholds are not changed.  Synchronous on
 * stream.  Errors: LODGE_E_INVALID for bad arguments or cameras. */
lodge_status lodge_select_thresholds(lodge_ctx* ctx, int32_t scene_id, const lodge_camera* views,
                                     int32_t n_views, const double* candidates,
                                     int32_t n_candidates, double* d_out, int64_t* keys_out,
                                     void* stream);

/* Eq. 5 (supplementary "Selecting chunk centers"): the number of chunk
 * clusters for n camera positions (host, 3n doubles, metres) and first depth
 * threshold d1 > 0: ceil((4 / d1) max_i |c_i - c_mean|), clamped to [1, n].
 * *k_out (host) receives it.  Host-only; needs no device. */
lodge_status lodge_num_clusters(const double* positions, int32_t n, double d1, int32_t* k_out);

/* Chunk centres by K-means on camera positions (supplementary "Selecting
 * chunk centers"), Lloyd's iteration in FP64: start from the k positions
 * positions[init[j]] (host, k distinct indices, 1 <= k <= n); then repeat
 * (a) assign each position to its nearest centre (squared Euclidean
 * distance, ties to the lower centre index) and stop if no assignment
 * changed, (b) move each centre to the mean of its positions (summed in
 * index order; a centre without positions stays), at most max_iter times.
 * centers_out (host, 3k) receives the centres, assign_out (host, n,
 * optional) each position's nearest returned centre, iters_out (optional)
 * the number of update steps done.  Host-only; needs no device. */
lodge_status lodge_kmeans_centers(const double* positions, int32_t n, int32_t k,
                                  const int32_t* init, int32_t max_iter, double* centers_out,
                                  int32_t* assign_out, int32_t* iters_out);

/* ---------------------------------------------------------------- render */

/* Size of the bins whose key lists the renders of this context sort and
 * composite from: squares of 2^log2_tiles x 2^log2_tiles 16x16 tiles
 * (0..3), or -1 (the context's start value) to choose per frame: per-tile
 * lists for active sets of 2^21 Gaussians or more, bins of 2x2 tiles below.
 * A Gaussian is keyed once per bin its tile rect touches (Sec. 3,
 * "Preliminaries: 3DGS", assigns it to every tile it overlaps); compositing
 * walks the bin's list for each of the bin's tiles and skips the Gaussians
 * that cannot reach a pixel of the tile, so images do not depend on the
 * setting, only the number of keys sorted and records walked do.  Frames
 * saved for the adjoint (save_for_backward) and the importance walk always
 * use per-tile lists (log2_tiles = 0).  Errors: LODGE_E_INVALID for a NULL
 * ctx or log2_tiles outside -1..3. */
lodge_status lodge_set_bin_size(lodge_ctx* ctx, int32_t log2_tiles);

/* Render n_cams cameras of one scene in `mode`.  d_rgb (device,
 * caller-owned) receives n_cams images back to back, each H x W x 3 of its
 * camera.  stats (host, optional) receives n_cams frame counters.  With
 * save_for_backward != 0 (n_cams must be 1) the frame's intermediate state
 * is kept under *handle_out until lodge_release.  Returns when every frame
 * has been enqueued and its counters read.  Frames of a resident scene
 * take turns on several streams (six; two for LODGE_FULL) and, once their
 * stream has seen a frame, run without a mid-frame synchronisation
 * (scratch sized by capacities, counts read at the end of the call); a
 * frame whose keys outgrow that capacity is rendered again
 * (lodge_profile.redone), so images and counters are those of rendering
 * each camera alone. */
lodge_status lodge_render(lodge_ctx* ctx, int32_t scene_id, lodge_mode mode,
                          const lodge_camera* cams, int32_t n_cams, float* d_rgb, void* stream,
                          int32_t save_for_backward, int64_t* handle_out,
                          lodge_frame_stats* stats);

/* Render n frames (1..64) of any scenes, modes and sizes as one batch:
 * each frame runs its stages up to the tile ranges on its own scratch, then
 * a single launch composites the tiles of all frames (the step of the
 * serving loop).  scene_ids, modes, cams: host arrays of n; d_rgb: host
 * array of n DEVICE image pointers (H x W x 3 each, caller-owned).  stats
 * and statuses (host, optional) receive per-frame counters and outcomes.
 * Images equal lodge_render's.  Synchronous on stream.  Returns
 * LODGE_E_INVALID if any frame failed (its status says why). */
lodge_status lodge_render_batch(lodge_ctx* ctx, int32_t n, const int32_t* scene_ids,
                                const int32_t* modes, const lodge_camera* cams, float* const* d_rgb,
                                void* stream, lodge_frame_stats* stats, int32_t* statuses);

/* Same as lodge_render but cameras and the image live in HOST memory: the
 * call copies the images back (device -> host) before returning, each one
 * as soon as its frame is done, so that the copies of earlier frames overlap
 * the rendering of later ones (page-locked h_rgb lets them run
 * asynchronously).  h_rgb: n_cams images, H x W x 3 float32 each.  Intended
 * for callers that do not manage device memory; device scratch is owned by
 * the context. */
lodge_status lodge_render_host(lodge_ctx* ctx, int32_t scene_id, lodge_mode mode,
                               const lodge_camera* cams, int32_t n_cams, float* h_rgb,
                               void* stream, lodge_frame_stats* stats);

/* LOD rendering (Eq. 2 at each camera centre) with thresholds given per
 * camera instead of the scene's: d_inner (host) holds n_cams rows of
 * num_levels - 1 non-negative, ascending distances (+inf allowed).  This is
 * the rendering of the LOD build loop (supplementary "LOD structure
 * optimization steps"), which draws d_l from U(0.7 d_l, 1.3 d_l) each step;
 * the caller draws the values.  Images and stats as lodge_render.
 * Resident scenes only.  Synchronous on stream. */
lodge_status lodge_render_lod(lodge_ctx* ctx, int32_t scene_id, const lodge_camera* cams,
                              int32_t n_cams, const double* d_inner, float* d_rgb, void* stream,
                              lodge_frame_stats* stats);

/* Importance score (Sec. 3 "Importance pruning" and "Visibility filtering",
 * which follow RadSplat): render each of the n_cams cameras (host array) and
 * raise d_score[gid] (DEVICE, n_total floats, caller-initialised, normally
 * to 0) to the largest blending weight T * alpha that the Gaussian receives
 * at any pixel where it is composited (Eq. 1, same decisions as
 * lodge_render).  Calls accumulate: the score over several calls is the
 * maximum over all their views.  chunk < 0: the mode's active set per camera;
 * chunk >= 0: chunk `chunk`'s own active set for every camera, with no
 * blending (resident scenes only; the views of a chunk's visibility
 * filtering).  Synchronous on stream.  Errors: LODGE_E_INVALID,
 * LODGE_E_NOT_RESIDENT. */
lodge_status lodge_importance(lodge_ctx* ctx, int32_t scene_id, lodge_mode mode, int32_t chunk,
                              const lodge_camera* cams, int32_t n_cams, float* d_score,
                              void* stream);

/* Visibility filtering of one chunk (Sec. 3): remove from chunk `chunk`'s
 * active set every Gaussian whose score in d_score (DEVICE, n_total floats,
 * from lodge_importance) is below threshold; the set keeps gid order.
 * *n_kept (host, optional) receives the new size.  Later CHUNK and
 * CHUNK_BLEND renders use the filtered set.  Resident scenes only; must not
 * run while frames of the scene are being rendered.  Synchronous.  Errors:
 * LODGE_E_INVALID, LODGE_E_NOT_RESIDENT, LODGE_E_BUDGET. */
lodge_status lodge_filter_chunk(lodge_ctx* ctx, int32_t scene_id, int32_t chunk,
                                const float* d_score, float threshold, int64_t* n_kept,
                                void* stream);

/* Render Gaussians given as raw DEVICE parameters (the fine-tuning path of
 * Sec. 3 "Building LOD", supplementary "LOD structure optimization steps":
 * only the trained level's parameters change between steps).  Activation is
 * done on the device in FP32.  Layout as lodge_level_desc.  d_rgb: H x W x 3. */
lodge_status lodge_render_params(lodge_ctx* ctx, int64_t n, const float* d_means,
                                 const float* d_log_scales, const float* d_quats,
                                 const float* d_opacity_logits, const float* d_sh,
                                 int32_t sh_degree, float filter_var, const lodge_camera* cam,
                                 float* d_rgb, void* stream, int32_t save_for_backward,
                                 int64_t* handle_out, lodge_frame_stats* stats);

/* LOD rendering of levels given as raw DEVICE parameters (supplementary
 * "LOD structure optimization steps": level l is built by fine-tuning G_l
 * with LOD rendering of the levels up to l, the threshold d_l drawn from
 * U(0.7 d_l, 1.3 d_l) per step; Sec. 3 "Building LOD").
 *   num_levels: 1 .. 8, finest first; level_n (host, num_levels): sizes.
 *   d_means .. d_sh (host arrays of num_levels DEVICE pointers, caller-owned,
 *     layouts as lodge_level_desc; SH 16-byte aligned); activated on the
 *     device in FP32 into one gid-ordered store (gid = index into the levels
 *     concatenated finest first).
 *   filter_var (host, num_levels): the Eq. 3 variance of each level.
 *   d_inner (host, num_levels - 1, ascending, metres): this frame's
 *     thresholds d_1 .. d_{L-1}; Eq. 2 at the camera centre selects level
 *     l's band [d_l, d_{l+1}).
 *   d_rgb: H x W x 3 (device).
 *   d_score (device, total Gaussians, optional): when given, the frame also
 *     raises the importance scores (as lodge_importance) and cannot be saved.
 *   save_for_backward: keep the frame for lodge_render_backward, which then
 *     gives gradients of level train_level only, into arrays of that level's
 *     size (the other levels are fixed, as in the build).
 * Synchronous on stream.  Errors: LODGE_E_INVALID (sizes, thresholds,
 * pointers, train_level), LODGE_E_OOM, LODGE_E_CUDA. */
lodge_status lodge_render_params_lod(lodge_ctx* ctx, int32_t num_levels, const int64_t* level_n,
                                     const float* const* d_means, const float* const* d_log_scales,
                                     const float* const* d_quats, const float* const* d_opacity_logits,
                                     const float* const* d_sh, int32_t sh_degree, const float* filter_var,
                                     const double* d_inner, const lodge_camera* cam, float* d_rgb,
                                     float* d_score, int32_t train_level, void* stream,
                                     int32_t save_for_backward, int64_t* handle_out,
                                     lodge_frame_stats* stats);

/* Gradients of a saved lodge_render_params frame.  d_dL_drgb: H x W x 3
 * (device).  Gradients (device, caller-owned, same layouts as the
 * parameters) are ACCUMULATED (+=) so several views can be summed; zero them
 * first.  Any gradient pointer may be NULL to skip that group. */
lodge_status lodge_render_backward(lodge_ctx* ctx, int64_t handle, const float* d_dL_drgb,
                                   float* d_g_means, float* d_g_log_scales, float* d_g_quats,
                                   float* d_g_opacity_logits, float* d_g_sh, void* stream);

/* Free a saved frame. */
lodge_status lodge_release(lodge_ctx* ctx, int64_t handle);

/* ---------------------------------------------------------------- inspection */

/* Sorted tile keys of a saved frame: key = tile_id << 32 | bits(FP32 depth),
 * tile_id = ty * tiles_x + tx, in the order they are composited, and the gid
 * of each key.  Device outputs with capacity cap; *n_keys (host) receives
 * the count; LODGE_E_OVERFLOW if it exceeds cap. */
lodge_status lodge_debug_keys(lodge_ctx* ctx, int64_t handle, uint64_t* d_keys, uint32_t* d_gids,
                              int64_t cap, int64_t* n_keys, void* stream);

/* Projection records of a saved frame, one per visible Gaussian in gid
 * order: d_gid, d_depth (FP32 key depth), d_rect (tx0, ty0, tx1, ty1 int32),
 * d_mean2 (2 floats), d_conic (3 floats: inverse 2D covariance xx, xy, yy),
 * d_opacity (final opacity), d_rgb (3 floats).  Any output may be NULL.
 * *n_visible (host) receives the count; LODGE_E_OVERFLOW if > cap. */
lodge_status lodge_debug_records(lodge_ctx* ctx, int64_t handle, uint32_t* d_gid, float* d_depth,
                                 int32_t* d_rect, float* d_mean2, float* d_conic,
                                 float* d_opacity, float* d_rgb, int64_t cap,
                                 int64_t* n_visible, void* stream);

/* Sort n (key, value) pairs of 32-bit unsigned integers by the key bits
 * [0, key_bits), stably, with the library's onesweep LSD radix sort.
 * d_keys/d_vals are sorted in place (device).  Exposed for testing the sort
 * (Sec. 3: Gaussians are sorted per tile by depth). */
lodge_status lodge_sort_pairs(lodge_ctx* ctx, uint32_t* d_keys, uint32_t* d_vals, int64_t n,
                              int32_t key_bits, void* stream);

/* Allocation-free variant of lodge_sort_pairs (the paper has no counterpart:
 * this is a convenience for callers that cannot allocate device memory, such
 * as an application that owns every device allocation itself, or a loop that
 * cannot afford an allocation's implicit synchronisation).  Same result as
 * lodge_sort_pairs: d_keys / d_vals (device, caller-owned, n pairs) are
 * sorted in place, stably, on key bits [0, key_bits).  No context is needed
 * and nothing is allocated: scratch is a fixed array in the library's device
 * memory, about 12.6 MB on every device that loads the library, kept until
 * the process exits.
 *   - n may be at most 1,048,576 (2^20); larger n returns LODGE_E_INVALID
 *     before any device work.
 *   - The first call on a device looks up the array's device address and
 *     caches it for the device; make that first call before capturing any
 *     stream.  The cached address is valid until cudaDeviceReset on that
 *     device; do not call this function after such a reset.
 *   - Every call on a device shares the array: calls whose device work
 *     overlaps (on different streams) race and give wrong results.  The call
 *     copies the status word to the host and synchronises `stream` before
 *     returning.
 *   - Errors: LODGE_E_INVALID (arguments), LODGE_E_CUDA, LODGE_E_TIMEOUT (a
 *     bounded device-side wait gave up), LODGE_E_OVERFLOW (any other error
 *     bit the sort's kernels set in the status word). */
lodge_status lodge_sort_pairs_noalloc(uint32_t* d_keys, uint32_t* d_vals, int64_t n,
                                      int32_t key_bits, void* stream);

/* Debug: the decoupled look-back that the library's scans (projection,
 * emission, sort passes) use to chain per-tile prefix sums, run alone over
 * n_tiles tiles of one warp each.  Tile i contributes i + 1; tile `missing`
 * (0 <= missing < n_tiles) never publishes its count, so its successors'
 * waits run out; missing < 0 lets every tile publish.  Every wait gives up
 * after spin_limit polls (1 .. 2^22; the library's own scans use 2^22),
 * records the timeout in a status word and counts the missing tile as 0, so
 * the kernel always ends.  h_prefix (host, n_tiles) receives each tile's
 * exclusive prefix (the tiles before `missing` get the exact sums).  The
 * call allocates its device words itself and synchronises `stream`.
 * Returns LODGE_E_TIMEOUT when a wait gave up (the context stays usable),
 * LODGE_E_INVALID for n_tiles outside 1 .. 1024 or a bad limit.  Exposed to
 * test the bounded waits that keep a stalled predecessor from hanging the
 * GPU (the paper has no counterpart). */
lodge_status lodge_debug_lookback(int32_t n_tiles, int32_t missing, uint32_t spin_limit,
                                  uint32_t* h_prefix, void* stream);

/* ---------------------------------------------------------------- serving */

/* One render request: scene, mode, camera and its arrival time in seconds
 * relative to the start of lodge_serve. */
typedef struct {
    int32_t scene;
    int32_t mode;          /* lodge_mode */
    lodge_camera cam;
    double arrival_s;
} lodge_request;

typedef struct {
    double start_s;        /* admitted: a slot picked it up */
    double finish_s;       /* image rendered (and copied to the host if asked) */
    int32_t status;        /* lodge_status of this request */
    int32_t slot;
    lodge_frame_stats stats;
    int32_t uploads;       /* chunk blocks gathered into HBM for this request */
    int32_t step_frames;   /* step mode: frames composited by the request's step */
} lodge_request_result;

typedef struct {
    int32_t slots;         /* requests in flight at once, 1..64 */
    int32_t realtime;      /* != 0: a request is not started before its arrival */
    float* h_images;       /* optional host buffer: the images back to back in
                              request order (H x W x 3 each) */
    double wait_limit_s;   /* how long a request may wait for HBM (0: 10 s) */
    int32_t batch;         /* 0: slot workers as above; B > 0: steps - each step
                              takes the requests that have arrived (at most B, in
                              arrival order), runs their stages up to the tile
                              ranges and composites all of them with one launch */
    int32_t pad_;
} lodge_serve_opts;

/* Serve n requests with continuous batching (the serving loop built around
 * the paper's renderer: chunk residency, sort buffers and images stay on the
 * device).  With opts->batch = 0, each slot is a worker with its own stream
 * and scratch; requests are admitted in arrival order as slots free up and
 * as their memory fits the HBM budget, and their work overlaps on the
 * device.  With opts->batch > 0, the loop runs in steps: every request that
 * has arrived when a step starts joins it (up to batch), and one launch
 * composites all of the step's frames; requests arriving meanwhile join the
 * next step, and a request whose memory does not fit waits for a later step
 * (up to wait_limit_s).  results[i] (host) receives request i's times, status
 * and frame counters (slot = its place in the step in batch mode); latency
 * = finish_s - arrival_s.  Returns LODGE_E_INVALID if any request failed
 * (its own status says why); the other requests still complete. */
lodge_status lodge_serve(lodge_ctx* ctx, const lodge_request* reqs, int32_t n,
                         const lodge_serve_opts* opts, lodge_request_result* results);

/* Residency counters of the context (streamed scenes). */
typedef struct {
    int64_t resident_blocks;
    int64_t block_hits, block_uploads, block_evictions;
    int64_t upload_bytes;       /* attribute bytes gathered into HBM */
    int64_t failed_uploads;
    int64_t hbm_used, hbm_budget;
} lodge_residency;

/* Copy the context's residency counters to *out (host).  Errors:
 * LODGE_E_INVALID for NULL arguments. */
lodge_status lodge_residency_stats(lodge_ctx* ctx, lodge_residency* out);

/* Fault injection for tests: the next n chunk uploads fail on the host side
 * (LODGE_E_CUDA for the requests that need them) without touching the
 * device. */
lodge_status lodge_inject_upload_failures(lodge_ctx* ctx, int32_t n);

/* ---------------------------------------------------------------- profiling */

/* Stages of a frame, in launch order. */
typedef enum {
    LODGE_STAGE_SELECT = 0,     /* K1 Eq. 2 selection (LOD mode) */
    LODGE_STAGE_UNION = 1,      /* K2 chunk-pair union (when the pair changes) */
    LODGE_STAGE_PROJECT = 2,    /* K3 projection + SH + compaction */
    LODGE_STAGE_DEPTH_SORT = 3, /* K5 onesweep sort by depth */
    LODGE_STAGE_EMIT = 4,       /* K4 bin emission */
    LODGE_STAGE_TILE_SORT = 5,  /* K5 onesweep sort by bin */
    LODGE_STAGE_RANGES = 6,     /* K6 bin ranges */
    LODGE_STAGE_BLEND = 7,      /* K7 compositing */
    LODGE_NUM_STAGES = 8
} lodge_stage;

/* Accumulated device time per stage, measured with CUDA events recorded on
 * the render stream around each stage (ms), the number of kernel launches per
 * stage, and the number of frames. */
typedef struct {
    double ms[LODGE_NUM_STAGES];
    int64_t launches[LODGE_NUM_STAGES];
    int64_t frames;
    int64_t keys;      /* sum of per-frame tile keys */
    int64_t visible;   /* sum of per-frame visible Gaussians */
    int64_t active;    /* sum of per-frame active Gaussians */
    int64_t packed_keys; /* bin keys of frames whose bin and record index fit
                          * one 32-bit word: sorted as single words, no values */
    int64_t bin_keys;    /* sum of per-frame keys emitted and sorted (one per
                          * record and bin; equals keys for per-tile bins) */
    int64_t bin_sort_passes; /* sum of per-frame passes of the bin sort */
    int64_t blend_pairs;      /* counting mode: (pixel, Gaussian) pairs the
                               * compositing evaluated (Eq. 1 alpha) */
    int64_t blend_pairs_used; /* counting mode: pairs composited (alpha >=
                               * 1/255 and the pixel not yet saturated) */
    int64_t redone;           /* frames of multi-camera calls rendered again
                               * because their bin keys outgrew the capacity
                               * sized from earlier frames */
    double host_ms;           /* host time lodge_render spent enqueuing its
                               * frames, up to the wait for their counts */
} lodge_profile;

/* Start (enable != 0, counters reset) or stop collecting the profile.
 * Launch counts are always collected; event timing only while enabled.
 * enable = 2 is the counting mode: single-frame compositing also counts its
 * (pixel, Gaussian) pairs (blend_pairs, blend_pairs_used) with a counting
 * variant of the kernel and every frame synchronises, so stage times taken
 * in this mode are not those of the plain kernels. */
lodge_status lodge_profile_enable(lodge_ctx* ctx, int enable);

/* Copy the accumulated profile to *out (host). */
lodge_status lodge_profile_read(lodge_ctx* ctx, lodge_profile* out);

#ifdef __cplusplus
}
#endif
#endif /* LODGE_H */
