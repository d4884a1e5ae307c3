/*
 * perch.h -- C ABI of libperch: PERCH 2.0 hypothesis scoring on one GB300 (sm_103a).
 *
 * The library scores object-pose hypotheses against an RGB-D observation the
 * way PERCH 2.0 does (Agarwal, Han, Likhachev, "PERCH 2.0: Fast and Accurate
 * GPU-based Perception via Search for Object Pose Estimation"):
 *   for each pose h the object mesh is rendered into an integer depth z-buffer
 *   (Sec. IV-A "Parallel Rendering"), the visible pixels are back-projected and
 *   down-sampled in image space (Sec. IV-A), pixels hidden behind the observed
 *   depth are removed as extraneous occluders (R_K \ C_K, Eq. 3), every
 *   remaining rendered point q is tested against the observed cloud I within
 *   radius delta (Eq. 2) and, optionally, by CIEDE2000 colour (Eq. 4), and the
 *   costs J_r (unexplained rendered points) and J_o (observed points of the
 *   admissible set V(O) not found as a nearest neighbour, Sec. IV-A "Parallel
 *   Cost Computation") are returned per hypothesis; perch_best takes the
 *   per-object argmin of J = J_o + J_r (Eq. 1, Sec. IV-A "Parallel Search").
 *
 * Conventions used by every call:
 *   - image W x H, pixel (u,v) has its centre at integer (u,v); intrinsics
 *     fx, fy, cx, cy map a camera point (X,Y,Z) to (fx X/Z + cx, fy Y/Z + cy);
 *   - depth is uint16 in 0.1 mm units, 0 = no return;
 *   - a pose is 12 float32, row-major 3x4 [R | t], object frame -> camera
 *     frame (x right, y down, z forward), metres;
 *   - a ROI is int32[4] = {u0, v0, u1, v1}, half-open, clipped to the image;
 *     NULL means the whole image;
 *   - costs are int32 pairs {J_o, J_r} per hypothesis.
 *
 * Error behaviour: every call returns a perch_status; nothing aborts or exits.
 * On failure the call has no effect on the caller's buffers beyond what the
 * message from perch_last_error() states; device-side failures are reported
 * as PERCH_E_CUDA.  There is no CPU fallback: a context cannot be created
 * without a CUDA device.
 *
 * Threading: a context may be used by one host thread at a time, with one
 * exception: while a served-form server runs on it (its own threads use the
 * context), other threads may load and release meshes and observations; every
 * other call on the context returns PERCH_E_BUSY until the server is stopped.
 *
 * Lifetime: releasing a mesh or an observation returns PERCH_E_BUSY, and
 * changes nothing, while anything may still read it -- a queued or running
 * served request, a batch graph that has not been destroyed, or an
 * asynchronous call (cuda_stream != NULL) whose stream has not yet passed it.
 */
#ifndef PERCH_H
#define PERCH_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PERCH_API __attribute__((visibility("default")))
#else
#define PERCH_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct perch_ctx perch_ctx;   /* opaque; owns all device memory it allocates */
typedef int32_t perch_status;

#define PERCH_OK          0
#define PERCH_E_INVALID  (-1)   /* bad argument (null pointer, size, id, range)          */
#define PERCH_E_NOMEM    (-2)   /* cudaMalloc or host allocation failed                   */
#define PERCH_E_BUDGET   (-3)   /* the allocation would exceed the context's HBM budget   */
#define PERCH_E_NOTFOUND (-4)   /* unknown scene, mesh or ticket id                       */
#define PERCH_E_CUDA     (-5)   /* a CUDA runtime call or kernel failed                   */
#define PERCH_E_TIMEOUT  (-6)   /* a bounded wait ran out                                 */
#define PERCH_E_BUSY     (-7)   /* resource in use (e.g. releasing a scene with work)     */

/* Scoring parameters, fixed per observation.
 *   delta_m          sensor resolution delta of Eq. 2, metres, 1e-4 <= delta_m <= 1.
 *   tau_c            CIEDE2000 threshold tau_c of Eq. 4 (the paper uses 12.5).
 *   color_check      0: Eq. 2 only; 1: Eq. 4 (distance and colour).
 *   stride           image-space down-sampling factor s >= 1 (Sec. IV-A): only
 *                    pixels with u % s == 0 and v % s == 0 enter I and R.
 *   occ_margin_units occluder margin m (0.1 mm): a rendered pixel of depth d is
 *                    an occluded one (in C_K, Eq. 3) iff the observed depth
 *                    d_obs > 0 and d_obs + m < d (and, when scoring by label,
 *                    the pixel's label differs from the object's, Sec. V-C).
 *                    -1 turns occluder marking off, which is the variant
 *                    PERCH 2.0-A of Sec. VI-A (rendered points are never
 *                    removed by the observed depth).
 *   z_near_m         triangles with a vertex nearer than this are culled.
 *   jo_mode          0: J_o as the J_o kernel of Sec. IV-A computes it -- an observed
 *                    point of V(O) is an inlier iff it is the nearest neighbour of a
 *                    rendered point it explains;
 *                    1: J_o as Eq. 3 writes it, OUTLIER(p | R \ C) with the test
 *                    applied from the observed side ("or vice-versa", Sec. IV-B):
 *                    an observed point p of V(O) is an inlier iff its nearest
 *                    rendered point q of R \ C (smallest squared distance, ties to
 *                    the lowest pixel index) lies within delta (Eq. 2) and, with
 *                    color_check on, the CIEDE2000 difference of q's and p's
 *                    colours is at most tau_c (Eq. 4).  Keeps a 64-bit key per
 *                    pixel of the admissible box in shared memory (row bands of
 *                    4 x mark_bits / 64 pixels); slower than mode 0. */
typedef struct perch_params {
    float delta_m;
    float tau_c;
    int32_t color_check;
    int32_t stride;
    int32_t occ_margin_units;
    float z_near_m;
    int32_t jo_mode;
} perch_params;

/* Fill *p with the defaults: delta 1 cm, tau_c 12.5, colour on, stride 1,
 * margin = delta (100 units), z_near 5 cm, jo_mode 0. */
PERCH_API perch_status perch_default_params(perch_params *p);

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the device
 * memory the context may hold (0 = no cap); every allocation is charged to it
 * and refused with PERCH_E_BUDGET when it would exceed it.  *out receives the
 * context (NULL on failure).  PERCH_E_CUDA if the device cannot be used. */
PERCH_API perch_status perch_create(perch_ctx **out, int32_t device, uint64_t hbm_budget_bytes);

/* Free every device allocation of the context and the context itself.  Waits
 * for the context's own work.  ctx may be NULL. */
PERCH_API perch_status perch_destroy(perch_ctx *ctx);

/* Message of the last failing call on this context ("" if none).  The string
 * is owned by the context and valid until its next call. */
PERCH_API const char *perch_last_error(const perch_ctx *ctx);

/* Bytes of device memory the context currently holds (charged to the budget). */
PERCH_API uint64_t perch_hbm_used(const perch_ctx *ctx);

/* Upload an object model (Sec. III-A: the 3-D models of the N objects).
 *   verts_xyz  host, n_verts*3 float32, object frame (z up, base on z = 0), metres
 *   rgb        host, n_verts*3 uint8 per-vertex colour
 *   tris       host, n_tris*3 int32 vertex indices (any winding; rendered two-sided)
 *   vol_radius_m, vol_height_m  the inscribed cylinder V(O) about the object's z axis,
 *              0 <= z <= height (notation table: admissible volume)
 * Limits: 1 <= n_verts, 1 <= n_tris <= 2^31-1, indices in [0, n_verts).
 * The data are copied; the caller keeps ownership.  *mesh_id receives the id. */
PERCH_API perch_status perch_load_mesh(perch_ctx *ctx, const float *verts_xyz, const uint8_t *rgb,
                             int32_t n_verts, const int32_t *tris, int32_t n_tris,
                             float vol_radius_m, float vol_height_m, int32_t *mesh_id);

/* Release a mesh and its device memory.  PERCH_E_BUSY while it is in use
 * (see "Lifetime" above); PERCH_E_NOTFOUND for an unknown id. */
PERCH_API perch_status perch_release_mesh(perch_ctx *ctx, int32_t mesh_id);

/* Upload an observation (Sec. III-B: the input cloud I from the RGB-D image and
 * the intrinsics) and build its device-resident data: the back-projected
 * cloud, per-pixel CIELAB, and a voxel hash over I with cells of edge
 * delta*(1+1/64) used for the radius search.
 *   depth   host, H*W uint16 (0.1 mm, 0 = invalid)
 *   rgb     host, H*W*3 uint8
 *   labels  host, H*W int32 segmentation labels, or NULL (Sec. V-C)
 *   W, H    1 <= W, H; W*H <= 466033 (keeps the fixed-point edge functions in int32)
 *   params  scoring parameters (copied)
 * The data are copied; *scene_id receives the id.  PERCH_E_INVALID when the
 * parameters are out of range or the image is too large for delta (the cell
 * coordinates of the cloud must stay below 1e5 cells). */
PERCH_API perch_status perch_set_observation(perch_ctx *ctx, const uint16_t *depth, const uint8_t *rgb,
                                   const int32_t *labels, int32_t W, int32_t H, float fx,
                                   float fy, float cx, float cy, const perch_params *params,
                                   int32_t *scene_id);

/* Release an observation and its device memory.  PERCH_E_BUSY while it is
 * in use (see "Lifetime" above); PERCH_E_NOTFOUND for an unknown id. */
PERCH_API perch_status perch_release_scene(perch_ctx *ctx, int32_t scene_id);

/* Score n pose hypotheses of one mesh against one observation.
 *   label  -1: V(O) is the mesh's cylinder at each pose (3-DoF, Sec. IV-A);
 *          >= 0: V(O) = {p in I : labels(p) == label, p inside the ROI} and
 *          occluders must carry a different label (6-DoF, Sec. V-C); needs labels.
 *   roi    rendering is restricted to this rectangle (NULL = whole image).
 *   poses  n*12 float32, costs n*2 int32 {J_o, J_r}.
 *   cuda_stream NULL: poses and costs are HOST pointers, the call copies them,
 *          runs and returns when costs are written.
 *          non-NULL (a cudaStream_t): poses and costs are DEVICE pointers; the
 *          work is enqueued on that stream and the call returns at once; both
 *          buffers must stay valid until the stream reaches that point.
 * n == 0 is a no-op.  Results do not depend on the order of the hypotheses. */
PERCH_API perch_status perch_score_hypotheses(perch_ctx *ctx, int32_t scene_id, int32_t mesh_id,
                                    int32_t label, const int32_t *roi, const float *poses,
                                    int64_t n, int32_t *costs, void *cuda_stream);

/* Argmin of J = J_o + J_r over n hypotheses (Eq. 1; "find the one
 * corresponding to the minimum cost for each object", Sec. IV-A), computed on
 * the device.  Ties go to the lowest id; ids = NULL uses the index.
 *   costs n*2 int32, ids n uint64 or NULL, n >= 1 (n < 2^31).
 *   best_index (int64) and best_cost (int32) receive the winner.
 * cuda_stream NULL: all pointers are host pointers; otherwise all are device
 * pointers and the result is written when the stream reaches the call.  The
 * context's argmin launches share one scratch buffer, so each is ordered on
 * the GPU after the context's previous one (an event), whatever the streams. */
PERCH_API perch_status perch_best(perch_ctx *ctx, const int32_t *costs, const uint64_t *ids, int64_t n,
                        int64_t *best_index, int32_t *best_cost, void *cuda_stream);

/* The argmin of perch_best as one 64-bit key, (J << 32) | id, for combining
 * searches sharded over several processes or GPUs: every shard computes its
 * key, and the minimum of the keys (one min-reduce, e.g. an all-reduce MIN) is
 * the key of the whole search's winner -- smallest J, ties to the lowest id,
 * exactly as one perch_best over all hypotheses decides (Sec. IV-A "Parallel
 * Search").  costs (n*2 int32), ids (n uint64, each below 2^32: the
 * hypotheses' ids in the whole search; NULL uses the index) and key (one
 * uint64) are DEVICE pointers on cuda_stream (required), ordered like
 * perch_best's launches.  1 <= n <= 2^31-1. */
PERCH_API perch_status perch_best_key(perch_ctx *ctx, const int32_t *costs, const uint64_t *ids, int64_t n,
                                      uint64_t *key, void *cuda_stream);

/* Wait for cuda_stream (NULL: the context's own stream) and report what the
 * kernels of earlier asynchronous calls found: the scoring kernels keep a
 * device error word (a hash table too small, a depth key out of range, a
 * bitset over capacity, a GICP source cloud over max_source_points) that an
 * asynchronous call cannot return.  PERCH_OK, or the status the synchronous
 * call would have returned (PERCH_E_CUDA or PERCH_E_INVALID, message in
 * perch_last_error); the word is cleared.  Synchronous calls check it too. */
PERCH_API perch_status perch_sync(perch_ctx *ctx, void *cuda_stream);

/* The same argmin as perch_best, for callers that cannot allocate device
 * memory -- for example a serving process that reserves all of its HBM at
 * start-up and may not call cudaMalloc afterwards (an allocation can
 * synchronise the device and stall every other stream), or a host framework
 * whose allocator owns the device memory.  Such callers cannot create a
 * perch_ctx, so this call takes none.  The paper has no counterpart; it is an
 * interface for these callers only.
 *   costs (n*2 int32), ids (n uint64 or NULL), best_index (int64) and
 *   best_cost (int32) are DEVICE pointers on the current CUDA device; the work
 *   is enqueued on cuda_stream (NULL: the default stream) and the result is
 *   written when the stream reaches it.
 *   1 <= n <= 2^31-1, otherwise PERCH_E_INVALID.  PERCH_E_INVALID too when a
 *   pointer is not device memory of the current device (host, pinned, managed
 *   or another GPU's memory: checked with cudaPointerGetAttributes before any
 *   launch); PERCH_E_CUDA if a CUDA call fails.
 * It allocates nothing.  Its scratch (the kernel's per-block partial results
 * and completion ticket, 24.8 KB for at most 1024 blocks) is a static device
 * array that every GPU loading the library holds until the process exits.
 * The first call on a device looks up that array's device address with
 * cudaGetSymbolAddress; make that first call before any stream capture.  All
 * calls share the one array: calls that overlap on the GPU (for instance on
 * two streams at once) race and must be ordered by the caller. */
PERCH_API perch_status perch_best_noalloc(const int32_t *costs, const uint64_t *ids, int64_t n,
                                          int64_t *best_index, int32_t *best_cost,
                                          void *cuda_stream);

/* Launch shape of the scoring kernel for this context: threads per block (128,
 * 256 or 512), the capacity of the shared-memory z-buffer in 32-bit words
 * (1024 <= zbuf_words <= 49152; a 32-bit key per pixel when the mesh has fewer
 * than 65536 triangles and the hypothesis lies within 6.5 m, else a 64-bit key
 * per pixel), and the capacity in bits of the bitset that marks nearest
 * neighbours inside the admissible box (1024 <= mark_bits <= 2^22, 0 = the
 * default 32768).  Pixel boxes larger than the z-buffer are processed in
 * tiles, admissible boxes larger than the bitset in row bands.  Results do not
 * depend on these choices; only speed and shared memory do.  A new context
 * uses 256 threads, 7064 words and 32768 bits (four blocks per SM).  The
 * autotuner of the batched form calls it.  PERCH_E_INVALID outside the
 * ranges. */
PERCH_API perch_status perch_set_launch_config(perch_ctx *ctx, int32_t threads, int32_t zbuf_words,
                                               int32_t mark_bits);

/* Tile bins of the rasteriser (Sec. IV-A "Parallel Rendering" renders every
 * triangle of a pose into its image; a pixel box larger than the shared-memory
 * z-buffer is rendered tile by tile).  bin_cap > 0: when a hypothesis's pixel
 * box needs 2 to 32 tiles, one pass first lists in each tile's bin the
 * triangles whose sample boxes meet it (at most bin_cap per tile), and each
 * tile is then rasterised from its bin alone instead of from the whole mesh;
 * a tile whose bin overflowed is rasterised from the whole mesh.  Plain
 * scoring (jo_mode 0) only.  The bins live in the vertex-cache slots (32 x
 * bin_cap x 4 bytes per resident block, charged to the budget).  Results do
 * not depend on it.  0 (the default) = no bins; otherwise 64 <= bin_cap <=
 * 65536, else PERCH_E_INVALID.  The autotuner sets it. */
PERCH_API perch_status perch_set_raster_bins(perch_ctx *ctx, int32_t bin_cap);

/* ---- batched form ----------------------------------------------------------
 * Hypotheses of many (scene, mesh) searches scored by ONE call: each item gets
 * a persistent launch of the whole resident grid with its scene and mesh in
 * the kernel parameters, and the launches are dealt round-robin over four
 * side streams, so the blocks of item j+1 start on the SMs that item j's
 * blocks leave at its tail -- searches of very different sizes (objects,
 * ROIs, hypothesis counts) share the GPU without a per-search tail.  Each
 * item is what perch_score_hypotheses takes (Sec. IV-A "Parallel Search":
 * every object of every scene is searched independently). */
typedef struct perch_work_item {
    int32_t scene_id;
    int32_t mesh_id;
    int32_t label;            /* as in perch_score_hypotheses */
    int32_t roi[4];           /* {u0,v0,u1,v1}; u1 <= u0 or v1 <= v0 means the whole image */
    int64_t pose_offset;      /* index of the item's first hypothesis in the batch arrays */
    int64_t n;                /* hypotheses of the item (>= 0) */
} perch_work_item;

/* Score all items of a batch.  poses holds 12 floats and costs 2 int32 per
 * hypothesis; item i uses entries [pose_offset, pose_offset + n).  Items may
 * not overlap.  cuda_stream NULL: HOST pointers, synchronous; otherwise DEVICE
 * pointers enqueued on that stream.  items is a host array, copied by the call.
 * Each item must hold fewer than 2^32 hypotheses. */
PERCH_API perch_status perch_score_batch(perch_ctx *ctx, const perch_work_item *items, int32_t n_items,
                                         const float *poses, int32_t *costs, void *cuda_stream);

/* A batch built once as a CUDA graph and replayed: one counter-reset node and
 * one persistent scoring kernel node per item with the whole resident grid,
 * node j depending on node j - 4 (the side-stream round robin of
 * perch_score_batch as a graph), so a single graph launch runs every search
 * (items read their scene and mesh from the kernel parameters).  The item list, the
 * device pose/cost arrays and the launch shape are fixed at creation; the
 * caller refills the pose array between replays.  The graph owns its scratch,
 * so replays of one graph must be ordered (one stream), while different graphs
 * and the context may run concurrently.  poses/costs are DEVICE pointers. */
typedef struct perch_batch_graph perch_batch_graph;
PERCH_API perch_status perch_batch_graph_create(perch_ctx *ctx, const perch_work_item *items,
                                                int32_t n_items, const float *poses,
                                                int32_t *costs, perch_batch_graph **out);
PERCH_API perch_status perch_batch_graph_launch(perch_batch_graph *g, void *cuda_stream);
PERCH_API perch_status perch_batch_graph_destroy(perch_batch_graph *g);

/* Autotuner: time the candidate launch shapes (threads per block x z-buffer
 * words x tile-bin capacity, the bins tried with the 2048- and 4096-word
 * z-buffers only) on a sample of this batch -- every 8th item in order of
 * size, whole; batches of fewer than 16 items whole (DEVICE poses/costs; the
 * sampled items' costs are overwritten) --, keep the fastest as the
 * context's launch configuration and remember it for batches of the same
 * class (largest ROI area and triangle count, each rounded to a power of
 * two); a later call for a known class returns the remembered shape without
 * timing.  *threads, *zbuf_words and *bin_cap (may be NULL) receive the
 * choice. */
PERCH_API perch_status perch_autotune(perch_ctx *ctx, const perch_work_item *items, int32_t n_items,
                                      const float *poses, int32_t *costs, int32_t *threads,
                                      int32_t *zbuf_words, int32_t *bin_cap);

/* ---- served form -----------------------------------------------------------
 * A continuous-batching server on a context: requests (one search each: a
 * scene, a mesh and its pose hypotheses) are queued as they arrive; a
 * scheduler thread packs the queued requests into launches of the batched
 * scorer whenever one of `slots` launch slots is free, so requests that
 * arrive while others are on the GPU join the next launch and launches overlap
 * on the device (each slot has its own scratch and stream).  Within a slot the
 * requests run smallest first and each one completes (its costs copied back,
 * its ticket done) as soon as its own scoring is finished.  Scenes and meshes
 * stay resident in the context; each slot's device staging for
 * max_batch_hypotheses poses and costs is allocated at start-up and charged
 * to the context's HBM budget, so admission is bounded by that budget.
 * While a server runs, other threads may load and release meshes and
 * observations (a release that a queued or running request still needs is
 * refused with PERCH_E_BUSY); every other call on the context returns
 * PERCH_E_BUSY until perch_server_stop. */
typedef struct perch_server perch_server;

typedef struct perch_server_config {
    int32_t slots;                 /* launches in flight, >= 1 (2 is typical) */
    int64_t max_batch_hypotheses;  /* hypotheses per launch; a larger request is refused */
    int32_t max_wait_us;           /* a free slot waits at most this long for more requests
                                      when fewer than max_batch_hypotheses are queued (0: none) */
} perch_server_config;

typedef struct perch_request {
    int32_t scene_id;
    int32_t mesh_id;
    int32_t label;                 /* as in perch_score_hypotheses */
    int32_t roi[4];                /* u1 <= u0 or v1 <= v0: the whole image */
    const float *poses;            /* HOST, n*12; copied by perch_submit */
    int64_t n;                     /* >= 1 */
    int32_t *costs;                /* HOST, n*2; written before the ticket completes and
                                      must stay valid until then */
} perch_request;

/* Start a server.  PERCH_E_BUDGET when the slots' staging does not fit the budget. */
PERCH_API perch_status perch_server_start(perch_ctx *ctx, const perch_server_config *cfg,
                                          perch_server **out);
/* Queue a request; *ticket identifies it.  PERCH_E_BUDGET if n exceeds
 * max_batch_hypotheses, PERCH_E_NOTFOUND for unknown ids, PERCH_E_INVALID for
 * bad arguments, PERCH_E_BUSY once the server is stopping. */
PERCH_API perch_status perch_submit(perch_server *srv, const perch_request *req, uint64_t *ticket);
/* PERCH_OK if the request completed, PERCH_E_BUSY if still queued or running,
 * the request's error otherwise (PERCH_E_NOTFOUND for an unknown ticket). */
PERCH_API perch_status perch_poll(perch_server *srv, uint64_t ticket);
/* Wait for a ticket at most timeout_us microseconds (< 0: no limit);
 * PERCH_E_TIMEOUT when the limit runs out. */
PERCH_API perch_status perch_wait(perch_server *srv, uint64_t ticket, int64_t timeout_us);
/* Steady-clock times (ns) of submission and completion of a finished ticket. */
PERCH_API perch_status perch_ticket_times(perch_server *srv, uint64_t ticket, int64_t *submit_ns,
                                          int64_t *done_ns);
/* Forget a finished ticket (its status and times).  The server keeps every
 * ticket until it is released or the server is stopped, so a long-running
 * caller releases each one once it has read it.  PERCH_E_BUSY while the
 * request is queued or running, PERCH_E_NOTFOUND for an unknown ticket. */
PERCH_API perch_status perch_ticket_release(perch_server *srv, uint64_t ticket);
/* Number of tickets the server holds (queued, running and finished but not
 * yet released). */
PERCH_API perch_status perch_server_tickets(perch_server *srv, int64_t *held);
/* Finish every queued request, stop the threads and free the server. */
PERCH_API perch_status perch_server_stop(perch_server *srv);

/* ---- 6-DoF pose proposals (Sec. V-B, Eq. 5 and Eq. 6) ------------------------
 * The hypothesis set H(O) = H_r x H_t of one object, generated on the device:
 *   H_r: M viewpoints v_i on the unit sphere -- a Fibonacci lattice
 *        (y_i = 1 - (2i+1)/M, azimuth i times the golden angle), the closest
 *        thing to M equidistant points -- times N in-plane angles
 *        theta_k = 2 pi k / N.  v_i is the direction from the object to the
 *        camera in the object frame; R_view(v_i) turns it onto the camera's
 *        -z axis (camera right = forward x object z, or x object y when
 *        forward is parallel to z), and R = Rz(theta_k) R_view(v_i) rotates
 *        about the optical axis.
 *   H_t: the centre (uc, vc) of the object's 2-D box back-projected at K
 *        depths z_j evenly spaced from z_min to z_max (K = 1: their mean),
 *        z_min / z_max = the nearest / farthest observed depth among pixels of
 *        the box whose label is `label`; t = c_j - R m, c_j the back-projected
 *        centre and m the centre of the mesh's bounding box.
 *   poses receives M*N*K poses (12 float32 each), ordered ((i N + k) K + j).
 *   bbox = {u0, v0, u1, v1} (half-open, clipped to the image); needs labels.
 *   z_range (int32[2], may be NULL) receives z_min, z_max in 0.1 mm units
 *   (both 0 when no pixel of the box carries the label: the poses then sit at
 *   depth 0 and every triangle is culled).
 * cuda_stream NULL: poses and z_range are HOST pointers, synchronous;
 * otherwise DEVICE pointers enqueued on that stream.
 * Limits: 1 <= M, N, K and M*N*K <= 2^26. */
PERCH_API perch_status perch_pose_proposals(perch_ctx *ctx, int32_t scene_id, int32_t mesh_id,
                                            int32_t label, const int32_t *bbox, int32_t M,
                                            int32_t N, int32_t K, float *poses, int32_t *z_range,
                                            void *cuda_stream);

/* ---- M2M GICP refinement (Sec. IV-A "Parallel M2M GICP"; Sec. III-A) ------------
 * Each hypothesis' pose is adjusted by generalised ICP before it is scored
 * (rendered again) with perch_score_hypotheses:
 *   source  = the hypothesis' rendered cloud R \ C at the input pose (visible,
 *             not occluded, on the scene's stride lattice, inside the ROI),
 *             each point with the camera-frame normal of its mesh triangle;
 *   target  = the observed cloud I of the scene, each point with the normal of
 *             the cross product of the depth image's central differences
 *             (zero at the border, next to a pixel without depth, or where a
 *             neighbour's depth differs by more than normal_max_jump_units);
 *   model   = every point a Gaussian flattened along its normal,
 *             C(n) = I - (1 - epsilon) n n^T (zero normal: C = I);
 *   step    = Gauss-Newton on sum r^T (C_b + R C_a R^T)^-1 r, r = b - (R a + t),
 *             b the nearest observed point within the scene's delta (the
 *             correspondence radius: set up a separate observation with the
 *             radius wanted), the increment linearised as (I + [w]x) p + v;
 *             the rotation update is the quaternion (1, w/2) normalised.
 * The per-correspondence terms are binary32, rounded to multiples of 2^-24 and
 * summed exactly in 64-bit integers; the 6x6 system is solved by Cholesky in
 * binary64.  So the result does not depend on the order of the sums: it is
 * bit-identical from run to run and to a sequential evaluation of the same
 * definitions.  A hypothesis stops after max_iterations updates, after a step
 * below both stop thresholds (that step is applied), with fewer than
 * min_correspondences matches, or when the system is not positive definite.
 * poses_out (n*12) receives R_inc R_0 | R_inc t_0 + t_inc rounded to binary32;
 * info (n*2 int32, may be NULL) the updates applied and the matches of the
 * last iteration evaluated, or (-1, source points) for a hypothesis whose
 * source cloud exceeded max_source_points (its pose is returned unchanged and
 * the call reports PERCH_E_INVALID when it synchronises).
 * cuda_stream NULL: poses, poses_out and info are HOST pointers, synchronous;
 * otherwise DEVICE pointers enqueued on that stream (no host synchronisation).
 * poses and poses_out may be the same array. */
typedef struct {
    int32_t max_iterations;          /* default 10; 0 returns the poses unchanged   */
    float epsilon;                   /* default 1e-3, in (0, 1)                     */
    int32_t normal_max_jump_units;   /* default 200 (2 cm), >= 0                     */
    int32_t min_correspondences;     /* default 6, >= 1                              */
    float stop_rotation_rad;         /* default 1e-5                                 */
    float stop_translation_m;        /* default 1e-5                                 */
    int32_t max_source_points;       /* per hypothesis; 0 = min(65536, ROI lattice)  */
} perch_gicp_params;

PERCH_API perch_status perch_default_gicp_params(perch_gicp_params *p);
PERCH_API perch_status perch_refine_hypotheses(perch_ctx *ctx, int32_t scene_id, int32_t mesh_id,
                                               int32_t label, const int32_t *roi, const float *poses,
                                               int64_t n, const perch_gicp_params *params,
                                               float *poses_out, int32_t *info, void *cuda_stream);

/* ---- Monotone Scene Generation tree search (Sec. III, Fig. 2; variant 2.0-B) -----
 * The K object instances are placed one per tree level; a state is the set
 * placed so far, kept on the device as its composed depth image (stride
 * lattice), the observed pixels its rendered points explain, and the observed
 * pixels inside its admissible volumes.  Adding object j at candidate pose h
 * to a state is an edge, scored on the GPU for every remaining object and
 * pose of every state of the level at once:
 *   refused  if j would cover a placed object: a lattice pixel where j
 *            renders at depth d, the state at s > 0 and d + m < s
 *            (m = occ_margin_units, or 0 when occluder marking is off);
 *   dJ_r     = j's visible rendered points (not behind the state, not behind
 *              the observed depth) that are unexplained (Eq. 2, Eq. 4);
 *   dJ_o     = observed points in V(j) not counted by an earlier object and
 *              explained neither by the state nor by j (Eq. 1).
 * The search keeps, level by level, the beam_width cheapest children ordered
 * by (path cost, parent rank, object, pose index) and returns the cheapest
 * goal: order[l] = the object placed at level l, pose_index[l] its pose
 * (index into that object's poses), level_cost[l] = the path cost after
 * level l.  A beam at least as wide as every level is an exhaustive search.
 * edges_scored (may be NULL) receives the number of edges evaluated.
 * Poses are HOST pointers; the call is synchronous.  Needs jo_mode 0.
 * Status PERCH_E_NOTFOUND when every path is refused.  Limits: 1 <= K <= 64,
 * 1 <= beam_width <= 4096. */
typedef struct {
    int32_t mesh_id;
    int32_t label;                   /* -1: cylinder V; >= 0: labels == label */
    int32_t roi[4];                  /* u0, v0, u1, v1; an empty box = whole image */
    const float *poses;              /* HOST, n*12 */
    int32_t n;
} perch_tree_object;

PERCH_API perch_status perch_tree_search(perch_ctx *ctx, int32_t scene_id, const perch_tree_object *objects,
                                         int32_t K, int32_t beam_width, int32_t *order,
                                         int32_t *pose_index, int64_t *level_cost, int64_t *edges_scored);

/* ---- Pose accuracy (the measures of Sec. VI) ---------------------------------
 * perch_add_s: for each of n pose pairs, the mean over the mesh's vertices x
 * of || P x - T x || (symmetric 0: ADD) or of the distance from P x to the
 * closest T y over the vertices y (symmetric 1: ADD-S), in metres; vertex
 * transforms and distances in binary32, the mean in binary64.  poses and
 * poses_true are n*12 row-major 3x4, add receives n doubles.  cuda_stream
 * NULL: HOST pointers, synchronous; otherwise DEVICE pointers on that stream.
 * ADD-S costs n * V^2 distance evaluations (V vertices).
 * perch_add_s_auc (host only): the area under the accuracy curve
 * acc(t) = |{i : add_i < t}| / n for t in [0, max_threshold], divided by
 * max_threshold: the mean of max(0, 1 - add_i / max_threshold). */
PERCH_API perch_status perch_add_s(perch_ctx *ctx, int32_t mesh_id, const float *poses, const float *poses_true,
                                   int64_t n, int32_t symmetric, double *add, void *cuda_stream);
PERCH_API perch_status perch_add_s_auc(const double *add, int64_t n, double max_threshold, double *auc);

/* Measured shared-memory atomicMin throughput of the device (operations per
 * second over all SMs, random addresses in a 32 KB array per block), the
 * ceiling of the rasteriser's z-buffer updates.  A measurement helper with no
 * counterpart in the paper; about 50 ms of GPU time. */
PERCH_API perch_status perch_measure_smem_atomics(int32_t device, double *u32_per_s, double *u64_per_s);

/* Debug view of the rasteriser used by perch_score_hypotheses: the z-buffer of
 * one pose as 64-bit keys (depth << 32) | triangle id, 0xFFFFFFFFFFFFFFFF where
 * nothing is covered.  keys is a HOST buffer of W*H uint64 of the scene; the
 * call is synchronous. */
PERCH_API perch_status perch_debug_render_keys(perch_ctx *ctx, int32_t scene_id, int32_t mesh_id,
                                     const int32_t *roi, const float *pose, uint64_t *keys);

#ifdef __cplusplus
}
#endif

#endif /* PERCH_H */
