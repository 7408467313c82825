/*
 * linprim.h -- C ABI of the GB300 (sm_103a) LinPrim rasterizer.
 *
 * Differentiable tile rasterization of transparent, homogeneous octahedra and
 * tetrahedra as defined in "LinPrim: Linear Primitives for Differentiable
 * Volumetric Rendering" (arXiv 2501.16312):
 *
 *   render(primitives, cameras) -> images                 Sec. 3.2
 *   render_backward(dL/dimage)  -> dL/d{centre, vertices, opacity, SH}
 *                                                          Sec. 3.4, App.
 *                                                          "Gradient Computation"
 *
 * Every step of both calls runs in hand-written CUDA kernels on the device
 * the context was created for; there is no CPU path.
 *
 * Conventions shared by all calls
 * -------------------------------
 * - Pointers named "device" are CUDA device pointers owned by the caller; the
 *   library never frees them.  "host" pointers are read (or written) before
 *   the call returns.
 * - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *   enqueued asynchronously on it; outputs are valid once the stream has
 *   reached the call's work.
 * - Every call returns an lp_status; nothing throws across the ABI.  On an
 *   error, lp_last_error(ctx) holds a one-line description.
 * - A context is not thread-safe; use one per host thread.
 * - Floating point is IEEE binary32 throughout.
 */
#ifndef LINPRIM_H
#define LINPRIM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LP_OK = 0,
    LP_ERR_INVALID = 1,      /* a bad argument (null pointer, bad size, bad enum) */
    LP_ERR_CAPACITY = 2,     /* a captured launch overflowed reserved capacity */
    LP_ERR_CUDA = 3,         /* a CUDA runtime error; see lp_last_error */
    LP_ERR_TIMEOUT = 4,      /* a bounded device-side wait expired */
    LP_ERR_UNSUPPORTED = 5,  /* valid but not implemented (e.g. tile size) */
    LP_ERR_STATE = 6         /* call order violated (backward without forward) */
} lp_status;

/* Primitive kinds; the value is the number of vertices per primitive. */
enum { LP_TETRAHEDRON = 4, LP_OCTAHEDRON = 6 };

/* Largest number of cameras rendered by one call. */
#define LP_MAX_CAMERAS 32

/* Pinhole camera (Sec. 3.2 "Preprocessing": primitives are transformed into
 * the camera's coordinate system and projected).
 *   viewmat  world -> camera, 4x4 row-major, OpenCV axes (x right, y down,
 *            z forward); the last row is ignored.
 *   fx, fy   focal lengths in pixels; cx, cy principal point in pixels.
 *            Pixel (x, y) is sampled at its centre (x + 0.5, y + 0.5).
 *   width, height  image size in pixels (each >= 1).                       */
typedef struct {
    float viewmat[16];
    float fx, fy, cx, cy;
    int width, height;
} lp_camera;

/* A population of primitives, structure of arrays, all device pointers.
 * (Sec. 3.1: features are position, vertices, opacity and SH colour.)
 *   kind       LP_OCTAHEDRON or LP_TETRAHEDRON (V = 6 or 4 vertices).
 *   n          number of primitives (>= 0).
 *   sh_degree  0..3; K = (sh_degree + 1)^2 coefficients per channel.
 *   centre     float[n][3]   world-space centre (the linearisation point of
 *              the ray-space map and the depth-sort key; Sec. 3.2).
 *   verts      float[n][V][3] world-space vertices.  Octahedra: the order is
 *              (+a0, -a0, +a1, -a1, +a2, -a2) for three axes a_i through the
 *              centre; faces take one vertex of each pair (8 faces).
 *              Tetrahedra: any order; face k omits vertex k (4 faces).
 *   opacity    float[n]      alpha in [0, 1) (after the sigmoid).
 *   sh         float[n][K][3] SH coefficients in 3DGS order.
 * Preconditions (not checked): each primitive is convex and its centre lies
 * strictly inside it, as the paper's parameterisation guarantees (Sec. 3.1);
 * all values are finite.                                                    */
typedef struct {
    int kind;
    int n;
    int sh_degree;
    const float* centre;
    const float* verts;
    const float* opacity;
    const float* sh;
} lp_prims;

/* Launch / algorithm parameters (the autotuner's search space).
 *   tile          tile edge in pixels: 8, 16 (the paper's patch size, App.
 *                 "Rendering Performance", Table 7) or 32.  Smaller tiles
 *                 give longer tile lists but fewer list entries per pixel.
 *   batch         projected primitives staged in shared memory per round of
 *                 the blend: 32, 64 or 128.
 *   blocks_per_sm resident blend blocks per SM for the persistent grid;
 *                 0 = as many as fit (occupancy query), else 1..32.
 *   sort_mode     0: one stable radix sort of 64-bit (tile << 32 | depth)
 *                 keys; 1: stable sort of records by depth, then a stable
 *                 sort of the tile ids; 2: stable sort of the tile ids of
 *                 entries emitted in record order, then a stable sort of
 *                 each tile's run by depth (all three give the same order).
 *   pixels_per_thread  1, 2 or 4 horizontally adjacent pixels per blend
 *                 thread (tile^2 / pixels_per_thread threads per tile);
 *                 built pairs: tile 8 with 1 or 2, tile 16 with 1, 2 or 4,
 *                 tile 32 with 2 or 4.  The exact-span mode takes 2 pixels
 *                 per thread on 8x8 tiles and 4 otherwise.
 *   chain_split   0: the backward's chain to world space in one pass per
 *                 primitive; 1: in two passes, geometry then colour, each
 *                 holding fewer registers (ignored while densification
 *                 statistics are gathered, which need one pass).
 *   radix_bits    widest digit of the radix sort passes: 4, 6, 8 or 11 bits.
 *                 A sort of k key bits takes p = ceil(k / radix_bits)
 *                 passes of ceil(k / p) bits each (at least 4), each with a
 *                 histogram of 2^bits bins per 4096 keys.
 *   tile_order    0: the persistent blends take tiles in index order; 1:
 *                 longest tile list first (tiles bucketed by the binary
 *                 logarithm of their list length), so that no long tile
 *                 starts last.
 *   onesweep      0: each radix pass is a histogram, a scan of it and a
 *                 scatter; 1: one histogram of every digit place up front,
 *                 then one kernel per pass whose blocks find their digit
 *                 offsets by decoupled look-back (below 2^30 entries).
 * Every setting renders bit-identical images (a pixel's arithmetic does not
 * depend on the schedule); tile lists are identical for one tile edge and in
 * the paper's per-tile order at each.  chain_split and the blend schedule
 * change the order in which gradient terms are summed, so gradients can differ in
 * the last bits between settings.  A backward, depth pass or pair count uses
 * the tile edge, batch and pixels per thread of its forward.                */
typedef struct {
    int tile;
    int batch;
    int blocks_per_sm;
    int sort_mode;
    int pixels_per_thread;
    int chain_split;
    int radix_bits;
    int tile_order;
    int onesweep;
} lp_tuning;

/* Sizes of the last forward call (filled by lp_get_stats).                 */
typedef struct {
    long long records;    /* n_cams * n (primitive, view) pairs */
    long long entries;    /* tile-list length E (0 until read back) */
    long long tiles;      /* tiles over all cameras */
    long long pixels;     /* pixels over all cameras */
    int sort_passes;      /* radix passes of the last sort */
    int key_bits;         /* key bits sorted */
    int launches_fwd;     /* kernels the last forward launched */
    int launches_bwd;     /* kernels a backward launches */
} lp_stats;

/* Stages timed by lp_stage_times, in launch order. */
enum {
    LP_STAGE_PREPROCESS = 0,   /* A1: project, planes, density, colour, rectangle */
    LP_STAGE_SCAN_EMIT = 1,    /* A2: scan of tile counts, key emission */
    LP_STAGE_SORT = 2,         /* A3: radix sort of the tile list */
    LP_STAGE_RANGES = 3,       /* A4: per-tile ranges */
    LP_STAGE_BLEND_FWD = 4,    /* A5: front-to-back blend */
    LP_STAGE_BLEND_BWD = 5,    /* A6: back-to-front blend backward */
    LP_STAGE_CHAIN = 6,        /* A7: chain to world-space features */
    LP_NUM_STAGES = 7
};

typedef struct lp_ctx lp_ctx;

/* Create a context bound to CUDA device `device` (made current for every
 * later call on this context).  *out receives the context.                  */
lp_status lp_create(lp_ctx** out, int device);

/* Free the context and its device workspace.  NULL is ignored.             */
void lp_destroy(lp_ctx* ctx);

/* Set / read the tuning parameters (defaults: tile 16, batch 64,
 * blocks_per_sm 0, sort_mode 0, pixels_per_thread 4, chain_split 0,
 * radix_bits 8, tile_order 0, onesweep 0).  LP_ERR_INVALID
 * for a value outside the sets above, or a (tile, pixels_per_thread) pair
 * that is not built.                                                        */
lp_status lp_set_tuning(lp_ctx* ctx, const lp_tuning* t);
lp_status lp_get_tuning(lp_ctx* ctx, lp_tuning* t);

/* Exact spans (App. "Ray Space Approximation", the variant without the
 * approximation).  exact = 1: later forwards clip each pixel's true
 * perspective ray -- from the camera centre through the pixel centre --
 * against the primitive's camera-space faces; the span and the depth are
 * distances along that ray.  The tile rectangle is then the box of the
 * perspectively projected vertices, a primitive with a vertex at camera depth
 * <= 0.2 is not drawn, and the 2D filter is not applied.  exact = 0 (the
 * default) uses the EWA ray-space approximation.  A backward, depth pass or
 * pair count uses the mode of its forward.  The exact mode runs one fixed
 * schedule (32 records per batch, 4 pixels per thread) whatever the tuning. */
lp_status lp_set_exact(lp_ctx* ctx, int exact);
lp_status lp_get_exact(lp_ctx* ctx, int* exact);

/* Depth map of the last forward on this context (App. "Depth and Surface
 * Reconstruction"): for every pixel, the distance along the ray (ray-space
 * depth, world units) at which it enters the first primitive after which the
 * cumulative opacity exceeds 0.5; 0 where the opacity never exceeds 0.5.
 * depth: device, float, packed [cam][H][W] like one channel of the images,
 * caller-owned, overwritten.  Runs a front-to-back pass over the forward's
 * tile lists that stops each pixel at opacity 0.5; it leaves the forward's
 * state (and so a later backward) untouched.  Asynchronous on `stream`.
 * Errors: LP_ERR_STATE without a forward, LP_ERR_INVALID for NULL.         */
lp_status lp_render_depth(lp_ctx* ctx, float* depth, void* stream);

/* The 2D anti-aliasing filter (Sec. 3.3; the paper uses a size of 0.1 px,
 * App. "Experimental Setting").  kernel_px = 0 turns it off (the default).
 * When on, every vertex on a primitive's projected (ray-space) bounding box
 * moves outward parallel to the screen -- in x for the x-extremes, in y for
 * the y-extremes -- by kernel_px / 2 for an octahedron (its opposite vertices
 * mirror the move) and kernel_px for a tetrahedron; the face planes, spans
 * and the tile rectangle then come from the moved vertices, and the backward
 * treats the move as a constant.  Applies to later forward calls on the
 * context (a backward uses the setting of its forward).  Errors:
 * LP_ERR_INVALID unless 0 <= kernel_px <= 16 and finite.                     */
lp_status lp_set_filter_2d(lp_ctx* ctx, float kernel_px);
lp_status lp_get_filter_2d(lp_ctx* ctx, float* kernel_px);

/* Densification statistics (Sec. 3.4 "Adaptive Population Control", App.
 * "Experimental Setting"), gathered into caller-owned device arrays of at
 * least n primitives, indexed like lp_prims, by every later call on the
 * context until they are unset:
 *   px_max      unsigned[n]: each forward raises it to the largest side, in
 *               pixels, of the primitive's pixel rectangle (clipped to the
 *               image) over the forward's cameras;
 *   grad_sum    float[n]: each backward adds, for every camera in which the
 *               primitive has a non-empty pixel rectangle, the norm of the
 *               view-space position gradient -- the gradient of the loss
 *               w.r.t. a translation of the whole primitive (centre and
 *               vertices) parallel to that camera's image plane, in NDC units
 *               (x_ndc = 2 x_px / W - 1);
 *   grad_count  unsigned[n]: each backward adds the number of those cameras.
 * The caller zeroes the arrays; one thread updates each primitive, so no two
 * calls may run concurrently on them.  All three NULL turns gathering off (the
 * default).  Calls with more than n primitives fail with LP_ERR_INVALID.
 * Errors: LP_ERR_INVALID if only some pointers are NULL or n < 0.          */
lp_status lp_set_densify_stats(lp_ctx* ctx, float* grad_sum, unsigned int* grad_count,
                               unsigned int* px_max, long long n);

/* Pre-size the library-owned workspace.  Needed before a forward/backward
 * pair is captured into a CUDA graph: a captured call cannot read the
 * tile-list length back, so it uses this capacity and latches
 * LP_ERR_CAPACITY (returned by lp_sync_status) if E exceeds it.  Outside
 * capture the workspace grows on demand and this call is optional.
 *   max_records  >= n_cams * n;  max_entries >= E;
 *   max_pixels   >= total pixels; max_tiles >= total tiles.                 */
lp_status lp_reserve(lp_ctx* ctx, long long max_records, long long max_entries,
                     long long max_pixels, long long max_tiles);

/* Forward render of n_cams cameras in one batched launch sequence
 * (Sec. 3.2: preprocess, global sort + tiling, per-tile rasterization and
 * front-to-back compositing with the stop at cumulative opacity 0.999).
 *   prims   host struct with device arrays, see lp_prims.
 *   cams    host array of n_cams cameras (1 <= n_cams <= LP_MAX_CAMERAS).
 *   bg      host float[3] background colour.
 *   images  device float, packed per camera as [3][H][W] planes, cameras
 *           back to back in order (sum of 3*W*H floats); overwritten.
 * The context keeps the sorted tile lists and per-pixel state (8 bytes per
 * pixel) for the next lp_render_backward.  Outside stream capture the call
 * synchronises `stream` once, to read the tile-list length and size its
 * workspace.
 * Limits: at most 2^30 pixels and 2^30 tiles over all cameras, each camera at
 * most 65536 pixels on a side (LP_ERR_INVALID otherwise).  Tile-list offsets
 * are 32-bit: the list (one entry per primitive, camera and covered tile)
 * must stay below 2^32 - 1 entries, about 51 GB of keys and values.  The
 * length is summed in 64 bits; a longer list returns LP_ERR_CAPACITY before
 * anything is sized for it (under stream capture it renders nothing and
 * lp_sync_status returns LP_ERR_CAPACITY).                                   */
lp_status lp_render_forward(lp_ctx* ctx, const lp_prims* prims, const lp_camera* cams,
                            int n_cams, const float bg[3], float* images, void* stream);

/* Backward of the last lp_render_forward on this context (Sec. 3.4
 * "Rasterization Backpropagation" and "Preprocessing Backpropagation").
 * The primitive arrays and cameras of that forward must be unchanged.
 *   dL_dimages  device float, same layout as the forward's images.
 *   dcentre     device float[n][3]
 *   dverts      device float[n][V][3]
 *   dopacity    device float[n]
 *   dsh         device float[n][K][3]
 *   accumulate  0: outputs are overwritten; 1: gradients are added to them.
 * Gradients are summed over the cameras of the forward.  The density
 * normaliser d_min carries no gradient (App. "Experimental Setting").
 * Returns LP_ERR_STATE if no forward preceded it on this context.          */
lp_status lp_render_backward(lp_ctx* ctx, const float* dL_dimages, float* dcentre,
                             float* dverts, float* dopacity, float* dsh, int accumulate,
                             void* stream);

/* Synchronise `stream`, then return (and clear) any status latched on the
 * device by earlier calls (LP_ERR_CAPACITY, LP_ERR_TIMEOUT), or LP_OK.     */
lp_status lp_sync_status(lp_ctx* ctx, void* stream);

/* Bounds canaries (a debugging aid; the paper has no counterpart).
 * lp_set_debug_guard(ctx, 1): every workspace buffer the context allocates
 * from then on carries a zone of 4096 bytes after its capacity, filled with
 * the byte 0xA5; each such allocation also synchronises the device.  Buffers
 * allocated earlier carry no zone (create the context, enable guards, then
 * call lp_reserve or render).  lp_check_guards synchronises the device and
 * reads every zone back: *checked receives the number of guarded buffers and
 * *damaged the number of zone bytes that changed -- 0 unless some kernel
 * wrote past a buffer's capacity (lp_last_error then names the first such
 * buffer).  Host pointers; errors: LP_ERR_INVALID for NULL, LP_ERR_CUDA.    */
lp_status lp_set_debug_guard(lp_ctx* ctx, int enabled);
lp_status lp_check_guards(lp_ctx* ctx, long long* checked, long long* damaged);

/* Failure-path test hook (the paper has no counterpart).  The tile-list sort
 * runs its passes with a decoupled look-back: each block waits for the
 * blocks before it to publish their digit counts, every wait bounded to
 * about a second, after which the block latches LP_ERR_TIMEOUT (returned by
 * lp_sync_status) and writes nothing outside its buffers.  With block >= 0
 * and the onesweep tuning on, that block of the first pass of later
 * forwards on this context publishes nothing, so the blocks after it time
 * out; the rendered result is then invalid.  -1 (the default) turns it off.
 * LP_ERR_INVALID below -1.                                                  */
lp_status lp_debug_sort_stall(lp_ctx* ctx, int block);

/* Test hook for the tile-count scan (Sec. 3.2 "Global Sorting and Tiling":
 * a record's entries start at the exclusive prefix sum of the tile counts).
 * Runs the forward's scan on n device counts: offsets[i] (device, n words)
 * receives the 32-bit exclusive prefix sum, and *total (host) the sum, or
 * 0xFFFFFFFF when the sum reaches 2^32 - 1: the scan keeps its total in 64
 * bits, and a forward whose tile list would be that long returns
 * LP_ERR_CAPACITY (with a stream capture, lp_sync_status does) rather than
 * wrap its 32-bit offsets.  Synchronises the stream.  Returns
 * LP_ERR_CAPACITY on such a total, LP_ERR_INVALID for bad arguments or a
 * status still latched from an earlier call, else LP_OK.  Invalidates the
 * context's last forward for lp_render_backward.                            */
lp_status lp_debug_scan(lp_ctx* ctx, const unsigned int* counts, long long n, unsigned int* offsets,
                        unsigned int* total, void* stream);

/* Sizes of the last forward (host struct).                                 */
lp_status lp_get_stats(lp_ctx* ctx, lp_stats* out);

/* Parity hooks (synchronise the device; host buffers):
 * lp_debug_keys copies the sorted tile list of the last forward -- keys
 * (global_tile << 32 | binary32 bits of the camera-space centre depth) and
 * values (record index cam * n + primitive) -- up to `cap` entries, and
 * stores E in *n.  lp_debug_counts copies the per-record tile counts
 * (n_cams * n).  lp_debug_pixel_state copies the per-pixel number of
 * tile-list entries up to the last contributor and the transmittance before
 * it (total pixels each).                                                   */
lp_status lp_debug_keys(lp_ctx* ctx, unsigned long long* keys, unsigned int* vals,
                        long long cap, long long* n);
lp_status lp_debug_counts(lp_ctx* ctx, unsigned int* counts, long long cap);
lp_status lp_debug_pixel_state(lp_ctx* ctx, unsigned int* last, float* T_last, long long cap);

/* Workload counters of the last forward (synchronises; runs an instrumented
 * copy of the blend).  counts: host long long[4] receiving the numbers of
 * (pixel, primitive) pairs
 *   [0] iterated: tile-list entries each pixel walks, front to back, up to
 *       the one that stops it (the whole list if none does),
 *   [1] evaluated: of those, pairs whose face planes the blend evaluates
 *       (not proven uncovered for the pixel's lane group by the staging
 *       test; the exact-span mode evaluates every iterated pair),
 *   [2] intersected: the pixel ray crosses the primitive,
 *   [3] iterated up to each pixel's last contributor: the entries the
 *       paper's backward walks, back to front from that contributor.
 * [0] and [2] are the "iterated" and "intersected" counts of the paper's
 * App. "Rendering Performance and Efficiency", Table 7.                     */
lp_status lp_count_pairs(lp_ctx* ctx, long long* counts);

/* Per-stage device timing.  When enabled, forward and backward record CUDA
 * events between their stages on the call's stream (inside stream capture
 * they become event-record nodes of the graph, re-recorded on each replay).
 * lp_stage_times waits for the last recorded events and writes the duration
 * of each stage of the most recent forward/backward, in milliseconds, to
 * ms[LP_NUM_STAGES] (host).  Stages not run yet read as 0.                  */
lp_status lp_set_timing(lp_ctx* ctx, int enabled);
lp_status lp_stage_times(lp_ctx* ctx, float* ms);

/* ------------------------------------------------------------------------
 * Optimisation step (context-free, asynchronous on `stream`, device pointers).
 * ------------------------------------------------------------------------ */

/* Parameter layer (Sec. 3.1): per primitive its centre c float[n][3], rotation
 * quaternion q = (w, x, y, z) float[n][4] (normalised here), distances
 * float[n][D] (D = 3 for octahedra: one per axis, shared by opposite vertices;
 * D = 4 for tetrahedra: one per corner) and opacity logit float[n].  Writes
 * verts float[n][V][3]: octahedra c + d_i R e_i, c - d_i R e_i for axis i in
 * the vertex order of lp_prims; tetrahedra c + d_k R b_k with b_k the four
 * directions (+1,+1,+1), (+1,-1,-1), (-1,+1,-1), (-1,-1,+1) over sqrt(3);
 * and opacity float[n] = sigmoid(logit).  Distances are used as given.       */
lp_status lp_params_forward(int kind, int n, const float* centre, const float* quat, const float* dist,
                            const float* logit, float* verts, float* opacity, void* stream);

/* Adjoint of lp_params_forward (Sec. 3.4: corner gradients split into the
 * rotation and the distances).  dverts float[n][V][3] and dopacity float[n]
 * are inputs; dcentre float[n][3] is ADDED to (pass the renderer's centre
 * gradient); dquat float[n][4], ddist float[n][D], dlogit float[n] are
 * overwritten.                                                               */
lp_status lp_params_backward(int kind, int n, const float* quat, const float* dist, const float* logit,
                             const float* dverts, const float* dopacity, float* dcentre, float* dquat,
                             float* ddist, float* dlogit, void* stream);

/* L1 image loss (the L1 term of Sec. 3.4's loss): grad[i] = sign(image[i] -
 * target[i]) / count for count floats; if loss (device double) is non-NULL,
 * mean |image - target| is ADDED to *loss.                                   */
lp_status lp_l1_loss_grad(const float* image, const float* target, long long count, float* grad,
                          double* loss, void* stream);

/* Fused Adam (Sec. 3.4; Kingma & Ba) over parameter groups of one flat float
 * array: groups[k] covers params[offset, offset + count); groups ascend and
 * do not overlap (1 <= n_groups <= LP_ADAM_MAX_GROUPS).
 * Learning rate of element j of a group (j counted from its offset) at step t
 * (1-based): lr_tail when period > 0 and j % period >= head -- so one
 * [n][K][3] SH array can give its DC term and its higher bands different
 * rates (period 3K, head 3) -- else lr, or, when decay_steps > 0, the
 * log-linear blend lr^(1-f) * lr_final^f with f = min(t / decay_steps, 1)
 * (the exponential position schedule of 3DGS, which the paper keeps).
 * m, v: first/second moments, same layout as params.  step: device int, the
 * number of completed steps; the call uses t = step + 1 and then increments
 * it on the device, so replays of a captured step advance.  */
#define LP_ADAM_MAX_GROUPS 8
typedef struct {
    long long offset;
    long long count;
    float lr;
    float lr_final;
    int decay_steps;
    int period;
    int head;
    float lr_tail;
} lp_adam_group;
lp_status lp_adam_step(float* params, const float* grads, float* m, float* v, const lp_adam_group* groups,
                       int n_groups, float beta1, float beta2, float eps, int* step, void* stream);

/* Population control (Sec. 3.4 "Adaptive Population Control"; thresholds of
 * App. "Experimental Setting": opacity 0.025, 40% of the scene, 20 pixels,
 * gradient 1.5e-4, 1% of the scene, children 1/1.2 the size).
 *
 * Size of a primitive: an octahedron's longest axis 2 max_i |d_i|, a
 * tetrahedron's sqrt(2) max_k |d_k| (binary32, single rounding).
 *
 * lp_population_decide: action[i] (unsigned char) =
 *   LP_POP_PRUNE if logit < (float)log(min_opacity / (1 - min_opacity)) or
 *                size > max_scene_frac * scene_extent or px_max > max_pixels;
 *   else LP_POP_CLONE / LP_POP_SPLIT if grad_count > 0 and
 *                grad_sum / grad_count > grad_threshold, cloned when size <
 *                clone_scene_frac * scene_extent, split otherwise;
 *   else LP_POP_KEEP.
 * (products and the quotient rounded to binary32 once each), dest[i] = the
 * exclusive prefix sum of the output counts 0 / 1 / 2 / 2, *n_out (device
 * unsigned) = their total.  dist float[n][D], logit float[n] and the
 * statistics (see lp_set_densify_stats) are inputs.  scratch: device,
 * lp_population_scratch(n) unsigned ints.  Errors: LP_ERR_INVALID for a bad
 * kind, n < 0, NULL pointers or rules outside (0, inf).                   */
#define LP_POP_PRUNE 0
#define LP_POP_KEEP 1
#define LP_POP_CLONE 2
#define LP_POP_SPLIT 3
typedef struct {
    float scene_extent;
    float min_opacity;
    float max_scene_frac;
    unsigned int max_pixels;
    float grad_threshold;
    float clone_scene_frac;
} lp_population_rules;
long long lp_population_scratch(long long n);
lp_status lp_population_decide(int kind, int n, const float* dist, const float* logit, const float* grad_sum,
                               const unsigned int* grad_count, const unsigned int* px_max,
                               const lp_population_rules* rules, unsigned char* action, unsigned int* dest,
                               unsigned int* n_out, unsigned int* scratch, void* stream);

/* lp_population_apply: the new population, written to dst[s] for each of
 * n_sets array sets (device float arrays in the layout of lp_params_forward:
 * centre [n][3], quat [n][4], dist [n][D], logit [n], sh [n][sh_coeffs][3]).
 * Set 0 holds the parameters, sets 1.. per-parameter optimiser state (Adam's
 * moments).  Primitive i goes to rows dest[i].. of every set:
 *   KEEP   one row, a copy;
 *   CLONE  two rows: the copy, then a clone with the same parameters and
 *          zero state (Sec. 3.4);
 *   SPLIT  two children with the origin's quat, logit and sh, distances
 *          d / 1.2, zero state, and centres c + R(q) (|d| * z_j) (octahedron:
 *          standard deviations equal to the distances along the rotated axes)
 *          or c + (max |d| / 2) z_j (tetrahedron), z_j = normals[i][j][0..2]
 *          (device float[n][2][3], standard-normal draws of the caller);
 *   PRUNE  nothing.
 * dst arrays hold at least *n_out rows and must not overlap src.  action and
 * dest come from lp_population_decide.  1 <= n_sets <= 4.
 * Errors: LP_ERR_INVALID for a bad kind, sh_coeffs not in {1, 4, 9, 16},
 * n < 0, NULL pointers.                                                    */
typedef struct {
    float* centre;
    float* quat;
    float* dist;
    float* logit;
    float* sh;
} lp_param_arrays;
lp_status lp_population_apply(int kind, int sh_coeffs, int n, const unsigned char* action,
                              const unsigned int* dest, const float* normals, const lp_param_arrays* src,
                              const lp_param_arrays* dst, int n_sets, void* stream);

/* Allocation-free forward render of ONE camera.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- services whose device memory belongs to a pool or budget they
 * may not bypass, embedded or real-time hosts that forbid allocation after
 * start-up.  It runs the same kernels as lp_render_forward (default tuning,
 * 64-bit key sort) and writes the same image, but takes no context and
 * allocates nothing: its scratch is one fixed array of about 10.6 MiB inside
 * the library, held by every GPU that uses it until the process exits.
 *   prims   as for lp_render_forward; n <= 16384.
 *   cam     one camera, width * height <= 262144 and at most 2048 16x16 tiles.
 *   bg      host float[3]; image: device float[3][H][W], overwritten.
 *   stream  must belong to the current device (LP_ERR_INVALID otherwise).
 * Returns LP_ERR_CAPACITY, before launching anything, when n, the pixel or
 * the tile count exceeds those limits, and after the key scan when the tile
 * list would exceed 262144 entries (the image is then not written).  The
 * call synchronises `stream` twice: after the key scan, to read the
 * tile-list length, and at the end, to read the status the kernels latch on
 * the device (returned as LP_ERR_CAPACITY or LP_ERR_TIMEOUT).
 * All calls share the scratch array and it keeps the previous call's
 * contents (each call clears what must start at zero): calls whose GPU work
 * overlaps -- on different streams or host threads -- race and must be
 * serialised by the caller.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  No backward state is kept
 * (lp_render_backward needs lp_render_forward).                            */
lp_status lp_render_forward_noalloc(const lp_prims* prims, const lp_camera* cam, const float bg[3],
                                    float* image, void* stream);

/* Description of the last error on this context ("" if none).             */
const char* lp_last_error(lp_ctx* ctx);

/* Static name of a status code.                                            */
const char* lp_status_string(lp_status s);

#ifdef __cplusplus
}
#endif

#endif /* LINPRIM_H */
