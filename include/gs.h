/*
 * gs.h -- C ABI of the B300 (sm_103a) online 3D Gaussian Splatting step.
 *
 * The paper (Streaming Real-Time Rendered Scenes as 3D Gaussians) keeps a
 * 3DGS scene model that an optimiser thread continuously refits to rendered
 * reference views: it "renders the present Gaussian model from those
 * viewpoints, compares the result to the captured ground-truth images, and
 * updates the trainable Gaussian parameters" (Sec. 3.1), with "the same
 * parameters as in prior 3DGS work" (Sec. 3.2.3), and streams the changed
 * Gaussians as tensor-delta packets between snapshots (Sec. 3.5).  The calls
 * below are the data-parallel steps of that loop.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every call returns gs_status_t and, unless stated, only ENQUEUES work on
 *    `stream` (a cudaStream_t passed as void*; NULL = legacy default stream).
 *    Argument errors are detected on the host before anything is enqueued and
 *    returned synchronously (GS_ERR_ARG).  Errors found by kernels (a key
 *    buffer too small, a bounded wait that ran out) are recorded in the
 *    context's device status word; read it with gs_get_status().
 *  - All array pointers are DEVICE pointers unless marked "host".  The caller
 *    owns every buffer it passes; the library only borrows them for the
 *    duration of the enqueued work.  The context owns its scratch workspace.
 *  - No call allocates device memory except gs_ctx_create / gs_ctx_reserve.
 *  - A context is used by one host thread and one stream at a time.
 *  - Float data are IEEE float32.  Integer keys/indices are uint32.
 *
 * Layouts
 * -------
 *  params  float [15][n][4]  "planes"; plane 0 = mean x,y,z + opacity logit,
 *          plane 1 = log-scale x,y,z + 0, plane 2 = quaternion (w,x,y,z),
 *          planes 3..14 = 48 SH coefficients, coefficient k (l=0..3,
 *          m=-l..l) of channel c at flat index 3k+c (plane 3 + idx/4).
 *  proj    float [V][n][16]  per (view, Gaussian): u, v, depth, opacity,
 *          A, B, C (conic), radius, r, g, b, clamp mask (uint32 bits),
 *          rect lo (uint32 x0 | y0<<16), rect hi (x1 | y1<<16),
 *          tiles touched (uint32), 0.  All zero when culled.
 *  images  float, views concatenated, each planar [3][H][W]; T_final and
 *          n_contrib are [H][W] per view, concatenated the same way.
 *  tiles   views in order; tile (tx, ty) of view v has global index
 *          tile_offset(v) + ty * ceil(W/B) + tx with B = the context's tile
 *          size (16 by default).  ranges uint32 [total_tiles][2] = [start, end).
 *  grad2d  float [V][n][12] per (view, Gaussian): dL/du, dL/dv, dL/dA, dL/dB,
 *          dL/dC, dL/dopacity, dL/dr, dL/dg, dL/db, 0, 0, 0.
 */
#ifndef GS_H_
#define GS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GS_OK = 0,
    GS_ERR_ARG = 1,       /* bad argument (null pointer, bad size or range)        */
    GS_ERR_CAPACITY = 2,  /* a caller buffer or the workspace is too small         */
    GS_ERR_CUDA = 3,      /* a CUDA runtime call failed                            */
    GS_ERR_OOM = 4,       /* workspace allocation failed                           */
    GS_ERR_TIMEOUT = 5    /* a bounded inter-block wait in a kernel ran out        */
} gs_status_t;

typedef struct gs_ctx gs_ctx;

/* Pinhole camera, world -> camera: x_cam = R x_world + t; x right, y down,
 * z forward; pixel (i, j) is sampled at (i + 0.5, j + 0.5).  80 bytes. */
typedef struct gs_camera {
    float R[9];          /* row-major */
    float t[3];
    float fx, fy, cx, cy;
    int32_t width, height;
    float near_plane;    /* Gaussians with camera z <= near_plane are culled */
    float _pad;
} gs_camera;

/* Scene dynamics (Sec. 3.4).  Rigid objects (Sec. 3.4.2): Gaussian i belongs
 * to object group[i]; its mean, rotation and SH appearance are stored in that
 * object's frame, and the object's current pose (rotation R_g, translation
 * t_g) is applied before rendering: mean_world = R_g mean + t_g, covariance
 * R_g Sigma R_g^T, SH evaluated at the view direction in the object frame.
 * Relighting (Sec. 3.4.1), simplified to a Lambertian factor of one
 * directional light on the DC coefficient:
 *   DC_used = DC * (ambient + diffuse * max(0, (R_g normal) . light)).
 * The poses and the light live in device memory so that a captured graph sees
 * each frame's values; they are inputs, never differentiated. */
typedef struct gs_dynamics {
    int32_t n_groups;        /* objects, 1..256 */
    int32_t _pad;
    const uint8_t* group;    /* device [n]: object of each Gaussian */
    const float* poses;      /* device [n_groups][8]: unit quaternion (w,x,y,z), translation (x,y,z), 0 */
    const float* normals;    /* device [n][4]: object-frame unit normal (x,y,z), 0; NULL: no relighting */
    const float* light;      /* device [4]: unit vector towards the light (world), 0 */
    float ambient, diffuse;
} gs_dynamics;

/* Preculling (Sec. 3.3): Gaussians belong to the cells of a regular grid
 * (cell of a world-space mean p: floor((p - origin) / cell_size) per axis,
 * float32, clamped to the grid); only Gaussians of kept cells are rendered and
 * optimised.  cell_visible comes from gs_cell_visibility (or the caller). */
typedef struct gs_precull {
    const uint8_t* cell_visible; /* device, [dims[2]][dims[1]][dims[0]], nonzero: kept */
    float origin[3];             /* world position of the grid's lowest corner */
    float cell_size;
    int32_t dims[3];
    int32_t _pad;
} gs_precull;

/* SH relighting (Sec. 3.4.1).  The Gaussian's SH coefficients are read as
 * its diffuse radiance transfer T_c(w) = sum_k c_{k,c} Y_k(w) in its object's
 * frame, and the lighting is given as SH coefficients as well.  The colour is
 * the integral over the sphere of the transfer times the incident lighting,
 * seen from the object's frame (rotation R_g of gs_dynamics, identity for a
 * static scene):
 *   rgb_c = max(0, sum_k c_{k,c} (e'_{k,c} + v E_c Y_k(R_g^T l)) + 0.5),
 * e' the world-frame environment coefficients e rotated into the object's
 * frame (Lenv'(w) = Lenv(R_g w)), l the unit vector towards the directional
 * light of radiance E_c, v = visibility / 255 its per-Gaussian light
 * visibility (only the direct light is attenuated).  The colour does not
 * depend on the view; the SH coefficients get its gradient, the mean none.
 * Exclusive with the Lambertian factor of gs_dynamics (normals must be NULL).
 * The buffers live in device memory so that a captured graph sees each
 * frame's values. */
typedef struct gs_lighting {
    const float* light;          /* device [56]: e[16][3] (k-major, rgb), then l (x, y, z, 0),
                                    then E (r, g, b, 0) */
    const uint8_t* visibility;   /* device [n] (train step: [n + n_frozen], active pool
                                    first), 255 = lit; NULL: every Gaussian lit */
} gs_lighting;

typedef struct gs_scene {
    int64_t n;           /* number of Gaussians, >= 0 */
    int32_t sh_degree;   /* 0..3 */
    int32_t _pad;
    const float* params; /* device, [15][n][4] */
    const gs_dynamics* dyn; /* host pointer; NULL: static scene */
    const gs_precull* precull; /* host pointer; NULL: every Gaussian takes part */
    const gs_lighting* lighting; /* host pointer; NULL: view-dependent SH colour */
} gs_scene;

/* Orthographic camera attached to the directional light (Sec. 3.4.1).  A
 * world point x maps to x_l = R (x - origin); texel coordinates
 * u = x_l / texel + width / 2, v = y_l / texel + height / 2, light depth
 * z_l; texel (i, j) is sampled at (i + 0.5, j + 0.5).  72 bytes. */
typedef struct gs_light_camera {
    float R[9];          /* row-major world -> light rotation: map x, map y, depth axis */
    float origin[3];     /* world point at the map's centre and depth 0 */
    float texel;         /* world units per texel, > 0 */
    int32_t width, height; /* texels, 1..16384 each */
    float alpha_min;     /* footprint threshold, 0 < alpha_min <= 0.99 */
    float bias;          /* depth bias of the visibility test (world units), >= 0 */
    float _pad;
} gs_light_camera;

/* ---------------------------------------------------------------- context */

/* Creates a context bound to CUDA device `device` with `workspace_bytes` of
 * scratch (may be 0; grow it later with gs_ctx_reserve).  Synchronous. */
gs_status_t gs_ctx_create(gs_ctx** out, int device, size_t workspace_bytes);
/* Destroys the context and frees its workspace.  Synchronous. */
gs_status_t gs_ctx_destroy(gs_ctx* ctx);
/* Ensures the workspace holds at least `bytes`; reallocates (after a device
 * synchronise) if it does not.  Synchronous; never call during capture. */
gs_status_t gs_ctx_reserve(gs_ctx* ctx, size_t bytes);
/* Tile size B in pixels (8 or 16; default 16).  Changes the tile grid
 * seen by every later call. */
gs_status_t gs_ctx_set_tile(gs_ctx* ctx, int32_t tile);
/* Radix digit width of the tile-key sort (4..8 bits; default 8). */
gs_status_t gs_ctx_set_sort_bits(gs_ctx* ctx, int32_t bits);
/* Keys per thread of a tile-key sort pass (8, 12 or 16; default 16): larger
 * tiles mean fewer look-back steps, smaller ones more resident blocks. */
gs_status_t gs_ctx_set_sort_items(gs_ctx* ctx, int32_t items);
/* How (tile, Gaussian) entries are binned; both give the identical sorted
 * arrays and ranges.
 *   GS_BINNING_TWO_LEVEL (default): one entry per touched super-tile of
 *     8 x 8 tiles is emitted in depth order and sorted stably by super-tile;
 *     each super-tile's list is then expanded into its tiles' lists, whose
 *     offsets come from a count and a scan.  The radix sort moves roughly
 *     (tiles per Gaussian / super-tiles per Gaussian) times fewer entries.
 *   GS_BINNING_DIRECT: one entry per touched tile, sorted stably by tile key.
 * Returns GS_ERR_ARG for any other mode. */
#define GS_BINNING_TWO_LEVEL 0
#define GS_BINNING_DIRECT 1
gs_status_t gs_ctx_set_binning(gs_ctx* ctx, int32_t mode);
/* Threads per pixel row of a 16 x 16 tile (2 or 4; default 4) in compositing
 * and in its adjoint: each thread owns 16 / threads_per_row adjacent pixels.
 * Fewer threads per row share each fragment's loads and gradient reduction
 * among more pixels; more threads per row give more warps per tile.  8 x 8
 * tiles always use 4.  Results are identical up to the order of
 * floating-point gradient sums.  gs_ctx_set_raster_threads sets both kernels,
 * gs_ctx_set_raster_bwd_threads the adjoint alone. */
gs_status_t gs_ctx_set_raster_threads(gs_ctx* ctx, int32_t threads_per_row);
gs_status_t gs_ctx_set_raster_bwd_threads(gs_ctx* ctx, int32_t threads_per_row);
/* The context's current binning mode (GS_BINNING_*), digit width, items per
 * thread and the compositing / adjoint threads per row (any pointer may be
 * NULL). */
gs_status_t gs_ctx_get_tuning(const gs_ctx* ctx, int32_t* binning, int32_t* sort_bits, int32_t* sort_items,
                              int32_t* raster_threads, int32_t* raster_bwd_threads);
/* One configuration timed by gs_autotune. */
typedef struct gs_tune_entry {
    int32_t binning;         /* GS_BINNING_* */
    int32_t sort_bits;       /* radix digit width */
    int32_t sort_items;      /* keys per thread per sort tile */
    int32_t raster_threads;  /* threads per pixel row (both compositing kernels) */
    float ms;                /* mean time of one pass */
    float ms_render_fwd;     /* of which compositing */
    float ms_render_bwd;     /* of which its adjoint */
} gs_tune_entry;

/* Autotuner.  Times projection, binning and sorting, compositing and the
 * compositing adjoint of `scene` for the cameras (device copy d_cams, host copy
 * host_cams) under every combination of binning {two-level, direct} x digit
 * bits {8, 7, 6} x items per thread {16, 12, 8} x threads per pixel row
 * {4, 2} (8-px tiles: 4 only), `reps` passes each after one warm-up pass.  It
 * leaves the context set to the binning and sort settings with the smallest
 * time outside compositing (the sorted lists, and so the compositing cost, do
 * not depend on them), and to the compositing and adjoint layouts that are
 * fastest on their own.  The tile size is kept (it defines the
 * caller's tile grid).  The adjoint is fed the rendered image as its image
 * gradient; its cost does not depend on the values.  Workspace: gs_workspace_size(ctx, host_cams, V,
 * n, keys_cap).  Synchronous (it waits on events), so not for stream capture;
 * a graph captured earlier keeps its old configuration until captured again.
 * results (may be NULL when max_results is 0) receives up to max_results
 * entries in the order tried, *n_results (may be NULL) their number.  A kernel
 * error (for example GS_ERR_CAPACITY when keys_cap is too small) stops the
 * search, restores the previous settings and is returned (the status word
 * keeps it). */
gs_status_t gs_autotune(gs_ctx* ctx, const gs_scene* scene, const gs_camera* d_cams, const gs_camera* host_cams,
                        int32_t n_views, int64_t keys_cap, int32_t reps, gs_tune_entry* results,
                        int32_t max_results, int32_t* n_results, void* stream);
/* Preculling visibility (Sec. 3.3: "each camera determines a set of visible
 * cells using depth testing").  d_depth holds each view's depth buffer
 * (camera-space z of the nearest surface, +inf where empty), views back to
 * back as [height][width] floats.  A cell is kept (d_cell_visible[c] = 1) when
 * some view sees it by a conservative hierarchical depth test, evaluated in
 * float32 with fused multiply-adds:
 *   - the 8 corners go to camera space (z = R[6]x + R[7]y + R[8]z + t[2] as
 *     nested FMAs); all at z <= near: not seen; some: the whole image at depth
 *     near; otherwise u = fx * (x / z) + cx (FMA), v likewise, and the pixel
 *     range floor(min u)..floor(max u) x floor(min v)..floor(max v), clipped
 *     (empty: not seen), at depth min z;
 *   - in the buffer's max pyramid (level k + 1 of size ((w+1)/2, (h+1)/2)
 *     holds 2x2 maxima), the first level at which the range spans at most 2
 *     texels per axis; seen when depth <= the max of those texels.
 * It never drops a cell whose pixels show something at or behind the cell.
 * Workspace: gs_precull_workspace_size(host_cams, V) bytes. */
gs_status_t gs_cell_visibility(gs_ctx* ctx, const gs_camera* d_cams, const gs_camera* host_cams, int32_t n_views,
                               const float* d_depth, const gs_precull* grid, uint8_t* d_cell_visible,
                               void* stream);
size_t gs_precull_workspace_size(const gs_camera* host_cams, int32_t n_views);
/* Light-space depth map (Sec. 3.4.1), rendered from the Gaussians of
 * `scene` (the paper's engine renders it from its meshes).  Texel (i, j) of
 * depth [height][width] (float32, device) receives the smallest light depth
 * z_l of the Gaussians whose splat alpha at the texel centre reaches
 * alpha_min: o exp(-q / 2) >= alpha_min, q = d^T Sigma2^-1 d, Sigma2 the
 * orthographic image of the world covariance in texel units plus 0.3 I,
 * d = texel centre - (u, v) of the mean.  Texels no Gaussian covers hold
 * +inf.  accumulate = 0 first fills the map with +inf; 1 adds this scene's
 * Gaussians to the map as it is (a second pool).  The scene's dynamics apply;
 * preculling and lighting are ignored (every Gaussian casts a shadow).  The
 * result does not depend on the order of the Gaussians.  No workspace. */
gs_status_t gs_light_depth_map(gs_ctx* ctx, const gs_scene* scene, const gs_light_camera* lcam, float* depth,
                               int32_t accumulate, void* stream);
/* Per-Gaussian light visibility (Sec. 3.4.1): visibility[i] (uint8, device)
 * = 255 when the mean of Gaussian i falls outside the map or its light depth
 * is at most depth[floor(v)][floor(u)] + bias, else 0.  No workspace. */
gs_status_t gs_light_visibility(gs_ctx* ctx, const gs_scene* scene, const gs_light_camera* lcam,
                                const float* depth, uint8_t* visibility, void* stream);
/* Bound of every wait of one block on another in the context's kernels
 * (the look-backs of the onesweep sort passes and of the key emission), in
 * SM clock cycles counted from the start of the wait; 0 restores the default
 * of 2e9 cycles (about one second at 2 GHz).  A wait that runs out records
 * GS_ERR_TIMEOUT in the status word, its block publishes what it has and
 * skips its scatter, and the kernel returns: results of that call are then
 * incomplete, never out of bounds.  Read by calls enqueued later; a graph
 * keeps the value it was captured with.  GS_ERR_ARG for cycles < 0. */
gs_status_t gs_ctx_set_wait_limit(gs_ctx* ctx, int64_t cycles);
/* Test hook of the bounded waits (failure detection without a GPU fault):
 * with tile >= 0, the next gs_bin_sort calls of this context with direct
 * binning (GS_BINNING_DIRECT) run the last pass of their tile-key sort with
 * onesweep tile `tile` withholding its digit counts, a flag that nothing
 * else sets, so that the waits of the tiles after it run out
 * (GS_ERR_TIMEOUT).  Only that pass is affected: its output goes to the
 * caller's arrays, which no later kernel of the call reads, and those arrays
 * are then incomplete.  Two-level binning and the fused calls ignore the
 * hook.  -1 (the default) turns it off; GS_ERR_ARG below -1. */
gs_status_t gs_ctx_set_wait_test(gs_ctx* ctx, int64_t tile);
/* Reads and clears the device status word (synchronises `stream`).
 * *status receives the first error a kernel recorded since the last read
 * (GS_OK if none); *detail receives the required size for GS_ERR_CAPACITY. */
gs_status_t gs_get_status(gs_ctx* ctx, void* stream, int32_t* status, int64_t* detail);
/* Workspace bytes the steps below need for V views (camera array on the
 * host), n Gaussians and a key capacity of keys_cap. */
size_t gs_workspace_size(const gs_ctx* ctx, const gs_camera* host_cams, int32_t n_views,
                         int64_t n, int64_t keys_cap);
/* Total tiles and pixels of a camera set (host array), for sizing buffers. */
int64_t gs_total_tiles(const gs_ctx* ctx, const gs_camera* host_cams, int32_t n_views);

/* ---------------------------------------------------------------- forward */

/* EWA projection with SH colour, for every (view, Gaussian).  Sec. 3.2.3
 * (3DGS parameters rendered by differentiable splatting), Sec. 3.2.2 / 3.4.1
 * (SH appearance).  Per view: t = R mu + t_cam; Sigma = R_q S S^T R_q^T;
 * Jacobian J of the pinhole map at t (x/z, y/z clamped to 1.3 tan(fov/2));
 * Sigma2D = J R Sigma R^T J^T + 0.3 I; conic = Sigma2D^-1; radius =
 * ceil(3 sqrt(lambda_max)), lambda_max = mid + sqrt(max(0.1, mid^2 - det));
 * tile rectangle: the tiles [floor((u - r) / B), floor((u + r + B - 1) / B))
 * (likewise in v) of the square of half-side r, cut to the tiles that hold
 * a pixel centre inside the bounding box of the ellipse where alpha reaches
 * 1/255 (half-widths sqrt(tau a), sqrt(tau c), tau = 2 ln(255 o), for the
 * 2D covariance (a, b; b, c), widened by 0.1 % + 0.01 px; none when
 * o < 1/255): every pixel the square's compositing takes the splat at lies
 * inside, so images and gradients are those of the square;
 * rgb = SH(dir) + 0.5 clamped at 0; opacity = sigmoid(logit).  Culled:
 * z <= near, det <= 0, or empty rect.
 * d_cams: device gs_camera[V].  Writes proj [V][n][16]. */
gs_status_t gs_project(gs_ctx* ctx, const gs_scene* scene, const gs_camera* d_cams,
                       int32_t n_views, float* proj, void* stream);

/* Tile binning + radix sort (Sec. 3.2.3: the model is refit by the
 * differentiable tile rasterisation of the cited 3DGS method, whose per-tile
 * lists are depth-sorted): every (view, Gaussian, touched tile) becomes one
 * (tile key, Gaussian index) entry, ordered by (view, tile, float32 depth,
 * Gaussian index); then per-tile [start, end) ranges.  Implemented as a
 * stable depth sort of the V*n projected Gaussians followed by a stable
 * LSD radix sort of the tile keys (both in-house onesweep sorts).
 * total_tiles: gs_total_tiles() of the camera set (host-known; a mismatch
 * with the device cameras records GS_ERR_ARG).
 * sorted_keys (may be NULL) / sorted_vals: uint32 [keys_cap];
 * ranges: uint32 [total_tiles][2]; d_num_keys: uint32 on the device.
 * If the entry count K exceeds keys_cap, nothing beyond keys_cap is written,
 * *d_num_keys = K, and the status word records GS_ERR_CAPACITY with K. */
gs_status_t gs_bin_sort(gs_ctx* ctx, const float* proj, const gs_camera* d_cams,
                        int32_t n_views, int64_t n, int64_t total_tiles, int64_t keys_cap,
                        uint32_t* sorted_keys, uint32_t* sorted_vals, uint32_t* ranges,
                        uint32_t* d_num_keys, void* stream);

/* Front-to-back alpha compositing per pixel over its tile's sorted list
 * (Sec. 3.1: the optimiser "renders the present Gaussian model from those
 * viewpoints"; Sec. 3.2.3: the cited 3DGS method's differentiable
 * rasteriser): alpha = min(0.99, o exp(P)), P = -(A dx^2 + C dy^2)/2 - B dx dy, skipped
 * when P > 0 or alpha < 1/255; stops before the fragment that would take
 * T below 1e-4.  image = sum c alpha T + T_final * bg.  n_contrib = 1-based
 * list position of the last fragment added (0 if none).
 * bg: host float[3].  T_final / n_contrib may be NULL (forward only). */
gs_status_t gs_render_fwd(gs_ctx* ctx, const float* proj, const gs_camera* d_cams,
                          int32_t n_views, int64_t n, int64_t total_tiles,
                          const uint32_t* sorted_vals,
                          const uint32_t* ranges, const float* bg, float* image,
                          float* T_final, uint32_t* n_contrib, void* stream);

/* --------------------------------------------------------------- loss */

/* L = w_l1 * mean|x - y| + w_ssim * (1 - mean SSIM) over V views of H x W x 3
 * (11x11 Gaussian window, sigma 1.5, C1 = 1e-4, C2 = 9e-4, zero padding),
 * and dL/dx.  Sec. 3.1 ("compares the result to the captured ground-truth
 * images ... using the configured loss").  d_loss: one float on the device.
 * dimage may alias nothing else.  All views must share H and W. */
gs_status_t gs_loss(gs_ctx* ctx, const float* image, const float* target, int32_t n_views,
                    int32_t height, int32_t width, float w_l1, float w_ssim,
                    float* d_loss, float* dimage, void* stream);

/* --------------------------------------------------------------- backward */

/* Reverse-order adjoint of gs_render_fwd (Sec. 3.2.3: the parameters are
 * refit by gradient descent through the differentiable rasteriser; Sec. 3.1:
 * "compares the result ... and updates the trainable Gaussian parameters"):
 * per pixel, walks its list back from n_contrib, recovering each T_j from
 * T_final (no per-fragment state is stored), and accumulates dL/d(u, v, A, B, C, opacity, rgb) per (view,
 * Gaussian) into grad2d (which it first zeroes). */
gs_status_t gs_raster_bwd(gs_ctx* ctx, const float* proj, const gs_camera* d_cams,
                          int32_t n_views, int64_t n, int64_t total_tiles,
                          const uint32_t* sorted_vals,
                          const uint32_t* ranges, const float* bg, const float* T_final,
                          const uint32_t* n_contrib, const float* dimage, float* grad2d,
                          void* stream);

/* Adjoint of gs_project (Sec. 3.2.3: gradients of the 3DGS parameters --
 * mean, scale, rotation, opacity, SH coefficients -- through the EWA
 * projection and the SH colour of Sec. 3.2.2 / 3.4.1): grad2d of every view
 * -> parameter gradients dparams [15][n][4], summed over views (accumulate != 0 adds to dparams,
 * else overwrites).  Zero through clamps, culls and rounding steps. */
gs_status_t gs_project_bwd(gs_ctx* ctx, const gs_scene* scene, const gs_camera* d_cams,
                           int32_t n_views, const float* proj, const float* grad2d,
                           float* dparams, int32_t accumulate, void* stream);

/* gs_raster_bwd followed by gs_project_bwd (overwriting dparams): the
 * gradient of the loss with respect to every trainable parameter of the
 * current model (Sec. 3.1, 3.2.3). */
gs_status_t gs_render_bwd(gs_ctx* ctx, const gs_scene* scene, const gs_camera* d_cams,
                          int32_t n_views, int64_t total_tiles, const float* proj,
                          const uint32_t* sorted_vals,
                          const uint32_t* ranges, const float* bg, const float* T_final,
                          const uint32_t* n_contrib, const float* dimage, float* grad2d,
                          float* dparams, void* stream);

/* --------------------------------------------------------------- update */

typedef struct gs_adam_cfg {
    float lr[60];        /* per element of a Gaussian's 60 floats (plane*4 + lane) */
    float beta1, beta2, eps;
    int32_t step;        /* 1-based step, used when d_step is NULL */
    const int32_t* d_step; /* optional device step counter: read (and, if
                              increment != 0, incremented by 1 after use) */
    int32_t increment;
    int32_t _pad;
} gs_adam_cfg;

/* Adam with bias correction over theta/grad/m/v [15][n][4] (Sec. 3.1
 * "configured ... learning rates"; Sec. 3.3 optimiser state).  Pad lanes get
 * zero gradient and stay put. */
gs_status_t gs_adam_step(gs_ctx* ctx, float* theta, const float* grad, float* m, float* v,
                         int64_t n, const gs_adam_cfg* cfg, void* stream);

/* Changed-set extraction for the incremental stream (Sec. 3.5: tensor-delta
 * packets between snapshots, residuals against the last transmitted state).
 * Gaussian i is changed when max_k |theta_k - baseline_k| > thr over its 60
 * floats (float32 arithmetic).  Writes changed indices ascending to d_idx
 * (uint32 [n]), one 128-byte record each to d_records (uint32 index, float32
 * mean xyz, then 56 float16 RNE: log-scale xyz, quaternion wxyz, opacity
 * logit, 48 SH), the count to *d_count, and copies theta into baseline for
 * every changed Gaussian. */
gs_status_t gs_extract_delta(gs_ctx* ctx, const float* theta, float* baseline, int64_t n,
                             float thr, uint32_t* d_idx, uint8_t* d_records,
                             uint32_t* d_count, void* stream);

/* Attribute groups of a Gaussian's 60 stored floats, for tensor deltas
 * (Sec. 3.5: tensor-delta packets per attribute, each tensor on its own
 * schedule; opacity and DC every frame, the others less often).  Flat float
 * indices and record encoding per group: */
#define GS_ATTR_MEAN 1      /* floats 0..2, float32 (12-byte record) */
#define GS_ATTR_OPACITY 2   /* float 3 (logit), float16 (2 B) */
#define GS_ATTR_SCALE 4     /* floats 4..6 (log-scale), float16 (6 B) */
#define GS_ATTR_ROTATION 8  /* floats 8..11 (quaternion), float16 (8 B) */
#define GS_ATTR_DC 16       /* floats 12..14 (SH degree 0), float16 (6 B) */
#define GS_ATTR_SH_REST 32  /* floats 15..59 (SH degrees 1-3), float16 (90 B) */

/* Record size in bytes of one group's tensor delta; -1 if `attr` is not one
 * GS_ATTR_* value. */
int32_t gs_tensor_record_bytes(int32_t attr);

/* Tensor delta of one attribute group.  Gaussian i is sent when max over the
 * group's floats of |theta - baseline| > thr (float32 compare).  Outputs, in
 * ascending index order: d_idx uint32[M], d_vals M records of
 * gs_tensor_record_bytes(attr) bytes packed densely (the group's floats in
 * flat order, float32 for GS_ATTR_MEAN, float16 round-to-nearest-even
 * otherwise), *d_count = M.  The sent Gaussians' group floats in `baseline`
 * take theta's values; its other floats are untouched.  Buffers hold n
 * entries.  Workspace as gs_extract_delta.  GS_ERR_ARG for a bad attr. */
gs_status_t gs_extract_tensor_delta(gs_ctx* ctx, const float* theta, float* baseline, int64_t n, int32_t attr,
                                    float thr, uint32_t* d_idx, void* d_vals, uint32_t* d_count, void* stream);
/* Client-side replay of a tensor delta into `params` (planes [15][n][4]):
 * the first *d_count records' decoded values replace the group's floats of
 * Gaussian d_idx[i].  Indices >= n are skipped and recorded as GS_ERR_ARG in
 * the status word.  No workspace. */
gs_status_t gs_apply_tensor_delta(gs_ctx* ctx, float* params, int64_t n, int32_t attr, const uint32_t* d_idx,
                                  const void* d_vals, const uint32_t* d_count, void* stream);
/* Client-side replay of gs_extract_delta's 128-byte records: mean exactly,
 * log-scale, quaternion, opacity logit and SH decoded from float16; the pad
 * float is untouched.  Indices >= n are skipped (GS_ERR_ARG in the status
 * word). */
gs_status_t gs_apply_delta(gs_ctx* ctx, float* params, int64_t n, const uint8_t* d_records,
                           const uint32_t* d_count, void* stream);

/* Largest n accepted by gs_extract_delta_noalloc. */
#define GS_NOALLOC_MAX_GAUSSIANS 4194304

/* gs_extract_delta for callers that cannot allocate device memory (the paper
 * has no counterpart; this is a property of the library, not of the method).
 * A sender on a real-time thread must not call cudaMalloc, which can block on
 * the device, and a host whose device memory belongs to another allocator may
 * have no workspace or context to give.  This call takes no context and
 * allocates nothing: its scratch (about 4.3 MB) is a fixed device array in
 * the library, held by every GPU that loads it until the process exits.
 * Same arguments, outputs and results as gs_extract_delta.  n above
 * GS_NOALLOC_MAX_GAUSSIANS returns GS_ERR_CAPACITY with nothing enqueued.
 * All calls on a device share the array (its old contents never matter, so
 * nothing is cleared); calls that overlap on the GPU race and must not be
 * issued.  The first call on a device looks the array's address up with that
 * device current and keeps it for the life of the process; make that call
 * outside any stream capture.  The kept address belongs to the device's
 * primary context: after that context is reset (cudaDeviceReset) or torn
 * down and created again, it is stale and the call must not be used. */
gs_status_t gs_extract_delta_noalloc(const float* theta, float* baseline, int64_t n, float thr,
                                     uint32_t* d_idx, uint8_t* d_records, uint32_t* d_count,
                                     void* stream);

/* --------------------------------------------------------------- serving */

/* Forward-only render of R client viewpoints (any mix of resolutions) of a
 * device-resident model (Sec. 3.1 / 3.5: the client "continuously render[s]
 * that model ... from the viewpoint of the camera that tracks the user").
 * image: views concatenated as for gs_render_fwd.  Scratch from the context
 * workspace (size with gs_workspace_size(ctx, cams, R, n, keys_cap)). */
gs_status_t gs_render_batch(gs_ctx* ctx, const gs_scene* scene, const gs_camera* d_cams,
                            int32_t n_requests, int64_t total_tiles, int64_t keys_cap,
                            const float* bg,
                            float* image, void* stream);

/* gs_render_batch with a host copy of the cameras (host_cams: R records,
 * read during the call, as d_cams holds them): the tile total comes from
 * their sizes, and with the exact super-tile total the super-tile sort takes
 * no more digit passes than that count needs and compositing takes the
 * longest tile lists first.  Same image, bit for bit.  A device view table
 * whose totals differ from host_cams' is reported as GS_ERR_ARG (device
 * status).  GS_ERR_ARG for null host_cams or a view of zero size. */
gs_status_t gs_render_batch_sized(gs_ctx* ctx, const gs_scene* scene, const gs_camera* d_cams,
                                  const gs_camera* host_cams, int32_t n_requests, int64_t keys_cap,
                                  const float* bg, float* image, void* stream);

/* ------------------------------------------------------------ fused step */

typedef struct gs_train_io {
    float* params;        /* [15][n][4], updated in place */
    float* grads;         /* [15][n][4], scratch (holds this step's gradient) */
    float* adam_m;        /* [15][n][4] */
    float* adam_v;        /* [15][n][4] */
    float* baseline;      /* [15][n][4], last transmitted values */
    const float* targets; /* V views, planar [3][H][W] each */
    float* image;         /* V views, this step's render */
    float* d_loss;        /* 1 float */
    uint32_t* d_delta_idx;   /* uint32 [n] */
    uint8_t* d_delta_records;/* [n][128] */
    uint32_t* d_delta_count; /* 1 uint32 */
    int32_t* d_step;      /* Adam step counter, incremented each step */
    const float* frozen;  /* [15][n_frozen][4] inference-only pool, or NULL */
} gs_train_io;

typedef struct gs_train_cfg {
    const gs_dynamics* dyn; /* host pointer; NULL: static scene.  Read when the
                               step is enqueued (or captured): pointers fixed */
    int64_t n;
    int32_t sh_degree;
    int32_t n_views;
    int32_t width, height; /* shared by all views */
    int64_t keys_cap;
    float w_l1, w_ssim;
    float bg[3];
    float delta_thr;
    gs_adam_cfg adam;     /* d_step / step fields are ignored: io.d_step is used */
    int64_t n_frozen;     /* Gaussians in io.frozen (0: none) */
    const gs_precull* precull; /* host pointer; NULL: no preculling.  Gaussians of
                               culled cells are not rendered and get no Adam
                               update (their parameters and moments stay) */
    const gs_lighting* lighting; /* host pointer; NULL: view-dependent SH colour */
    int32_t phases;       /* GS_TRAIN_* parts to run; 0 = GS_TRAIN_ALL */
    int32_t _pad2;
} gs_train_cfg;

/* Parts of the training step (gs_train_cfg.phases).  GS_TRAIN_GRADIENT runs
 * projection, binning, compositing, the loss and both adjoints and leaves
 * dL/dparams of this call's views in io->grads (parameters, Adam moments,
 * baseline and step counter untouched); GS_TRAIN_UPDATE runs Adam on
 * io->grads, the delta extraction and the step counter increment.  Splitting
 * the step lets a caller combine the gradients of several calls in between:
 * the views of one step spread over GPUs (Sec. 3.1 renders the model from
 * all ready reference cameras; each GPU takes some of them, with w_l1 and
 * w_ssim scaled by its share of the views, and the rank gradients are summed
 * before the update), or mini-batches of views accumulated on one GPU. */
#define GS_TRAIN_GRADIENT 1
#define GS_TRAIN_UPDATE 2
#define GS_TRAIN_ALL 3

/* One whole optimisation step over all V reference views (Sec. 3.1: "iterates
 * over ready reference cameras, optionally grouping them as mini batches"):
 * project, bin/sort, composite, loss, backward, Adam, delta extraction (or
 * the part of it cfg->phases selects).
 * Enqueue-only, no host synchronisation and no allocation: safe to capture
 * into a CUDA graph.
 * Gaussian freezing (Sec. 3.3): the n_frozen Gaussians of io.frozen are
 * rendered with the n active ones (they follow them as indices n ..
 * n + n_frozen - 1 of the sorted lists, and of the dynamics arrays when the
 * scene is dynamic) but get no gradient, no Adam update and no delta; only the
 * active pool needs grads, Adam moments and a baseline.
 * Workspace: gs_workspace_size(ctx, cams, V, n + n_frozen, keys_cap). */
gs_status_t gs_train_step(gs_ctx* ctx, const gs_camera* d_cams, const gs_train_io* io,
                          const gs_train_cfg* cfg, void* stream);

/* Number of phase boundaries gs_train_step can mark with events: before
 * projection, after projection, after the depth sort, after key emission,
 * after the tile-key sort (ranges included), after compositing, after the
 * loss, after the raster adjoint, after the projection adjoint, after Adam,
 * after delta extraction. */
#define GS_TRAIN_PHASE_EVENTS 11

/* gs_train_step that also records `events` (GS_TRAIN_PHASE_EVENTS cudaEvent_t
 * handles passed as void*, created by the caller with timing enabled) at the
 * phase boundaries, so that a caller can time each kernel phase with CUDA
 * events on the stream the kernels run on.  Under stream capture the records
 * become external event-record nodes of the graph. */
gs_status_t gs_train_step_events(gs_ctx* ctx, const gs_camera* d_cams, const gs_train_io* io,
                                 const gs_train_cfg* cfg, void* const* events, void* stream);

/* Captures gs_train_step into a CUDA graph held by the context (replacing any
 * earlier one) and replays it with gs_graph_launch.  Synchronous capture. */
gs_status_t gs_train_graph_capture(gs_ctx* ctx, const gs_camera* d_cams,
                                   const gs_train_io* io, const gs_train_cfg* cfg,
                                   void* stream);
/* As gs_train_graph_capture, with phase events recorded by every replay. */
gs_status_t gs_train_graph_capture_events(gs_ctx* ctx, const gs_camera* d_cams,
                                          const gs_train_io* io, const gs_train_cfg* cfg,
                                          void* const* events, void* stream);
gs_status_t gs_graph_launch(gs_ctx* ctx, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GS_H_ */
