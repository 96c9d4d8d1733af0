/*
 * vr.h -- C ABI of libvr, a B300 (sm_103a) implementation of the data-parallel hot path of
 * Brix, Prassni, Hinrichs, "Visualization of Large Volumetric Multi-Channel Microscopy Data
 * Streams on Standard PCs" (arXiv 1407.2074):
 *   - incremental construction of a bricked multi-channel octree while slices stream in
 *     (Sec. "Incremental Construction", steps 1-3; Sec. "Handling Volumes of Arbitrary
 *     Dimensions"; Sec. "Handling Multi-Channel Data");
 *   - front-to-back ray casting of that octree (Algorithm 1 and Sec. "Basic Ray-Casting":
 *     screen-space-error level of detail, descent, trilinear brick sampling, per-channel
 *     transfer functions, emission-absorption compositing, clip planes, early termination);
 *   - the adjoint of the compositing with respect to the transfer functions and the
 *     per-channel intensity scales (an addition of this library; the paper has none).
 *
 * Conventions shared by every call:
 *   - Every call returns a vr_status.  After a device-side error (reported through the
 *     library's error word) the context answers VR_ERR_STATE until vr_destroy.
 *   - Stream-ordered calls take a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Borrowed input pointers must stay valid until the stream reaches the call.
 *   - The library owns its device memory (brick pool, node tables, staging); callers own
 *     images and gradient buffers.  A context is not thread-safe, and its render calls share
 *     the context's work queue and scratch buffers: calls of one context issued on different
 *     streams must not overlap on the GPU (use one stream, or order the streams).
 *   - Coordinates are level-0 voxel units; voxel i is centred at i + 0.5.
 *   - There is no CPU fallback: without a CUDA device vr_create fails with VR_ERR_CUDA.
 */
#ifndef VR_H
#define VR_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vr_ctx vr_ctx;

typedef enum {
    VR_OK = 0,
    VR_ERR_INVALID_ARG = 1,
    VR_ERR_OUT_OF_MEMORY = 2,
    VR_ERR_CUDA = 3,
    VR_ERR_STATE = 4,
    VR_ERR_TIMEOUT = 5,
    VR_ERR_DEVICE_ASSERT = 6
} vr_status;

enum { VR_FP32 = 0, VR_FP16_INTERP = 1 };
enum { VR_MODE_DVR = 0, VR_MODE_MIP = 1 };
/* OR-ed into vr_render's mode: this call interpolates samples and reads the transfer functions in
 * FP16 (normalised intensities), compositing in FP32 -- as if the context had VR_FP16_INTERP. */
#define VR_RENDER_FP16 0x10
enum { VR_HOST_BLOCK = 0, VR_DEVICE_BLOCK = 1, VR_HOST_ASYNC = 2 }; /* vr_insert_block on_device */
#define VR_MAX_CHANNELS 4
#define VR_MAX_LEVELS 16
#define VR_MAX_CLIP 3

/* Optional device allocator (for instance PyTorch's caching allocator).  alloc returns NULL on
 * failure.  Both are called on the host, with the context's device current. */
typedef struct {
    void* (*alloc)(size_t bytes, void* user, void* stream);
    void (*free)(void* p, void* user, void* stream);
    void* user;
} vr_allocator;

typedef struct {
    uint16_t background;        /* value of never-inserted voxels (Sec. "Incremental Construction") */
    uint16_t homog_threshold;   /* tau: a brick is homogeneous if max - min < tau in every channel
                                   (Sec. "CPU Data Structure"); 0 disables pruning */
    size_t pool_capacity_bytes; /* brick pool size; 0 = room for every brick of the full tree */
    int precision;              /* VR_FP32 or VR_FP16_INTERP: default precision of vr_render's DVR
                                   (FP16 sample interpolation and TF lookup, FP32 compositing) */
    size_t cache_capacity_bytes; /* > 0: out-of-core rendering -- renders read bricks only from a
                                    device render cache of this size, filled on request (Sec.
                                    "GPU Data Structure", brick buffer + flag buffer); 0: renders
                                    read the brick store directly */
    int store_on_host;          /* 1: the brick store lives in mapped pinned host memory (the
                                   construction kernels write it over the bus); 0: device memory */
} vr_options;

/* One view.  The camera looks from eye at target; up fixes the roll.  fov_y_deg is the vertical
 * field of view.  Pixel (0,0) is the top-left corner.  lod_error_px is the screen-space error
 * epsilon: level L is used from the distance t_L = 2^L H / (2 eps tan(fov/2)) on (Sec. "Basic
 * Ray-Casting", optimal LOD).  step_voxels is the sampling step (Alg. 1 samplingStep, >= 1e-3;
 * a ray takes at most 2^24 samples).
 * ert_alpha stops a ray once its opacity reaches it (a value > 1 disables early termination).
 * clip[i] = (n, d) keeps the half-space n.p + d >= 0 (up to three planes, Sec. "Integration
 * into Voreen").  n_clip = -1 selects the context's planes set by vr_set_clip_planes. */
typedef struct {
    float eye[3], target[3], up[3];
    float fov_y_deg;
    int width, height;
    float lod_error_px, step_voxels, ert_alpha;
    int n_clip;
    float clip[VR_MAX_CLIP][4];
} vr_camera;

typedef struct {
    int64_t dims[3];
    int channels, brick_size, levels; /* levels = N + 1 */
    int64_t nodes;                    /* entries of the dense node tables (all levels) */
    int64_t slots_capacity, slots_used;
    int64_t pool_bytes, node_table_bytes;
    int64_t last_render_samples;      /* samples composited by the last vr_render (all cameras) */
    int64_t last_render_rays;         /* rays with a non-empty interval */
    int64_t last_render_continued;    /* rays of the last vr_render finished by its second launch
                                         (vr_set_ray_continuation) */
} vr_stats_t;

/* Create a context for a volume of final resolution dims (X, Y, Z), channels 1..4 and brick
 * edge brick_size (even, >= 4).  Only the final resolution and the channel count are known in
 * advance (Sec. "Incremental Construction").  The volume is virtually extended to
 * brick_size * 2^N per axis (Eq. 1, Sec. "Handling Volumes of Arbitrary Dimensions").  The root
 * exists from the start and holds the background value.  opts and alloc may be NULL (defaults:
 * background 0, tau 0, full-tree pool, FP32; cudaMalloc).  The current CUDA device is used.
 * Errors: VR_ERR_INVALID_ARG (bad dims/channels/brick size), VR_ERR_OUT_OF_MEMORY, VR_ERR_CUDA. */
vr_status vr_create(const int64_t dims[3], int channels, int brick_size, const vr_options* opts,
                    const vr_allocator* alloc, vr_ctx** out);

/* Release every resource of the context (synchronises the device first).  A library utility, not
 * a step of the method: the paper's renderer lives as long as its application.  Also the one call
 * that still succeeds after a device error (VR_ERR_STATE).  Errors: VR_ERR_INVALID_ARG (NULL). */
vr_status vr_destroy(vr_ctx* ctx);

/* Insert the cuboid block [origin, origin + extent) of values block[ez][ey][ex][C] (uint16, the
 * channels interleaved per voxel as in Sec. "Handling Multi-Channel Data").  Already inserted
 * values are overwritten (Sec. "Incremental Construction", step 1); every level on the
 * insertion path is updated by 2x2x2 round-half-up half-sampling (step 2) and the homogeneity
 * flags and AVG values of the touched nodes are refreshed (step 3).
 * on_device: 1 (VR_DEVICE_BLOCK) block is a device pointer; 0 (VR_HOST_BLOCK) a host pointer
 * copied by the library on cuda_stream (pinned memory makes the copy asynchronous; pageable
 * memory is copied before the call returns); 2 (VR_HOST_ASYNC) a host pointer whose copy runs on
 * the library's own upload stream without waiting for earlier work on cuda_stream, so that it
 * overlaps the rendering already queued there (the paper builds the octree beside the renderer,
 * Sec. "Incremental Construction"): the block must hold its values at the call and stay unchanged
 * until cuda_stream has passed this insert; two staging buffers alternate, so at most two such
 * uploads are in flight.  The updates themselves are ordered on cuda_stream in every mode.
 * Errors: VR_ERR_INVALID_ARG (block outside the volume, NULL block), VR_ERR_OUT_OF_MEMORY (the
 * brick pool is exhausted; nothing is modified), VR_ERR_STATE, VR_ERR_CUDA. */
vr_status vr_insert_block(vr_ctx* ctx, const int64_t origin[3], const int64_t extent[3], const uint16_t* block,
                          int on_device, void* cuda_stream);

/* The slice-wise form of vr_insert_block: slice z (0 <= z < Z) of values slice[Y][X][C]. */
vr_status vr_insert_slice(vr_ctx* ctx, int64_t z, const uint16_t* slice, int on_device, void* cuda_stream);

/* Per-channel transfer functions: tf[C][256][4] RGBA (alpha = opacity per level-0 voxel of
 * path length) and intensity scales scale[C]; intensity I maps to x = clamp(s I / 65535, 0, 1)
 * and the table is read linearly at 255 x (Alg. 1 applyTF).  Device pointers; copied on the
 * stream.  Errors: VR_ERR_INVALID_ARG (NULL pointers). */
vr_status vr_set_transfer_functions(vr_ctx* ctx, const float* tf, const float* scale, void* cuda_stream);

/* Per-channel affine sample transforms (Sec. "Correction of Chromatic Aberration": each sampling
 * point is multiplied by the channel's matrix before the volume is sampled).  m is a host array
 * [C][3][4] (row-major 3x4: rotation/scale and translation, level-0 voxel units), copied; NULL
 * or all-identity restores the untransformed path.  With transforms, each channel descends the
 * octree from its own point (FP32 interpolation; VR_RENDER_FP16 is ignored).  Used by vr_render,
 * plans and vr_render_backward.  Errors: VR_ERR_INVALID_ARG (non-finite entries). */
vr_status vr_set_channel_transforms(vr_ctx* ctx, const float* m);

/* Context-wide clip planes (up to three half-spaces n.p + d >= 0, Sec. "Integration into
 * Voreen"), used by every camera whose n_clip is -1.  planes[n][4] is a host array, copied.
 * Errors: VR_ERR_INVALID_ARG (n outside 0..3, NULL planes with n > 0). */
vr_status vr_set_clip_planes(vr_ctx* ctx, int n, const float* planes);

/* Render n_cams views in one launch.  images[i] is a device buffer [H_i][W_i][4] of
 * premultiplied RGBA FP32 (caller-owned); mode VR_MODE_DVR (Algorithm 1) or VR_MODE_MIP, optionally
 * | VR_RENDER_FP16 (DVR only; MIP always interpolates in FP32).
 * Stream-ordered.  Errors: VR_ERR_INVALID_ARG (bad camera, NULL image, no transfer functions
 * set), VR_ERR_STATE, VR_ERR_CUDA. */
vr_status vr_render(vr_ctx* ctx, const vr_camera* cams, int n_cams, float* const* images, int mode,
                    void* cuda_stream);

/* vr_render for callers that cannot let the library allocate memory during a call -- an
 * application that reserved its GPU memory up front, or a host that must not have its other
 * streams stalled by the device-wide synchronisation cudaMalloc/cudaFree can cause.  The paper
 * has no counterpart.  Same arguments, checks and images as vr_render (the context, its brick pool
 * and transfer functions must exist already), but the ray-tile queue, the sample counters and the
 * per-camera constants live in one fixed device array of libvr (about 15 KB, held by every GPU
 * that loads the library until the process exits) instead of buffers the library allocates.
 * The launch shape is the context's (vr_set_launch_shape); DVR tiles run in raster order (no
 * cost-ordered queue, whose order buffers are allocated), which changes no pixel.
 * At most VR_NOALLOC_MAX_CAMERAS cameras per call (VR_ERR_INVALID_ARG beyond).  The first call on
 * a device looks the array up (cudaGetSymbolAddress).  The per-camera constants are copied from the
 * caller's host stack by cudaMemcpyAsync, so a call must not be recorded into a CUDA graph by
 * stream capture (render plans, vr_plan_*, are the capturable form).  Every call reuses the same
 * array: calls that can overlap on the GPU (other streams, other contexts on the same device) race
 * and must be serialised by the caller.  The call does not update vr_stats' last_render_* counters. */
#define VR_NOALLOC_MAX_CAMERAS 64
vr_status vr_render_noalloc(vr_ctx* ctx, const vr_camera* cams, int n_cams, float* const* images, int mode,
                            void* cuda_stream);

/* Adjoint of vr_render (DVR) for dL/dimage given per view (device [H_i][W_i][4]): writes
 * dl_dtf[C][256][4] and dl_dscale[C] (device, overwritten).  Each ray's forward march is
 * recomputed, never stored.  Stream-ordered.  The paper has no counterpart. */
vr_status vr_render_backward(vr_ctx* ctx, const vr_camera* cams, int n_cams, const float* const* dl_dimages,
                             float* dl_dtf, float* dl_dscale, void* cuda_stream);

/* vr_render_backward given also the DVR images (FP32 interpolation) that vr_render wrote for the
 * same cameras, volume state, transfer functions and scales (device [H_i][W_i][4], unchanged
 * since): each ray's final colour and transmittance (1 - alpha) are read from its pixel instead of
 * being recomputed by a forward march, so each ray is marched once, by the sweep, which still
 * takes the forward's decisions (samples, runs, early termination) itself.  The transmittance
 * recovered as 1 - alpha carries alpha's rounding (absolute ~6e-8).  In the FP64 gradient-check
 * mode the images are not used (the double forward is recomputed).  Errors as
 * vr_render_backward, and VR_ERR_INVALID_ARG for NULL images.  The paper has no counterpart. */
vr_status vr_render_backward_with_images(vr_ctx* ctx, const vr_camera* cams, int n_cams, const float* const* images,
                                         const float* const* dl_dimages, float* dl_dtf, float* dl_dscale,
                                         void* cuda_stream);

/* Accumulation precision of vr_render_backward.  0 (default): single precision throughout.
 * 1 (FP64 gradient-check mode): the per-ray transmittance and colour of the sweep, the gradient
 * terms and their sums are double precision, for checks of the gradient element by element
 * against an FP64 reference; the decisions (samples, runs, early termination) stay those of the
 * single-precision forward.  Much slower on GPUs with few FP64 units; not for training loops.
 * The double sums (24 KB) are allocated on the first backward call in this mode.  The paper has
 * no counterpart.  Errors: VR_ERR_INVALID_ARG (fp64 not 0 or 1), VR_ERR_STATE. */
vr_status vr_set_gradient_precision(vr_ctx* ctx, int fp64);

/* Measurement hook: vr_render (DVR) that also sets, for every distinct level-L voxel read by a
 * trilinear corner, bit (z*Y_L + y)*X_L + x of voxel_marks[L] (device, N+1 bitmaps of
 * ceil(X_L*Y_L*Z_L/32) words, caller-zeroed), and bit n of node_marks for every node entry the
 * descent reads (global index over all levels, ceil(nodes/32) words).  The counts give the
 * algorithmic bytes a frame must move.  The paper has no counterpart. */
vr_status vr_render_footprint(vr_ctx* ctx, const vr_camera* cams, int n_cams, float* const* images,
                              uint32_t* const* voxel_marks, uint32_t* node_marks, void* cuda_stream);

/* ---- out-of-core rendering (contexts created with cache_capacity_bytes > 0) ----
 * vr_render then reads bricks only from the render cache.  A sample whose brick is missing
 * requests it and uses the nearest resident brick of its parent or grandparent on the descent
 * path, else the node's AVG, requesting those too (full-frame ray casting, Sec. "Full-Frame
 * Ray-Casting").  Every sampled brick is flagged as used.  vr_cache_update then uploads requested
 * bricks, coarser levels first: free slots first, then slots whose brick was not used in the last
 * pass, then (full-frame) used bricks of finer levels than the request (Sec. "Brick Upload from
 * RAM to GPU"); in refinement mode any slot may be replaced.  Inserting data drops the cached
 * copies of every brick the insert changed (Sec. "Incremental Octree Updates on the GPU"). */
typedef struct {
    int64_t requested; /* distinct bricks requested by the passes since the last update */
    int64_t uploaded, evicted, resident, capacity;
} vr_cache_report;
/* Uploads up to max_uploads requested bricks (synchronises the stream) and clears the flags. */
vr_status vr_cache_update(vr_ctx* ctx, int max_uploads, int refinement, void* cuda_stream, vr_cache_report* out);
/* Makes the bricks of the listed nodes resident (dense node numbering: levels 0..N in order,
 * each level's node grid x fastest); nodes without a brick are skipped.  Synchronises. */
vr_status vr_cache_load(vr_ctx* ctx, int64_t n, const int64_t* nodes, void* cuda_stream);
/* Test hook: per node (dense numbering) residency and the used / requested flags of the passes
 * since the last update (host arrays of vr_stats().nodes bytes).  Synchronises. */
vr_status vr_cache_read(vr_ctx* ctx, uint8_t* resident, uint8_t* used, uint8_t* requested, void* cuda_stream);

/* Refinement ray casting (Sec. "Refinement Ray-Casting") of one view into a device image: each
 * pass resumes every unfinished ray from its saved sample and colour and runs it until it ends
 * (pixel written) or reaches a brick that is not resident (request set, state saved).  The
 * caller alternates vr_refine_pass and vr_cache_update(..., refinement = 1, ...) until *pending
 * is 0; the image is then the full-quality render. */
typedef struct vr_refine vr_refine;
vr_status vr_refine_begin(vr_ctx* ctx, const vr_camera* cam, float* image, vr_refine** out);
vr_status vr_refine_pass(vr_refine* r, void* cuda_stream, int64_t* pending, int64_t* samples);
vr_status vr_refine_end(vr_refine* r);

/* Test hook: level L of the volume as out[Z_L][Y_L][X_L][C] (host buffer), gathered from the
 * brick pool (never-touched bricks read as the background).  Synchronises the stream.  Reads back
 * the state the paper defines in Sec. "CPU Data Structure" (level L is the iterated 2x2x2
 * half-sampling of level 0, Eq. 1) so that it can be checked voxel for voxel; not a step of the
 * method.  Errors: VR_ERR_INVALID_ARG (level outside 0..N, NULL out), VR_ERR_DEVICE_ASSERT,
 * VR_ERR_STATE, VR_ERR_CUDA. */
vr_status vr_read_level(vr_ctx* ctx, int level, uint16_t* out, void* cuda_stream);

/* Test hook: values of n level-L voxels, xyz[n][3] (host) -> out[n][C] (host).  Synchronises.
 * Errors: VR_ERR_INVALID_ARG for a coordinate outside level L. */
vr_status vr_read_voxels(vr_ctx* ctx, int level, int64_t n, const int64_t* xyz, uint16_t* out, void* cuda_stream);

/* Test hook: the render record of node (level, i, j, k): flags bit0 has_children, bit1
 * has_brick, bit2 touched; avg[C].  Synchronises.  Errors: VR_ERR_INVALID_ARG outside the grid. */
vr_status vr_read_node(vr_ctx* ctx, int level, int64_t i, int64_t j, int64_t k, uint32_t* flags, uint16_t* avg,
                       void* cuda_stream);

/* Library utility (no counterpart in the paper): sizes of the tree and the pool, and the sample,
 * ray and continued-ray counts of the last vr_render (the work units of the measurement), read
 * from the device: waits for the work queued so far.  Errors: VR_ERR_INVALID_ARG (NULL),
 * VR_ERR_CUDA. */
vr_status vr_stats(vr_ctx* ctx, vr_stats_t* out);

/* Test hook (no counterpart in the paper): writes code (!= 0) into the context's device error
 * word, exactly as a failed device-side check of a kernel would (the kernels never trap; they set
 * this word and return).  The next call that polls the word (vr_read_level, vr_read_voxels,
 * vr_read_node) returns VR_ERR_DEVICE_ASSERT and every later call VR_ERR_STATE, until
 * vr_destroy, which still releases everything.  Lets the error path be tested without a fault.
 * Errors: VR_ERR_INVALID_ARG (NULL context or code 0), VR_ERR_STATE, VR_ERR_CUDA. */
vr_status vr_debug_raise_error(vr_ctx* ctx, int code);

/* Render plan: a fixed batch of views of uneven resolution rendered by ONE persistent launch,
 * captured once into a CUDA graph (queue reset + kernel) and replayed by vr_plan_launch.  The
 * plan owns the per-camera constants; images, the context's brick pool and its transfer
 * functions are read at replay time, so inserts and vr_set_transfer_functions between replays
 * take effect.  mode as in vr_render (| VR_RENDER_FP16).  The launch shape (vr_set_launch_shape)
 * is fixed at creation.  An addition of this library; the paper has no counterpart. */
typedef struct vr_render_plan vr_render_plan;
vr_status vr_plan_create(vr_ctx* ctx, const vr_camera* cams, int n_cams, float* const* images, int mode,
                         vr_render_plan** out);
vr_status vr_plan_launch(vr_render_plan* plan, void* cuda_stream);
/* Samples composited and rays of the last replay (synchronises). */
vr_status vr_plan_samples(vr_render_plan* plan, int64_t* samples, int64_t* rays);
/* Destroys a plan; plans must be destroyed before their context (vr_destroy). */
vr_status vr_plan_destroy(vr_render_plan* plan);

/* Launch shape of the ray caster: warp tile tile_w x tile_h (product 32), threads per CTA (64, 128,
 * 256, 512 or 768) and CTAs per SM of the persistent grid (up to 768 threads are resident per SM).
 * Defaults 8 x 4, 768, 1: one CTA per SM keeps one copy of the transfer-function tables there. */
vr_status vr_set_launch_shape(vr_ctx* ctx, int tile_w, int tile_h, int threads_per_cta, int ctas_per_sm);

/* MIP ray segments (vr_render and render plans in VR_MODE_MIP that read the store directly, no
 * per-channel transforms): with samples = n > 0, the samples k in [j n, (j+1) n) of every ray form
 * segment j, the segments are separate work items (so the longest rays no longer run in one warp
 * each), and a merge takes the per-channel maximum over them before the transfer functions.  A
 * maximum does not round: the image and sample counts are the whole-ray ones bit for bit.  Used
 * when some ray can be longer than one segment; the segment buffers (20 bytes per pixel and
 * segment, 4 per tile and segment) are allocated through the context's allocator on first use.
 * 0 turns segments off; otherwise 4 <= n <= 2^24.  Default 1024.  Not a step of the paper's
 * method: a work decomposition of the MIP ray loop (Sec. "Basic Ray-Casting"). */
vr_status vr_set_mip_segment_length(vr_ctx* ctx, int samples);

/* Order of the ray-tile queue of vr_render for DVR (FP32 or FP16, with or without per-channel
 * transforms or the out-of-core render cache).  0: raster order.  1 (default): when the previous DVR vr_render call of this context
 * had the same tile grid (the same number of views, image sizes and tile shape), its tiles are
 * queued by the SM clock cycles each took there, costliest first (longest-processing-time-first
 * list scheduling in 128 cost classes, four per power of two); the first call of a grid is in
 * raster order.  Early ray termination makes tile costs very uneven, and in raster order a frame
 * ends with a tail in which a few warps finish the longest rays while the rest of the GPU has run
 * out of tiles.  A pixel does not depend on when its tile runs: images and sample counts are the
 * same in either order.  MIP stays in raster order (its rays all run to the end; the cost order
 * measured slower there).  Not part of the paper's method. */
vr_status vr_set_tile_order(vr_ctx* ctx, int mode);

/* How level 0 of an insert reads the block (Sec. "Incremental Construction", step 2: the
 * inserted voxels are copied into the level-0 bricks).  1 (default): the rows of each brick slot's
 * changed planes are staged in shared memory by bulk tensor copies (TMA), one copy per plane,
 * when the block allows it: its base address and its row pitch (extent[0] x channels x 2 bytes)
 * multiples of 16 bytes, and the brick edge small enough for one copy box ((M + 2) x channels + 7
 * elements and M + 2 rows, each at most 256); other blocks take the per-thread loads.  0: always
 * the per-thread loads.  The tree is the same bit for bit either way.  A staged copy that has not
 * landed after about two seconds sets device error bit 4 (read back as VR_ERR_DEVICE_ASSERT by
 * the next call that polls it) instead of waiting forever.  Errors: VR_ERR_INVALID_ARG (NULL
 * context, mode not 0 or 1). */
vr_status vr_set_insert_staging(vr_ctx* ctx, int mode);

/* Ray continuation of vr_render (DVR, FP32 or FP16, reading the store directly with no
 * per-channel transforms).  Early ray termination makes ray lengths very uneven: once the ray-tile
 * queue has run dry, the rest of a frame is a tail in which a few warps march the longest rays
 * while the others idle.  With continuation on, a lane whose ray still has more than
 * min_samples_left segment lengths to go at that point (checked every 16 steps) records the ray's
 * state -- the next sample, transmittance and colour -- and a second launch resumes each recorded
 * ray with lanes_per_ray lanes in lockstep: lane j shades samples k + j, and every lane of the group
 * composites the step's shaded samples in order (the composite is split into a per-sample shading
 * and an in-order ray update; runs of equal samples through brick-less nodes start at the same
 * samples).  Images and sample counts are those of one lane per ray, bit for bit.  The buffers
 * (32 bytes per thread of the render grid) are allocated through the context's allocator on first
 * use.  lanes_per_ray: 0 (off) or 1, 2, 4, 8, 16, 32; min_samples_left >= 0; VR_ERR_INVALID_ARG
 * otherwise.  Defaults 16 and 32.  Not part of the paper's method: a work decomposition of the ray
 * loop of Algorithm 1. */
vr_status vr_set_ray_continuation(vr_ctx* ctx, int lanes_per_ray, int min_samples_left);

/* Ray-tile shape of the render queue: each warp renders tile_w x tile_h pixels (tile_w * tile_h
 * must be 32).  Default 8 x 4.  Chosen per workload by the autotuner of the Python package. */
vr_status vr_set_tile_shape(vr_ctx* ctx, int tile_w, int tile_h);

/* Library utility (no counterpart in the paper): message of the last error of this context (or of
 * the last failed vr_create when ctx is NULL).  The string is owned by the library and valid
 * until the next call on the same context. */
const char* vr_last_error(const vr_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
