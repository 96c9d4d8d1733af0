/*
 * oracle.h -- plain, slow FP64 CPU oracle of the multi-channel octree ray
 * caster (Brix, Prassni, Hinrichs: "Visualization of Large Volumetric
 * Multi-Channel Microscopy Data Streams on Standard PCs").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this code; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no source with the CUDA path.
 *
 * What it computes (each function cites the passage it follows):
 *   - volume state: level-0 values (last writer wins, background where never
 *     inserted), the mip levels by iterated round-half-up 2x2x2 means over
 *     in-volume children (Sec. "CPU Data Structure", Eq. 1, "Incremental
 *     Construction" step 2, "Handling Volumes of Arbitrary Dimensions"),
 *     per-node min/max/AVG and the homogeneity flags (same sections, and
 *     "Handling Multi-Channel Data");
 *   - the render of Algorithm 1: per ray, fixed-step march, node at the
 *     screen-space-error level by descent from the root, AVG or trilinear
 *     sample per channel, per-channel transfer function, emission-absorption
 *     compositing inside the channel loop, early ray termination;
 *   - the exact FP64 adjoint of that render with respect to the transfer
 *     function tables and the per-channel intensity scales.
 *
 * Precision: values, interpolation, transfer functions, compositing and
 * gradients are FP64.  Ray GEOMETRY (directions, entry/exit, sample
 * positions, level and node choice) is evaluated in one of two ways:
 *   OR_GEOM_FP64 (or_render, or_render_xf, or_render_check): in double
 *     precision, the definition.  Some decisions are discontinuous -- the
 *     level floor at t_L and the child choice at a split plane -- and a
 *     single-precision implementation may correctly take either branch when
 *     the quantity lies within its rounding error of the threshold.  Such
 *     decisions (whose two branches also sample differently) are flagged;
 *     or_render_check marches every combination of the first OR_MAXFLAG of
 *     them per ray and compares a given pixel with the nearest admissible
 *     result; a ray with more flagged decisions is "unresolved".
 *   OR_GEOM_FP32 (or_render_geo, or_render_cache and the adjoint): in IEEE
 *     single precision in a fixed operation order, mirroring a single-
 *     precision implementation decision for decision (the brick-cache flags
 *     are compared bit for bit; the adjoint is the derivative of the render at
 *     the forward's own decisions).
 * The ERT decision (A >= ert) compares accumulated opacity; every state in
 * the band |A - ert| < OR_ERT_BAND is an admissible stopping state.
 *
 * Parity pins: see tests/test_oracle_*.py (closed forms, hand-computed
 * golden values, invariants, brute force on tiny inputs).
 */
#ifndef VR_ORACLE_H
#define VR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_MAXL 16
#define OR_MAXC 4
#define OR_MAXCAND 4
#define OR_ERT_BAND 2e-4
#define OR_MAXFLAG 3 /* knife-edge decisions enumerated per ray: up to 2^3 variants */
#define OR_GEOM_FP32 0
#define OR_GEOM_FP64 1

typedef struct {
    int64_t dim[3];          /* level-0 extent X, Y, Z */
    int C;                   /* channels */
    int M;                   /* brick interior edge (even) */
    int N;                   /* levels 0..N */
    int64_t ldim[OR_MAXL][3]; /* real extent of level L: ceil(ldim[L-1] / 2) */
    int64_t nb[OR_MAXL][3];   /* node grid of level L: ceil(ldim[L] / M) */
    uint16_t bg;             /* background value of never-inserted voxels */
    uint16_t tau;            /* homogeneity threshold (max - min < tau) */
} or_geom;

typedef struct {
    int touched;      /* some in-volume level-0 voxel of the region was inserted */
    int has_children; /* L > 0 and touched and not subtree-homogeneous */
    int has_brick;    /* touched and not brick-homogeneous */
    int brick_homog, subtree_homog;
    uint16_t avg[OR_MAXC];
    uint16_t bmin[OR_MAXC], bmax[OR_MAXC]; /* over the brick's in-volume level-L voxels */
    uint16_t smin[OR_MAXC], smax[OR_MAXC]; /* over the node's in-volume level-0 voxels */
    int64_t count;                         /* in-volume level-L voxels of the brick */
} or_node;

typedef struct or_volume or_volume;

/* Geometry of the level hierarchy; returns 0 or -1 on invalid arguments. */
int or_geom_init(or_geom* g, const int64_t dim[3], int C, int M, uint16_t bg, uint16_t tau);

/* ---- dense volume: every level held as a flat array ---- */
or_volume* or_dense_create(const int64_t dim[3], int C, int M, uint16_t bg, uint16_t tau);
/* Insert a block (origin, extent) of values [ez][ey][ex][C]; overwrites (last writer wins). */
int or_dense_insert(or_volume* v, const int64_t origin[3], const int64_t extent[3], const uint16_t* block);
/* Recompute levels 1..N and all node records from level 0 and the inserted mask. */
int or_dense_build(or_volume* v, int threads);
/* Level L as [Z_L][Y_L][X_L][C] (pointer valid until destroy). */
const uint16_t* or_dense_level(or_volume* v, int L);

/* ---- lazy volume: level 0 from a generator callback, inserted z-range [z_lo, z_hi);
 *      levels and nodes computed on demand and memoised ---- */
typedef void (*or_gen_fn)(void* user, int64_t x, int64_t y, int64_t z, uint16_t* out);
or_volume* or_lazy_create(const int64_t dim[3], int C, int M, uint16_t bg, uint16_t tau, or_gen_fn gen, void* user,
                          int64_t z_lo, int64_t z_hi);

/* ---- streamed volume: the state of a fully inserted volume whose level 0 is fed once, slab by
 *      slab in z order (slab [nz][Y][X][C], z0 = the next slice), and read back through gen;
 *      levels 1..N and node records are complete after or_stream_finish ---- */
or_volume* or_stream_create(const int64_t dim[3], int C, int M, uint16_t bg, uint16_t tau, or_gen_fn gen, void* user);
int or_stream_feed(or_volume* v, int64_t z0, int64_t nz, const uint16_t* slab, int threads);
int or_stream_finish(or_volume* v, int threads);

void or_volume_destroy(or_volume* v);
const or_geom* or_volume_geom(const or_volume* v);
uint16_t or_value(or_volume* v, int L, int64_t x, int64_t y, int64_t z, int c);
int or_node_info(or_volume* v, int L, int64_t i, int64_t j, int64_t k, or_node* out);

/* ---- render ---- */
typedef struct {
    float eye[3], target[3], up[3];
    float fov_y_deg;
    int width, height;
    float lod_error_px; /* epsilon of the screen-space error, pixels */
    float step_voxels;  /* sampling step, level-0 voxel units */
    float ert_alpha;    /* early ray termination threshold */
    int n_clip;         /* 0..3 half-spaces n.p + d >= 0 */
    float clip[3][4];
} or_camera;

typedef struct {
    int n_cand;                      /* 1..OR_MAXCAND admissible RGBA results */
    double rgba[OR_MAXCAND][4];      /* rgba[0] is the FP64-natural result */
    int64_t samples;                 /* samples composited with the natural decisions */
} or_pixel;

/* Renders the listed pixels with double-precision geometry and the natural branch of every
 * decision.  tf: [C][256][4] (table entries in [0,1]), scale: [C].
 * mode 0 = emission-absorption (Algorithm 1), mode 1 = maximum intensity projection. */
int or_render(or_volume* v, const or_camera* cam, const float* tf, const float* scale, int mode, int64_t n,
              const int32_t* px, const int32_t* py, or_pixel* out, int threads);

/* As or_render, with a per-channel affine sample transform (Sec. "Correction of Chromatic
 * Aberration"): channel c samples the volume at xf[c] * p, xf [C][3][4] (NULL = identity). */
int or_render_xf(or_volume* v, const or_camera* cam, const float* tf, const float* scale, const float* xf, int mode,
                 int64_t n, const int32_t* px, const int32_t* py, or_pixel* out, int threads);
/* As or_render_xf with the geometry chosen: OR_GEOM_FP64 or OR_GEOM_FP32. */
int or_render_geo(or_volume* v, const or_camera* cam, const float* tf, const float* scale, const float* xf, int mode,
                  int geometry, int64_t n, const int32_t* px, const int32_t* py, or_pixel* out, int threads);

/* Parity check of rendered pixels (A16 reading: several results are correct).  For pixel i,
 * err = the smallest max-abs difference between rgba[i] (RGBA, e.g. a GPU image's pixel) and an
 * admissible result: any stopping state within the early-termination band, on any combination of
 * branches of the ray's first OR_MAXFLAG knife-edge decisions (OR_GEOM_FP64; with OR_GEOM_FP32 the
 * mirrored decisions only).  Enumeration of a ray stops once a variant is within stop_err (0:
 * march every variant). */
typedef struct {
    double err;        /* smallest max-abs RGBA difference to an admissible result */
    double rgba[4];    /* natural result */
    int64_t samples;   /* natural sample count */
    int flagged;       /* knife-edge decisions met on the natural march */
    int variants;      /* decision variants marched */
    int unresolved;    /* some march met more than OR_MAXFLAG knife-edge decisions */
} or_check;
/* Knife-edge margins (defaults 8 and 1.5): the bound on the single-precision error of the unit ray
 * direction, in units of 2^-24 per component, and the factor applied to the resulting bounds on
 * the sample parameter and position.  Global; set before rendering. */
void or_set_edge_margins(double dir_ulps, double safety);
int or_render_check(or_volume* v, const or_camera* cam, const float* tf, const float* scale, const float* xf, int mode,
                    int geometry, int64_t n, const int32_t* px, const int32_t* py, const float* rgba, double stop_err,
                    or_check* out, int threads);

int or_render_grad_xf(or_volume* v, const or_camera* cam, const float* tf, const float* scale, const float* xf,
                      int64_t n, const int32_t* px, const int32_t* py, const double* dl, double* dtf, double* dscale,
                      int threads);

/* Algorithmic footprint of one DVR frame of cam (every pixel, single-precision decisions): the
 * number of distinct voxels of each level 0..N read by a trilinear corner of some sample
 * (voxels[L]) and of distinct node entries read on some sample's descent from the root (nodes),
 * over the samples up to the natural early-termination stop.  What a frame must read at least;
 * border duplicates and padding of a brick layout are not part of it. */
int or_render_footprint(or_volume* v, const or_camera* cam, const float* tf, const float* scale, int64_t* voxels,
                        int64_t* nodes, int threads);

/* Full-frame rendering with a partial brick cache (Sec. "Full-Frame Ray-Casting"): resident[n]
 * != 0 when node n's brick is in the render cache (dense numbering of or_node_index).  A sample
 * whose node's brick is missing requests it and uses the nearest present brick of the parent or
 * grandparent on its descent path, else the node's AVG; missing ancestors' bricks are requested
 * too.  used/requested (per node, zeroed by the caller) receive the flags the render sets. */
int or_render_cache(or_volume* v, const or_camera* cam, const float* tf, const float* scale, int mode, int64_t n,
                    const int32_t* px, const int32_t* py, const uint8_t* resident, uint8_t* used, uint8_t* requested,
                    or_pixel* out, int threads);
int64_t or_node_count(const or_geom* g);
int64_t or_node_index(const or_geom* g, int L, int64_t i, int64_t j, int64_t k);

/* As or_render_grad_xf; also marks in ert_edge[n] (optional) the rays whose opacity after some
 * sample up to the stopping one lies within ert_margin of the early-termination threshold: there
 * a single-precision accumulation may stop a sample earlier or later, and the gradient of the ray
 * changes discontinuously (A16 reading for the adjoint). */
int or_render_grad_edges(or_volume* v, const or_camera* cam, const float* tf, const float* scale, const float* xf,
                         int64_t n, const int32_t* px, const int32_t* py, const double* dl, double* dtf,
                         double* dscale, uint8_t* ert_edge, double ert_margin, int threads);

/* Gradient of sum_pixels sum_k dl[p][k] * I[p][k] with respect to tf and scale (FP64 values,
 * single-precision decisions as the forward's, the natural stop).  dl: [n][4].  Outputs are
 * overwritten. */
int or_render_grad(or_volume* v, const or_camera* cam, const float* tf, const float* scale, int64_t n,
                   const int32_t* px, const int32_t* py, const double* dl, double* dtf, double* dscale, int threads);

/* Single steps, exposed for the pins: trilinear value of level L at p (level-0 units),
 * and the transfer-function lookup of intensity I with scale s in one channel's table [256][4]. */
double or_sample_trilinear(or_volume* v, int L, const float p[3], int c);
void or_tf_eval(const float* tf_channel, double s, double I, double rgba[4]);

/* Derived camera quantities, exposed for the tests: ray direction of a pixel,
 * [t0, t1) of its ray, and the level thresholds t_L (L = 1..N). */
int or_ray(const or_geom* g, const or_camera* cam, int px, int py, float dir[3], float* t0, float* t1);
int or_lod_thresholds(const or_geom* g, const or_camera* cam, float* tl /* [N+1], tl[0] = 0 */);

#ifdef __cplusplus
}
#endif
#endif
