// vr_internal.h -- device data layout and kernel launchers shared by the host code (vr_api.cpp)
// and the kernels (vr_insert.cu, vr_render.cu).
//
// HBM layout:
//   pool      brick slots of S^3 voxels, S = M + 2 (one border voxel per side, Sec. "Filtering
//             across Brick Boundaries"); a voxel holds VS uint16 (C channels interleaved, Sec.
//             "Handling Multi-Channel Data"; C = 3 is padded to 4 so that a voxel is one 8-byte
//             load).  Slot position l along an axis holds the level value at
//             clamp(b*M - 1 + l, 0, extent - 1): borders equal the neighbours, clamp-replicated at
//             the real extent, so trilinear filtering never leaves the slot.
//   rnodes    one 16-byte render record per node of the COMPLETE real node grid of every level
//             (dense, x fastest; level offsets noff[L]), so inserts never move entries (the paper's
//             node buffer is also laid out for the complete tree, Sec. "GPU Data Structure").
//   nstat     per node: brick min/max/sum and subtree min/max per channel (homogeneity, AVG).
//   pstat     per slot and interior plane: min/max/sum per channel, so that a slice insert
//             refreshes a brick's statistics without re-reading the brick.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace vrk {

constexpr int MAXL = 16;
constexpr int MAXC = 4;
constexpr int MAXCLIP = 3;

enum : uint32_t { F_CHILDREN = 1u, F_BRICK = 2u, F_TOUCHED = 4u };

struct __align__(16) RNode {
    int32_t slot;   // brick slot (valid when allocated), -1 = none
    uint32_t flags; // F_CHILDREN | F_BRICK | F_TOUCHED
    uint16_t avg[4];
};

struct NStat {
    uint16_t bmin[MAXC], bmax[MAXC], smin[MAXC], smax[MAXC];
    unsigned long long bsum[MAXC];
    long long count;
};

struct PStat {
    uint16_t mn, mx;
    uint32_t sum;
};

struct Geo {
    int C, M, S, N, VS; // channels, brick edge, slot edge, top level, uint16 per voxel
    int pow2;           // M is a power of two
    uint16_t bg, tau;
    long long ldim[MAXL][3];
    long long nb[MAXL][3];
    long long noff[MAXL + 1];
    long long slot_elems; // S^3 * VS
    long long n_slots_cap;
};

// Error word bits set by kernels (never trap).
enum : int { ERR_SLOT_RANGE = 1, ERR_NODE_RANGE = 2, ERR_COPY_TIMEOUT = 4 };

struct SlotInit {
    long long node; // global node index
    int level, slot;
    int bi, bj, bk;
};

struct CamParam {
    float eye[3], ff[3], rr[3], uu[3];
    float kx, ky, dt, ert;
    float tl[MAXL + 1]; // tl[0] = 0, tl[N+1] = +inf
    int W, H, n_clip, tiles_x;
    float clip[MAXCLIP][4];
    float* img;
    const float* dimg; // adjoint input (backward only)
    long long tile_begin;
};

// Out-of-core render cache (Sec. "GPU Data Structure": brick buffer + flag buffer).
struct CacheArgs {
    int* cslot;             // per node: its brick's slot in the render cache, -1 = not resident
    unsigned char* used;    // per node: brick sampled in this pass
    unsigned char* req;     // per node: brick requested in this pass
    const uint16_t* cache;  // render cache slots (same slot layout as the store)
    int refine;             // refinement pass: suspend a ray at its first missing brick
};

struct RefineState { // one pixel of a refinement session
    float C[3], T; // premultiplied colour and transmittance (1 - opacity) so far
    int k;      // next sample index
    int status; // 0 = not started, 1 = suspended, 2 = done
    int pad[2];
};

struct RayCont { // a DVR ray stopped at sample k with transmittance T and colour C, to be resumed
    int ci, px, py, k;
    float T, Cr, Cg, Cb;
};

struct RenderArgs {
    Geo g;
    const uint16_t* pool;
    const RNode* rnodes;
    const float4* tf;    // [C][256][2]: entry, next - entry
    const float* scl;    // [MAXC] s / 65535, then [MAXC] s
    const CamParam* cams;
    int n_cams;
    long long total_tiles;
    int tile_w, tile_h;
    unsigned int* counter;              // tile queue head (reset before each launch)
    unsigned long long* stats;          // [0] samples, [1] rays
    CacheArgs cache;                    // cache.cslot == nullptr: the store is read directly
    RefineState* refine_state;          // MODE 3: per pixel of the single camera
    unsigned int* pending;              // MODE 3: rays still suspended after the pass
    int has_xf;                         // per-channel sample transforms active
    float xf[MAXC][12];                 // channel c samples at xf[c] (3x4, row-major) applied to p
    unsigned int* vmark[MAXL];          // footprint mode: one bit per level-L voxel
    unsigned int* nmark;                // footprint mode: one bit per node
    // MIP ray segments: samples k in [j kseg, (j+1) kseg) of a ray are segment j (nseg == 0: whole rays)
    int kseg, nseg;
    float4* seg_v;                      // [nseg][total_tiles][32] per-channel maxima of the segment
    unsigned int* seg_meta;             // [nseg][total_tiles][32] samples << 2 | 2 when the ray goes on
    unsigned int* seg_done;             // [nseg][total_tiles] 0 pending, 1 done, 3 done and rays go on
    const unsigned int* tile_order;     // queue position -> tile (nullptr: raster order)
    // Ray continuation (plain DVR): once the tile queue runs dry, a lane whose ray has more than
    // cont_min samples left stops, records its state in cont[] and a second launch finishes it
    // with 2^cont_lg lanes per ray.  cont_ctl: [0] queue dry, [1] records, [2] records taken.
    RayCont* cont;                      // nullptr: rays are marched to their end in one launch
    unsigned int* cont_ctl;
    int cont_min, cont_lg;
    unsigned int* tile_cost;            // per tile: SM clock cycles / 64 it took (nullptr: not kept)
    int fwd_img;                        // backward: cams[].img hold the forward's DVR images
    float* dtf;                         // backward: [C][256][4]
    float* dscale;                      // backward: [C]
    double* dacc;                       // backward, FP64 check mode: [C * 1024 + C] sums (zeroed)
    int* err;
};

// ---- launchers (defined in the .cu files) ----
cudaError_t launch_init_nodes(const Geo& g, RNode* rn, NStat* ns, cudaStream_t st);
cudaError_t launch_slot_init(const Geo& g, uint16_t* pool, RNode* rn, PStat* ps, const SlotInit* list, int n,
                             cudaStream_t st);
cudaError_t launch_level_update(const Geo& g, int L, const long long lo[3], const long long hi[3],
                                const uint16_t* block, const long long org[3], const long long ext[3], uint16_t* pool,
                                RNode* rn, NStat* ns, PStat* ps, int* err, cudaStream_t st, bool stage_rows = true);
cudaError_t launch_read_level(const Geo& g, int L, const uint16_t* pool, const RNode* rn, uint16_t* out,
                              cudaStream_t st);
cudaError_t launch_read_voxels(const Geo& g, int L, const uint16_t* pool, const RNode* rn, const long long* xyz,
                               long long n, uint16_t* out, cudaStream_t st);
cudaError_t launch_prepare_tf(int C, const float* tf, const float* scale, float4* tf2, float* scl, cudaStream_t st);
// pdl: launched as a programmatic dependent of the kernel before it on st (vr_render's own chain)
cudaError_t launch_render(const RenderArgs& a, int mode, int fp16, int blocks, int threads, cudaStream_t st,
                          bool pdl = false);
cudaError_t launch_render_backward(const RenderArgs& a, int blocks, int threads, cudaStream_t st);
// the second launch of a continued DVR render: the recorded rays, 2^a.cont_lg lanes each
cudaError_t launch_render_tail(const RenderArgs& a, int fp16, int blocks, int threads, cudaStream_t st,
                               bool pdl = false);
cudaError_t launch_tile_order(const unsigned int* cost, long long tiles, unsigned int* aux, unsigned int* order,
                              cudaStream_t st);
cudaError_t launch_cache_gather(const uint16_t* store, uint16_t* cache, const int2* list, int n, long long slot_elems,
                                cudaStream_t st);

} // namespace vrk
