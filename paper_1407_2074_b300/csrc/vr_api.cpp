// vr_api.cpp -- host side of libvr: the C ABI declared in include/vr.h.
//
// The host keeps only what it needs to allocate brick slots (a mirror of the slot index of every
// node) and to derive per-camera constants; volume values, node records, homogeneity and images
// live on the device and are produced by the kernels in vr_insert.cu and vr_render.cu.
// Build with -ffp-contract=off: the camera constants below are double-precision expressions whose
// rounding must not depend on FMA contraction (they decide sample levels).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "vr.h"
#include "vr_internal.h"

using namespace vrk;

// Buffers of MIP ray segments (grown on demand; a render plan owns its own).
struct SegBuf {
    float4* v = nullptr;
    unsigned int* meta = nullptr;
    unsigned int* done = nullptr;
    long long cap_entries = 0; // (segment, tile, lane) entries of v and meta
    long long cap_done = 0;    // (segment, tile) flags
};

struct vr_ctx {
    int dev = 0;
    Geo g{};
    vr_options opt{};
    vr_allocator alloc{};
    bool has_alloc = false;
    int sms = 148;
    uint16_t* pool = nullptr;
    RNode* rn = nullptr;
    NStat* ns = nullptr;
    PStat* ps = nullptr;
    int* err = nullptr;
    float4* tf2 = nullptr;
    float* scl = nullptr;
    bool tf_set = false;
    unsigned int* counter = nullptr;
    unsigned long long* stats = nullptr;
    std::vector<int32_t> h_slot;
    long long slots_used = 0;
    uint16_t* stage = nullptr;
    size_t stage_bytes = 0;
    // overlapped host uploads (VR_HOST_ASYNC): two staging buffers filled on the library's own
    // upload stream; stage_free[b] is recorded on the caller's stream once level 0 has read buffer b
    cudaStream_t up_stream = nullptr;
    uint16_t* up_stage[2] = {nullptr, nullptr};
    size_t up_bytes[2] = {0, 0};
    cudaEvent_t stage_free[2] = {nullptr, nullptr};
    cudaEvent_t up_done[2] = {nullptr, nullptr};
    int up_next = 0;
    SlotInit* d_list = nullptr;
    SlotInit* h_list = nullptr;
    int list_cap = 0;
    cudaEvent_t list_ev = nullptr;
    CamParam* d_cams = nullptr;
    CamParam* h_cams = nullptr;
    int cams_cap = 0;
    cudaEvent_t cams_ev = nullptr;
    int n_clip_default = 0;
    float clip_default[VR_MAX_CLIP][4] = {};
    int tile_w = 8, tile_h = 4;
    int threads = 768, ctas_per_sm = 1; // render launch shape (autotuned per workload)
    // tile queue order from the previous render of the same tile grid (costliest tiles first)
    int tile_order_mode = 1;
    int insert_staging = 1; // level 0 of an insert reads the block through TMA-staged rows when it can
    // ray continuation (plain DVR): once the queue runs dry, rays with more than cont_min samples
    // left are finished by a second launch with 2^cont_lg lanes per ray (cont_lg < 0: off)
    int cont_lg = 4;
    int cont_min = 32;
    RayCont* cont = nullptr;
    unsigned int* cont_ctl = nullptr;
    long long cont_cap = 0;
    int kseg_mip = 1024; // MIP: samples per ray segment (0: rays marched whole)
    SegBuf seg;
    unsigned int* lpt_cost = nullptr;
    unsigned int* lpt_order = nullptr;
    unsigned int* lpt_aux = nullptr;
    long long lpt_cap = 0;
    unsigned long long lpt_sig = 0;
    bool lpt_have = false;
    bool last_cont = false;       // the last vr_render continued rays (their number in cont_ctl[1])
    // out-of-core render cache (cache_cap slots; 0 = renders read the store directly)
    long long cache_cap = 0;
    uint16_t* cache = nullptr;
    int* d_cslot = nullptr;
    unsigned char* d_used = nullptr;
    unsigned char* d_req = nullptr;
    std::vector<int> h_cslot;        // node -> cache slot
    std::vector<long long> h_owner;  // cache slot -> node
    std::vector<unsigned char> h_used, h_req;
    std::vector<signed char> node_level;
    int2* d_glist = nullptr;
    int2* h_glist = nullptr;
    int glist_cap = 0;
    bool store_host = false;
    int has_xf = 0;                     // per-channel sample transforms (identity when 0)
    float xf[VR_MAX_CHANNELS][12] = {};
    int grad_fp64 = 0;                  // vr_render_backward: FP64 gradient-check mode
    double* d_gacc = nullptr;           // its double sums [C * 1024 + C]
    bool failed = false;
    std::string msg;
};

static std::string g_create_error;

static vr_status fail(vr_ctx* c, vr_status s, const std::string& m) {
    if (c) {
        c->msg = m;
        if (s == VR_ERR_CUDA || s == VR_ERR_DEVICE_ASSERT) c->failed = true;
    } else {
        g_create_error = m;
    }
    return s;
}

static vr_status cuda_fail(vr_ctx* c, cudaError_t e, const char* where) {
    return fail(c, VR_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(ctx, expr)                                          \
    do {                                                       \
        cudaError_t e_ = (expr);                               \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #expr); \
    } while (0)

static void* dalloc(vr_ctx* c, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (c->has_alloc) return c->alloc.alloc(bytes, c->alloc.user, nullptr);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

static void dfree(vr_ctx* c, void* p) {
    if (!p) return;
    if (c->has_alloc)
        c->alloc.free(p, c->alloc.user, nullptr);
    else
        cudaFree(p);
}

// The tile grid of a call (FNV-1a over the views' sizes and the tile shape): tile costs measured
// by one call order the queue of another only when both have the same grid.
static unsigned long long grid_sig(const vr_ctx* c, const CamParam* cams, int n) {
    unsigned long long sig = 1469598103934665603ull;
    auto mix = [&](long long v) {
        sig ^= (unsigned long long)v;
        sig *= 1099511628211ull;
    };
    mix(n);
    mix(c->tile_w);
    mix(c->tile_h);
    for (int i = 0; i < n; ++i) {
        mix(cams[i].W);
        mix(cams[i].H);
    }
    return sig;
}

// Tile order of a vr_render call: when the previous call had the same tile grid, its measured tile
// costs order the queue (costliest first); this call's costs are kept for the next.
static vr_status order_prepare(vr_ctx* c, RenderArgs& a, const CamParam* cams, int n, long long tiles, cudaStream_t st) {
    if (!c->tile_order_mode) return VR_OK;
    const unsigned long long sig = grid_sig(c, cams, n);
    if (tiles > c->lpt_cap) {
        CK(c, cudaDeviceSynchronize()); // the old buffers may still be in use (any stream)
        dfree(c, c->lpt_cost);
        dfree(c, c->lpt_order);
        dfree(c, c->lpt_aux);
        c->lpt_cap = 0;
        c->lpt_have = false;
        c->lpt_cost = (unsigned int*)dalloc(c, sizeof(unsigned int) * (size_t)tiles);
        c->lpt_order = (unsigned int*)dalloc(c, sizeof(unsigned int) * (size_t)tiles);
        c->lpt_aux = (unsigned int*)dalloc(c, sizeof(unsigned int) * 256);
        if (!c->lpt_cost || !c->lpt_order || !c->lpt_aux) return fail(c, VR_ERR_OUT_OF_MEMORY, "tile order buffers");
        c->lpt_cap = tiles;
    }
    if (c->lpt_have && sig == c->lpt_sig) {
        CK(c, launch_tile_order(c->lpt_cost, tiles, c->lpt_aux, c->lpt_order, st));
        a.tile_order = c->lpt_order;
    }
    a.tile_cost = c->lpt_cost;
    c->lpt_sig = sig;
    c->lpt_have = true;
    return VR_OK;
}

// Ray continuation buffers for a render grid of `lanes` threads (each lane records at most one ray).
static vr_status cont_prepare(vr_ctx* c, RenderArgs& a, long long lanes, cudaStream_t st) {
    if (c->cont_lg < 0) return VR_OK;
    if (lanes > c->cont_cap) {
        CK(c, cudaDeviceSynchronize()); // the old buffers may still be in use (any stream)
        dfree(c, c->cont);
        c->cont_cap = 0;
        c->cont = (RayCont*)dalloc(c, sizeof(RayCont) * (size_t)lanes);
        if (!c->cont_ctl) c->cont_ctl = (unsigned int*)dalloc(c, sizeof(unsigned int) * 4);
        if (!c->cont || !c->cont_ctl) return fail(c, VR_ERR_OUT_OF_MEMORY, "ray continuation buffers");
        c->cont_cap = lanes;
    }
    CK(c, cudaMemsetAsync(c->cont_ctl, 0, sizeof(unsigned int) * 4, st));
    a.cont = c->cont;
    a.cont_ctl = c->cont_ctl;
    a.cont_min = c->cont_min;
    a.cont_lg = c->cont_lg;
    return VR_OK;
}

static void seg_free(vr_ctx* c, SegBuf& b) {
    dfree(c, b.v);
    dfree(c, b.meta);
    dfree(c, b.done);
    b = SegBuf();
}

// MIP segments for these cameras (a ray inside the volume box is at most its diagonal long); fills
// the segment fields of `a` and grows `b`, or leaves nseg = 0 when every ray fits one segment.
static vr_status seg_prepare(vr_ctx* c, SegBuf& b, RenderArgs& a, const CamParam* cams, int n, long long tiles,
                             cudaStream_t st) {
    a.nseg = 0;
    if (c->kseg_mip <= 0 || a.cache.cslot || a.has_xf) return VR_OK;
    const double dx = (double)c->g.ldim[0][0], dy = (double)c->g.ldim[0][1], dz = (double)c->g.ldim[0][2];
    const double diag = std::sqrt(dx * dx + dy * dy + dz * dz);
    long long ns = 0;
    for (int i = 0; i < n; ++i) {
        double k = std::ceil(diag / (double)cams[i].dt) + 2.0;
        if (k > (double)(1 << 24)) k = (double)(1 << 24);
        ns = std::max(ns, ((long long)k + c->kseg_mip - 1) / c->kseg_mip);
    }
    if (ns <= 1 || ns * tiles >= 0xffffffffLL) return VR_OK;
    const long long entries = ns * tiles * 32, done = ns * tiles;
    if (entries > b.cap_entries || done > b.cap_done) {
        CK(c, cudaDeviceSynchronize()); // the old buffers may still be in use (any stream)
        seg_free(c, b);
        b.v = (float4*)dalloc(c, sizeof(float4) * (size_t)entries);
        b.meta = (unsigned int*)dalloc(c, sizeof(unsigned int) * (size_t)entries);
        b.done = (unsigned int*)dalloc(c, sizeof(unsigned int) * (size_t)done);
        if (!b.v || !b.meta || !b.done) {
            seg_free(c, b);
            return fail(c, VR_ERR_OUT_OF_MEMORY, "ray segment buffers");
        }
        b.cap_entries = entries;
        b.cap_done = done;
    }
    a.kseg = c->kseg_mip;
    a.nseg = (int)ns;
    a.seg_v = b.v;
    a.seg_meta = b.meta;
    a.seg_done = b.done;
    return VR_OK;
}

static void destroy_all(vr_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->dev);
    cudaDeviceSynchronize();
    seg_free(c, c->seg);
    dfree(c, c->lpt_cost);
    dfree(c, c->lpt_order);
    dfree(c, c->lpt_aux);
    dfree(c, c->cont);
    dfree(c, c->cont_ctl);
    if (c->store_host) {
        if (c->pool) cudaFreeHost(c->pool);
    } else {
        dfree(c, c->pool);
    }
    dfree(c, c->cache);
    dfree(c, c->d_cslot);
    dfree(c, c->d_used);
    dfree(c, c->d_req);
    dfree(c, c->d_glist);
    if (c->h_glist) cudaFreeHost(c->h_glist);
    dfree(c, c->rn);
    dfree(c, c->ns);
    dfree(c, c->ps);
    dfree(c, c->err);
    dfree(c, c->tf2);
    dfree(c, c->scl);
    dfree(c, c->counter);
    dfree(c, c->stats);
    dfree(c, c->stage);
    if (c->up_stream) cudaStreamSynchronize(c->up_stream);
    for (int b = 0; b < 2; ++b) {
        dfree(c, c->up_stage[b]);
        if (c->stage_free[b]) cudaEventDestroy(c->stage_free[b]);
        if (c->up_done[b]) cudaEventDestroy(c->up_done[b]);
    }
    if (c->up_stream) cudaStreamDestroy(c->up_stream);
    dfree(c, c->d_list);
    dfree(c, c->d_gacc);
    dfree(c, c->d_cams);
    if (c->h_list) cudaFreeHost(c->h_list);
    if (c->h_cams) cudaFreeHost(c->h_cams);
    if (c->list_ev) cudaEventDestroy(c->list_ev);
    if (c->cams_ev) cudaEventDestroy(c->cams_ev);
    delete c;
}

extern "C" {

vr_status vr_create(const int64_t dims[3], int channels, int brick_size, const vr_options* opts,
                    const vr_allocator* alloc, vr_ctx** out) {
    if (!out) return fail(nullptr, VR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!dims) return fail(nullptr, VR_ERR_INVALID_ARG, "dims is NULL");
    for (int a = 0; a < 3; ++a)
        if (dims[a] <= 0 || dims[a] >= (1 << 21)) return fail(nullptr, VR_ERR_INVALID_ARG, "dims must be in 1..2^21-1");
    if (channels < 1 || channels > VR_MAX_CHANNELS) return fail(nullptr, VR_ERR_INVALID_ARG, "channels must be 1..4");
    if (brick_size < 4 || brick_size > 128 || (brick_size & 1))
        return fail(nullptr, VR_ERR_INVALID_ARG, "brick_size must be even and in 4..128");
    if (alloc && (!alloc->alloc || !alloc->free)) return fail(nullptr, VR_ERR_INVALID_ARG, "allocator incomplete");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    int ndev = 0;
    if (e != cudaSuccess || cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(nullptr, VR_ERR_CUDA, "no CUDA device");
    }
    vr_ctx* c = new vr_ctx();
    c->dev = dev;
    if (opts) c->opt = *opts;
    if (c->opt.precision != VR_FP32 && c->opt.precision != VR_FP16_INTERP) {
        delete c;
        return fail(nullptr, VR_ERR_INVALID_ARG, "unknown precision");
    }
    if (alloc) {
        c->alloc = *alloc;
        c->has_alloc = true;
    }
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);
    Geo& g = c->g;
    g.C = channels;
    g.M = brick_size;
    g.S = brick_size + 2;
    g.VS = channels == 1 ? 1 : (channels == 2 ? 2 : 4);
    g.pow2 = (brick_size & (brick_size - 1)) == 0;
    g.bg = c->opt.background;
    g.tau = c->opt.homog_threshold;
    long long nbmax = 1;
    for (int a = 0; a < 3; ++a) nbmax = std::max<long long>(nbmax, (dims[a] + brick_size - 1) / brick_size);
    int N = 0;
    while ((1LL << N) < nbmax) ++N;
    if (N + 1 > MAXL) {
        delete c;
        return fail(nullptr, VR_ERR_INVALID_ARG, "too many levels");
    }
    g.N = N;
    for (int a = 0; a < 3; ++a) g.ldim[0][a] = dims[a];
    for (int L = 1; L <= N; ++L)
        for (int a = 0; a < 3; ++a) g.ldim[L][a] = (g.ldim[L - 1][a] + 1) / 2;
    long long nodes = 0, full_slots = 0;
    for (int L = 0; L <= N; ++L) {
        for (int a = 0; a < 3; ++a) g.nb[L][a] = (g.ldim[L][a] + brick_size - 1) / brick_size;
        g.noff[L] = nodes;
        nodes += g.nb[L][0] * g.nb[L][1] * g.nb[L][2];
    }
    g.noff[N + 1] = nodes;
    full_slots = nodes;
    g.slot_elems = (long long)g.S * g.S * g.S * g.VS;
    const long long slot_bytes = g.slot_elems * 2;
    long long cap = full_slots;
    if (c->opt.pool_capacity_bytes > 0) cap = std::min<long long>(full_slots, (long long)(c->opt.pool_capacity_bytes / slot_bytes));
    if (cap < 1) {
        delete c;
        return fail(nullptr, VR_ERR_INVALID_ARG, "pool capacity below one brick");
    }
    g.n_slots_cap = cap;
    c->h_slot.assign((size_t)nodes, -1);
    if (c->opt.store_on_host) {
        c->store_host = true;
        void* hp = nullptr;
        if (cudaHostAlloc(&hp, (size_t)(cap * slot_bytes), cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            hp = nullptr;
        }
        void* dp = nullptr;
        if (hp && cudaHostGetDevicePointer(&dp, hp, 0) != cudaSuccess) {
            cudaGetLastError();
            dp = nullptr;
        }
        if (hp && dp != hp) { // unified addressing is expected on this platform
            cudaFreeHost(hp);
            hp = nullptr;
        }
        c->pool = (uint16_t*)hp;
    } else {
        c->pool = (uint16_t*)dalloc(c, (size_t)(cap * slot_bytes));
    }
    if (c->opt.cache_capacity_bytes > 0) {
        c->cache_cap = std::min<long long>(full_slots, (long long)(c->opt.cache_capacity_bytes / slot_bytes));
        if (c->cache_cap < 1) c->cache_cap = 1;
        c->cache = (uint16_t*)dalloc(c, (size_t)(c->cache_cap * slot_bytes));
        c->d_cslot = (int*)dalloc(c, sizeof(int) * (size_t)nodes);
        c->d_used = (unsigned char*)dalloc(c, (size_t)nodes);
        c->d_req = (unsigned char*)dalloc(c, (size_t)nodes);
        if (!c->cache || !c->d_cslot || !c->d_used || !c->d_req) {
            destroy_all(c);
            return fail(nullptr, VR_ERR_OUT_OF_MEMORY, "render cache allocation failed");
        }
        cudaMemset(c->d_cslot, 0xff, sizeof(int) * (size_t)nodes);
        cudaMemset(c->d_used, 0, (size_t)nodes);
        cudaMemset(c->d_req, 0, (size_t)nodes);
        c->h_cslot.assign((size_t)nodes, -1);
        c->h_owner.assign((size_t)c->cache_cap, -1);
        c->h_used.assign((size_t)nodes, 0);
        c->h_req.assign((size_t)nodes, 0);
        c->node_level.assign((size_t)nodes, 0);
        for (int L = 0; L <= N; ++L)
            for (long long n = g.noff[L]; n < g.noff[L + 1]; ++n) c->node_level[(size_t)n] = (signed char)L;
    }
    c->rn = (RNode*)dalloc(c, sizeof(RNode) * (size_t)nodes);
    c->ns = (NStat*)dalloc(c, sizeof(NStat) * (size_t)nodes);
    c->ps = (PStat*)dalloc(c, sizeof(PStat) * (size_t)(cap * brick_size * channels));
    c->err = (int*)dalloc(c, sizeof(int));
    c->tf2 = (float4*)dalloc(c, sizeof(float4) * 512 * channels);
    c->scl = (float*)dalloc(c, sizeof(float) * 2 * MAXC);
    c->counter = (unsigned int*)dalloc(c, sizeof(unsigned int) * 4);
    c->stats = (unsigned long long*)dalloc(c, sizeof(unsigned long long) * 4);
    if (!c->pool || !c->rn || !c->ns || !c->ps || !c->err || !c->tf2 || !c->scl || !c->counter || !c->stats) {
        destroy_all(c);
        return fail(nullptr, VR_ERR_OUT_OF_MEMORY, "device allocation failed");
    }
    if (cudaEventCreateWithFlags(&c->list_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->cams_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->stage_free[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->stage_free[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->up_done[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->up_done[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->up_stream, cudaStreamNonBlocking) != cudaSuccess) {
        destroy_all(c);
        return fail(nullptr, VR_ERR_CUDA, "event creation failed");
    }
    cudaMemset(c->err, 0, sizeof(int));
    cudaMemset(c->stats, 0, sizeof(unsigned long long) * 4);
    e = launch_init_nodes(g, c->rn, c->ns, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        std::string m = std::string("init: ") + cudaGetErrorString(e);
        destroy_all(c);
        return fail(nullptr, VR_ERR_CUDA, m);
    }
    *out = c;
    return VR_OK;
}

vr_status vr_destroy(vr_ctx* c) {
    if (!c) return VR_ERR_INVALID_ARG;
    destroy_all(c);
    return VR_OK;
}

static vr_status check_ctx(vr_ctx* c) {
    if (!c) return VR_ERR_INVALID_ARG;
    if (c->failed) return fail(c, VR_ERR_STATE, "context failed earlier: " + c->msg);
    cudaSetDevice(c->dev);
    return VR_OK;
}

static long long ceil_div(long long a, long long b) { return (a + b - 1) / b; }

vr_status vr_insert_block(vr_ctx* c, const int64_t origin[3], const int64_t extent[3], const uint16_t* block,
                          int on_device, void* stream) {
    vr_status s = check_ctx(c);
    if (s != VR_OK) return s;
    if (!origin || !extent || !block) return fail(c, VR_ERR_INVALID_ARG, "NULL argument");
    if (on_device != VR_HOST_BLOCK && on_device != VR_DEVICE_BLOCK && on_device != VR_HOST_ASYNC)
        return fail(c, VR_ERR_INVALID_ARG, "on_device must be VR_HOST_BLOCK, VR_DEVICE_BLOCK or VR_HOST_ASYNC");
    const Geo& g = c->g;
    for (int a = 0; a < 3; ++a)
        if (origin[a] < 0 || extent[a] <= 0 || origin[a] + extent[a] > g.ldim[0][a])
            return fail(c, VR_ERR_INVALID_ARG, "block outside the volume");
    cudaStream_t st = (cudaStream_t)stream;
    // slots for every brick whose interior the block reaches, on every level (step 1: nodes and
    // bricks on the insertion path are created); count first so that a full pool changes nothing
    long long lo[MAXL][3], hi[MAXL][3];
    long long need = 0;
    for (int L = 0; L <= g.N; ++L) {
        for (int a = 0; a < 3; ++a) {
            lo[L][a] = origin[a] >> L;
            hi[L][a] = (origin[a] + extent[a] - 1) >> L;
        }
        for (long long k = lo[L][2] / g.M; k <= hi[L][2] / g.M; ++k)
            for (long long j = lo[L][1] / g.M; j <= hi[L][1] / g.M; ++j)
                for (long long i = lo[L][0] / g.M; i <= hi[L][0] / g.M; ++i)
                    if (c->h_slot[(size_t)(g.noff[L] + (k * g.nb[L][1] + j) * g.nb[L][0] + i)] < 0) ++need;
    }
    if (c->slots_used + need > g.n_slots_cap) return fail(c, VR_ERR_OUT_OF_MEMORY, "brick pool exhausted");
    // stage host data
    const uint16_t* src = block;
    const size_t bytes = (size_t)extent[0] * extent[1] * extent[2] * g.C * sizeof(uint16_t);
    int up = -1; // staging buffer of an overlapped upload
    if (on_device == VR_HOST_ASYNC) {
        // the copy waits only until level 0 of the insert before last has read this buffer, not
        // for earlier work on the caller's stream; the caller's stream waits for the copy
        up = c->up_next;
        c->up_next ^= 1;
        if (bytes > c->up_bytes[up]) {
            CK(c, cudaEventSynchronize(c->stage_free[up]));
            CK(c, cudaStreamSynchronize(c->up_stream));
            dfree(c, c->up_stage[up]);
            c->up_stage[up] = (uint16_t*)dalloc(c, bytes);
            c->up_bytes[up] = c->up_stage[up] ? bytes : 0;
            if (!c->up_stage[up]) return fail(c, VR_ERR_OUT_OF_MEMORY, "staging allocation failed");
        }
        CK(c, cudaStreamWaitEvent(c->up_stream, c->stage_free[up], 0));
        CK(c, cudaMemcpyAsync(c->up_stage[up], block, bytes, cudaMemcpyHostToDevice, c->up_stream));
        CK(c, cudaEventRecord(c->up_done[up], c->up_stream));
        CK(c, cudaStreamWaitEvent(st, c->up_done[up], 0));
        src = c->up_stage[up];
    } else if (!on_device) {
        if (bytes > c->stage_bytes) {
            CK(c, cudaStreamSynchronize(st));
            dfree(c, c->stage);
            c->stage = (uint16_t*)dalloc(c, bytes);
            c->stage_bytes = c->stage ? bytes : 0;
            if (!c->stage) return fail(c, VR_ERR_OUT_OF_MEMORY, "staging allocation failed");
        }
        CK(c, cudaMemcpyAsync(c->stage, block, bytes, cudaMemcpyHostToDevice, st));
        src = c->stage;
    }
    if (need > 0) {
        if (need > c->list_cap) {
            CK(c, cudaEventSynchronize(c->list_ev));
            CK(c, cudaStreamSynchronize(st));
            dfree(c, c->d_list);
            if (c->h_list) cudaFreeHost(c->h_list);
            c->h_list = nullptr;
            int cap = (int)std::max<long long>(need, 4096);
            c->d_list = (SlotInit*)dalloc(c, sizeof(SlotInit) * (size_t)cap);
            if (!c->d_list || cudaMallocHost(&c->h_list, sizeof(SlotInit) * (size_t)cap) != cudaSuccess) {
                c->list_cap = 0;
                return fail(c, VR_ERR_OUT_OF_MEMORY, "slot list allocation failed");
            }
            c->list_cap = cap;
        }
        CK(c, cudaEventSynchronize(c->list_ev));
        int n = 0;
        for (int L = 0; L <= g.N; ++L)
            for (long long k = lo[L][2] / g.M; k <= hi[L][2] / g.M; ++k)
                for (long long j = lo[L][1] / g.M; j <= hi[L][1] / g.M; ++j)
                    for (long long i = lo[L][0] / g.M; i <= hi[L][0] / g.M; ++i) {
                        long long nid = g.noff[L] + (k * g.nb[L][1] + j) * g.nb[L][0] + i;
                        if (c->h_slot[(size_t)nid] >= 0) continue;
                        int slot = (int)c->slots_used++;
                        c->h_slot[(size_t)nid] = slot;
                        c->h_list[n++] = SlotInit{nid, L, slot, (int)i, (int)j, (int)k};
                    }
        CK(c, cudaMemcpyAsync(c->d_list, c->h_list, sizeof(SlotInit) * (size_t)n, cudaMemcpyHostToDevice, st));
        CK(c, cudaEventRecord(c->list_ev, st));
        CK(c, launch_slot_init(g, c->pool, c->rn, c->ps, c->d_list, n, st));
    }
    const long long org[3] = {origin[0], origin[1], origin[2]}, ext[3] = {extent[0], extent[1], extent[2]};
    // one launch per level, 0 .. N: each level reads the one below (step 2 of the construction).
    // Levels 2 .. N in one launch, each parent updated by the CTA finishing its last child slot,
    // measured slower (228 vs 84 us on the 24 GiB workload): a CTA that completes several parents
    // updates them one after another, and one slot's update already takes ~13 us.
    for (int L = 0; L <= g.N; ++L) {
        CK(c, launch_level_update(g, L, lo[L], hi[L], src, org, ext, c->pool, c->rn, c->ns, c->ps, c->err, st,
                                  c->insert_staging != 0));
        if (L == 0 && up >= 0) CK(c, cudaEventRecord(c->stage_free[up], st));
    }
    if (c->cache_cap > 0) {
        // cached copies of every brick this insert rewrote (interior or border) are stale now
        bool dropped = false;
        for (int L = 0; L <= g.N; ++L) {
            long long b0[3], b1[3];
            for (int a = 0; a < 3; ++a) {
                b0[a] = std::max<long long>(0, (lo[L][a] + g.M - 1) / g.M - 1);
                b1[a] = std::min<long long>(g.nb[L][a] - 1, (hi[L][a] + 1) / g.M);
            }
            for (long long k = b0[2]; k <= b1[2]; ++k)
                for (long long j = b0[1]; j <= b1[1]; ++j)
                    for (long long i = b0[0]; i <= b1[0]; ++i) {
                        const size_t nid = (size_t)(g.noff[L] + (k * g.nb[L][1] + j) * g.nb[L][0] + i);
                        const int cs = c->h_cslot[nid];
                        if (cs >= 0) {
                            c->h_owner[(size_t)cs] = -1;
                            c->h_cslot[nid] = -1;
                            dropped = true;
                        }
                    }
        }
        if (dropped)
            CK(c, cudaMemcpyAsync(c->d_cslot, c->h_cslot.data(), sizeof(int) * c->h_cslot.size(), cudaMemcpyHostToDevice,
                                  st));
    }
    return VR_OK;
}

vr_status vr_insert_slice(vr_ctx* c, int64_t z, const uint16_t* slice, int on_device, void* stream) {
    if (!c) return VR_ERR_INVALID_ARG;
    if (z < 0 || z >= c->g.ldim[0][2]) return fail(c, VR_ERR_INVALID_ARG, "slice z outside the volume");
    const int64_t o[3] = {0, 0, z}, e[3] = {c->g.ldim[0][0], c->g.ldim[0][1], 1};
    return vr_insert_block(c, o, e, slice, on_device, stream);
}

vr_status vr_set_transfer_functions(vr_ctx* c, const float* tf, const float* scale, void* stream) {
    vr_status s = check_ctx(c);
    if (s != VR_OK) return s;
    if (!tf || !scale) return fail(c, VR_ERR_INVALID_ARG, "NULL transfer function or scale");
    CK(c, launch_prepare_tf(c->g.C, tf, scale, c->tf2, c->scl, (cudaStream_t)stream));
    c->tf_set = true;
    return VR_OK;
}

vr_status vr_set_channel_transforms(vr_ctx* c, const float* m) {
    vr_status s = check_ctx(c);
    if (s != VR_OK) return s;
    if (!m) {
        c->has_xf = 0;
        return VR_OK;
    }
    bool identity = true;
    for (int ch = 0; ch < c->g.C; ++ch)
        for (int q = 0; q < 12; ++q) {
            const float v = m[12 * ch + q];
            if (!std::isfinite(v)) return fail(c, VR_ERR_INVALID_ARG, "non-finite transform");
            c->xf[ch][q] = v;
            const float id = (q == 0 || q == 5 || q == 10) ? 1.0f : 0.0f;
            if (v != id) identity = false;
        }
    c->has_xf = identity ? 0 : 1;
    return VR_OK;
}

vr_status vr_set_clip_planes(vr_ctx* c, int n, const float* planes) {
    vr_status s = check_ctx(c);
    if (s != VR_OK) return s;
    if (n < 0 || n > VR_MAX_CLIP || (n > 0 && !planes)) return fail(c, VR_ERR_INVALID_ARG, "bad clip planes");
    c->n_clip_default = n;
    for (int i = 0; i < n; ++i)
        for (int q = 0; q < 4; ++q) c->clip_default[i][q] = planes[4 * i + q];
    return VR_OK;
}

// Per-camera constants.  The expressions and their evaluation order are part of the
// contract: sample levels and sample positions depend on their rounding.
static bool derive_camera(const vr_ctx* c, const vr_camera& cam, CamParam& cp) {
    if (cam.width <= 0 || cam.height <= 0 || !(cam.step_voxels >= 1e-3f) || !(cam.lod_error_px > 0.0f) ||
        !(cam.fov_y_deg > 0.0f && cam.fov_y_deg < 180.0f) || cam.n_clip < -1 || cam.n_clip > VR_MAX_CLIP)
        return false;
    const Geo& g = c->g;
    const double th = std::tan(((double)cam.fov_y_deg * M_PI) / 360.0);
    double f[3], r[3], u[3], up[3];
    for (int a = 0; a < 3; ++a) {
        f[a] = (double)cam.target[a] - (double)cam.eye[a];
        up[a] = (double)cam.up[a];
    }
    const double nf = std::sqrt((f[0] * f[0] + f[1] * f[1]) + f[2] * f[2]);
    if (!(nf > 0.0)) return false;
    for (int a = 0; a < 3; ++a) f[a] = f[a] / nf;
    r[0] = f[1] * up[2] - f[2] * up[1];
    r[1] = f[2] * up[0] - f[0] * up[2];
    r[2] = f[0] * up[1] - f[1] * up[0];
    const double nr = std::sqrt((r[0] * r[0] + r[1] * r[1]) + r[2] * r[2]);
    if (!(nr > 0.0)) return false;
    for (int a = 0; a < 3; ++a) r[a] = r[a] / nr;
    u[0] = r[1] * f[2] - r[2] * f[1];
    u[1] = r[2] * f[0] - r[0] * f[2];
    u[2] = r[0] * f[1] - r[1] * f[0];
    for (int a = 0; a < 3; ++a) {
        cp.eye[a] = cam.eye[a];
        cp.ff[a] = (float)f[a];
        cp.rr[a] = (float)r[a];
        cp.uu[a] = (float)u[a];
    }
    cp.kx = (float)((th * (double)cam.width) / (double)cam.height);
    cp.ky = (float)th;
    cp.dt = cam.step_voxels;
    cp.ert = cam.ert_alpha;
    for (int L = 0; L <= MAXL; ++L) cp.tl[L] = INFINITY;
    cp.tl[0] = 0.0f;
    for (int L = 1; L <= g.N; ++L)
        cp.tl[L] = (float)(std::ldexp((double)cam.height, L) / ((2.0 * (double)cam.lod_error_px) * th));
    cp.W = cam.width;
    cp.H = cam.height;
    const int nc = cam.n_clip < 0 ? c->n_clip_default : cam.n_clip;
    cp.n_clip = nc;
    for (int i = 0; i < VR_MAX_CLIP; ++i)
        for (int q = 0; q < 4; ++q) cp.clip[i][q] = (i < nc) ? (cam.n_clip < 0 ? c->clip_default[i][q] : cam.clip[i][q]) : 0.0f;
    return true;
}

static vr_status prepare_cams(vr_ctx* c, const vr_camera* cams, int n, float* const* imgs, const float* const* dimgs,
                              cudaStream_t st, long long* total_tiles) {
    if (n > c->cams_cap) {
        CK(c, cudaEventSynchronize(c->cams_ev));
        CK(c, cudaStreamSynchronize(st));
        dfree(c, c->d_cams);
        if (c->h_cams) cudaFreeHost(c->h_cams);
        c->h_cams = nullptr;
        int cap = std::max(n, 64);
        c->d_cams = (CamParam*)dalloc(c, sizeof(CamParam) * (size_t)cap);
        if (!c->d_cams || cudaMallocHost(&c->h_cams, sizeof(CamParam) * (size_t)cap) != cudaSuccess) {
            c->cams_cap = 0;
            return fail(c, VR_ERR_OUT_OF_MEMORY, "camera buffer allocation failed");
        }
        c->cams_cap = cap;
    }
    CK(c, cudaEventSynchronize(c->cams_ev));
    long long tiles = 0;
    for (int i = 0; i < n; ++i) {
        CamParam& cp = c->h_cams[i];
        std::memset(&cp, 0, sizeof cp);
        if (!derive_camera(c, cams[i], cp)) return fail(c, VR_ERR_INVALID_ARG, "invalid camera " + std::to_string(i));
        if (imgs) {
            if (!imgs[i]) return fail(c, VR_ERR_INVALID_ARG, "NULL image");
            cp.img = imgs[i];
        }
        if (dimgs) {
            if (!dimgs[i]) return fail(c, VR_ERR_INVALID_ARG, "NULL image gradient");
            cp.dimg = dimgs[i];
        }
        cp.tiles_x = (int)ceil_div(cp.W, c->tile_w);
        cp.tile_begin = tiles;
        tiles += (long long)cp.tiles_x * ceil_div(cp.H, c->tile_h);
    }
    if (tiles >= 0xffffffffLL) return fail(c, VR_ERR_INVALID_ARG, "too many pixels in one call");
    CK(c, cudaMemcpyAsync(c->d_cams, c->h_cams, sizeof(CamParam) * (size_t)n, cudaMemcpyHostToDevice, st));
    CK(c, cudaEventRecord(c->cams_ev, st));
    *total_tiles = tiles;
    return VR_OK;
}

static RenderArgs make_args(vr_ctx* c, int n, long long tiles) {
    RenderArgs a;
    std::memset(&a, 0, sizeof a);
    a.g = c->g;
    a.pool = c->pool;
    a.rnodes = c->rn;
    a.tf = c->tf2;
    a.scl = c->scl;
    a.cams = c->d_cams;
    a.n_cams = n;
    a.total_tiles = tiles;
    a.tile_w = c->tile_w;
    a.tile_h = c->tile_h;
    a.counter = c->counter;
    a.stats = c->stats;
    a.err = c->err;
    a.has_xf = c->has_xf;
    std::memcpy(a.xf, c->xf, sizeof a.xf);
    if (c->cache_cap > 0) {
        a.cache.cslot = c->d_cslot;
        a.cache.used = c->d_used;
        a.cache.req = c->d_req;
        a.cache.cache = c->cache;
        a.cache.refine = 0;
    }
    return a;
}

static int grid_for(vr_ctx* c, long long tiles, int threads, int per_sm) {
    long long warps = tiles, per_block = threads / 32;
    long long need = (warps + per_block - 1) / per_block;
    long long maxb = (long long)c->sms * per_sm;
    if (need > maxb) need = maxb;
    return (int)(need < 1 ? 1 : need);
}

vr_status vr_render(vr_ctx* c, const vr_camera* cams, int n, float* const* images, int mode, void* stream) {
    vr_status s = check_ctx(c);
    if (s != VR_OK) return s;
    if (!cams || n <= 0 || !images) return fail(c, VR_ERR_INVALID_ARG, "no cameras or images");
    const int fp16 = (mode & VR_RENDER_FP16) || c->opt.precision == VR_FP16_INTERP;
    mode &= ~VR_RENDER_FP16;
    if (mode != VR_MODE_DVR && mode != VR_MODE_MIP) return fail(c, VR_ERR_INVALID_ARG, "unknown mode");
    if (!c->tf_set) return fail(c, VR_ERR_INVALID_ARG, "transfer functions not set");
    cudaStream_t st = (cudaStream_t)stream;
    long long tiles = 0;
    s = prepare_cams(c, cams, n, images, nullptr, st, &tiles);
    if (s != VR_OK) return s;
    CK(c, cudaMemsetAsync(c->counter, 0, sizeof(unsigned long long), st));
    CK(c, cudaMemsetAsync(c->stats, 0, 2 * sizeof(unsigned long long), st));
    RenderArgs a = make_args(c, n, tiles);
    const int blocks = grid_for(c, tiles, c->threads, c->ctas_per_sm);
    const bool cont = mode == VR_MODE_DVR && !a.has_xf && !a.cache.cslot && c->cont_lg >= 0;
    if (cont) { // before the tile order: its reset is no kernel, and the kernels below form one chain
        s = cont_prepare(c, a, (long long)blocks * c->threads, st);
        if (s != VR_OK) return s;
    }
    if (mode == VR_MODE_DVR) { // whole-ray, per-channel-transform and render-cache passes alike
        s = order_prepare(c, a, c->h_cams, n, tiles, st);
        if (s != VR_OK) return s;
    }
    if (mode == VR_MODE_MIP) {
        s = seg_prepare(c, c->seg, a, c->h_cams, n, tiles, st);
        if (s != VR_OK) return s;
    }
    // the tile-order scatter, the ray caster and the continuation as programmatic dependents, each
    // of the kernel before it
    CK(c, launch_render(a, mode, fp16 && mode == VR_MODE_DVR, blocks, c->threads, st, true));
    if (cont) CK(c, launch_render_tail(a, fp16, blocks, c->threads, st, true));
    c->last_cont = cont;
    return VR_OK;
}

static vr_status render_backward(vr_ctx* c, const vr_camera* cams, int n, const float* const* images,
                                 const float* const* dl, float* dtf, float* dscale, void* stream) {
    vr_status s = check_ctx(c);
    if (s != VR_OK) return s;
    if (!cams || n <= 0 || !dl || !dtf || !dscale) return fail(c, VR_ERR_INVALID_ARG, "NULL argument");
    if (!c->tf_set) return fail(c, VR_ERR_INVALID_ARG, "transfer functions not set");
    cudaStream_t st = (cudaStream_t)stream;
    long long tiles = 0;
    s = prepare_cams(c, cams, n, const_cast<float* const*>(images), dl, st, &tiles);
    if (s != VR_OK) return s;
    CK(c, cudaMemsetAsync(dtf, 0, sizeof(float) * 1024 * c->g.C, st));
    CK(c, cudaMemsetAsync(dscale, 0, sizeof(float) * c->g.C, st));
    CK(c, cudaMemsetAsync(c->counter, 0, sizeof(unsigned long long), st));
    RenderArgs a = make_args(c, n, tiles);
    a.stats = nullptr;
    a.dtf = dtf;
    a.dscale = dscale;
    a.fwd_img = images != nullptr && !c->grad_fp64;
    if (c->grad_fp64) {
        const size_t nb = sizeof(double) * (size_t)(c->g.C * 1024 + c->g.C);
        if (!c->d_gacc) {
            c->d_gacc = (double*)dalloc(c, nb);
            if (!c->d_gacc) return fail(c, VR_ERR_OUT_OF_MEMORY, "FP64 gradient buffer");
        }
        CK(c, cudaMemsetAsync(c->d_gacc, 0, nb, st));
        a.dacc = c->d_gacc;
    }
    CK(c, launch_render_backward(a, grid_for(c, tiles, 128, 4), 128, st));
    return VR_OK;
}

vr_status vr_render_backward(vr_ctx* c, const vr_camera* cams, int n, const float* const* dl, float* dtf,
                             float* dscale, void* stream) {
    return render_backward(c, cams, n, nullptr, dl, dtf, dscale, stream);
}

vr_status vr_render_backward_with_images(vr_ctx* c, const vr_camera* cams, int n, const float* const* images,
                                         const float* const* dl, float* dtf, float* dscale, void* stream) {
    if (c && !images) return fail(c, VR_ERR_INVALID_ARG, "NULL images");
    return render_backward(c, cams, n, images, dl, dtf, dscale, stream);
}

vr_status vr_render_footprint(vr_ctx* c, const vr_camera* cams, int n, float* const* images,
                              uint32_t* const* voxel_marks, uint32_t* node_marks, void* stream) {
    vr_status s = check_ctx(c);
    if (s != VR_OK) return s;
    if (!cams || n <= 0 || !images || !voxel_marks || !node_marks) return fail(c, VR_ERR_INVALID_ARG, "NULL argument");
    for (int L = 0; L <= c->g.N; ++L)
        if (!voxel_marks[L]) return fail(c, VR_ERR_INVALID_ARG, "NULL voxel bitmap");
    if (!c->tf_set) return fail(c, VR_ERR_INVALID_ARG, "transfer functions not set");
    cudaStream_t st = (cudaStream_t)stream;
    long long tiles = 0;
    s = prepare_cams(c, cams, n, images, nullptr, st, &tiles);
    if (s != VR_OK) return s;
    CK(c, cudaMemsetAsync(c->counter, 0, sizeof(unsigned long long), st));
    CK(c, cudaMemsetAsync(c->stats, 0, 2 * sizeof(unsigned long long), st));
    RenderArgs a = make_args(c, n, tiles);
    for (int L = 0; L <= c->g.N; ++L) a.vmark[L] = voxel_marks[L];
    a.nmark = node_marks;
    CK(c, launch_render(a, 2, 0, grid_for(c, tiles, 256, 8), 256, st));
    return VR_OK;
}

static vr_status cache_upload(vr_ctx* c, const std::vector<std::pair<long long, int>>& moves, cudaStream_t st) {
    // moves: (node, cache slot); copies store slot -> cache slot for each, then publishes the table
    const int n = (int)moves.size();
    if (n > 0) {
        if (n > c->glist_cap) {
            CK(c, cudaStreamSynchronize(st));
            dfree(c, c->d_glist);
            if (c->h_glist) cudaFreeHost(c->h_glist);
            c->h_glist = nullptr;
            const int cap = std::max(n, 1024);
            c->d_glist = (int2*)dalloc(c, sizeof(int2) * (size_t)cap);
            if (!c->d_glist || cudaMallocHost(&c->h_glist, sizeof(int2) * (size_t)cap) != cudaSuccess) {
                c->glist_cap = 0;
                return fail(c, VR_ERR_OUT_OF_MEMORY, "cache upload list allocation failed");
            }
            c->glist_cap = cap;
        }
        CK(c, cudaStreamSynchronize(st));
        for (int i = 0; i < n; ++i) c->h_glist[i] = make_int2(c->h_slot[(size_t)moves[i].first], moves[i].second);
        CK(c, cudaMemcpyAsync(c->d_glist, c->h_glist, sizeof(int2) * (size_t)n, cudaMemcpyHostToDevice, st));
        CK(c, launch_cache_gather(c->pool, c->cache, c->d_glist, n, c->g.slot_elems, st));
    }
    CK(c, cudaMemcpyAsync(c->d_cslot, c->h_cslot.data(), sizeof(int) * c->h_cslot.size(), cudaMemcpyHostToDevice, st));
    CK(c, cudaStreamSynchronize(st));
    return VR_OK;
}

vr_status vr_cache_update(vr_ctx* c, int max_uploads, int refinement, void* stream, vr_cache_report* out) {
    vr_status s = check_ctx(c);
    if (s != VR_OK) return s;
    if (c->cache_cap <= 0) return fail(c, VR_ERR_INVALID_ARG, "context has no render cache");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nn = c->h_cslot.size();
    CK(c, cudaMemcpyAsync(c->h_used.data(), c->d_used, nn, cudaMemcpyDeviceToHost, st));
    CK(c, cudaMemcpyAsync(c->h_req.data(), c->d_req, nn, cudaMemcpyDeviceToHost, st));
    CK(c, cudaStreamSynchronize(st));
    std::vector<long long> reqs;
    for (size_t n = 0; n < nn; ++n)
        if (c->h_req[n] && c->h_cslot[n] < 0 && c->h_slot[n] >= 0) reqs.push_back((long long)n);
    // coarser levels first (they cover more of the volume), then node order
    std::stable_sort(reqs.begin(), reqs.end(),
                     [&](long long a, long long b) { return c->node_level[(size_t)a] > c->node_level[(size_t)b]; });
    // victims in order of preference: free, unused in the last pass, then (by request) finer used
    std::vector<int> free_slots, unused, used_by_level[MAXL];
    for (long long sl = c->cache_cap - 1; sl >= 0; --sl) {
        const long long owner = c->h_owner[(size_t)sl];
        if (owner < 0)
            free_slots.push_back((int)sl);
        else if (refinement || !c->h_used[(size_t)owner])
            unused.push_back((int)sl);
        else
            used_by_level[c->node_level[(size_t)owner]].push_back((int)sl);
    }
    std::vector<std::pair<long long, int>> moves;
    long long evicted = 0;
    for (long long node : reqs) {
        if ((int)moves.size() >= max_uploads) break;
        int slot = -1;
        if (!free_slots.empty()) {
            slot = free_slots.back();
            free_slots.pop_back();
        } else if (!unused.empty()) {
            slot = unused.back();
            unused.pop_back();
        } else {
            const int lr = c->node_level[(size_t)node];
            for (int L = 0; L < lr && slot < 0; ++L)
                if (!used_by_level[L].empty()) {
                    slot = used_by_level[L].back();
                    used_by_level[L].pop_back();
                }
        }
        if (slot < 0) break;
        const long long prev = c->h_owner[(size_t)slot];
        if (prev >= 0) {
            c->h_cslot[(size_t)prev] = -1;
            ++evicted;
        }
        c->h_owner[(size_t)slot] = node;
        c->h_cslot[(size_t)node] = slot;
        moves.push_back({node, slot});
    }
    s = cache_upload(c, moves, st);
    if (s != VR_OK) return s;
    CK(c, cudaMemsetAsync(c->d_used, 0, nn, st));
    CK(c, cudaMemsetAsync(c->d_req, 0, nn, st));
    if (out) {
        out->requested = (int64_t)reqs.size();
        out->uploaded = (int64_t)moves.size();
        out->evicted = evicted;
        long long res = 0;
        for (long long o : c->h_owner) res += o >= 0;
        out->resident = res;
        out->capacity = c->cache_cap;
    }
    return VR_OK;
}

vr_status vr_cache_load(vr_ctx* c, int64_t n, const int64_t* nodes, void* stream) {
    vr_status s = check_ctx(c);
    if (s != VR_OK) return s;
    if (c->cache_cap <= 0) return fail(c, VR_ERR_INVALID_ARG, "context has no render cache");
    if (n < 0 || (n > 0 && !nodes)) return fail(c, VR_ERR_INVALID_ARG, "bad node list");
    const long long nn = (long long)c->h_cslot.size();
    std::vector<unsigned char> keep((size_t)nn, 0);
    for (int64_t i = 0; i < n; ++i) {
        if (nodes[i] < 0 || nodes[i] >= nn) return fail(c, VR_ERR_INVALID_ARG, "node outside the tree");
        keep[(size_t)nodes[i]] = 1;
    }
    std::vector<int> victims;
    for (long long sl = c->cache_cap - 1; sl >= 0; --sl)
        if (c->h_owner[(size_t)sl] < 0) victims.push_back((int)sl);
    for (long long sl = c->cache_cap - 1; sl >= 0; --sl) {
        const long long o = c->h_owner[(size_t)sl];
        if (o >= 0 && !keep[(size_t)o]) victims.push_back((int)sl);
    }
    std::reverse(victims.begin(), victims.end()); // free slots are taken first (from the back)
    std::vector<std::pair<long long, int>> moves;
    for (int64_t i = 0; i < n; ++i) {
        const long long node = nodes[i];
        if (c->h_slot[(size_t)node] < 0 || c->h_cslot[(size_t)node] >= 0) continue;
        if (victims.empty()) return fail(c, VR_ERR_OUT_OF_MEMORY, "render cache smaller than the node list");
        const int slot = victims.back();
        victims.pop_back();
        const long long prev = c->h_owner[(size_t)slot];
        if (prev >= 0) c->h_cslot[(size_t)prev] = -1;
        c->h_owner[(size_t)slot] = node;
        c->h_cslot[(size_t)node] = slot;
        moves.push_back({node, slot});
    }
    return cache_upload(c, moves, (cudaStream_t)stream);
}

vr_status vr_cache_read(vr_ctx* c, uint8_t* resident, uint8_t* used, uint8_t* requested, void* stream) {
    vr_status s = check_ctx(c);
    if (s != VR_OK) return s;
    if (c->cache_cap <= 0) return fail(c, VR_ERR_INVALID_ARG, "context has no render cache");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nn = c->h_cslot.size();
    if (used) CK(c, cudaMemcpyAsync(used, c->d_used, nn, cudaMemcpyDeviceToHost, st));
    if (requested) CK(c, cudaMemcpyAsync(requested, c->d_req, nn, cudaMemcpyDeviceToHost, st));
    CK(c, cudaStreamSynchronize(st));
    if (resident)
        for (size_t n = 0; n < nn; ++n) resident[n] = c->h_cslot[n] >= 0;
    return VR_OK;
}

struct vr_refine {
    vr_ctx* c = nullptr;
    CamParam* d_cam = nullptr;
    RefineState* state = nullptr;
    unsigned int* pending = nullptr;
    long long tiles = 0;
};

vr_status vr_refine_begin(vr_ctx* c, const vr_camera* cam, float* image, vr_refine** out) {
    vr_status s = check_ctx(c);
    if (s != VR_OK) return s;
    if (!cam || !image || !out) return fail(c, VR_ERR_INVALID_ARG, "NULL argument");
    if (c->cache_cap <= 0) return fail(c, VR_ERR_INVALID_ARG, "refinement needs a render cache");
    if (!c->tf_set) return fail(c, VR_ERR_INVALID_ARG, "transfer functions not set");
    CamParam cp;
    std::memset(&cp, 0, sizeof cp);
    if (!derive_camera(c, *cam, cp)) return fail(c, VR_ERR_INVALID_ARG, "invalid camera");
    cp.img = image;
    cp.tiles_x = (int)ceil_div(cp.W, c->tile_w);
    cp.tile_begin = 0;
    vr_refine* r = new vr_refine();
    r->c = c;
    r->tiles = (long long)cp.tiles_x * ceil_div(cp.H, c->tile_h);
    r->d_cam = (CamParam*)dalloc(c, sizeof(CamParam));
    r->state = (RefineState*)dalloc(c, sizeof(RefineState) * (size_t)cp.W * (size_t)cp.H);
    r->pending = (unsigned int*)dalloc(c, sizeof(unsigned int) * 4);
    if (!r->d_cam || !r->state || !r->pending) {
        dfree(c, r->d_cam);
        dfree(c, r->state);
        dfree(c, r->pending);
        delete r;
        return fail(c, VR_ERR_OUT_OF_MEMORY, "refinement state allocation failed");
    }
    cudaError_t e = cudaMemcpy(r->d_cam, &cp, sizeof cp, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(r->state, 0, sizeof(RefineState) * (size_t)cp.W * (size_t)cp.H);
    if (e != cudaSuccess) {
        dfree(c, r->d_cam);
        dfree(c, r->state);
        dfree(c, r->pending);
        delete r;
        return cuda_fail(c, e, "refine_begin");
    }
    *out = r;
    return VR_OK;
}

vr_status vr_refine_pass(vr_refine* r, void* stream, int64_t* pending, int64_t* samples) {
    if (!r) return VR_ERR_INVALID_ARG;
    vr_ctx* c = r->c;
    vr_status s = check_ctx(c);
    if (s != VR_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    RenderArgs a = make_args(c, 1, r->tiles);
    a.cams = r->d_cam;
    a.cache.refine = 1;
    a.refine_state = r->state;
    a.pending = r->pending;
    CK(c, cudaMemsetAsync(r->pending, 0, sizeof(unsigned int), st));
    CK(c, cudaMemsetAsync(c->counter, 0, sizeof(unsigned long long), st));
    CK(c, cudaMemsetAsync(c->stats, 0, 2 * sizeof(unsigned long long), st));
    CK(c, launch_render(a, 3, 0, grid_for(c, r->tiles, 256, 8), 256, st));
    unsigned int hp = 0;
    unsigned long long hs[2] = {0, 0};
    CK(c, cudaMemcpyAsync(&hp, r->pending, sizeof hp, cudaMemcpyDeviceToHost, st));
    CK(c, cudaMemcpyAsync(hs, c->stats, sizeof hs, cudaMemcpyDeviceToHost, st));
    CK(c, cudaStreamSynchronize(st));
    if (pending) *pending = hp;
    if (samples) *samples = (int64_t)hs[0];
    return VR_OK;
}

vr_status vr_refine_end(vr_refine* r) {
    if (!r) return VR_ERR_INVALID_ARG;
    cudaSetDevice(r->c->dev);
    cudaDeviceSynchronize();
    dfree(r->c, r->d_cam);
    dfree(r->c, r->state);
    dfree(r->c, r->pending);
    delete r;
    return VR_OK;
}

static vr_status poll_error(vr_ctx* c, cudaStream_t st) {
    int h = 0;
    CK(c, cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(c, cudaStreamSynchronize(st));
    if (h) return fail(c, VR_ERR_DEVICE_ASSERT, "device check failed (code " + std::to_string(h) + ")");
    return VR_OK;
}

vr_status vr_read_level(vr_ctx* c, int level, uint16_t* out, void* stream) {
    vr_status s = check_ctx(c);
    if (s != VR_OK) return s;
    if (!out || level < 0 || level > c->g.N) return fail(c, VR_ERR_INVALID_ARG, "bad level or NULL output");
    const Geo& g = c->g;
    cudaStream_t st = (cudaStream_t)stream;
    size_t bytes = (size_t)g.ldim[level][0] * g.ldim[level][1] * g.ldim[level][2] * g.C * sizeof(uint16_t);
    uint16_t* tmp = (uint16_t*)dalloc(c, bytes);
    if (!tmp) return fail(c, VR_ERR_OUT_OF_MEMORY, "read buffer allocation failed");
    cudaError_t e = launch_read_level(g, level, c->pool, c->rn, tmp, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(c, tmp);
    if (e != cudaSuccess) return cuda_fail(c, e, "read_level");
    return poll_error(c, st);
}

vr_status vr_read_voxels(vr_ctx* c, int level, int64_t n, const int64_t* xyz, uint16_t* out, void* stream) {
    vr_status s = check_ctx(c);
    if (s != VR_OK) return s;
    const Geo& g = c->g;
    if (level < 0 || level > g.N || n < 0 || (n > 0 && (!xyz || !out))) return fail(c, VR_ERR_INVALID_ARG, "bad arguments");
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a)
            if (xyz[3 * i + a] < 0 || xyz[3 * i + a] >= g.ldim[level][a])
                return fail(c, VR_ERR_INVALID_ARG, "voxel outside the level");
    if (n == 0) return VR_OK;
    cudaStream_t st = (cudaStream_t)stream;
    long long* dxyz = (long long*)dalloc(c, sizeof(long long) * 3 * (size_t)n);
    uint16_t* dout = (uint16_t*)dalloc(c, sizeof(uint16_t) * (size_t)(n * g.C));
    cudaError_t e = (!dxyz || !dout) ? cudaErrorMemoryAllocation : cudaSuccess;
    if (e == cudaSuccess) e = cudaMemcpyAsync(dxyz, xyz, sizeof(long long) * 3 * (size_t)n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_read_voxels(g, level, c->pool, c->rn, dxyz, n, dout, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, sizeof(uint16_t) * (size_t)(n * g.C), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(c, dxyz);
    dfree(c, dout);
    if (e != cudaSuccess) return cuda_fail(c, e, "read_voxels");
    return poll_error(c, st);
}

vr_status vr_read_node(vr_ctx* c, int level, int64_t i, int64_t j, int64_t k, uint32_t* flags, uint16_t* avg,
                       void* stream) {
    vr_status s = check_ctx(c);
    if (s != VR_OK) return s;
    const Geo& g = c->g;
    if (level < 0 || level > g.N || i < 0 || j < 0 || k < 0 || i >= g.nb[level][0] || j >= g.nb[level][1] ||
        k >= g.nb[level][2] || !flags)
        return fail(c, VR_ERR_INVALID_ARG, "node outside the grid");
    cudaStream_t st = (cudaStream_t)stream;
    RNode r;
    CK(c, cudaMemcpyAsync(&r, c->rn + g.noff[level] + (k * g.nb[level][1] + j) * g.nb[level][0] + i, sizeof(RNode),
                          cudaMemcpyDeviceToHost, st));
    CK(c, cudaStreamSynchronize(st));
    *flags = r.flags;
    if (avg)
        for (int q = 0; q < g.C; ++q) avg[q] = r.avg[q];
    return poll_error(c, st);
}

vr_status vr_debug_raise_error(vr_ctx* c, int code) {
    vr_status s = check_ctx(c);
    if (s != VR_OK) return s;
    if (code == 0) return fail(c, VR_ERR_INVALID_ARG, "code must be non-zero");
    CK(c, cudaMemcpy(c->err, &code, sizeof(int), cudaMemcpyHostToDevice));
    return VR_OK;
}

vr_status vr_stats(vr_ctx* c, vr_stats_t* out) {
    if (!c || !out) return VR_ERR_INVALID_ARG;
    cudaSetDevice(c->dev);
    const Geo& g = c->g;
    std::memset(out, 0, sizeof *out);
    for (int a = 0; a < 3; ++a) out->dims[a] = g.ldim[0][a];
    out->channels = g.C;
    out->brick_size = g.M;
    out->levels = g.N + 1;
    out->nodes = g.noff[g.N + 1];
    out->slots_capacity = g.n_slots_cap;
    out->slots_used = c->slots_used;
    out->pool_bytes = g.n_slots_cap * g.slot_elems * 2;
    out->node_table_bytes = out->nodes * (long long)(sizeof(RNode) + sizeof(NStat));
    unsigned long long h[2] = {0, 0};
    if (cudaMemcpy(h, c->stats, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess)
        return cuda_fail(c, cudaGetLastError(), "stats");
    out->last_render_samples = (int64_t)h[0];
    out->last_render_rays = (int64_t)h[1];
    if (c->last_cont) {
        unsigned n = 0;
        if (cudaMemcpy(&n, c->cont_ctl + 1, sizeof n, cudaMemcpyDeviceToHost) != cudaSuccess)
            return cuda_fail(c, cudaGetLastError(), "stats");
        out->last_render_continued = n;
    }
    return VR_OK;
}

const char* vr_last_error(const vr_ctx* c) { return c ? c->msg.c_str() : g_create_error.c_str(); }

// Tile shape of the ray queue (tw x th pixels per warp, tw * th = 32).  Used by the autotuner.
vr_status vr_set_tile_shape(vr_ctx* c, int tw, int th) {
    if (!c || tw <= 0 || th <= 0 || tw * th != 32) return VR_ERR_INVALID_ARG;
    c->tile_w = tw;
    c->tile_h = th;
    return VR_OK;
}

vr_status vr_set_mip_segment_length(vr_ctx* c, int samples) {
    if (!c || samples < 0 || (samples > 0 && samples < 4) || samples > (1 << 24)) return VR_ERR_INVALID_ARG;
    c->kseg_mip = samples;
    return VR_OK;
}

vr_status vr_set_gradient_precision(vr_ctx* c, int fp64) {
    vr_status s = check_ctx(c);
    if (s != VR_OK) return s;
    if (fp64 != 0 && fp64 != 1) return fail(c, VR_ERR_INVALID_ARG, "gradient precision must be 0 or 1");
    c->grad_fp64 = fp64;
    return VR_OK;
}

vr_status vr_set_tile_order(vr_ctx* c, int mode) {
    if (!c || (mode != 0 && mode != 1)) return VR_ERR_INVALID_ARG;
    c->tile_order_mode = mode;
    c->lpt_have = false;
    return VR_OK;
}

vr_status vr_set_insert_staging(vr_ctx* c, int mode) {
    if (!c || (mode != 0 && mode != 1)) return VR_ERR_INVALID_ARG;
    c->insert_staging = mode;
    return VR_OK;
}

vr_status vr_set_ray_continuation(vr_ctx* c, int lanes_per_ray, int min_samples_left) {
    if (!c) return VR_ERR_INVALID_ARG;
    int lg = 0;
    while (lg <= 5 && (1 << lg) != lanes_per_ray) ++lg;
    if (lanes_per_ray != 0 && lg > 5) return fail(c, VR_ERR_INVALID_ARG, "ray continuation: 0 or 1..32 lanes (a power of two)");
    if (min_samples_left < 0) return fail(c, VR_ERR_INVALID_ARG, "ray continuation: min_samples_left < 0");
    c->cont_lg = lanes_per_ray == 0 ? -1 : lg;
    c->cont_min = min_samples_left;
    return VR_OK;
}

vr_status vr_set_launch_shape(vr_ctx* c, int tw, int th, int threads, int ctas_per_sm) {
    if (!c || tw <= 0 || th <= 0 || tw * th != 32 ||
        (threads != 64 && threads != 128 && threads != 256 && threads != 512 && threads != 768) ||
        ctas_per_sm < 1 || ctas_per_sm > 32)
        return VR_ERR_INVALID_ARG;
    c->tile_w = tw;
    c->tile_h = th;
    c->threads = threads;
    c->ctas_per_sm = ctas_per_sm;
    return VR_OK;
}

struct vr_render_plan {
    vr_ctx* c = nullptr;
    SegBuf seg;
    CamParam* d_cams = nullptr;
    unsigned int* counter = nullptr;
    unsigned long long* stats = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

static void plan_free(vr_render_plan* p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    seg_free(p->c, p->seg);
    dfree(p->c, p->d_cams);
    dfree(p->c, p->counter);
    dfree(p->c, p->stats);
    delete p;
}

vr_status vr_plan_create(vr_ctx* c, const vr_camera* cams, int n, float* const* images, int mode,
                         vr_render_plan** out) {
    vr_status s = check_ctx(c);
    if (s != VR_OK) return s;
    if (!out || !cams || n <= 0 || !images) return fail(c, VR_ERR_INVALID_ARG, "no cameras or images");
    *out = nullptr;
    const int fp16 = (mode & VR_RENDER_FP16) || c->opt.precision == VR_FP16_INTERP;
    mode &= ~VR_RENDER_FP16;
    if (mode != VR_MODE_DVR && mode != VR_MODE_MIP) return fail(c, VR_ERR_INVALID_ARG, "unknown mode");
    if (!c->tf_set) return fail(c, VR_ERR_INVALID_ARG, "transfer functions not set");
    std::vector<CamParam> h((size_t)n);
    long long tiles = 0;
    for (int i = 0; i < n; ++i) {
        CamParam& cp = h[(size_t)i];
        std::memset(&cp, 0, sizeof cp);
        if (!derive_camera(c, cams[i], cp)) return fail(c, VR_ERR_INVALID_ARG, "invalid camera " + std::to_string(i));
        if (!images[i]) return fail(c, VR_ERR_INVALID_ARG, "NULL image");
        cp.img = images[i];
        cp.tiles_x = (int)ceil_div(cp.W, c->tile_w);
        cp.tile_begin = tiles;
        tiles += (long long)cp.tiles_x * ceil_div(cp.H, c->tile_h);
    }
    if (tiles >= 0xffffffffLL) return fail(c, VR_ERR_INVALID_ARG, "too many pixels in one plan");
    vr_render_plan* p = new vr_render_plan();
    p->c = c;
    p->d_cams = (CamParam*)dalloc(c, sizeof(CamParam) * (size_t)n);
    p->counter = (unsigned int*)dalloc(c, sizeof(unsigned int) * 4);
    p->stats = (unsigned long long*)dalloc(c, sizeof(unsigned long long) * 4);
    if (!p->d_cams || !p->counter || !p->stats) {
        plan_free(p);
        return fail(c, VR_ERR_OUT_OF_MEMORY, "plan allocation failed");
    }
    cudaError_t e = cudaMemcpy(p->d_cams, h.data(), sizeof(CamParam) * (size_t)n, cudaMemcpyHostToDevice);
    RenderArgs a = make_args(c, n, tiles);
    a.cams = p->d_cams;
    a.counter = p->counter;
    a.stats = p->stats;
    if (e == cudaSuccess && mode == VR_MODE_MIP) {
        s = seg_prepare(c, p->seg, a, h.data(), n, tiles, nullptr);
        if (s != VR_OK) {
            plan_free(p);
            return s;
        }
    }
    cudaStream_t cs = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        cudaMemsetAsync(p->counter, 0, sizeof(unsigned long long), cs);
        cudaMemsetAsync(p->stats, 0, 2 * sizeof(unsigned long long), cs);
        launch_render(a, mode, fp16 && mode == VR_MODE_DVR, grid_for(c, tiles, c->threads, c->ctas_per_sm), c->threads, cs);
        e = cudaStreamEndCapture(cs, &p->graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    if (cs) cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        plan_free(p);
        return cuda_fail(c, e, "plan capture");
    }
    *out = p;
    return VR_OK;
}

vr_status vr_plan_launch(vr_render_plan* p, void* stream) {
    if (!p) return VR_ERR_INVALID_ARG;
    vr_status s = check_ctx(p->c);
    if (s != VR_OK) return s;
    CK(p->c, cudaGraphLaunch(p->exec, (cudaStream_t)stream));
    return VR_OK;
}

vr_status vr_plan_samples(vr_render_plan* p, int64_t* samples, int64_t* rays) {
    if (!p) return VR_ERR_INVALID_ARG;
    unsigned long long h[2] = {0, 0};
    CK(p->c, cudaMemcpy(h, p->stats, sizeof h, cudaMemcpyDeviceToHost));
    if (samples) *samples = (int64_t)h[0];
    if (rays) *rays = (int64_t)h[1];
    return VR_OK;
}

vr_status vr_plan_destroy(vr_render_plan* p) {
    if (!p) return VR_ERR_INVALID_ARG;
    cudaSetDevice(p->c->dev);
    cudaDeviceSynchronize();
    plan_free(p);
    return VR_OK;
}

} // extern "C"

// Validation and camera constants for vr_render_noalloc (vr_noalloc.cu): exactly what vr_render
// computes, written into a host array the caller provides, with no allocation of any kind.
namespace vrk {

vr_status prepare_render_noalloc(vr_ctx* c, const vr_camera* cams, int n, float* const* images, int mode,
                                 CamParam* params, RenderArgs* args, int* blocks, int* threads, int* fp16) {
    vr_status s = check_ctx(c);
    if (s != VR_OK) return s;
    if (!cams || n <= 0 || !images || !params || !args || !blocks || !threads || !fp16)
        return fail(c, VR_ERR_INVALID_ARG, "no cameras or images");
    // the same mode word as vr_render: DVR or MIP, optionally | VR_RENDER_FP16 (DVR only)
    const int want_fp16 = (mode & VR_RENDER_FP16) || c->opt.precision == VR_FP16_INTERP;
    mode &= ~VR_RENDER_FP16;
    if (mode != VR_MODE_DVR && mode != VR_MODE_MIP) return fail(c, VR_ERR_INVALID_ARG, "unknown mode");
    *fp16 = want_fp16 && mode == VR_MODE_DVR;
    if (!c->tf_set) return fail(c, VR_ERR_INVALID_ARG, "transfer functions not set");
    long long tiles = 0;
    for (int i = 0; i < n; ++i) {
        CamParam& cp = params[i];
        std::memset(&cp, 0, sizeof cp);
        if (!derive_camera(c, cams[i], cp)) return fail(c, VR_ERR_INVALID_ARG, "invalid camera " + std::to_string(i));
        if (!images[i]) return fail(c, VR_ERR_INVALID_ARG, "NULL image");
        cp.img = images[i];
        cp.tiles_x = (int)ceil_div(cp.W, c->tile_w);
        cp.tile_begin = tiles;
        tiles += (long long)cp.tiles_x * ceil_div(cp.H, c->tile_h);
    }
    if (tiles >= 0xffffffffLL) return fail(c, VR_ERR_INVALID_ARG, "too many pixels in one call");
    *args = make_args(c, n, tiles);
    // the context's launch shape (vr_set_launch_shape), as vr_render uses it
    *threads = c->threads;
    *blocks = grid_for(c, tiles, c->threads, c->ctas_per_sm);
    return VR_OK;
}

vr_status noalloc_fail(vr_ctx* c, vr_status s, const char* msg) { return fail(c, s, msg); }

} // namespace vrk
