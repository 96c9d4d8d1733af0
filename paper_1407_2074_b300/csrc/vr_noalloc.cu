// vr_noalloc.cu -- vr_render_noalloc: the ray-casting launch of vr_render without any memory
// allocation by the library during the call.
//
// Who needs it: applications that budget GPU memory once, up front (for instance a viewer that
// sizes its brick pool to nearly all of the device and then renders frame after frame), and
// hosts that hand the library a stream but forbid it to allocate -- cudaMalloc/cudaFree may
// synchronise the whole device and would stall every other stream of the process on each call.
// vr_render allocates its camera buffer (device + pinned host) the first time it sees a larger
// batch; this entry point instead keeps the ray-tile queue head, the sample counters and the
// per-camera constants in one fixed array in device memory, defined below, which every GPU that
// loads libvr holds until the process exits (about 15 KB).
#include <cuda_runtime.h>

#include <mutex>

#include "vr.h"
#include "vr_internal.h"

namespace vrk {
vr_status prepare_render_noalloc(vr_ctx* c, const vr_camera* cams, int n, float* const* images, int mode,
                                 CamParam* params, RenderArgs* args, int* blocks, int* threads, int* fp16);
vr_status noalloc_fail(vr_ctx* c, vr_status s, const char* msg);
} // namespace vrk

using namespace vrk;

namespace {
struct NoAllocScratch {
    CamParam cams[VR_NOALLOC_MAX_CAMERAS];
    unsigned int counter[4];        // ray-tile queue head
    unsigned long long stats[4];    // samples, rays
};
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};
} // namespace

// The scratch itself.  In host code this name is only a stand-in for the symbol, never a device
// address: the address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char vr_noalloc_scratch[sizeof(NoAllocScratch)];

extern "C" vr_status vr_render_noalloc(vr_ctx* ctx, const vr_camera* cams, int n_cams, float* const* images, int mode,
                                       void* cuda_stream) {
    if (!ctx) return VR_ERR_INVALID_ARG;
    if (n_cams > VR_NOALLOC_MAX_CAMERAS)
        return noalloc_fail(ctx, VR_ERR_INVALID_ARG, "vr_render_noalloc: more than VR_NOALLOC_MAX_CAMERAS (64) cameras");
    CamParam params[VR_NOALLOC_MAX_CAMERAS]; // host stack, no heap
    RenderArgs a;
    int blocks = 0, threads = 0, fp16 = 0;
    // validates like vr_render and makes ctx's device current
    vr_status s = prepare_render_noalloc(ctx, cams, n_cams, images, mode, params, &a, &blocks, &threads, &fp16);
    if (s != VR_OK) return s;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return noalloc_fail(ctx, VR_ERR_CUDA, "vr_render_noalloc: no usable current device");
    }
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_addr[dev]) { // first call on this device: look the array up, with the device current
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, vr_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return noalloc_fail(ctx, VR_ERR_CUDA, "vr_render_noalloc: cudaGetSymbolAddress failed");
            }
            g_scratch_addr[dev] = p;
        }
        base = g_scratch_addr[dev];
    }
    NoAllocScratch* sc = static_cast<NoAllocScratch*>(base);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaMemcpyAsync(sc->cams, params, sizeof(CamParam) * (size_t)n_cams, cudaMemcpyHostToDevice, st);
    // the array keeps the previous call's contents: the queue head and counters must restart at 0
    if (e == cudaSuccess) e = cudaMemsetAsync(sc->counter, 0, sizeof(sc->counter), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc->stats, 0, sizeof(sc->stats), st);
    if (e != cudaSuccess) return noalloc_fail(ctx, VR_ERR_CUDA, cudaGetErrorString(e));
    a.cams = sc->cams;
    a.counter = sc->counter;
    a.stats = sc->stats;
    e = launch_render(a, mode & ~VR_RENDER_FP16, fp16, blocks, threads, st);
    if (e != cudaSuccess) return noalloc_fail(ctx, VR_ERR_CUDA, cudaGetErrorString(e));
    return VR_OK;
}
