// vr_render.cu -- ray casting of the bricked octree (Algorithm 1 and Sec. "Basic Ray-Casting")
// and its adjoint with respect to the transfer functions and intensity scales.
//
// Work decomposition: a persistent grid; every warp takes 32-ray tiles (tile_w x tile_h pixels)
// from one queue spanning all cameras of the call (batched views of uneven resolution share one
// launch).  Per ray:
//   setup      pinhole ray, slab test against the real volume box, clip half-spaces, t >= 0;
//   march      t_k = t0 + k dt while t_k < t1, last segment l = t1 - t_k;
//   LOD        L* = largest L with t_k >= t_L (thresholds precomputed per camera);
//   node       descent from the root to level L* through the dense node tables, stopping at a
//              node without children; the node is cached until the sample leaves its box or L*
//              rises above its level;
//   intensity  AVG of a brick-less node, else trilinear inside the node's slot (the border
//              voxels make the eight corners one slot); the eight corners are cached per cell;
//   TF         x = sat(I s / 65535), entry i = min(floor(255 x), 254), linear (smem table);
//   composite  a = 1 - (1 - alpha)^l, C += (1 - A) a rgb, A += (1 - A) a per channel in order;
//   ERT        stop once A >= ert after a sample.
// Geometry (ray direction, interval, t_k, sample positions, level and node choice) uses only
// correctly rounded single-precision operations (_rn intrinsics, never contracted) in a fixed
// order, so these integer-valued decisions are reproducible off the GPU; interpolation, TF and
// compositing are ordinary FP32 with FMA.
#include <cuda_runtime.h>
#include <math_constants.h>

#include "vr_internal.h"

namespace vrk {

__device__ __forceinline__ bool ray_setup(const CamParam& cp, const Geo& g, int px, int py, float d[3], float& t0,
                                          float& t1) {
    const float a = (float)(2 * px + 1);
    const float cxp = __fsub_rn(__fdiv_rn(a, (float)cp.W), 1.0f);
    const float b = (float)(2 * py + 1);
    const float cyp = __fsub_rn(1.0f, __fdiv_rn(b, (float)cp.H));
    const float x = __fmul_rn(cxp, cp.kx), y = __fmul_rn(cyp, cp.ky);
    float dd[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) dd[i] = __fadd_rn(__fadd_rn(cp.ff[i], __fmul_rn(x, cp.rr[i])), __fmul_rn(y, cp.uu[i]));
    const float n2 = __fadd_rn(__fadd_rn(__fmul_rn(dd[0], dd[0]), __fmul_rn(dd[1], dd[1])), __fmul_rn(dd[2], dd[2]));
    const float s = __fsqrt_rn(n2);
#pragma unroll
    for (int i = 0; i < 3; ++i) d[i] = __fdiv_rn(dd[i], s);
    t0 = 0.0f;
    t1 = CUDART_INF_F;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float o = cp.eye[i], D = (float)g.ldim[0][i];
        if (d[i] != 0.0f) {
            const float ta = __fdiv_rn(__fsub_rn(0.0f, o), d[i]), tb = __fdiv_rn(__fsub_rn(D, o), d[i]);
            t0 = fmaxf(t0, fminf(ta, tb));
            t1 = fminf(t1, fmaxf(ta, tb));
        } else if (o < 0.0f || o > D) {
            return false;
        }
    }
    for (int p = 0; p < cp.n_clip; ++p) {
        const float* n = cp.clip[p];
        const float sv = __fadd_rn(
            __fadd_rn(__fadd_rn(__fmul_rn(n[0], cp.eye[0]), __fmul_rn(n[1], cp.eye[1])), __fmul_rn(n[2], cp.eye[2])), n[3]);
        const float q = __fadd_rn(__fadd_rn(__fmul_rn(n[0], d[0]), __fmul_rn(n[1], d[1])), __fmul_rn(n[2], d[2]));
        if (q == 0.0f) {
            if (sv < 0.0f) return false;
        } else {
            const float tc = __fdiv_rn(-sv, q);
            if (q > 0.0f)
                t0 = fmaxf(t0, tc);
            else
                t1 = fminf(t1, tc);
        }
    }
    return t0 < t1;
}

// Opacity correction a = 1 - (1 - alpha)^l and its complement (1 - alpha)^l, accurate for small
// alpha (no 1 - (1 - x) cancellation).
__device__ __forceinline__ void opacity(float al, float ell, float& a, float& oma) {
    if (ell == 0.5f) {
        const float s = sqrtf(1.0f - al);
        a = al / (1.0f + s);
        oma = s;
    } else if (ell == 1.0f) {
        a = al;
        oma = 1.0f - al;
    } else {
        const float lg = log1pf(-al);
        a = -expm1f(ell * lg);
        oma = expf(ell * lg);
    }
}

constexpr float ALPHA_MAX = 1.0f - 1e-6f;
constexpr long long MAX_SAMPLES = 1LL << 24; // (float)k stays exact; bounds every ray

template <int C>
struct TFLookup {
    float r, g, b, al; // interpolated entry (al before clamping)
    float lam, xr;     // position between entries, unclamped x
    int i;
    __device__ __forceinline__ void eval(const float4* __restrict__ s_tf, const float* s_scl, int c, float I) {
        xr = I * s_scl[c];
        const float x = __saturatef(xr);
        const float w = x * 255.0f;
        i = min((int)w, 254);
        lam = w - (float)i;
        const float4 T = s_tf[(c * 256 + i) * 2], D = s_tf[(c * 256 + i) * 2 + 1];
        r = fmaf(lam, D.x, T.x);
        g = fmaf(lam, D.y, T.y);
        b = fmaf(lam, D.z, T.z);
        al = fmaf(lam, D.w, T.w);
    }
};

// Marches one ray; calls f.sample(I[C], ell) for every sample until it returns true.
template <int C, int VS, bool POW2, class F>
__device__ __forceinline__ long long march(const Geo& g, const uint16_t* __restrict__ pool,
                                           const RNode* __restrict__ rn, const CamParam& cp, const float d[3], float t0,
                                           float t1, F& f) {
    const float dt = cp.dt;
    const int N = g.N, M = g.M, S = g.S;
    int Lstar = 0;
    float tnext = cp.tl[1 <= N ? 1 : N + 1];
    if (N < 1) tnext = CUDART_INF_F;
    // node cache
    int nlev = -1;
    float tl_limit = 0.0f; // t at which L* would exceed the cached node's level
    float lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    long long cidx[3] = {0, 0, 0};
    bool brick = false;
    const uint16_t* sbase = nullptr;
    float avg[C];
    float off[3] = {0, 0, 0};
    float inv_vox = 1.0f;
    // cell cache
    const uint16_t* cell = nullptr;
    float cv[8][C];
    long long k = 0;
    for (;; ++k) {
        const float tk = __fadd_rn(t0, __fmul_rn((float)k, dt));
        if (!(tk < t1) || k >= MAX_SAMPLES) break;
        const float ell = fminf(dt, __fsub_rn(t1, tk));
        float p[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) p[a] = __fadd_rn(cp.eye[a], __fmul_rn(tk, d[a]));
        while (tk >= tnext) {
            ++Lstar;
            tnext = (Lstar < N) ? cp.tl[Lstar + 1] : CUDART_INF_F;
        }
        bool valid = nlev >= 0 && tk < tl_limit;
        if (valid) {
            if (POW2) {
#pragma unroll
                for (int a = 0; a < 3; ++a) valid = valid && (p[a] >= lo[a]) && (p[a] < hi[a]);
            } else {
                const float size = (float)(M << nlev);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    long long q = (long long)floorf(__fdiv_rn(p[a], size));
                    q = q < 0 ? 0 : (q > g.nb[nlev][a] - 1 ? g.nb[nlev][a] - 1 : q);
                    valid = valid && (q == cidx[a]);
                }
            }
        }
        if (!valid) {
            // getNodeAtPosition: descend from the root towards L*
            int lev = N;
            long long idx[3] = {0, 0, 0};
            RNode nd = rn[g.noff[N]];
            f.on_node(g.noff[N]);
            while (lev > Lstar && (nd.flags & F_CHILDREN)) {
                --lev;
                const float size = (float)(M << lev);
                const float inv = 1.0f / size;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    long long q = POW2 ? (long long)floorf(__fmul_rn(p[a], inv)) : (long long)floorf(__fdiv_rn(p[a], size));
                    const long long c0 = 2 * idx[a];
                    q = q < c0 ? c0 : (q > c0 + 1 ? c0 + 1 : q);
                    if (q > g.nb[lev][a] - 1) q = g.nb[lev][a] - 1;
                    idx[a] = q;
                }
                const long long nid = g.noff[lev] + (idx[2] * g.nb[lev][1] + idx[1]) * g.nb[lev][0] + idx[0];
                nd = rn[nid];
                f.on_node(nid);
            }
            nlev = lev;
            tl_limit = (lev < N) ? cp.tl[lev + 1] : CUDART_INF_F;
            const float size = (float)(M << lev);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                cidx[a] = idx[a];
                lo[a] = (idx[a] == 0) ? -CUDART_INF_F : (float)idx[a] * size;
                hi[a] = (idx[a] == g.nb[lev][a] - 1) ? CUDART_INF_F : (float)(idx[a] + 1) * size;
                off[a] = (float)(idx[a] * M) - 0.5f;
            }
            inv_vox = 1.0f / (float)(1 << lev);
            brick = (nd.flags & F_BRICK) && nd.slot >= 0 && nd.slot < g.n_slots_cap;
            sbase = brick ? pool + (long long)nd.slot * g.slot_elems : nullptr;
#pragma unroll
            for (int c = 0; c < C; ++c) avg[c] = (float)nd.avg[c];
            cell = nullptr;
        }
        float I[C];
        if (brick) {
            float fr[3];
            int i0[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float u = __fsub_rn(__fmul_rn(p[a], inv_vox), off[a]);
                const float fl = floorf(u);
                int ii = (int)fl;
                fr[a] = __fsub_rn(u, fl);
                i0[a] = ii < 0 ? 0 : (ii > M ? M : ii);
            }
            const uint16_t* cp0 = sbase + ((long long)(i0[2] * S + i0[1]) * S + i0[0]) * VS;
            if (cp0 != cell) {
                cell = cp0;
                f.on_cell(g, nlev, cidx, i0);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const uint16_t* v = cp0 + ((long long)(((q >> 2) & 1) * S + ((q >> 1) & 1)) * S + (q & 1)) * VS;
                    if (VS == 4) {
                        const uint2 w = __ldg(reinterpret_cast<const uint2*>(v));
                        const uint32_t ws[2] = {w.x, w.y};
#pragma unroll
                        for (int c = 0; c < C; ++c) cv[q][c] = (float)((ws[c >> 1] >> (16 * (c & 1))) & 0xffffu);
                    } else if (VS == 2) {
                        const uint32_t w = __ldg(reinterpret_cast<const unsigned int*>(v));
#pragma unroll
                        for (int c = 0; c < C; ++c) cv[q][c] = (float)((w >> (16 * c)) & 0xffffu);
                    } else {
                        cv[q][0] = (float)__ldg(reinterpret_cast<const unsigned short*>(v));
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const float c00 = fmaf(fr[0], cv[1][c] - cv[0][c], cv[0][c]);
                const float c10 = fmaf(fr[0], cv[3][c] - cv[2][c], cv[2][c]);
                const float c01 = fmaf(fr[0], cv[5][c] - cv[4][c], cv[4][c]);
                const float c11 = fmaf(fr[0], cv[7][c] - cv[6][c], cv[6][c]);
                const float c0 = fmaf(fr[1], c10 - c00, c00);
                const float c1 = fmaf(fr[1], c11 - c01, c01);
                I[c] = fmaf(fr[2], c1 - c0, c0);
            }
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) I[c] = avg[c];
        }
        if (f.sample(I, ell)) {
            ++k;
            break;
        }
    }
    return k;
}

struct NoHooks {
    __device__ __forceinline__ void on_node(long long) {}
    __device__ __forceinline__ void on_cell(const Geo&, int, const long long*, const int*) {}
};

template <int C>
struct DVRComposite : NoHooks {
    const float4* s_tf;
    const float* s_scl;
    float ert;
    float A = 0.0f, Cr = 0.0f, Cg = 0.0f, Cb = 0.0f;
    __device__ __forceinline__ bool sample(const float (&I)[C], float ell) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            TFLookup<C> t;
            t.eval(s_tf, s_scl, c, I[c]);
            const float al = fminf(fmaxf(t.al, 0.0f), ALPHA_MAX);
            float a, oma;
            opacity(al, ell, a, oma);
            const float w = (1.0f - A) * a;
            Cr = fmaf(w, t.r, Cr);
            Cg = fmaf(w, t.g, Cg);
            Cb = fmaf(w, t.b, Cb);
            A += w;
        }
        return A >= ert;
    }
};

// DVR that also records the distinct (level, voxel) pairs read by trilinear corners and the
// node entries visited: the algorithmic footprint of a frame (measurement only).
template <int C>
struct DVRFootprint : DVRComposite<C> {
    unsigned int* const* vmark;
    unsigned int* nmark;
    __device__ __forceinline__ void on_node(long long nid) {
        atomicOr(&nmark[nid >> 5], 1u << (nid & 31));
    }
    __device__ __forceinline__ void on_cell(const Geo& g, int L, const long long* idx, const int* i0) {
        for (int q = 0; q < 8; ++q) {
            long long v[3];
            for (int a = 0; a < 3; ++a) {
                long long x = idx[a] * g.M - 1 + i0[a] + ((q >> a) & 1);
                v[a] = x < 0 ? 0 : (x > g.ldim[L][a] - 1 ? g.ldim[L][a] - 1 : x);
            }
            const long long bit = (v[2] * g.ldim[L][1] + v[1]) * g.ldim[L][0] + v[0];
            atomicOr(&vmark[L][bit >> 5], 1u << (bit & 31));
        }
    }
};

template <int C>
struct MIPMax : NoHooks {
    float mx[C];
    __device__ __forceinline__ MIPMax() {
#pragma unroll
        for (int c = 0; c < C; ++c) mx[c] = -1.0f;
    }
    __device__ __forceinline__ bool sample(const float (&I)[C], float) {
#pragma unroll
        for (int c = 0; c < C; ++c) mx[c] = fmaxf(mx[c], I[c]);
        return false;
    }
};

__device__ __forceinline__ int find_camera(const CamParam* __restrict__ cams, int n, long long tile) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cams[mid].tile_begin <= tile)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void load_tables(const RenderArgs& a, int C, float4* s_tf, float* s_scl) {
    for (int i = threadIdx.x; i < C * 512; i += blockDim.x) s_tf[i] = a.tf[i];
    if (threadIdx.x < C) s_scl[threadIdx.x] = a.scl[threadIdx.x];
    __syncthreads();
}

template <int C, int VS, int MODE, bool POW2>
__global__ void __launch_bounds__(256) render_kernel(RenderArgs a) {
    extern __shared__ float4 s_tf[];
    __shared__ float s_scl[MAXC];
    load_tables(a, C, s_tf, s_scl);
    const int lane = threadIdx.x & 31;
    unsigned long long my_samples = 0, my_rays = 0;
    for (;;) {
        unsigned int tile = 0;
        if (lane == 0) tile = atomicAdd(a.counter, 1u);
        tile = __shfl_sync(0xffffffffu, tile, 0);
        if ((long long)tile >= a.total_tiles) break;
        const int ci = find_camera(a.cams, a.n_cams, tile);
        const CamParam& cp = a.cams[ci];
        const long long lt = (long long)tile - cp.tile_begin;
        const int px = (int)(lt % cp.tiles_x) * a.tile_w + lane % a.tile_w;
        const int py = (int)(lt / cp.tiles_x) * a.tile_h + lane / a.tile_w;
        if (px >= cp.W || py >= cp.H) continue;
        float d[3], t0, t1;
        float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ray_setup(cp, a.g, px, py, d, t0, t1)) {
            ++my_rays;
            if (MODE == 0) {
                DVRComposite<C> f{{}, s_tf, s_scl, cp.ert};
                my_samples += march<C, VS, POW2>(a.g, a.pool, a.rnodes, cp, d, t0, t1, f);
                out = make_float4(f.Cr, f.Cg, f.Cb, f.A);
            } else if (MODE == 2) {
                DVRFootprint<C> f;
                f.s_tf = s_tf;
                f.s_scl = s_scl;
                f.ert = cp.ert;
                f.vmark = a.vmark;
                f.nmark = a.nmark;
                my_samples += march<C, VS, POW2>(a.g, a.pool, a.rnodes, cp, d, t0, t1, f);
                out = make_float4(f.Cr, f.Cg, f.Cb, f.A);
            } else {
                MIPMax<C> f;
                const long long n = march<C, VS, POW2>(a.g, a.pool, a.rnodes, cp, d, t0, t1, f);
                my_samples += n;
                if (n > 0) {
                    float A = 0.f, Cr = 0.f, Cg = 0.f, Cb = 0.f;
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        TFLookup<C> t;
                        t.eval(s_tf, s_scl, c, f.mx[c]);
                        const float al = fminf(fmaxf(t.al, 0.0f), ALPHA_MAX);
                        const float w = (1.0f - A) * al;
                        Cr = fmaf(w, t.r, Cr);
                        Cg = fmaf(w, t.g, Cg);
                        Cb = fmaf(w, t.b, Cb);
                        A += w;
                    }
                    out = make_float4(Cr, Cg, Cb, A);
                }
            }
        }
        reinterpret_cast<float4*>(cp.img)[(long long)py * cp.W + px] = out;
    }
    for (int o = 16; o > 0; o >>= 1) {
        my_samples += __shfl_xor_sync(0xffffffffu, my_samples, o);
        my_rays += __shfl_xor_sync(0xffffffffu, my_rays, o);
    }
    if (lane == 0 && a.stats) {
        atomicAdd(&a.stats[0], my_samples);
        atomicAdd(&a.stats[1], my_rays);
    }
}

// Reverse-mode sweep in forward order.  With the final (C_f, A_f) of the ray known, the adjoint
// of the opacity after channel-step j is
//   gA_j+ = [ -gC.(C_f - C_j+) + gA_f (1 - A_f) ] / (1 - A_j+),
// and for the update C += (1-A) a rgb, A += (1-A) a:
//   dL/da_j   = (1 - A_j-) gC.rgb_j + [ -gC.(C_f - C_j+) + gA_f (1 - A_f) ] / (1 - a_j),
//   dL/drgb_j = gC (1 - A_j-) a_j,     da/dalpha = l (1 - a) / (1 - alpha).
template <int C>
struct DVRAdjoint : NoHooks {
    const float4* s_tf;
    const float* s_scl;
    float* s_dtf; // [C][256][4]
    float ert;
    float gC[3], gAf, Cf[3], Af;
    float A = 0.0f, Cp[3] = {0.0f, 0.0f, 0.0f};
    float dsc[C];
    __device__ __forceinline__ bool sample(const float (&I)[C], float ell) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            TFLookup<C> t;
            t.eval(s_tf, s_scl, c, I[c]);
            const bool clamped = !(t.al >= 0.0f && t.al <= ALPHA_MAX);
            const float al = fminf(fmaxf(t.al, 0.0f), ALPHA_MAX);
            float a, oma;
            opacity(al, ell, a, oma);
            const float T = 1.0f - A;
            const float w = T * a;
            Cp[0] = fmaf(w, t.r, Cp[0]);
            Cp[1] = fmaf(w, t.g, Cp[1]);
            Cp[2] = fmaf(w, t.b, Cp[2]);
            A += w;
            const float suffix = -(gC[0] * (Cf[0] - Cp[0]) + gC[1] * (Cf[1] - Cp[1]) + gC[2] * (Cf[2] - Cp[2])) +
                                 gAf * (1.0f - Af);
            const float ga = T * (gC[0] * t.r + gC[1] * t.g + gC[2] * t.b) + suffix / oma;
            const float gq[4] = {gC[0] * w, gC[1] * w, gC[2] * w, clamped ? 0.0f : ga * ell * oma / (1.0f - al)};
            float* e0 = s_dtf + (c * 256 + t.i) * 4;
            const float4 D = s_tf[(c * 256 + t.i) * 2 + 1];
            const float glam = gq[0] * D.x + gq[1] * D.y + gq[2] * D.z + gq[3] * D.w;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (gq[q] != 0.0f) {
                    atomicAdd(e0 + q, (1.0f - t.lam) * gq[q]);
                    atomicAdd(e0 + 4 + q, t.lam * gq[q]);
                }
            }
            if (t.xr > 0.0f && t.xr < 1.0f) dsc[c] += glam * 255.0f * I[c] * (1.0f / 65535.0f);
        }
        return A >= ert;
    }
};

template <int C, int VS, bool POW2>
__global__ void __launch_bounds__(256) render_backward_kernel(RenderArgs a) {
    extern __shared__ float4 s_tf[];
    __shared__ float s_scl[MAXC];
    float* s_dtf = reinterpret_cast<float*>(s_tf + C * 512);
    for (int i = threadIdx.x; i < C * 1024; i += blockDim.x) s_dtf[i] = 0.0f;
    load_tables(a, C, s_tf, s_scl);
    const int lane = threadIdx.x & 31;
    float dsc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) dsc[c] = 0.0f;
    for (;;) {
        unsigned int tile = 0;
        if (lane == 0) tile = atomicAdd(a.counter, 1u);
        tile = __shfl_sync(0xffffffffu, tile, 0);
        if ((long long)tile >= a.total_tiles) break;
        const int ci = find_camera(a.cams, a.n_cams, tile);
        const CamParam& cp = a.cams[ci];
        const long long lt = (long long)tile - cp.tile_begin;
        const int px = (int)(lt % cp.tiles_x) * a.tile_w + lane % a.tile_w;
        const int py = (int)(lt / cp.tiles_x) * a.tile_h + lane / a.tile_w;
        if (px >= cp.W || py >= cp.H) continue;
        float d[3], t0, t1;
        if (!ray_setup(cp, a.g, px, py, d, t0, t1)) continue;
        const float4 gl = reinterpret_cast<const float4*>(cp.dimg)[(long long)py * cp.W + px];
        if (gl.x == 0.0f && gl.y == 0.0f && gl.z == 0.0f && gl.w == 0.0f) continue;
        DVRComposite<C> fw{{}, s_tf, s_scl, cp.ert};
        march<C, VS, POW2>(a.g, a.pool, a.rnodes, cp, d, t0, t1, fw);
        DVRAdjoint<C> bw;
        bw.s_tf = s_tf;
        bw.s_scl = s_scl;
        bw.s_dtf = s_dtf;
        bw.ert = cp.ert;
        bw.gC[0] = gl.x;
        bw.gC[1] = gl.y;
        bw.gC[2] = gl.z;
        bw.gAf = gl.w;
        bw.Cf[0] = fw.Cr;
        bw.Cf[1] = fw.Cg;
        bw.Cf[2] = fw.Cb;
        bw.Af = fw.A;
#pragma unroll
        for (int c = 0; c < C; ++c) bw.dsc[c] = 0.0f;
        march<C, VS, POW2>(a.g, a.pool, a.rnodes, cp, d, t0, t1, bw);
#pragma unroll
        for (int c = 0; c < C; ++c) dsc[c] += bw.dsc[c];
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
        float v = dsc[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && v != 0.0f) atomicAdd(&a.dscale[c], v);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < C * 1024; i += blockDim.x)
        if (s_dtf[i] != 0.0f) atomicAdd(&a.dtf[i], s_dtf[i]);
}

template <int C, int VS>
static cudaError_t launch_fwd_c(const RenderArgs& a, int mode, int blocks, int threads, cudaStream_t st) {
    const size_t smem = (size_t)C * 512 * sizeof(float4);
    if (mode == 0) {
        if (a.g.pow2)
            render_kernel<C, VS, 0, true><<<blocks, threads, smem, st>>>(a);
        else
            render_kernel<C, VS, 0, false><<<blocks, threads, smem, st>>>(a);
    } else if (mode == 2) {
        if (a.g.pow2)
            render_kernel<C, VS, 2, true><<<blocks, threads, smem, st>>>(a);
        else
            render_kernel<C, VS, 2, false><<<blocks, threads, smem, st>>>(a);
    } else {
        if (a.g.pow2)
            render_kernel<C, VS, 1, true><<<blocks, threads, smem, st>>>(a);
        else
            render_kernel<C, VS, 1, false><<<blocks, threads, smem, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_render(const RenderArgs& a, int mode, int fp16, int blocks, int threads, cudaStream_t st) {
    (void)fp16;
    switch (a.g.C) {
        case 1: return launch_fwd_c<1, 1>(a, mode, blocks, threads, st);
        case 2: return launch_fwd_c<2, 2>(a, mode, blocks, threads, st);
        case 3: return launch_fwd_c<3, 4>(a, mode, blocks, threads, st);
        default: return launch_fwd_c<4, 4>(a, mode, blocks, threads, st);
    }
}

template <int C, int VS>
static cudaError_t launch_bwd_c(const RenderArgs& a, int blocks, int threads, cudaStream_t st) {
    const size_t smem = (size_t)C * 512 * sizeof(float4) + (size_t)C * 1024 * sizeof(float);
    if (a.g.pow2) {
        cudaFuncSetAttribute(render_backward_kernel<C, VS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        render_backward_kernel<C, VS, true><<<blocks, threads, smem, st>>>(a);
    } else {
        cudaFuncSetAttribute(render_backward_kernel<C, VS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        render_backward_kernel<C, VS, false><<<blocks, threads, smem, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_render_backward(const RenderArgs& a, int blocks, int threads, cudaStream_t st) {
    switch (a.g.C) {
        case 1: return launch_bwd_c<1, 1>(a, blocks, threads, st);
        case 2: return launch_bwd_c<2, 2>(a, blocks, threads, st);
        case 3: return launch_bwd_c<3, 4>(a, blocks, threads, st);
        default: return launch_bwd_c<4, 4>(a, blocks, threads, st);
    }
}

} // namespace vrk
