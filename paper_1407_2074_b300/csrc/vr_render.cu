// vr_render.cu -- ray casting of the bricked octree (Algorithm 1 and Sec. "Basic Ray-Casting")
// and its adjoint with respect to the transfer functions and intensity scales.
//
// Work decomposition: a persistent grid; every warp takes 32-ray tiles (tile_w x tile_h pixels)
// from one queue spanning all cameras of the call (batched views of uneven resolution share one
// launch).  Per ray:
//   setup      pinhole ray, slab test against the real volume box, clip half-spaces, t >= 0;
//   march      t_k = t0 + k dt while t_k < t1, last segment l = t1 - t_k;
//   LOD        L* = largest L with t_k >= t_L (thresholds precomputed per camera);
//   node       descent to level L* through the dense node tables, stopping at a node without
//              children; the node is cached until the sample leaves its box or L* rises above its
//              level, and the next lookup restarts at the lowest cached ancestor holding the sample
//              (the same node as a descent from the root);
//   intensity  AVG of a brick-less node, else trilinear inside the node's slot (the border
//              voxels make the eight corners one slot), corners re-read at every sample; two
//              consecutive samples of one brick node are shaded together before compositing;
//              a run of equal samples through a brick-less node is composited in closed form;
//   TF         x = sat(I s / 65535), entry i = min(floor(255 x), 254), linear (smem table);
//   composite  a = 1 - (1 - alpha)^l, C += T a rgb, T <- T (1 - a) per channel in order (T = 1 - A);
//   ERT        stop once A >= ert after a sample.
// Geometry (ray direction, interval, t_k, sample positions, level and node choice) uses only
// correctly rounded single-precision operations (_rn intrinsics, never contracted) in a fixed
// order, so these integer-valued decisions are reproducible off the GPU; interpolation, TF and
// compositing are ordinary FP32 with FMA.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math_constants.h>

#include <type_traits>

#include "vr_internal.h"

namespace vrk {

// Programmatic dependent launch within one vr_render: the tile-order scatter, the ray caster and
// the continuation are launched with programmatic stream serialization, so each launch is
// processed while the kernel before it drains; a kernel does its independent set-up (tables into
// shared memory, its own counting) and then waits here for the kernel before it to complete and
// its writes to be visible.  No kernel triggers its dependents early.  The wait does nothing in a
// kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

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

// Hardware square root and reciprocal approximations (one SFU operation each, relative error
// about 2^-22; flush-to-zero is harmless: the operands lie in [1e-6, 2]).
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Opacity correction a = 1 - (1 - alpha)^l and its complement (1 - alpha)^l, accurate for small
// alpha (no 1 - (1 - x) cancellation): for l = 1/2, a = alpha / (1 + sqrt(1 - alpha)).
__device__ __forceinline__ void opacity(float al, float ell, float& a, float& oma) {
    if (ell == 0.5f) {
        const float s = sqrt_approx(1.0f - al); // 1 - al >= 1e-6
        a = al * rcp_approx(1.0f + s);
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

// A uint16 voxel value h as the float 2^23 + h (exponent bits or'ed in, no conversion).  Sums and
// differences of such values are exact, so only the constant term of a cell removes the offset.
constexpr float VBIAS = 8388608.0f;
__device__ __forceinline__ float biased(uint32_t h) { return __uint_as_float(0x4B000000u | h); }

// 2^-e as a float, exactly (0 <= e < 126): the reciprocal of a power-of-two size without a division
__device__ __forceinline__ float pow2_neg(int e) { return __int_as_float((127 - e) << 23); }

constexpr float ALPHA_MAX = 1.0f - 1e-6f;
constexpr int MAX_SAMPLES = 1 << 24; // (float)k stays exact; bounds every ray

template <int C>
struct TFLookup {
    float r, g, b, al; // interpolated entry (al before clamping)
    float lam, xr;     // position between entries, unclamped x
    int i;
    __device__ __forceinline__ void eval(const float4* __restrict__ s_tf, const float* s_scl, int c, float I) {
        xr = I * s_scl[c];
        const float x = __saturatef(xr);
        const float w = x * 255.0f;
        // entry floor(255 x): at x = 1 that is entry 255 with lam = 0, whose difference to the next
        // entry is stored as 0, so it reads entry 255 itself (the value the segment 254..255
        // reaches at its end)
        i = (int)w;
        lam = w - (float)i;
        const float4 T = s_tf[c * 256 + i], D = s_tf[(C + c) * 256 + i];
        // two packed FP32 FMAs (each element rounded as fmaf)
        const float2 l2 = make_float2(lam, lam);
        const float2 rg = __ffma2_rn(l2, make_float2(D.x, D.y), make_float2(T.x, T.y));
        const float2 ba = __ffma2_rn(l2, make_float2(D.z, D.w), make_float2(T.z, T.w));
        r = rg.x;
        g = rg.y;
        b = ba.x;
        al = ba.y;
    }
};

// Emission-absorption compositing runs in two steps (DVRComposite below): a sample is shaded on
// its own over the channels into its local colour rgb_s and transmittance q_s, and then composited
// into the ray, C += T rgb_s, T *= q_s.  Only the second step depends on the ray's state.
struct Shaded {
    float r, g, b, q;
};

// Traversal state of one ray, shared by the one-lane march and the lane-group march: the level of
// detail L* of the current sample and the cached node -- its level, grid index, the faces of its
// box the ray heads for, and its brick slot or AVG.  Sample positions, L* and the node choice use
// only correctly rounded single-precision operations in a fixed order.  SK > 0: the slot edge
// M + 2 known at compile time (corner offsets become immediates); 0: read from the geometry.
template <int C, int VS, bool POW2, int SK = 0>
struct RayCursor {
    const Geo& g;
    const uint16_t* __restrict__ pool;
    const RNode* __restrict__ rn;
    const float* tl; // the camera's LOD thresholds (global memory)
    float eye[3], d[3];
    int N, M, S, mlog;
    int Lstar = 0;
    float tnext;
    // node cache
    int nlev = -1;
    float tl_limit = 0.0f;   // t at which L* would exceed the cached node's level
    float bnd[3] = {0, 0, 0}; // the node-box face each axis is heading for (+-inf at the grid ends)
    bool neg[3];
    int cidx[3] = {0, 0, 0};
    bool brick = false;
    const uint16_t* sbase = nullptr;
    float avg[C];
    float off[3] = {0, 0, 0};
    float inv_vox = 1.0f;

    __device__ __forceinline__ RayCursor(const Geo& g_, const uint16_t* pool_, const RNode* rn_, const CamParam& cp,
                                         const float dd[3])
        : g(g_), pool(pool_), rn(rn_), tl(cp.tl) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            eye[a] = cp.eye[a]; // in registers: cp lives in global memory
            d[a] = dd[a];
            neg[a] = !(dd[a] > 0.0f);
        }
        N = g.N;
        M = SK > 0 ? SK - 2 : g.M; // the launch picks SK == g.S
        S = SK > 0 ? SK : g.S;
        mlog = __ffs(M) - 1; // log2(M) when POW2
        tnext = N >= 1 ? cp.tl[1] : CUDART_INF_F;
    }
    __device__ __forceinline__ void position(float tk, float (&p)[3]) const {
#pragma unroll
        for (int a = 0; a < 3; ++a) p[a] = __fadd_rn(eye[a], __fmul_rn(tk, d[a]));
    }
    // L* = the largest L with tk >= t_L (t grows along the ray, so L* only rises)
    __device__ __forceinline__ void advance_lod(float tk) {
        while (tk >= tnext) {
            ++Lstar;
            tnext = (Lstar < N) ? tl[Lstar + 1] : CUDART_INF_F;
        }
    }
    // p inside the cached node's box.  With power-of-two node sizes positions move monotonically
    // along each axis, so only the face the ray is heading for can be crossed: (p < hi) for d > 0,
    // (p >= lo) otherwise.
    __device__ __forceinline__ bool in_box(const float (&p)[3]) const {
        bool in = true;
        if (POW2) {
#pragma unroll
            for (int a = 0; a < 3; ++a) in = in && ((p[a] < bnd[a]) != neg[a]);
        } else {
            const float size = (float)(M << nlev);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                int q = (int)floorf(__fdiv_rn(p[a], size));
                const int qm = (int)g.nb[nlev][a] - 1;
                q = q < 0 ? 0 : (q > qm ? qm : q);
                in = in && (q == cidx[a]);
            }
        }
        return in;
    }
    // the cached node is the one a descent would give for the sample at tk, p
    __device__ __forceinline__ bool holds(float tk, const float (&p)[3]) const {
        return nlev >= 0 && tk < tl_limit && in_box(p);
    }
    __device__ __forceinline__ long long node_id(int lev, const int (&idx)[3]) const {
        return g.noff[lev] + ((long long)idx[2] * g.nb[lev][1] + idx[1]) * g.nb[lev][0] + idx[0];
    }
    // getNodeAtPosition: descend from the root towards L*, stopping at a node without children,
    // and cache the node.  With power-of-two node sizes the descent restarts at the lowest
    // ancestor of the cached node whose box holds p (at level L* or above): every ancestor has
    // children, and from there the descent visits exactly the nodes the root descent would.
    template <class F>
    __device__ __forceinline__ void descend(const float (&p)[3], F& f) {
        int lev = N;
        int idx[3] = {0, 0, 0};
        if (POW2 && nlev >= 0) {
            for (int A = nlev + 1 > Lstar ? nlev + 1 : Lstar; A < N; ++A) {
                const int sh = A - nlev;
                const float inv = pow2_neg(mlog + A);
                bool in = true;
#pragma unroll
                for (int a = 0; a < 3; ++a) in = in && ((int)floorf(__fmul_rn(p[a], inv)) == (cidx[a] >> sh));
                if (in) {
                    lev = A;
#pragma unroll
                    for (int a = 0; a < 3; ++a) idx[a] = cidx[a] >> sh;
                    break;
                }
            }
        }
        const long long nid0 = node_id(lev, idx);
        RNode nd = rn[nid0];
        f.on_node(nid0);
        while (lev > Lstar && (nd.flags & F_CHILDREN)) {
            --lev;
            const float size = (float)(M << lev);
            const float inv = POW2 ? pow2_neg(mlog + lev) : 0.0f;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float qf = POW2 ? floorf(__fmul_rn(p[a], inv)) : floorf(__fdiv_rn(p[a], size));
                const int c0 = 2 * idx[a];
                int q = qf < (float)c0 ? c0 : (qf > (float)(c0 + 1) ? c0 + 1 : (int)qf);
                const int qm = (int)g.nb[lev][a] - 1;
                if (q > qm) q = qm;
                idx[a] = q;
            }
            const long long nid = node_id(lev, idx);
            nd = rn[nid];
            f.on_node(nid);
        }
        nlev = lev;
        tl_limit = (lev < N) ? tl[lev + 1] : CUDART_INF_F;
        const float size = (float)(M << lev);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cidx[a] = idx[a];
            if (d[a] > 0.0f)
                bnd[a] = (idx[a] == (int)g.nb[lev][a] - 1) ? CUDART_INF_F : (float)(idx[a] + 1) * size;
            else
                bnd[a] = (idx[a] == 0) ? -CUDART_INF_F : (float)idx[a] * size;
            off[a] = (float)(idx[a] * M) - 0.5f;
        }
        inv_vox = pow2_neg(lev);
        brick = (nd.flags & F_BRICK) && nd.slot >= 0 && nd.slot < g.n_slots_cap;
        sbase = brick ? pool + (long long)nd.slot * g.slot_elems : nullptr;
#pragma unroll
        for (int c = 0; c < C; ++c) avg[c] = (float)nd.avg[c];
    }
    // cell of position pp in the cached brick: corner index i0 (clamped into the slot) and fractions
    __device__ __forceinline__ const uint16_t* cell(const float (&pp)[3], float (&fr)[3], int (&i0)[3]) const {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float u = fmaf(pp[a], inv_vox, -off[a]); // == (p * 2^-L) - off: the product is exact
            const float fl = floorf(u);
            const int ii = (int)fl;
            fr[a] = __fsub_rn(u, fl);
            // in [0, M] with one unsigned minimum: the node's box keeps ii in [0, M]; any other
            // value (a negative one reads as a large unsigned) still lands inside the slot
            i0[a] = (int)min((unsigned)ii, (unsigned)M);
        }
        return sbase + ((i0[2] * S + i0[1]) * S + i0[0]) * VS;
    }
    __device__ __forceinline__ const uint16_t* corner(const uint16_t* cp0, int q) const {
        return cp0 + ((long long)(((q >> 2) & 1) * S + ((q >> 1) & 1)) * S + (q & 1)) * VS;
    }
    // FP32 trilinear at position pp inside the cached node's brick.  The eight corners of the cell
    // are re-read at every sample (L1 hits): a per-lane cell cache made the reload a branch that
    // some lane of the warp takes at almost every sample (lanes enter new cells at different
    // samples), which cost more than the loads it saved.  Corners are 2^23 + value (biased()), so
    // the polynomial coefficients are exact differences and only the constant term drops 2^23:
    //   I = k0 + kx fx + ky fy + kz fz + kxy fx fy + kxz fx fz + kyz fy fz + kxyz fx fy fz
    template <class F>
    __device__ __forceinline__ void trilinear(const float (&pp)[3], float (&out)[C], F& f) const {
        float fr[3];
        int i0[3];
        const uint16_t* cp0 = cell(pp, fr, i0);
        f.on_cell(g, nlev, cidx, i0);
        float w[8][C];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const uint16_t* v = corner(cp0, q);
            if (VS == 4) {
                const uint2 x = __ldg(reinterpret_cast<const uint2*>(v));
                const uint32_t ws[2] = {x.x, x.y};
#pragma unroll
                for (int c = 0; c < C; ++c) w[q][c] = biased((c & 1) ? (ws[c >> 1] >> 16) : (ws[c >> 1] & 0xffffu));
            } else if (VS == 2) {
                const uint32_t x = __ldg(reinterpret_cast<const unsigned int*>(v));
#pragma unroll
                for (int c = 0; c < C; ++c) w[q][c] = biased(c ? (x >> 16) : (x & 0xffffu));
            } else {
                w[q][0] = biased(__ldg(reinterpret_cast<const unsigned short*>(v)));
            }
        }
        const float fxy = fr[0] * fr[1], fxz = fr[0] * fr[2], fyz = fr[1] * fr[2], fxyz = fxy * fr[2];
        // channel pairs in packed FP32 (each element rounded as its scalar operation)
        auto sub2 = [](float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); };
        auto bcast2 = [](float x) { return make_float2(x, x); };
#pragma unroll
        for (int c = 0; c + 1 < C; c += 2) {
            float2 W[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) W[q] = make_float2(w[q][c], w[q][c + 1]);
            const float2 d10 = sub2(W[1], W[0]), d20 = sub2(W[2], W[0]), d40 = sub2(W[4], W[0]);
            const float2 d32 = sub2(W[3], W[2]), d54 = sub2(W[5], W[4]), d64 = sub2(W[6], W[4]);
            float2 v = __ffma2_rn(bcast2(fr[0]), d10, sub2(W[0], bcast2(VBIAS)));
            v = __ffma2_rn(bcast2(fr[1]), d20, v);
            v = __ffma2_rn(bcast2(fr[2]), d40, v);
            v = __ffma2_rn(bcast2(fxy), sub2(d32, d10), v);
            v = __ffma2_rn(bcast2(fxz), sub2(d54, d10), v);
            v = __ffma2_rn(bcast2(fyz), sub2(d64, d20), v);
            v = __ffma2_rn(bcast2(fxyz), sub2(sub2(sub2(W[7], W[6]), d54), sub2(d32, d10)), v);
            out[c] = v.x;
            out[c + 1] = v.y;
        }
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float v0 = w[0][c], v1 = w[1][c], v2 = w[2][c], v3 = w[3][c];
            const float v4 = w[4][c], v5 = w[5][c], v6 = w[6][c], v7 = w[7][c];
            if (c == C - 1 && (C & 1)) { // the odd channel out
                float v = fmaf(fr[0], v1 - v0, v0 - VBIAS);
                v = fmaf(fr[1], v2 - v0, v);
                v = fmaf(fr[2], v4 - v0, v);
                v = fmaf(fxy, (v3 - v2) - (v1 - v0), v);
                v = fmaf(fxz, (v5 - v4) - (v1 - v0), v);
                v = fmaf(fyz, (v6 - v4) - (v2 - v0), v);
                out[c] = fmaf(fxyz, ((v7 - v6) - (v5 - v4)) - ((v3 - v2) - (v1 - v0)), v);
            }
            if constexpr (F::kExactI) {
                // the same polynomial in double: its coefficients are exact integers and the
                // fractions exact floats, so this is the trilinear value to double rounding
                const double fx = fr[0], fy = fr[1], fz = fr[2];
                double e = (double)(v0 - VBIAS) + fx * (double)(v1 - v0);
                e += fy * (double)(v2 - v0) + fz * (double)(v4 - v0);
                e += fx * fy * (double)((v3 - v2) - (v1 - v0)) + fx * fz * (double)((v5 - v4) - (v1 - v0));
                e += fy * fz * (double)((v6 - v4) - (v2 - v0));
                f.Id[c] = e + fx * fy * fz * (double)(((v7 - v6) - (v5 - v4)) - ((v3 - v2) - (v1 - v0)));
            }
        }
    }
    // FP16 trilinear: corners as normalised half pairs, interpolated in half2
    template <class F>
    __device__ __forceinline__ void trilinear_h(const float (&pp)[3], float (&out)[C], F& f) const {
        constexpr int CP = (C + 1) / 2;
        float fr[3];
        int i0[3];
        const uint16_t* cp0 = cell(pp, fr, i0);
        f.on_cell(g, nlev, cidx, i0);
        __half2 hv[8][CP];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const uint16_t* v = corner(cp0, q);
            float cv[C];
            if (VS == 4) {
                const uint2 w = __ldg(reinterpret_cast<const uint2*>(v));
                const uint32_t ws[2] = {w.x, w.y};
#pragma unroll
                for (int c = 0; c < C; ++c) cv[c] = (float)((c & 1) ? (ws[c >> 1] >> 16) : (ws[c >> 1] & 0xffffu));
            } else if (VS == 2) {
                const uint32_t w = __ldg(reinterpret_cast<const unsigned int*>(v));
#pragma unroll
                for (int c = 0; c < C; ++c) cv[c] = (float)(c ? (w >> 16) : (w & 0xffffu));
            } else {
                cv[0] = (float)__ldg(reinterpret_cast<const unsigned short*>(v));
            }
            constexpr float inv = 1.0f / 65535.0f;
#pragma unroll
            for (int j = 0; j < CP; ++j)
                hv[q][j] = __floats2half2_rn(cv[2 * j] * inv, (2 * j + 1 < C) ? cv[2 * j + 1] * inv : 0.0f);
        }
        const __half2 fx = __float2half2_rn(fr[0]), fy = __float2half2_rn(fr[1]), fz = __float2half2_rn(fr[2]);
#pragma unroll
        for (int j = 0; j < CP; ++j) {
            const __half2 c00 = __hfma2(fx, __hsub2(hv[1][j], hv[0][j]), hv[0][j]);
            const __half2 c10 = __hfma2(fx, __hsub2(hv[3][j], hv[2][j]), hv[2][j]);
            const __half2 c01 = __hfma2(fx, __hsub2(hv[5][j], hv[4][j]), hv[4][j]);
            const __half2 c11 = __hfma2(fx, __hsub2(hv[7][j], hv[6][j]), hv[6][j]);
            const __half2 c0 = __hfma2(fy, __hsub2(c10, c00), c00);
            const __half2 c1 = __hfma2(fy, __hsub2(c11, c01), c01);
            const float2 r = __half22float2(__hfma2(fz, __hsub2(c1, c0), c0));
            out[2 * j] = r.x;
            if (2 * j + 1 < C) out[2 * j + 1] = r.y;
        }
    }
    // sample intensity inside a brick node: FP32 or (H) FP16 interpolation
    template <bool H, class F>
    __device__ __forceinline__ void interpolate(const float (&pp)[3], float (&out)[C], F& f) const {
        if constexpr (H)
            trilinear_h(pp, out, f);
        else
            trilinear(pp, out, f);
    }
    // intensity of a brick-less node: its AVG (normalised and rounded to FP16 when H)
    template <bool H, class F>
    __device__ __forceinline__ void average(float (&out)[C], F& f) const {
#pragma unroll
        for (int c = 0; c < C; ++c) out[c] = H ? __half2float(__float2half_rn(avg[c] * (1.0f / 65535.0f))) : avg[c];
        if constexpr (F::kExactI) {
#pragma unroll
            for (int c = 0; c < C; ++c) f.Id[c] = (double)avg[c];
        }
    }
    // sample kk has a full segment and lies in the cached node at the same level
    __device__ __forceinline__ bool in_run(int kk, float t0, float t1, float dt, int klim) const {
        if (kk >= klim) return false;
        const float t = __fadd_rn(t0, __fmul_rn((float)kk, dt));
        if (!(t < t1) || !(t < tl_limit) || !(__fsub_rn(t1, t) >= dt)) return false;
        float p[3];
        position(t, p);
        if (POW2) {
#pragma unroll
            for (int a = 0; a < 3; ++a)
                if ((p[a] < bnd[a]) == neg[a]) return false;
            return true;
        }
        return in_box(p);
    }
    // A brick-less node gives every sample the same intensity: the number n >= 1 of samples
    // k, k+1, ... (sample k, at tk, in the node with a full segment) that stay in the node with a
    // full segment, found with the same per-sample single-precision tests (monotone in k).
    __device__ __forceinline__ int run_length(int k, float tk, float t0, float t1, float dt, int klim) const {
        // estimate of the last sample in the node (fast divisions: the exact per-sample tests decide)
        float te = fminf(tl_limit, t1 - dt);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (d[a] != 0.0f) te = fminf(te, __fdividef(bnd[a] - eye[a], d[a]));
        }
        const float steps = floorf(__fdividef(te - tk, dt));
        const int ke = k + (steps > 0.0f ? (int)fminf(steps, 16777216.0f) : 0);
        int aa = k, bb;
        if (ke > k && in_run(ke, t0, t1, dt, klim)) {
            aa = ke;
            int st = 1;
            bb = ke + 1;
            while (in_run(bb, t0, t1, dt, klim)) {
                aa = bb;
                st *= 2;
                bb = aa + st;
            }
        } else {
            bb = ke > k ? ke : k + 1;
        }
        while (bb - aa > 1) {
            const int m = aa + (bb - aa) / 2;
            if (in_run(m, t0, t1, dt, klim))
                aa = m;
            else
                bb = m;
        }
        return aa - k + 1;
    }
};

// Marches one ray; calls f.sample(I[C], ell) for every sample until it returns true.
// H = false: I in raw uint16 units, FP32 interpolation.  H = true: the eight corners are cached as
// normalised FP16 channel pairs (value / 65535), interpolated in half2; I is that FP16 result.
// With a render cache (ca != nullptr) a node's brick is read from the cache when resident;
// otherwise it is requested and, in a full-frame pass, the brick of the parent or grandparent on
// the descent path stands in when resident (nearest first; missing ones are requested too), else
// the node's AVG (Sec. "Full-Frame Ray-Casting").  In a refinement pass (ca->refine) the ray
// stops at its first missing brick instead and march returns -(k + 1), k the sample to resume
// from (Sec. "Refinement Ray-Casting").  k0 is the first sample index.  With dry != nullptr the
// march also stops, returning -(k + 1), once *dry is set (checked every 16 steps) and more than
// min_left segment lengths of the ray remain: f then holds the state before sample k.
template <int C, int VS, bool POW2, bool H, class F, int SK = 0>
__device__ __forceinline__ long long march(const Geo& g, const uint16_t* __restrict__ pool,
                                           const RNode* __restrict__ rn, const CamParam& cp, const float d[3], float t0,
                                           float t1, F& f, const CacheArgs* ca = nullptr, int k0 = 0,
                                           int kend = MAX_SAMPLES, const unsigned* dry = nullptr, int min_left = 0) {
    // samples k0 <= k < min(kend, MAX_SAMPLES) inside [t0, t1)
    const float dt = cp.dt;
    const int klim = kend < MAX_SAMPLES ? kend : MAX_SAMPLES;
    RayCursor<C, VS, POW2, SK> cur(g, pool, rn, cp, d);
    const int N = cur.N, M = cur.M;
    int k = k0;
    float kf = (float)k0; // == (float)k, exact below 2^24
    unsigned steps = 0;
    for (;; ++k, kf += 1.0f) {
        const float tk = __fadd_rn(t0, __fmul_rn(kf, dt));
        if (!(tk < t1) || k >= klim) break;
        if (dry && (++steps & 15u) == 0u && *(volatile const unsigned*)dry != 0u &&
            __fsub_rn(t1, tk) > (float)min_left * dt)
            return -(long long)(k + 1);
        const float ell = fminf(dt, __fsub_rn(t1, tk));
        float p[3];
        cur.position(tk, p);
        cur.advance_lod(tk);
        if (!cur.holds(tk, p)) {
            cur.descend(p, f);
            if (ca && cur.brick) {
                const int lev = cur.nlev;
                const long long nid = cur.node_id(lev, cur.cidx);
                const int cs = ca->cslot[nid];
                if (cs >= 0) {
                    ca->used[nid] = 1;
                    cur.sbase = ca->cache + (long long)cs * g.slot_elems;
                } else {
                    ca->req[nid] = 1;
                    if (ca->refine) return -(long long)(k + 1);
                    cur.brick = false;
                    cur.sbase = nullptr;
                    for (int up = 1; up <= 2 && lev + up <= N; ++up) {
                        const int L2 = lev + up;
                        const int i2[3] = {cur.cidx[0] >> up, cur.cidx[1] >> up, cur.cidx[2] >> up};
                        const long long n2 = cur.node_id(L2, i2);
                        if (!(rn[n2].flags & F_BRICK)) continue;
                        const int c2 = ca->cslot[n2];
                        if (c2 < 0) {
                            ca->req[n2] = 1;
                        } else if (!cur.brick) {
                            cur.brick = true;
                            ca->used[n2] = 1;
                            cur.sbase = ca->cache + (long long)c2 * g.slot_elems;
#pragma unroll
                            for (int a = 0; a < 3; ++a) cur.off[a] = (float)(i2[a] * M) - 0.5f;
                            cur.inv_vox = pow2_neg(L2);
                        }
                    }
                }
            }
        }
        float I[C];
        if constexpr (F::kPairs) {
            // A brick sample takes the next sample too when it lies in the same brick node at the
            // same level with a full segment: both are shaded before the two are composited in
            // order, so the gathers and lookups of the second overlap those of the first.  A sample
            // without such a partner -- and a sample of a brick-less node that starts no run --
            // takes the same code with itself as the partner, composited once: every lane of the
            // warp meets at one copy of the shading in the loop.
            bool two = false;
            const float kf2 = kf + 1.0f;
            float I2[C];
            if (cur.brick) {
                float p2[3] = {p[0], p[1], p[2]};
                if (ell == dt && k + 1 < klim) {
                    const float tk2 = __fadd_rn(t0, __fmul_rn(kf2, dt));
                    if (tk2 < t1 && __fsub_rn(t1, tk2) >= dt && tk2 < cur.tnext && tk2 < cur.tl_limit) {
                        float q[3];
                        cur.position(tk2, q);
                        if (cur.in_box(q)) {
                            two = true;
#pragma unroll
                            for (int a = 0; a < 3; ++a) p2[a] = q[a];
                        }
                    }
                }
                cur.template interpolate<H>(p, I, f);
                cur.template interpolate<H>(p2, I2, f);
            } else {
                cur.template average<H>(I, f);
                if constexpr (F::kRuns) if (ell == dt) {
                    // composite the run of equal samples through this brick-less node in one step
                    const int n = cur.run_length(k, tk, t0, t1, dt, klim);
                    if (n >= 2) {
                        bool stop = false;
                        const int used = (int)f.run(I, n, dt, stop);
                        k += used - 1;
                        kf = (float)k;
                        if (stop) {
                            ++k;
                            break;
                        }
                        continue;
                    }
                }
#pragma unroll
                for (int c = 0; c < C; ++c) I2[c] = I[c];
            }
            const int st = f.sample2(I, I2, ell, two);
            if (st == 1) {
                ++k;
                break;
            }
            if (two) {
                ++k;
                kf = kf2;
                if (st == 2) {
                    ++k;
                    break;
                }
            }
        } else {
            if (cur.brick) {
                cur.template interpolate<H>(p, I, f);
            } else {
                cur.template average<H>(I, f);
                if constexpr (F::kRuns) if (ell == dt) {
                    // composite the run of equal samples through this brick-less node in one step
                    const int n = cur.run_length(k, tk, t0, t1, dt, klim);
                    if (n >= 2) {
                        bool stop = false;
                        const int used = (int)f.run(I, n, dt, stop);
                        k += used - 1;
                        kf = (float)k;
                        if (stop) {
                            ++k;
                            break;
                        }
                        continue;
                    }
                }
            }
            if (f.sample(I, ell)) {
                ++k;
                break;
            }
        }
    }
    return k;
}

// Lane-group march (DVR): the 2^lg lanes of one group march one ray together, lane j shading
// samples k + j of each step in lockstep; every lane of the group then composites the shaded
// samples in order (the second step of the two-step composite), so the group ends
// each step with the same ray state in every lane and stops at the same sample.  A step ends at the
// group's first sample in a brick-less node with a full segment: as in the one-lane march, that
// sample starts a run of equal samples, which its lane composites in closed form and shares.  The
// samples composited, the runs and the stop are those of march(), so the image is bit for bit the
// one-lane image.  gmask: the group's lanes; gbase: its first lane; j: this lane's place in it;
// k0: the first sample (f holds the ray state before it); s_grp: the warp's 32 shared-memory slots.
template <int C, int VS, bool POW2, bool H, class F, int SK = 0>
__device__ __forceinline__ long long march_group(const Geo& g, const uint16_t* __restrict__ pool,
                                                 const RNode* __restrict__ rn, const CamParam& cp, const float d[3],
                                                 float t0, float t1, F& f, int lg, unsigned gmask, int gbase, int j,
                                                 int k0, float4* s_grp) {
    const float dt = cp.dt;
    const int G = 1 << lg;
    const int lane = gbase + j;
    const unsigned gbits = gmask >> gbase; // the group's lanes as bits 0 .. G-1
    RayCursor<C, VS, POW2, SK> cur(g, pool, rn, cp, d);
    int k = k0;
    for (;;) {
        const int kk = k + j;
        const float tk = __fadd_rn(t0, __fmul_rn((float)kk, dt));
        const bool act = tk < t1 && kk < MAX_SAMPLES;
        bool starts_run = false;
        Shaded s{0.0f, 0.0f, 0.0f, 1.0f};
        float I[C];
        float ell = dt;
        if (act) {
            ell = fminf(dt, __fsub_rn(t1, tk));
            float p[3];
            cur.position(tk, p);
            cur.advance_lod(tk);
            if (!cur.holds(tk, p)) cur.descend(p, f);
            if (cur.brick) {
                cur.template interpolate<H>(p, I, f);
                s = f.shade(I, ell);
            } else {
                cur.template average<H>(I, f);
                if (F::kRuns && ell == dt)
                    starts_run = true;
                else
                    s = f.shade(I, ell);
            }
        }
        const unsigned run_bits = (__ballot_sync(gmask, starts_run) >> gbase) & gbits;
        const unsigned end_bits = (__ballot_sync(gmask, !act) >> gbase) & gbits;
        const int jr = run_bits ? __ffs(run_bits) - 1 : G; // first sample that starts a run
        const int je = end_bits ? __ffs(end_bits) - 1 : G; // first sample past the ray's end
        const int jl = jr < je ? jr : je;
        // The in-order update of the ray by the step's shaded samples 0 .. jl-1, through the warp's
        // shared-memory slots (one store per lane, broadcast reads): the reads do not depend on the
        // chain, so they run ahead of it, and no branch leaves the loop early -- once the ray
        // stops, the later samples are skipped, leaving the same state as update() one by one.
        s_grp[lane] = make_float4(s.r, s.g, s.b, s.q);
        __syncwarp(gmask);
        int stop_at = -1;
#pragma unroll 4
        for (int q = 0; q < jl; ++q) {
            const float4 v = s_grp[gbase + q];
            if (stop_at < 0) {
                f.Cr = fmaf(f.T, v.x, f.Cr);
                f.Cg = fmaf(f.T, v.y, f.Cg);
                f.Cb = fmaf(f.T, v.z, f.Cb);
                f.T *= v.w;
                if (1.0f - f.T >= f.ert) stop_at = q;
            }
        }
        __syncwarp(gmask); // the slots are read before the next step writes them
        if (stop_at >= 0) return k + stop_at + 1;
        if (jl == G) {
            k += G;
            continue;
        }
        if (je < jr) return k + je;
        // sample k + jr starts a run: its lane finds the run's length and composites it
        k += jr;
        int used = 0;
        bool stop = false;
        if (j == jr) {
            const int n = cur.run_length(kk, tk, t0, t1, dt, MAX_SAMPLES);
            if (n >= 2) {
                used = (int)f.run(I, n, dt, stop);
            } else {
                stop = f.sample(I, ell);
                used = 1;
            }
        }
        f.bcast(gmask, gbase + jr);
        used = __shfl_sync(gmask, used, gbase + jr);
        stop = __shfl_sync(gmask, (int)stop, gbase + jr) != 0;
        k += used;
        if (stop) return k;
    }
}

// March with a per-channel affine sample transform (Sec. "Correction of Chromatic Aberration"):
// channel c samples at q_c = X_c p, X_c a 3x4 matrix applied in single precision in a fixed order
// (((m0 p0 + m1 p1) + m2 p2) + m3).  Each channel descends from its own point and keeps its own
// node cache; the node test checks both faces because rounded transformed positions
// need not be monotone.  Samples are composited one by one (no closed-form runs).
template <int C, int VS, bool POW2, class F, int SK = 0>
__device__ __forceinline__ long long march_xf(const Geo& g, const uint16_t* __restrict__ pool,
                                              const RNode* __restrict__ rn, const CamParam& cp, const float d[3],
                                              float t0, float t1, const float (*xf)[12], F& f) {
    const float dt = cp.dt;
    // SK: the slot edge as a compile-time constant (0: read from the geometry)
    const int N = g.N, M = SK > 0 ? SK - 2 : g.M, S = SK > 0 ? SK : g.S;
    int Lstar = 0;
    float tnext = (N >= 1) ? cp.tl[1] : CUDART_INF_F;
    int nlev[C];
    float tl_limit[C], lo[C][3], hi[C][3], off[C][3], inv_vox[C], avg[C], cv[C][8];
    const uint16_t* sbase[C];
    bool brick[C];
    int cidx[C][3];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        nlev[c] = -1;
        tl_limit[c] = 0.0f;
        brick[c] = false;
        sbase[c] = nullptr;
    }
    int k = 0;
    float kf = 0.0f;
    for (;; ++k, kf += 1.0f) {
        const float tk = __fadd_rn(t0, __fmul_rn(kf, dt));
        if (!(tk < t1) || k >= MAX_SAMPLES) break;
        const float ell = fminf(dt, __fsub_rn(t1, tk));
        float p[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) p[a] = __fadd_rn(cp.eye[a], __fmul_rn(tk, d[a]));
        while (tk >= tnext) {
            ++Lstar;
            tnext = (Lstar < N) ? cp.tl[Lstar + 1] : CUDART_INF_F;
        }
        float I[C];
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float* m = xf[c];
            float q[3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
                q[i] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(m[4 * i], p[0]), __fmul_rn(m[4 * i + 1], p[1])),
                                           __fmul_rn(m[4 * i + 2], p[2])),
                                 m[4 * i + 3]);
            bool valid = nlev[c] >= 0 && tk < tl_limit[c];
            if (valid) {
                if (POW2) {
#pragma unroll
                    for (int a = 0; a < 3; ++a) valid = valid && (q[a] >= lo[c][a]) && (q[a] < hi[c][a]);
                } else {
                    const float size = (float)(M << nlev[c]);
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        int qq = (int)floorf(__fdiv_rn(q[a], size));
                        const int qm = (int)g.nb[nlev[c]][a] - 1;
                        qq = qq < 0 ? 0 : (qq > qm ? qm : qq);
                        valid = valid && (qq == cidx[c][a]);
                    }
                }
            }
            if (!valid) {
                int lev = N;
                int idx[3] = {0, 0, 0};
                if (POW2 && nlev[c] >= 0) {
                    // restart at the lowest ancestor of the channel's cached node that holds q
                    const int mlog = __ffs(M) - 1;
                    for (int A = nlev[c] + 1 > Lstar ? nlev[c] + 1 : Lstar; A < N; ++A) {
                        const int sh = A - nlev[c];
                        const float inv = pow2_neg(mlog + A);
                        bool in = true;
#pragma unroll
                        for (int a = 0; a < 3; ++a) in = in && ((int)floorf(__fmul_rn(q[a], inv)) == (cidx[c][a] >> sh));
                        if (in) {
                            lev = A;
#pragma unroll
                            for (int a = 0; a < 3; ++a) idx[a] = cidx[c][a] >> sh;
                            break;
                        }
                    }
                }
                RNode nd = rn[g.noff[lev] + ((long long)idx[2] * g.nb[lev][1] + idx[1]) * g.nb[lev][0] + idx[0]];
                while (lev > Lstar && (nd.flags & F_CHILDREN)) {
                    --lev;
                    const float size = (float)(M << lev);
                    const float inv = 1.0f / size;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const float qf = POW2 ? floorf(__fmul_rn(q[a], inv)) : floorf(__fdiv_rn(q[a], size));
                        const int c0 = 2 * idx[a];
                        int qq = qf < (float)c0 ? c0 : (qf > (float)(c0 + 1) ? c0 + 1 : (int)qf);
                        const int qm = (int)g.nb[lev][a] - 1;
                        if (qq > qm) qq = qm;
                        idx[a] = qq;
                    }
                    nd = rn[g.noff[lev] + ((long long)idx[2] * g.nb[lev][1] + idx[1]) * g.nb[lev][0] + idx[0]];
                }
                nlev[c] = lev;
                tl_limit[c] = (lev < N) ? cp.tl[lev + 1] : CUDART_INF_F;
                const float size = (float)(M << lev);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    cidx[c][a] = idx[a];
                    lo[c][a] = (idx[a] == 0) ? -CUDART_INF_F : (float)idx[a] * size;
                    hi[c][a] = (idx[a] == (int)g.nb[lev][a] - 1) ? CUDART_INF_F : (float)(idx[a] + 1) * size;
                    off[c][a] = (float)(idx[a] * M) - 0.5f;
                }
                inv_vox[c] = 1.0f / (float)(1 << lev);
                brick[c] = (nd.flags & F_BRICK) && nd.slot >= 0 && nd.slot < g.n_slots_cap;
                sbase[c] = brick[c] ? pool + (long long)nd.slot * g.slot_elems : nullptr;
                avg[c] = (float)nd.avg[c];
            }
            if (brick[c]) {
                float fr[3];
                int i0[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float u = fmaf(q[a], inv_vox[c], -off[c][a]); // exact product, one rounding
                    const float fl = floorf(u);
                    const int ii = (int)fl;
                    fr[a] = __fsub_rn(u, fl);
                    i0[a] = ii < 0 ? 0 : (ii > M ? M : ii); // a transformed point may leave the volume
                }
                const int coff = ((i0[2] * S + i0[1]) * S + i0[0]) * VS;
                {
                    // corners re-read at every sample (no divergent per-lane cell cache)
                    float v[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        v[e] = biased(__ldg(sbase[c] + coff + ((((e >> 2) & 1) * S + ((e >> 1) & 1)) * S + (e & 1)) * VS + c));
                    cv[c][0] = v[0] - VBIAS;
                    cv[c][1] = v[1] - v[0];
                    cv[c][2] = v[2] - v[0];
                    cv[c][4] = v[4] - v[0];
                    cv[c][3] = (v[3] - v[2]) - (v[1] - v[0]);
                    cv[c][5] = (v[5] - v[4]) - (v[1] - v[0]);
                    cv[c][6] = (v[6] - v[4]) - (v[2] - v[0]);
                    cv[c][7] = ((v[7] - v[6]) - (v[5] - v[4])) - ((v[3] - v[2]) - (v[1] - v[0]));
                }
                float r = fmaf(fr[0], cv[c][1], cv[c][0]);
                r = fmaf(fr[1], cv[c][2], r);
                r = fmaf(fr[2], cv[c][4], r);
                r = fmaf(fr[0] * fr[1], cv[c][3], r);
                r = fmaf(fr[0] * fr[2], cv[c][5], r);
                r = fmaf(fr[1] * fr[2], cv[c][6], r);
                I[c] = fmaf(fr[0] * fr[1] * fr[2], cv[c][7], r);
                if constexpr (F::kExactI) {
                    const double fx = fr[0], fy = fr[1], fz = fr[2];
                    double e = (double)cv[c][0] + fx * (double)cv[c][1] + fy * (double)cv[c][2] + fz * (double)cv[c][4];
                    e += fx * fy * (double)cv[c][3] + fx * fz * (double)cv[c][5] + fy * fz * (double)cv[c][6];
                    f.Id[c] = e + fx * fy * fz * (double)cv[c][7];
                }
            } else {
                I[c] = avg[c];
                if constexpr (F::kExactI) f.Id[c] = (double)avg[c];
            }
        }
        if (f.sample(I, ell)) {
            ++k;
            break;
        }
    }
    return k;
}

struct NoHooks {
    static constexpr bool kRuns = false; // composites runs of equal samples in closed form
    static constexpr bool kPairs = false; // has sample2 (two samples shaded together)
    static constexpr bool kExactI = false; // the march also stores the double intensity in Id[C]
    __device__ __forceinline__ void on_node(long long) {}
    __device__ __forceinline__ void on_cell(const Geo&, int, const int*, const int*) {}
};

// n samples of one constant intensity, each a per-sample transfer T' = T q, C' = C + T K:
// after j samples T_j = T q^j and C_j = C + T K (1 - q^j) / (1 - q).  Early termination at the
// first j with 1 - T q^j >= ert.  ln q and 1 - q^j come from log1p/expm1 (no cancellation).
// State in transmittance form (T = 1 - A).
__device__ __forceinline__ long long composite_run(float lnq, const float K[3], long long n, float ert, float& T,
                                                   float& Cr, float& Cg, float& Cb, bool& stop) {
    const float T0 = T;
    long long j = n;
    stop = false;
    if (lnq < 0.0f && ert <= 1.0f) {
        const float target = (1.0f - ert) / T0;
        float jj = (target >= 1.0f) ? 1.0f : ceilf(logf(target) / lnq);
        if (jj < 1.0f) jj = 1.0f;
        if (jj <= (float)n) {
            j = (long long)jj;
            stop = true;
        }
    }
    const float S = (lnq < 0.0f) ? expm1f((float)j * lnq) / expm1f(lnq) : (float)j;
    Cr = fmaf(T0 * K[0], S, Cr);
    Cg = fmaf(T0 * K[1], S, Cg);
    Cb = fmaf(T0 * K[2], S, Cb);
    T = T0 * expf((float)j * lnq);
    return j;
}

// Emission-absorption compositing in two steps.  A sample is first shaded on its own, over the
// channels in order (the composite sits inside the channel loop of Algorithm 1):
//   P_0 = 1,  rgb_s += P_c a_c rgb_c,  P_{c+1} = P_c (1 - a_c),  q_s = P_C;
// then composited into the ray: C += T rgb_s, T *= q_s (T = 1 - A, the transmittance), and the ray
// stops once 1 - T >= ert.  Only the second step depends on the ray's state, so samples shaded by
// different lanes and composited in order by each of them give the same bits as one lane marching
// alone, in single steps, in pairs or in any grouping.
template <int C, bool RUNS = true, bool PAIRS = RUNS>
struct DVRComposite : NoHooks {
    static constexpr bool kRuns = RUNS;
    static constexpr bool kPairs = PAIRS;
    const float4* s_tf;
    const float* s_scl;
    float ert;
    float T = 1.0f, Cr = 0.0f, Cg = 0.0f, Cb = 0.0f;
    __device__ __forceinline__ Shaded shade(const float (&I)[C], float ell) const {
        Shaded s{0.0f, 0.0f, 0.0f, 1.0f};
#pragma unroll
        for (int c = 0; c < C; ++c) {
            TFLookup<C> t;
            t.eval(s_tf, s_scl, c, I[c]);
            const float al = fminf(fmaxf(t.al, 0.0f), ALPHA_MAX);
            float a, oma;
            opacity(al, ell, a, oma);
            const float w = s.q * a;
            const float2 rg = __ffma2_rn(make_float2(w, w), make_float2(t.r, t.g), make_float2(s.r, s.g));
            s.r = rg.x;
            s.g = rg.y;
            s.b = fmaf(w, t.b, s.b);
            s.q *= oma;
        }
        return s;
    }
    __device__ __forceinline__ bool update(const Shaded& s) {
        const float2 rg = __ffma2_rn(make_float2(T, T), make_float2(s.r, s.g), make_float2(Cr, Cg));
        Cr = rg.x;
        Cg = rg.y;
        Cb = fmaf(T, s.b, Cb);
        T *= s.q;
        return 1.0f - T >= ert;
    }
    __device__ __forceinline__ long long run(const float (&I)[C], long long n, float ell, bool& stop) {
        float lnq = 0.0f, K[3];
        const Shaded s = shade(I, ell);
        K[0] = s.r;
        K[1] = s.g;
        K[2] = s.b;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            TFLookup<C> t;
            t.eval(s_tf, s_scl, c, I[c]);
            lnq += ell * log1pf(-fminf(fmaxf(t.al, 0.0f), ALPHA_MAX));
        }
        return composite_run(lnq, K, n, ert, T, Cr, Cg, Cb, stop);
    }
    // Two samples shaded first (their gathers and lookups overlap), the first with segment ell,
    // the second with a full one, then composited in order -- the second only when two.  Returns 1
    // when the first sample terminates the ray (the second is dropped), 2 when the second does,
    // else 0.
    __device__ __forceinline__ int sample2(const float (&I1)[C], const float (&I2)[C], float ell, bool two) {
        const Shaded s1 = shade(I1, ell), s2 = shade(I2, ell);
        if (update(s1)) return 1;
        if (!two) return 0;
        return update(s2) ? 2 : 0;
    }
    __device__ __forceinline__ bool sample(const float (&I)[C], float ell) { return update(shade(I, ell)); }
    __device__ __forceinline__ float alpha() const { return 1.0f - T; }
    // the ray state of lane src to the lanes of mask (lane-group march)
    __device__ __forceinline__ void bcast(unsigned mask, int src) {
        T = __shfl_sync(mask, T, src);
        Cr = __shfl_sync(mask, Cr, src);
        Cg = __shfl_sync(mask, Cg, src);
        Cb = __shfl_sync(mask, Cb, src);
    }
};

// FP16 variant of the DVR functor: I is the FP16-interpolated normalised intensity; the
// transfer-function lookup reads a half table (entry, next - entry) and interpolates in half2;
// opacity correction and compositing stay FP32 (the same two steps as above).
struct __align__(16) HalfEntry {
    __half2 rg, ba, drg, dba;
};

template <int C>
struct DVRCompositeH : NoHooks {
    static constexpr bool kRuns = true;
    static constexpr bool kPairs = true;
    const HalfEntry* s_tfh;
    const __half* s_sh; // per-channel scale s (normalised intensities)
    float ert;
    float T = 1.0f, Cr = 0.0f, Cg = 0.0f, Cb = 0.0f;
    __device__ __forceinline__ void lookup(int c, float I, float2& rg, float2& ba) const {
        const __half x = __hmul_sat(__float2half_rn(I), s_sh[c]);
        const float w = __half2float(x) * 255.0f;
        const int i = (int)w; // entry 255 at x = 1 (its difference is 0), as in TFLookup
        const __half2 lam = __float2half2_rn(w - (float)i);
        const HalfEntry e = s_tfh[c * 256 + i];
        rg = __half22float2(__hfma2(lam, e.drg, e.rg));
        ba = __half22float2(__hfma2(lam, e.dba, e.ba));
    }
    __device__ __forceinline__ Shaded shade(const float (&I)[C], float ell) const {
        Shaded s{0.0f, 0.0f, 0.0f, 1.0f};
#pragma unroll
        for (int c = 0; c < C; ++c) {
            float2 rg, ba;
            lookup(c, I[c], rg, ba);
            const float al = fminf(fmaxf(ba.y, 0.0f), ALPHA_MAX);
            float a, oma;
            opacity(al, ell, a, oma);
            const float w = s.q * a;
            s.r = fmaf(w, rg.x, s.r);
            s.g = fmaf(w, rg.y, s.g);
            s.b = fmaf(w, ba.x, s.b);
            s.q *= oma;
        }
        return s;
    }
    __device__ __forceinline__ bool update(const Shaded& s) {
        Cr = fmaf(T, s.r, Cr);
        Cg = fmaf(T, s.g, Cg);
        Cb = fmaf(T, s.b, Cb);
        T *= s.q;
        return 1.0f - T >= ert;
    }
    __device__ __forceinline__ long long run(const float (&I)[C], long long n, float ell, bool& stop) {
        float lnq = 0.0f, K[3];
        const Shaded s = shade(I, ell);
        K[0] = s.r;
        K[1] = s.g;
        K[2] = s.b;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            float2 rg, ba;
            lookup(c, I[c], rg, ba);
            lnq += ell * log1pf(-fminf(fmaxf(ba.y, 0.0f), ALPHA_MAX));
        }
        return composite_run(lnq, K, n, ert, T, Cr, Cg, Cb, stop);
    }
    __device__ __forceinline__ int sample2(const float (&I1)[C], const float (&I2)[C], float ell, bool two) {
        const Shaded s1 = shade(I1, ell), s2 = shade(I2, ell);
        if (update(s1)) return 1;
        if (!two) return 0;
        return update(s2) ? 2 : 0;
    }
    __device__ __forceinline__ bool sample(const float (&I)[C], float ell) { return update(shade(I, ell)); }
    __device__ __forceinline__ float alpha() const { return 1.0f - T; }
    // the ray state of lane src to the lanes of mask (lane-group march)
    __device__ __forceinline__ void bcast(unsigned mask, int src) {
        T = __shfl_sync(mask, T, src);
        Cr = __shfl_sync(mask, Cr, src);
        Cg = __shfl_sync(mask, Cg, src);
        Cb = __shfl_sync(mask, Cb, src);
    }
};

// DVR that also records the distinct (level, voxel) pairs read by trilinear corners and the
// node entries visited: the algorithmic footprint of a frame (measurement only).  Samples one by one
// (no pairs), so that no sample past the stop is read.
template <int C>
struct DVRFootprint : DVRComposite<C, true, false> {
    unsigned int* const* vmark;
    unsigned int* nmark;
    __device__ __forceinline__ void on_node(long long nid) {
        atomicOr(&nmark[nid >> 5], 1u << (nid & 31));
    }
    __device__ __forceinline__ void on_cell(const Geo& g, int L, const int* idx, const int* i0) {
        for (int q = 0; q < 8; ++q) {
            long long v[3];
            for (int a = 0; a < 3; ++a) {
                long long x = (long long)idx[a] * g.M - 1 + i0[a] + ((q >> a) & 1);
                v[a] = x < 0 ? 0 : (x > g.ldim[L][a] - 1 ? g.ldim[L][a] - 1 : x);
            }
            const long long bit = (v[2] * g.ldim[L][1] + v[1]) * g.ldim[L][0] + v[0];
            atomicOr(&vmark[L][bit >> 5], 1u << (bit & 31));
        }
    }
};

template <int C>
struct MIPMax : NoHooks {
    static constexpr bool kRuns = true;
    float mx[C];
    __device__ __forceinline__ long long run(const float (&I)[C], long long n, float, bool& stop) {
#pragma unroll
        for (int c = 0; c < C; ++c) mx[c] = fmaxf(mx[c], I[c]);
        stop = false;
        return n;
    }
    __device__ __forceinline__ MIPMax() {
#pragma unroll
        for (int c = 0; c < C; ++c) mx[c] = -1.0f;
    }
    __device__ __forceinline__ bool sample(const float (&I)[C], float) {
#pragma unroll
        for (int c = 0; c < C; ++c) mx[c] = fmaxf(mx[c], I[c]);
        return false;
    }
    static constexpr bool kPairs = true;
    __device__ __forceinline__ int sample2(const float (&I1)[C], const float (&I2)[C], float, bool) {
#pragma unroll
        for (int c = 0; c < C; ++c) mx[c] = fmaxf(mx[c], fmaxf(I1[c], I2[c]));
        return 0;
    }
};

// Pixel of a lane in tile lt of its camera: tiles in raster order, tile_w x tile_h lanes (both
// powers of two, tile_w * tile_h = 32); 32-bit index arithmetic (a camera has < 2^31 tiles).
__device__ __forceinline__ void tile_pixel(long long lt, int tiles_x, int tile_w, int tile_h, int lane, int& px, int& py) {
    const unsigned t = (unsigned)lt, tx = (unsigned)tiles_x;
    const unsigned row = t / tx;
    const int sh = __ffs(tile_w) - 1;
    px = (int)(t - row * tx) * tile_w + (lane & (tile_w - 1));
    py = (int)row * tile_h + (lane >> sh);
}

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
    // entries in s_tf[0, C*256), differences in s_tf[C*256, 2*C*256): 16-byte strides keep lanes
    // with different entries on different banks
    for (int i = threadIdx.x; i < C * 512; i += blockDim.x) s_tf[(i & 1) * C * 256 + (i >> 1)] = a.tf[i];
    if (threadIdx.x < C) s_scl[threadIdx.x] = a.scl[threadIdx.x];
    __syncthreads();
}

#ifndef VR_RENDER_MIN_CTAS
#define VR_RENDER_MIN_CTAS 3 // resident 256-thread CTAs per SM the register budget is sized for
#endif
// The persistent ray casters run 768 resident threads per SM in CTAs of 64 to 768 threads: the
// same register budget as three 256-thread CTAs (at most 85 per thread), and by default one
// 768-thread CTA per SM, so that the SM holds one copy of the transfer-function tables (24 KB)
// and leaves the rest to L1 (24 GiB orbit: 1.835 -> 1.790 ms per frame against 3 x 256).
constexpr int RENDER_MAX_THREADS = 768;
constexpr int RENDER_MAX_WARPS = RENDER_MAX_THREADS / 32;

// The tables of the forward kernels: FP32 entries and differences, and with H their half
// copies (entry, difference) after them and the half scales.
template <int C, bool H>
__device__ __forceinline__ void load_render_tables(const RenderArgs& a, float4* s_tf, float* s_scl, __half* s_sh) {
    load_tables(a, C, s_tf, s_scl);
    if (H) {
        HalfEntry* s_tfh = reinterpret_cast<HalfEntry*>(s_tf + C * 512);
        for (int i = threadIdx.x; i < C * 256; i += blockDim.x) {
            const float4 T = s_tf[i], D = s_tf[C * 256 + i];
            HalfEntry e;
            e.rg = __floats2half2_rn(T.x, T.y);
            e.ba = __floats2half2_rn(T.z, T.w);
            e.drg = __floats2half2_rn(D.x, D.y);
            e.dba = __floats2half2_rn(D.z, D.w);
            s_tfh[i] = e;
        }
        if (threadIdx.x < C) s_sh[threadIdx.x] = __float2half_rn(s_scl[threadIdx.x] * 65535.0f);
        __syncthreads();
    }
}

template <int C, int VS, int MODE, bool POW2, bool H, bool XF = false, bool CACHE = false, int SK = 0>
__global__ void __launch_bounds__(RENDER_MAX_THREADS, 1) render_kernel(RenderArgs a) {
    extern __shared__ float4 s_tf[];
    __shared__ float s_scl[MAXC];
    __shared__ __half s_sh[MAXC];
    HalfEntry* s_tfh = reinterpret_cast<HalfEntry*>(s_tf + C * 512);
    load_render_tables<C, H>(a, s_tf, s_scl, s_sh);
    // Warp tiles: a warp takes one tile_w x tile_h pixel tile at a time and its lanes march their
    // rays in lockstep.  Neighbouring rays at the same depth read the same cache lines; refilling
    // lanes with new rays as soon as theirs end (tried) loses that coherence and is ~3.6x slower.
    using F = std::conditional_t<MODE == 1, MIPMax<C>,
                                 std::conditional_t<MODE == 2, DVRFootprint<C>,
                                                    std::conditional_t<H, DVRCompositeH<C>, DVRComposite<C>>>>;
    const int lane = threadIdx.x & 31;
    unsigned long long* counter = reinterpret_cast<unsigned long long*>(a.counter);
    unsigned long long my_samples = 0, my_rays = 0;
    // Ray continuation (plain DVR, a.cont set): the first warp to find the queue empty raises the
    // dry flag; from then on, lanes whose rays still have far to go stop and record their state
    // for the second launch (render_tail_kernel), which marches each of them with a lane group.
    constexpr bool CONT = MODE == 0 && !XF && !CACHE;
    const unsigned* dry = (CONT && a.cont) ? a.cont_ctl : nullptr;
    // per-tile cost (optional): lane 0 notes the tile and the SM clock when it takes a tile and
    // stores the difference when it takes the next one (the warp has converged there)
    __shared__ unsigned s_ct_tile[RENDER_MAX_WARPS];
    __shared__ long long s_ct_clk[RENDER_MAX_WARPS];
    const int wib = threadIdx.x >> 5;
    if (lane == 0) s_ct_tile[wib] = 0xffffffffu;
    pdl_wait(); // the tile order of this call (tile_scatter_kernel) is complete
    for (;;) {
        unsigned long long tile = 0;
        if (lane == 0) tile = atomicAdd(counter, 1ull);
        tile = __shfl_sync(0xffffffffu, tile, 0);
        if (a.tile_cost && lane == 0 && s_ct_tile[wib] != 0xffffffffu) {
            const long long cyc = (clock64() - s_ct_clk[wib]) >> 6;
            a.tile_cost[s_ct_tile[wib]] = cyc < 0xffffffffLL ? (unsigned)cyc : 0xffffffffu;
        }
        if ((long long)tile >= a.total_tiles) {
            if (dry && lane == 0 && *(volatile const unsigned*)dry == 0u) *(volatile unsigned*)a.cont_ctl = 1u;
            break;
        }
        if (a.tile_order) tile = a.tile_order[tile];
        if (a.tile_cost && lane == 0) {
            s_ct_tile[wib] = (unsigned)tile;
            s_ct_clk[wib] = clock64();
        }
        const int ci = find_camera(a.cams, a.n_cams, (long long)tile);
        const CamParam* cp = &a.cams[ci];
        const long long lt = (long long)tile - cp->tile_begin;
        int px, py;
        tile_pixel(lt, cp->tiles_x, a.tile_w, a.tile_h, lane, px, py);
        if (px >= cp->W || py >= cp->H) continue;
        float dd[3], r0, r1;
        float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ray_setup(*cp, a.g, px, py, dd, r0, r1)) {
            ++my_rays;
            F f;
            if constexpr (MODE == 1) {
                f = MIPMax<C>();
            } else if constexpr (MODE == 2) {
                f.s_tf = s_tf;
                f.s_scl = s_scl;
                f.ert = cp->ert;
                f.vmark = a.vmark;
                f.nmark = a.nmark;
            } else if constexpr (H) {
                f = DVRCompositeH<C>{{}, s_tfh, s_sh, cp->ert};
            } else {
                f = DVRComposite<C>{{}, s_tf, s_scl, cp->ert};
            }
            long long n;
            if constexpr (XF) {
                n = march_xf<C, VS, POW2, F, SK>(a.g, a.pool, a.rnodes, *cp, dd, r0, r1, a.xf, f);
            } else if constexpr (CONT) {
                n = march<C, VS, POW2, H, F, SK>(a.g, a.pool, a.rnodes, *cp, dd, r0, r1, f, nullptr, 0, MAX_SAMPLES, dry,
                                          a.cont_min);
                if (n < 0) { // stopped at sample -n - 1: record the ray for the second launch
                    const unsigned slot = atomicAdd(&a.cont_ctl[1], 1u);
                    my_samples += (unsigned long long)(-n - 1);
                    a.cont[slot] = RayCont{ci, px, py, (int)(-n - 1), f.T, f.Cr, f.Cg, f.Cb};
                    continue; // the pixel is written by the second launch
                }
            } else {
                n = march<C, VS, POW2, H, F, SK>(a.g, a.pool, a.rnodes, *cp, dd, r0, r1, f, CACHE ? &a.cache : nullptr);
            }
            my_samples += (unsigned long long)n;
            if constexpr (MODE == 1) {
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
            } else {
                out = make_float4(f.Cr, f.Cg, f.Cb, f.alpha());
            }
        }
        reinterpret_cast<float4*>(cp->img)[(long long)py * cp->W + px] = out;
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

// Second launch of a continued DVR render: every ray recorded by render_kernel once the tile queue
// ran dry is resumed at its recorded sample and state and marched to its end by a group of
// 2^a.cont_lg lanes (march_group), which then writes its pixel.  The first launch was latency-bound
// by then -- few warps left, each with long rays -- and a lane group advances a ray by up to
// 2^cont_lg samples per step; the samples composited, and so the pixel, are those of one lane.
template <int C, int VS, bool POW2, bool H, int SK = 0>
__global__ void __launch_bounds__(RENDER_MAX_THREADS, 1) render_tail_kernel(RenderArgs a) {
    extern __shared__ float4 s_tf[];
    __shared__ float s_scl[MAXC];
    __shared__ __half s_sh[MAXC];
    __shared__ float4 s_grp[RENDER_MAX_WARPS][32]; // per warp: the shaded samples of a step
    const HalfEntry* s_tfh = reinterpret_cast<const HalfEntry*>(s_tf + C * 512);
    load_render_tables<C, H>(a, s_tf, s_scl, s_sh);
    using F = std::conditional_t<H, DVRCompositeH<C>, DVRComposite<C>>;
    const int lane = threadIdx.x & 31;
    const int lg = a.cont_lg, per = 32 >> lg;
    const int j = lane & ((1 << lg) - 1), gbase = lane - j;
    const unsigned gmask = lg == 5 ? 0xffffffffu : (((1u << (1 << lg)) - 1u) << gbase);
    pdl_wait(); // the rays recorded by render_kernel are complete
    const unsigned n_cont = a.cont_ctl[1];
    unsigned long long my_samples = 0;
    for (;;) {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(&a.cont_ctl[2], (unsigned)per);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n_cont) break;
        const unsigned gi = base + (unsigned)(lane >> lg);
        if (gi >= n_cont) continue; // the whole group
        const RayCont rc = a.cont[gi];
        const CamParam* cp = &a.cams[rc.ci];
        float dd[3], r0, r1;
        ray_setup(*cp, a.g, rc.px, rc.py, dd, r0, r1); // the recorded ray: a non-empty interval
        F f;
        if constexpr (H)
            f = DVRCompositeH<C>{{}, s_tfh, s_sh, cp->ert};
        else
            f = DVRComposite<C>{{}, s_tf, s_scl, cp->ert};
        f.T = rc.T;
        f.Cr = rc.Cr;
        f.Cg = rc.Cg;
        f.Cb = rc.Cb;
        const long long n =
            march_group<C, VS, POW2, H, F, SK>(a.g, a.pool, a.rnodes, *cp, dd, r0, r1, f, lg, gmask, gbase, j, rc.k,
                                        s_grp[threadIdx.x >> 5]);
        if (j == 0) {
            my_samples += (unsigned long long)(n - rc.k);
            reinterpret_cast<float4*>(cp->img)[(long long)rc.py * cp->W + rc.px] =
                make_float4(f.Cr, f.Cg, f.Cb, f.alpha());
        }
    }
    for (int o = 16; o > 0; o >>= 1) my_samples += __shfl_xor_sync(0xffffffffu, my_samples, o);
    if (lane == 0 && a.stats) atomicAdd(&a.stats[0], my_samples);
}

// Opacity correction in double precision: a = 1 - (1 - alpha)^l and its complement.
__device__ __forceinline__ void opacity_d(double al, float ell, double& a, double& oma) {
    if (ell == 0.5f) {
        oma = sqrt(1.0 - al);
        a = al / (1.0 + oma);
    } else if (ell == 1.0f) {
        a = al;
        oma = 1.0 - al;
    } else {
        const double lg = log1p(-al);
        a = -expm1((double)ell * lg);
        oma = exp((double)ell * lg);
    }
}

constexpr double ALPHA_MAX_D = 1.0 - 1e-6;

// One sample's shading in double precision (the FP64 gradient-check mode): the table entry i and
// the position lam between entries i and i + 1, the interpolated entry, the opacity correction
// and the sample's local colour K and transmittance q = P_C, all from the exact intensity Id and
// the unrounded intensity scale, as in the FP64 definition.  The entry is not a decision of the
// march (the table is continuous across entries), so it is taken from the double position: with
// the single-precision one, a position that rounds across an entry would put a gradient of
// relative size ~1e-5 on the neighbouring entry.
template <int C>
struct ShadeD {
    int i[C];
    bool clamped[C], inside[C];
    double lam[C], rgb[C][3], dT[C][4], al[C], a[C], oma[C];
    double P[C], R[C][3], K[3], q, lnq;
    __device__ __forceinline__ void eval(const float4* s_tf, const float* s_raw, const double (&Id)[C], float ell) {
        double pre = 1.0;
        K[0] = K[1] = K[2] = 0.0;
        lnq = 0.0;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const double xr = (double)s_raw[c] * Id[c] / 65535.0;
            inside[c] = xr > 0.0 && xr < 1.0;
            const double w = (xr < 0.0 ? 0.0 : (xr > 1.0 ? 1.0 : xr)) * 255.0;
            i[c] = min((int)floor(w), 254);
            lam[c] = w - (double)i[c];
            const float4 T0 = s_tf[c * 256 + i[c]], T1 = s_tf[c * 256 + i[c] + 1];
            dT[c][0] = (double)T1.x - (double)T0.x;
            dT[c][1] = (double)T1.y - (double)T0.y;
            dT[c][2] = (double)T1.z - (double)T0.z;
            dT[c][3] = (double)T1.w - (double)T0.w;
            rgb[c][0] = (double)T0.x + lam[c] * dT[c][0];
            rgb[c][1] = (double)T0.y + lam[c] * dT[c][1];
            rgb[c][2] = (double)T0.z + lam[c] * dT[c][2];
            const double alr = (double)T0.w + lam[c] * dT[c][3];
            clamped[c] = !(alr >= 0.0 && alr <= ALPHA_MAX_D);
            al[c] = alr < 0.0 ? 0.0 : (alr > ALPHA_MAX_D ? ALPHA_MAX_D : alr);
            opacity_d(al[c], ell, a[c], oma[c]);
            P[c] = pre;
            const double wa = pre * a[c];
            K[0] += wa * rgb[c][0];
            K[1] += wa * rgb[c][1];
            K[2] += wa * rgb[c][2];
            R[c][0] = K[0];
            R[c][1] = K[1];
            R[c][2] = K[2];
            pre *= oma[c];
            lnq += (double)ell * log1p(-al[c]);
        }
        q = pre;
    }
};

// The adjoint's forward pass in the FP64 check mode: the single-precision march decides (the
// same samples, runs and stop as DVRComposite), and the ray's colour and transmittance are
// accumulated alongside in double precision from the double shading.
template <int C>
struct DVRForwardD : DVRComposite<C, true, false> {
    using B = DVRComposite<C, true, false>;
    static constexpr bool kExactI = true;
    const float* s_raw;
    double Id[C];
    double Cd[3] = {0.0, 0.0, 0.0}, Td = 1.0;
    __device__ __forceinline__ bool sample(const float (&I)[C], float ell) {
        ShadeD<C> sd;
        sd.eval(B::s_tf, s_raw, Id, ell);
#pragma unroll
        for (int i = 0; i < 3; ++i) Cd[i] += Td * sd.K[i];
        Td *= sd.q;
        return B::sample(I, ell);
    }
    __device__ __forceinline__ long long run(const float (&I)[C], long long n, float ell, bool& stop) {
        ShadeD<C> sd;
        sd.eval(B::s_tf, s_raw, Id, ell);
        const long long j = B::run(I, n, ell, stop);
        const double nj = (double)j;
        const double S = sd.lnq < 0.0 ? expm1(nj * sd.lnq) / expm1(sd.lnq) : nj;
#pragma unroll
        for (int i = 0; i < 3; ++i) Cd[i] += Td * sd.K[i] * S;
        Td *= exp(nj * sd.lnq);
        return j;
    }
};

// Reverse-mode sweep in forward order.  With the final (C_f, T_f) of the ray known, the adjoint
// of channel-step j of the update C += T a rgb, T <- T (1 - a) (T = 1 - A) is
//   dL/da_j   = T_j gC.rgb_j + [ -gC.(C_f - C_j+) + gA_f T_f ] / (1 - a_j),
//   dL/drgb_j = gC T_j a_j,     da/dalpha = l (1 - a) / (1 - alpha).
// The sweep repeats the forward's single-precision arithmetic (DVRComposite: the two-step
// composite, closed-form runs through brick-less nodes) so that it stops at the same sample.  A run
// of n equal samples contributes the sums over its samples in closed form: sample s, channel c has
// T_{s,c} = T_0 q^s P_c (P_c = prod_{c' < c} (1 - a_c'), q = P_C) and
// C_(s,c)+ = C_0 + T_0 K (1 - q^s) / (1 - q) + T_0 q^s R_c (R_c = sum_{c' <= c} P_c' a_c' rgb_c',
// K = R_{C-1}), so every term is a geometric series in q.
// D = true (FP64 gradient-check mode): every value downstream of the sample positions -- the
// intensity, the table interpolation, the opacity correction, transmittance, colour, the gradient
// terms and their sums -- is double precision (ShadeD); the decisions (samples, table entries,
// runs, the stop) stay those of the single-precision forward.  The table-entry sums go to double
// shared-memory accumulators.
template <int C, bool D = false>
struct DVRAdjoint : NoHooks {
    using R = std::conditional_t<D, double, float>;
    static constexpr bool kRuns = true;
    static constexpr bool kExactI = D;
    const float4* s_tf;
    const float* s_scl;
    const float* s_raw; // unrounded scales (D mode)
    R* s_dtf;           // [C][256][4]
    float ert;
    R gC[3], gAf, Cf[3], Tf;
    double Id[C]; // the sample's double intensity (D mode; set by the march)
    // the forward's single-precision state (decides the stop); in the D mode also a double copy
    float T = 1.0f, Cp[3] = {0.0f, 0.0f, 0.0f};
    R Td = 1.0, Cd[3] = {0.0, 0.0, 0.0};
    R dsc[C];
    // Per channel, the table-entry pair (i, i+1) this lane is accumulating into and the pending
    // sums S = sum g and L = sum lam g (entry i receives S - L, entry i+1 receives L).  Samples
    // of one ray mostly stay on one pair, so shared-memory atomics happen once per change of
    // pair instead of once per sample (32 lanes hitting one entry serialise).  A sample's colour
    // gradient is gC w (gC the ray's image gradient, w the sample's weight), so for colour only
    // the weights are summed (pW, pWL) and gC is applied at the flush; opacity keeps pA, pAL.
    // Four sums per channel instead of eight keep the lane's state in registers.
    int pk[C];
    R pW[C], pWL[C], pA[C], pAL[C];
    __device__ __forceinline__ void reset() {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            pk[c] = -1;
            pW[c] = pWL[c] = pA[c] = pAL[c] = (R)0;
        }
    }
    __device__ __forceinline__ void flush(int c) {
        if (pk[c] < 0) return;
        R* e0 = s_dtf + (c * 256 + pk[c]) * 4;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const R S = q < 3 ? gC[q] * pW[c] : pA[c], L = q < 3 ? gC[q] * pWL[c] : pAL[c];
            const R lo = S - L;
            if (lo != (R)0) atomicAdd(e0 + q, lo);
            if (L != (R)0) atomicAdd(e0 + 4 + q, L);
        }
        pW[c] = pWL[c] = pA[c] = pAL[c] = (R)0;
    }
    __device__ __forceinline__ void flush_all() {
#pragma unroll
        for (int c = 0; c < C; ++c) flush(c);
    }
    // table gradient (gC w, ga) (rgba) of channel c at entry i, position lam, slope dT = T[i+1] -
    // T[i], and the scale gradient (x = s I / 65535 inside (0, 1))
    __device__ __forceinline__ void accumulate(int c, int i, R lam, const R (&dT)[4], bool inside, R w, R ga, R I) {
        const R glam = w * (gC[0] * dT[0] + gC[1] * dT[1] + gC[2] * dT[2]) + ga * dT[3];
        if (i != pk[c]) {
            flush(c);
            pk[c] = i;
        }
        pW[c] += w;
        pWL[c] += lam * w;
        pA[c] += ga;
        pAL[c] += lam * ga;
        if (inside) dsc[c] += glam * (R)255.0f * I * (R)(1.0f / 65535.0f);
    }
    __device__ __forceinline__ void accumulate(int c, const TFLookup<C>& t, R w, R ga, float I) {
        const float4 Dv = s_tf[(C + c) * 256 + t.i];
        const R dT[4] = {(R)Dv.x, (R)Dv.y, (R)Dv.z, (R)Dv.w};
        accumulate(c, t.i, (R)t.lam, dT, t.xr > 0.0f && t.xr < 1.0f, w, ga, (R)I);
    }
    __device__ __forceinline__ R suffix(const R (&Cj)[3]) const {
        return -(gC[0] * (Cf[0] - Cj[0]) + gC[1] * (Cf[1] - Cj[1]) + gC[2] * (Cf[2] - Cj[2])) + gAf * Tf;
    }
    // the forward's single-precision update of one sample (decides the stop)
    __device__ __forceinline__ bool forward_update(const float (&I)[C], float ell) {
        const DVRComposite<C, true, false> fw{{}, s_tf, s_scl, ert};
        const Shaded s = fw.shade(I, ell);
        Cp[0] = fmaf(T, s.r, Cp[0]);
        Cp[1] = fmaf(T, s.g, Cp[1]);
        Cp[2] = fmaf(T, s.b, Cp[2]);
        T *= s.q;
        return 1.0f - T >= ert;
    }
    __device__ __forceinline__ bool sample(const float (&I)[C], float ell) {
        if constexpr (D) {
            ShadeD<C> sd;
            sd.eval(s_tf, s_raw, Id, ell);
            const double T0 = Td;
            const double C0[3] = {Cd[0], Cd[1], Cd[2]};
#pragma unroll
            for (int c = 0; c < C; ++c) {
                double Cj[3];
#pragma unroll
                for (int i = 0; i < 3; ++i) Cj[i] = C0[i] + T0 * sd.R[c][i];
                const double Tc = T0 * sd.P[c];
                const double w = Tc * sd.a[c];
                const double ga = Tc * (gC[0] * sd.rgb[c][0] + gC[1] * sd.rgb[c][1] + gC[2] * sd.rgb[c][2]) +
                                  suffix(Cj) / sd.oma[c];
                accumulate(c, sd.i[c], sd.lam[c], sd.dT[c], sd.inside[c], w,
                           sd.clamped[c] ? 0.0 : ga * (double)ell * sd.oma[c] / (1.0 - sd.al[c]), Id[c]);
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) Cd[i] += Td * sd.K[i];
            Td *= sd.q;
            return forward_update(I, ell);
        } else {
            const float T0 = T;
            const float C0[3] = {Cp[0], Cp[1], Cp[2]};
            Shaded s{0.0f, 0.0f, 0.0f, 1.0f}; // the forward's single-precision shading
#pragma unroll
            for (int c = 0; c < C; ++c) {
                TFLookup<C> t;
                t.eval(s_tf, s_scl, c, I[c]);
                const bool clamped = !(t.al >= 0.0f && t.al <= ALPHA_MAX);
                const float al = fminf(fmaxf(t.al, 0.0f), ALPHA_MAX);
                float a, oma;
                opacity(al, ell, a, oma);
                const float Pc = s.q;
                const float w32 = s.q * a;
                s.r = fmaf(w32, t.r, s.r);
                s.g = fmaf(w32, t.g, s.g);
                s.b = fmaf(w32, t.b, s.b);
                s.q *= oma;
                const float Cj[3] = {fmaf(T0, s.r, C0[0]), fmaf(T0, s.g, C0[1]), fmaf(T0, s.b, C0[2])};
                const float Tc = T0 * Pc;
                const float w = Tc * a;
                const float ga = Tc * (gC[0] * t.r + gC[1] * t.g + gC[2] * t.b) + suffix(Cj) / oma;
                accumulate(c, t, w, clamped ? 0.0f : ga * ell * oma / (1.0f - al), I[c]);
            }
            Cp[0] = fmaf(T, s.r, Cp[0]);
            Cp[1] = fmaf(T, s.g, Cp[1]);
            Cp[2] = fmaf(T, s.b, Cp[2]);
            T *= s.q;
            return 1.0f - T >= ert;
        }
    }
    __device__ __forceinline__ long long run(const float (&I)[C], long long n, float ell, bool& stop) {
        const R T0 = D ? Td : (R)T;
        const R C0[3] = {D ? Cd[0] : (R)Cp[0], D ? Cd[1] : (R)Cp[1], D ? Cd[2] : (R)Cp[2]};
        const R alpha0 = suffix(C0); // before the run
        // the forward's single-precision closed form decides the samples used and the stop
        DVRComposite<C, true, false> fw{{}, s_tf, s_scl, ert};
        fw.T = T;
        fw.Cr = Cp[0];
        fw.Cg = Cp[1];
        fw.Cb = Cp[2];
        const long long j = fw.run(I, n, ell, stop);
        T = fw.T;
        Cp[0] = fw.Cr;
        Cp[1] = fw.Cg;
        Cp[2] = fw.Cb;
        const R nj = (R)j;
        if constexpr (D) {
            // geometric sums over the run from the double shading of the (exact) AVG intensity
            ShadeD<C> sd;
            sd.eval(s_tf, s_raw, Id, ell);
            const double em1 = expm1(sd.lnq);
            const double Sg = sd.lnq < 0.0 ? expm1(nj * sd.lnq) / em1 : nj; // sum_{s<j} q^s
            const double beta = sd.lnq < 0.0 ? T0 * (gC[0] * sd.K[0] + gC[1] * sd.K[1] + gC[2] * sd.K[2]) / -em1 : 0.0;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const double gamma = T0 * (gC[0] * sd.R[c][0] + gC[1] * sd.R[c][1] + gC[2] * sd.R[c][2]);
                const double ga =
                    T0 * sd.P[c] * (gC[0] * sd.rgb[c][0] + gC[1] * sd.rgb[c][1] + gC[2] * sd.rgb[c][2]) * Sg +
                    (alpha0 * nj + beta * (nj - Sg) + gamma * Sg) / sd.oma[c];
                const double wsum = T0 * sd.P[c] * sd.a[c] * Sg;
                accumulate(c, sd.i[c], sd.lam[c], sd.dT[c], sd.inside[c], wsum,
                           sd.clamped[c] ? 0.0 : ga * (double)ell * sd.oma[c] / (1.0 - sd.al[c]), Id[c]);
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) Cd[i] += Td * sd.K[i] * Sg;
            Td *= exp(nj * sd.lnq);
        } else {
            // geometric sums over the run, in single precision
            TFLookup<C> t[C];
            float a[C], oma[C], al[C];
            float Pw[C], Rc[C][3], K[3] = {0.0f, 0.0f, 0.0f}, pre = 1.0f, lnq = 0.0f;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                t[c].eval(s_tf, s_scl, c, I[c]);
                al[c] = fminf(fmaxf(t[c].al, 0.0f), ALPHA_MAX);
                opacity(al[c], ell, a[c], oma[c]);
                Pw[c] = pre;
                const float w = pre * a[c];
                K[0] += w * t[c].r;
                K[1] += w * t[c].g;
                K[2] += w * t[c].b;
                Rc[c][0] = K[0];
                Rc[c][1] = K[1];
                Rc[c][2] = K[2];
                pre *= oma[c];
                lnq += ell * log1pf(-al[c]);
            }
            const float em1 = expm1f(lnq);
            const float Sg = lnq < 0.0f ? expm1f(nj * lnq) / em1 : nj;
            const float beta = lnq < 0.0f ? T0 * (gC[0] * K[0] + gC[1] * K[1] + gC[2] * K[2]) / -em1 : 0.0f;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const float gamma = T0 * (gC[0] * Rc[c][0] + gC[1] * Rc[c][1] + gC[2] * Rc[c][2]);
                const float ga = T0 * Pw[c] * (gC[0] * t[c].r + gC[1] * t[c].g + gC[2] * t[c].b) * Sg +
                                 (alpha0 * nj + beta * (nj - Sg) + gamma * Sg) / oma[c];
                const float wsum = T0 * Pw[c] * a[c] * Sg;
                const bool clamped = !(t[c].al >= 0.0f && t[c].al <= ALPHA_MAX);
                accumulate(c, t[c], wsum, clamped ? 0.0f : ga * ell * oma[c] / (1.0f - al[c]), I[c]);
            }
        }
        return j;
    }
};

constexpr unsigned BWD_REFILL = 8; // idle lanes of a warp that make it regroup (per-lane ray queue)

// 4 resident 128-thread CTAs per SM (128 registers, no spills of the lane's state): on the 512^3
// view 3.45 ms against 3.64 ms with 5 CTAs at 96 registers (272 bytes of spill loads); tiles in
// raster order (the forward's costliest-first order measured 3.55-3.66 ms here: neighbouring
// tiles share bricks in L1).
// D: the FP64 gradient-check mode (double sums; per-CTA sums added into a double buffer, a.dacc).
// SK: the slot edge as a compile-time constant (0: read from the geometry), as in render_kernel.
template <int C, int VS, bool POW2, bool XF = false, bool D = false, int SK = 0>
__global__ void __launch_bounds__(128, 4) render_backward_kernel(RenderArgs a) {
    using R = std::conditional_t<D, double, float>;
    extern __shared__ float4 s_tf[];
    __shared__ float s_scl[MAXC];
    __shared__ float s_raw[MAXC];
    R* s_dtf = reinterpret_cast<R*>(s_tf + C * 512);
    for (int i = threadIdx.x; i < C * 1024; i += blockDim.x) s_dtf[i] = (R)0;
    if (threadIdx.x < C) s_raw[threadIdx.x] = a.scl[MAXC + threadIdx.x];
    load_tables(a, C, s_tf, s_scl);
    const int lane = threadIdx.x & 31;
    R dsc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) dsc[c] = (R)0;
    bool lane_queue = false;
    if constexpr (!XF && !D) lane_queue = a.fwd_img != 0;
    if constexpr (!XF && !D) if (lane_queue) {
        // Rays handed out one per lane (ray r: lane r % 32 of tile r / 32), so that a lane whose
        // ray has ended takes the next ray instead of idling until the warp's longest ray ends.
        // Once BWD_REFILL lanes of a warp are idle, the marching lanes stop at their next 16-step
        // check (march's exact stop: the state before sample k stays in bw) and the warp regroups:
        // idle lanes take new rays, stopped lanes resume at their sample.  After the queue is
        // empty every lane marches its ray to the end.
        __shared__ unsigned s_stop[4], s_idle[4]; // per warp of the 128-thread CTA
        unsigned long long* rq = reinterpret_cast<unsigned long long*>(a.counter);
        const unsigned long long nrays = (unsigned long long)a.total_tiles * 32ull;
        const int wib = threadIdx.x >> 5;
        bool have = false, empty = false;
        int k0 = 0;
        const CamParam* cpp = a.cams;
        float d[3] = {0.0f, 0.0f, 0.0f}, t0 = 0.0f, t1 = 0.0f;
        DVRAdjoint<C, false> bw;
        for (;;) {
            unsigned need = __ballot_sync(0xffffffffu, !have);
            while (need != 0u && !empty) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(rq, (unsigned long long)__popc(need));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (base + (unsigned long long)__popc(need) >= nrays) empty = true; // uniform in the warp
                if (!have) {
                    const unsigned long long r = base + (unsigned long long)__popc(need & ((1u << lane) - 1u));
                    if (r < nrays) {
                        const long long tile = (long long)(r >> 5);
                        cpp = &a.cams[find_camera(a.cams, a.n_cams, tile)];
                        int px, py;
                        tile_pixel(tile - cpp->tile_begin, cpp->tiles_x, a.tile_w, a.tile_h, (int)(r & 31u), px, py);
                        if (px < cpp->W && py < cpp->H && ray_setup(*cpp, a.g, px, py, d, t0, t1)) {
                            const long long pix = (long long)py * cpp->W + px;
                            const float4 gl = reinterpret_cast<const float4*>(cpp->dimg)[pix];
                            if (gl.x != 0.0f || gl.y != 0.0f || gl.z != 0.0f || gl.w != 0.0f) {
                                // the ray's final colour and transmittance from the forward image
                                const float4 im = reinterpret_cast<const float4*>(cpp->img)[pix];
                                bw = DVRAdjoint<C, false>();
                                bw.s_tf = s_tf;
                                bw.s_scl = s_scl;
                                bw.s_raw = s_raw;
                                bw.s_dtf = s_dtf;
                                bw.ert = cpp->ert;
                                bw.gC[0] = gl.x;
                                bw.gC[1] = gl.y;
                                bw.gC[2] = gl.z;
                                bw.gAf = gl.w;
                                bw.Cf[0] = im.x;
                                bw.Cf[1] = im.y;
                                bw.Cf[2] = im.z;
                                bw.Tf = 1.0f - im.w;
#pragma unroll
                                for (int c = 0; c < C; ++c) bw.dsc[c] = 0.0f;
                                bw.reset();
                                k0 = 0;
                                have = true;
                            }
                        }
                    }
                }
                need = __ballot_sync(0xffffffffu, !have);
            }
            if (__ballot_sync(0xffffffffu, have) == 0u) break; // the queue is empty and no lane holds a ray
            if (lane == 0) {
                s_stop[wib] = 0u;
                s_idle[wib] = 0u;
            }
            __syncwarp();
            if (have) {
                const long long r = march<C, VS, POW2, false, DVRAdjoint<C, false>, SK>(
                    a.g, a.pool, a.rnodes, *cpp, d, t0, t1, bw, nullptr, k0, MAX_SAMPLES, empty ? nullptr : &s_stop[wib], 0);
                if (r < 0) {
                    k0 = (int)(-(r + 1)); // stopped for a regrouping: resume at sample k0
                } else {
                    bw.flush_all();
#pragma unroll
                    for (int c = 0; c < C; ++c) dsc[c] += bw.dsc[c];
                    have = false;
                    if (!empty && atomicAdd(&s_idle[wib], 1u) + 1u >= BWD_REFILL) *(volatile unsigned*)&s_stop[wib] = 1u;
                }
            }
        }
    }
    for (;;) {
        if (lane_queue) break;
        unsigned int tile = 0;
        if (lane == 0) tile = atomicAdd(a.counter, 1u);
        tile = __shfl_sync(0xffffffffu, tile, 0);
        if ((long long)tile >= a.total_tiles) break;
        const int ci = find_camera(a.cams, a.n_cams, tile);
        const CamParam& cp = a.cams[ci];
        const long long lt = (long long)tile - cp.tile_begin;
        int px, py;
        tile_pixel(lt, cp.tiles_x, a.tile_w, a.tile_h, lane, px, py);
        if (px >= cp.W || py >= cp.H) continue;
        float d[3], t0, t1;
        if (!ray_setup(cp, a.g, px, py, d, t0, t1)) continue;
        const float4 gl = reinterpret_cast<const float4*>(cp.dimg)[(long long)py * cp.W + px];
        if (gl.x == 0.0f && gl.y == 0.0f && gl.z == 0.0f && gl.w == 0.0f) continue;
        // the forward pass: the sweep's arithmetic (runs, no pairs) -- or, given the forward's
        // images (a.fwd_img; single precision only), the final colour and transmittance of the ray
        // read from its pixel: the forward render composited the same samples in the same order
        std::conditional_t<D, DVRForwardD<C>, DVRComposite<C, true, false>> fw;
        fw.s_tf = s_tf;
        fw.s_scl = s_scl;
        fw.ert = cp.ert;
        if constexpr (D) fw.s_raw = s_raw;
        if (!D && a.fwd_img) {
            const float4 im = reinterpret_cast<const float4*>(cp.img)[(long long)py * cp.W + px];
            fw.Cr = im.x;
            fw.Cg = im.y;
            fw.Cb = im.z;
            fw.T = 1.0f - im.w;
        } else if constexpr (XF) {
            march_xf<C, VS, POW2>(a.g, a.pool, a.rnodes, cp, d, t0, t1, a.xf, fw);
        } else {
            march<C, VS, POW2, false, decltype(fw), SK>(a.g, a.pool, a.rnodes, cp, d, t0, t1, fw);
        }
        DVRAdjoint<C, D> bw;
        bw.s_tf = s_tf;
        bw.s_scl = s_scl;
        bw.s_raw = s_raw;
        bw.s_dtf = s_dtf;
        bw.ert = cp.ert;
        bw.gC[0] = gl.x;
        bw.gC[1] = gl.y;
        bw.gC[2] = gl.z;
        bw.gAf = gl.w;
        if constexpr (D) {
            bw.Cf[0] = fw.Cd[0];
            bw.Cf[1] = fw.Cd[1];
            bw.Cf[2] = fw.Cd[2];
            bw.Tf = fw.Td;
        } else {
            bw.Cf[0] = fw.Cr;
            bw.Cf[1] = fw.Cg;
            bw.Cf[2] = fw.Cb;
            bw.Tf = fw.T;
        }
#pragma unroll
        for (int c = 0; c < C; ++c) bw.dsc[c] = (R)0;
        bw.reset();
        if constexpr (XF)
            march_xf<C, VS, POW2>(a.g, a.pool, a.rnodes, cp, d, t0, t1, a.xf, bw);
        else
            march<C, VS, POW2, false, decltype(bw), SK>(a.g, a.pool, a.rnodes, cp, d, t0, t1, bw);
        bw.flush_all();
#pragma unroll
        for (int c = 0; c < C; ++c) dsc[c] += bw.dsc[c];
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
        R v = dsc[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && v != (R)0) {
            if constexpr (D) atomicAdd(&a.dacc[C * 1024 + c], v);
            else atomicAdd(&a.dscale[c], v);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < C * 1024; i += blockDim.x)
        if (s_dtf[i] != (R)0) {
            if constexpr (D) atomicAdd(&a.dacc[i], s_dtf[i]);
            else atomicAdd(&a.dtf[i], s_dtf[i]);
        }
}

// FP64 gradient-check mode: the double sums rounded once to the float outputs.
__global__ void grad_convert_kernel(int C, const double* __restrict__ acc, float* __restrict__ dtf,
                                    float* __restrict__ dscale) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < C * 1024) dtf[i] = (float)acc[i];
    if (i < C) dscale[i] = (float)acc[C * 1024 + i];
}

// Queue order from the tile costs of an earlier frame of the same tile grid: costliest first
// (longest-processing-time-first list scheduling), in NCLS classes of cost, four per power of
// two (exponent and the two bits below the leading one); the order inside a class is whatever the
// atomics give (a pixel does not depend on when its tile runs).
// aux: [0, NCLS) class sizes, [NCLS, 2 NCLS) class cursors, zeroed before.
constexpr int NCLS = 128;
__device__ __forceinline__ int cost_class(unsigned c) {
    if (c < 4u) return (int)c;
    const int e = 31 - __clz(c);
    return e * 4 + (int)((c >> (e - 2)) & 3u);
}

__global__ void tile_hist_kernel(const unsigned* __restrict__ cost, long long n, unsigned* aux) {
    __shared__ unsigned h[NCLS];
    if (threadIdx.x < NCLS) h[threadIdx.x] = 0;
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        atomicAdd(&h[cost_class(cost[i])], 1u);
    __syncthreads();
    if (threadIdx.x < NCLS && h[threadIdx.x]) atomicAdd(&aux[threadIdx.x], h[threadIdx.x]);
}

__global__ void tile_scatter_kernel(const unsigned* __restrict__ cost, long long n, unsigned* aux,
                                    unsigned* __restrict__ order) {
    __shared__ unsigned base[NCLS], cnt[NCLS];
    if (threadIdx.x < NCLS) cnt[threadIdx.x] = 0;
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        atomicAdd(&cnt[cost_class(cost[i])], 1u);
    pdl_wait(); // the class sizes (tile_hist_kernel) are complete
    if (threadIdx.x == 0) {
        unsigned acc = 0;
        for (int c = NCLS - 1; c >= 0; --c) {
            base[c] = acc;
            acc += aux[c];
        }
    }
    __syncthreads();
    if (threadIdx.x < NCLS) {
        base[threadIdx.x] += cnt[threadIdx.x] ? atomicAdd(&aux[NCLS + threadIdx.x], cnt[threadIdx.x]) : 0u;
        cnt[threadIdx.x] = 0;
    }
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int c = cost_class(cost[i]);
        order[base[c] + atomicAdd(&cnt[c], 1u)] = (unsigned)i;
    }
}

// ---- MIP ray segments ----
// A MIP ray is the per-channel maximum over its samples, so it splits without approximation: the
// samples k in [j kseg, (j+1) kseg) of every ray of a tile are work item j * total_tiles + tile
// (segment-major), each records its per-channel maxima and sample count, and a merge takes the
// maximum over the segments and applies the transfer functions.  The image is the whole-ray
// image bit for bit; the longest rays no longer run in one warp each.
constexpr unsigned SEG_END_RAY = 0u, SEG_GOES_ON = 2u;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// seg_done[segment][tile]: 0 pending, 1 done and no ray of the tile goes on, 3 done and some do
template <int C, int VS, bool POW2, int SK = 0>
__global__ void __launch_bounds__(RENDER_MAX_THREADS, 1) mip_seg_kernel(RenderArgs a) {
    const int lane = threadIdx.x & 31;
    unsigned long long* counter = reinterpret_cast<unsigned long long*>(a.counter);
    unsigned long long my_rays = 0;
    const unsigned long long items = (unsigned long long)(a.total_tiles * a.nseg);
    for (;;) {
        unsigned long long q = 0;
        if (lane == 0) q = atomicAdd(counter, 1ull);
        q = __shfl_sync(0xffffffffu, q, 0);
        if (q >= items) break;
        const int seg = (int)(q / (unsigned long long)a.total_tiles);
        const long long tile = (long long)q - (long long)seg * a.total_tiles;
        const CamParam* cp = &a.cams[find_camera(a.cams, a.n_cams, tile)];
        int px, py;
        tile_pixel(tile - cp->tile_begin, cp->tiles_x, a.tile_w, a.tile_h, lane, px, py);
        const bool inimg = px < cp->W && py < cp->H;
        const long long slot = ((long long)seg * a.total_tiles + tile) * 32 + lane;
        bool work = inimg;
        if (seg > 0) {
            unsigned pd = 0;
            if (lane == 0) pd = ld_acquire_u32(&a.seg_done[(long long)(seg - 1) * a.total_tiles + tile]);
            pd = __shfl_sync(0xffffffffu, pd, 0);
            __syncwarp();
            if (pd == 1u) { // every ray of the tile ended before this segment
                if (lane == 0) st_release_u32(&a.seg_done[(long long)seg * a.total_tiles + tile], 1u);
                continue;
            }
            // previous segment done: only the rays that went on; not done yet: every ray (a ray
            // that ended before this segment finds no sample in it)
            if (pd == 3u && work) work = (__ldcg(&a.seg_meta[slot - a.total_tiles * 32]) & 3u) == SEG_GOES_ON;
        }
        float4 part = make_float4(-1.0f, -1.0f, -1.0f, -1.0f);
        unsigned meta = SEG_END_RAY;
        float dd[3], r0, r1;
        if (work && ray_setup(*cp, a.g, px, py, dd, r0, r1)) {
            if (seg == 0) ++my_rays;
            MIPMax<C> f;
            const int k0 = seg * a.kseg, k1 = k0 + a.kseg;
            const long long k =
                march<C, VS, POW2, false, decltype(f), SK>(a.g, a.pool, a.rnodes, *cp, dd, r0, r1, f, nullptr, k0, k1);
            const bool cont = k == k1 && __fadd_rn(r0, __fmul_rn((float)k1, cp->dt)) < r1;
            meta = ((unsigned)(k - k0) << 2) | (cont ? SEG_GOES_ON : SEG_END_RAY);
#pragma unroll
            for (int c = 0; c < C; ++c) (&part.x)[c] = f.mx[c];
        }
        if (inimg) {
            a.seg_v[slot] = part;
            a.seg_meta[slot] = meta;
        }
        const bool any = __ballot_sync(0xffffffffu, (meta & 3u) == SEG_GOES_ON) != 0u;
        __syncwarp();
        if (lane == 0) {
            __threadfence();
            st_release_u32(&a.seg_done[(long long)seg * a.total_tiles + tile], any ? 3u : 1u);
        }
    }
    for (int o = 16; o > 0; o >>= 1) my_rays += __shfl_xor_sync(0xffffffffu, my_rays, o);
    if (lane == 0 && a.stats) atomicAdd(&a.stats[1], my_rays);
}

// merge: one warp per tile (grid-stride), a lane per pixel; the same transfer-function step as
// the whole-ray MIP pass
template <int C>
__global__ void __launch_bounds__(256) mip_merge_kernel(RenderArgs a) {
    extern __shared__ float4 s_tf[];
    __shared__ float s_scl[MAXC];
    load_tables(a, C, s_tf, s_scl);
    const int lane = threadIdx.x & 31;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    unsigned long long my_samples = 0;
    for (long long tile = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); tile < a.total_tiles;
         tile += nwarps) {
        const CamParam* cp = &a.cams[find_camera(a.cams, a.n_cams, tile)];
        int px, py;
        tile_pixel(tile - cp->tile_begin, cp->tiles_x, a.tile_w, a.tile_h, lane, px, py);
        if (px >= cp->W || py >= cp->H) continue;
        float mx[C];
        unsigned long long n = 0;
        for (int j = 0; j < a.nseg; ++j) {
            const long long slot = ((long long)j * a.total_tiles + tile) * 32 + lane;
            const unsigned m = a.seg_meta[slot];
            const float4 v = a.seg_v[slot];
#pragma unroll
            for (int c = 0; c < C; ++c) mx[c] = j == 0 ? (&v.x)[c] : fmaxf(mx[c], (&v.x)[c]);
            n += m >> 2;
            if ((m & 3u) != SEG_GOES_ON) break;
        }
        float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
        if (n > 0) {
            float A = 0.f, Cr = 0.f, Cg = 0.f, Cb = 0.f;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                TFLookup<C> t;
                t.eval(s_tf, s_scl, c, mx[c]);
                const float al = fminf(fmaxf(t.al, 0.0f), ALPHA_MAX);
                const float w = (1.0f - A) * al;
                Cr = fmaf(w, t.r, Cr);
                Cg = fmaf(w, t.g, Cg);
                Cb = fmaf(w, t.b, Cb);
                A += w;
            }
            out = make_float4(Cr, Cg, Cb, A);
        }
        reinterpret_cast<float4*>(cp->img)[(long long)py * cp->W + px] = out;
        my_samples += n;
    }
    for (int o = 16; o > 0; o >>= 1) my_samples += __shfl_xor_sync(0xffffffffu, my_samples, o);
    if (lane == 0 && a.stats) atomicAdd(&a.stats[0], my_samples);
}

// One refinement pass over the pixels of a single camera: every unfinished ray resumes from its
// saved sample index and compositing state, and either ends (pixel written) or stops again at its
// next missing brick (state saved, counted in *pending).
template <int C, int VS, bool POW2>
__global__ void __launch_bounds__(256, VR_RENDER_MIN_CTAS) refine_kernel(RenderArgs a) {
    extern __shared__ float4 s_tf[];
    __shared__ float s_scl[MAXC];
    load_tables(a, C, s_tf, s_scl);
    const int lane = threadIdx.x & 31;
    unsigned long long* counter = reinterpret_cast<unsigned long long*>(a.counter);
    unsigned long long my_samples = 0;
    unsigned int my_pending = 0;
    const CamParam* cp = &a.cams[0];
    for (;;) {
        unsigned long long tile = 0;
        if (lane == 0) tile = atomicAdd(counter, 1ull);
        tile = __shfl_sync(0xffffffffu, tile, 0);
        if ((long long)tile >= a.total_tiles) break;
        const long long lt = (long long)tile;
        int px, py;
        tile_pixel(lt, cp->tiles_x, a.tile_w, a.tile_h, lane, px, py);
        if (px >= cp->W || py >= cp->H) continue;
        const long long pix = (long long)py * cp->W + px;
        RefineState st = a.refine_state[pix];
        if (st.status == 2) continue;
        float dd[3], r0, r1;
        if (!ray_setup(*cp, a.g, px, py, dd, r0, r1)) {
            reinterpret_cast<float4*>(cp->img)[pix] = make_float4(0.f, 0.f, 0.f, 0.f);
            st.status = 2;
            a.refine_state[pix] = st;
            continue;
        }
        DVRComposite<C> f{{}, s_tf, s_scl, cp->ert};
        const int k0 = st.status == 1 ? st.k : 0;
        if (st.status == 1) {
            f.Cr = st.C[0];
            f.Cg = st.C[1];
            f.Cb = st.C[2];
            f.T = st.T;
        }
        const long long r = march<C, VS, POW2, false>(a.g, a.pool, a.rnodes, *cp, dd, r0, r1, f, &a.cache, k0);
        if (r < 0) {
            st.k = (int)(-r - 1);
            st.C[0] = f.Cr;
            st.C[1] = f.Cg;
            st.C[2] = f.Cb;
            st.T = f.T;
            st.status = 1;
            my_samples += (unsigned long long)(st.k - k0);
            ++my_pending;
        } else {
            reinterpret_cast<float4*>(cp->img)[pix] = make_float4(f.Cr, f.Cg, f.Cb, f.alpha());
            st.status = 2;
            my_samples += (unsigned long long)(r - k0);
        }
        a.refine_state[pix] = st;
    }
    for (int o = 16; o > 0; o >>= 1) {
        my_samples += __shfl_xor_sync(0xffffffffu, my_samples, o);
        my_pending += __shfl_xor_sync(0xffffffffu, my_pending, o);
    }
    if (lane == 0) {
        if (a.stats) atomicAdd(&a.stats[0], my_samples);
        if (my_pending) atomicAdd(a.pending, my_pending);
    }
}

__global__ void cache_gather_kernel(const uint16_t* __restrict__ store, uint16_t* __restrict__ cache,
                                    const int2* __restrict__ list, long long slot_elems) {
    const int2 e = list[blockIdx.x]; // (store slot, cache slot)
    const uint4* src = reinterpret_cast<const uint4*>(store + (long long)e.x * slot_elems);
    uint4* dst = reinterpret_cast<uint4*>(cache + (long long)e.y * slot_elems);
    const long long n16 = slot_elems * 2 / 16;
    for (long long i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = src[i];
}

cudaError_t launch_cache_gather(const uint16_t* store, uint16_t* cache, const int2* list, int n, long long slot_elems,
                                cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    cache_gather_kernel<<<n, 256, 0, st>>>(store, cache, list, slot_elems);
    return cudaGetLastError();
}

// The shared-memory carve-out of a persistent render kernel: just what its resident CTAs need
// (by registers, at `threads` per CTA), so that the rest of the SM's unified L1/shared memory
// caches the brick gathers (24 GiB orbit: 1.87 -> 1.84 ms per frame against the driver's default).
static void prefer_l1(const void* kernel, int threads, size_t dyn_smem) {
    cudaFuncAttributes fa;
    int dev = 0, smem_sm = 0;
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        smem_sm <= 0 || fa.numRegs <= 0) {
        cudaGetLastError();
        return;
    }
    int ctas = 65536 / (threads * fa.numRegs);
    if (ctas < 1) ctas = 1;
    const double need = (double)ctas * ((double)dyn_smem + (double)fa.sharedSizeBytes + 1024.0);
    int pct = (int)(100.0 * need / smem_sm) + 1;
    if (pct > 100) pct = 100;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct) != cudaSuccess)
        cudaGetLastError();
}

// One launch of kernel k, as a programmatic dependent of the kernel before it on st when pdl.
template <class K>
static cudaError_t launch_k(K k, int blocks, int threads, size_t smem, cudaStream_t st, bool pdl, const RenderArgs& a) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, a);
}

template <int C, int VS, int MODE, bool POW2, bool H, bool XF = false, bool CACHE = false, int SK = 0>
static void launch_one(const RenderArgs& a, int blocks, int threads, cudaStream_t st, bool pdl = false) {
    const size_t smem = (size_t)C * 512 * sizeof(float4) + (H ? (size_t)C * 256 * sizeof(HalfEntry) : 0);
    cudaFuncSetAttribute(render_kernel<C, VS, MODE, POW2, H, XF, CACHE, SK>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    prefer_l1(reinterpret_cast<const void*>(render_kernel<C, VS, MODE, POW2, H, XF, CACHE, SK>), threads, smem);
    launch_k(render_kernel<C, VS, MODE, POW2, H, XF, CACHE, SK>, blocks, threads, smem, st, pdl, a);
}

// The slot edges the plain DVR kernels are also built for as compile-time constants (M = 32, the
// brick size of the large workloads, and M = 16): their corner offsets become immediates.
constexpr int SK_DVR = 34, SK_DVR16 = 18;

template <int C, int VS>
static cudaError_t launch_fwd_c(const RenderArgs& a, int mode, int fp16, int blocks, int threads, cudaStream_t st,
                                bool pdl) {
    const bool p2 = a.g.pow2 != 0;
    if (mode == 3) {
        const size_t smem = (size_t)C * 512 * sizeof(float4);
        if (p2) {
            cudaFuncSetAttribute(refine_kernel<C, VS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            refine_kernel<C, VS, true><<<blocks, threads, smem, st>>>(a);
        } else {
            cudaFuncSetAttribute(refine_kernel<C, VS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            refine_kernel<C, VS, false><<<blocks, threads, smem, st>>>(a);
        }
        return cudaGetLastError();
    }
    if (a.cache.cslot && (mode == 0 || mode == 1 || mode == 2)) { // full-frame pass over the render cache
        if (mode == 0) {
            if (p2) launch_one<C, VS, 0, true, false, false, true>(a, blocks, threads, st);
            else launch_one<C, VS, 0, false, false, false, true>(a, blocks, threads, st);
        } else if (mode == 1) {
            if (p2) launch_one<C, VS, 1, true, false, false, true>(a, blocks, threads, st);
            else launch_one<C, VS, 1, false, false, false, true>(a, blocks, threads, st);
        } else {
            if (p2) launch_one<C, VS, 2, true, false, false, true>(a, blocks, threads, st);
            else launch_one<C, VS, 2, false, false, false, true>(a, blocks, threads, st);
        }
        return cudaGetLastError();
    }
    if (a.has_xf && (mode == 0 || mode == 1)) { // per-channel transforms: FP32 interpolation
        if (mode == 0) {
            if (p2 && a.g.S == SK_DVR) launch_one<C, VS, 0, true, false, true, false, SK_DVR>(a, blocks, threads, st);
            else if (p2 && a.g.S == SK_DVR16)
                launch_one<C, VS, 0, true, false, true, false, SK_DVR16>(a, blocks, threads, st);
            else if (p2) launch_one<C, VS, 0, true, false, true>(a, blocks, threads, st);
            else launch_one<C, VS, 0, false, false, true>(a, blocks, threads, st);
        } else {
            if (p2) launch_one<C, VS, 1, true, false, true>(a, blocks, threads, st);
            else launch_one<C, VS, 1, false, false, true>(a, blocks, threads, st);
        }
        return cudaGetLastError();
    }
    if (mode == 1 && a.nseg > 0) { // MIP in ray segments: segments, then the merge
        cudaMemsetAsync(a.seg_done, 0, sizeof(unsigned) * (size_t)a.nseg * (size_t)a.total_tiles, st);
        if (p2 && a.g.S == SK_DVR) mip_seg_kernel<C, VS, true, SK_DVR><<<blocks, threads, 0, st>>>(a);
        else if (p2) mip_seg_kernel<C, VS, true><<<blocks, threads, 0, st>>>(a);
        else mip_seg_kernel<C, VS, false><<<blocks, threads, 0, st>>>(a);
        const long long mb = (a.total_tiles + 7) / 8;
        const int mblocks = (int)(mb < 1 ? 1 : (mb > 4096 ? 4096 : mb));
        const size_t smem = (size_t)C * 512 * sizeof(float4);
        cudaFuncSetAttribute(mip_merge_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        mip_merge_kernel<C><<<mblocks, 256, smem, st>>>(a);
        return cudaGetLastError();
    }
    const bool sk = p2 && a.g.S == SK_DVR, sk16 = p2 && a.g.S == SK_DVR16;
    if (mode == 0 && fp16) {
        if (sk) launch_one<C, VS, 0, true, true, false, false, SK_DVR>(a, blocks, threads, st, pdl);
        else if (sk16) launch_one<C, VS, 0, true, true, false, false, SK_DVR16>(a, blocks, threads, st, pdl);
        else if (p2) launch_one<C, VS, 0, true, true>(a, blocks, threads, st, pdl);
        else launch_one<C, VS, 0, false, true>(a, blocks, threads, st, pdl);
    } else if (mode == 0) {
        if (sk) launch_one<C, VS, 0, true, false, false, false, SK_DVR>(a, blocks, threads, st, pdl);
        else if (sk16) launch_one<C, VS, 0, true, false, false, false, SK_DVR16>(a, blocks, threads, st, pdl);
        else if (p2) launch_one<C, VS, 0, true, false>(a, blocks, threads, st, pdl);
        else launch_one<C, VS, 0, false, false>(a, blocks, threads, st, pdl);
    } else if (mode == 2) {
        if (p2) launch_one<C, VS, 2, true, false>(a, blocks, threads, st);
        else launch_one<C, VS, 2, false, false>(a, blocks, threads, st);
    } else {
        if (p2) launch_one<C, VS, 1, true, false>(a, blocks, threads, st);
        else launch_one<C, VS, 1, false, false>(a, blocks, threads, st);
    }
    return cudaGetLastError();
}

template <int C, int VS, bool POW2, bool H, int SK = 0>
static void launch_tail_one(const RenderArgs& a, int blocks, int threads, cudaStream_t st, bool pdl) {
    const size_t smem = (size_t)C * 512 * sizeof(float4) + (H ? (size_t)C * 256 * sizeof(HalfEntry) : 0);
    cudaFuncSetAttribute(render_tail_kernel<C, VS, POW2, H, SK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    prefer_l1(reinterpret_cast<const void*>(render_tail_kernel<C, VS, POW2, H, SK>), threads, smem);
    launch_k(render_tail_kernel<C, VS, POW2, H, SK>, blocks, threads, smem, st, pdl, a);
}

template <int C, int VS>
static cudaError_t launch_tail_c(const RenderArgs& a, int fp16, int blocks, int threads, cudaStream_t st, bool pdl) {
    if (a.g.pow2 && a.g.S == SK_DVR) {
        if (fp16) launch_tail_one<C, VS, true, true, SK_DVR>(a, blocks, threads, st, pdl);
        else launch_tail_one<C, VS, true, false, SK_DVR>(a, blocks, threads, st, pdl);
    } else if (a.g.pow2 && a.g.S == SK_DVR16) {
        if (fp16) launch_tail_one<C, VS, true, true, SK_DVR16>(a, blocks, threads, st, pdl);
        else launch_tail_one<C, VS, true, false, SK_DVR16>(a, blocks, threads, st, pdl);
    } else if (a.g.pow2) {
        if (fp16) launch_tail_one<C, VS, true, true>(a, blocks, threads, st, pdl);
        else launch_tail_one<C, VS, true, false>(a, blocks, threads, st, pdl);
    } else {
        if (fp16) launch_tail_one<C, VS, false, true>(a, blocks, threads, st, pdl);
        else launch_tail_one<C, VS, false, false>(a, blocks, threads, st, pdl);
    }
    return cudaGetLastError();
}

cudaError_t launch_render_tail(const RenderArgs& a, int fp16, int blocks, int threads, cudaStream_t st, bool pdl) {
    if (!a.cont || a.cont_lg < 0 || a.cont_lg > 5) return cudaErrorInvalidValue;
    switch (a.g.C) {
        case 1: return launch_tail_c<1, 1>(a, fp16, blocks, threads, st, pdl);
        case 2: return launch_tail_c<2, 2>(a, fp16, blocks, threads, st, pdl);
        case 3: return launch_tail_c<3, 4>(a, fp16, blocks, threads, st, pdl);
        default: return launch_tail_c<4, 4>(a, fp16, blocks, threads, st, pdl);
    }
}

cudaError_t launch_render(const RenderArgs& a, int mode, int fp16, int blocks, int threads, cudaStream_t st, bool pdl) {
    switch (a.g.C) {
        case 1: return launch_fwd_c<1, 1>(a, mode, fp16, blocks, threads, st, pdl);
        case 2: return launch_fwd_c<2, 2>(a, mode, fp16, blocks, threads, st, pdl);
        case 3: return launch_fwd_c<3, 4>(a, mode, fp16, blocks, threads, st, pdl);
        default: return launch_fwd_c<4, 4>(a, mode, fp16, blocks, threads, st, pdl);
    }
}

template <int C, int VS, bool POW2, bool XF, bool D, int SK = 0>
static void launch_bwd_one(const RenderArgs& a, int blocks, int threads, cudaStream_t st) {
    const size_t smem = (size_t)C * 512 * sizeof(float4) + (size_t)C * 1024 * (D ? sizeof(double) : sizeof(float));
    cudaFuncSetAttribute(render_backward_kernel<C, VS, POW2, XF, D, SK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    render_backward_kernel<C, VS, POW2, XF, D, SK><<<blocks, threads, smem, st>>>(a);
    if (D) grad_convert_kernel<<<(C * 1024 + 255) / 256, 256, 0, st>>>(C, a.dacc, a.dtf, a.dscale);
}

template <int C, int VS, bool D>
static void launch_bwd_d(const RenderArgs& a, int blocks, int threads, cudaStream_t st) {
    if constexpr (!D) { // the training path: the slot edge as a constant where it is one of two
        if (a.g.pow2 && !a.has_xf && a.g.S == SK_DVR)
            return launch_bwd_one<C, VS, true, false, D, SK_DVR>(a, blocks, threads, st);
        if (a.g.pow2 && !a.has_xf && a.g.S == SK_DVR16)
            return launch_bwd_one<C, VS, true, false, D, SK_DVR16>(a, blocks, threads, st);
    }
    if (a.g.pow2) {
        if (a.has_xf) launch_bwd_one<C, VS, true, true, D>(a, blocks, threads, st);
        else launch_bwd_one<C, VS, true, false, D>(a, blocks, threads, st);
    } else {
        if (a.has_xf) launch_bwd_one<C, VS, false, true, D>(a, blocks, threads, st);
        else launch_bwd_one<C, VS, false, false, D>(a, blocks, threads, st);
    }
}

template <int C, int VS>
static cudaError_t launch_bwd_c(const RenderArgs& a, int blocks, int threads, cudaStream_t st) {
    if (a.dacc) launch_bwd_d<C, VS, true>(a, blocks, threads, st);
    else launch_bwd_d<C, VS, false>(a, blocks, threads, st);
    return cudaGetLastError();
}

cudaError_t launch_tile_order(const unsigned* cost, long long tiles, unsigned* aux, unsigned* order, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(aux, 0, 2 * NCLS * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    const long long b = (tiles + 1023) / 1024;
    const int blocks = (int)(b < 1 ? 1 : (b > 148 ? 148 : b));
    tile_hist_kernel<<<blocks, 1024, 0, st>>>(cost, tiles, aux);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(1024u);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, tile_scatter_kernel, cost, tiles, aux, order);
    if (e != cudaSuccess) return e;
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
