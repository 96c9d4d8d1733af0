// vr_insert.cu -- incremental octree construction on the device (Sec. "Incremental
// Construction", steps 1-3; Sec. "Handling Volumes of Arbitrary Dimensions"; Sec. "Handling
// Multi-Channel Data").
//
// One launch per level L = 0..N, each over the bricks of level L whose slot (interior + border)
// covers the part of level L changed by the inserted block.  A CTA owns one slot, so no two CTAs
// write the same memory:
//   L = 0   copy the block's voxels into the slot positions that map onto them (interior and
//           the one-voxel borders of neighbouring bricks, clamp-replicated at the real extent);
//   L > 0   recompute those positions as the round-half-up mean of their in-volume children
//           (2x2x2, read from ONE child slot: with an even M and a one-voxel border the eight
//           children of any slot position lie in the child brick that holds 2x);
//   then    refresh the per-plane min/max/sum of the touched interior planes and finalize the
//           node: brick min/max/AVG, subtree min/max from the children (already final: previous
//           launch), homogeneity (max - min < tau in every channel) and the render record.
// The launches are ordered on the caller's stream; level L reads only level L-1 and its own
// slot, so the result is independent of scheduling.
#include <cuda.h> // CUtensorMap and its enums; the encoder is fetched from the driver at run time
#include <cuda_runtime.h>

#include "vr_internal.h"

namespace vrk {

__device__ __forceinline__ long long clampll(long long v, long long lo, long long hi) {
    return v < lo ? lo : (v > hi ? hi : v);
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ uint16_t rhu(unsigned long long S, unsigned long long k) {
    return (uint16_t)((2ull * S + k) / (2ull * k));
}

// rhu for k = 2^sh children (always the case: k is a product of factors 1 or 2 per axis):
// floor((2S + k) / (2k)) = (S + k/2) >> sh.  S <= 8 * 65535 keeps everything in 32 bits.
__device__ __forceinline__ uint32_t rhu_pow2(uint32_t S, uint32_t sh) { return (S + ((1u << sh) >> 1)) >> sh; }

__global__ void init_nodes_kernel(Geo g, RNode* rn, NStat* ns) {
    long long n = g.noff[g.N + 1];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        RNode r;
        r.slot = -1;
        r.flags = 0;
        for (int c = 0; c < 4; ++c) r.avg[c] = g.bg;
        rn[i] = r;
        NStat s;
        for (int c = 0; c < MAXC; ++c) {
            s.bmin[c] = s.bmax[c] = s.smin[c] = s.smax[c] = g.bg;
            s.bsum[c] = 0;
        }
        s.count = 0;
        ns[i] = s;
    }
}

cudaError_t launch_init_nodes(const Geo& g, RNode* rn, NStat* ns, cudaStream_t st) {
    long long n = g.noff[g.N + 1];
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    init_nodes_kernel<<<blocks, 256, 0, st>>>(g, rn, ns);
    return cudaGetLastError();
}

// Fill a newly allocated slot with the current level values at its positions: its own interior
// is untouched (background); borders come from touched neighbours, else background.
__global__ void slot_init_kernel(Geo g, uint16_t* __restrict__ pool, RNode* __restrict__ rn, PStat* __restrict__ ps,
                                 const SlotInit* __restrict__ list) {
    const SlotInit e = list[blockIdx.x];
    const int L = e.level, M = g.M, S = g.S, VS = g.VS, C = g.C;
    const long long b[3] = {e.bi, e.bj, e.bk};
    uint16_t* dst = pool + (long long)e.slot * g.slot_elems;
    const long long n = (long long)S * S * S;
    for (long long t = threadIdx.x; t < n; t += blockDim.x) {
        int l[3] = {(int)(t % S), (int)((t / S) % S), (int)(t / ((long long)S * S))};
        long long xc[3], ob[3];
        bool own = true;
        for (int a = 0; a < 3; ++a) {
            xc[a] = clampll(b[a] * M - 1 + l[a], 0, g.ldim[L][a] - 1);
            ob[a] = xc[a] / M;
            own = own && (ob[a] == b[a]);
        }
        uint16_t v[4] = {g.bg, g.bg, g.bg, g.bg};
        if (C < 4) v[3] = 0;
        if (C == 3) v[3] = 0;
        if (!own) {
            long long nid = g.noff[L] + (ob[2] * g.nb[L][1] + ob[1]) * g.nb[L][0] + ob[0];
            RNode r = rn[nid];
            if ((r.flags & F_TOUCHED) && r.slot >= 0 && r.slot < g.n_slots_cap) {
                const uint16_t* src = pool + (long long)r.slot * g.slot_elems +
                                      (((xc[2] - ob[2] * M + 1) * S + (xc[1] - ob[1] * M + 1)) * S +
                                       (xc[0] - ob[0] * M + 1)) * VS;
                for (int c = 0; c < C; ++c) v[c] = src[c];
            }
        }
        uint16_t* d = dst + t * VS;
        for (int c = 0; c < VS; ++c) d[c] = (c < C) ? v[c] : (uint16_t)0;
    }
    // plane statistics of a background brick
    long long nin[3];
    for (int a = 0; a < 3; ++a) {
        long long r = g.ldim[L][a] - b[a] * M;
        nin[a] = r < M ? (r > 0 ? r : 0) : M;
    }
    for (int t = threadIdx.x; t < M * C; t += blockDim.x) {
        PStat p;
        p.mn = p.mx = g.bg;
        p.sum = (uint32_t)((unsigned long long)g.bg * (unsigned long long)(nin[0] * nin[1]));
        ps[((long long)e.slot * M) * C + t] = p;
    }
    if (threadIdx.x == 0) rn[e.node].slot = e.slot;
}

cudaError_t launch_slot_init(const Geo& g, uint16_t* pool, RNode* rn, PStat* ps, const SlotInit* list, int n,
                             cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    slot_init_kernel<<<n, 256, 0, st>>>(g, pool, rn, ps, list);
    return cudaGetLastError();
}

struct LevelArgs {
    Geo g;
    int L;
    long long lo[3], hi[3];  // changed box of level L, inclusive
    long long blo[3], bn[3]; // brick range of the grid
    const uint16_t* block;   // L = 0 input
    long long org[3], ext[3];
    int mshift; // log2(M) when M is a power of two, else -1
    uint16_t* pool;
    RNode* rn;
    NStat* ns;
    PStat* ps;
    int* err;
};

template <int C>
__device__ __forceinline__ void block_reduce_stats(uint32_t (&mn)[C], uint32_t (&mx)[C], unsigned long long (&sm)[C]) {
    __shared__ uint32_t s_mn[32][C], s_mx[32][C];
    __shared__ unsigned long long s_sm[32][C];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        for (int o = 16; o > 0; o >>= 1) {
            mn[c] = min(mn[c], __shfl_xor_sync(0xffffffffu, mn[c], o));
            mx[c] = max(mx[c], __shfl_xor_sync(0xffffffffu, mx[c], o));
            sm[c] += __shfl_xor_sync(0xffffffffu, sm[c], o);
        }
        if (lane == 0) {
            s_mn[wid][c] = mn[c];
            s_mx[wid][c] = mx[c];
            s_sm[wid][c] = sm[c];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; ++w)
            for (int c = 0; c < C; ++c) {
                mn[c] = min(mn[c], s_mn[w][c]);
                mx[c] = max(mx[c], s_mx[w][c]);
                sm[c] += s_sm[w][c];
            }
    }
    __syncthreads();
}

constexpr int MAX_S = 130; // slot edge for the largest brick (M = 128)

// Programmatic dependent launch between the levels of one insert: a level >= 1 is launched with
// programmatic stream serialization, so its launch is processed while the level below drains and
// its CTAs look up their own slot before they wait (griddepcontrol.wait) for the level below to
// complete and its writes to be visible; nothing that level writes is read before the wait.  The
// levels do not trigger their dependents early: a trigger at the start of each CTA measured 0.400
// ms per 8-slice insert of the 2048^2 x 1024 workload, one before the node finalize 0.321 ms,
// none 0.319 ms (0.332 ms with plain launches).  The wait does nothing in a kernel launched
// without the attribute (level 0).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// One position of level L > 0: round-half-up mean of its in-volume children (2x2x2, one child slot).
template <int C, int VS>
__device__ __forceinline__ void half_sample(const LevelArgs& a, int L, int x, int y, int z, int msh, uint16_t (&v)[VS]) {
    const Geo& g = a.g;
    const int M = g.M, S = g.S;
    const int cx = 2 * x, cy = 2 * y, cz = 2 * z;
    const bool hx = cx + 1 < (int)g.ldim[L - 1][0], hy = cy + 1 < (int)g.ldim[L - 1][1],
               hz = cz + 1 < (int)g.ldim[L - 1][2];
    const int cbx = msh >= 0 ? cx >> msh : cx / M, cby = msh >= 0 ? cy >> msh : cy / M,
              cbz = msh >= 0 ? cz >> msh : cz / M;
    const long long cnid = g.noff[L - 1] + ((long long)cbz * g.nb[L - 1][1] + cby) * g.nb[L - 1][0] + cbx;
    const int cs = a.rn[cnid].slot;
    const uint32_t ksh = (uint32_t)hx + (uint32_t)hy + (uint32_t)hz; // k = 2^ksh children
    if (cs < 0 || cs >= g.n_slots_cap) {
#pragma unroll
        for (int c = 0; c < C; ++c) v[c] = g.bg;
        if (cs >= g.n_slots_cap) atomicOr(a.err, ERR_SLOT_RANGE);
        return;
    }
    const uint16_t* cp = a.pool + (long long)cs * g.slot_elems +
                         (((cz - cbz * M + 1) * S + (cy - cby * M + 1)) * S + (cx - cbx * M + 1)) * VS;
    uint32_t sum[C];
#pragma unroll
    for (int c = 0; c < C; ++c) sum[c] = 0;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int dx = e & 1, dy = (e >> 1) & 1, dz = e >> 2;
        if ((dx && !hx) || (dy && !hy) || (dz && !hz)) continue;
        const uint16_t* q = cp + ((dz * S + dy) * S + dx) * VS;
        if (VS == 4) {
            const uint2 w = *reinterpret_cast<const uint2*>(q); // one 8-byte voxel
            const uint32_t ws[2] = {w.x, w.y};
#pragma unroll
            for (int c = 0; c < C; ++c) sum[c] += (c & 1) ? (ws[c >> 1] >> 16) : (ws[c >> 1] & 0xffffu);
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) sum[c] += q[c];
        }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) v[c] = (uint16_t)rhu_pow2(sum[c], ksh);
}

// The node finalize's inputs that do not depend on the positions a launch writes: the statistics
// of the slot's interior planes outside the changed range [pz0, pz1] and the children's subtree
// minima and maxima (level L - 1, complete once the launch's pdl_wait has returned).  With whole
// changed planes (gather) one warp loads them before the positions -- lane l the planes l + 1,
// l + 33, ... and lane l < 8 child l -- so that they arrive while the positions are written; the
// finalize then adds the changed planes from the shared per-plane sums instead of reading back
// what its CTA has just written.  Same values as reading every plane after the write.  (Level 0's
// staged kernel, throughput-bound over thousands of slots, measured slower with it: 0.318 against
// 0.313 ms per 8-slice insert of the 2048^2 x 1024 workload; levels >= 1 gain 0.319 -> 0.313.)
template <int C>
struct FinalizeInputs {
    uint32_t bmn[32][C], bmx[32][C], cmn[32][C], cmx[32][C];
    unsigned long long bsm[32][C];
};

template <int C>
__device__ __forceinline__ void finalize_inputs(const LevelArgs& a, const long long (&b)[3], int slot, int pz0,
                                                int pz1, int nin2, FinalizeInputs<C>& fi) {
    const Geo& g = a.g;
    const int L = a.L, M = g.M;
    const int lane = threadIdx.x & 31; // one warp
    uint32_t bmn[C], bmx[C], cmn[C], cmx[C];
    unsigned long long bsm[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        bmn[c] = cmn[c] = 0xffffu;
        bmx[c] = cmx[c] = 0u;
        bsm[c] = 0ull;
    }
    for (int lz = 1 + lane; lz <= nin2; lz += 32) {
        if (lz >= pz0 && lz <= pz1) continue; // changed by this launch: from the shared plane sums
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const PStat p = a.ps[((long long)slot * M + (lz - 1)) * C + c];
            bmn[c] = min(bmn[c], (uint32_t)p.mn);
            bmx[c] = max(bmx[c], (uint32_t)p.mx);
            bsm[c] += p.sum;
        }
    }
    if (L > 0 && lane < 8) {
        const long long ci = 2 * b[0] + (lane & 1), cj = 2 * b[1] + ((lane >> 1) & 1), ck = 2 * b[2] + (lane >> 2);
        if (ci < g.nb[L - 1][0] && cj < g.nb[L - 1][1] && ck < g.nb[L - 1][2]) {
            const long long cn = g.noff[L - 1] + (ck * g.nb[L - 1][1] + cj) * g.nb[L - 1][0] + ci;
            const uint32_t flags = a.rn[cn].flags;
            uint32_t smn[C], smx[C];
#pragma unroll
            for (int c = 0; c < C; ++c) {
                smn[c] = a.ns[cn].smin[c];
                smx[c] = a.ns[cn].smax[c];
            }
            const bool t = (flags & F_TOUCHED) != 0;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                cmn[c] = t ? smn[c] : (uint32_t)g.bg;
                cmx[c] = t ? smx[c] : (uint32_t)g.bg;
            }
        }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
        fi.bmn[lane][c] = bmn[c];
        fi.bmx[lane][c] = bmx[c];
        fi.bsm[lane][c] = bsm[c];
        fi.cmn[lane][c] = cmn[c];
        fi.cmx[lane][c] = cmx[c];
    }
}

// After a slot's positions are written: the plane statistics of its changed interior planes
// (gathered while writing, or re-read), then the node's finalize in warp 0.
template <int C, int VS>
__device__ __forceinline__ void finish_slot(const LevelArgs& a, const long long (&b)[3], long long nid, int slot,
                                            const uint16_t* dst, const int (&l0)[3], const int (&l1)[3],
                                            const int (&nin)[3], bool interior, bool full_xy, bool gather,
                                            uint32_t (*s_pmn)[C], uint32_t (*s_pmx)[C], uint32_t (*s_psm)[C],
                                            const FinalizeInputs<C>* fi = nullptr) {
    const Geo& g = a.g;
    const int L = a.L, M = g.M, S = g.S;
    if (gather) {
        __syncthreads();
        const int pz0 = l0[2] > 1 ? l0[2] : 1, pz1 = l1[2] < nin[2] ? l1[2] : nin[2];
        for (int i = threadIdx.x; i < (pz1 - pz0 + 1) * C; i += blockDim.x) {
            const int lz = pz0 + i / C, c = i % C;
            PStat p;
            p.mn = (uint16_t)s_pmn[lz][c];
            p.mx = (uint16_t)s_pmx[lz][c];
            p.sum = s_psm[lz][c];
            a.ps[((long long)slot * M + (lz - 1)) * C + c] = p;
        }
    }
    if (!interior) return; // only border copies changed: the node's own statistics did not
    if (!full_xy) {
        __syncthreads();
        // per-plane statistics of the changed interior planes, re-read (in-volume voxels only)
        const int pz0 = l0[2] > 1 ? l0[2] : 1, pz1 = l1[2] < M ? l1[2] : M;
        for (int lz = pz0; lz <= pz1; ++lz) {
            if (lz > nin[2]) break; // plane beyond the real extent: unused
            uint32_t mn[C], mx[C];
            unsigned long long sm[C];
#pragma unroll
            for (int c = 0; c < C; ++c) {
                mn[c] = 0xffffu;
                mx[c] = 0;
                sm[c] = 0;
            }
            const int npl = nin[0] * nin[1];
            for (int t = threadIdx.x; t < npl; t += blockDim.x) {
                const int ty = t / nin[0];
                const int lx = 1 + (t - ty * nin[0]), ly = 1 + ty;
                const uint16_t* q = dst + ((lz * S + ly) * S + lx) * VS;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const uint32_t val = q[c];
                    mn[c] = min(mn[c], val);
                    mx[c] = max(mx[c], val);
                    sm[c] += val;
                }
            }
            block_reduce_stats<C>(mn, mx, sm);
            if (threadIdx.x == 0) {
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    PStat p;
                    p.mn = (uint16_t)mn[c];
                    p.mx = (uint16_t)mx[c];
                    p.sum = (uint32_t)sm[c];
                    a.ps[((long long)slot * M + (lz - 1)) * C + c] = p;
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x >= 32) return;
    // finalize the node in warp 0 (Sec. "CPU Data Structure": homogeneity, AVG; all channels must
    // be homogeneous, Sec. "Handling Multi-Channel Data").  Lane l reads the plane statistics of
    // planes l, l+32, ... and lane l < 8 the subtree statistics of child l; warp reductions.
    const int lane = threadIdx.x;
    uint32_t bmn[C], bmx[C], cmn[C], cmx[C];
    unsigned long long bsm[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        bmn[c] = cmn[c] = 0xffffu;
        bmx[c] = cmx[c] = 0u;
        bsm[c] = 0ull;
    }
    if (fi && gather) {
        // the other planes and the children from the early loads, the changed planes from the
        // shared sums (the values just written to the plane statistics)
        const int pz0 = l0[2] > 1 ? l0[2] : 1, pz1 = l1[2] < nin[2] ? l1[2] : nin[2];
#pragma unroll
        for (int c = 0; c < C; ++c) {
            bmn[c] = fi->bmn[lane][c];
            bmx[c] = fi->bmx[lane][c];
            bsm[c] = fi->bsm[lane][c];
            cmn[c] = fi->cmn[lane][c];
            cmx[c] = fi->cmx[lane][c];
        }
        for (int lz = 1 + lane; lz <= nin[2]; lz += 32) {
            if (lz < pz0 || lz > pz1) continue;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                bmn[c] = min(bmn[c], s_pmn[lz][c]);
                bmx[c] = max(bmx[c], s_pmx[lz][c]);
                bsm[c] += s_psm[lz][c];
            }
        }
    } else {
        for (int lz = 1 + lane; lz <= nin[2]; lz += 32) {
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const PStat p = a.ps[((long long)slot * M + (lz - 1)) * C + c];
                bmn[c] = min(bmn[c], (uint32_t)p.mn);
                bmx[c] = max(bmx[c], (uint32_t)p.mx);
                bsm[c] += p.sum;
            }
        }
        if (L > 0 && lane < 8) {
            const long long ci = 2 * b[0] + (lane & 1), cj = 2 * b[1] + ((lane >> 1) & 1),
                            ck = 2 * b[2] + (lane >> 2);
            if (ci < g.nb[L - 1][0] && cj < g.nb[L - 1][1] && ck < g.nb[L - 1][2]) {
                const long long cn = g.noff[L - 1] + (ck * g.nb[L - 1][1] + cj) * g.nb[L - 1][0] + ci;
                const bool t = (a.rn[cn].flags & F_TOUCHED) != 0;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    cmn[c] = t ? (uint32_t)a.ns[cn].smin[c] : (uint32_t)g.bg;
                    cmx[c] = t ? (uint32_t)a.ns[cn].smax[c] : (uint32_t)g.bg;
                }
            }
        }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
        for (int o = 16; o > 0; o >>= 1) {
            bmn[c] = min(bmn[c], __shfl_xor_sync(0xffffffffu, bmn[c], o));
            bmx[c] = max(bmx[c], __shfl_xor_sync(0xffffffffu, bmx[c], o));
            bsm[c] += __shfl_xor_sync(0xffffffffu, bsm[c], o);
            cmn[c] = min(cmn[c], __shfl_xor_sync(0xffffffffu, cmn[c], o));
            cmx[c] = max(cmx[c], __shfl_xor_sync(0xffffffffu, cmx[c], o));
        }
    }
    if (lane != 0) return;
    NStat s;
    bool bh = true, sh = true;
    s.count = nin[0] * nin[1] * nin[2];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        s.bmin[c] = (uint16_t)bmn[c];
        s.bmax[c] = (uint16_t)bmx[c];
        s.bsum[c] = bsm[c];
        const uint32_t smn = (L > 0) ? cmn[c] : bmn[c];
        const uint32_t smx = (L > 0) ? cmx[c] : bmx[c];
        s.smin[c] = (uint16_t)smn;
        s.smax[c] = (uint16_t)smx;
        if (!((int)bmx[c] - (int)bmn[c] < (int)g.tau)) bh = false;
        if (!((int)smx - (int)smn < (int)g.tau)) sh = false;
    }
    for (int c = C; c < MAXC; ++c) {
        s.bmin[c] = s.bmax[c] = s.smin[c] = s.smax[c] = 0;
        s.bsum[c] = 0;
    }
    a.ns[nid] = s;
    RNode r;
    r.slot = slot;
    r.flags = F_TOUCHED | ((L > 0 && !sh) ? F_CHILDREN : 0u) | (!bh ? F_BRICK : 0u);
    for (int c = 0; c < 4; ++c)
        r.avg[c] = (c < C) ? rhu(s.bsum[c], (unsigned long long)s.count) : (uint16_t)0;
    a.rn[nid] = r;
}

template <int C, int VS, bool LEVEL0, bool WIDE = false>
__global__ void __launch_bounds__(WIDE ? 1024 : 256) level_update_kernel(LevelArgs a) {
    const Geo& g = a.g;
    const int L = a.L, M = g.M, S = g.S;
    long long bb = blockIdx.x;
    long long b[3];
    b[0] = a.blo[0] + bb % a.bn[0];
    bb /= a.bn[0];
    b[1] = a.blo[1] + bb % a.bn[1];
    b[2] = a.blo[2] + bb / a.bn[1];
    const long long nid = g.noff[L] + (b[2] * g.nb[L][1] + b[1]) * g.nb[L][0] + b[0];
    const int slot = a.rn[nid].slot;
    if (slot < 0) return; // untouched neighbour without a slot: nothing stored to update
    if (slot >= g.n_slots_cap) {
        if (threadIdx.x == 0) atomicOr(a.err, ERR_SLOT_RANGE);
        return;
    }
    // slot positions whose clamped coordinate lies in [lo, hi]
    int l0[3], l1[3];
    bool interior = true;
    for (int d = 0; d < 3; ++d) {
        long long base = b[d] * M - 1, ext = g.ldim[L][d];
        long long s0 = (a.lo[d] == 0) ? 0 : a.lo[d] - base;
        long long s1 = (a.hi[d] == ext - 1) ? S - 1 : a.hi[d] - base;
        if (s0 < 0) s0 = 0;
        if (s1 > S - 1) s1 = S - 1;
        l0[d] = (int)s0;
        l1[d] = (int)s1;
        if (s0 > s1) return;
        interior = interior && (b[d] * M <= a.hi[d]) && (b[d] * M + M - 1 >= a.lo[d]);
    }
    uint16_t* dst = a.pool + (long long)slot * g.slot_elems;
    const int nx = l1[0] - l0[0] + 1, ny = l1[1] - l0[1] + 1;
    const int np = nx * ny;
    int nin[3]; // in-volume interior extent of this brick
    for (int d = 0; d < 3; ++d) {
        const long long r = g.ldim[L][d] - b[d] * M;
        nin[d] = (int)(r < M ? r : M);
    }
    // When the change covers every interior in-volume position of a plane (always for whole
    // slices) the plane statistics are gathered while writing: per thread, per warp (reduce
    // instructions), then one shared atomic per warp and plane; otherwise re-read afterwards.
    const bool full_xy = l0[0] <= 1 && l1[0] >= nin[0] && l0[1] <= 1 && l1[1] >= nin[1];
    const bool gather = interior && full_xy; // uniform in the CTA
    __shared__ uint32_t s_pmn[MAX_S][C], s_pmx[MAX_S][C], s_psm[MAX_S][C];
    __shared__ FinalizeInputs<C> s_fi;
    if (gather) {
        for (int i = threadIdx.x; i < S * C; i += blockDim.x) {
            s_pmn[i / C][i % C] = 0xffffu;
            s_pmx[i / C][i % C] = 0u;
            s_psm[i / C][i % C] = 0u;
        }
        __syncthreads();
    }
    const int bx0 = (int)(b[0] * M) - 1, by0 = (int)(b[1] * M) - 1, bz0 = (int)(b[2] * M) - 1;
    const int X = (int)g.ldim[L][0], Y = (int)g.ldim[L][1], Z = (int)g.ldim[L][2];
    const int msh = a.mshift; // log2(M) when M is a power of two, else -1
    // t / nx as a multiply-high: exact because t * nx < S^3 < 2^32
    const uint32_t mnx = nx > 1 ? (uint32_t)((0x100000000ull + (unsigned)nx - 1) / (unsigned)nx) : 0u;
    // U positions per thread per round: their loads are issued before any of their stores
    constexpr int U = LEVEL0 ? 4 : 2;
    const uint16_t* __restrict__ blk = a.block;
    // the slot lookups above read only what the insert's slot set-up wrote (complete before level
    // 0 starts); the children (level L - 1) are complete once this returns
    pdl_wait();
    if (gather && threadIdx.x < 32)
        finalize_inputs<C>(a, b, slot, l0[2] > 1 ? l0[2] : 1, l1[2] < nin[2] ? l1[2] : nin[2], nin[2], s_fi);
    for (int lz = l0[2]; lz <= l1[2]; ++lz) {
        const int z = clampi(bz0 + lz, 0, Z - 1);
        const bool stats_here = gather && lz >= 1 && lz <= nin[2]; // uniform in the CTA
        uint32_t mn[C], mx[C], sm32[C]; // a thread's share of one plane stays below 2^32
#pragma unroll
        for (int c = 0; c < C; ++c) {
            mn[c] = 0xffffu;
            mx[c] = 0;
            sm32[c] = 0;
        }
        const uint16_t* src_plane = LEVEL0 ? blk + (long long)(z - a.org[2]) * a.ext[1] * a.ext[0] * C : nullptr;
        for (int t0 = threadIdx.x; t0 < np; t0 += U * blockDim.x) {
            uint16_t v[U][VS];
            int lxs[U], lys[U];
            bool ok[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int t = t0 + u * (int)blockDim.x;
                ok[u] = t < np;
#pragma unroll
                for (int c = 0; c < VS; ++c) v[u][c] = 0;
                const int ty = nx > 1 ? (int)__umulhi((uint32_t)t, mnx) : t;
                lxs[u] = l0[0] + (t - ty * nx);
                lys[u] = l0[1] + ty;
                if (!ok[u]) continue;
                const int x = clampi(bx0 + lxs[u], 0, X - 1), y = clampi(by0 + lys[u], 0, Y - 1);
                if (LEVEL0) {
                    const uint16_t* src = src_plane + ((long long)(y - a.org[1]) * a.ext[0] + (x - a.org[0])) * C;
#pragma unroll
                    for (int c = 0; c < C; ++c) v[u][c] = src[c];
                } else {
                    half_sample<C, VS>(a, L, x, y, z, msh, v[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (!ok[u]) continue;
                uint16_t* d = dst + ((lz * S + lys[u]) * S + lxs[u]) * VS;
                if (VS == 4) {
                    uint2 w;
                    w.x = (uint32_t)v[u][0] | ((uint32_t)v[u][VS > 1 ? 1 : 0] << 16);
                    w.y = (uint32_t)v[u][VS > 2 ? 2 : 0] | ((uint32_t)v[u][VS > 3 ? 3 : 0] << 16);
                    *reinterpret_cast<uint2*>(d) = w;
                } else if (VS == 2) {
                    *reinterpret_cast<uint32_t*>(d) = (uint32_t)v[u][0] | ((uint32_t)v[u][VS > 1 ? 1 : 0] << 16);
                } else {
                    d[0] = v[u][0];
                }
                if (stats_here && lxs[u] >= 1 && lxs[u] <= nin[0] && lys[u] >= 1 && lys[u] <= nin[1]) {
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        mn[c] = min(mn[c], (uint32_t)v[u][c]);
                        mx[c] = max(mx[c], (uint32_t)v[u][c]);
                        sm32[c] += v[u][c];
                    }
                }
            }
        }
        if (stats_here) {
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const uint32_t wmn = __reduce_min_sync(0xffffffffu, mn[c]);
                const uint32_t wmx = __reduce_max_sync(0xffffffffu, mx[c]);
                const uint32_t wsm = __reduce_add_sync(0xffffffffu, sm32[c]);
                if ((threadIdx.x & 31) == 0) {
                    atomicMin(&s_pmn[lz][c], wmn);
                    atomicMax(&s_pmx[lz][c], wmx);
                    atomicAdd(&s_psm[lz][c], wsm);
                }
            }
        }
    }
    finish_slot<C, VS>(a, b, nid, slot, dst, l0, l1, nin, interior, full_xy, gather, s_pmn, s_pmx, s_psm, &s_fi);
}

// ---- level 0 with the block's rows staged in shared memory by the tensor memory accelerator ----
//
// One CTA per level-0 slot as above.  For each chunk of up to `pb_max` changed planes, thread 0
// issues one bulk tensor copy per plane: the box of bw x bh elements of the block that holds the
// plane's (M+2)^2 clamped positions, its x origin rounded down to a 16-byte boundary (the copy's
// alignment rule); positions past the block's end read zeros that no position uses.  The CTA
// waits on one mbarrier (bounded), then each warp converts one plane (or its share of one) from
// shared memory into 8-byte slot voxels, gathering that plane's statistics in registers.

constexpr long long COPY_WAIT_CYCLES = 4000000000ll; // ~2 s at 2 GHz: a copy that never lands

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// true once the barrier's phase `parity` has completed; false after COPY_WAIT_CYCLES
__device__ __forceinline__ bool wait_phase(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > COPY_WAIT_CYCLES) return false;
    }
}

template <int C, int VS>
__global__ void __launch_bounds__(256) level0_staged_kernel(LevelArgs a, const __grid_constant__ CUtensorMap tm,
                                                            int bw, int bh, int plane_bytes, int pb_max) {
    extern __shared__ __align__(128) unsigned char s_dyn[];
    __shared__ __align__(8) unsigned long long s_bar;
    // the copies' destinations on a 128-byte boundary (the launch adds 128 bytes of slack)
    unsigned char* const s_box = s_dyn + ((128u - (smem_u32(s_dyn) & 127u)) & 127u);
    __shared__ uint32_t s_pmn[MAX_S][C], s_pmx[MAX_S][C], s_psm[MAX_S][C];
    const Geo& g = a.g;
    const int M = g.M, S = g.S;
    long long bb = blockIdx.x;
    long long b[3];
    b[0] = a.blo[0] + bb % a.bn[0];
    bb /= a.bn[0];
    b[1] = a.blo[1] + bb % a.bn[1];
    b[2] = a.blo[2] + bb / a.bn[1];
    const long long nid = g.noff[0] + (b[2] * g.nb[0][1] + b[1]) * g.nb[0][0] + b[0];
    const int slot = a.rn[nid].slot;
    if (slot < 0) return;
    if (slot >= g.n_slots_cap) {
        if (threadIdx.x == 0) atomicOr(a.err, ERR_SLOT_RANGE);
        return;
    }
    int l0[3], l1[3];
    bool interior = true;
    for (int d = 0; d < 3; ++d) {
        long long base = b[d] * M - 1, ext = g.ldim[0][d];
        long long s0 = (a.lo[d] == 0) ? 0 : a.lo[d] - base;
        long long s1 = (a.hi[d] == ext - 1) ? S - 1 : a.hi[d] - base;
        if (s0 < 0) s0 = 0;
        if (s1 > S - 1) s1 = S - 1;
        l0[d] = (int)s0;
        l1[d] = (int)s1;
        if (s0 > s1) return;
        interior = interior && (b[d] * M <= a.hi[d]) && (b[d] * M + M - 1 >= a.lo[d]);
    }
    uint16_t* dst = a.pool + (long long)slot * g.slot_elems;
    const int nx = l1[0] - l0[0] + 1, ny = l1[1] - l0[1] + 1;
    const int np = nx * ny;
    int nin[3];
    for (int d = 0; d < 3; ++d) {
        const long long r = g.ldim[0][d] - b[d] * M;
        nin[d] = (int)(r < M ? r : M);
    }
    const bool full_xy = l0[0] <= 1 && l1[0] >= nin[0] && l0[1] <= 1 && l1[1] >= nin[1];
    const bool gather = interior && full_xy;
    const uint32_t bar = smem_u32(&s_bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (gather)
        for (int i = threadIdx.x; i < S * C; i += blockDim.x) {
            s_pmn[i / C][i % C] = 0xffffu;
            s_pmx[i / C][i % C] = 0u;
            s_psm[i / C][i % C] = 0u;
        }
    __syncthreads();
    const int bx0 = (int)(b[0] * M) - 1, by0 = (int)(b[1] * M) - 1, bz0 = (int)(b[2] * M) - 1;
    const int X = (int)g.ldim[0][0], Y = (int)g.ldim[0][1], Z = (int)g.ldim[0][2];
    const int ox = (int)a.org[0], oy = (int)a.org[1], oz = (int)a.org[2];
    // the box: rows from the first position's clamped y, elements from its clamped x (times C)
    // rounded down to a multiple of 8 (16 bytes)
    const int ya = clampi(by0 + l0[1], 0, Y - 1);
    const int ex = ((clampi(bx0 + l0[0], 0, X - 1) - ox) * C) & ~7;
    const uint32_t mnx = nx > 1 ? (uint32_t)((0x100000000ull + (unsigned)nx - 1) / (unsigned)nx) : 0u;
    const int nw = (int)(blockDim.x >> 5), w = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
    constexpr int U = 4;
    uint32_t parity = 0;
    for (int pz0 = l0[2]; pz0 <= l1[2]; pz0 += pb_max) {
        const int pb = min(pb_max, l1[2] - pz0 + 1);
        if (threadIdx.x == 0) {
            // the previous chunk's reads of these buffers (ordered by the barrier below) come first
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(pb * bw * bh * 2)
                         : "memory");
            for (int p = 0; p < pb; ++p) {
                const int z = clampi(bz0 + pz0 + p, 0, Z - 1) - oz;
                asm volatile(
                    "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                    ::"r"(smem_u32(s_box + p * plane_bytes)), "l"(reinterpret_cast<unsigned long long>(&tm)), "r"(ex),
                      "r"(ya - oy), "r"(z), "r"(bar)
                    : "memory");
            }
        }
        const bool late = !wait_phase(bar, parity);
        parity ^= 1u;
        if (__syncthreads_or(late)) {
            if (threadIdx.x == 0) atomicOr(a.err, ERR_COPY_TIMEOUT);
            return;
        }
        // warps to planes: gw warps share one plane when the chunk has fewer planes than warps
        const int gw = pb >= nw ? 1 : nw / pb;
        for (int p = w / gw; p < pb; p += nw / gw) {
            const int lz = pz0 + p;
            const bool stats_here = gather && lz >= 1 && lz <= nin[2];
            const uint16_t* sp = reinterpret_cast<const uint16_t*>(s_box + p * plane_bytes);
            uint32_t mn[C], mx[C], sm32[C];
#pragma unroll
            for (int c = 0; c < C; ++c) {
                mn[c] = 0xffffu;
                mx[c] = 0;
                sm32[c] = 0;
            }
            const int stride = gw * 32;
            for (int t0 = (w % gw) * 32 + lane; t0 < np; t0 += U * stride) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int t = t0 + u * stride;
                    if (t >= np) break;
                    const int ty = nx > 1 ? (int)__umulhi((uint32_t)t, mnx) : t;
                    const int lx = l0[0] + (t - ty * nx), ly = l0[1] + ty;
                    const int x = clampi(bx0 + lx, 0, X - 1), y = clampi(by0 + ly, 0, Y - 1);
                    const uint16_t* q = sp + (y - ya) * bw + ((x - ox) * C - ex);
                    uint16_t v[VS];
#pragma unroll
                    for (int c = 0; c < VS; ++c) v[c] = c < C ? q[c] : (uint16_t)0;
                    uint16_t* d = dst + ((lz * S + ly) * S + lx) * VS;
                    if (VS == 4) {
                        uint2 wv;
                        wv.x = (uint32_t)v[0] | ((uint32_t)v[VS > 1 ? 1 : 0] << 16);
                        wv.y = (uint32_t)v[VS > 2 ? 2 : 0] | ((uint32_t)v[VS > 3 ? 3 : 0] << 16);
                        *reinterpret_cast<uint2*>(d) = wv;
                    } else if (VS == 2) {
                        *reinterpret_cast<uint32_t*>(d) = (uint32_t)v[0] | ((uint32_t)v[VS > 1 ? 1 : 0] << 16);
                    } else {
                        d[0] = v[0];
                    }
                    if (stats_here && lx >= 1 && lx <= nin[0] && ly >= 1 && ly <= nin[1]) {
#pragma unroll
                        for (int c = 0; c < C; ++c) {
                            mn[c] = min(mn[c], (uint32_t)v[c]);
                            mx[c] = max(mx[c], (uint32_t)v[c]);
                            sm32[c] += v[c];
                        }
                    }
                }
            }
            if (stats_here) {
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const uint32_t wmn = __reduce_min_sync(0xffffffffu, mn[c]);
                    const uint32_t wmx = __reduce_max_sync(0xffffffffu, mx[c]);
                    const uint32_t wsm = __reduce_add_sync(0xffffffffu, sm32[c]);
                    if (lane == 0) {
                        atomicMin(&s_pmn[lz][c], wmn);
                        atomicMax(&s_pmx[lz][c], wmx);
                        atomicAdd(&s_psm[lz][c], wsm);
                    }
                }
            }
        }
        // every warp is done with this chunk's planes before the next chunk's copies land
        __syncthreads();
    }
    finish_slot<C, VS>(a, b, nid, slot, dst, l0, l1, nin, interior, full_xy, gather, s_pmn, s_pmx, s_psm);
}

template <int C, int VS>
static cudaError_t launch_level(const LevelArgs& a, bool level0, long long nblocks, cudaStream_t st) {
    if (level0) {
        level_update_kernel<C, VS, true><<<(unsigned)nblocks, 256, 0, st>>>(a);
        return cudaGetLastError();
    } else {
        // the upper levels have a few slots only: wider CTAs shorten each slot's chain of
        // dependent loads (child slot, then children) instead of leaving SMs idle.  Launched as
        // programmatic dependents of the level below (pdl_wait in the kernel).
        const bool wide = nblocks < 2 * 148;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)nblocks);
        cfg.blockDim = dim3(wide ? 1024u : 256u);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        return wide ? cudaLaunchKernelEx(&cfg, level_update_kernel<C, VS, false, true>, a)
                    : cudaLaunchKernelEx(&cfg, level_update_kernel<C, VS, false>, a);
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        else
            cudaGetLastError();
    }
    return fn;
}

constexpr int STAGE_SMEM_MAX = 32 * 1024; // staged planes of one level-0 CTA (+ 128 bytes of alignment slack)
constexpr int STAGE_PLANES_MAX = 8;

// Level 0 through level0_staged_kernel when the block allows it: base and rows 16-byte aligned,
// and the box of one slot plane within the copy engine's 256-element box limit.  Returns false
// (nothing launched) otherwise.
template <int C, int VS>
static bool launch_level0_staged(const LevelArgs& a, long long nblocks, cudaStream_t st, cudaError_t* e) {
    const Geo& g = a.g;
    const int S = g.S;
    const int bw = ((S * C + 7) + 7) & ~7, bh = S;
    const unsigned long long row = (unsigned long long)a.ext[0] * C * sizeof(uint16_t);
    if (bw > 256 || bh > 256 || ((uintptr_t)a.block & 15u) != 0 || (row & 15u) != 0) return false;
    const int plane_bytes = (bw * bh * 2 + 127) & ~127;
    int pb_max = STAGE_SMEM_MAX / plane_bytes;
    if (pb_max > STAGE_PLANES_MAX) pb_max = STAGE_PLANES_MAX;
    if (pb_max < 1) return false;
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    CUtensorMap tm;
    const cuuint64_t dims[3] = {(cuuint64_t)a.ext[0] * C, (cuuint64_t)a.ext[1], (cuuint64_t)a.ext[2]};
    const cuuint64_t strides[2] = {row, row * (cuuint64_t)a.ext[1]};
    const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<uint16_t*>(a.block), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    const int smem = pb_max * plane_bytes + 128;
    *e = cudaFuncSetAttribute(level0_staged_kernel<C, VS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (*e != cudaSuccess) return true;
    level0_staged_kernel<C, VS><<<(unsigned)nblocks, 256, smem, st>>>(a, tm, bw, bh, plane_bytes, pb_max);
    *e = cudaGetLastError();
    return true;
}

cudaError_t launch_level_update(const Geo& g, int L, const long long lo[3], const long long hi[3],
                                const uint16_t* block, const long long org[3], const long long ext[3], uint16_t* pool,
                                RNode* rn, NStat* ns, PStat* ps, int* err, cudaStream_t st, bool stage_rows) {
    LevelArgs a;
    a.g = g;
    a.L = L;
    long long nblocks = 1;
    for (int d = 0; d < 3; ++d) {
        a.lo[d] = lo[d];
        a.hi[d] = hi[d];
        // bricks whose clamped slot range [b M - 1, b M + M] meets [lo, hi]
        long long b0 = (lo[d] + g.M - 1) / g.M - 1; // ceil(lo / M) - 1
        long long b1 = (hi[d] + 1) / g.M;
        if (b0 < 0) b0 = 0;
        if (b1 > g.nb[L][d] - 1) b1 = g.nb[L][d] - 1;
        a.blo[d] = b0;
        a.bn[d] = b1 - b0 + 1;
        nblocks *= a.bn[d];
        a.org[d] = org ? org[d] : 0;
        a.ext[d] = ext ? ext[d] : 0;
    }
    a.block = block;
    a.mshift = -1;
    if (g.pow2)
        for (int sft = 0; sft < 31; ++sft)
            if ((1 << sft) == g.M) a.mshift = sft;
    a.pool = pool;
    a.rn = rn;
    a.ns = ns;
    a.ps = ps;
    a.err = err;
    if (nblocks <= 0) return cudaSuccess;
    if (nblocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (L == 0 && stage_rows) {
        cudaError_t e = cudaSuccess;
        bool done = false;
        switch (g.C) {
            case 1: done = launch_level0_staged<1, 1>(a, nblocks, st, &e); break;
            case 2: done = launch_level0_staged<2, 2>(a, nblocks, st, &e); break;
            case 3: done = launch_level0_staged<3, 4>(a, nblocks, st, &e); break;
            default: done = launch_level0_staged<4, 4>(a, nblocks, st, &e); break;
        }
        if (done) return e;
    }
    switch (g.C) {
        case 1: return launch_level<1, 1>(a, L == 0, nblocks, st);
        case 2: return launch_level<2, 2>(a, L == 0, nblocks, st);
        case 3: return launch_level<3, 4>(a, L == 0, nblocks, st);
        default: return launch_level<4, 4>(a, L == 0, nblocks, st);
    }
}

__global__ void read_level_kernel(Geo g, int L, const uint16_t* __restrict__ pool, const RNode* __restrict__ rn,
                                  uint16_t* __restrict__ out) {
    const long long X = g.ldim[L][0], Y = g.ldim[L][1], Z = g.ldim[L][2];
    const long long n = X * Y * Z;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        long long x = i % X, y = (i / X) % Y, z = i / (X * Y);
        long long bx = x / g.M, by = y / g.M, bz = z / g.M;
        int slot = rn[g.noff[L] + (bz * g.nb[L][1] + by) * g.nb[L][0] + bx].slot;
        for (int c = 0; c < g.C; ++c) {
            uint16_t v = g.bg;
            if (slot >= 0 && slot < g.n_slots_cap)
                v = pool[(long long)slot * g.slot_elems +
                         (((z - bz * g.M + 1) * g.S + (y - by * g.M + 1)) * g.S + (x - bx * g.M + 1)) * g.VS + c];
            out[i * g.C + c] = v;
        }
    }
}

cudaError_t launch_read_level(const Geo& g, int L, const uint16_t* pool, const RNode* rn, uint16_t* out,
                              cudaStream_t st) {
    long long n = g.ldim[L][0] * g.ldim[L][1] * g.ldim[L][2];
    long long blocks = (n + 255) / 256;
    if (blocks > 148 * 32) blocks = 148 * 32;
    if (blocks < 1) blocks = 1;
    read_level_kernel<<<(unsigned)blocks, 256, 0, st>>>(g, L, pool, rn, out);
    return cudaGetLastError();
}

__global__ void read_voxels_kernel(Geo g, int L, const uint16_t* __restrict__ pool, const RNode* __restrict__ rn,
                                   const long long* __restrict__ xyz, long long n, uint16_t* __restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
        const long long bx = x / g.M, by = y / g.M, bz = z / g.M;
        const int slot = rn[g.noff[L] + (bz * g.nb[L][1] + by) * g.nb[L][0] + bx].slot;
        for (int c = 0; c < g.C; ++c) {
            uint16_t v = g.bg;
            if (slot >= 0 && slot < g.n_slots_cap)
                v = pool[(long long)slot * g.slot_elems +
                         (((z - bz * g.M + 1) * g.S + (y - by * g.M + 1)) * g.S + (x - bx * g.M + 1)) * g.VS + c];
            out[i * g.C + c] = v;
        }
    }
}

cudaError_t launch_read_voxels(const Geo& g, int L, const uint16_t* pool, const RNode* rn, const long long* xyz,
                               long long n, uint16_t* out, cudaStream_t st) {
    long long blocks = (n + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    if (blocks < 1) return cudaSuccess;
    read_voxels_kernel<<<(unsigned)blocks, 256, 0, st>>>(g, L, pool, rn, xyz, n, out);
    return cudaGetLastError();
}

__global__ void prepare_tf_kernel(int C, const float* __restrict__ tf, const float* __restrict__ scale,
                                  float4* __restrict__ tf2, float* __restrict__ scl) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < C * 256) {
        int e = i & 255;
        float4 v = make_float4(tf[4 * i], tf[4 * i + 1], tf[4 * i + 2], tf[4 * i + 3]);
        float4 w = v;
        if (e < 255) w = make_float4(tf[4 * i + 4], tf[4 * i + 5], tf[4 * i + 6], tf[4 * i + 7]);
        tf2[2 * i] = v;
        tf2[2 * i + 1] = make_float4(w.x - v.x, w.y - v.y, w.z - v.z, w.w - v.w);
    }
    if (i < C) {
        scl[i] = scale[i] / 65535.0f; // what the render multiplies raw intensities by
        scl[MAXC + i] = scale[i];     // unrounded, for the double-precision gradient check
    }
}

cudaError_t launch_prepare_tf(int C, const float* tf, const float* scale, float4* tf2, float* scl, cudaStream_t st) {
    prepare_tf_kernel<<<(C * 256 + 255) / 256, 256, 0, st>>>(C, tf, scale, tf2, scl);
    return cudaGetLastError();
}

} // namespace vrk
