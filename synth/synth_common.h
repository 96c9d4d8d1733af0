/*
 * synth_common.h -- seeded, counter-based generator of synthetic multi-channel
 * microscopy volumes (SPIM-like stand-ins for the paper's data sets D1-D3,
 * Table 1).  This module produces INPUTS only: it holds none of the renderer's
 * or the oracle's arithmetic (no downsampling, no octree, no compositing).
 *
 * The same inline functions are compiled twice: by gcc for the host
 * generator (synth_host.c, built with -ffp-contract=off) and by nvcc for the
 * device generator (synth_dev.cu).  Every floating-point step below is an
 * IEEE correctly-rounded single-precision operation (+, -, *, /, sqrt) in a
 * fixed order; on the device the _rn intrinsics forbid FMA contraction.  The
 * exponential is this file's own (Cody-Waite range reduction by ln 2 and a
 * degree-9 Taylor polynomial), so no libm/libdevice routine enters the value.
 * Host and device therefore produce bit-identical voxels for the same
 * (seed, channel, x, y, z).
 *
 * Voxel model:
 *   lambda_c(x,y,z) = base(x,y,z) + sum_j peak_{j,c} * exp(-q_{j,c})
 *   q_{j,c} = ((dx^2 + dy^2) * ia_{j,c}) + (dz^2 * ib_{j,c}),  d = voxel centre - centre_j
 *   terms with q >= 12.5 are dropped (support radius 5 sigma)
 *   value_c = Poisson(lambda_c): Knuth's product-of-uniforms method for
 *             lambda < 30, else the normal approximation
 *             floor(lambda + sqrt(lambda) * Z + 0.5), Z = (sum of 12 uniforms) - 6
 *             (Irwin-Hall), clamped to [0, 65535].
 *   base = 0 for the blob volumes; 100 (+200 inside the tissue ellipsoid)
 *   for the SPIM-like volumes.
 * Randomness is SplitMix64 (Steele, Lea, Flood 2014) keyed by
 * (seed, channel, x, y, z), so any slice can be produced independently.
 */
#ifndef SYNTH_COMMON_H
#define SYNTH_COMMON_H
#include <stdint.h>

#if defined(__CUDACC__)
#define SY_FN __host__ __device__ static inline
#else
#define SY_FN static inline
#endif

#if defined(__CUDA_ARCH__)
#define SY_MUL(a, b) __fmul_rn((a), (b))
#define SY_ADD(a, b) __fadd_rn((a), (b))
#define SY_SUB(a, b) __fsub_rn((a), (b))
#define SY_SQRT(a) __fsqrt_rn(a)
#define SY_FLOOR(a) floorf(a)
#define SY_F2BITS(f) __float_as_uint(f)
#define SY_BITS2F(u) __uint_as_float(u)
#else
#include <math.h>
#include <string.h>
#define SY_MUL(a, b) ((a) * (b))
#define SY_ADD(a, b) ((a) + (b))
#define SY_SUB(a, b) ((a) - (b))
#define SY_SQRT(a) sqrtf(a)
#define SY_FLOOR(a) floorf(a)
static inline uint32_t sy_f2bits_(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static inline float sy_bits2f_(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
#define SY_F2BITS(f) sy_f2bits_(f)
#define SY_BITS2F(u) sy_bits2f_(u)
#endif

#define SY_GOLDEN 0x9e3779b97f4a7c15ULL
#define SY_MAXC 4
#define SY_QCUT 12.5f

/* Kinds of synthetic volume. */
#define SY_KIND_BLOBS 0 /* isotropic Gaussian blobs per channel, no offset */
#define SY_KIND_SPIM 1  /* tissue ellipsoid + anisotropic nuclei, offset 100 (+200 in tissue) */

/* One emitter: centre and, per channel, peak and the two inverse widths
 * ia = 1/(2 sigma_xy^2), ib = 1/(2 sigma_z^2).  peak == 0 means absent. */
typedef struct {
    float cx, cy, cz, pad;
    float peak[SY_MAXC];
    float ia[SY_MAXC];
    float ib[SY_MAXC];
} sy_nucleus;

/* Plain-pointer view of a generator specification (host or device memory). */
typedef struct {
    int kind, C;
    int64_t X, Y, Z;
    uint64_t seed;
    float mask_c[3];  /* tissue ellipsoid centre */
    float mask_ia[3]; /* 1 / semi-axis */
    int cell;         /* cell edge of the spatial index, voxels */
    int ncx, ncy, ncz;
    const sy_nucleus* nuclei;
    const int64_t* cell_start; /* ncx*ncy*ncz + 1 offsets into cell_idx */
    const int32_t* cell_idx;   /* nucleus ids, ascending within a cell */
} sy_view;

SY_FN uint64_t sy_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* Next uniform float in [0,1) with 24 random bits (exact conversion). */
SY_FN float sy_uniform(uint64_t* st) {
    *st += SY_GOLDEN;
    uint64_t r = sy_mix64(*st);
    return (float)(uint32_t)(r >> 40) * (1.0f / 16777216.0f);
}

SY_FN uint64_t sy_voxel_key(uint64_t seed, int c, int64_t x, int64_t y, int64_t z) {
    uint64_t k = sy_mix64(seed ^ ((uint64_t)(c + 1) * 0xd1b54a32d192ed03ULL));
    uint64_t p = (uint64_t)x | ((uint64_t)y << 21) | ((uint64_t)z << 42);
    return sy_mix64(k ^ sy_mix64(p));
}

/* exp(-q) for q >= 0: q = k ln2 + r with r in [0, ln2) (Cody-Waite split of
 * ln 2 into a 16-bit head and a tail), e^-r by its Taylor series to degree 9
 * (truncation error < 3e-9), times 2^-k built from the exponent bits. */
SY_FN float sy_expneg(float q) {
    if (!(q < 87.0f)) return 0.0f;
    const float LOG2E = 1.44269502f;
    const float LN2_HI = 0.693145751953125f; /* 16 significant bits: k*LN2_HI exact */
    const float LN2_LO = 1.42860677e-06f;
    float kf = SY_FLOOR(SY_MUL(q, LOG2E));
    float r = SY_SUB(SY_SUB(q, SY_MUL(kf, LN2_HI)), SY_MUL(kf, LN2_LO));
    /* Horner: 1 - r(1 - r/2(1 - r/3(... (1 - r/9)))) */
    float t = 1.0f;
    t = SY_SUB(1.0f, SY_MUL(SY_MUL(r, 0.111111112f), t));
    t = SY_SUB(1.0f, SY_MUL(SY_MUL(r, 0.125f), t));
    t = SY_SUB(1.0f, SY_MUL(SY_MUL(r, 0.142857149f), t));
    t = SY_SUB(1.0f, SY_MUL(SY_MUL(r, 0.166666672f), t));
    t = SY_SUB(1.0f, SY_MUL(SY_MUL(r, 0.2f), t));
    t = SY_SUB(1.0f, SY_MUL(SY_MUL(r, 0.25f), t));
    t = SY_SUB(1.0f, SY_MUL(SY_MUL(r, 0.333333343f), t));
    t = SY_SUB(1.0f, SY_MUL(SY_MUL(r, 0.5f), t));
    t = SY_SUB(1.0f, SY_MUL(r, t));
    int k = (int)kf;
    float scale = SY_BITS2F((uint32_t)(127 - k) << 23); /* 2^-k, k in [0,125] */
    return SY_MUL(t, scale);
}

SY_FN uint16_t sy_poisson(float lam, uint64_t key) {
    uint64_t st = key;
    if (lam < 30.0f) {
        float L = sy_expneg(lam);
        float p = 1.0f;
        int k = 0;
        for (;;) {
            p = SY_MUL(p, sy_uniform(&st));
            if (p <= L || k >= 1000) break;
            ++k;
        }
        return (uint16_t)k;
    }
    float s = 0.0f;
    for (int i = 0; i < 12; ++i) s = SY_ADD(s, sy_uniform(&st));
    float zn = SY_SUB(s, 6.0f);
    float v = SY_FLOOR(SY_ADD(SY_ADD(lam, SY_MUL(SY_SQRT(lam), zn)), 0.5f));
    if (v < 0.0f) v = 0.0f;
    if (v > 65535.0f) v = 65535.0f;
    return (uint16_t)(int)v;
}

/* All C channel values of voxel (x, y, z) (voxel centre at +0.5). */
SY_FN void sy_voxel(const sy_view* s, int64_t x, int64_t y, int64_t z, uint16_t* out) {
    float xf = (float)x + 0.5f, yf = (float)y + 0.5f, zf = (float)z + 0.5f;
    float base = 0.0f;
    if (s->kind == SY_KIND_SPIM) {
        float ex = SY_MUL(SY_SUB(xf, s->mask_c[0]), s->mask_ia[0]);
        float ey = SY_MUL(SY_SUB(yf, s->mask_c[1]), s->mask_ia[1]);
        float ez = SY_MUL(SY_SUB(zf, s->mask_c[2]), s->mask_ia[2]);
        float e = SY_ADD(SY_ADD(SY_MUL(ex, ex), SY_MUL(ey, ey)), SY_MUL(ez, ez));
        base = (e <= 1.0f) ? 300.0f : 100.0f;
    }
    float lam[SY_MAXC];
    for (int c = 0; c < s->C; ++c) lam[c] = base;
    int64_t cx = x / s->cell, cy = y / s->cell, cz = z / s->cell;
    int64_t cell = (cz * s->ncy + cy) * s->ncx + cx;
    for (int64_t j = s->cell_start[cell]; j < s->cell_start[cell + 1]; ++j) {
        const sy_nucleus* n = &s->nuclei[s->cell_idx[j]];
        float dx = SY_SUB(xf, n->cx), dy = SY_SUB(yf, n->cy), dz = SY_SUB(zf, n->cz);
        float dxy2 = SY_ADD(SY_MUL(dx, dx), SY_MUL(dy, dy));
        float dz2 = SY_MUL(dz, dz);
        for (int c = 0; c < s->C; ++c) {
            if (n->peak[c] > 0.0f) {
                float q = SY_ADD(SY_MUL(dxy2, n->ia[c]), SY_MUL(dz2, n->ib[c]));
                if (q < SY_QCUT) lam[c] = SY_ADD(lam[c], SY_MUL(n->peak[c], sy_expneg(q)));
            }
        }
    }
    for (int c = 0; c < s->C; ++c) out[c] = sy_poisson(lam[c], sy_voxel_key(s->seed, c, x, y, z));
}

#endif
