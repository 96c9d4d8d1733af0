/*
 * oracle_render.c -- TEST INFRASTRUCTURE (FP64 CPU oracle; see oracle.h).
 *
 * Algorithm 1 (DVR ray traversal) and the surrounding text of Sec. "Basic
 * Ray-Casting", written out sample by sample:
 *
 *   ray setup      pinhole camera; [t0, t1) = the ray inside the real volume
 *                  box [0,X]x[0,Y]x[0,Z], inside every clip half-space
 *                  n.p + d >= 0 (up to three clipping planes, Sec. "Integration
 *                  into Voreen"), and t >= 0;
 *   march          t_k = t0 + k*step while t_k < t1; segment length
 *                  l_k = min(step, t1 - t_k);
 *   LOD            the level whose voxel projects to the pixel size: the
 *                  largest L <= N with t_k >= t_L,
 *                  t_L = 2^L H / (2 eps tan(fov/2));
 *   node           descend from the root to the child whose box holds the
 *                  sample, until the desired level or a node without
 *                  children (getNodeAtPosition);
 *   intensity      per channel: the node's AVG if it has no brick, else
 *                  trilinear interpolation of that level's values
 *                  (clamp-to-edge at the real extent);
 *   TF             x = clamp(s_c I / 65535, 0, 1), linear interpolation in the
 *                  channel's 256-entry RGBA table;
 *   composite      inside the channel loop (accumulation-level intermixing):
 *                  a = 1 - (1 - alpha)^l, C += (1-A) a rgb, A += (1-A) a;
 *   ERT            stop after a sample once A >= ert.
 *
 * Geometry (ray direction, interval, sample parameter and position, level
 * and node choice) is evaluated either in double precision (OR_GEOM_FP64, the
 * definition; decisions that lie within the single-precision error of their
 * threshold are flagged and both branches enumerated by or_render_check) or
 * in IEEE single precision in the operation order written here
 * (OR_GEOM_FP32, a mirror of a single-precision implementation); everything
 * downstream of the sample position is double.  See oracle.h.
 * This file must be compiled with -ffp-contract=off.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"
#include "oracle_internal.h"

typedef struct {
    float ff[3], rr[3], uu[3]; /* forward, right, up (unit), rounded to single precision */
    float kx, ky;              /* tan(fov/2) * W/H, tan(fov/2) */
    float tl[OR_MAXL];         /* level thresholds, tl[0] = 0 */
    double f64[3], r64[3], u64[3], kx64, ky64, tl64[OR_MAXL]; /* the same, unrounded */
} cam_derived;

static void cam_setup(const or_geom* g, const or_camera* cam, cam_derived* cd) {
    double th = tan(((double)cam->fov_y_deg * M_PI) / 360.0);
    double f[3], r[3], u[3], up[3];
    for (int a = 0; a < 3; ++a) {
        f[a] = (double)cam->target[a] - (double)cam->eye[a];
        up[a] = (double)cam->up[a];
    }
    double nf = sqrt((f[0] * f[0] + f[1] * f[1]) + f[2] * f[2]);
    for (int a = 0; a < 3; ++a) f[a] = f[a] / nf;
    r[0] = f[1] * up[2] - f[2] * up[1];
    r[1] = f[2] * up[0] - f[0] * up[2];
    r[2] = f[0] * up[1] - f[1] * up[0];
    double nr = sqrt((r[0] * r[0] + r[1] * r[1]) + r[2] * r[2]);
    for (int a = 0; a < 3; ++a) r[a] = r[a] / nr;
    u[0] = r[1] * f[2] - r[2] * f[1];
    u[1] = r[2] * f[0] - r[0] * f[2];
    u[2] = r[0] * f[1] - r[1] * f[0];
    for (int a = 0; a < 3; ++a) {
        cd->ff[a] = (float)f[a];
        cd->rr[a] = (float)r[a];
        cd->uu[a] = (float)u[a];
        cd->f64[a] = f[a];
        cd->r64[a] = r[a];
        cd->u64[a] = u[a];
    }
    cd->kx64 = (th * (double)cam->width) / (double)cam->height;
    cd->ky64 = th;
    cd->kx = (float)cd->kx64;
    cd->ky = (float)th;
    cd->tl[0] = 0.0f;
    cd->tl64[0] = 0.0;
    for (int L = 1; L <= g->N; ++L) {
        cd->tl64[L] = ldexp((double)cam->height, L) / ((2.0 * (double)cam->lod_error_px) * th);
        cd->tl[L] = (float)cd->tl64[L];
    }
}

/* ---- double-precision geometry and its knife-edge decisions (A16 reading) ----
 *
 * The quantities a single-precision implementation computes from the same camera differ from the
 * double-precision ones by rounding.  For each ray we bound that difference by forward error
 * analysis with unit roundoff u = 2^-24: the unit direction within OR_DIR_ULPS u per component
 * (the sum f + x r + y u, the norm and the division, with headroom for approximate square roots and
 * divisions), the entry parameter t0 within |t0| (ddir / |d_a| + 4u) for a box face of axis a (and
 * the corresponding bound for a clip plane), the sample parameter t_k = t0 + k dt within
 * dt0 + 2u t_k, and the sample position p = eye + t_k d within
 * dt_k |d_a| + t_k ddir + 2u (|eye_a| + t_k |d_a|) + u |p_a| per axis; OR_EDGE_SAFETY multiplies both.
 * A decision whose double-precision quantity lies within that bound of its threshold -- the level
 * choice t_k >= t_L, or the child choice at the parent's split plane -- is a knife edge when its
 * two branches sample differently (a different level or brick state, or a different AVG); either
 * branch is then a correct result. */
static const double U32 = 5.9604644775390625e-08; /* 2^-24 */
static double OR_DIR_ULPS = 8.0;    /* measured: <= 2.4 u for IEEE-rounded single-precision setup */
static double OR_EDGE_SAFETY = 1.5;

void or_set_edge_margins(double dir_ulps, double safety) {
    OR_DIR_ULPS = dir_ulps;
    OR_EDGE_SAFETY = safety;
}

typedef struct {
    const unsigned char* force; /* forced branches of the first nforce flagged decisions (1 = other) */
    int nforce;
    int nflag; /* flagged decisions met (output) */
} edge_ctl;

static int edge_take_other(edge_ctl* e) {
    int j = e->nflag++;
    return j < e->nforce ? (int)e->force[j] : 0;
}

/* Ray direction and [t0, t1) in double precision; *dt0 bounds the single-precision error of t0. */
static int ray_setup64(const or_geom* g, const or_camera* cam, const cam_derived* cd, int px, int py, double dir[3],
                       double* t0o, double* t1o, double* dt0) {
    double x = ((double)(2 * px + 1) / (double)cam->width - 1.0) * cd->kx64;
    double y = (1.0 - (double)(2 * py + 1) / (double)cam->height) * cd->ky64;
    double d[3];
    for (int i = 0; i < 3; ++i) d[i] = cd->f64[i] + x * cd->r64[i] + y * cd->u64[i];
    double s = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int i = 0; i < 3; ++i) dir[i] = d[i] / s;
    const double ddir = OR_DIR_ULPS * U32;
    double t0 = 0.0, t1 = INFINITY, e0 = 0.0;
    for (int i = 0; i < 3; ++i) {
        double o = (double)cam->eye[i], D = (double)g->dim[i];
        if (dir[i] != 0.0) {
            double ta = (0.0 - o) / dir[i], tb = (D - o) / dir[i];
            double lo = fmin(ta, tb), hi = fmax(ta, tb);
            double e = fabs(lo) * (ddir / fabs(dir[i]) + 4.0 * U32);
            if (lo > t0) {
                t0 = lo;
                e0 = e;
            } else if (lo == t0 && e > e0) {
                e0 = e;
            }
            t1 = fmin(t1, hi);
        } else if (o < 0.0 || o > D) {
            return 0;
        }
    }
    for (int p = 0; p < cam->n_clip; ++p) {
        const float* n = cam->clip[p];
        double sv = (double)n[0] * cam->eye[0] + (double)n[1] * cam->eye[1] + (double)n[2] * cam->eye[2] + (double)n[3];
        double q = (double)n[0] * dir[0] + (double)n[1] * dir[1] + (double)n[2] * dir[2];
        if (q == 0.0) {
            if (sv < 0.0) return 0;
        } else {
            double tc = -sv / q;
            double n1 = fabs((double)n[0]) + fabs((double)n[1]) + fabs((double)n[2]);
            double X = fabs((double)n[0] * cam->eye[0]) + fabs((double)n[1] * cam->eye[1]) +
                       fabs((double)n[2] * cam->eye[2]) + fabs((double)n[3]);
            double e = fabs(tc) * (n1 * ddir + 4.0 * U32) / fabs(q) + 4.0 * U32 * X / fabs(q);
            if (q > 0.0) {
                if (tc > t0) {
                    t0 = tc;
                    e0 = e;
                } else if (tc == t0 && e > e0) {
                    e0 = e;
                }
            } else {
                t1 = fmin(t1, tc);
            }
        }
    }
    *t0o = t0;
    *t1o = t1;
    *dt0 = e0;
    return t0 < t1;
}

/* Ray direction and [t0, t1); returns 0 for an empty interval. */
static int ray_setup(const or_geom* g, const or_camera* cam, const cam_derived* cd, int px, int py, float dir[3],
                     float* t0o, float* t1o) {
    float a = (float)(2 * px + 1);
    float cxp = a / (float)cam->width - 1.0f;
    float b = (float)(2 * py + 1);
    float cyp = 1.0f - b / (float)cam->height;
    float x = cxp * cd->kx, y = cyp * cd->ky;
    float d[3];
    for (int i = 0; i < 3; ++i) d[i] = (cd->ff[i] + x * cd->rr[i]) + y * cd->uu[i];
    float n2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
    float s = sqrtf(n2);
    for (int i = 0; i < 3; ++i) dir[i] = d[i] / s;
    float t0 = 0.0f, t1 = INFINITY;
    for (int i = 0; i < 3; ++i) {
        float o = cam->eye[i], D = (float)g->dim[i];
        if (dir[i] != 0.0f) {
            float ta = (0.0f - o) / dir[i], tb = (D - o) / dir[i];
            t0 = fmaxf(t0, fminf(ta, tb));
            t1 = fminf(t1, fmaxf(ta, tb));
        } else if (o < 0.0f || o > D) {
            return 0;
        }
    }
    for (int p = 0; p < cam->n_clip; ++p) {
        const float* n = cam->clip[p];
        float sv = ((n[0] * cam->eye[0] + n[1] * cam->eye[1]) + n[2] * cam->eye[2]) + n[3];
        float q = (n[0] * dir[0] + n[1] * dir[1]) + n[2] * dir[2];
        if (q == 0.0f) {
            if (sv < 0.0f) return 0;
        } else {
            float tc = (-sv) / q;
            if (q > 0.0f)
                t0 = fmaxf(t0, tc);
            else
                t1 = fminf(t1, tc);
        }
    }
    *t0o = t0;
    *t1o = t1;
    return t0 < t1;
}

int or_ray(const or_geom* g, const or_camera* cam, int px, int py, float dir[3], float* t0, float* t1) {
    cam_derived cd;
    cam_setup(g, cam, &cd);
    return ray_setup(g, cam, &cd, px, py, dir, t0, t1);
}

int or_lod_thresholds(const or_geom* g, const or_camera* cam, float* tl) {
    cam_derived cd;
    cam_setup(g, cam, &cd);
    for (int L = 0; L <= g->N; ++L) tl[L] = cd.tl[L];
    return 0;
}

/* getNodeAtPosition (Algorithm 1, and the descent described after it): start at the
 * root and descend to the child whose box contains p until level Lstar is reached or
 * the current node has no children.  Child boxes follow from halving the parent box;
 * the child index along an axis is floor(p / size) clamped to the parent's two
 * children and to the real node grid. */
static int descend_path(or_volume* v, const float p[3], int Lstar, or_node* nd, int64_t path[OR_MAXL][3]) {
    const or_geom* g = or_volume_geom(v);
    int lev = g->N;
    int64_t idx[3] = {0, 0, 0};
    or_node_info(v, lev, 0, 0, 0, nd);
    if (path) path[lev][0] = path[lev][1] = path[lev][2] = 0;
    while (lev > Lstar && nd->has_children) {
        --lev;
        float size = (float)((int64_t)g->M << lev);
        for (int a = 0; a < 3; ++a) {
            int64_t q = (int64_t)floorf(p[a] / size);
            int64_t c0 = 2 * idx[a];
            if (q < c0) q = c0;
            if (q > c0 + 1) q = c0 + 1;
            if (q > g->nb[lev][a] - 1) q = g->nb[lev][a] - 1;
            idx[a] = q;
        }
        or_node_info(v, lev, idx[0], idx[1], idx[2], nd);
        if (path)
            for (int a = 0; a < 3; ++a) path[lev][a] = idx[a];
    }
    return lev;
}

static int descend(or_volume* v, const float p[3], int Lstar, or_node* nd) { return descend_path(v, p, Lstar, nd, NULL); }

/* What a sample takes from the node a descent ends at: the level's trilinear value when the node
 * has a brick (the same value for every node of that level holding p: borders make the level one
 * continuous field), else the node's AVG. */
typedef struct {
    int lev, brick;
    uint16_t avg[OR_MAXC];
} outcome_t;

static int outcome_same(const outcome_t* a, const outcome_t* b, int C) {
    if (a->brick != b->brick) return 0;
    if (a->brick) return a->lev == b->lev;
    for (int c = 0; c < C; ++c)
        if (a->avg[c] != b->avg[c]) return 0;
    return 1;
}

/* The descent of getNodeAtPosition in double precision from node (lev, idx) towards Lstar.  With
 * ctl != NULL, a child choice along axis a whose coordinate lies within dp[a] of the parent's split
 * plane, with both children in the real node grid and sampling differently, is a knife edge:
 * ctl decides the branch. */
static int descend64(or_volume* v, const double p[3], const double dp[3], int Lstar, int lev, const int64_t idx0[3],
                     edge_ctl* ctl, outcome_t* oc) {
    const or_geom* g = or_volume_geom(v);
    int64_t idx[3] = {idx0[0], idx0[1], idx0[2]};
    or_node nd;
    or_node_info(v, lev, idx[0], idx[1], idx[2], &nd);
    while (lev > Lstar && nd.has_children) {
        --lev;
        double size = (double)((int64_t)g->M << lev);
        int64_t q[3];
        for (int a = 0; a < 3; ++a) {
            int64_t c0 = 2 * idx[a];
            q[a] = (p[a] < (double)(c0 + 1) * size) ? c0 : c0 + 1;
            if (q[a] > g->nb[lev][a] - 1) q[a] = g->nb[lev][a] - 1;
        }
        if (ctl) {
            for (int a = 0; a < 3; ++a) {
                int64_t c0 = 2 * idx[a];
                if (c0 + 1 > g->nb[lev][a] - 1) continue; /* one child only along this axis */
                if (fabs(p[a] - (double)(c0 + 1) * size) > dp[a]) continue;
                int64_t qo[3] = {q[0], q[1], q[2]};
                qo[a] = (q[a] == c0) ? c0 + 1 : c0;
                outcome_t o1, o2;
                descend64(v, p, dp, Lstar, lev, q, NULL, &o1);
                descend64(v, p, dp, Lstar, lev, qo, NULL, &o2);
                if (outcome_same(&o1, &o2, g->C)) continue;
                if (edge_take_other(ctl)) q[a] = qo[a];
            }
        }
        for (int a = 0; a < 3; ++a) idx[a] = q[a];
        or_node_info(v, lev, idx[0], idx[1], idx[2], &nd);
    }
    oc->lev = lev;
    oc->brick = nd.has_brick;
    for (int c = 0; c < g->C; ++c) oc->avg[c] = nd.avg[c];
    return lev;
}

/* The level choice L* = max{L <= N : t >= t_L} in double precision; a threshold within dtk of t
 * whose two levels sample differently is a knife edge (ctl decides). */
static int lod64(or_volume* v, const cam_derived* cd, double t, double dtk, const double p[3], const double dp[3],
                 edge_ctl* ctl) {
    const or_geom* g = or_volume_geom(v);
    int Lstar = 0;
    for (int L = 1; L <= g->N; ++L)
        if (t >= cd->tl64[L]) Lstar = L;
    if (!ctl) return Lstar;
    const int64_t root[3] = {0, 0, 0};
    for (int L = 1; L <= g->N; ++L) {
        if (fabs(t - cd->tl64[L]) > dtk + 2.0 * U32 * cd->tl64[L]) continue;
        int alt = (t >= cd->tl64[L]) ? L - 1 : L;
        if (alt == Lstar) continue;
        outcome_t o1, o2;
        descend64(v, p, dp, Lstar, g->N, root, NULL, &o1);
        descend64(v, p, dp, alt, g->N, root, NULL, &o2);
        if (outcome_same(&o1, &o2, g->C)) continue;
        if (edge_take_other(ctl)) Lstar = alt;
    }
    return Lstar;
}

int64_t or_node_count(const or_geom* g) {
    int64_t n = 0;
    for (int L = 0; L <= g->N; ++L) n += g->nb[L][0] * g->nb[L][1] * g->nb[L][2];
    return n;
}

/* Dense node numbering used for residency and flag arrays: levels 0..N in order, each level's
 * node grid x fastest. */
int64_t or_node_index(const or_geom* g, int L, int64_t i, int64_t j, int64_t k) {
    int64_t off = 0;
    for (int l = 0; l < L; ++l) off += g->nb[l][0] * g->nb[l][1] * g->nb[l][2];
    return off + (k * g->nb[L][1] + j) * g->nb[L][0] + i;
}

/* Trilinear interpolation of level L at p (level-0 units; voxel i centred at (i+0.5) 2^L). */
static double trilinear(or_volume* v, int L, const double p[3], int c) {
    const or_geom* g = or_volume_geom(v);
    int64_t i0[3], i1[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double u = ldexp(p[a], -L) - 0.5;
        double fl = floor(u);
        f[a] = u - fl;
        int64_t i = (int64_t)fl, hi = g->ldim[L][a] - 1;
        i0[a] = i < 0 ? 0 : (i > hi ? hi : i);
        i1[a] = i + 1 < 0 ? 0 : (i + 1 > hi ? hi : i + 1);
    }
    double s = 0.0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
                s += w * (double)or_value(v, L, dx ? i1[0] : i0[0], dy ? i1[1] : i0[1], dz ? i1[2] : i0[2], c);
            }
    return s;
}

double or_sample_trilinear(or_volume* v, int L, const float p[3], int c) {
    const double q[3] = {p[0], p[1], p[2]};
    return trilinear(v, L, q, c);
}

/* Transfer function (Alg. 1 applyTF): x = clamp(s I / 65535, 0, 1) indexes the 256 entries
 * at x * 255; the value is linear between the two neighbouring entries. */
static int tf_index(double s, double I, double* lam, double* xr_out) {
    double xr = s * I / 65535.0;
    double x = xr < 0.0 ? 0.0 : (xr > 1.0 ? 1.0 : xr);
    double w = x * 255.0;
    int i = (int)floor(w);
    if (i > 254) i = 254;
    *lam = w - (double)i;
    if (xr_out) *xr_out = xr;
    return i;
}

void or_tf_eval(const float* tfc, double s, double I, double rgba[4]) {
    double lam;
    int i = tf_index(s, I, &lam, NULL);
    for (int q = 0; q < 4; ++q) rgba[q] = (1.0 - lam) * (double)tfc[4 * i + q] + lam * (double)tfc[4 * i + 4 + q];
}

/* Per-(sample, channel) record for the adjoint. */
typedef struct {
    double I, lam, alpha, a, ell, A_before;
    int i, inside, aclamped, c;
} rec_t;

typedef struct {
    rec_t* r;
    int64_t n, cap;
} recbuf;

static void rec_push(recbuf* b, const rec_t* r) {
    if (b->n == b->cap) {
        b->cap = b->cap ? 2 * b->cap : 4096;
        b->r = (rec_t*)realloc(b->r, sizeof(rec_t) * (size_t)b->cap);
    }
    b->r[b->n++] = *r;
}

#define ALPHA_MAX (1.0 - 1e-6)

/* One ray.  mode 0: emission-absorption with ERT candidates; mode 1: MIP.
 * rec != NULL records the natural-decision forward for the adjoint. */
/* Per-channel affine sample transform (Sec. "Correction of Chromatic Aberration": each sampling
 * point is multiplied by the matrix of the current channel).  m is [3][4] (rows x, y, z; last
 * column the translation), evaluated in single precision in this order. */
static void channel_point(const float* m, const float p[3], float q[3]) {
    for (int i = 0; i < 3; ++i) q[i] = ((m[4 * i] * p[0] + m[4 * i + 1] * p[1]) + m[4 * i + 2] * p[2]) + m[4 * i + 3];
}

/* Brick cache state for out-of-core rendering (NULL res = every brick present). */
typedef struct {
    const uint8_t* res; /* per node: its brick is in the render cache */
    uint8_t* used;      /* per node: its brick was sampled (output) */
    uint8_t* req;       /* per node: its brick was requested (output) */
} cache_io;

/* Algorithmic footprint of a render (or_render_footprint): one bit per (level, voxel) read by a
 * trilinear corner and one per node entry read on a descent, for the samples up to the natural
 * stop.  Set with atomic ORs (rays run on several threads). */
typedef struct {
    uint8_t* vox[OR_MAXL];
    uint8_t* nodes;
} fp_io;

static void bit_set(uint8_t* bits, int64_t i) { __atomic_fetch_or(&bits[i >> 3], (uint8_t)(1u << (i & 7)), __ATOMIC_RELAXED); }

/* The eight corners of the trilinear cell of p at level L (the same cell as trilinear()). */
static void fp_corners(const or_geom* g, fp_io* fp, int L, const double p[3]) {
    int64_t c[3][2];
    for (int a = 0; a < 3; ++a) {
        double u = ldexp(p[a], -L) - 0.5;
        int64_t i = (int64_t)floor(u), hi = g->ldim[L][a] - 1;
        c[a][0] = i < 0 ? 0 : (i > hi ? hi : i);
        c[a][1] = i + 1 < 0 ? 0 : (i + 1 > hi ? hi : i + 1);
    }
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx)
                bit_set(fp->vox[L], (c[2][dz] * g->ldim[L][1] + c[1][dy]) * g->ldim[L][0] + c[0][dx]);
}

/* Admissible results of one march, for or_render_check: with target != NULL, *best receives the
 * smallest max-abs RGBA difference between target and a state the ray may correctly end in. */
typedef struct {
    const float* target;
    double best;
} adm_t;

static void adm_offer(adm_t* ad, const double st[4]) {
    if (!ad || !ad->target) return;
    double e = 0.0;
    for (int q = 0; q < 4; ++q) {
        double d = fabs(st[q] - (double)ad->target[q]);
        if (d > e) e = d;
    }
    if (e < ad->best) ad->best = e;
}

/* One ray.  mode 0: emission-absorption with ERT candidates; mode 1: MIP.  geometry: OR_GEOM_FP64
 * (ctl != NULL decides the knife edges met, see ray_setup64) or OR_GEOM_FP32 (the mirrored
 * single-precision decisions; required with a brick cache).  rec != NULL records the
 * natural-decision forward for the adjoint; ad != NULL collects the admissible end states. */
static void march(or_volume* v, const or_camera* cam, const cam_derived* cd, const float* tf, const float* scale,
                  const float* xf, int mode, int geometry, int px, int py, or_pixel* out, recbuf* rec,
                  const cache_io* cio, edge_ctl* ctl, adm_t* ad, fp_io* fp) {
    const or_geom* g = or_volume_geom(v);
    int C = g->C;
    const int fp64 = geometry == OR_GEOM_FP64;
    memset(out, 0, sizeof(*out));
    out->n_cand = 1;
    float dirf[3], t0f = 0.0f, t1f = 0.0f;
    double dir[3], t0 = 0.0, t1 = 0.0, dt0 = 0.0;
    int hit = fp64 ? ray_setup64(g, cam, cd, px, py, dir, &t0, &t1, &dt0)
                   : ray_setup(g, cam, cd, px, py, dirf, &t0f, &t1f);
    if (!hit) {
        const double zero[4] = {0, 0, 0, 0};
        adm_offer(ad, zero);
        return;
    }
    const float dt = cam->step_voxels;
    const double ert = (double)cam->ert_alpha;
    double Cacc[3] = {0, 0, 0}, A = 0.0;
    double mip[OR_MAXC];
    for (int c = 0; c < C; ++c) mip[c] = -1.0;
    int have_nat = 0, have_early = 0;
    double st_nat[4] = {0}, st_early[4] = {0}, st_prev[4] = {0}, st_late[4] = {0};
    int have_prev = 0, have_late = 0;
    int64_t nsamp = 0;
    for (int64_t k = 0;; ++k) {
        double p[3], dp[3] = {0, 0, 0};
        float pf[3];
        double ell;
        int Lstar = 0, lev;
        or_node nd;
        int64_t path[OR_MAXL][3];
        outcome_t oc;
        if (fp64) {
            double tk = t0 + (double)k * (double)dt;
            if (!(tk < t1) || k >= ((int64_t)1 << 24)) break; /* at most 2^24 samples per ray */
            ell = fmin((double)dt, t1 - tk);
            double dtk = OR_EDGE_SAFETY * (dt0 + 2.0 * U32 * tk);
            for (int a = 0; a < 3; ++a) {
                p[a] = (double)cam->eye[a] + tk * dir[a];
                dp[a] = OR_EDGE_SAFETY * (dtk * fabs(dir[a]) + tk * OR_DIR_ULPS * U32 +
                                          2.0 * U32 * (fabs((double)cam->eye[a]) + tk * fabs(dir[a])) +
                                          U32 * fabs(p[a]));
            }
            Lstar = lod64(v, cd, tk, dtk, p, dp, ctl);
            const int64_t root[3] = {0, 0, 0};
            lev = descend64(v, p, dp, Lstar, g->N, root, ctl, &oc);
            nd.has_brick = oc.brick;
            for (int c = 0; c < C; ++c) nd.avg[c] = oc.avg[c];
        } else {
            float tk = t0f + (float)k * dt;
            if (!(tk < t1f) || k >= ((int64_t)1 << 24)) break;
            ell = (double)fminf(dt, t1f - tk);
            for (int a = 0; a < 3; ++a) {
                pf[a] = cam->eye[a] + tk * dirf[a];
                p[a] = (double)pf[a];
            }
            for (int L = 1; L <= g->N; ++L)
                if (tk >= cd->tl[L]) Lstar = L;
            lev = descend_path(v, pf, Lstar, &nd, path);
        }
        /* Full-frame ray casting with a partial brick cache (Sec. "Full-Frame Ray-Casting"): a
         * missing brick is requested; the brick of the parent or grandparent on the descent path,
         * if present, stands in (nearest first), else the node's AVG; those missing are requested
         * as well. */
        int samp_lev = nd.has_brick ? lev : -1;
        if (!fp64 && cio && cio->res && nd.has_brick) {
            const or_geom* gg = or_volume_geom(v);
            int64_t nid = or_node_index(gg, lev, path[lev][0], path[lev][1], path[lev][2]);
            if (cio->res[nid]) {
                cio->used[nid] = 1;
            } else {
                cio->req[nid] = 1;
                samp_lev = -1;
                for (int up = 1; up <= 2 && lev + up <= gg->N; ++up) {
                    int L2 = lev + up;
                    or_node n2;
                    or_node_info(v, L2, path[L2][0], path[L2][1], path[L2][2], &n2);
                    if (!n2.has_brick) continue;
                    int64_t nid2 = or_node_index(gg, L2, path[L2][0], path[L2][1], path[L2][2]);
                    if (cio->res[nid2]) {
                        if (samp_lev < 0) {
                            samp_lev = L2;
                            cio->used[nid2] = 1;
                        }
                    } else {
                        cio->req[nid2] = 1;
                    }
                }
            }
        }
        or_node ndc[OR_MAXC];
        int levc[OR_MAXC];
        double pc[OR_MAXC][3];
        if (xf) /* every channel descends from its own transformed point */
            for (int c = 0; c < C; ++c) {
                const float* m = xf + 12 * c;
                if (fp64) {
                    double dq[3];
                    for (int i = 0; i < 3; ++i) {
                        pc[c][i] = m[4 * i] * p[0] + m[4 * i + 1] * p[1] + m[4 * i + 2] * p[2] + (double)m[4 * i + 3];
                        dq[i] = fabs((double)m[4 * i]) * dp[0] + fabs((double)m[4 * i + 1]) * dp[1] +
                                fabs((double)m[4 * i + 2]) * dp[2] +
                                OR_EDGE_SAFETY * 4.0 * U32 *
                                    (fabs(m[4 * i] * p[0]) + fabs(m[4 * i + 1] * p[1]) + fabs(m[4 * i + 2] * p[2]) +
                                     fabs((double)m[4 * i + 3]));
                    }
                    const int64_t root[3] = {0, 0, 0};
                    outcome_t occ;
                    levc[c] = descend64(v, pc[c], dq, Lstar, g->N, root, ctl, &occ);
                    ndc[c].has_brick = occ.brick;
                    for (int cc = 0; cc < C; ++cc) ndc[c].avg[cc] = occ.avg[cc];
                } else {
                    float qf[3];
                    channel_point(m, pf, qf);
                    for (int i = 0; i < 3; ++i) pc[c][i] = (double)qf[i];
                    levc[c] = descend(v, qf, Lstar, &ndc[c]);
                }
            }
        if (!have_nat || mode == 1) ++nsamp;
        if (fp && !fp64 && !xf && !have_nat) { /* the descent path and the cell of this sample */
            for (int L = lev; L <= g->N; ++L) bit_set(fp->nodes, or_node_index(g, L, path[L][0], path[L][1], path[L][2]));
            if (samp_lev >= 0) fp_corners(g, fp, samp_lev, p);
        }
        for (int c = 0; c < C; ++c) {
            double I;
            if (xf)
                I = ndc[c].has_brick ? trilinear(v, levc[c], pc[c], c) : (double)ndc[c].avg[c];
            else
                I = samp_lev >= 0 ? trilinear(v, samp_lev, p, c) : (double)nd.avg[c];
            if (mode == 1) {
                if (I > mip[c]) mip[c] = I;
                continue;
            }
            double lam, xr, rgba[4];
            int i = tf_index((double)scale[c], I, &lam, &xr);
            or_tf_eval(tf + (size_t)c * 1024, (double)scale[c], I, rgba);
            double alpha = rgba[3];
            int acl = 0;
            if (alpha > ALPHA_MAX) {
                alpha = ALPHA_MAX;
                acl = 1;
            }
            if (alpha < 0.0) {
                alpha = 0.0;
                acl = 1;
            }
            double aa = 1.0 - pow(1.0 - alpha, ell);
            if (rec && !have_nat) {
                rec_t r = {I, lam, alpha, aa, ell, A, i, (xr > 0.0 && xr < 1.0), acl, c};
                rec_push(rec, &r);
            }
            for (int q = 0; q < 3; ++q) Cacc[q] += (1.0 - A) * aa * rgba[q];
            A += (1.0 - A) * aa;
        }
        if (mode == 1) continue;
        double st[4] = {Cacc[0], Cacc[1], Cacc[2], A};
        if (A >= ert - OR_ERT_BAND) adm_offer(ad, st); /* every state in the band is a correct stop */
        if (!have_early && A >= ert - OR_ERT_BAND) {
            have_early = 1;
            memcpy(st_early, st, sizeof st);
        }
        if (!have_nat && A >= ert) {
            have_nat = 1;
            memcpy(st_nat, st, sizeof st);
            out->samples = nsamp;
        }
        if (A >= ert + OR_ERT_BAND) {
            have_late = 1;
            memcpy(st_late, st, sizeof st);
            break;
        }
        if (have_early) {
            have_prev = 1;
            memcpy(st_prev, st, sizeof st);
        }
    }
    if (mode == 1) {
        out->samples = nsamp;
        if (nsamp == 0) {
            const double zero[4] = {0, 0, 0, 0};
            adm_offer(ad, zero);
            return;
        }
        double Cm[3] = {0, 0, 0}, Am = 0.0;
        for (int c = 0; c < C; ++c) {
            double rgba[4];
            or_tf_eval(tf + (size_t)c * 1024, (double)scale[c], mip[c], rgba);
            double alpha = rgba[3] > ALPHA_MAX ? ALPHA_MAX : rgba[3];
            for (int q = 0; q < 3; ++q) Cm[q] += (1.0 - Am) * alpha * rgba[q];
            Am += (1.0 - Am) * alpha;
        }
        out->rgba[0][0] = Cm[0];
        out->rgba[0][1] = Cm[1];
        out->rgba[0][2] = Cm[2];
        out->rgba[0][3] = Am;
        adm_offer(ad, out->rgba[0]);
        return;
    }
    double fin[4] = {Cacc[0], Cacc[1], Cacc[2], A};
    if (!have_late) adm_offer(ad, fin); /* the ray ran to its end */
    if (!have_nat) {
        out->samples = nsamp;
        memcpy(out->rgba[0], fin, sizeof fin);
    } else {
        memcpy(out->rgba[0], st_nat, sizeof st_nat);
    }
    /* admissible alternatives: the stopping states an FP32 accumulation may reach */
    int n = 1;
    double* cands[3] = {have_early ? st_early : NULL, have_prev ? st_prev : NULL,
                        have_late ? st_late : (have_early ? fin : NULL)};
    for (int q = 0; q < 3; ++q) {
        if (!cands[q]) continue;
        int dup = 0;
        for (int m = 0; m < n; ++m)
            if (memcmp(out->rgba[m], cands[q], sizeof(double) * 4) == 0) dup = 1;
        if (!dup && n < OR_MAXCAND) memcpy(out->rgba[n++], cands[q], sizeof(double) * 4);
    }
    out->n_cand = n;
}

typedef struct {
    or_volume* v;
    const or_camera* cam;
    cam_derived cd;
    const float* tf;
    const float* scale;
    const float* xf; /* NULL or [C][3][4] per-channel transforms */
    cache_io cio;
    int mode, geometry;
    const int32_t* px;
    const int32_t* py;
    or_pixel* out;
    fp_io* fp;           /* or_render_footprint: bitmaps to mark, else NULL */
    const float* target; /* or_render_check: the pixels to compare [n][4] */
    or_check* chk;
    double stop_err; /* or_render_check: stop enumerating once a variant is this close */
} render_job;

static void render_range(void* p, int64_t b, int64_t e) {
    render_job* j = (render_job*)p;
    for (int64_t i = b; i < e; ++i)
        march(j->v, j->cam, &j->cd, j->tf, j->scale, j->xf, j->mode, j->geometry, j->px[i], j->py[i], &j->out[i],
              NULL, &j->cio, NULL, NULL, j->fp);
}

static int cam_valid(const or_camera* cam) {
    if (!cam || cam->width <= 0 || cam->height <= 0 || !(cam->step_voxels > 0.0f) || !(cam->lod_error_px > 0.0f) ||
        cam->n_clip < 0 || cam->n_clip > 3 || !(cam->fov_y_deg > 0.0f && cam->fov_y_deg < 180.0f))
        return 0;
    return 1;
}

static void job_init(render_job* j, or_volume* v, const or_camera* cam, const float* tf, const float* scale,
                     const float* xf, int mode, int geometry, const int32_t* px, const int32_t* py) {
    memset(j, 0, sizeof *j);
    j->v = v;
    j->cam = cam;
    cam_setup(or_volume_geom(v), cam, &j->cd);
    j->tf = tf;
    j->scale = scale;
    j->xf = xf;
    j->mode = mode;
    j->geometry = geometry;
    j->px = px;
    j->py = py;
}

int or_render_geo(or_volume* v, const or_camera* cam, const float* tf, const float* scale, const float* xf, int mode,
                  int geometry, int64_t n, const int32_t* px, const int32_t* py, or_pixel* out, int threads) {
    if (!v || !cam_valid(cam) || !tf || !scale || !px || !py || !out || (mode != 0 && mode != 1) ||
        (geometry != OR_GEOM_FP32 && geometry != OR_GEOM_FP64))
        return -1;
    render_job j;
    job_init(&j, v, cam, tf, scale, xf, mode, geometry, px, py);
    j.out = out;
    or_parallel_for(n, 16, threads, render_range, &j);
    return 0;
}

int or_render_xf(or_volume* v, const or_camera* cam, const float* tf, const float* scale, const float* xf, int mode,
                 int64_t n, const int32_t* px, const int32_t* py, or_pixel* out, int threads) {
    return or_render_geo(v, cam, tf, scale, xf, mode, OR_GEOM_FP64, n, px, py, out, threads);
}

int or_render(or_volume* v, const or_camera* cam, const float* tf, const float* scale, int mode, int64_t n,
              const int32_t* px, const int32_t* py, or_pixel* out, int threads) {
    return or_render_xf(v, cam, tf, scale, NULL, mode, n, px, py, out, threads);
}

static int64_t popcount_bytes(const uint8_t* b, int64_t n) {
    int64_t s = 0;
    for (int64_t i = 0; i < n; ++i) s += __builtin_popcount(b[i]);
    return s;
}

int or_render_footprint(or_volume* v, const or_camera* cam, const float* tf, const float* scale, int64_t* voxels,
                        int64_t* nodes, int threads) {
    if (!v || !cam_valid(cam) || !tf || !scale || !voxels || !nodes) return -1;
    const or_geom* g = or_volume_geom(v);
    const int64_t n = (int64_t)cam->width * cam->height;
    int32_t* px = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int32_t* py = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    or_pixel* out = (or_pixel*)malloc(sizeof(or_pixel) * (size_t)n);
    fp_io fp;
    memset(&fp, 0, sizeof fp);
    int ok = px && py && out;
    for (int L = 0; L <= g->N && ok; ++L) {
        fp.vox[L] = (uint8_t*)calloc((size_t)((g->ldim[L][0] * g->ldim[L][1] * g->ldim[L][2] + 7) / 8), 1);
        ok = fp.vox[L] != NULL;
    }
    if (ok) ok = (fp.nodes = (uint8_t*)calloc((size_t)((or_node_count(g) + 7) / 8), 1)) != NULL;
    if (ok) {
        for (int64_t i = 0; i < n; ++i) {
            px[i] = (int32_t)(i % cam->width);
            py[i] = (int32_t)(i / cam->width);
        }
        render_job j;
        job_init(&j, v, cam, tf, scale, NULL, 0, OR_GEOM_FP32, px, py);
        j.out = out;
        j.fp = &fp;
        or_parallel_for(n, 16, threads, render_range, &j);
        for (int L = 0; L <= g->N; ++L)
            voxels[L] = popcount_bytes(fp.vox[L], (g->ldim[L][0] * g->ldim[L][1] * g->ldim[L][2] + 7) / 8);
        *nodes = popcount_bytes(fp.nodes, (or_node_count(g) + 7) / 8);
    }
    for (int L = 0; L <= g->N; ++L) free(fp.vox[L]);
    free(fp.nodes);
    free(px);
    free(py);
    free(out);
    return ok ? 0 : -2;
}

/* Every variant of the ray's knife-edge decisions, depth first: the march with the branches in
 * script[0..len) forced and the natural branch beyond, then, for each later flagged decision j
 * (up to OR_MAXFLAG), the march that takes the other branch there and the natural one between. */
static void explore(render_job* j, int64_t i, const unsigned char* script, int len, or_check* out) {
    edge_ctl e = {script, len, 0};
    adm_t ad = {j->target + 4 * i, INFINITY};
    or_pixel pix;
    march(j->v, j->cam, &j->cd, j->tf, j->scale, j->xf, j->mode, j->geometry, j->px[i], j->py[i], &pix, NULL, NULL,
          j->geometry == OR_GEOM_FP64 ? &e : NULL, &ad, NULL);
    out->variants++;
    if (ad.best < out->err) out->err = ad.best;
    if (len == 0) {
        memcpy(out->rgba, pix.rgba[0], sizeof out->rgba);
        out->samples = pix.samples;
        out->flagged = e.nflag;
    }
    if (e.nflag > OR_MAXFLAG) out->unresolved = 1;
    int lim = e.nflag < OR_MAXFLAG ? e.nflag : OR_MAXFLAG;
    for (int k = len; k < lim && out->err > j->stop_err; ++k) {
        unsigned char s2[OR_MAXFLAG] = {0};
        if (len > 0) memcpy(s2, script, (size_t)len);
        s2[k] = 1;
        explore(j, i, s2, k + 1, out);
    }
}

static void check_range(void* p, int64_t b, int64_t e) {
    render_job* j = (render_job*)p;
    for (int64_t i = b; i < e; ++i) {
        or_check* o = &j->chk[i];
        memset(o, 0, sizeof *o);
        o->err = INFINITY;
        explore(j, i, NULL, 0, o);
    }
}

int or_render_check(or_volume* v, const or_camera* cam, const float* tf, const float* scale, const float* xf, int mode,
                    int geometry, int64_t n, const int32_t* px, const int32_t* py, const float* rgba, double stop_err,
                    or_check* out, int threads) {
    if (!v || !cam_valid(cam) || !tf || !scale || !px || !py || !rgba || !out || (mode != 0 && mode != 1) ||
        (geometry != OR_GEOM_FP32 && geometry != OR_GEOM_FP64))
        return -1;
    render_job j;
    job_init(&j, v, cam, tf, scale, xf, mode, geometry, px, py);
    j.target = rgba;
    j.chk = out;
    j.stop_err = stop_err;
    or_parallel_for(n, 16, threads, check_range, &j);
    return 0;
}

int or_render_cache(or_volume* v, const or_camera* cam, const float* tf, const float* scale, int mode, int64_t n,
                    const int32_t* px, const int32_t* py, const uint8_t* resident, uint8_t* used, uint8_t* requested,
                    or_pixel* out, int threads) {
    if (!v || !cam_valid(cam) || !tf || !scale || !px || !py || !out || !resident || !used || !requested ||
        (mode != 0 && mode != 1))
        return -1;
    render_job j;
    /* single-precision (mirrored) geometry: the used/requested flags are compared bit for bit */
    job_init(&j, v, cam, tf, scale, NULL, mode, OR_GEOM_FP32, px, py);
    j.cio.res = resident;
    j.cio.used = used;
    j.cio.req = requested;
    j.out = out;
    or_parallel_for(n, 16, threads, render_range, &j);
    return 0;
}

/* ---- adjoint ---- */
typedef struct {
    render_job rj;
    const double* dl;
    double* dtf;    /* [threads][C*256*4] */
    double* dscale; /* [threads][C] */
    int64_t next, n;
    int nthreads;
    uint8_t* ert_edge; /* optional [n]: some sample state lies within ert_margin of the threshold */
    double ert_margin;
} grad_job;

/* Whether the opacity after some sample of the recorded (natural) march -- up to and including
 * the stopping sample -- lies within margin of the termination threshold: there a single-precision
 * accumulation may stop one sample earlier or later (A16 reading). */
static int ert_knife_edge(const recbuf* rb, double ert, double margin) {
    for (int64_t n = 1; n < rb->n; ++n)
        if (rb->r[n].c == 0 && fabs(rb->r[n].A_before - ert) < margin) return 1;
    if (rb->n > 0) {
        const rec_t* r = &rb->r[rb->n - 1];
        double A = r->A_before + (1.0 - r->A_before) * r->a;
        if (fabs(A - ert) < margin) return 1;
    }
    return 0;
}

typedef struct {
    grad_job* g;
    int tid;
} grad_worker_arg;

/* Reverse sweep over the recorded (sample, channel) updates
 *   C' = C + (1-A) a rgb,  A' = A + (1-A) a,
 * with a = 1 - (1 - alpha)^l and (rgb, alpha) = (1-lam) T[i] + lam T[i+1],
 * lam = 255 x - i, x = s I / 65535 (clamped to [0,1]). */
static void ray_grad(const or_geom* g, const float* tf, const recbuf* rb, const double* dl, double* dtf, double* dscale) {
    double gC[3] = {dl[0], dl[1], dl[2]}, gA = dl[3];
    (void)g;
    for (int64_t n = rb->n - 1; n >= 0; --n) {
        const rec_t* r = &rb->r[n];
        const float* T0 = tf + ((size_t)r->c * 256 + (size_t)r->i) * 4;
        const float* T1 = T0 + 4;
        double rgba[4];
        for (int q = 0; q < 4; ++q) rgba[q] = (1.0 - r->lam) * (double)T0[q] + r->lam * (double)T1[q];
        double A = r->A_before, a = r->a;
        double gCrgb = gC[0] * rgba[0] + gC[1] * rgba[1] + gC[2] * rgba[2];
        double ga = (1.0 - A) * (gA + gCrgb);
        double gv[4];
        for (int q = 0; q < 3; ++q) gv[q] = gC[q] * (1.0 - A) * a;
        double dadal = r->aclamped ? 0.0 : r->ell * pow(1.0 - r->alpha, r->ell - 1.0);
        gv[3] = ga * dadal;
        double* D0 = dtf + ((size_t)r->c * 256 + (size_t)r->i) * 4;
        double glam = 0.0;
        for (int q = 0; q < 4; ++q) {
            D0[q] += (1.0 - r->lam) * gv[q];
            D0[q + 4] += r->lam * gv[q];
            glam += gv[q] * ((double)T1[q] - (double)T0[q]);
        }
        if (r->inside) dscale[r->c] += glam * 255.0 * r->I / 65535.0;
        gA = gA * (1.0 - a) - a * gCrgb;
    }
}

static void* grad_worker(void* p) {
    grad_worker_arg* wa = (grad_worker_arg*)p;
    grad_job* j = wa->g;
    const or_geom* g = or_volume_geom(j->rj.v);
    double* dtf = j->dtf + (size_t)wa->tid * (size_t)g->C * 1024;
    double* dsc = j->dscale + (size_t)wa->tid * (size_t)g->C;
    recbuf rb = {NULL, 0, 0};
    for (;;) {
        int64_t i = __atomic_fetch_add(&j->next, 1, __ATOMIC_RELAXED);
        if (i >= j->n) break;
        rb.n = 0;
        or_pixel px;
        march(j->rj.v, j->rj.cam, &j->rj.cd, j->rj.tf, j->rj.scale, j->rj.xf, 0, OR_GEOM_FP32, j->rj.px[i],
              j->rj.py[i], &px, &rb, NULL, NULL, NULL, NULL);
        ray_grad(g, j->rj.tf, &rb, j->dl + 4 * i, dtf, dsc);
        if (j->ert_edge) j->ert_edge[i] = (uint8_t)ert_knife_edge(&rb, (double)j->rj.cam->ert_alpha, j->ert_margin);
    }
    free(rb.r);
    return NULL;
}

int or_render_grad_edges(or_volume* v, const or_camera* cam, const float* tf, const float* scale, const float* xf,
                         int64_t n, const int32_t* px, const int32_t* py, const double* dl, double* dtf,
                         double* dscale, uint8_t* ert_edge, double ert_margin, int threads) {
    if (!v || !cam_valid(cam) || !tf || !scale || !px || !py || !dl || !dtf || !dscale) return -1;
    const or_geom* g = or_volume_geom(v);
    int C = g->C;
    threads = or_threads(threads);
    grad_job j;
    memset(&j, 0, sizeof j);
    j.rj.v = v;
    j.rj.cam = cam;
    cam_setup(g, cam, &j.rj.cd);
    j.rj.tf = tf;
    j.rj.scale = scale;
    j.rj.xf = xf;
    j.rj.px = px;
    j.rj.py = py;
    j.n = n;
    j.dl = dl;
    j.nthreads = threads;
    j.ert_edge = ert_edge;
    j.ert_margin = ert_margin;
    j.dtf = (double*)calloc((size_t)threads * (size_t)C * 1024, sizeof(double));
    j.dscale = (double*)calloc((size_t)threads * (size_t)C, sizeof(double));
    pthread_t th[256];
    grad_worker_arg wa[256];
    for (int t = 0; t < threads; ++t) {
        wa[t].g = &j;
        wa[t].tid = t;
        pthread_create(&th[t], NULL, grad_worker, &wa[t]);
    }
    for (int t = 0; t < threads; ++t) pthread_join(th[t], NULL);
    memset(dtf, 0, sizeof(double) * (size_t)C * 1024);
    memset(dscale, 0, sizeof(double) * (size_t)C);
    for (int t = 0; t < threads; ++t) {
        for (int q = 0; q < C * 1024; ++q) dtf[q] += j.dtf[(size_t)t * C * 1024 + q];
        for (int c = 0; c < C; ++c) dscale[c] += j.dscale[(size_t)t * C + c];
    }
    free(j.dtf);
    free(j.dscale);
    return 0;
}

int or_render_grad_xf(or_volume* v, const or_camera* cam, const float* tf, const float* scale, const float* xf,
                      int64_t n, const int32_t* px, const int32_t* py, const double* dl, double* dtf, double* dscale,
                      int threads) {
    return or_render_grad_edges(v, cam, tf, scale, xf, n, px, py, dl, dtf, dscale, NULL, 0.0, threads);
}

int or_render_grad(or_volume* v, const or_camera* cam, const float* tf, const float* scale, int64_t n,
                   const int32_t* px, const int32_t* py, const double* dl, double* dtf, double* dscale, int threads) {
    return or_render_grad_xf(v, cam, tf, scale, NULL, n, px, py, dl, dtf, dscale, threads);
}
