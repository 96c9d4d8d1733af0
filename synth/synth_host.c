/*
 * synth_host.c -- host side of the seeded input generator (see synth_common.h).
 *
 * Builds a generator specification (emitter list + a CSR spatial index over
 * cubic cells) from (kind, dims, channels, count, seed) and evaluates voxels
 * on the host, multithreaded over rows.  Build with -ffp-contract=off: the
 * per-voxel arithmetic must be plain IEEE single operations so that it
 * matches the device generator bit for bit.
 */
#include "synth_common.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

typedef struct {
    sy_view v;
    sy_nucleus* nuclei;
    int64_t* cell_start;
    int32_t* cell_idx;
    int64_t n_nuclei;
    int64_t n_idx;
} sy_spec;

static double u01(uint64_t* st) {
    *st += SY_GOLDEN;
    return (double)(sy_mix64(*st) >> 11) * (1.0 / 9007199254740992.0);
}

static double uab(uint64_t* st, double a, double b) { return a + (b - a) * u01(st); }

/* Per-channel width factors of the SPIM-like point spread (anisotropic blur). */
static const double SPIM_B[SY_MAXC] = {1.0, 1.1, 1.2, 1.3};
static const double SPIM_A[SY_MAXC] = {1.5, 2.0, 2.5, 3.0};

static void build_index(sy_spec* s) {
    sy_view* v = &s->v;
    int cs = v->cell;
    v->ncx = (int)((v->X + cs - 1) / cs);
    v->ncy = (int)((v->Y + cs - 1) / cs);
    v->ncz = (int)((v->Z + cs - 1) / cs);
    int64_t ncell = (int64_t)v->ncx * v->ncy * v->ncz;
    int64_t* count = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
    int64_t(*box)[6] = (int64_t(*)[6])malloc(sizeof(int64_t[6]) * (size_t)(s->n_nuclei > 0 ? s->n_nuclei : 1));
    for (int64_t j = 0; j < s->n_nuclei; ++j) {
        const sy_nucleus* n = &s->nuclei[j];
        double rxy = 0.0, rz = 0.0;
        for (int c = 0; c < v->C; ++c) {
            if (n->peak[c] > 0.0f) {
                double a = sqrt((double)SY_QCUT / n->ia[c]), b = sqrt((double)SY_QCUT / n->ib[c]);
                if (a > rxy) rxy = a;
                if (b > rz) rz = b;
            }
        }
        double cen[3] = {n->cx, n->cy, n->cz}, r[3] = {rxy, rxy, rz};
        int64_t dim[3] = {v->X, v->Y, v->Z};
        int nc[3] = {v->ncx, v->ncy, v->ncz};
        for (int a = 0; a < 3; ++a) {
            int64_t lo = (int64_t)floor(cen[a] - r[a] - 0.5) - 1, hi = (int64_t)ceil(cen[a] + r[a] - 0.5) + 1;
            if (lo < 0) lo = 0;
            if (hi > dim[a] - 1) hi = dim[a] - 1;
            box[j][2 * a] = lo / cs;
            box[j][2 * a + 1] = (hi < lo) ? -1 : hi / cs;
            if (box[j][2 * a + 1] >= nc[a]) box[j][2 * a + 1] = nc[a] - 1;
        }
        for (int64_t z = box[j][4]; z <= box[j][5]; ++z)
            for (int64_t y = box[j][2]; y <= box[j][3]; ++y)
                for (int64_t x = box[j][0]; x <= box[j][1]; ++x) count[(z * v->ncy + y) * v->ncx + x + 1]++;
    }
    for (int64_t i = 0; i < ncell; ++i) count[i + 1] += count[i];
    s->n_idx = count[ncell];
    s->cell_idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(s->n_idx > 0 ? s->n_idx : 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ncell + 1));
    memcpy(fill, count, sizeof(int64_t) * (size_t)(ncell + 1));
    for (int64_t j = 0; j < s->n_nuclei; ++j) /* ascending ids within each cell */
        for (int64_t z = box[j][4]; z <= box[j][5]; ++z)
            for (int64_t y = box[j][2]; y <= box[j][3]; ++y)
                for (int64_t x = box[j][0]; x <= box[j][1]; ++x)
                    s->cell_idx[fill[(z * v->ncy + y) * v->ncx + x]++] = (int32_t)j;
    free(fill);
    free(box);
    s->cell_start = count;
    v->cell_start = s->cell_start;
    v->cell_idx = s->cell_idx;
    v->nuclei = s->nuclei;
}

/*
 * kind SY_KIND_BLOBS: per channel `count` isotropic Gaussian blobs, centres
 *   uniform in [dim/8, 7 dim/8) per axis, sigma ~ U(2,6), peak ~ U(1000,60000).
 * kind SY_KIND_SPIM: `count` nuclei with centres uniform in the tissue
 *   ellipsoid (semi-axes 0.45 dims, centred), radius r ~ U(3,8); present in
 *   channel c with probability 0.7, peak ~ U(2000,30000),
 *   sigma_xy = r/2 * b_c, sigma_z = sigma_xy * a_c.
 */
void* sy_spec_create(int kind, int64_t X, int64_t Y, int64_t Z, int C, int64_t count, uint64_t seed) {
    if (C < 1 || C > SY_MAXC || X <= 0 || Y <= 0 || Z <= 0 || count < 0) return NULL;
    if (X >= (1 << 21) || Y >= (1 << 21) || Z >= (1 << 21)) return NULL;
    sy_spec* s = (sy_spec*)calloc(1, sizeof(sy_spec));
    s->v.kind = kind;
    s->v.C = C;
    s->v.X = X;
    s->v.Y = Y;
    s->v.Z = Z;
    s->v.seed = seed;
    s->v.cell = 32;
    double dims[3] = {(double)X, (double)Y, (double)Z};
    for (int a = 0; a < 3; ++a) {
        s->v.mask_c[a] = (float)(0.5 * dims[a]);
        s->v.mask_ia[a] = (float)(1.0 / (0.45 * dims[a]));
    }
    uint64_t st = sy_mix64(seed ^ 0x6a09e667f3bcc909ULL) ^ ((uint64_t)kind << 32);
    if (kind == SY_KIND_BLOBS) {
        s->n_nuclei = count * C;
        s->nuclei = (sy_nucleus*)calloc((size_t)(s->n_nuclei > 0 ? s->n_nuclei : 1), sizeof(sy_nucleus));
        for (int c = 0; c < C; ++c)
            for (int64_t i = 0; i < count; ++i) {
                sy_nucleus* n = &s->nuclei[c * count + i];
                n->cx = (float)uab(&st, dims[0] / 8, dims[0] * 7 / 8);
                n->cy = (float)uab(&st, dims[1] / 8, dims[1] * 7 / 8);
                n->cz = (float)uab(&st, dims[2] / 8, dims[2] * 7 / 8);
                double sigma = uab(&st, 2.0, 6.0);
                n->peak[c] = (float)uab(&st, 1000.0, 60000.0);
                n->ia[c] = n->ib[c] = (float)(1.0 / (2.0 * sigma * sigma));
            }
    } else if (kind == SY_KIND_SPIM) {
        s->n_nuclei = count;
        s->nuclei = (sy_nucleus*)calloc((size_t)(count > 0 ? count : 1), sizeof(sy_nucleus));
        for (int64_t i = 0; i < count; ++i) {
            sy_nucleus* n = &s->nuclei[i];
            double p[3];
            for (;;) { /* rejection sampling inside the ellipsoid */
                double e = 0.0;
                for (int a = 0; a < 3; ++a) {
                    p[a] = uab(&st, 0.05 * dims[a], 0.95 * dims[a]);
                    double t = (p[a] - 0.5 * dims[a]) / (0.45 * dims[a]);
                    e += t * t;
                }
                if (e <= 1.0) break;
            }
            n->cx = (float)p[0];
            n->cy = (float)p[1];
            n->cz = (float)p[2];
            double r = uab(&st, 3.0, 8.0);
            for (int c = 0; c < C; ++c) {
                double present = u01(&st), peak = uab(&st, 2000.0, 30000.0);
                if (present < 0.7) {
                    double sxy = r / 2.0 * SPIM_B[c], sz = sxy * SPIM_A[c];
                    n->peak[c] = (float)peak;
                    n->ia[c] = (float)(1.0 / (2.0 * sxy * sxy));
                    n->ib[c] = (float)(1.0 / (2.0 * sz * sz));
                }
            }
        }
    } else {
        free(s);
        return NULL;
    }
    build_index(s);
    return s;
}

void sy_spec_destroy(void* h) {
    sy_spec* s = (sy_spec*)h;
    if (!s) return;
    free(s->nuclei);
    free(s->cell_start);
    free(s->cell_idx);
    free(s);
}

/* Raw arrays for upload to the device generator. */
void sy_spec_arrays(void* h, const void** nuclei, int64_t* n_nuclei, const int64_t** cell_start, int64_t* n_cells,
                    const int32_t** cell_idx, int64_t* n_idx) {
    sy_spec* s = (sy_spec*)h;
    *nuclei = s->nuclei;
    *n_nuclei = s->n_nuclei;
    *cell_start = s->cell_start;
    *n_cells = (int64_t)s->v.ncx * s->v.ncy * s->v.ncz;
    *cell_idx = s->cell_idx;
    *n_idx = s->n_idx;
}

const sy_view* sy_spec_view(void* h) { return &((sy_spec*)h)->v; }

/* One voxel, all channels: the entry point handed to the oracle's lazy volume. */
void sy_host_voxel(void* h, int64_t x, int64_t y, int64_t z, uint16_t* out) {
    sy_voxel(&((sy_spec*)h)->v, x, y, z, out);
}

/* Arbitrary list of voxels: coords [n][3] (x, y, z) -> out [n][C]. */
void sy_host_voxels(void* h, int64_t n, const int64_t* coords, uint16_t* out) {
    sy_spec* s = (sy_spec*)h;
    for (int64_t i = 0; i < n; ++i) sy_voxel(&s->v, coords[3 * i], coords[3 * i + 1], coords[3 * i + 2], out + i * s->v.C);
}

typedef struct {
    sy_spec* s;
    int64_t x0, x1, y0, y1, z0, z1;
    uint16_t* out;
    int64_t next_row;
    pthread_mutex_t* mu;
} job_t;

static void* worker(void* arg) {
    job_t* j = (job_t*)arg;
    int64_t nx = j->x1 - j->x0, ny = j->y1 - j->y0, nrows = ny * (j->z1 - j->z0);
    int C = j->s->v.C;
    for (;;) {
        pthread_mutex_lock(j->mu);
        int64_t r = j->next_row;
        j->next_row += 4;
        pthread_mutex_unlock(j->mu);
        if (r >= nrows) break;
        int64_t rend = r + 4 < nrows ? r + 4 : nrows;
        for (; r < rend; ++r) {
            int64_t z = j->z0 + r / ny, y = j->y0 + r % ny;
            uint16_t* o = j->out + r * nx * C;
            for (int64_t x = j->x0; x < j->x1; ++x) sy_voxel(&j->s->v, x, y, z, o + (x - j->x0) * C);
        }
    }
    return NULL;
}

/* Box [x0,x1) x [y0,y1) x [z0,z1) -> out[z][y][x][C]; threads <= 0 means all cores. */
int sy_host_generate_box(void* h, int64_t x0, int64_t x1, int64_t y0, int64_t y1, int64_t z0, int64_t z1, uint16_t* out,
                         int threads) {
    sy_spec* s = (sy_spec*)h;
    if (!s || x0 < 0 || y0 < 0 || z0 < 0 || x1 > s->v.X || y1 > s->v.Y || z1 > s->v.Z || x1 < x0 || y1 < y0 || z1 < z0)
        return -1;
    if (threads <= 0) threads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    pthread_mutex_t mu = PTHREAD_MUTEX_INITIALIZER;
    job_t j = {s, x0, x1, y0, y1, z0, z1, out, 0, &mu};
    pthread_t th[256];
    for (int i = 0; i < threads; ++i) pthread_create(&th[i], NULL, worker, &j);
    for (int i = 0; i < threads; ++i) pthread_join(th[i], NULL);
    return 0;
}
