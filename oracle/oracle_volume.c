/*
 * oracle_volume.c -- TEST INFRASTRUCTURE (FP64/integer CPU oracle; see oracle.h).
 *
 * The volume state as a pure function of what has been inserted:
 *   V_0[v]   = the last value inserted at v, or the background value where
 *              nothing was inserted ("Incremental Construction": the root
 *              starts with only the background value; already inserted data
 *              can be overwritten; unknown values are the background).
 *   V_L[j]   = RHU( sum of V_{L-1}[2j + d], d in {0,1}^3, 2j+d inside the
 *              level-(L-1) real extent ; number k of such children ),
 *              RHU(S, k) = floor((2S + k) / (2k))  (round half up).
 *              Levels are built by iterated half-sampling of the previous
 *              level (Sec. "CPU Data Structure"; step 2 of the incremental
 *              construction), and voxels outside the real volume never
 *              enter a mean (Sec. "Handling Volumes of Arbitrary Dimensions").
 *   node (L, i, j, k) covers level-L voxels [iM, (i+1)M) x ... of the
 *              virtual extension M*2^N (Eq. 1) and level-0 voxels
 *              [iM 2^L, (i+1)M 2^L) x ... ; only in-volume voxels count.
 *   brick_homog   <=> for every channel, max - min over the brick's in-volume
 *                     level-L voxels is below tau (Sec. "CPU Data Structure";
 *                     all channels must be homogeneous, Sec. "Handling
 *                     Multi-Channel Data").
 *   subtree_homog <=> the same over the node's in-volume level-0 voxels.
 *   AVG_c         = RHU(mean of the brick's in-volume level-L voxels).
 *   has_children  = L > 0 and touched and not subtree_homog.
 *   has_brick     = touched and not brick_homog.
 * Deleting a homogeneous brick changes only what the render reads, never the
 * stored values (a reading of the paper, which is silent on re-inserting into
 * a deleted brick): the state depends on the current level-0 values only.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#include "oracle.h"
#include "oracle_internal.h"

int or_geom_init(or_geom* g, const int64_t dim[3], int C, int M, uint16_t bg, uint16_t tau) {
    if (!g || !dim || C < 1 || C > OR_MAXC || M < 2 || (M & 1)) return -1;
    for (int a = 0; a < 3; ++a)
        if (dim[a] <= 0 || dim[a] >= ((int64_t)1 << 21)) return -1;
    memset(g, 0, sizeof(*g));
    for (int a = 0; a < 3; ++a) g->dim[a] = dim[a];
    g->C = C;
    g->M = M;
    g->bg = bg;
    g->tau = tau;
    int64_t nbmax = 1;
    for (int a = 0; a < 3; ++a) {
        int64_t nb = (dim[a] + M - 1) / M;
        if (nb > nbmax) nbmax = nb;
    }
    int N = 0;
    while (((int64_t)1 << N) < nbmax) ++N;
    if (N + 1 > OR_MAXL) return -1;
    g->N = N;
    for (int a = 0; a < 3; ++a) g->ldim[0][a] = dim[a];
    for (int L = 1; L <= N; ++L)
        for (int a = 0; a < 3; ++a) g->ldim[L][a] = (g->ldim[L - 1][a] + 1) / 2;
    for (int L = 0; L <= N; ++L)
        for (int a = 0; a < 3; ++a) g->nb[L][a] = (g->ldim[L][a] + M - 1) / M;
    return 0;
}

static inline uint16_t rhu(uint64_t S, uint64_t k) { return (uint16_t)((2 * S + k) / (2 * k)); }

/* ------------------------------------------------------------------------------------------ */
/* parallel for                                                                               */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int64_t n, next, chunk;
    pthread_mutex_t mu;
    void (*fn)(void*, int64_t, int64_t);
    void* arg;
} pf_t;

static void* pf_worker(void* p) {
    pf_t* j = (pf_t*)p;
    for (;;) {
        pthread_mutex_lock(&j->mu);
        int64_t b = j->next;
        j->next += j->chunk;
        pthread_mutex_unlock(&j->mu);
        if (b >= j->n) break;
        int64_t e = b + j->chunk < j->n ? b + j->chunk : j->n;
        j->fn(j->arg, b, e);
    }
    return NULL;
}

int or_threads(int threads) {
    if (threads <= 0) threads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    return threads;
}

void or_parallel_for(int64_t n, int64_t chunk, int threads, void (*fn)(void*, int64_t, int64_t), void* arg) {
    threads = or_threads(threads);
    if (n <= 0) return;
    if (threads == 1 || n <= chunk) {
        fn(arg, 0, n);
        return;
    }
    pf_t j;
    j.n = n;
    j.next = 0;
    j.chunk = chunk;
    j.fn = fn;
    j.arg = arg;
    pthread_mutex_init(&j.mu, NULL);
    pthread_t th[256];
    for (int i = 0; i < threads; ++i) pthread_create(&th[i], NULL, pf_worker, &j);
    for (int i = 0; i < threads; ++i) pthread_join(th[i], NULL);
    pthread_mutex_destroy(&j.mu);
}

/* ------------------------------------------------------------------------------------------ */
/* volume object                                                                              */
/* ------------------------------------------------------------------------------------------ */
#define MEMO_SHARDS 256

typedef struct {
    uint64_t* keys; /* 0 = empty; stored key = packed + 1 */
    uint16_t* vals; /* [cap][OR_MAXC] */
    int64_t cap, used;
    pthread_mutex_t mu;
} memo_shard;

typedef struct {
    uint64_t* keys;
    or_node* vals;
    int64_t cap, used;
    pthread_mutex_t mu;
} node_shard;

struct or_volume {
    or_geom g;
    int lazy;
    /* dense */
    uint16_t* V[OR_MAXL];
    uint8_t* ins;
    or_node* nodes[OR_MAXL];
    int built;
    /* lazy */
    or_gen_fn gen;
    void* user;
    int64_t z_lo, z_hi;
    memo_shard* vmemo[OR_MAXL];
    node_shard* nmemo;
    /* streamed: level 0 fed once in z order and read back through gen; levels >= 1 in V[] */
    int streamed;
    int64_t next_z;     /* first level-0 slice not fed yet */
    uint16_t* carry;    /* an even slice whose odd partner comes with the next feed */
    int have_carry;
    uint64_t* sum0;     /* [level-0 node][C] running sums */
};

const or_geom* or_volume_geom(const or_volume* v) { return &v->g; }

static inline int64_t vidx(const or_geom* g, int L, int64_t x, int64_t y, int64_t z) {
    return (z * g->ldim[L][1] + y) * g->ldim[L][0] + x;
}

static inline int64_t nidx(const or_geom* g, int L, int64_t i, int64_t j, int64_t k) {
    return (k * g->nb[L][1] + j) * g->nb[L][0] + i;
}

or_volume* or_dense_create(const int64_t dim[3], int C, int M, uint16_t bg, uint16_t tau) {
    or_volume* v = (or_volume*)calloc(1, sizeof(or_volume));
    if (!v || or_geom_init(&v->g, dim, C, M, bg, tau) != 0) {
        free(v);
        return NULL;
    }
    const or_geom* g = &v->g;
    for (int L = 0; L <= g->N; ++L) {
        int64_t n = g->ldim[L][0] * g->ldim[L][1] * g->ldim[L][2] * C;
        v->V[L] = (uint16_t*)malloc(sizeof(uint16_t) * (size_t)n);
        if (!v->V[L]) {
            or_volume_destroy(v);
            return NULL;
        }
        for (int64_t i = 0; i < n; ++i) v->V[L][i] = bg;
        int64_t nn = g->nb[L][0] * g->nb[L][1] * g->nb[L][2];
        v->nodes[L] = (or_node*)calloc((size_t)nn, sizeof(or_node));
        if (!v->nodes[L]) {
            or_volume_destroy(v);
            return NULL;
        }
    }
    v->ins = (uint8_t*)calloc((size_t)(dim[0] * dim[1] * dim[2]), 1);
    if (!v->ins) {
        or_volume_destroy(v);
        return NULL;
    }
    return v;
}

int or_dense_insert(or_volume* v, const int64_t o[3], const int64_t e[3], const uint16_t* block) {
    if (!v || v->lazy || v->streamed) return -1;
    const or_geom* g = &v->g;
    for (int a = 0; a < 3; ++a)
        if (o[a] < 0 || e[a] < 0 || o[a] + e[a] > g->dim[a]) return -1;
    int C = g->C;
    for (int64_t z = 0; z < e[2]; ++z)
        for (int64_t y = 0; y < e[1]; ++y)
            for (int64_t x = 0; x < e[0]; ++x) {
                int64_t d = vidx(g, 0, o[0] + x, o[1] + y, o[2] + z);
                const uint16_t* s = block + ((z * e[1] + y) * e[0] + x) * C;
                for (int c = 0; c < C; ++c) v->V[0][d * C + c] = s[c];
                v->ins[d] = 1;
            }
    v->built = 0;
    return 0;
}

/* ---- dense build ---- */
typedef struct {
    or_volume* v;
    int L;
} lvl_arg;

static void build_level_rows(void* p, int64_t b, int64_t e) {
    lvl_arg* a = (lvl_arg*)p;
    const or_geom* g = &a->v->g;
    int L = a->L, C = g->C;
    const uint16_t* P = a->v->V[L - 1];
    uint16_t* Q = a->v->V[L];
    const int64_t* pd = g->ldim[L - 1];
    for (int64_t r = b; r < e; ++r) { /* r = z * Y_L + y */
        int64_t z = r / g->ldim[L][1], y = r % g->ldim[L][1];
        for (int64_t x = 0; x < g->ldim[L][0]; ++x)
            for (int c = 0; c < C; ++c) {
                uint64_t S = 0, k = 0;
                for (int dz = 0; dz < 2; ++dz)
                    for (int dy = 0; dy < 2; ++dy)
                        for (int dx = 0; dx < 2; ++dx) {
                            int64_t cx = 2 * x + dx, cy = 2 * y + dy, cz = 2 * z + dz;
                            if (cx < pd[0] && cy < pd[1] && cz < pd[2]) {
                                S += P[vidx(g, L - 1, cx, cy, cz) * C + c];
                                ++k;
                            }
                        }
                Q[vidx(g, L, x, y, z) * C + c] = rhu(S, k);
            }
    }
}

/* Node record by brute force over the node's regions (dense storage). */
static void node_brute(or_volume* v, int L, int64_t i, int64_t j, int64_t k, or_node* n) {
    const or_geom* g = &v->g;
    int C = g->C, M = g->M;
    memset(n, 0, sizeof(*n));
    int64_t lo[3] = {i * M, j * M, k * M}, hi[3];
    for (int a = 0; a < 3; ++a) hi[a] = lo[a] + M < g->ldim[L][a] ? lo[a] + M : g->ldim[L][a];
    uint64_t sum[OR_MAXC] = {0};
    for (int c = 0; c < C; ++c) {
        n->bmin[c] = n->smin[c] = 0xffff;
        n->bmax[c] = n->smax[c] = 0;
    }
    for (int64_t z = lo[2]; z < hi[2]; ++z)
        for (int64_t y = lo[1]; y < hi[1]; ++y)
            for (int64_t x = lo[0]; x < hi[0]; ++x) {
                for (int c = 0; c < C; ++c) {
                    uint16_t val = or_value(v, L, x, y, z, c);
                    sum[c] += val;
                    if (val < n->bmin[c]) n->bmin[c] = val;
                    if (val > n->bmax[c]) n->bmax[c] = val;
                }
                n->count++;
            }
    int64_t s = (int64_t)M << L, l0[3] = {i * s, j * s, k * s}, h0[3];
    for (int a = 0; a < 3; ++a) h0[a] = l0[a] + s < g->dim[a] ? l0[a] + s : g->dim[a];
    for (int64_t z = l0[2]; z < h0[2]; ++z)
        for (int64_t y = l0[1]; y < h0[1]; ++y)
            for (int64_t x = l0[0]; x < h0[0]; ++x) {
                if (!v->lazy) {
                    if (v->ins[vidx(g, 0, x, y, z)]) n->touched = 1;
                } else if (z >= v->z_lo && z < v->z_hi) {
                    n->touched = 1;
                }
                for (int c = 0; c < C; ++c) {
                    uint16_t val = or_value(v, 0, x, y, z, c);
                    if (val < n->smin[c]) n->smin[c] = val;
                    if (val > n->smax[c]) n->smax[c] = val;
                }
            }
    n->brick_homog = 1;
    n->subtree_homog = 1;
    for (int c = 0; c < C; ++c) {
        if (!((int)n->bmax[c] - (int)n->bmin[c] < (int)g->tau)) n->brick_homog = 0;
        if (!((int)n->smax[c] - (int)n->smin[c] < (int)g->tau)) n->subtree_homog = 0;
        n->avg[c] = n->touched ? rhu(sum[c], (uint64_t)n->count) : g->bg;
    }
    n->has_children = (L > 0) && n->touched && !n->subtree_homog;
    n->has_brick = n->touched && !n->brick_homog;
}

static void build_nodes_range(void* p, int64_t b, int64_t e) {
    lvl_arg* a = (lvl_arg*)p;
    const or_geom* g = &a->v->g;
    int L = a->L;
    for (int64_t r = b; r < e; ++r) {
        int64_t i = r % g->nb[L][0], j = (r / g->nb[L][0]) % g->nb[L][1], k = r / (g->nb[L][0] * g->nb[L][1]);
        node_brute(a->v, L, i, j, k, &a->v->nodes[L][r]);
    }
}

int or_dense_build(or_volume* v, int threads) {
    if (!v || v->lazy || v->streamed) return -1;
    const or_geom* g = &v->g;
    for (int L = 1; L <= g->N; ++L) {
        lvl_arg a = {v, L};
        or_parallel_for(g->ldim[L][1] * g->ldim[L][2], 4, threads, build_level_rows, &a);
    }
    v->built = 1; /* or_value reads the arrays from here on */
    for (int L = 0; L <= g->N; ++L) {
        lvl_arg a = {v, L};
        or_parallel_for(g->nb[L][0] * g->nb[L][1] * g->nb[L][2], 1, threads, build_nodes_range, &a);
    }
    return 0;
}

const uint16_t* or_dense_level(or_volume* v, int L) {
    if (!v || v->lazy || L < 0 || L > v->g.N) return NULL;
    return v->V[L]; /* NULL for level 0 of a streamed volume */
}

/* ---- lazy volume ---- */
or_volume* or_lazy_create(const int64_t dim[3], int C, int M, uint16_t bg, uint16_t tau, or_gen_fn gen, void* user,
                          int64_t z_lo, int64_t z_hi) {
    or_volume* v = (or_volume*)calloc(1, sizeof(or_volume));
    if (!v || !gen || or_geom_init(&v->g, dim, C, M, bg, tau) != 0) {
        free(v);
        return NULL;
    }
    v->lazy = 1;
    v->built = 1;
    v->gen = gen;
    v->user = user;
    v->z_lo = z_lo < 0 ? 0 : z_lo;
    v->z_hi = z_hi > dim[2] ? dim[2] : z_hi;
    for (int L = 0; L <= v->g.N; ++L) {
        v->vmemo[L] = (memo_shard*)calloc(MEMO_SHARDS, sizeof(memo_shard));
        for (int s = 0; s < MEMO_SHARDS; ++s) pthread_mutex_init(&v->vmemo[L][s].mu, NULL);
    }
    v->nmemo = (node_shard*)calloc(MEMO_SHARDS, sizeof(node_shard));
    for (int s = 0; s < MEMO_SHARDS; ++s) pthread_mutex_init(&v->nmemo[s].mu, NULL);
    return v;
}

static inline uint64_t hash64(uint64_t z) {
    z = (z ^ (z >> 33)) * 0xff51afd7ed558ccdULL;
    z = (z ^ (z >> 33)) * 0xc4ceb9fe1a85ec53ULL;
    return z ^ (z >> 33);
}

static int memo_get(memo_shard* s, uint64_t key, uint16_t* out) {
    int found = 0;
    pthread_mutex_lock(&s->mu);
    if (s->cap) {
        uint64_t h = hash64(key) & (uint64_t)(s->cap - 1);
        while (s->keys[h]) {
            if (s->keys[h] == key + 1) {
                memcpy(out, &s->vals[h * OR_MAXC], sizeof(uint16_t) * OR_MAXC);
                found = 1;
                break;
            }
            h = (h + 1) & (uint64_t)(s->cap - 1);
        }
    }
    pthread_mutex_unlock(&s->mu);
    return found;
}

static void memo_put(memo_shard* s, uint64_t key, const uint16_t* val) {
    pthread_mutex_lock(&s->mu);
    if (2 * (s->used + 1) > s->cap) {
        int64_t nc = s->cap ? 2 * s->cap : 1024;
        uint64_t* nk = (uint64_t*)calloc((size_t)nc, sizeof(uint64_t));
        uint16_t* nv = (uint16_t*)malloc(sizeof(uint16_t) * OR_MAXC * (size_t)nc);
        for (int64_t i = 0; i < s->cap; ++i)
            if (s->keys[i]) {
                uint64_t h = hash64(s->keys[i] - 1) & (uint64_t)(nc - 1);
                while (nk[h]) h = (h + 1) & (uint64_t)(nc - 1);
                nk[h] = s->keys[i];
                memcpy(&nv[h * OR_MAXC], &s->vals[i * OR_MAXC], sizeof(uint16_t) * OR_MAXC);
            }
        free(s->keys);
        free(s->vals);
        s->keys = nk;
        s->vals = nv;
        s->cap = nc;
    }
    uint64_t h = hash64(key) & (uint64_t)(s->cap - 1);
    while (s->keys[h] && s->keys[h] != key + 1) h = (h + 1) & (uint64_t)(s->cap - 1);
    if (!s->keys[h]) s->used++;
    s->keys[h] = key + 1;
    memcpy(&s->vals[h * OR_MAXC], val, sizeof(uint16_t) * OR_MAXC);
    pthread_mutex_unlock(&s->mu);
}

static void lazy_voxel(or_volume* v, int L, int64_t x, int64_t y, int64_t z, uint16_t* out) {
    const or_geom* g = &v->g;
    uint64_t key = (uint64_t)x | ((uint64_t)y << 21) | ((uint64_t)z << 42);
    memo_shard* sh = &v->vmemo[L][hash64(key * 31 + (uint64_t)L) % MEMO_SHARDS];
    if (memo_get(sh, key, out)) return;
    uint16_t val[OR_MAXC] = {0};
    if (L == 0) {
        if (z >= v->z_lo && z < v->z_hi)
            v->gen(v->user, x, y, z, val);
        else
            for (int c = 0; c < g->C; ++c) val[c] = g->bg;
    } else {
        uint64_t S[OR_MAXC] = {0}, k = 0;
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    int64_t cx = 2 * x + dx, cy = 2 * y + dy, cz = 2 * z + dz;
                    if (cx < g->ldim[L - 1][0] && cy < g->ldim[L - 1][1] && cz < g->ldim[L - 1][2]) {
                        uint16_t ch[OR_MAXC];
                        lazy_voxel(v, L - 1, cx, cy, cz, ch);
                        for (int c = 0; c < g->C; ++c) S[c] += ch[c];
                        ++k;
                    }
                }
        for (int c = 0; c < g->C; ++c) val[c] = rhu(S[c], k);
    }
    memo_put(sh, key, val);
    memcpy(out, val, sizeof(uint16_t) * OR_MAXC);
}

uint16_t or_value(or_volume* v, int L, int64_t x, int64_t y, int64_t z, int c) {
    const or_geom* g = &v->g;
    if (v->streamed && L == 0) {
        uint16_t val[OR_MAXC] = {0};
        v->gen(v->user, x, y, z, val);
        return val[c];
    }
    if (v->lazy) {
        uint16_t val[OR_MAXC];
        lazy_voxel(v, L, x, y, z, val);
        return val[c];
    }
    return v->V[L][vidx(g, L, x, y, z) * g->C + c];
}

/* Lazy node: when tau == 0 no brick or subtree can be homogeneous (max - min < 0 never
 * holds), so the flags follow from `touched` alone and no scan is needed. */
static void lazy_node(or_volume* v, int L, int64_t i, int64_t j, int64_t k, or_node* n) {
    const or_geom* g = &v->g;
    if (g->tau != 0) {
        uint64_t key = (uint64_t)i | ((uint64_t)j << 20) | ((uint64_t)k << 40) | ((uint64_t)L << 60);
        node_shard* sh = &v->nmemo[hash64(key) % MEMO_SHARDS];
        pthread_mutex_lock(&sh->mu);
        for (int64_t t = 0; t < sh->used; ++t)
            if (sh->keys[t] == key) {
                *n = sh->vals[t];
                pthread_mutex_unlock(&sh->mu);
                return;
            }
        pthread_mutex_unlock(&sh->mu);
        node_brute(v, L, i, j, k, n);
        pthread_mutex_lock(&sh->mu);
        if (sh->used == sh->cap) {
            sh->cap = sh->cap ? 2 * sh->cap : 64;
            sh->keys = (uint64_t*)realloc(sh->keys, sizeof(uint64_t) * (size_t)sh->cap);
            sh->vals = (or_node*)realloc(sh->vals, sizeof(or_node) * (size_t)sh->cap);
        }
        sh->keys[sh->used] = key;
        sh->vals[sh->used] = *n;
        sh->used++;
        pthread_mutex_unlock(&sh->mu);
        return;
    }
    memset(n, 0, sizeof(*n));
    int64_t s = (int64_t)g->M << L;
    int64_t zlo = k * s, zhi = zlo + s < g->dim[2] ? zlo + s : g->dim[2];
    n->touched = (zlo < v->z_hi && v->z_lo < zhi);
    n->has_children = (L > 0) && n->touched;
    n->has_brick = n->touched;
    for (int c = 0; c < g->C; ++c) n->avg[c] = g->bg; /* read only when there is no brick */
}

/* ---- streamed volume ----
 * The same state as a dense volume into which the whole level 0 was inserted, for volumes whose
 * level 0 does not fit in host memory: level 0 is fed once, slab by slab in z order, and is not
 * stored (or_value reads it back through the generator that produced it); level 1 is half-sampled
 * from each pair of level-0 slices as the pair arrives; levels 2..N by build_level_rows.  Node
 * records: level-0 brick min/max/sum accumulate while feeding; a level-L brick (L >= 1) is scanned
 * in V[L]; the level-0 region of a node is the union of its children's level-0 regions, so its
 * subtree min/max is the min/max over the children's. */
or_volume* or_stream_create(const int64_t dim[3], int C, int M, uint16_t bg, uint16_t tau, or_gen_fn gen, void* user) {
    or_volume* v = (or_volume*)calloc(1, sizeof(or_volume));
    if (!v || !gen || or_geom_init(&v->g, dim, C, M, bg, tau) != 0) {
        free(v);
        return NULL;
    }
    const or_geom* g = &v->g;
    v->streamed = 1;
    v->gen = gen;
    v->user = user;
    for (int L = 0; L <= g->N; ++L) {
        if (L >= 1) {
            v->V[L] = (uint16_t*)malloc(sizeof(uint16_t) * (size_t)(g->ldim[L][0] * g->ldim[L][1] * g->ldim[L][2] * C));
            if (!v->V[L]) {
                or_volume_destroy(v);
                return NULL;
            }
        }
        v->nodes[L] = (or_node*)calloc((size_t)(g->nb[L][0] * g->nb[L][1] * g->nb[L][2]), sizeof(or_node));
        if (!v->nodes[L]) {
            or_volume_destroy(v);
            return NULL;
        }
    }
    const int64_t n0 = g->nb[0][0] * g->nb[0][1] * g->nb[0][2];
    v->sum0 = (uint64_t*)calloc((size_t)(n0 * C), sizeof(uint64_t));
    v->carry = (uint16_t*)malloc(sizeof(uint16_t) * (size_t)(dim[0] * dim[1] * C));
    if (!v->sum0 || !v->carry) {
        or_volume_destroy(v);
        return NULL;
    }
    for (int64_t i = 0; i < n0; ++i)
        for (int c = 0; c < C; ++c) {
            v->nodes[0][i].bmin[c] = 0xffff;
            v->nodes[0][i].bmax[c] = 0;
        }
    return v;
}

typedef struct {
    or_volume* v;
    const uint16_t* s0; /* level-0 slice z (and s1 = slice z + 1, or NULL) */
    const uint16_t* s1;
    int64_t z;
} feed_arg;

/* level-0 brick statistics of slice z, one task per row of bricks (disjoint node sets) */
static void feed_stats_rows(void* p, int64_t b, int64_t e) {
    feed_arg* a = (feed_arg*)p;
    or_volume* v = a->v;
    const or_geom* g = &v->g;
    const int C = g->C, M = g->M;
    const int64_t X = g->dim[0], Y = g->dim[1], k = a->z / M;
    for (int64_t j = b; j < e; ++j) {
        const int64_t y1 = (j + 1) * M < Y ? (j + 1) * M : Y;
        for (int64_t y = j * M; y < y1; ++y)
            for (int64_t x = 0; x < X; ++x) {
                const int64_t nid = nidx(g, 0, x / M, j, k);
                or_node* n = &v->nodes[0][nid];
                const uint16_t* val = a->s0 + (y * X + x) * C;
                for (int c = 0; c < C; ++c) {
                    if (val[c] < n->bmin[c]) n->bmin[c] = val[c];
                    if (val[c] > n->bmax[c]) n->bmax[c] = val[c];
                    v->sum0[nid * C + c] += val[c];
                }
                n->count++;
            }
    }
}

/* level-1 slice z / 2 from level-0 slices z and z + 1 (s1 == NULL: z + 1 is outside the volume) */
static void feed_level1_rows(void* p, int64_t b, int64_t e) {
    feed_arg* a = (feed_arg*)p;
    or_volume* v = a->v;
    const or_geom* g = &v->g;
    const int C = g->C;
    const int64_t X = g->dim[0], Y = g->dim[1];
    uint16_t* Q = v->V[1];
    for (int64_t y = b; y < e; ++y)
        for (int64_t x = 0; x < g->ldim[1][0]; ++x)
            for (int c = 0; c < C; ++c) {
                uint64_t S = 0, k = 0;
                for (int dz = 0; dz < 2; ++dz) {
                    const uint16_t* P = dz ? a->s1 : a->s0;
                    if (!P) continue;
                    for (int dy = 0; dy < 2; ++dy)
                        for (int dx = 0; dx < 2; ++dx) {
                            const int64_t cx = 2 * x + dx, cy = 2 * y + dy;
                            if (cx < X && cy < Y) {
                                S += P[(cy * X + cx) * C + c];
                                ++k;
                            }
                        }
                }
                Q[vidx(g, 1, x, y, a->z / 2) * C + c] = rhu(S, k);
            }
}

int or_stream_feed(or_volume* v, int64_t z0, int64_t nz, const uint16_t* slab, int threads) {
    if (!v || !v->streamed || z0 != v->next_z || nz <= 0 || z0 + nz > v->g.dim[2] || !slab) return -1;
    const or_geom* g = &v->g;
    const int64_t X = g->dim[0], Y = g->dim[1], plane = X * Y * g->C, Z = g->dim[2];
    for (int64_t z = z0; z < z0 + nz; ++z) {
        const uint16_t* sz = slab + (z - z0) * plane;
        feed_arg a = {v, sz, NULL, z};
        or_parallel_for(g->nb[0][1], 1, threads, feed_stats_rows, &a);
        if (g->N >= 1) {
            if ((z & 1) == 0) {
                if (z + 1 < z0 + nz) { /* partner in this slab */
                    a.s1 = sz + plane;
                    or_parallel_for(g->ldim[1][1], 8, threads, feed_level1_rows, &a);
                } else if (z + 1 == Z) { /* last slice of an odd extent */
                    or_parallel_for(g->ldim[1][1], 8, threads, feed_level1_rows, &a);
                } else {
                    memcpy(v->carry, sz, sizeof(uint16_t) * (size_t)plane);
                    v->have_carry = 1;
                }
            } else if (z == z0 && v->have_carry) { /* odd partner of the carried slice */
                feed_arg b = {v, v->carry, sz, z - 1};
                or_parallel_for(g->ldim[1][1], 8, threads, feed_level1_rows, &b);
                v->have_carry = 0;
            }
        }
    }
    v->next_z = z0 + nz;
    return 0;
}

static void stream_nodes_range(void* p, int64_t b, int64_t e) {
    lvl_arg* a = (lvl_arg*)p;
    or_volume* v = a->v;
    const or_geom* g = &v->g;
    const int L = a->L, C = g->C, M = g->M;
    for (int64_t r = b; r < e; ++r) {
        const int64_t i = r % g->nb[L][0], j = (r / g->nb[L][0]) % g->nb[L][1], k = r / (g->nb[L][0] * g->nb[L][1]);
        or_node* n = &v->nodes[L][r];
        uint64_t sum[OR_MAXC] = {0};
        if (L == 0) {
            for (int c = 0; c < C; ++c) {
                sum[c] = v->sum0[r * C + c];
                n->smin[c] = n->bmin[c];
                n->smax[c] = n->bmax[c];
            }
        } else {
            n->count = 0;
            for (int c = 0; c < C; ++c) {
                n->bmin[c] = n->smin[c] = 0xffff;
                n->bmax[c] = n->smax[c] = 0;
            }
            const int64_t lo[3] = {i * M, j * M, k * M};
            int64_t hi[3];
            for (int q = 0; q < 3; ++q) hi[q] = lo[q] + M < g->ldim[L][q] ? lo[q] + M : g->ldim[L][q];
            for (int64_t z = lo[2]; z < hi[2]; ++z)
                for (int64_t y = lo[1]; y < hi[1]; ++y)
                    for (int64_t x = lo[0]; x < hi[0]; ++x) {
                        const uint16_t* val = &v->V[L][vidx(g, L, x, y, z) * C];
                        for (int c = 0; c < C; ++c) {
                            sum[c] += val[c];
                            if (val[c] < n->bmin[c]) n->bmin[c] = val[c];
                            if (val[c] > n->bmax[c]) n->bmax[c] = val[c];
                        }
                        n->count++;
                    }
            for (int d = 0; d < 8; ++d) {
                const int64_t ci = 2 * i + (d & 1), cj = 2 * j + ((d >> 1) & 1), ck = 2 * k + (d >> 2);
                if (ci >= g->nb[L - 1][0] || cj >= g->nb[L - 1][1] || ck >= g->nb[L - 1][2]) continue;
                const or_node* ch = &v->nodes[L - 1][nidx(g, L - 1, ci, cj, ck)];
                for (int c = 0; c < C; ++c) {
                    if (ch->smin[c] < n->smin[c]) n->smin[c] = ch->smin[c];
                    if (ch->smax[c] > n->smax[c]) n->smax[c] = ch->smax[c];
                }
            }
        }
        n->touched = 1; /* the whole volume was fed */
        n->brick_homog = 1;
        n->subtree_homog = 1;
        for (int c = 0; c < C; ++c) {
            if (!((int)n->bmax[c] - (int)n->bmin[c] < (int)g->tau)) n->brick_homog = 0;
            if (!((int)n->smax[c] - (int)n->smin[c] < (int)g->tau)) n->subtree_homog = 0;
            n->avg[c] = rhu(sum[c], (uint64_t)n->count);
        }
        n->has_children = (L > 0) && !n->subtree_homog;
        n->has_brick = !n->brick_homog;
    }
}

int or_stream_finish(or_volume* v, int threads) {
    if (!v || !v->streamed || v->next_z != v->g.dim[2] || v->built) return -1;
    const or_geom* g = &v->g;
    for (int L = 2; L <= g->N; ++L) {
        lvl_arg a = {v, L};
        or_parallel_for(g->ldim[L][1] * g->ldim[L][2], 4, threads, build_level_rows, &a);
    }
    for (int L = 0; L <= g->N; ++L) { /* children before parents */
        lvl_arg a = {v, L};
        or_parallel_for(g->nb[L][0] * g->nb[L][1] * g->nb[L][2], 1, threads, stream_nodes_range, &a);
    }
    v->built = 1;
    return 0;
}

int or_node_info(or_volume* v, int L, int64_t i, int64_t j, int64_t k, or_node* out) {
    const or_geom* g = &v->g;
    if (L < 0 || L > g->N || i < 0 || j < 0 || k < 0 || i >= g->nb[L][0] || j >= g->nb[L][1] || k >= g->nb[L][2])
        return -1;
    if (v->lazy) {
        lazy_node(v, L, i, j, k, out);
        return 0;
    }
    if (!v->built) return -2;
    *out = v->nodes[L][nidx(g, L, i, j, k)];
    return 0;
}

void or_volume_destroy(or_volume* v) {
    if (!v) return;
    for (int L = 0; L < OR_MAXL; ++L) {
        free(v->V[L]);
        free(v->nodes[L]);
        if (v->vmemo[L]) {
            for (int s = 0; s < MEMO_SHARDS; ++s) {
                free(v->vmemo[L][s].keys);
                free(v->vmemo[L][s].vals);
                pthread_mutex_destroy(&v->vmemo[L][s].mu);
            }
            free(v->vmemo[L]);
        }
    }
    if (v->nmemo) {
        for (int s = 0; s < MEMO_SHARDS; ++s) {
            free(v->nmemo[s].keys);
            free(v->nmemo[s].vals);
            pthread_mutex_destroy(&v->nmemo[s].mu);
        }
        free(v->nmemo);
    }
    free(v->ins);
    free(v->carry);
    free(v->sum0);
    free(v);
}
