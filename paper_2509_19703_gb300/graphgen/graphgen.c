/*
 * Seeded synthetic graph generators.
 *
 * This module produces the input graphs that both the CUDA path and the CPU
 * oracle consume. It holds none of the method's arithmetic (no BFS, no
 * distances, no weights): only random-graph models and a CSR builder.
 *
 * The paper evaluates on real scale-free, GION (large-diameter RNA) and mesh
 * graphs (Section 4.1.2, Table 2), which are not available here. These models
 * stand in for them: Barabasi-Albert for scale-free, 2-D grids for meshes,
 * G(n,p) and uniform random trees to bracket the dense and the large-diameter
 * ends. The paper uses the largest connected component of each graph; every
 * model here except G(n,p) at low density is connected by construction.
 *
 * Random numbers: xoshiro256** (Blackman & Vigna, 2018) seeded through
 * splitmix64 (Steele, Lea & Flood, 2014), both written from their published
 * definitions. Only integer arithmetic decides graph structure, except the
 * geometric skip of G(n,p) (Batagelj & Brandes, 2005) which uses log().
 *
 * Output is CSR over int32 ids in generator order: rows sorted ascending,
 * symmetric, no self loops, no duplicate entries.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct {
    int32_t n;
    int64_t nnz;      /* directed entries = 2 * undirected edges */
    int32_t *row_ptr; /* n + 1 (int32: nnz must stay below 2^31) */
    int32_t *col;     /* nnz */
} gg_csr;

/* ---------------- random numbers ---------------- */

typedef struct { uint64_t s[4]; } gg_rng;

static uint64_t splitmix64_next(uint64_t *x) {
    uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static void rng_seed(gg_rng *r, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64_next(&x);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t rng_next(gg_rng *r) {
    uint64_t *s = r->s;
    uint64_t result = rotl64(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}

/* uniform integer in [0, bound) by 64x64->128 multiply-shift */
static inline uint64_t rng_below(gg_rng *r, uint64_t bound) {
    return (uint64_t)(((unsigned __int128)rng_next(r) * bound) >> 64);
}

/* uniform double in [0, 1) with 53 random bits */
static inline double rng_unit(gg_rng *r) {
    return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0);
}

/* ---------------- edge list -> CSR ---------------- */

typedef struct {
    int64_t len, cap;
    int32_t *u, *v;
} edge_buf;

static int eb_init(edge_buf *e, int64_t cap) {
    if (cap < 16) cap = 16;
    e->len = 0;
    e->cap = cap;
    e->u = (int32_t *)malloc(sizeof(int32_t) * cap);
    e->v = (int32_t *)malloc(sizeof(int32_t) * cap);
    return (e->u && e->v) ? 0 : -1;
}

static int eb_push(edge_buf *e, int32_t a, int32_t b) {
    if (e->len == e->cap) {
        int64_t nc = e->cap * 2;
        int32_t *nu = (int32_t *)realloc(e->u, sizeof(int32_t) * nc);
        if (!nu) return -1;
        e->u = nu;
        int32_t *nv = (int32_t *)realloc(e->v, sizeof(int32_t) * nc);
        if (!nv) return -1;
        e->v = nv;
        e->cap = nc;
    }
    e->u[e->len] = a;
    e->v[e->len] = b;
    e->len++;
    return 0;
}

static void eb_free(edge_buf *e) {
    free(e->u);
    free(e->v);
    e->u = e->v = NULL;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

void gg_free(gg_csr *g) {
    if (!g) return;
    free(g->row_ptr);
    free(g->col);
    free(g);
}

/* Symmetrise, drop self loops and duplicates, sort rows. */
gg_csr *gg_from_edges(int32_t n, int64_t ne, const int32_t *eu, const int32_t *ev) {
    if (n < 0) return NULL;
    gg_csr *g = (gg_csr *)calloc(1, sizeof(gg_csr));
    if (!g) return NULL;
    g->n = n;
    int64_t *deg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!deg) { free(g); return NULL; }
    for (int64_t e = 0; e < ne; ++e) {
        int32_t a = eu[e], b = ev[e];
        if (a == b || a < 0 || b < 0 || a >= n || b >= n) continue;
        deg[a]++;
        deg[b]++;
    }
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int32_t *tmp = NULL;
    int64_t total = 0;
    for (int32_t i = 0; i < n; ++i) { pos[i] = total; total += deg[i]; }
    pos[n] = total;
    tmp = (int32_t *)malloc(sizeof(int32_t) * (total > 0 ? total : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!pos || !tmp || !fill) { free(deg); free(pos); free(tmp); free(fill); free(g); return NULL; }
    memcpy(fill, pos, sizeof(int64_t) * ((size_t)n + 1));
    for (int64_t e = 0; e < ne; ++e) {
        int32_t a = eu[e], b = ev[e];
        if (a == b || a < 0 || b < 0 || a >= n || b >= n) continue;
        tmp[fill[a]++] = b;
        tmp[fill[b]++] = a;
    }
    /* sort and dedup each row in place */
    int64_t out = 0;
    g->row_ptr = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    if (!g->row_ptr) { free(deg); free(pos); free(tmp); free(fill); free(g); return NULL; }
    for (int32_t i = 0; i < n; ++i) {
        int64_t b0 = pos[i], b1 = pos[i + 1];
        qsort(tmp + b0, (size_t)(b1 - b0), sizeof(int32_t), cmp_i32);
        g->row_ptr[i] = (int32_t)out;
        for (int64_t t = b0; t < b1; ++t)
            if (t == b0 || tmp[t] != tmp[t - 1]) tmp[out++] = tmp[t];
    }
    g->row_ptr[n] = (int32_t)out;
    g->nnz = out;
    g->col = (int32_t *)malloc(sizeof(int32_t) * (out > 0 ? out : 1));
    if (!g->col) { free(deg); free(pos); free(tmp); free(fill); free(g->row_ptr); free(g); return NULL; }
    memcpy(g->col, tmp, sizeof(int32_t) * (size_t)out);
    free(deg);
    free(pos);
    free(tmp);
    free(fill);
    return g;
}

static gg_csr *finish(int32_t n, edge_buf *e) {
    gg_csr *g = gg_from_edges(n, e->len, e->u, e->v);
    eb_free(e);
    return g;
}

/* ---------------- deterministic families ---------------- */

/* W x H grid, vertex id = row * W + column (row-major). */
gg_csr *gg_grid(int32_t W, int32_t H) {
    if (W < 1 || H < 1) return NULL;
    int64_t n = (int64_t)W * H;
    if (n > INT32_MAX) return NULL;
    edge_buf e;
    if (eb_init(&e, 2 * n)) return NULL;
    for (int32_t r = 0; r < H; ++r)
        for (int32_t c = 0; c < W; ++c) {
            int32_t v = r * W + c;
            if (c + 1 < W) eb_push(&e, v, v + 1);
            if (r + 1 < H) eb_push(&e, v, v + W);
        }
    return finish((int32_t)n, &e);
}

gg_csr *gg_path(int32_t n) {
    edge_buf e;
    if (n < 1 || eb_init(&e, n)) return NULL;
    for (int32_t i = 0; i + 1 < n; ++i) eb_push(&e, i, i + 1);
    return finish(n, &e);
}

gg_csr *gg_cycle(int32_t n) {
    edge_buf e;
    if (n < 3 || eb_init(&e, n)) return NULL;
    for (int32_t i = 0; i < n; ++i) eb_push(&e, i, (i + 1) % n);
    return finish(n, &e);
}

/* star with centre 0 and leaves 1..n-1 */
gg_csr *gg_star(int32_t n) {
    edge_buf e;
    if (n < 2 || eb_init(&e, n)) return NULL;
    for (int32_t i = 1; i < n; ++i) eb_push(&e, 0, i);
    return finish(n, &e);
}

gg_csr *gg_complete(int32_t n) {
    edge_buf e;
    if (n < 1 || n > 46000 || eb_init(&e, (int64_t)n * (n - 1) / 2 + 1)) return NULL;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = i + 1; j < n; ++j) eb_push(&e, i, j);
    return finish(n, &e);
}

/* ---------------- random families ---------------- */

/*
 * Barabasi-Albert preferential attachment: a clique on m0 + 1 vertices, then
 * each new vertex v attaches to m0 distinct earlier vertices chosen with
 * probability proportional to degree (uniform draws from the endpoint list).
 */
gg_csr *gg_ba(int32_t n, int32_t m0, uint64_t seed) {
    if (m0 < 1 || n < m0 + 1) return NULL;
    gg_rng r;
    rng_seed(&r, seed);
    int64_t ne_max = (int64_t)m0 * (m0 + 1) / 2 + (int64_t)(n - m0 - 1) * m0;
    edge_buf e;
    if (eb_init(&e, ne_max + 1)) return NULL;
    int32_t *ends = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * ne_max + 2));
    int32_t *pick = (int32_t *)malloc(sizeof(int32_t) * (size_t)m0);
    if (!ends || !pick) { free(ends); free(pick); eb_free(&e); return NULL; }
    int64_t ne = 0;
    for (int32_t i = 0; i <= m0; ++i)
        for (int32_t j = i + 1; j <= m0; ++j) {
            eb_push(&e, i, j);
            ends[ne++] = i;
            ends[ne++] = j;
        }
    for (int32_t v = m0 + 1; v < n; ++v) {
        int32_t got = 0;
        while (got < m0) {
            int32_t t = ends[rng_below(&r, (uint64_t)ne)];
            int dup = 0;
            for (int32_t q = 0; q < got; ++q)
                if (pick[q] == t) { dup = 1; break; }
            if (!dup) pick[got++] = t;
        }
        for (int32_t q = 0; q < m0; ++q) {
            eb_push(&e, v, pick[q]);
            ends[ne++] = v;
            ends[ne++] = pick[q];
        }
    }
    free(ends);
    free(pick);
    return finish(n, &e);
}

/* G(n, p) by geometric skipping over the lower triangle (Batagelj & Brandes). */
gg_csr *gg_gnp(int32_t n, double p, uint64_t seed) {
    if (n < 1 || !(p >= 0.0) || p > 1.0) return NULL;
    gg_rng r;
    rng_seed(&r, seed);
    double expect = p * (double)n * (double)(n - 1) / 2.0;
    edge_buf e;
    if (eb_init(&e, (int64_t)(expect * 1.1) + 64)) return NULL;
    if (p > 0.0) {
        if (p >= 1.0) {
            for (int32_t i = 0; i < n; ++i)
                for (int32_t j = 0; j < i; ++j) eb_push(&e, i, j);
        } else {
            double lq = log(1.0 - p);
            int64_t v = 1, w = -1;
            while (v < n) {
                double u = rng_unit(&r);
                w += 1 + (int64_t)floor(log(1.0 - u) / lq);
                while (w >= v && v < n) { w -= v; v++; }
                if (v < n) eb_push(&e, (int32_t)v, (int32_t)w);
            }
        }
    }
    return finish(n, &e);
}

/* Uniform random labelled tree by decoding a random Pruefer sequence. */
gg_csr *gg_tree(int32_t n, uint64_t seed) {
    if (n < 1) return NULL;
    edge_buf e;
    if (eb_init(&e, n)) return NULL;
    if (n == 2) eb_push(&e, 0, 1);
    if (n > 2) {
        gg_rng r;
        rng_seed(&r, seed);
        int32_t L = n - 2;
        int32_t *seq = (int32_t *)malloc(sizeof(int32_t) * L);
        int32_t *deg = (int32_t *)malloc(sizeof(int32_t) * n);
        if (!seq || !deg) { free(seq); free(deg); eb_free(&e); return NULL; }
        for (int32_t i = 0; i < n; ++i) deg[i] = 1;
        for (int32_t i = 0; i < L; ++i) {
            seq[i] = (int32_t)rng_below(&r, (uint64_t)n);
            deg[seq[i]]++;
        }
        /* linear-time decoding with a moving pointer to the smallest leaf */
        int32_t ptr = 0;
        while (deg[ptr] != 1) ptr++;
        int32_t leaf = ptr;
        for (int32_t i = 0; i < L; ++i) {
            int32_t v = seq[i];
            eb_push(&e, leaf, v);
            if (--deg[v] == 1 && v < ptr) {
                leaf = v;
            } else {
                ptr++;
                while (deg[ptr] != 1) ptr++;
                leaf = ptr;
            }
        }
        /* join the last leaf to n-1 */
        eb_push(&e, leaf, n - 1);
        free(seq);
        free(deg);
    }
    return finish(n, &e);
}

/* Seeded uniform doubles in [0, 1), used to draw workload mixes. */
void gg_uniform(uint64_t seed, int64_t count, double *out) {
    gg_rng r;
    rng_seed(&r, seed);
    for (int64_t i = 0; i < count; ++i) out[i] = rng_unit(&r);
}
