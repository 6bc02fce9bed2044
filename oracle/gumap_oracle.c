/*
 * CPU ORACLE for the graph-theoretic kNN path of GUMAP / SL-GUMAP.
 *
 * This file is TEST INFRASTRUCTURE. It is a plain, slow, obviously correct
 * restatement of what the path computes, used only by the tests, by the
 * smoke check and by the benchmark's CPU-baseline leg. It shares no code,
 * header, table or helper with the CUDA library and must never be linked
 * into it.
 *
 * What it computes (each function cites the passage it follows):
 *   - hop distances by breadth-first search from each source
 *       (Algorithm 1, all-pairs distances; Algorithm 4, partial BFS);
 *   - the kNN list of each source: the first k other vertices in
 *       (distance, vertex id) order (Section 3.3.1; the paper breaks ties at
 *       random, this library fixes the tie rule to ascending vertex id);
 *   - rho_i and sigma_i of the UMAP similarity
 *       h_ij = exp(-(d_ij - rho_i) / sigma_i)   (Section 2.1)
 *     with sigma_i solving sum_j exp(-max(0, d_ij - rho_i)/sigma_i) = log2 k;
 *   - the fuzzy union w_ij = a_ij + a_ji - a_ij * a_ji (the symmetrisation of
 *     the UMAP implementation the paper builds on, Section 4.1.1);
 *   - the quality metrics of a drawing X (Section 4.1.3): neighbourhood
 *     preservation with radius r and the aggregated stress.
 * Floating point is FP64 throughout, except the drawing's squared distances
 * that order N_D(v, r): those are FP32 (the layout's own precision), each
 * step rounded to float; the file is compiled with -ffp-contract=off so no
 * a*b+c is fused into one rounding.
 *
 * Readings taken where the paper is silent or garbled:
 *   - the source itself is not in its own list and has distance 0; the list
 *     holds k OTHER vertices (Section 3.3.1, "k other vertices");
 *   - partial BFS finishes the level at which k vertices are reached and then
 *     keeps the k smallest by (distance, id), instead of the paper's
 *     insertion-order break;
 *   - fewer than k reachable vertices: pad with id -1, distance 0xFFFF,
 *     weight 0 (unreachable pairs carry an "infinite" value, Section 3.2);
 *   - no root of the sigma equation: if the row has at most log2 k valid
 *     entries, sigma = +inf (all weights 1); if at least log2 k entries sit at
 *     distance rho, sigma -> 0+ and is lifted to the floor below;
 *   - sigma floor: sigma = max(sigma*, 1e-3 * mean valid distance);
 *   - neighbourhood preservation: N_G(v, r) excludes v; N_D(v, r) is ordered
 *     by (FP32 squared distance, id), the squared distance being a monotone
 *     function of the distance; a vertex with an empty N_G(v, r) counts 1
 *     (two empty sets are identical); the printed sum over v is returned;
 *   - stress: a pair with no connecting path contributes 1, the limit of its
 *     term as d_ij grows without bound ("infinite" distance, Section 3.2).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORACLE_INF16 0xFFFFu

/* ------------------------------------------------------------------ */
/* Breadth-first search (hop distances): Algorithm 1's distances.     */
/* dist[v] = -1 for unreachable vertices.                              */
/* ------------------------------------------------------------------ */
int oracle_bfs(const int32_t *row_ptr, const int32_t *col, int32_t n, int32_t s,
               int32_t *dist, int32_t *queue) {
    if (s < 0 || s >= n) return -1;
    for (int32_t v = 0; v < n; ++v) dist[v] = -1;
    int32_t head = 0, tail = 0;
    dist[s] = 0;
    queue[tail++] = s;
    while (head < tail) {
        int32_t u = queue[head++];
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            int32_t w = col[e];
            if (dist[w] < 0) {
                dist[w] = dist[u] + 1;
                queue[tail++] = w;
            }
        }
    }
    return 0;
}

/* All-pairs hop distances as an n x n uint16 matrix (0xFFFF = unreachable). */
int oracle_apsp(const int32_t *row_ptr, const int32_t *col, int32_t n, uint16_t *D) {
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!dist || !queue) { free(dist); free(queue); return -1; }
    for (int32_t s = 0; s < n; ++s) {
        oracle_bfs(row_ptr, col, n, s, dist, queue);
        for (int32_t v = 0; v < n; ++v)
            D[(size_t)s * n + v] = dist[v] < 0 ? (uint16_t)ORACLE_INF16 : (uint16_t)dist[v];
    }
    free(dist);
    free(queue);
    return 0;
}

/* (distance, id) pairs sorted ascending: the fixed tie rule. */
typedef struct { int32_t d, v; } dv_pair;

static int cmp_dv(const void *a, const void *b) {
    const dv_pair *x = (const dv_pair *)a, *y = (const dv_pair *)b;
    if (x->d != y->d) return (x->d > y->d) - (x->d < y->d);
    return (x->v > y->v) - (x->v < y->v);
}

static void write_row(const dv_pair *p, int32_t cnt, int32_t k, int32_t *idx, uint16_t *dst) {
    for (int32_t t = 0; t < k; ++t) {
        if (t < cnt) {
            idx[t] = p[t].v;
            dst[t] = (uint16_t)p[t].d;
        } else {
            idx[t] = -1;
            dst[t] = (uint16_t)ORACLE_INF16;
        }
    }
}

/*
 * Full form (GUMAP, Algorithm 1: all-pairs distances, then the k nearest):
 * for each source run BFS to completion, then sort every reachable vertex
 * other than the source by (distance, id) and keep the first k.
 * sources == NULL means all vertices 0..n-1 in order.
 */
int oracle_knn_full(const int32_t *row_ptr, const int32_t *col, int32_t n, int32_t k,
                    const int32_t *sources, int32_t n_src, int32_t *out_idx, uint16_t *out_dist) {
    if (k < 1) return -1;
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    dv_pair *pairs = (dv_pair *)malloc(sizeof(dv_pair) * (size_t)(n > 0 ? n : 1));
    if (!dist || !queue || !pairs) { free(dist); free(queue); free(pairs); return -1; }
    for (int32_t i = 0; i < n_src; ++i) {
        int32_t s = sources ? sources[i] : i;
        if (s < 0 || s >= n) { free(dist); free(queue); free(pairs); return -1; }
        oracle_bfs(row_ptr, col, n, s, dist, queue);
        int32_t cnt = 0;
        for (int32_t v = 0; v < n; ++v)
            if (v != s && dist[v] >= 0) { pairs[cnt].d = dist[v]; pairs[cnt].v = v; cnt++; }
        qsort(pairs, (size_t)cnt, sizeof(dv_pair), cmp_dv);
        write_row(pairs, cnt, k, out_idx + (size_t)i * k, out_dist + (size_t)i * k);
    }
    free(dist);
    free(queue);
    free(pairs);
    return 0;
}

/*
 * Partial form (SL-GUMAP, Algorithm 4 PartialBFS): level-by-level BFS from
 * the source, marking vertices on discovery; after each level the number of
 * vertices found so far is compared with k, and the search stops once the
 * level that reaches k is complete. The found vertices are then sorted by
 * (distance, id) and the first k kept.
 *
 * work_edges (optional, per source): the adjacency entries scanned by the
 * vertices expanded before the stopping level, i.e. sum of deg(u) over
 * d(u) < D_s, which is the traversal work of this form.
 */
int oracle_knn_partial(const int32_t *row_ptr, const int32_t *col, int32_t n, int32_t k,
                       const int32_t *sources, int32_t n_src, int32_t *out_idx,
                       uint16_t *out_dist, int64_t *work_edges) {
    if (k < 1) return -1;
    int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *cur = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *nxt = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    dv_pair *found = (dv_pair *)malloc(sizeof(dv_pair) * (size_t)(n > 0 ? n : 1));
    if (!mark || !cur || !nxt || !found) { free(mark); free(cur); free(nxt); free(found); return -1; }
    /* mark[v] == i means v was visited by the i-th source (stamps never repeat) */
    for (int32_t v = 0; v < n; ++v) mark[v] = -1;
    for (int32_t i = 0; i < n_src; ++i) {
        int32_t s = sources ? sources[i] : i;
        if (s < 0 || s >= n) { free(mark); free(cur); free(nxt); free(found); return -1; }
        int32_t stamp = i;
        int64_t work = 0;
        int32_t n_found = 0, n_cur = 1, level = 0;
        cur[0] = s;
        mark[s] = stamp;
        while (n_found < k && n_cur > 0) {
            level++;
            int32_t n_nxt = 0;
            for (int32_t q = 0; q < n_cur; ++q) {
                int32_t u = cur[q];
                work += row_ptr[u + 1] - row_ptr[u];
                for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
                    int32_t w = col[e];
                    if (mark[w] != stamp) {
                        mark[w] = stamp;
                        nxt[n_nxt++] = w;
                        found[n_found].d = level;
                        found[n_found].v = w;
                        n_found++;
                    }
                }
            }
            int32_t *t = cur; cur = nxt; nxt = t;
            n_cur = n_nxt;
        }
        qsort(found, (size_t)n_found, sizeof(dv_pair), cmp_dv);
        write_row(found, n_found, k, out_idx + (size_t)i * k, out_dist + (size_t)i * k);
        if (work_edges) work_edges[i] = work;
    }
    free(mark);
    free(cur);
    free(nxt);
    free(found);
    return 0;
}

/* ------------------------------------------------------------------ */
/* rho_i, sigma_i and directed weights (Section 2.1, h_ij).            */
/* ------------------------------------------------------------------ */

/* f(sigma) = sum over valid j of exp(-max(0, d_j - rho) / sigma) */
static double f_sigma(const uint16_t *d, int32_t kv, double rho, double sigma) {
    double acc = 0.0;
    for (int32_t j = 0; j < kv; ++j) {
        double x = (double)d[j] - rho;
        if (x < 0.0) x = 0.0;
        acc += exp(-x / sigma);
    }
    return acc;
}

/*
 * For each row (k slots, valid slots first, distances ascending, padding
 * 0xFFFF): rho = smallest valid distance; sigma from the calibration
 * equation by bisection on a doubling bracket, run until the bracket stops
 * shrinking; a_ij = exp(-max(0, d_ij - rho)/sigma); padding weight 0.
 * Rows with no valid slot get rho = 0, sigma = 0.
 */
void oracle_smooth_knn(const uint16_t *dist, int32_t n_rows, int32_t k, double *rho_out,
                       double *sigma_out, double *a_out) {
    const double T = log2((double)k);
    for (int32_t i = 0; i < n_rows; ++i) {
        const uint16_t *d = dist + (size_t)i * k;
        double *a = a_out + (size_t)i * k;
        int32_t kv = 0;
        while (kv < k && d[kv] != ORACLE_INF16) kv++;
        if (kv == 0) {
            rho_out[i] = 0.0;
            sigma_out[i] = 0.0;
            for (int32_t j = 0; j < k; ++j) a[j] = 0.0;
            continue;
        }
        double rho = (double)d[0];
        double mean = 0.0;
        int32_t c_eq = 0;
        for (int32_t j = 0; j < kv; ++j) {
            if ((double)d[j] < rho) rho = (double)d[j];
            mean += (double)d[j];
        }
        mean /= (double)kv;
        for (int32_t j = 0; j < kv; ++j)
            if ((double)d[j] == rho) c_eq++;
        double sigma;
        if ((double)kv <= T) {
            sigma = INFINITY;            /* f(sigma) < T for every sigma */
        } else if ((double)c_eq >= T) {
            sigma = 0.0;                 /* f(sigma) > T for every sigma > 0 */
        } else {
            double lo = 0.0, hi = 1.0;
            while (f_sigma(d, kv, rho, hi) < T) hi *= 2.0;
            for (;;) {
                double mid = 0.5 * (lo + hi);
                if (!(mid > lo && mid < hi)) break;
                if (f_sigma(d, kv, rho, mid) > T) hi = mid;
                else lo = mid;
            }
            sigma = 0.5 * (lo + hi);
        }
        double floor_ = 1e-3 * mean;
        if (sigma < floor_) sigma = floor_;
        rho_out[i] = rho;
        sigma_out[i] = sigma;
        for (int32_t j = 0; j < k; ++j) {
            if (j < kv) {
                double x = (double)d[j] - rho;
                if (x < 0.0) x = 0.0;
                a[j] = isinf(sigma) ? 1.0 : exp(-x / sigma);
            } else {
                a[j] = 0.0;
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* Fuzzy union w_ij = a_ij + a_ji - a_ij a_ji (absent direction = 0).  */
/* ------------------------------------------------------------------ */

/* weight of j's slot pointing at i, or 0 if i is not in j's list */
static double lookup(const int32_t *idx, const double *a, int32_t k, int32_t j, int32_t i) {
    for (int32_t t = 0; t < k; ++t)
        if (idx[(size_t)j * k + t] == i) return a[(size_t)j * k + t];
    return 0.0;
}

/* Per-slot union weight for a list built over ALL vertices (row i = vertex i). */
void oracle_slot_union(const int32_t *idx, const double *a, int32_t n, int32_t k, double *w) {
    for (int32_t i = 0; i < n; ++i)
        for (int32_t t = 0; t < k; ++t) {
            int32_t j = idx[(size_t)i * k + t];
            if (j < 0) { w[(size_t)i * k + t] = 0.0; continue; }
            double aij = a[(size_t)i * k + t];
            double aji = lookup(idx, a, k, j, i);
            w[(size_t)i * k + t] = aij + aji - aij * aji;
        }
}

typedef struct { int64_t key; double val; } kv_pair;

static int cmp_kv(const void *a, const void *b) {
    int64_t x = ((const kv_pair *)a)->key, y = ((const kv_pair *)b)->key;
    return (x > y) - (x < y);
}

/*
 * Symmetric COO of the union, sorted by (row, col): every directed entry
 * (i, j, a_ij) and its transpose (j, i, a_ij) keyed by row * n + col, sorted,
 * equal keys merged with a + b - a b. Returns nnz (or -1 on failure).
 * Output buffers must hold 2 * n * k entries.
 */
int64_t oracle_coo_union(const int32_t *idx, const double *a, int32_t n, int32_t k,
                         int32_t *row, int32_t *colo, double *w) {
    size_t cap = (size_t)2 * n * k;
    kv_pair *e = (kv_pair *)malloc(sizeof(kv_pair) * (cap > 0 ? cap : 1));
    if (!e) return -1;
    size_t m = 0;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t t = 0; t < k; ++t) {
            int32_t j = idx[(size_t)i * k + t];
            if (j < 0) continue;
            double v = a[(size_t)i * k + t];
            e[m].key = (int64_t)i * n + j; e[m].val = v; m++;
            e[m].key = (int64_t)j * n + i; e[m].val = v; m++;
        }
    qsort(e, m, sizeof(kv_pair), cmp_kv);
    int64_t nnz = 0;
    for (size_t p = 0; p < m;) {
        double v = e[p].val;
        size_t q = p + 1;
        while (q < m && e[q].key == e[p].key) {
            v = v + e[q].val - v * e[q].val;
            q++;
        }
        row[nnz] = (int32_t)(e[p].key / n);
        colo[nnz] = (int32_t)(e[p].key % n);
        w[nnz] = v;
        nnz++;
        p = q;
    }
    free(e);
    return nnz;
}

/* ------------------------------------------------------------------ */
/* Quality metrics of a drawing (Section 4.1.3).                       */
/* X is the drawing, float[n][dim] row-major.                          */
/* ------------------------------------------------------------------ */

/* Squared Euclidean distance of rows u and v in FP32: per coordinate the
 * difference, its square, then the running sum in coordinate order, every
 * step rounded to float. */
static float sqdist32(const float *X, int32_t dim, int32_t u, int32_t v) {
    float acc = 0.0f;
    for (int32_t c = 0; c < dim; ++c) {
        float dx = X[(size_t)u * dim + c] - X[(size_t)v * dim + c];
        float sq = dx * dx;
        acc = acc + sq;
    }
    return acc;
}

/* (squared distance, id): the order of the geometric neighbourhood. */
typedef struct { float d2; int32_t v; } gd_pair;

static int cmp_gd(const void *a, const void *b) {
    const gd_pair *x = (const gd_pair *)a, *y = (const gd_pair *)b;
    if (x->d2 < y->d2) return -1;
    if (x->d2 > y->d2) return 1;
    return x->v < y->v ? -1 : (x->v > y->v);
}

/*
 * Neighbourhood preservation (Section 4.1.3). For each vertex v:
 *   N_G(v, r) = the other vertices at hop distance at most r (BFS);
 *   N_D(v, r) = the |N_G(v, r)| other vertices closest to v in the drawing,
 *               by (FP32 squared distance, id);
 * For the vertices verts[0 .. n_verts) (verts NULL: all n in order) it writes
 * out_c[i] = |N_G(v, r)|, out_inter[i] = |N_G(v, r) ∩ N_D(v, r)|, and returns
 * the printed sum over them of |∩| / |∪|, where |∪| = 2 |N_G| - |∩| because
 * both sets have |N_G| elements; a vertex with an empty N_G(v, r) adds 1.
 * Returns -1 on failure.
 */
double oracle_np(const int32_t *row_ptr, const int32_t *col, int32_t n, const float *X, int32_t dim, int32_t r,
                 const int32_t *verts, int32_t n_verts, int32_t *out_c, int32_t *out_inter) {
    if (n < 1 || dim < 1 || r < 1) return -1.0;
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    gd_pair *geo = (gd_pair *)malloc(sizeof(gd_pair) * (size_t)n);
    if (!dist || !queue || !geo) { free(dist); free(queue); free(geo); return -1.0; }
    double total = 0.0;
    for (int32_t vi = 0; vi < n_verts; ++vi) {
        int32_t v = verts ? verts[vi] : vi;
        if (v < 0 || v >= n) { free(dist); free(queue); free(geo); return -1.0; }
        oracle_bfs(row_ptr, col, n, v, dist, queue);
        int32_t c = 0;
        for (int32_t u = 0; u < n; ++u)
            if (u != v && dist[u] >= 0 && dist[u] <= r) c++;
        int32_t m = 0;
        for (int32_t u = 0; u < n; ++u)
            if (u != v) { geo[m].d2 = sqdist32(X, dim, u, v); geo[m].v = u; m++; }
        qsort(geo, (size_t)m, sizeof(gd_pair), cmp_gd);
        int32_t inter = 0;
        for (int32_t t = 0; t < c; ++t) {
            int32_t u = geo[t].v;
            if (dist[u] >= 0 && dist[u] <= r) inter++;
        }
        out_c[vi] = c;
        out_inter[vi] = inter;
        total += c == 0 ? 1.0 : (double)inter / (double)(2 * c - inter);
    }
    free(dist);
    free(queue);
    free(geo);
    return total;
}

/*
 * Aggregated stress (Section 4.1.3):
 *   1/(n^2 - n) * sum over ordered pairs i != j of ((d_ij - ||X_i - X_j||) / d_ij)^2
 * with d_ij the hop distance (BFS) and ||.|| the Euclidean distance in FP64.
 * A pair with no connecting path adds 1. row_out (optional) receives the sum
 * over j of each row i = verts[ii] (verts NULL: all n rows in order); the
 * return value is the sum of those rows / (n^2 - n), the stress itself when
 * every row is taken. Returns -1 on failure.
 */
double oracle_stress(const int32_t *row_ptr, const int32_t *col, int32_t n, const float *X, int32_t dim,
                     const int32_t *verts, int32_t n_verts, double *row_out) {
    if (n < 2 || dim < 1) return -1.0;
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!dist || !queue) { free(dist); free(queue); return -1.0; }
    double total = 0.0;
    for (int32_t ii = 0; ii < n_verts; ++ii) {
        int32_t i = verts ? verts[ii] : ii;
        if (i < 0 || i >= n) { free(dist); free(queue); return -1.0; }
        oracle_bfs(row_ptr, col, n, i, dist, queue);
        double row = 0.0;
        for (int32_t j = 0; j < n; ++j) {
            if (j == i) continue;
            if (dist[j] < 0) { row += 1.0; continue; }
            double sq = 0.0;
            for (int32_t c = 0; c < dim; ++c) {
                double dx = (double)X[(size_t)i * dim + c] - (double)X[(size_t)j * dim + c];
                sq += dx * dx;
            }
            double t = ((double)dist[j] - sqrt(sq)) / (double)dist[j];
            row += t * t;
        }
        if (row_out) row_out[ii] = row;
        total += row;
    }
    free(dist);
    free(queue);
    return total / ((double)n * (double)n - (double)n);
}
