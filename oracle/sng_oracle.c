/*
 * sng_oracle.c -- plain, slow, single-threaded FP64 oracle for SNG-DBSCAN.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code, header, table or constant generator with the CUDA path: every
 * definition below is written out again from the paper and from the published
 * SplitMix64 output function.
 *
 * What it computes follows Algorithm 1 ("Subsampled Neighborhood Graph DBSCAN")
 * of Jiang, Jang & Lacki, "Faster DBSCAN via subsampled similarity queries"
 * (NeurIPS 2020), Section 3, step by step:
 *   step 1  G = (X, {})                         -> empty edge list
 *   step 2  for each x, ceil(s n) sampled partners x_ij, edge if |x-x_ij| <= eps
 *                                                -> orc_build_rows
 *   step 3  components of the subgraph induced by vertices of degree >= MinPts
 *                                                -> orc_degrees, orc_components_bfs,
 *                                                   orc_components_uf
 *   step 4  every non-core x connected to some K_i joins one of them
 *                                                -> orc_border_labels
 *   step 5  return the clusters; all other points are noise (label -1)
 *
 * Readings where the paper is silent (each is stated again where it is used):
 *  - Partners are drawn with replacement, never the point itself, by a
 *    counter-based hash: k_i = mix(seed ^ mix(i)), h = mix(k_i ^ j),
 *    r = h mod (n-1), partner = r + (r >= i); mix = SplitMix64 output function
 *    (Steele, Lea & Flood, OOPSLA 2014).  Duplicate draws are multi-edges.
 *  - Distance: d2 = sum_k ((double)a_k - (double)b_k)^2 summed left to right,
 *    every operation rounded separately (built with -ffp-contract=off);
 *    edge iff d2 <= (double)eps * (double)eps (closed ball, step 2).  The
 *    method needs only similarity queries (Section 1), so other neighbourhood
 *    tests are offered as well, each in a stated FP64 order: inner product
 *    and cosine similarity (edge iff sim >= eps), Manhattan and Chebyshev
 *    distance (edge iff dist <= eps; orc_l1, orc_linf).
 *  - Degree (step 3) default: undirected multigraph degree, each kept draw
 *    (i,p) adds one to both endpoints.  Mode 1: out-degree only (the count
 *    that the proof of Lemma 2 thresholds).  Mode 2: simple-graph degree
 *    (distinct neighbours in either direction), documentation only.
 *  - A border point adjacent to several components (step 4, "choose one
 *    arbitrarily") takes the smallest component label; a component's label
 *    is the smallest point index among its core points.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -fPIC -shared.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ hash */

/* SplitMix64 output function (Steele, Lea & Flood 2014): one increment of the
 * golden-gamma constant followed by the two xor-shift-multiply rounds and a
 * final xor-shift.  mix(0) is the generator's first output from state 0. */
uint64_t orc_mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Partner number j of point i (Algorithm 1, step 2: "sample ceil(sn) examples
 * from X").  sample_all != 0 enumerates every other point instead (j + [j>=i]),
 * which turns step 2 into the full eps-neighbourhood graph of textbook DBSCAN. */
int64_t orc_partner(uint64_t seed, int64_t i, int64_t j, int64_t n, int32_t sample_all)
{
    if (sample_all)
        return j + (j >= i ? 1 : 0);
    uint64_t key = orc_mix64(seed ^ orc_mix64((uint64_t)i));
    uint64_t h = orc_mix64(key ^ (uint64_t)j);
    uint64_t r = h % (uint64_t)(n - 1);
    return (int64_t)r + ((int64_t)r >= i ? 1 : 0);
}

/* Partners of rows i0..i0+ni-1, draws 0..m-1, row-major into out[ni*m]. */
void orc_partners(uint64_t seed, int64_t n, int64_t i0, int64_t ni, int64_t m,
                  int32_t sample_all, int64_t *out)
{
    for (int64_t r = 0; r < ni; ++r)
        for (int64_t j = 0; j < m; ++j)
            out[r * m + j] = orc_partner(seed, i0 + r, j, n, sample_all);
}

/* Squared Euclidean distance in FP64, left to right, no fused operations. */
double orc_dist2(const float *a, const float *b, int32_t d)
{
    double s = 0.0;
    for (int32_t k = 0; k < d; ++k) {
        double t = (double)a[k] - (double)b[k];
        double t2 = t * t;
        s = s + t2;
    }
    return s;
}

/* ------------------------------------------------------------ graph build */

typedef struct {
    int64_t n_rows;      /* number of source rows listed */
    int64_t num_edges;   /* kept draws */
    int64_t *row_ptr;    /* n_rows + 1 */
    int32_t *col;        /* num_edges partners, in draw order j within a row */
    int64_t band_pairs;  /* draws with |d2 - eps^2| <= band_rel * eps^2 */
} orc_graph;

void orc_graph_free(orc_graph *g)
{
    if (!g) return;
    free(g->row_ptr);
    free(g->col);
    g->row_ptr = NULL;
    g->col = NULL;
}

/*
 * Algorithm 1, step 2 for a list of source rows (rows == NULL: all n rows in
 * order).  Row r of the result lists, in draw order j = 0..m-1, the partners p
 * of point rows[r] with d2(x_i, x_p) <= eps^2.  band_point (length n, may be
 * NULL) gets a 1 at both ends of every draw whose FP64 d2 lies within
 * band_rel * eps^2 of eps^2.  Returns 0, or -1 on bad arguments / no memory.
 */
int32_t orc_build_rows_m(int64_t n, int32_t d, int64_t ld, const float *x, float eps,
                         uint64_t seed, int64_t m, int32_t sample_all, double band_rel,
                         const int64_t *rows, int64_t n_rows, orc_graph *out,
                         uint8_t *band_point, const int32_t *m_row);
int32_t orc_build_rows_metric(int64_t n, int32_t d, int64_t ld, const float *x, float eps,
                              uint64_t seed, int64_t m, int32_t sample_all, double band_rel,
                              const int64_t *rows, int64_t n_rows, orc_graph *out,
                              uint8_t *band_point, const int32_t *m_row, int32_t metric);

int32_t orc_build_rows(int64_t n, int32_t d, int64_t ld, const float *x, float eps,
                       uint64_t seed, int64_t m, int32_t sample_all, double band_rel,
                       const int64_t *rows, int64_t n_rows, orc_graph *out,
                       uint8_t *band_point)
{
    return orc_build_rows_m(n, d, ld, x, eps, seed, m, sample_all, band_rel, rows, n_rows, out,
                            band_point, NULL);
}

/*
 * As orc_build_rows, but point i draws only its first m_row[i] partners of
 * the same stream (m_row == NULL: m for every point).  This is the graph of
 * the surrogate-gated form: a point the gate calls noise draws nothing, one it
 * calls core draws a prefix of its draws, an uncertain one draws all m.
 */
int32_t orc_build_rows_m(int64_t n, int32_t d, int64_t ld, const float *x, float eps,
                         uint64_t seed, int64_t m, int32_t sample_all, double band_rel,
                         const int64_t *rows, int64_t n_rows, orc_graph *out,
                         uint8_t *band_point, const int32_t *m_row)
{
    return orc_build_rows_metric(n, d, ld, x, eps, seed, m, sample_all, band_rel, rows, n_rows,
                                 out, band_point, m_row, 0);
}

/* Inner product <a, b> in FP64: products and sums left to right, each
 * operation rounded on its own. */
double orc_dot(const float *a, const float *b, int32_t d)
{
    double s = 0.0;
    for (int32_t k = 0; k < d; ++k) {
        double t = (double)a[k] * (double)b[k];
        s = s + t;
    }
    return s;
}

/* Cosine similarity <a, b> / (|a| |b|): the inner product and both squared
 * norms as in orc_dot, then sqrt(|a|^2) * sqrt(|b|^2), the quotient last; a
 * zero vector gives NaN, which is never similar to anything. */
double orc_cosine(const float *a, const float *b, int32_t d)
{
    double ab = orc_dot(a, b, d);
    double aa = orc_dot(a, a, d);
    double bb = orc_dot(b, b, d);
    double den = sqrt(aa) * sqrt(bb);
    return ab / den;
}

/* Manhattan distance sum_k |a_k - b_k| in FP64: each difference, its
 * absolute value and each sum left to right; a NaN difference makes the
 * distance NaN (never within eps). */
double orc_l1(const float *a, const float *b, int32_t d)
{
    double s = 0.0;
    for (int32_t k = 0; k < d; ++k) {
        double t = (double)a[k] - (double)b[k];
        s = s + fabs(t);
    }
    return s;
}

/* Chebyshev distance max_k |a_k - b_k| in FP64; a NaN difference makes the
 * distance NaN (fmax would drop it). */
double orc_linf(const float *a, const float *b, int32_t d)
{
    double s = 0.0;
    for (int32_t k = 0; k < d; ++k) {
        double t = fabs((double)a[k] - (double)b[k]);
        if (t != t) return t;
        if (t > s) s = t;
    }
    return s;
}

/* Algorithm 1, step 2 with the neighbourhood test of `metric`: 0 = Euclidean
 * ball (d2 <= eps^2, band |d2 - eps^2| <= band_rel eps^2); 1 = inner product,
 * 2 = cosine similarity (edge iff sim >= eps, band |sim - eps| <= band_rel
 * |eps|); 3 = Manhattan, 4 = Chebyshev distance (edge iff dist <= eps, band
 * |dist - eps| <= band_rel eps). */
int32_t orc_build_rows_metric(int64_t n, int32_t d, int64_t ld, const float *x, float eps,
                              uint64_t seed, int64_t m, int32_t sample_all, double band_rel,
                              const int64_t *rows, int64_t n_rows, orc_graph *out,
                              uint8_t *band_point, const int32_t *m_row, int32_t metric)
{
    if (n < 2 || d < 1 || ld < d || m < 0 || !out) return -1;
    if (sample_all && m != n - 1) return -1;
    if (metric < 0 || metric > 4) return -1;
    if (!rows) n_rows = n;
    double eps2 = (double)eps * (double)eps;
    double band = band_rel * eps2;
    double tau = (double)eps;
    if (metric != 0) band = band_rel * fabs(tau);
    int64_t cap = 1024, e = 0;
    int32_t *col = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    int64_t *row_ptr = (int64_t *)malloc((size_t)(n_rows + 1) * sizeof(int64_t));
    if (!col || !row_ptr) { free(col); free(row_ptr); return -1; }
    int64_t band_pairs = 0;
    row_ptr[0] = 0;
    for (int64_t r = 0; r < n_rows; ++r) {
        int64_t i = rows ? rows[r] : r;
        const float *xi = x + i * ld;
        int64_t mi = m_row ? (int64_t)m_row[i] : m;
        if (mi > m) mi = m;
        for (int64_t j = 0; j < mi; ++j) {
            int64_t p = orc_partner(seed, i, j, n, sample_all);
            double v, gap;
            int keep;
            if (metric == 0) {
                v = orc_dist2(xi, x + p * ld, d);
                gap = v - eps2;
                keep = v <= eps2;
            } else if (metric >= 3) {
                v = metric == 3 ? orc_l1(xi, x + p * ld, d) : orc_linf(xi, x + p * ld, d);
                gap = v - tau;
                keep = v <= tau;
            } else {
                v = metric == 1 ? orc_dot(xi, x + p * ld, d) : orc_cosine(xi, x + p * ld, d);
                gap = v - tau;
                keep = v >= tau;
            }
            if (gap < 0) gap = -gap;
            if (gap <= band) {
                ++band_pairs;
                if (band_point) { band_point[i] = 1; band_point[p] = 1; }
            }
            if (keep) {
                if (e == cap) {
                    cap *= 2;
                    int32_t *nc = (int32_t *)realloc(col, (size_t)cap * sizeof(int32_t));
                    if (!nc) { free(col); free(row_ptr); return -1; }
                    col = nc;
                }
                col[e++] = (int32_t)p;
            }
        }
        row_ptr[r + 1] = e;
    }
    out->n_rows = n_rows;
    out->num_edges = e;
    out->row_ptr = row_ptr;
    out->col = col;
    out->band_pairs = band_pairs;
    return 0;
}

/*
 * Step 2 over the source rows 0..n_rows-1 (n_rows = n: all of them), cut into
 * blocks of `block` consecutive rows that orc_build_rows_metric builds one by
 * one and that are then joined in row order, so the graph equals the
 * one-call result row for row.  Built with
 * OpenMP (-fopenmp) the blocks are shared among the host cores: this is the
 * multi-core timing of the CPU baseline.  Without OpenMP the pragma is
 * ignored and the blocks run in order.  No band points (NULL) are recorded.
 */
int32_t orc_build_rows_blocks(int64_t n, int32_t d, int64_t ld, const float *x, float eps,
                              uint64_t seed, int64_t m, int32_t sample_all, double band_rel,
                              int64_t block, int64_t n_rows, orc_graph *out)
{
    if (n < 2 || block < 1 || n_rows < 1 || n_rows > n || !out) return -1;
    int64_t nb = (n_rows + block - 1) / block;
    orc_graph *part = (orc_graph *)calloc((size_t)nb, sizeof(orc_graph));
    if (!part) return -1;
    int failed = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : failed)
    for (int64_t b = 0; b < nb; ++b) {
        int64_t lo = b * block, hi = lo + block < n_rows ? lo + block : n_rows;
        int64_t *rows = (int64_t *)malloc((size_t)(hi - lo) * sizeof(int64_t));
        if (!rows) { failed |= 1; continue; }
        for (int64_t r = lo; r < hi; ++r) rows[r - lo] = r;
        failed |= orc_build_rows_metric(n, d, ld, x, eps, seed, m, sample_all, band_rel, rows,
                                        hi - lo, &part[b], NULL, NULL, 0) != 0;
        free(rows);
    }
    int64_t e = 0, bp = 0;
    for (int64_t b = 0; b < nb && !failed; ++b) { e += part[b].num_edges; bp += part[b].band_pairs; }
    int64_t *row_ptr = failed ? NULL : (int64_t *)malloc((size_t)(n_rows + 1) * sizeof(int64_t));
    int32_t *col = failed ? NULL : (int32_t *)malloc((size_t)(e > 0 ? e : 1) * sizeof(int32_t));
    if (!row_ptr || !col) failed = 1;
    if (!failed) {
        int64_t at = 0;
        row_ptr[0] = 0;
        for (int64_t b = 0; b < nb; ++b) {
            int64_t lo = b * block;
            for (int64_t r = 0; r < part[b].n_rows; ++r) row_ptr[lo + r + 1] = at + part[b].row_ptr[r + 1];
            if (part[b].num_edges)
                memcpy(col + at, part[b].col, (size_t)part[b].num_edges * sizeof(int32_t));
            at += part[b].num_edges;
        }
    }
    for (int64_t b = 0; b < nb; ++b) orc_graph_free(&part[b]);
    free(part);
    if (failed) { free(row_ptr); free(col); return -1; }
    out->n_rows = n_rows;
    out->num_edges = e;
    out->row_ptr = row_ptr;
    out->col = col;
    out->band_pairs = bp;
    return 0;
}

/* Host threads the blocks above may use (1 without OpenMP). */
#ifdef _OPENMP
#include <omp.h>
#endif
int32_t orc_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------ graph processing */

/* Degree of every vertex of G (Algorithm 1, step 3).  mode 0: undirected
 * multigraph (both ends of every kept draw); 1: out-degree; 2: number of
 * distinct neighbours in either direction. */
int32_t orc_degrees(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t mode,
                    int32_t *deg)
{
    memset(deg, 0, (size_t)n * sizeof(int32_t));
    if (mode == 0 || mode == 1) {
        for (int64_t i = 0; i < n; ++i)
            for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                deg[i] += 1;
                if (mode == 0) deg[col[e]] += 1;
            }
        return 0;
    }
    if (mode != 2) return -1;
    /* simple graph: gather both directions, then count distinct entries */
    int64_t E = row_ptr[n];
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *adj = (int32_t *)malloc((size_t)(2 * E + 1) * sizeof(int32_t));
    int32_t *seen = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!cnt || !adj || !seen) { free(cnt); free(adj); free(seen); return -1; }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            cnt[i + 1]++;
            cnt[col[e] + 1]++;
        }
    for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    int64_t *fill = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!fill) { free(cnt); free(adj); free(seen); return -1; }
    for (int64_t i = 0; i < n; ++i) fill[i] = cnt[i];
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            adj[fill[i]++] = col[e];
            adj[fill[col[e]]++] = (int32_t)i;
        }
    for (int64_t i = 0; i < n; ++i) seen[i] = -1;
    for (int64_t i = 0; i < n; ++i) {
        int32_t c = 0;
        for (int64_t e = cnt[i]; e < cnt[i + 1]; ++e)
            if (seen[adj[e]] != (int32_t)i) { seen[adj[e]] = (int32_t)i; ++c; }
        deg[i] = c;
    }
    free(cnt); free(adj); free(seen); free(fill);
    return 0;
}

/* Undirected adjacency restricted to core-core edges (both directions). */
static int32_t core_adjacency(int64_t n, const int64_t *row_ptr, const int32_t *col,
                              const uint8_t *core, int64_t **a_ptr, int32_t **a_col)
{
    int64_t *ptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!ptr) return -1;
    for (int64_t i = 0; i < n; ++i) {
        if (!core[i]) continue;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t p = col[e];
            if (core[p]) { ptr[i + 1]++; ptr[p + 1]++; }
        }
    }
    for (int64_t i = 0; i < n; ++i) ptr[i + 1] += ptr[i];
    int32_t *adj = (int32_t *)malloc((size_t)(ptr[n] + 1) * sizeof(int32_t));
    int64_t *fill = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    if (!adj || !fill) { free(ptr); free(adj); free(fill); return -1; }
    for (int64_t i = 0; i < n; ++i) fill[i] = ptr[i];
    for (int64_t i = 0; i < n; ++i) {
        if (!core[i]) continue;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t p = col[e];
            if (core[p]) { adj[fill[i]++] = p; adj[fill[p]++] = (int32_t)i; }
        }
    }
    free(fill);
    *a_ptr = ptr;
    *a_col = adj;
    return 0;
}

/*
 * Connected components K_1..K_l of the subgraph induced by core vertices
 * (Algorithm 1, step 3), by breadth-first search started from every unvisited
 * core in increasing index order, so the first vertex reached in a component
 * is its smallest index and becomes its label.  comp[i] = -1 for non-cores.
 * Returns the number of components, or -1 on no memory.
 */
int64_t orc_components_bfs(int64_t n, const int64_t *row_ptr, const int32_t *col,
                           const uint8_t *core, int32_t *comp)
{
    int64_t *aptr;
    int32_t *adj;
    if (core_adjacency(n, row_ptr, col, core, &aptr, &adj)) return -1;
    int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!queue) { free(aptr); free(adj); return -1; }
    for (int64_t i = 0; i < n; ++i) comp[i] = -1;
    int64_t ncomp = 0;
    for (int64_t s = 0; s < n; ++s) {
        if (!core[s] || comp[s] != -1) continue;
        ++ncomp;
        int64_t head = 0, tail = 0;
        queue[tail++] = (int32_t)s;
        comp[s] = (int32_t)s;
        while (head < tail) {
            int32_t u = queue[head++];
            for (int64_t e = aptr[u]; e < aptr[u + 1]; ++e) {
                int32_t v = adj[e];
                if (comp[v] == -1) { comp[v] = (int32_t)s; queue[tail++] = v; }
            }
        }
    }
    free(queue); free(aptr); free(adj);
    return ncomp;
}

static int32_t uf_find(int32_t *parent, int32_t x)
{
    while (parent[x] != x) x = parent[x];
    return x;
}

/*
 * The same components by sequential union-find: for each core-core edge the
 * two roots are joined, the larger root placed under the smaller, so each
 * final root is the smallest index of its component.  Independent of the BFS
 * version; the two must agree.
 */
int64_t orc_components_uf(int64_t n, const int64_t *row_ptr, const int32_t *col,
                          const uint8_t *core, int32_t *comp)
{
    int32_t *parent = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!parent) return -1;
    for (int64_t i = 0; i < n; ++i) parent[i] = (int32_t)i;
    for (int64_t i = 0; i < n; ++i) {
        if (!core[i]) continue;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t p = col[e];
            if (!core[p]) continue;
            int32_t a = uf_find(parent, (int32_t)i), b = uf_find(parent, p);
            if (a == b) continue;
            if (a < b) parent[b] = a; else parent[a] = b;
        }
    }
    int64_t ncomp = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!core[i]) { comp[i] = -1; continue; }
        comp[i] = uf_find(parent, (int32_t)i);
        if (comp[i] == (int32_t)i) ++ncomp;
    }
    free(parent);
    return ncomp;
}

/*
 * Algorithm 1, steps 4-5.  Cores keep their component label.  A non-core
 * point with a kept draw in either direction to some core takes the smallest
 * label among those cores; every other point is noise (-1).
 */
void orc_border_labels(int64_t n, const int64_t *row_ptr, const int32_t *col,
                       const uint8_t *core, const int32_t *comp, int32_t *labels)
{
    const int32_t NONE = 0x7fffffff;
    for (int64_t i = 0; i < n; ++i) labels[i] = core[i] ? comp[i] : NONE;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int32_t p = col[e];
            if (core[i] && !core[p] && comp[i] < labels[p]) labels[p] = comp[i];
            if (!core[i] && core[p] && comp[p] < labels[i]) labels[i] = comp[p];
        }
    for (int64_t i = 0; i < n; ++i)
        if (labels[i] == NONE) labels[i] = -1;
}

/* stats[0..7]: queries, kept, band_pairs, band_points, cores, clusters, noise, 0 */
int32_t orc_cluster_graph_forced(int64_t n, const int64_t *row_ptr, const int32_t *col,
                                 int32_t deg_mode, int32_t min_pts, const uint8_t *forced,
                                 int32_t *labels, uint8_t *core, int32_t *deg, int64_t *stats);

int32_t orc_cluster_graph(int64_t n, const int64_t *row_ptr, const int32_t *col,
                          int32_t deg_mode, int32_t min_pts, int32_t *labels,
                          uint8_t *core, int32_t *deg, int64_t *stats)
{
    return orc_cluster_graph_forced(n, row_ptr, col, deg_mode, min_pts, NULL, labels, core, deg,
                                    stats);
}

int32_t orc_cluster_graph_gated(int64_t n, const int64_t *row_ptr, const int32_t *col,
                                int32_t deg_mode, int32_t min_pts, const uint8_t *forced,
                                const int32_t *w_row, int32_t *labels, uint8_t *core,
                                int32_t *deg, int64_t *stats);

/* Steps 3-5 with an optional per-point override of the core test:
 * forced[i] = 1 makes i core, 2 makes it non-core, 0 leaves deg >= MinPts. */
int32_t orc_cluster_graph_forced(int64_t n, const int64_t *row_ptr, const int32_t *col,
                                 int32_t deg_mode, int32_t min_pts, const uint8_t *forced,
                                 int32_t *labels, uint8_t *core, int32_t *deg, int64_t *stats)
{
    return orc_cluster_graph_gated(n, row_ptr, col, deg_mode, min_pts, forced, NULL, labels,
                                   core, deg, stats);
}

/*
 * Degrees where every kept draw of row i counts w_row[i] (at both ends in
 * multigraph mode, at i only in out-degree mode): the gated form's estimate
 * of the plain degree when point i drew only some of its partners.
 */
static void degrees_weighted(int64_t n, const int64_t *row_ptr, const int32_t *col,
                             int32_t mode, const int32_t *w_row, int32_t *deg)
{
    memset(deg, 0, (size_t)n * sizeof(int32_t));
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            deg[i] += w_row[i];
            if (mode == 0) deg[col[e]] += w_row[i];
        }
}

/* Steps 3-5 of the gated form: forced core flags as above and, if w_row is
 * given, weighted degrees (min_pts is then in the weights' units). */
int32_t orc_cluster_graph_gated(int64_t n, const int64_t *row_ptr, const int32_t *col,
                                int32_t deg_mode, int32_t min_pts, const uint8_t *forced,
                                const int32_t *w_row, int32_t *labels, uint8_t *core,
                                int32_t *deg, int64_t *stats)
{
    int32_t *dg = deg ? deg : (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *comp = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!dg || !comp) { if (!deg) free(dg); free(comp); return -1; }
    if (w_row && (deg_mode == 0 || deg_mode == 1)) {
        degrees_weighted(n, row_ptr, col, deg_mode, w_row, dg);
    } else if (orc_degrees(n, row_ptr, col, deg_mode, dg)) {
        if (!deg) free(dg);
        free(comp);
        return -1;
    }
    int64_t ncores = 0;
    for (int64_t i = 0; i < n; ++i) {
        core[i] = dg[i] >= min_pts ? 1 : 0;
        if (forced && forced[i] == 1) core[i] = 1;
        if (forced && forced[i] == 2) core[i] = 0;
        ncores += core[i];
    }
    int64_t ncomp = orc_components_bfs(n, row_ptr, col, core, comp);
    if (ncomp < 0) { if (!deg) free(dg); free(comp); return -1; }
    orc_border_labels(n, row_ptr, col, core, comp, labels);
    int64_t noise = 0;
    for (int64_t i = 0; i < n; ++i) noise += labels[i] < 0;
    if (stats) {
        stats[1] = row_ptr[n];
        stats[4] = ncores;
        stats[5] = ncomp;
        stats[6] = noise;
    }
    if (!deg) free(dg);
    free(comp);
    return 0;
}

/*
 * The whole of Algorithm 1: graph (step 2), degrees and core mask (step 3),
 * components (step 3), borders and noise (steps 4-5).  labels, core (length n)
 * are outputs; deg may be NULL; band_point (length n) may be NULL.
 */
int32_t orc_cluster_metric(int64_t n, int32_t d, int64_t ld, const float *x, float eps,
                           uint64_t seed, int64_t m, int32_t sample_all, int32_t deg_mode,
                           int32_t min_pts, double band_rel, int32_t *labels, uint8_t *core,
                           int32_t *deg, uint8_t *band_point, int64_t *stats, int32_t metric);

int32_t orc_cluster(int64_t n, int32_t d, int64_t ld, const float *x, float eps,
                    uint64_t seed, int64_t m, int32_t sample_all, int32_t deg_mode,
                    int32_t min_pts, double band_rel, int32_t *labels, uint8_t *core,
                    int32_t *deg, uint8_t *band_point, int64_t *stats)
{
    return orc_cluster_metric(n, d, ld, x, eps, seed, m, sample_all, deg_mode, min_pts,
                              band_rel, labels, core, deg, band_point, stats, 0);
}

/* The whole of Algorithm 1 with the neighbourhood test of `metric` (see
 * orc_build_rows_metric). */
int32_t orc_cluster_metric(int64_t n, int32_t d, int64_t ld, const float *x, float eps,
                           uint64_t seed, int64_t m, int32_t sample_all, int32_t deg_mode,
                           int32_t min_pts, double band_rel, int32_t *labels, uint8_t *core,
                           int32_t *deg, uint8_t *band_point, int64_t *stats, int32_t metric)
{
    orc_graph g;
    uint8_t *bp = band_point ? band_point : (uint8_t *)calloc((size_t)n, 1);
    if (!bp) return -1;
    if (band_point) memset(bp, 0, (size_t)n);
    if (orc_build_rows_metric(n, d, ld, x, eps, seed, m, sample_all, band_rel, NULL, 0, &g, bp,
                              NULL, metric)) {
        if (!band_point) free(bp);
        return -1;
    }
    int32_t rc = orc_cluster_graph(n, g.row_ptr, g.col, deg_mode, min_pts, labels, core, deg,
                                   stats);
    if (stats) {
        int64_t nb = 0;
        for (int64_t i = 0; i < n; ++i) nb += bp[i];
        stats[0] = n * m;
        stats[2] = g.band_pairs;
        stats[3] = nb;
        stats[7] = 0;
    }
    orc_graph_free(&g);
    if (!band_point) free(bp);
    return rc;
}

/* ---------------------------------------------------- textbook DBSCAN */

/*
 * Brute-force DBSCAN (Ester et al. 1996) in the same FP64 arithmetic: the full
 * eps-neighbourhood of every point (the point itself included) from all n^2
 * pairs, cores = neighbourhoods of at least min_pts_db points, clusters =
 * connected components of cores under eps-adjacency, a border point joins the
 * adjacent cluster with the smallest label.  This is the s = 1 limit that the
 * paper describes SNG-DBSCAN as a sampled version of (Section 3).
 */
int32_t orc_dbscan_bruteforce(int64_t n, int32_t d, int64_t ld, const float *x, float eps,
                              int32_t min_pts_db, int32_t *labels, uint8_t *core)
{
    double eps2 = (double)eps * (double)eps;
    uint8_t *nb = (uint8_t *)malloc((size_t)(n * n));
    int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!nb || !queue) { free(nb); free(queue); return -1; }
    for (int64_t i = 0; i < n; ++i) {
        int32_t cnt = 0;
        for (int64_t j = 0; j < n; ++j) {
            nb[i * n + j] = orc_dist2(x + i * ld, x + j * ld, d) <= eps2;
            cnt += nb[i * n + j];
        }
        core[i] = cnt >= min_pts_db;
    }
    for (int64_t i = 0; i < n; ++i) labels[i] = -1;
    for (int64_t s = 0; s < n; ++s) {
        if (!core[s] || labels[s] != -1) continue;
        int64_t head = 0, tail = 0;
        queue[tail++] = (int32_t)s;
        labels[s] = (int32_t)s;
        while (head < tail) {
            int32_t u = queue[head++];
            for (int64_t v = 0; v < n; ++v)
                if (core[v] && labels[v] == -1 && nb[u * n + v]) {
                    labels[v] = (int32_t)s;
                    queue[tail++] = (int32_t)v;
                }
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        if (core[i]) continue;
        int32_t best = -1;
        for (int64_t j = 0; j < n; ++j)
            if (core[j] && nb[i * n + j] && (best < 0 || labels[j] < best)) best = labels[j];
        labels[i] = best;
    }
    free(nb);
    free(queue);
    return 0;
}
