/*
 * gdgen.c -- seeded synthetic graph generators.
 *
 * This file holds no graphlet arithmetic at all: it only turns a seed into an
 * undirected simple graph in sorted int32 CSR (both directions of every edge,
 * neighbour ids ascending, no self-loops, no duplicates).  The paper's
 * experiments drop weights, self-loops and direction from every input graph
 * (Sec. 5) and its problem statement is posed on an undirected simple graph
 * (Sec. 2.1); the generators produce exactly that form.
 *
 * Cross-machine determinism: the same seed must give the same graph on x86-64
 * and aarch64.  All randomness comes from splitmix64 (Steele, Lea, Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014) applied to a
 * counter; floating point uses only + - * / and sqrt, which IEEE 754 rounds
 * correctly everywhere, and the build passes -ffp-contract=off so that no
 * multiply-add is fused on one machine and not on the other.  Logarithms and
 * powers are computed by the series below rather than by libm, whose last-bit
 * results differ between platforms.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------------ */
/* random numbers                                                           */
/* ------------------------------------------------------------------------ */

typedef struct { uint64_t state; } rng_t;

static uint64_t splitmix64_next(rng_t *r) {
    uint64_t z = (r->state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static rng_t rng_make(uint64_t seed, uint64_t stream) {
    rng_t r;
    r.state = seed * 0xD1B54A32D192ED03ULL + stream * 0x8CB92BA72F3D8DD7ULL + 0x2545F4914F6CDD1DULL;
    (void)splitmix64_next(&r);
    return r;
}

/* uniform double in [0,1) with 53 random bits */
static double rng_unit(rng_t *r) {
    return (double)(splitmix64_next(r) >> 11) * (1.0 / 9007199254740992.0);
}

/* uniform integer in [0, bound) (bound > 0), multiply-shift without bias fix:
 * the bias is below 2^-32 for every bound used here. */
static uint64_t rng_below(rng_t *r, uint64_t bound) {
    unsigned __int128 p = (unsigned __int128)splitmix64_next(r) * bound;
    return (uint64_t)(p >> 64);
}

/* ------------------------------------------------------------------------ */
/* portable log / exp (argument reduction + series, no libm transcendental) */
/* ------------------------------------------------------------------------ */

static const double LN2 = 0.69314718055994530942;

/* natural log for x > 0 */
static double plog(double x) {
    int k;
    double m = frexp(x, &k);          /* x = m * 2^k, m in [0.5,1): exact */
    if (m < 0.70710678118654752440) { m *= 2.0; k -= 1; }   /* m in [0.707,1.414) */
    double s = (m - 1.0) / (m + 1.0); /* |s| < 0.1716 */
    double s2 = s * s, term = s, sum = 0.0;
    for (int i = 1; i < 60; i += 2) { sum += term / (double)i; term *= s2; }
    return 2.0 * sum + (double)k * LN2;
}

/* e^y for moderate y */
static double pexp(double y) {
    double t = y / LN2;
    double kf = floor(t);
    double f = (t - kf) * LN2;        /* f in [0, ln2) */
    double term = 1.0, sum = 1.0;
    for (int i = 1; i < 30; i++) { term *= f / (double)i; sum += term; }
    return ldexp(sum, (int)kf);
}

static double ppow(double x, double e) { return pexp(e * plog(x)); }

/* ------------------------------------------------------------------------ */
/* CSR assembly from an edge-pair list                                      */
/* ------------------------------------------------------------------------ */

typedef struct gdgen_graph {
    int32_t n;
    int64_t nnz;
    int32_t *row_ptr;   /* n+1 */
    int32_t *col_idx;   /* nnz */
} gdgen_graph;

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static void sort_row(int32_t *a, int64_t len) {
    if (len < 32) {
        for (int64_t i = 1; i < len; i++) {
            int32_t v = a[i]; int64_t j = i - 1;
            while (j >= 0 && a[j] > v) { a[j + 1] = a[j]; j--; }
            a[j + 1] = v;
        }
    } else {
        qsort(a, (size_t)len, sizeof(int32_t), cmp_i32);
    }
}

/* Build a simple undirected CSR from `cnt` pairs (src[i], dst[i]); self-loops
 * are dropped, both directions added, duplicates removed. */
static gdgen_graph *csr_from_pairs(int32_t n, int64_t cnt, const int32_t *src, const int32_t *dst) {
    gdgen_graph *g = (gdgen_graph *)calloc(1, sizeof(gdgen_graph));
    if (!g) return NULL;
    g->n = n;
    int64_t *deg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!deg) { free(g); return NULL; }
    for (int64_t i = 0; i < cnt; i++) {
        if (src[i] == dst[i]) continue;
        deg[src[i]]++; deg[dst[i]]++;
    }
    int64_t *off = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!off) { free(deg); free(g); return NULL; }
    off[0] = 0;
    for (int32_t v = 0; v < n; v++) off[v + 1] = off[v] + deg[v];
    int64_t total = off[n];
    int32_t *tmp = (int32_t *)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
    if (!tmp) { free(off); free(deg); free(g); return NULL; }
    for (int32_t v = 0; v < n; v++) deg[v] = off[v];
    for (int64_t i = 0; i < cnt; i++) {
        int32_t a = src[i], b = dst[i];
        if (a == b) continue;
        tmp[deg[a]++] = b;
        tmp[deg[b]++] = a;
    }
    /* sort + dedup in place, compacting */
    int64_t w = 0;
    int32_t *rp = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    if (!rp) { free(tmp); free(off); free(deg); free(g); return NULL; }
    for (int32_t v = 0; v < n; v++) {
        int64_t b = off[v], e = off[v + 1];
        sort_row(tmp + b, e - b);
        rp[v] = (int32_t)w;
        for (int64_t i = b; i < e; i++) {
            if (i > b && tmp[i] == tmp[i - 1]) continue;
            tmp[w++] = tmp[i];
        }
    }
    rp[n] = (int32_t)w;
    g->row_ptr = rp;
    g->nnz = w;
    g->col_idx = (int32_t *)realloc(tmp, (size_t)(w > 0 ? w : 1) * sizeof(int32_t));
    if (!g->col_idx) g->col_idx = tmp;
    free(off); free(deg);
    return g;
}

/* ------------------------------------------------------------------------ */
/* public API                                                               */
/* ------------------------------------------------------------------------ */

int32_t gdgen_n(const gdgen_graph *g) { return g ? g->n : -1; }
int64_t gdgen_nnz(const gdgen_graph *g) { return g ? g->nnz : -1; }

void gdgen_copy(const gdgen_graph *g, int32_t *row_ptr, int32_t *col_idx) {
    memcpy(row_ptr, g->row_ptr, ((size_t)g->n + 1) * sizeof(int32_t));
    if (g->nnz > 0) memcpy(col_idx, g->col_idx, (size_t)g->nnz * sizeof(int32_t));
}

void gdgen_free(gdgen_graph *g) {
    if (!g) return;
    free(g->row_ptr); free(g->col_idx); free(g);
}

/* G(n, p): every pair i < j is an edge independently with probability p.
 * Pairs are visited in row-major order of the strict upper triangle and the
 * gaps between successive edges are drawn from the geometric distribution
 * (skip = floor(log(U) / log(1-p))), which gives exactly the Bernoulli law. */
gdgen_graph *gdgen_erdos_renyi(int32_t n, double p, uint64_t seed) {
    if (n < 0) return NULL;
    rng_t r = rng_make(seed, 1);
    int64_t cap = 1024, cnt = 0;
    int32_t *src = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    int32_t *dst = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    if (!src || !dst) { free(src); free(dst); return NULL; }
    if (p > 0.0 && n > 1) {
        const int64_t total = (int64_t)n * (n - 1) / 2;
        const double lq = (p < 1.0) ? plog(1.0 - p) : 0.0;
        int64_t pos = -1;                  /* linear index into the pair list */
        int32_t row = 0; int64_t row_start = 0;   /* first linear index of `row` */
        for (;;) {
            int64_t skip;
            if (p >= 1.0) skip = 0;
            else {
                double u = 1.0 - rng_unit(&r);     /* (0,1] */
                double s = plog(u) / lq;
                skip = (s >= 9.0e18) ? total : (int64_t)s;
            }
            if (skip >= total - pos) break;
            pos += skip + 1;
            if (pos >= total) break;
            while (pos >= row_start + (n - 1 - row)) { row_start += n - 1 - row; row++; }
            int32_t col = (int32_t)(row + 1 + (pos - row_start));
            if (cnt == cap) {
                cap *= 2;
                int32_t *s2 = (int32_t *)realloc(src, (size_t)cap * sizeof(int32_t));
                int32_t *d2 = (int32_t *)realloc(dst, (size_t)cap * sizeof(int32_t));
                if (!s2 || !d2) { free(s2 ? s2 : src); free(d2 ? d2 : dst); return NULL; }
                src = s2; dst = d2;
            }
            src[cnt] = row; dst[cnt] = col; cnt++;
        }
    }
    gdgen_graph *g = csr_from_pairs(n, cnt, src, dst);
    free(src); free(dst);
    return g;
}

/* Chung-Lu: node weights w_i are Pareto with density exponent gamma
 * (P(x) ~ x^-gamma, x >= 1), rescaled so that sum w = 2 * draws (w_i is then
 * the expected degree before duplicates are removed), capped at `cap`; then
 * `draws` endpoint pairs are sampled i.i.d. with P(i) ~ w_i by inverse CDF on
 * the prefix sums; self-loops and duplicates are dropped.  cap <= 0 selects
 * the cap sqrt(sum w) (the Chung-Lu validity bound). */
gdgen_graph *gdgen_chung_lu(int32_t n, double gamma, int64_t draws, double cap, uint64_t seed) {
    if (n <= 0 || draws < 0 || !(gamma > 1.0)) return NULL;
    rng_t r = rng_make(seed, 2);
    double *w = (double *)malloc((size_t)n * sizeof(double));
    double *cdf = (double *)malloc(((size_t)n + 1) * sizeof(double));
    int32_t *src = (int32_t *)malloc((size_t)(draws > 0 ? draws : 1) * sizeof(int32_t));
    int32_t *dst = (int32_t *)malloc((size_t)(draws > 0 ? draws : 1) * sizeof(int32_t));
    if (!w || !cdf || !src || !dst) { free(w); free(cdf); free(src); free(dst); return NULL; }
    const double ex = -1.0 / (gamma - 1.0);
    double sum = 0.0;
    for (int32_t i = 0; i < n; i++) {
        double u = 1.0 - rng_unit(&r);     /* (0,1] */
        w[i] = ppow(u, ex);
        sum += w[i];
    }
    const double scale = (draws > 0) ? (2.0 * (double)draws) / sum : 1.0;
    double ssum = 0.0;
    for (int32_t i = 0; i < n; i++) { w[i] *= scale; ssum += w[i]; }
    if (cap <= 0.0) cap = sqrt(ssum);
    cdf[0] = 0.0;
    for (int32_t i = 0; i < n; i++) {
        double wi = w[i] > cap ? cap : w[i];
        cdf[i + 1] = cdf[i] + wi;
    }
    const double tot = cdf[n];
    for (int64_t k = 0; k < 2 * draws; k++) {
        double x = rng_unit(&r) * tot;
        /* largest i with cdf[i] <= x */
        int32_t lo = 0, hi = n;      /* invariant cdf[lo] <= x < cdf[hi] */
        while (hi - lo > 1) {
            int32_t mid = lo + (hi - lo) / 2;
            if (cdf[mid] <= x) lo = mid; else hi = mid;
        }
        if (k & 1) dst[k >> 1] = lo; else src[k >> 1] = lo;
    }
    gdgen_graph *g = csr_from_pairs(n, draws, src, dst);
    free(w); free(cdf); free(src); free(dst);
    return g;
}

/* R-MAT (Chakrabarti, Zhan, Faloutsos 2004) on 2^scale nodes: each sample
 * descends `scale` levels choosing quadrant a/b/c/d with the given
 * probabilities (no noise).  With relabel != 0 the node ids are passed through
 * a seeded uniform random permutation (Graph500 practice). */
gdgen_graph *gdgen_rmat(int scale, int64_t samples, double a, double b, double c,
                        uint64_t seed, int relabel) {
    if (scale < 1 || scale > 30 || samples < 0) return NULL;
    const int32_t n = (int32_t)1 << scale;
    rng_t r = rng_make(seed, 3);
    const uint64_t ta = (uint64_t)(a * 9007199254740992.0);
    const uint64_t tb = (uint64_t)((a + b) * 9007199254740992.0);
    const uint64_t tc = (uint64_t)((a + b + c) * 9007199254740992.0);
    int32_t *src = (int32_t *)malloc((size_t)(samples > 0 ? samples : 1) * sizeof(int32_t));
    int32_t *dst = (int32_t *)malloc((size_t)(samples > 0 ? samples : 1) * sizeof(int32_t));
    int32_t *perm = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!src || !dst || !perm) { free(src); free(dst); free(perm); return NULL; }
    for (int64_t k = 0; k < samples; k++) {
        uint32_t i = 0, j = 0;
        for (int l = 0; l < scale; l++) {
            uint64_t x = splitmix64_next(&r) >> 11;
            i <<= 1; j <<= 1;
            if (x < ta) { }
            else if (x < tb) { j |= 1; }
            else if (x < tc) { i |= 1; }
            else { i |= 1; j |= 1; }
        }
        src[k] = (int32_t)i; dst[k] = (int32_t)j;
    }
    for (int32_t v = 0; v < n; v++) perm[v] = v;
    if (relabel) {
        rng_t pr = rng_make(seed, 33);
        for (int32_t v = n - 1; v > 0; v--) {
            int32_t s = (int32_t)rng_below(&pr, (uint64_t)v + 1);
            int32_t t = perm[v]; perm[v] = perm[s]; perm[s] = t;
        }
        for (int64_t k = 0; k < samples; k++) { src[k] = perm[src[k]]; dst[k] = perm[dst[k]]; }
    }
    gdgen_graph *g = csr_from_pairs(n, samples, src, dst);
    free(src); free(dst); free(perm);
    return g;
}

/* Barabasi-Albert preferential attachment: start from the clique on m+1
 * nodes; each later node attaches to m distinct earlier nodes, each chosen
 * with probability proportional to its current degree (uniform pick from the
 * list of edge endpoints, repeated until m distinct targets are found). */
gdgen_graph *gdgen_barabasi_albert(int32_t n, int32_t m, uint64_t seed) {
    if (n < 0 || m < 1) return NULL;
    rng_t r = rng_make(seed, 4);
    int32_t k0 = (m + 1 < n) ? m + 1 : n;
    int64_t max_e = (int64_t)k0 * (k0 - 1) / 2 + (int64_t)(n > k0 ? n - k0 : 0) * m;
    int32_t *src = (int32_t *)malloc((size_t)(max_e > 0 ? max_e : 1) * sizeof(int32_t));
    int32_t *dst = (int32_t *)malloc((size_t)(max_e > 0 ? max_e : 1) * sizeof(int32_t));
    int32_t *ends = (int32_t *)malloc((size_t)(2 * max_e > 0 ? 2 * max_e : 1) * sizeof(int32_t));
    int32_t *pick = (int32_t *)malloc((size_t)m * sizeof(int32_t));
    if (!src || !dst || !ends || !pick) { free(src); free(dst); free(ends); free(pick); return NULL; }
    int64_t cnt = 0, ne = 0;
    for (int32_t i = 0; i < k0; i++)
        for (int32_t j = i + 1; j < k0; j++) {
            src[cnt] = i; dst[cnt] = j; cnt++;
            ends[ne++] = i; ends[ne++] = j;
        }
    for (int32_t v = k0; v < n; v++) {
        int32_t got = 0;
        while (got < m) {
            int32_t t = ends[rng_below(&r, (uint64_t)ne)];
            int dup = 0;
            for (int32_t q = 0; q < got; q++) if (pick[q] == t) { dup = 1; break; }
            if (!dup) pick[got++] = t;
        }
        for (int32_t q = 0; q < m; q++) {
            src[cnt] = v; dst[cnt] = pick[q]; cnt++;
            ends[ne++] = v; ends[ne++] = pick[q];
        }
    }
    gdgen_graph *g = csr_from_pairs(n, cnt, src, dst);
    free(src); free(dst); free(ends); free(pick);
    return g;
}

/* A graph from an explicit pair list (used for hand-built test graphs). */
gdgen_graph *gdgen_from_pairs(int32_t n, int64_t cnt, const int32_t *src, const int32_t *dst) {
    for (int64_t i = 0; i < cnt; i++)
        if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n) return NULL;
    return csr_from_pairs(n, cnt, src, dst);
}

/* Seeded draws used by the batch and request-trace recipes, exposed so that
 * the Python side draws its per-graph parameters from the same generator:
 * out[i] = uniform double in [0,1) for i < count, stream `stream`. */
void gdgen_uniforms(uint64_t seed, uint64_t stream, int64_t count, double *out) {
    rng_t r = rng_make(seed, stream);
    for (int64_t i = 0; i < count; i++) out[i] = rng_unit(&r);
}

/* Portable exp/log for recipe parameters (log-uniform sizes). */
double gdgen_log(double x) { return plog(x); }
double gdgen_exp(double x) { return pexp(x); }
