/*
 * gd_oracle.c -- CPU oracle for exact 3- and 4-node graphlet counts.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The CUDA library never
 * links, includes or calls anything here, and this file includes nothing of it.
 *
 * Paper: N. K. Ahmed, J. Neville, R. A. Rossi, N. Duffield, T. L. Willke,
 * "Graphlet Decomposition: Framework, Algorithms, and Applications" (2015).
 *
 * Input: undirected simple graph, int32 CSR, both directions stored, each row
 * sorted ascending (Sec. 2.1 problem statement; Sec. 5 drops weights,
 * self-loops and direction).  n counts every row, isolated nodes included.
 *
 * Output order of the 15 counts (Table 1 numbering):
 *   [g31 g32 g33 g34 g41 g42 g43 g44 g45 g46 g47 g48 g49 g4_10 g4_11]
 * Global counts are exact unsigned 128-bit integers, returned as (lo, hi)
 * u64 pairs; per-edge counts are u64.  Per-edge rows follow CSR order of the
 * undirected edges (u, v) with u < v.
 *
 * Two methods live here:
 *
 *  O1 "literal": Algorithm 2 (GraphletCounting) -- Step 1 marks N(u) and N(v)
 *     in a marker array X with values 1/2/3, CliqueCount and CycleCount scan
 *     the neighbourhoods of Tri_e and Star_u, Step 3 adds the unrestricted
 *     counts, Step 4 applies the Lemmas (Sec. 4.3) and Eqs. for g49 / g4_11.
 *     Single thread.  Algorithm 1 (TriadCensus) is here as well.  The
 *     per-edge O1 record counts every restricted count N^(e)_{a,b,1} of
 *     Sec. 4.2 straight from its definition (class of w, class of r, edge wr)
 *     and evaluates Corollaries 1-14 per edge.
 *
 *  O2 "independent": a different algorithm for graphs too large for O1's
 *     CycleCount.  Triangles per edge by marking the larger endpoint's list;
 *     4-cliques by enumerating each one once under a degree ordering and
 *     crediting its six edges; 4-cycles through an edge from 2-hop codegree
 *     counts around one endpoint; the restricted counts per edge from the
 *     identities below (each checked against brute force in the tests):
 *       A_u = sum_{w in Tri} T(u,w)       N_TSu1  = A_u - T - 2 cliq
 *       t(u) = edges inside N(u)          N_SuSu1 = t(u) - T - cliq - N_TSu1
 *       D_T = sum_{w in Tri} d(w)         N_TI1   = D_T - 2T - 2 cliq - N_TS1
 *       S1(u) = sum_{x in N(u)} d(x)
 *       N_SuI1 = (S1(u) - d(v) - D_T - Su) - N_TSu1 - 2 N_SuSu1 - cyc
 *       C4(e) = sum_{y in N(v)\{u}} (codeg(u,y) - 1)   (4-cycles through e)
 *       cyc   = C4(e) - N_TS1 - 2 cliq
 *     OpenMP threads, per-edge counters updated with relaxed atomics.
 *
 * Readings where the paper is silent (each listed in the design notes):
 *  - each undirected edge is visited once, as (u, v) with u < v (Alg. 2 runs
 *    "for e in E"; the 1/3, 1/2, 1/6 divisors need one visit per edge);
 *  - one marker array per worker; O1 is single-threaded so there is one X;
 *  - |V| is the CSR row count, isolated nodes included;
 *  - every entry of X that a step sets is cleared before the next edge;
 *  - counts are exact: u64 per edge, u128 for sums and completion; every
 *    division is exact and a remainder or an underflow is reported as an
 *    error (ORACLE_EARITH) instead of being wrapped.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

enum { ORACLE_OK = 0, ORACLE_EINVAL = 1, ORACLE_ENOMEM = 2, ORACLE_EARITH = 3 };

/* per-edge raw record layout (u64 each) */
enum {
    R_T = 0, R_SU, R_SV, R_I, R_CLIQ, R_CYC,
    R_TSU1, R_TSV1, R_SUSU1, R_SVSV1, R_TI1, R_SUI1, R_SVI1, R_II1,
    R_NUM
};

/* ------------------------------------------------------------------------ */
/* exact helpers                                                            */
/* ------------------------------------------------------------------------ */

static u128 choose2(u128 x) { return x < 2 ? 0 : (x * (x - 1)) / 2; }
static u128 choose3(u128 x) { return x < 3 ? 0 : (x * (x - 1) / 2) * (x - 2) / 3; }
static u128 choose4(u128 x) { return x < 4 ? 0 : ((x * (x - 1) / 2) * (x - 2) / 3) * (x - 3) / 4; }

static int sub_ok(u128 a, u128 b, u128 *r) { if (b > a) return 0; *r = a - b; return 1; }
static int div_ok(u128 a, u128 d, u128 *r) { if (a % d) return 0; *r = a / d; return 1; }

static void put128(uint64_t *out, int i, u128 x) {
    out[2 * i] = (uint64_t)x;
    out[2 * i + 1] = (uint64_t)(x >> 64);
}

/* Edge-summed quantities of Alg. 2 (Step 1-3 accumulators). */
typedef struct {
    u128 sT;      /* sum |Tri_e|                                Eq. triangle   */
    u128 sS;      /* sum |Star_u| + |Star_v|                    Eq. 2-star     */
    u128 sI;      /* sum |V| - |N(u) u N(v)|                    Eq. g3_3       */
    u128 sCliq;   /* sum CliqueCount = sum N_TT1                Cor. 1         */
    u128 sCyc;    /* sum CycleCount  = sum N_SuSv1              Cor. 3         */
    u128 nTT;     /* sum C(T,2)                                 Eq. comb       */
    u128 nSuSv;   /* sum Su*Sv                                                 */
    u128 nTS;     /* sum T*(Su+Sv)                                             */
    u128 nSS;     /* sum C(Su,2)+C(Sv,2)                                       */
    u128 nTI;     /* sum T*I                                                   */
    u128 nSI;     /* sum (Su+Sv)*I                                             */
    u128 nII;     /* sum C(I,2)                                                */
    u128 nII1;    /* sum |E| - (du-1) - (dv-1) - 1                 L. g4_9 */
} sums_t;

/* Step 4: Lemmas of Sec. 4.3, Eq. g4_9 and Eq. g4_11.  f[0..14] in Table 1
 * order.  Returns 0 on success, ORACLE_EARITH on a remainder/underflow. */
static int complete_counts(const sums_t *s, u128 n, u128 f[15]) {
    u128 t;
    /* k = 3 (Alg. 1) */
    if (!div_ok(s->sT, 3, &f[0])) return ORACLE_EARITH;          /* g31 */
    if (!div_ok(s->sS, 2, &f[1])) return ORACLE_EARITH;          /* g32 */
    f[2] = s->sI;                                                /* g33 */
    if (!sub_ok(choose3(n), f[0] + f[1] + f[2], &f[3])) return ORACLE_EARITH;  /* g34 */
    /* k = 4 */
    u128 f41, f42, f43, f44, f45, f46, f47, f48, f49, f410, f411;
    if (!div_ok(s->sCliq, 6, &f41)) return ORACLE_EARITH;        /* Lemma 1: each 4-clique on 6 edges */
    if (!div_ok(s->sCyc, 4, &f44)) return ORACLE_EARITH;         /* Lemma 2: each 4-cycle on 4 edges */
    if (!sub_ok(s->nTT, 6 * f41, &f42)) return ORACLE_EARITH;    /* Lemma 1 */
    if (!sub_ok(s->nSuSv, 4 * f44, &f46)) return ORACLE_EARITH;  /* Lemma 2 */
    if (!sub_ok(s->nTS, 4 * f42, &t) || !div_ok(t, 2, &f43)) return ORACLE_EARITH;   /* Lemma 3 */
    if (!sub_ok(s->nSS, f43, &t) || !div_ok(t, 3, &f45)) return ORACLE_EARITH;       /* Lemma 4 */
    if (!sub_ok(s->nTI, f43, &t) || !div_ok(t, 3, &f47)) return ORACLE_EARITH;       /* Lemma 5 */
    if (!sub_ok(s->nSI, 2 * f46, &t) || !div_ok(t, 2, &f48)) return ORACLE_EARITH;   /* Lemma 6 */
    if (!sub_ok(s->nII1, 6 * f41 + 4 * f42 + 2 * f43 + 4 * f44 + 2 * f46, &t)
        || !div_ok(t, 2, &f49)) return ORACLE_EARITH;                                 /* Eq. g4_9 */
    if (!sub_ok(s->nII, 2 * f49, &f410)) return ORACLE_EARITH;  /* Lemma 7 */
    if (!sub_ok(choose4(n), f41 + f42 + f43 + f44 + f45 + f46 + f47 + f48 + f49 + f410, &f411))
        return ORACLE_EARITH;                                    /* Eq. g4_11 */
    f[4] = f41; f[5] = f42; f[6] = f43; f[7] = f44; f[8] = f45; f[9] = f46;
    f[10] = f47; f[11] = f48; f[12] = f49; f[13] = f410; f[14] = f411;
    return ORACLE_OK;
}

/* Per-edge columns from a raw record: Corollaries 1-14 evaluated per edge. */
static int edge_columns(const uint64_t *r, uint64_t *c) {
    u128 T = r[R_T], Su = r[R_SU], Sv = r[R_SV], I = r[R_I];
    u128 cliq = r[R_CLIQ], cyc = r[R_CYC];
    u128 TS1 = (u128)r[R_TSU1] + r[R_TSV1];
    u128 SS1 = (u128)r[R_SUSU1] + r[R_SVSV1];
    u128 SI1 = (u128)r[R_SUI1] + r[R_SVI1];
    u128 TI1 = r[R_TI1], II1 = r[R_II1];
    u128 x;
    c[0] = (uint64_t)T;
    c[1] = (uint64_t)(Su + Sv);
    c[2] = (uint64_t)I;
    c[3] = 0;
    c[4] = (uint64_t)cliq;                                           /* Cor. 1          */
    if (!sub_ok(choose2(T), cliq, &x)) return ORACLE_EARITH;         /* Cor. 2 + Cor. 6 */
    c[5] = (uint64_t)(x + TS1);
    if (!sub_ok(T * (Su + Sv), TS1, &x)) return ORACLE_EARITH;       /* Cor. 5, 7, 10   */
    c[6] = (uint64_t)(x + TI1 + SS1);
    c[7] = (uint64_t)cyc;                                            /* Cor. 3          */
    if (!sub_ok(choose2(Su) + choose2(Sv), SS1, &x)) return ORACLE_EARITH;  /* Cor. 8   */
    c[8] = (uint64_t)x;
    if (!sub_ok(Su * Sv, cyc, &x)) return ORACLE_EARITH;             /* Cor. 4 + Cor. 11 */
    c[9] = (uint64_t)(x + SI1);
    if (!sub_ok(T * I, TI1, &x)) return ORACLE_EARITH;               /* Cor. 9          */
    c[10] = (uint64_t)x;
    if (!sub_ok((Su + Sv) * I, SI1, &x)) return ORACLE_EARITH;       /* Cor. 12         */
    c[11] = (uint64_t)x;
    c[12] = (uint64_t)II1;                                           /* Cor. 13         */
    if (!sub_ok(choose2(I), II1, &x)) return ORACLE_EARITH;          /* Cor. 14         */
    c[13] = (uint64_t)x;
    c[14] = 0;
    return ORACLE_OK;
}

/* Basic CSR sanity (the oracle trusts nothing it is handed). */
static int check_csr(int32_t n, const int32_t *rp, const int32_t *ci) {
    if (n < 0 || !rp) return ORACLE_EINVAL;
    if (rp[0] != 0) return ORACLE_EINVAL;
    for (int32_t u = 0; u < n; u++) {
        if (rp[u + 1] < rp[u]) return ORACLE_EINVAL;
        for (int32_t p = rp[u]; p < rp[u + 1]; p++) {
            if (ci[p] < 0 || ci[p] >= n || ci[p] == u) return ORACLE_EINVAL;
            if (p > rp[u] && ci[p] <= ci[p - 1]) return ORACLE_EINVAL;
        }
    }
    return ORACLE_OK;
}

/* ======================================================================== */
/* O1: Algorithm 1 (TriadCensus) and Algorithm 2 (GraphletCounting)        */
/* ======================================================================== */

/* Algorithm 1: all 3-node graphlet counts. out: 4 x (lo,hi). */
int oracle_triad_census(int32_t n, const int32_t *rp, const int32_t *ci, uint64_t *out) {
    int rc = check_csr(n, rp, ci);
    if (rc) return rc;
    uint8_t *X = (uint8_t *)calloc((size_t)n + 1, 1);
    if (!X) return ORACLE_ENOMEM;
    u128 f31 = 0, f32 = 0, f33 = 0;
    for (int32_t u = 0; u < n; u++) {
        for (int32_t p = rp[u]; p < rp[u + 1]; p++) {
            int32_t v = ci[p];
            if (v <= u) continue;                 /* each undirected edge once */
            int64_t star_u = 0, star_v = 0, tri = 0;
            for (int32_t q = rp[u]; q < rp[u + 1]; q++) {
                int32_t w = ci[q];
                if (w == v) continue;
                star_u++; X[w] = 1;
            }
            for (int32_t q = rp[v]; q < rp[v + 1]; q++) {
                int32_t w = ci[q];
                if (w == u) continue;
                if (X[w] == 1) { tri++; star_u--; }   /* found triangle */
                else star_v++;
            }
            f31 += (u128)tri;
            f32 += (u128)(star_u + star_v);
            f33 += (u128)n - (u128)(tri + star_u + star_v + 2);   /* |N(u) u N(v)| = T + S + 2 */
            for (int32_t q = rp[u]; q < rp[u + 1]; q++) X[ci[q]] = 0;
        }
    }
    free(X);
    u128 f[4];
    if (f31 % 3 || f32 % 2) return ORACLE_EARITH;
    f[0] = f31 / 3; f[1] = f32 / 2; f[2] = f33;
    if (!sub_ok(choose3((u128)n), f[0] + f[1] + f[2], &f[3])) return ORACLE_EARITH;
    for (int i = 0; i < 4; i++) put128(out, i, f[i]);
    return ORACLE_OK;
}

/* Algorithm 2, literal.  out: 15 x (lo,hi); sums_out (nullable): 13 x (lo,hi)
 * in the field order of sums_t. */
int oracle_alg2_global(int32_t n, const int32_t *rp, const int32_t *ci,
                       uint64_t *out, uint64_t *sums_out) {
    int rc = check_csr(n, rp, ci);
    if (rc) return rc;
    const int64_t m = (int64_t)rp[n] / 2;
    uint8_t *X = (uint8_t *)calloc((size_t)n + 1, 1);
    int32_t *tri = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    int32_t *staru = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    if (!X || !tri || !staru) { free(X); free(tri); free(staru); return ORACLE_ENOMEM; }
    sums_t s;
    memset(&s, 0, sizeof(s));
    for (int32_t u = 0; u < n; u++) {
        for (int32_t p = rp[u]; p < rp[u + 1]; p++) {
            int32_t v = ci[p];
            if (v <= u) continue;
            /* Step 1: Star_u <- N(u)\{v} with X=1; scan N(v): X=1 -> Tri (X=2),
             * else Star_v (X=3). */
            int64_t nsu = 0, nt = 0, nsv = 0;
            for (int32_t q = rp[u]; q < rp[u + 1]; q++) {
                int32_t w = ci[q];
                if (w == v) continue;
                staru[nsu++] = w; X[w] = 1;
            }
            for (int32_t q = rp[v]; q < rp[v + 1]; q++) {
                int32_t w = ci[q];
                if (w == u) continue;
                if (X[w] == 1) { tri[nt++] = w; X[w] = 2; }
                else { nsv++; X[w] = 3; }
            }
            /* remove Tri members from Star_u */
            int64_t k = 0;
            for (int64_t i = 0; i < nsu; i++) if (X[staru[i]] == 1) staru[k++] = staru[i];
            nsu = k;
            const u128 T = (u128)nt, Su = (u128)nsu, Sv = (u128)nsv;
            const u128 I = (u128)n - (T + Su + Sv + 2);
            /* f3 updates (Alg. 1 lines for g31, g32, g33) */
            s.sT += T; s.sS += Su + Sv; s.sI += I;
            /* Step 2: CliqueCount(X, Tri_e) */
            u128 cliq = 0;
            for (int64_t i = 0; i < nt; i++) {
                int32_t w = tri[i];
                for (int32_t q = rp[w]; q < rp[w + 1]; q++) if (X[ci[q]] == 2) cliq++;
                X[w] = 0;
            }
            /* Step 2: CycleCount(X, Star_u) */
            u128 cyc = 0;
            for (int64_t i = 0; i < nsu; i++) {
                int32_t w = staru[i];
                for (int32_t q = rp[w]; q < rp[w + 1]; q++) if (X[ci[q]] == 3) cyc++;
                X[w] = 0;
            }
            s.sCliq += cliq; s.sCyc += cyc;
            /* Step 3: unrestricted counts */
            s.nTT += choose2(T);
            s.nSuSv += Su * Sv;
            s.nTS += T * (Su + Sv);
            s.nSS += choose2(Su) + choose2(Sv);
            s.nTI += T * I;
            s.nSI += Su * I + Sv * I;
            s.nII += choose2(I);
            s.nII1 += (u128)m - (u128)(rp[u + 1] - rp[u] - 1) - (u128)(rp[v + 1] - rp[v] - 1) - 1;
            /* reset every entry of X set for this edge */
            for (int32_t q = rp[v]; q < rp[v + 1]; q++) X[ci[q]] = 0;
            for (int32_t q = rp[u]; q < rp[u + 1]; q++) X[ci[q]] = 0;
        }
    }
    free(X); free(tri); free(staru);
    u128 f[15];
    rc = complete_counts(&s, (u128)n, f);
    if (sums_out) {
        const u128 *sv = (const u128 *)&s;
        for (int i = 0; i < 13; i++) put128(sums_out, i, sv[i]);
    }
    if (rc) return rc;
    for (int i = 0; i < 15; i++) put128(out, i, f[i]);
    return ORACLE_OK;
}

/* O1 per-edge record for one edge (u, v): every restricted count straight
 * from its definition.  cls[] must be all zero on entry and is left so. */
static int edge_record_direct(int32_t n, const int32_t *rp, const int32_t *ci, int64_t m,
                              int32_t u, int32_t v, uint8_t *cls, int32_t *list, uint64_t *rec) {
    /* node classes w.r.t. e: 1 = S_u, 2 = T, 3 = S_v, 4 = endpoint, 0 = I */
    enum { CI = 0, CSU = 1, CT = 2, CSV = 3, CEND = 4 };
    int64_t len = 0;
    for (int32_t q = rp[u]; q < rp[u + 1]; q++) {
        int32_t w = ci[q];
        if (w == v) continue;
        cls[w] = CSU; list[len++] = w;
    }
    for (int32_t q = rp[v]; q < rp[v + 1]; q++) {
        int32_t w = ci[q];
        if (w == u) continue;
        if (cls[w] == CSU) cls[w] = CT;
        else { cls[w] = CSV; list[len++] = w; }
    }
    cls[u] = CEND; cls[v] = CEND;
    uint64_t cnt[4] = {0, 0, 0, 0};
    for (int64_t i = 0; i < len; i++) cnt[cls[list[i]]]++;
    /* ordered counts of edges (w, r), w in the egonet, r not an endpoint */
    uint64_t M[4][4];
    memset(M, 0, sizeof(M));
    for (int64_t i = 0; i < len; i++) {
        int32_t w = list[i];
        for (int32_t q = rp[w]; q < rp[w + 1]; q++) {
            int32_t r = ci[q];
            if (cls[r] == CEND) continue;
            M[cls[w]][cls[r]]++;
        }
    }
    /* N_{a,b,1}: an edge between two egonet classes a != b appears once in
     * M[a][b] and once in M[b][a]; within one class it appears twice in M[a][a];
     * an edge from the egonet to I appears once, in M[a][I]. */
    const uint64_t T = cnt[CT], Su = cnt[CSU], Sv = cnt[CSV];
    const uint64_t I = (uint64_t)n - T - Su - Sv - 2;
    rec[R_T] = T; rec[R_SU] = Su; rec[R_SV] = Sv; rec[R_I] = I;
    rec[R_CLIQ] = M[CT][CT] / 2;
    rec[R_CYC] = M[CSU][CSV];
    rec[R_TSU1] = M[CT][CSU];
    rec[R_TSV1] = M[CT][CSV];
    rec[R_SUSU1] = M[CSU][CSU] / 2;
    rec[R_SVSV1] = M[CSV][CSV] / 2;
    rec[R_TI1] = M[CT][CI];
    rec[R_SUI1] = M[CSU][CI];
    rec[R_SVI1] = M[CSV][CI];
    /* N_II1: edges with both ends independent of e (Sec. 4.3, before Eq. g4_9):
     * |E| - (du-1) - (dv-1) - 1 minus every edge touching the egonet. */
    const uint64_t du = (uint64_t)(rp[u + 1] - rp[u]), dv = (uint64_t)(rp[v + 1] - rp[v]);
    const u128 touched = (u128)rec[R_CLIQ] + rec[R_TSU1] + rec[R_TSV1] + rec[R_TI1]
                       + rec[R_SUSU1] + rec[R_SVSV1] + rec[R_CYC] + rec[R_SUI1] + rec[R_SVI1];
    u128 ii1;
    if (!sub_ok((u128)m - (du - 1) - (dv - 1) - 1, touched, &ii1)) return ORACLE_EARITH;
    rec[R_II1] = (uint64_t)ii1;
    for (int64_t i = 0; i < len; i++) cls[list[i]] = 0;
    cls[u] = 0; cls[v] = 0;
    return ORACLE_OK;
}

static int find_slot(const int32_t *rp, const int32_t *ci, int32_t u, int32_t v) {
    int32_t lo = rp[u], hi = rp[u + 1];
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (ci[mid] < v) lo = mid + 1; else hi = mid;
    }
    return (lo < rp[u + 1] && ci[lo] == v) ? lo : -1;
}

/* O1 per edge for a list of edges (eu[i], ev[i]) (each must be an edge; any
 * orientation).  cols: k x 15 u64 (may be NULL); raw: k x R_NUM u64 (may be
 * NULL).  Records are computed for the orientation u = min, v = max. */
int oracle_edges_direct(int32_t n, const int32_t *rp, const int32_t *ci,
                        int64_t k, const int32_t *eu, const int32_t *ev,
                        uint64_t *cols, uint64_t *raw) {
    int rc = check_csr(n, rp, ci);
    if (rc) return rc;
    const int64_t m = (int64_t)rp[n] / 2;
    uint8_t *cls = (uint8_t *)calloc((size_t)n + 1, 1);
    int32_t *list = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    if (!cls || !list) { free(cls); free(list); return ORACLE_ENOMEM; }
    uint64_t rec[R_NUM];
    for (int64_t i = 0; i < k; i++) {
        int32_t u = eu[i] < ev[i] ? eu[i] : ev[i];
        int32_t v = eu[i] < ev[i] ? ev[i] : eu[i];
        if (u < 0 || v >= n || find_slot(rp, ci, u, v) < 0) { rc = ORACLE_EINVAL; break; }
        rc = edge_record_direct(n, rp, ci, m, u, v, cls, list, rec);
        if (rc) break;
        if (raw) memcpy(raw + i * R_NUM, rec, sizeof(rec));
        if (cols && (rc = edge_columns(rec, cols + i * 15))) break;
    }
    free(cls); free(list);
    return rc;
}

/* O1 per edge over all edges in CSR order (u < v). */
int oracle_alg2_per_edge(int32_t n, const int32_t *rp, const int32_t *ci,
                         uint64_t *cols, uint64_t *raw) {
    int rc = check_csr(n, rp, ci);
    if (rc) return rc;
    const int64_t m = (int64_t)rp[n] / 2;
    uint8_t *cls = (uint8_t *)calloc((size_t)n + 1, 1);
    int32_t *list = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    if (!cls || !list) { free(cls); free(list); return ORACLE_ENOMEM; }
    uint64_t rec[R_NUM];
    int64_t e = 0;
    for (int32_t u = 0; u < n && !rc; u++)
        for (int32_t p = rp[u]; p < rp[u + 1]; p++) {
            int32_t v = ci[p];
            if (v <= u) continue;
            rc = edge_record_direct(n, rp, ci, m, u, v, cls, list, rec);
            if (rc) break;
            if (raw) memcpy(raw + e * R_NUM, rec, sizeof(rec));
            if (cols && (rc = edge_columns(rec, cols + e * 15))) break;
            e++;
        }
    free(cls); free(list);
    return rc;
}

/* ======================================================================== */
/* O2: independent method                                                   */
/* ======================================================================== */

static int owner_is_u(const int32_t *rp, int32_t u, int32_t v) {
    /* the endpoint with the larger (degree, id) marks its list; the other scans */
    int32_t du = rp[u + 1] - rp[u], dv = rp[v + 1] - rp[v];
    return du > dv || (du == dv && u > v);
}

static int rank_less(const int32_t *rp, int32_t a, int32_t b) {
    int32_t da = rp[a + 1] - rp[a], db = rp[b + 1] - rp[b];
    return da < db || (da == db && a < b);
}

static void atomic_add_u64(uint64_t *p, uint64_t x) {
    __atomic_fetch_add(p, x, __ATOMIC_RELAXED);
}

/* raw: m x R_NUM (CSR order of u<v edges), required.  threads <= 0: default. */
static int o2_raw(int32_t n, const int32_t *rp, const int32_t *ci, int threads, uint64_t *raw) {
    const int64_t nnz = rp[n];
    const int64_t m = nnz / 2;
    int rc = ORACLE_OK;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
    /* edge id of every slot: id of the undirected edge, CSR order of u<v */
    int64_t *eid = (int64_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int64_t));
    uint32_t *Tslot = (uint32_t *)calloc((size_t)(nnz > 0 ? nnz : 1), sizeof(uint32_t));
    uint64_t *tnode = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    uint64_t *s1 = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    uint64_t *Au = (uint64_t *)calloc((size_t)(m > 0 ? m : 1), sizeof(uint64_t));
    uint64_t *Av = (uint64_t *)calloc((size_t)(m > 0 ? m : 1), sizeof(uint64_t));
    uint64_t *DT = (uint64_t *)calloc((size_t)(m > 0 ? m : 1), sizeof(uint64_t));
    uint64_t *cliq = (uint64_t *)calloc((size_t)(m > 0 ? m : 1), sizeof(uint64_t));
    uint64_t *c4 = (uint64_t *)calloc((size_t)(m > 0 ? m : 1), sizeof(uint64_t));
    if (!eid || !Tslot || !tnode || !s1 || !Au || !Av || !DT || !cliq || !c4) { rc = ORACLE_ENOMEM; goto done; }
    {
        int64_t e = 0;
        for (int32_t u = 0; u < n; u++)
            for (int32_t p = rp[u]; p < rp[u + 1]; p++)
                if (ci[p] > u) eid[p] = e++;
        for (int32_t u = 0; u < n; u++)
            for (int32_t p = rp[u]; p < rp[u + 1]; p++)
                if (ci[p] < u) eid[p] = eid[find_slot(rp, ci, ci[p], u)];
    }
    /* pass 1: T per slot (mark the larger list, scan the smaller) */
    #pragma omp parallel
    {
        int32_t *stamp = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
        #pragma omp for schedule(dynamic, 64)
        for (int32_t u = 0; u < n; u++) {
            if (!stamp) continue;
            for (int32_t p = rp[u]; p < rp[u + 1]; p++) stamp[ci[p]] = u + 1;
            for (int32_t p = rp[u]; p < rp[u + 1]; p++) {
                int32_t v = ci[p];
                if (!owner_is_u(rp, u, v)) continue;
                uint32_t t = 0; int32_t mirror = -1;
                for (int32_t q = rp[v]; q < rp[v + 1]; q++) {
                    int32_t y = ci[q];
                    if (y == u) mirror = q;
                    else if (stamp[y] == u + 1) t++;
                }
                Tslot[p] = t;
                Tslot[mirror] = t;
            }
        }
        if (!stamp) {
            #pragma omp atomic write
            rc = ORACLE_ENOMEM;
        }
        free(stamp);
    }
    if (rc) goto done;
    /* node quantities: t(x) = edges inside N(x) = sum_y T(x,y) / 2; S1(x) */
    #pragma omp parallel for schedule(static)
    for (int32_t x = 0; x < n; x++) {
        uint64_t a = 0, b = 0;
        for (int32_t p = rp[x]; p < rp[x + 1]; p++) { a += Tslot[p]; b += (uint64_t)(rp[ci[p] + 1] - rp[ci[p]]); }
        tnode[x] = a / 2; s1[x] = b;
    }
    /* pass 2: A_u, A_v, D_T per edge (u = smaller id) */
    #pragma omp parallel
    {
        int32_t *stamp = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
        int32_t *pos = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
        #pragma omp for schedule(dynamic, 64)
        for (int32_t u = 0; u < n; u++) {
            if (!stamp || !pos) continue;
            for (int32_t p = rp[u]; p < rp[u + 1]; p++) { stamp[ci[p]] = u + 1; pos[ci[p]] = p; }
            for (int32_t p = rp[u]; p < rp[u + 1]; p++) {
                int32_t v = ci[p];
                if (!owner_is_u(rp, u, v)) continue;
                uint64_t a_own = 0, a_oth = 0, dsum = 0;
                for (int32_t q = rp[v]; q < rp[v + 1]; q++) {
                    int32_t y = ci[q];
                    if (y != u && stamp[y] == u + 1) {
                        a_own += Tslot[pos[y]];
                        a_oth += Tslot[q];
                        dsum += (uint64_t)(rp[y + 1] - rp[y]);
                    }
                }
                int64_t e = eid[p];
                if (u < v) { Au[e] = a_own; Av[e] = a_oth; } else { Au[e] = a_oth; Av[e] = a_own; }
                DT[e] = dsum;
            }
        }
        if (!stamp || !pos) {
            #pragma omp atomic write
            rc = ORACLE_ENOMEM;
        }
        free(stamp); free(pos);
    }
    if (rc) goto done;
    /* pass 3: 4-cliques, each enumerated once from its lowest-ranked edge
     * (orientation: a -> b when rank(a) < rank(b)); +1 on its six edges */
    #pragma omp parallel
    {
        int32_t *stamp = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
        int32_t *pos_a = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
        int32_t *tmark = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
        int32_t *pos_b = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
        int32_t *trl = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
        #pragma omp for schedule(dynamic, 16)
        for (int32_t a = 0; a < n; a++) {
            if (!stamp || !pos_a || !tmark || !pos_b || !trl) continue;
            for (int32_t p = rp[a]; p < rp[a + 1]; p++)
                if (rank_less(rp, a, ci[p])) { stamp[ci[p]] = a + 1; pos_a[ci[p]] = p; }
            for (int32_t p = rp[a]; p < rp[a + 1]; p++) {
                int32_t b = ci[p];
                if (!rank_less(rp, a, b)) continue;
                /* Tri+ = N+(a) n N+(b), ascending ids */
                int32_t nt = 0;
                for (int32_t q = rp[b]; q < rp[b + 1]; q++) {
                    int32_t c = ci[q];
                    if (rank_less(rp, b, c) && stamp[c] == a + 1) { pos_b[c] = q; trl[nt++] = c; }
                }
                /* pairs {c, d} of Tri+ joined by an edge: binary search of
                 * the later one in the earlier one's list */
                for (int32_t i = 0; i < nt; i++) {
                    int32_t c = trl[i];
                    for (int32_t j = i + 1; j < nt; j++) {
                        int32_t d = trl[j];
                        int32_t q = find_slot(rp, ci, c, d);
                        if (q < 0) continue;
                        /* 4-clique {a, b, c, d} */
                        atomic_add_u64(&cliq[eid[p]], 1);
                        atomic_add_u64(&cliq[eid[pos_a[c]]], 1);
                        atomic_add_u64(&cliq[eid[pos_a[d]]], 1);
                        atomic_add_u64(&cliq[eid[pos_b[c]]], 1);
                        atomic_add_u64(&cliq[eid[pos_b[d]]], 1);
                        atomic_add_u64(&cliq[eid[q]], 1);
                    }
                }
            }
        }
        if (!stamp || !pos_a || !tmark || !pos_b || !trl) {
            #pragma omp atomic write
            rc = ORACLE_ENOMEM;
        }
        free(stamp); free(pos_a); free(tmark); free(pos_b); free(trl);
    }
    if (rc) goto done;
    /* pass 4: 4-cycles (not necessarily induced) through each edge (u, v),
     * u < v:  C4(e) = sum_{y in N(v)\{u}} (codeg(u, y) - 1) */
    #pragma omp parallel
    {
        uint32_t *cnt = (uint32_t *)calloc((size_t)n + 1, sizeof(uint32_t));
        int32_t *touched = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
        #pragma omp for schedule(dynamic, 16)
        for (int32_t u = 0; u < n; u++) {
            if (!cnt || !touched) continue;
            int hasup = 0;
            for (int32_t p = rp[u]; p < rp[u + 1]; p++) if (ci[p] > u) { hasup = 1; break; }
            if (!hasup) continue;
            int64_t nt = 0;
            for (int32_t p = rp[u]; p < rp[u + 1]; p++) {
                int32_t x = ci[p];
                for (int32_t q = rp[x]; q < rp[x + 1]; q++) {
                    int32_t y = ci[q];
                    if (y == u) continue;
                    if (cnt[y]++ == 0) touched[nt++] = y;
                }
            }
            for (int32_t p = rp[u]; p < rp[u + 1]; p++) {
                int32_t v = ci[p];
                if (v < u) continue;
                uint64_t c = 0;
                for (int32_t q = rp[v]; q < rp[v + 1]; q++) {
                    int32_t y = ci[q];
                    if (y == u) continue;
                    c += (uint64_t)cnt[y] - 1;   /* cnt[y] >= 1: v itself */
                }
                c4[eid[p]] = c;
            }
            for (int64_t i = 0; i < nt; i++) cnt[touched[i]] = 0;
        }
        if (!cnt || !touched) {
            #pragma omp atomic write
            rc = ORACLE_ENOMEM;
        }
        free(cnt); free(touched);
    }
    if (rc) goto done;
    /* assemble raw records */
    {
        int64_t e = 0;
        int bad = 0;
        for (int32_t u = 0; u < n; u++)
            for (int32_t p = rp[u]; p < rp[u + 1]; p++) {
                int32_t v = ci[p];
                if (v <= u) continue;
                uint64_t *r = raw + e * R_NUM;
                const int64_t du = rp[u + 1] - rp[u], dv = rp[v + 1] - rp[v];
                const int64_t T = Tslot[p];
                const int64_t Su = du - 1 - T, Sv = dv - 1 - T;
                const int64_t I = (int64_t)n - du - dv + T;
                const int64_t cq = (int64_t)cliq[e];
                const int64_t tsu = (int64_t)Au[e] - T - 2 * cq;
                const int64_t tsv = (int64_t)Av[e] - T - 2 * cq;
                const int64_t susu = (int64_t)tnode[u] - T - cq - tsu;
                const int64_t svsv = (int64_t)tnode[v] - T - cq - tsv;
                const int64_t ti = (int64_t)DT[e] - 2 * T - 2 * cq - tsu - tsv;
                const int64_t cy = (int64_t)c4[e] - tsu - tsv - 2 * cq;
                const int64_t sui = ((int64_t)s1[u] - dv - (int64_t)DT[e] - Su) - tsu - 2 * susu - cy;
                const int64_t svi = ((int64_t)s1[v] - du - (int64_t)DT[e] - Sv) - tsv - 2 * svsv - cy;
                const int64_t touched = cq + tsu + tsv + ti + susu + svsv + cy + sui + svi;
                const int64_t ii1 = m - (du - 1) - (dv - 1) - 1 - touched;
                if (Su < 0 || Sv < 0 || I < 0 || tsu < 0 || tsv < 0 || susu < 0 || svsv < 0 ||
                    ti < 0 || cy < 0 || sui < 0 || svi < 0 || ii1 < 0) bad = 1;
                r[R_T] = (uint64_t)T; r[R_SU] = (uint64_t)Su; r[R_SV] = (uint64_t)Sv; r[R_I] = (uint64_t)I;
                r[R_CLIQ] = (uint64_t)cq; r[R_CYC] = (uint64_t)cy;
                r[R_TSU1] = (uint64_t)tsu; r[R_TSV1] = (uint64_t)tsv;
                r[R_SUSU1] = (uint64_t)susu; r[R_SVSV1] = (uint64_t)svsv;
                r[R_TI1] = (uint64_t)ti; r[R_SUI1] = (uint64_t)sui; r[R_SVI1] = (uint64_t)svi;
                r[R_II1] = (uint64_t)ii1;
                e++;
            }
        if (bad) rc = ORACLE_EARITH;
    }
done:
    free(eid); free(Tslot); free(tnode); free(s1); free(Au); free(Av); free(DT); free(cliq); free(c4);
    return rc;
}

/* O2 per edge: raw (m x R_NUM, nullable) and cols (m x 15, nullable). */
int oracle_o2_per_edge(int32_t n, const int32_t *rp, const int32_t *ci, int threads,
                       uint64_t *cols, uint64_t *raw_out) {
    int rc = check_csr(n, rp, ci);
    if (rc) return rc;
    const int64_t m = (int64_t)rp[n] / 2;
    uint64_t *raw = raw_out ? raw_out : (uint64_t *)malloc((size_t)(m > 0 ? m : 1) * R_NUM * sizeof(uint64_t));
    if (!raw) return ORACLE_ENOMEM;
    rc = o2_raw(n, rp, ci, threads, raw);
    if (!rc && cols)
        for (int64_t e = 0; e < m && !rc; e++) rc = edge_columns(raw + e * R_NUM, cols + e * 15);
    if (!raw_out) free(raw);
    return rc;
}

/* O2 global: out 15 x (lo,hi); sums_out (nullable) 13 x (lo,hi). */
int oracle_o2_global(int32_t n, const int32_t *rp, const int32_t *ci, int threads,
                     uint64_t *out, uint64_t *sums_out) {
    int rc = check_csr(n, rp, ci);
    if (rc) return rc;
    const int64_t m = (int64_t)rp[n] / 2;
    uint64_t *raw = (uint64_t *)malloc((size_t)(m > 0 ? m : 1) * R_NUM * sizeof(uint64_t));
    if (!raw) return ORACLE_ENOMEM;
    rc = o2_raw(n, rp, ci, threads, raw);
    if (rc) { free(raw); return rc; }
    sums_t s;
    memset(&s, 0, sizeof(s));
    int64_t e = 0;
    for (int32_t u = 0; u < n; u++)
        for (int32_t p = rp[u]; p < rp[u + 1]; p++) {
            int32_t v = ci[p];
            if (v <= u) continue;
            const uint64_t *r = raw + e * R_NUM;
            const u128 T = r[R_T], Su = r[R_SU], Sv = r[R_SV], I = r[R_I];
            s.sT += T; s.sS += Su + Sv; s.sI += I;
            s.sCliq += r[R_CLIQ]; s.sCyc += r[R_CYC];
            s.nTT += choose2(T); s.nSuSv += Su * Sv; s.nTS += T * (Su + Sv);
            s.nSS += choose2(Su) + choose2(Sv); s.nTI += T * I; s.nSI += (Su + Sv) * I;
            s.nII += choose2(I);
            s.nII1 += (u128)m - (u128)(rp[u + 1] - rp[u] - 1) - (u128)(rp[v + 1] - rp[v] - 1) - 1;
            e++;
        }
    free(raw);
    u128 f[15];
    rc = complete_counts(&s, (u128)n, f);
    if (sums_out) {
        const u128 *sv = (const u128 *)&s;
        for (int i = 0; i < 13; i++) put128(sums_out, i, sv[i]);
    }
    if (rc) return rc;
    for (int i = 0; i < 15; i++) put128(out, i, f[i]);
    return ORACLE_OK;
}

/* Completion alone, for tests that feed hand-made sums: sums 13 x (lo,hi). */
int oracle_complete(const uint64_t *sums_in, uint64_t n, uint64_t *out) {
    sums_t s;
    u128 *sv = (u128 *)&s;
    for (int i = 0; i < 13; i++) sv[i] = (u128)sums_in[2 * i] | ((u128)sums_in[2 * i + 1] << 64);
    u128 f[15];
    int rc = complete_counts(&s, (u128)n, f);
    if (rc) return rc;
    for (int i = 0; i < 15; i++) put128(out, i, f[i]);
    return ORACLE_OK;
}

int oracle_raw_width(void) { return R_NUM; }

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
