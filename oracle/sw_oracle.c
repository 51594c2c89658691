/*
 * CPU oracle for exact Smith-Waterman scoring with affine gaps.
 *
 * TEST INFRASTRUCTURE ONLY. This file exists to check the GPU library. It is
 * compiled and called by the tests, by __graft_entry__.smoke() and by the
 * CPU-baseline leg of bench.py, and by nothing else. It shares no code,
 * header or table with the CUDA path.
 *
 * What it computes: recurrence (1) of Section II.A, with S1 = the query
 * (index i, 1..m) and S2 = a database sequence (index j, 1..n):
 *
 *   H[i][j] = max{ 0, H[i-1][j-1] + fsbt(S1[i], S2[j]), E[i][j], F[i][j] }
 *   E[i][j] = max{ E[i-1][j] - alpha, H[i-1][j] - beta }
 *   F[i][j] = max{ F[i][j-1] - alpha, H[i][j-1] - beta }
 *
 * with H[i][0] = H[0][j] = E[0][j] = F[i][0] = 0, and the score is the
 * largest H[i][j]. alpha is the gap extension penalty and beta the sum of
 * the gap open and extension penalties; fsbt(a, b) = matrix[a * A + b] with
 * the row indexed by the query residue. Arithmetic is plain scalar int32.
 *
 * The search result (stage iv of the workflow in Section III) is every score
 * plus the top_k list ordered by score descending; equal scores are ordered
 * by ascending database index.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

static inline int32_t max2(int32_t a, int32_t b) { return a > b ? a : b; }

/*
 * Recurrence (1) in linear space (Section II.A: the score "can be calculated
 * in linear space"). Row i-1 of H and E is kept in H[] and E[]; F[i][j-1]
 * and H[i][j-1] are carried along the row.
 */
int32_t oracle_sw_score(const uint8_t* S1, uint32_t m, const uint8_t* S2, uint32_t n,
                        const int8_t* fsbt, uint32_t A, int32_t alpha, int32_t beta) {
    if (m == 0 || n == 0) return 0;
    int32_t* H = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t)); /* H[i-1][j] */
    int32_t* E = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t)); /* E[i-1][j] */
    if (!H || !E) { free(H); free(E); return -1; }
    int32_t best = 0;
    for (uint32_t i = 1; i <= m; ++i) {
        const int8_t* row = fsbt + (size_t)S1[i - 1] * A;
        int32_t diag = H[0];   /* H[i-1][0] = 0 */
        int32_t Hleft = 0;     /* H[i][0] = 0 */
        int32_t F = 0;         /* F[i][0] = 0 */
        for (uint32_t j = 1; j <= n; ++j) {
            const int32_t e = max2(E[j] - alpha, H[j] - beta);   /* E[i][j] */
            const int32_t f = max2(F - alpha, Hleft - beta);     /* F[i][j] */
            int32_t h = max2(0, diag + (int32_t)row[S2[j - 1]]);
            h = max2(h, max2(e, f));                             /* H[i][j] */
            diag = H[j];                                         /* H[i-1][j] */
            H[j] = h;
            E[j] = e;
            F = f;
            Hleft = h;
            if (h > best) best = h;
        }
    }
    free(H);
    free(E);
    return best;
}

/*
 * The same recurrence with the full (m+1) x (n+1) matrices, exactly as
 * printed. Used only to cross-check the linear-space form on small inputs.
 */
int32_t oracle_sw_score_full(const uint8_t* S1, uint32_t m, const uint8_t* S2, uint32_t n,
                             const int8_t* fsbt, uint32_t A, int32_t alpha, int32_t beta) {
    const size_t W = (size_t)n + 1;
    int32_t* H = (int32_t*)calloc(((size_t)m + 1) * W, sizeof(int32_t));
    int32_t* E = (int32_t*)calloc(((size_t)m + 1) * W, sizeof(int32_t));
    int32_t* F = (int32_t*)calloc(((size_t)m + 1) * W, sizeof(int32_t));
    if (!H || !E || !F) { free(H); free(E); free(F); return -1; }
    int32_t best = 0;
    for (uint32_t i = 1; i <= m; ++i) {
        for (uint32_t j = 1; j <= n; ++j) {
            E[i * W + j] = max2(E[(i - 1) * W + j] - alpha, H[(i - 1) * W + j] - beta);
            F[i * W + j] = max2(F[i * W + j - 1] - alpha, H[i * W + j - 1] - beta);
            const int32_t s = fsbt[(size_t)S1[i - 1] * A + S2[j - 1]];
            int32_t h = max2(0, H[(i - 1) * W + j - 1] + s);
            h = max2(h, E[i * W + j]);
            h = max2(h, F[i * W + j]);
            H[i * W + j] = h;
            if (h > best) best = h;
        }
    }
    free(H);
    free(E);
    free(F);
    return best;
}

typedef struct {
    const uint8_t* q;
    uint32_t m;
    const uint8_t* db;
    const uint64_t* offsets;
    const uint64_t* which;  /* NULL: all sequences */
    uint64_t count;
    const int8_t* fsbt;
    uint32_t A;
    int32_t alpha, beta;
    int32_t* scores;
    uint64_t next;          /* shared work counter */
    pthread_mutex_t lock;
} score_job;

static void* score_worker(void* arg) {
    score_job* J = (score_job*)arg;
    const uint64_t chunk = 64;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        const uint64_t b = J->next;
        J->next = b + chunk;
        pthread_mutex_unlock(&J->lock);
        if (b >= J->count) break;
        const uint64_t e = b + chunk < J->count ? b + chunk : J->count;
        for (uint64_t k = b; k < e; ++k) {
            const uint64_t s = J->which ? J->which[k] : k;
            const uint64_t o = J->offsets[s];
            const uint32_t n = (uint32_t)(J->offsets[s + 1] - o);
            J->scores[k] = oracle_sw_score(J->q, J->m, J->db + o, n, J->fsbt, J->A, J->alpha,
                                           J->beta);
        }
    }
    return NULL;
}

/*
 * scores[k] = score(query, sequence which[k]) for k < count (which == NULL:
 * sequence k), spread over nthreads threads.
 */
int oracle_scores(const uint8_t* query, uint32_t m, const uint8_t* db, const uint64_t* offsets,
                  const uint64_t* which, uint64_t count, const int8_t* fsbt, uint32_t A,
                  int32_t alpha, int32_t beta, int32_t* scores, int nthreads) {
    score_job J = {query, m, db, offsets, which, count, fsbt, A, alpha, beta, scores, 0};
    pthread_mutex_init(&J.lock, NULL);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    int started[256] = {0};
    for (int t = 1; t < nthreads; ++t)
        started[t] = pthread_create(&th[t], NULL, score_worker, &J) == 0;
    score_worker(&J);
    for (int t = 1; t < nthreads; ++t)
        if (started[t]) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&J.lock);
    return 0;
}

typedef struct { int32_t score; uint64_t index; } ranked;

static int by_score_then_index(const void* a, const void* b) {
    const ranked* x = (const ranked*)a;
    const ranked* y = (const ranked*)b;
    if (x->score != y->score) return x->score > y->score ? -1 : 1;
    return x->index < y->index ? -1 : (x->index > y->index ? 1 : 0);
}

/*
 * Stage (iv): sort all (score, index) pairs by score descending, index
 * ascending, and keep the first min(top_k, n) of them.
 */
int oracle_top_k(const int32_t* scores, uint64_t n, uint32_t top_k, int32_t* top_scores,
                 uint64_t* top_index, uint32_t* n_top) {
    ranked* r = (ranked*)malloc((n ? n : 1) * sizeof(ranked));
    if (!r) return -1;
    for (uint64_t s = 0; s < n; ++s) { r[s].score = scores[s]; r[s].index = s; }
    qsort(r, n, sizeof(ranked), by_score_then_index);
    const uint32_t k = (uint64_t)top_k < n ? top_k : (uint32_t)n;
    for (uint32_t i = 0; i < k; ++i) { top_scores[i] = r[i].score; top_index[i] = r[i].index; }
    *n_top = k;
    free(r);
    return 0;
}

/* Full search of one query: every score (database order) and the top_k list. */
int oracle_search(const uint8_t* query, uint32_t m, const uint8_t* db, const uint64_t* offsets,
                  uint64_t n_seqs, const int8_t* fsbt, uint32_t A, int32_t alpha, int32_t beta,
                  uint32_t top_k, int32_t* scores, int32_t* top_scores, uint64_t* top_index,
                  uint32_t* n_top, int nthreads) {
    oracle_scores(query, m, db, offsets, NULL, n_seqs, fsbt, A, alpha, beta, scores, nthreads);
    return oracle_top_k(scores, n_seqs, top_k, top_scores, top_index, n_top);
}

/*
 * One optimal local alignment of S1 (query, m) and S2 (database sequence, n):
 * the traceback that Section IV.C leaves to future work. What is returned
 * (the paper does not define it; these are the readings the tests check):
 *
 *  - the score S = max H[i][j] of recurrence (1);
 *  - the end cell: the first (i, j), in order of i then j, with H[i][j] = S;
 *    for S > 0 the alignment ends by aligning S1[i] with S2[j];
 *  - the start cell: of the cells (i', j') from which an alignment that
 *    begins by aligning S1[i'] with S2[j'] and ends by aligning S1[i] with
 *    S2[j] scores S, the one with the largest i', then the largest j';
 *  - the path: the three-state dynamic programme (M: S1[u] aligned with
 *    S2[v]; E: S1[u] against a gap; F: S2[v] against a gap) anchored at both
 *    cells, with the gap costs of recurrence (1) (a gap of either kind opens
 *    from H = max(M, E, F) at cost beta and extends at cost alpha), traced
 *    back from M at the end cell; H prefers M, then E, then F, and a gap state
 *    prefers extending to opening when both give its value.
 *
 * out = {S, q_begin, q_end, d_begin, d_end} with 0-based half-open residue
 * ranges; ops = one letter per alignment column in order: 'M' (a residue of
 * each), 'I' (a query residue against a gap), 'D' (a database residue against
 * a gap). S = 0 gives empty ranges and no ops. Returns 0, or -1 when ops_cap
 * is too small or memory runs out.
 */
#define ORACLE_NEG (-(1 << 29))

static int32_t max3i(int32_t a, int32_t b, int32_t c) { return max2(a, max2(b, c)); }

int oracle_sw_align(const uint8_t* S1, uint32_t m, const uint8_t* S2, uint32_t n,
                    const int8_t* fsbt, uint32_t A, int32_t alpha, int32_t beta, int32_t* out,
                    char* ops, uint32_t ops_cap, uint32_t* ops_len) {
    out[0] = out[1] = out[2] = out[3] = out[4] = 0;
    *ops_len = 0;
    if (m == 0 || n == 0) return 0;
    /* 1. score and end cell: recurrence (1) row by row, the first strict maximum */
    int32_t* H = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t));
    int32_t* E = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t));
    if (!H || !E) { free(H); free(E); return -1; }
    int32_t S = 0;
    uint32_t ie = 0, je = 0;
    for (uint32_t i = 1; i <= m; ++i) {
        int32_t diag = 0, Hleft = 0, F = 0;
        for (uint32_t j = 1; j <= n; ++j) {
            const int32_t e = max2(E[j] - alpha, H[j] - beta);
            F = max2(F - alpha, Hleft - beta);
            int32_t h = diag + fsbt[(uint32_t)S1[i - 1] * A + S2[j - 1]];
            h = max2(max2(h, 0), max2(e, F));
            diag = H[j];
            H[j] = h;
            E[j] = e;
            Hleft = h;
            if (h > S) { S = h; ie = i; je = j; }
        }
    }
    free(H);
    free(E);
    if (S == 0) return 0;

    /* 2. start cell: the same gap model run backwards from the end cell, anchored
     * there; Mr[i][j] is the best score of an alignment that begins by aligning
     * S1[i] with S2[j] and ends at the end cell (i <= ie, j <= je) */
    const uint32_t a0 = ie, b0 = je;  /* reversed extents */
    int32_t* Mr = (int32_t*)malloc(((size_t)a0 + 1) * (b0 + 1) * sizeof(int32_t));
    int32_t* Er = (int32_t*)malloc(((size_t)a0 + 1) * (b0 + 1) * sizeof(int32_t));
    int32_t* Fr = (int32_t*)malloc(((size_t)a0 + 1) * (b0 + 1) * sizeof(int32_t));
    if (!Mr || !Er || !Fr) { free(Mr); free(Er); free(Fr); return -1; }
#define R_(X, u, v) X[(size_t)(u) * (b0 + 1) + (v)]
    /* reversed coordinates u = ie - i + 1, v = je - j + 1 (1-based) */
    uint32_t is = 0, js = 0;
    for (uint32_t u = 0; u <= a0; ++u)
        for (uint32_t v = 0; v <= b0; ++v) {
            if (u == 0 || v == 0) {
                R_(Mr, u, v) = R_(Er, u, v) = R_(Fr, u, v) = ORACLE_NEG;
                continue;
            }
            const uint32_t i = ie - u + 1, j = je - v + 1;
            const int32_t s = fsbt[(uint32_t)S1[i - 1] * A + S2[j - 1]];
            int32_t mv;
            if (u == 1 && v == 1) mv = s;
            else {
                const int32_t hp = max3i(R_(Mr, u - 1, v - 1), R_(Er, u - 1, v - 1), R_(Fr, u - 1, v - 1));
                mv = hp <= ORACLE_NEG / 2 ? ORACLE_NEG : hp + s;
            }
            const int32_t hu = max3i(R_(Mr, u - 1, v), R_(Er, u - 1, v), R_(Fr, u - 1, v));
            const int32_t ev = max2(R_(Er, u - 1, v) - alpha, hu - beta);
            const int32_t hv = max3i(R_(Mr, u, v - 1), R_(Er, u, v - 1), R_(Fr, u, v - 1));
            const int32_t fv = max2(R_(Fr, u, v - 1) - alpha, hv - beta);
            R_(Mr, u, v) = mv;
            R_(Er, u, v) = ev <= ORACLE_NEG / 2 ? ORACLE_NEG : ev;
            R_(Fr, u, v) = fv <= ORACLE_NEG / 2 ? ORACLE_NEG : fv;
            if (mv == S && is == 0) { is = i; js = j; }  /* first in (u, v) order */
        }
    free(Mr);
    free(Er);
    free(Fr);
#undef R_
    if (is == 0) return -1; /* cannot happen: the alignment found in step 1 starts somewhere */

    /* 3. the path: anchored three-state programme over the box, full matrices */
    const uint32_t a = ie - is + 1, b = je - js + 1;
    int32_t* M3 = (int32_t*)malloc(((size_t)a + 1) * (b + 1) * sizeof(int32_t));
    int32_t* E3 = (int32_t*)malloc(((size_t)a + 1) * (b + 1) * sizeof(int32_t));
    int32_t* F3 = (int32_t*)malloc(((size_t)a + 1) * (b + 1) * sizeof(int32_t));
    if (!M3 || !E3 || !F3) { free(M3); free(E3); free(F3); return -1; }
#define B_(X, u, v) X[(size_t)(u) * (b + 1) + (v)]
    for (uint32_t u = 0; u <= a; ++u)
        for (uint32_t v = 0; v <= b; ++v) {
            if (u == 0 || v == 0) {
                B_(M3, u, v) = B_(E3, u, v) = B_(F3, u, v) = ORACLE_NEG;
                continue;
            }
            const int32_t s = fsbt[(uint32_t)S1[is + u - 2] * A + S2[js + v - 2]];
            int32_t mv;
            if (u == 1 && v == 1) mv = s;
            else {
                const int32_t hp = max3i(B_(M3, u - 1, v - 1), B_(E3, u - 1, v - 1), B_(F3, u - 1, v - 1));
                mv = hp <= ORACLE_NEG / 2 ? ORACLE_NEG : hp + s;
            }
            const int32_t hu = max3i(B_(M3, u - 1, v), B_(E3, u - 1, v), B_(F3, u - 1, v));
            const int32_t ev = max2(B_(E3, u - 1, v) - alpha, hu - beta);
            const int32_t hv = max3i(B_(M3, u, v - 1), B_(E3, u, v - 1), B_(F3, u, v - 1));
            const int32_t fv = max2(B_(F3, u, v - 1) - alpha, hv - beta);
            B_(M3, u, v) = mv;
            B_(E3, u, v) = ev <= ORACLE_NEG / 2 ? ORACLE_NEG : ev;
            B_(F3, u, v) = fv <= ORACLE_NEG / 2 ? ORACLE_NEG : fv;
        }
    int rc = 0;
    if (B_(M3, a, b) != S) rc = -1;
    /* trace back from M at (a, b); letters come out reversed */
    uint32_t u = a, v = b, len = 0;
    int state = 0; /* 0 = M, 1 = E, 2 = F */
    while (rc == 0) {
        if (len >= ops_cap) { rc = -1; break; }
        if (state == 0) {
            ops[len++] = 'M';
            if (u == 1 && v == 1) break;
            --u;
            --v;
        } else if (state == 1) {
            ops[len++] = 'I';
            const int extend = B_(E3, u, v) == B_(E3, u - 1, v) - alpha;
            --u;
            if (extend) continue;
        } else {
            ops[len++] = 'D';
            const int extend = B_(F3, u, v) == B_(F3, u, v - 1) - alpha;
            --v;
            if (extend) continue;
        }
        /* entering H at (u, v): M, then E, then F */
        const int32_t hm = B_(M3, u, v), he = B_(E3, u, v), hf = B_(F3, u, v);
        state = (hm >= he && hm >= hf) ? 0 : (he >= hf ? 1 : 2);
    }
    free(M3);
    free(E3);
    free(F3);
#undef B_
    if (rc != 0) return rc;
    for (uint32_t k = 0; k < len / 2; ++k) {
        const char c = ops[k];
        ops[k] = ops[len - 1 - k];
        ops[len - 1 - k] = c;
    }
    *ops_len = len;
    out[0] = S;
    out[1] = (int32_t)(is - 1);
    out[2] = (int32_t)ie;
    out[3] = (int32_t)(js - 1);
    out[4] = (int32_t)je;
    return 0;
}
