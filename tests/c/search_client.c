/*
 * A plain C client of the library's C ABI (include/sw.h): loads a small
 * database, searches one query, aligns its best hit, saves and reopens the
 * database, and prints what it got as one line of "key=value" pairs. The
 * tests build it with gcc against libswgb300.so and compare with the oracle.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "sw.h"

static int die(const char* what, sw_status st) {
    fprintf(stderr, "%s failed (%d): %s\n", what, (int)st, sw_last_error());
    return 1;
}

int main(int argc, char** argv) {
    if (argc < 2) {
        fprintf(stderr, "usage: %s <scratch file>\n", argv[0]);
        return 2;
    }
    /* database: n sequences of a fixed pattern over 20 codes; the query is a piece of #3 */
    enum { N = 64, A = 20 };
    uint64_t offsets[N + 1];
    static uint8_t residues[N * 300];
    uint64_t total = 0;
    for (int s = 0; s < N; ++s) {
        offsets[s] = total;
        const int len = 20 + (s * 37) % 260;
        for (int i = 0; i < len; ++i) residues[total++] = (uint8_t)((s * 7 + i * 13 + i / 5) % A);
    }
    offsets[N] = total;
    uint8_t query[60];
    for (int i = 0; i < 60; ++i) query[i] = residues[offsets[3] + 5 + i];
    int8_t matrix[A * A];
    for (int a = 0; a < A; ++a)
        for (int b = 0; b < A; ++b) matrix[a * A + b] = (int8_t)(a == b ? 5 : -(1 + (a + b) % 3));

    sw_db_opts opts;
    memset(&opts, 0, sizeof opts);
    sw_db* db = NULL;
    sw_status st = sw_db_load(residues, offsets, N, A, &opts, &db);
    if (st != SW_OK) return die("sw_db_load", st);
    int32_t scores[N], top_s[5];
    uint64_t top_i[5];
    uint32_t n_top = 0;
    sw_stats stats;
    st = sw_search(db, query, 60, matrix, 1, 11, 5, scores, top_s, top_i, &n_top, &stats);
    if (st != SW_OK) return die("sw_search", st);
    sw_alignment al;
    char ops[512];
    uint64_t used = 0;
    st = sw_align(db, query, 60, matrix, 1, 11, &top_i[0], 1, &al, ops, sizeof ops, &used);
    if (st != SW_OK) return die("sw_align", st);
    st = sw_db_save(db, argv[1]);
    if (st != SW_OK) return die("sw_db_save", st);
    sw_db_free(db);
    sw_db* db2 = NULL;
    st = sw_db_open(argv[1], NULL, &db2);
    if (st != SW_OK) return die("sw_db_open", st);
    int32_t scores2[N];
    st = sw_search(db2, query, 60, matrix, 1, 11, 0, scores2, NULL, NULL, NULL, NULL);
    if (st != SW_OK) return die("sw_search (reopened)", st);
    sw_db_free(db2);
    /* an error path: a code outside the alphabet */
    query[0] = 25;
    sw_db* db3 = NULL;
    sw_db_load(residues, offsets, N, A, &opts, &db3);
    st = sw_search(db3, query, 60, matrix, 1, 11, 0, NULL, NULL, NULL, NULL, NULL);
    const int rejected = st == SW_ERR_INVALID_ARG && strstr(sw_last_error(), "alphabet") != NULL;
    sw_db_free(db3);

    long sum = 0;
    int same = 1;
    for (int s = 0; s < N; ++s) {
        sum += scores[s];
        same &= scores[s] == scores2[s];
    }
    printf("n_top=%u top_index=%llu top_score=%d sum=%ld reopened_same=%d rejected=%d "
           "align_score=%d q=%u-%u d=%u-%u ops=%.*s cells=%llu\n",
           n_top, (unsigned long long)top_i[0], top_s[0], sum, same, rejected, al.score,
           al.q_begin, al.q_end, al.d_begin, al.d_end, (int)al.ops_len, ops + al.ops_offset,
           (unsigned long long)stats.cells);
    /* every score and the whole top-k list, one line each */
    printf("scores=");
    for (int s = 0; s < N; ++s) printf(s ? ",%d" : "%d", scores[s]);
    printf("\ntop=");
    for (uint32_t k = 0; k < n_top; ++k)
        printf(k ? ",%d:%llu" : "%d:%llu", top_s[k], (unsigned long long)top_i[k]);
    printf("\n");
    return 0;
}
