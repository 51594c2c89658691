/*
 * swgb300 — exact Smith-Waterman protein database search on one GB300 GPU.
 *
 * C ABI of the library (libswgb300.so). Every entry point scores protein
 * queries against a protein database with recurrence (1) of Section II.A of
 * Liu & Schmidt, "SWAPHI: Smith-Waterman Protein Database Search on Xeon Phi
 * Coprocessors" (arXiv:1404.4152):
 *
 *   H[i][j] = max{ 0, H[i-1][j-1] + fsbt(S1[i], S2[j]), E[i][j], F[i][j] }
 *   E[i][j] = max{ E[i-1][j] - alpha, H[i-1][j] - beta }
 *   F[i][j] = max{ F[i][j-1] - alpha, H[i][j-1] - beta }
 *
 * with H = E = F = 0 on the borders; the score of a pair is the largest H.
 * S1 is the query (rows) and S2 a database sequence (columns); fsbt(a, b) =
 * matrix[a * alphabet + b], row = query residue. alpha is the gap extension
 * penalty and beta the sum of the gap open and extension penalties, exactly as
 * the recurrence uses them. Every score is exact (bit-identical to scalar int32
 * arithmetic); no result is approximated.
 *
 * A search returns every score (database order) and the top_k hits ordered by
 * score descending, equal scores by ascending database index (stage (iv) of
 * the workflow in Section III).
 *
 * Conventions for every call:
 *  - Status codes: SW_OK or an error; on error nothing is written to any
 *    output and sw_last_error() returns a message for the calling thread.
 *  - Pointers marked HOST are ordinary host memory (pageable or pinned);
 *    pointers marked DEVICE are CUDA device memory on the database's device.
 *    The caller owns every buffer it passes; the library copies what it needs
 *    before returning (or, for the _device calls, before the work it enqueued
 *    on the caller's stream completes).
 *  - Residue codes are 0 .. alphabet-1, alphabet <= 32 (Section III.B.2:
 *    |Sigma| < 32 for biological sequences). Scoring-matrix entries are int8.
 *  - 0 <= alpha, beta <= 32767; top_k <= SW_MAX_TOP_K; a query has >= 1
 *    residue; database sequences may be empty (score 0).
 *  - Threads: a database handle may be searched from one thread at a time;
 *    different handles are independent. A server handle is thread-safe.
 *  - No exception crosses this interface.
 */
#ifndef SWGB300_SW_H
#define SWGB300_SW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SW_MAX_ALPHABET 32u
#define SW_MAX_TOP_K 1024u

typedef enum {
    SW_OK = 0,
    SW_ERR_INVALID_ARG = 1, /* a bad pointer, size, code, penalty or option */
    SW_ERR_OOM = 2,         /* device or host memory (or the configured budget) exhausted */
    SW_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    SW_ERR_TIMEOUT = 4,     /* a bounded wait ran out */
    SW_ERR_BUSY = 5,        /* the server queue is full or the ticket is unknown */
    SW_ERR_INTERNAL = 6     /* a broken internal invariant */
} sw_status;

/* Options for sw_db_load. Zero-initialise and set what you need; zero fields take defaults. */
typedef struct {
    int device;                 /* CUDA device ordinal (default 0) */
    uint32_t long_threshold;    /* sequences longer than this go to the warp-per-pair kernel
                                   (default 3000) */
    uint64_t device_budget;     /* cap on the bytes this handle may allocate on the device
                                   (0 = no cap); exceeding it gives SW_ERR_OOM */
    uint32_t flags;             /* SW_DB_FLAG_* */
    uint32_t block_threshold;   /* sequences longer than this (and than long_threshold) are
                                   scored by a whole block of 8 warps each, the multi-warp
                                   wavefront of the intra-sequence model (Section III.C),
                                   beside the warp-per-pair kernel, so one very long
                                   sequence does not leave one warp working after the
                                   others finish. 0 = automatic: max(4 * long_threshold,
                                   total residues / (32 * SM count)), the length at which a
                                   pair unit outgrows one warp's share of the search;
                                   UINT32_MAX = never */
} sw_db_opts;

#define SW_DB_FLAG_FORCE_INT32 1u   /* skip the packed 16-bit kernels; everything in int32 */
#define SW_DB_FLAG_PROFILE 2u       /* time every kernel phase with CUDA events (sw_db_get_profile) */
#define SW_DB_FLAG_QUERY_PROFILE 4u /* single queries use the int8 query-profile kernel instead of
                                       the score-profile ring (Section III.B.2 compares the two) */

typedef struct sw_db sw_db;

typedef struct {
    uint64_t n_seqs;
    uint64_t total_residues;     /* sum of database sequence lengths */
    uint64_t device_bytes;       /* bytes this handle holds on the device */
    uint32_t alphabet;
    uint32_t max_length;
    uint64_t n_long;             /* sequences above long_threshold */
    int device;
    uint64_t n_block;            /* sorted positions scored by the block wavefront (whole
                                    tiles of 8 that hold a sequence above block_threshold) */
    uint32_t block_threshold;    /* the threshold in effect */
} sw_db_info;

/* Per-call statistics (optional output of the search calls). */
typedef struct {
    uint64_t cells;              /* sum over pairs of |query| * |db sequence| (real residues) */
    uint64_t recomputed;         /* sequences rescored in int32 after the 16-bit lanes saturated */
    double kernel_ms;            /* device time from the first to the last kernel of the call */
    double total_ms;             /* wall time of the whole call, copies included */
} sw_stats;

/*
 * Load a database onto the device (stage (i)/(ii) set-up of Section III: the
 * subject sequences are ordered by length, as the paper's offline index does,
 * and laid out for the kernels).
 *
 *   residues : HOST, uint8 codes of all sequences concatenated (offsets[n_seqs] bytes)
 *   offsets  : HOST, n_seqs + 1 ascending byte offsets; sequence s is
 *              residues[offsets[s] .. offsets[s+1])
 *   n_seqs   : number of sequences (>= 1)
 *   alphabet : number of residue codes (1 .. 32); every code must be < alphabet
 *   opts     : HOST, may be NULL (defaults)
 *   out      : receives the handle; free it with sw_db_free
 *
 * Errors: SW_ERR_INVALID_ARG (bad code, offsets not ascending, ...), SW_ERR_OOM,
 * SW_ERR_CUDA. The host arrays may be freed as soon as the call returns.
 */
sw_status sw_db_load(const uint8_t* residues, const uint64_t* offsets, uint64_t n_seqs,
                     uint32_t alphabet, const sw_db_opts* opts, sw_db** out);

/*
 * Save a loaded database (its length-sorted tiles and index: the offline index
 * of Section III) to a file, and open such a file later without sorting or
 * re-tiling. The file is little-endian and written by this library; sw_db_open
 * checks its magic, version, size and internal consistency (every sequence
 * once in the sorted order, lengths and tile sizes adding up, every byte a
 * residue code below the alphabet or the pad code) and fails with
 * SW_ERR_INVALID_ARG otherwise. The long-sequence threshold is the one the
 * database was loaded with (opts->long_threshold is ignored); device,
 * device_budget, flags and block_threshold come from opts (NULL = defaults).
 * Searches on an opened database give the same results as on the original.
 */
sw_status sw_db_save(const sw_db* db, const char* path);
sw_status sw_db_open(const char* path, const sw_db_opts* opts, sw_db** out);

/* Release a database and all its device memory. NULL is ignored. */
void sw_db_free(sw_db* db);

/* Describe a loaded database. */
sw_status sw_db_get_info(const sw_db* db, sw_db_info* info);

/*
 * Search one query (HOST buffers; copies in and out are part of the call).
 *
 *   query      : HOST, qlen residue codes (< alphabet)
 *   matrix     : HOST, alphabet * alphabet int8 scores, row = query residue
 *   alpha,beta : gap extension / open-plus-extension penalties of recurrence (1)
 *   top_k      : number of hits wanted (0 .. SW_MAX_TOP_K)
 *   scores     : HOST, n_seqs int32, database order; may be NULL
 *   top_scores : HOST, top_k int32; may be NULL when top_k == 0
 *   top_index  : HOST, top_k uint64 database indices
 *   n_top      : HOST, receives min(top_k, n_seqs)
 *   stats      : HOST, may be NULL
 */
sw_status sw_search(sw_db* db, const uint8_t* query, uint32_t qlen, const int8_t* matrix,
                    int32_t alpha, int32_t beta, uint32_t top_k, int32_t* scores,
                    int32_t* top_scores, uint64_t* top_index, uint32_t* n_top, sw_stats* stats);

/*
 * Search one query with DEVICE buffers, enqueued on a caller stream
 * (cudaStream_t passed as void*; NULL = the legacy default stream). The call
 * returns after enqueueing; results are valid once the stream reaches them.
 *
 *   d_query      : DEVICE, qlen codes
 *   d_matrix     : DEVICE, alphabet * alphabet int8
 *   d_scores     : DEVICE, n_seqs int32 (database order); may be NULL
 *   d_top_scores : DEVICE, top_k int32;  d_top_index : DEVICE, top_k uint64
 *
 * Codes in d_query are checked on the device: a code >= alphabet makes the
 * result undefined but never an out-of-bounds access (it is clamped to the pad
 * code, which scores 0). Use sw_search for validated input.
 *
 * When the database has sequences above its block threshold, their kernel runs
 * on a stream of the handle, forked from the caller's stream by an event before
 * the search kernel and joined back into it after: the caller's stream order
 * holds, and the enqueued work can be captured into a CUDA graph. One handle
 * serves one such call at a time.
 */
sw_status sw_search_device(sw_db* db, const uint8_t* d_query, uint32_t qlen,
                           const int8_t* d_matrix, int32_t alpha, int32_t beta, uint32_t top_k,
                           int32_t* d_scores, int32_t* d_top_scores, uint64_t* d_top_index,
                           void* stream);

/*
 * Search nq queries against the database in one batched launch sequence
 * (HOST buffers). queries[q] has qlens[q] codes; scores may be NULL, else
 * scores[q] is NULL or n_seqs int32. top_scores / top_index hold nq * top_k
 * entries (row q = query q); n_top[q] receives min(top_k, n_seqs).
 */
sw_status sw_search_batch(sw_db* db, uint32_t nq, const uint8_t* const* queries,
                          const uint32_t* qlens, const int8_t* matrix, int32_t alpha,
                          int32_t beta, uint32_t top_k, int32_t* const* scores,
                          int32_t* top_scores, uint64_t* top_index, uint32_t* n_top,
                          sw_stats* stats);

/*
 * Per-phase kernel timing of a handle loaded with SW_DB_FLAG_PROFILE (the
 * tracing subsystem). Phases: 0 = the wavefront search kernel (both
 * length bins), 1 = int32 rescoring, 2 = top-k, 3 = the batched search
 * kernel. ms[p] is the summed device time of phase p measured
 * with CUDA events on the stream it ran on, calls[p] the number of timed
 * launches, cells[p] the DP cells it processed (sum of |query| * |sequence|
 * over real residues). launches counts every kernel the handle enqueued since
 * load or the last reset, timed or not. Reading waits for the timed work.
 */
typedef struct {
    uint64_t launches;
    uint64_t calls[4];
    uint64_t cells[4];
    double ms[4];
} sw_profile;

sw_status sw_db_get_profile(sw_db* db, sw_profile* out);
sw_status sw_db_reset_profile(sw_db* db);

/*
 * Search nq queries with DEVICE buffers in one batched launch sequence,
 * enqueued on a caller stream (cudaStream_t as void*).
 *
 *   d_queries    : DEVICE, all queries concatenated
 *   qoffsets     : HOST, nq + 1 ascending offsets into d_queries (query q is
 *                  d_queries[qoffsets[q] .. qoffsets[q+1]), at least 1 residue)
 *   d_matrix     : DEVICE, alphabet * alphabet int8
 *   d_scores     : DEVICE, nq * n_seqs int32, row q = query q, database order
 *   d_top_scores : DEVICE, nq * top_k int32; d_top_index : DEVICE, nq * top_k uint64
 *
 * Queries are paired by length and each pair shares the 16-bit halves of the
 * lanes; all pairs run in one persistent launch. The launch sequence is
 * captured in a CUDA graph and replayed when the next call has the same
 * buffers, lengths, penalties and stream. The call returns after enqueueing.
 * If more (query, sequence) pairs saturate the 16-bit lanes than the
 * rescoring list holds (max(n_seqs, 2^20) entries), the excess keep the score
 * -1; sw_search_batch detects this and searches again in int32.
 */
sw_status sw_search_batch_device(sw_db* db, uint32_t nq, const uint8_t* d_queries,
                                 const uint64_t* qoffsets, const int8_t* d_matrix, int32_t alpha,
                                 int32_t beta, uint32_t top_k, int32_t* d_scores,
                                 int32_t* d_top_scores, uint64_t* d_top_index, void* stream);

/*
 * Autotuning (no counterpart in the paper, which fixes its kernel shapes; the
 * score-profile width N = 8 of Section III.B.3 is the nearest analogue).
 * Times the search kernel on a sample of this database for every kernel mode
 * (index 0: one query against pairs of database sequences, int8 query profile;
 * 1: two queries per lane pair, used by batches and the server; 2: int32;
 * 3: one query against pairs with the score-profile ring of Section III.B.2,
 * the default for single queries) and every rows-per-lane
 * choice R in {8, 12, 16, 20, 24}, and stores the device time per query row
 * and database residue. Later searches on the handle pick R by minimising
 * padded rows x measured cost, and single queries take the faster of modes 0
 * and 3. int32_over_int16 is the measured speed ratio;
 * cutover_fraction the share of saturating pairs above which a search would be
 * cheaper in int32 (the 16/32-bit cutover). cache_path (may be NULL) names a
 * JSON file reused when its GPU name and SM count match.
 */
typedef struct {
    double ns_per_row_residue[4][5];
    uint32_t fastest_R[4];
    double int32_over_int16;
    double cutover_fraction;
    int from_cache;
} sw_tuning;

sw_status sw_db_autotune(sw_db* db, const int8_t* matrix, int32_t alpha, int32_t beta,
                         const char* cache_path, sw_tuning* out);

/*
 * Serving: a continuous-batching server over a loaded database (the paper
 * searches one query at a time; this keeps the database resident and takes
 * queries as they arrive).
 *
 * The database is cut into `slices` parts of about equal work. A scheduler
 * thread runs waves; one wave advances every admitted query by one slice in
 * persistent launches (two queries at the same slice share the 16-bit lane
 * halves when their lengths are close enough for the pair to cost less than
 * the two alone; the others run one query against two sequences). A query is
 * admitted at a wave boundary when a slot is free: a
 * slot reserves the device memory one query needs (a score row of n_seqs
 * int32 and max_qlen code bytes), and the number of slots is bounded by
 * max_active and by device_budget, so admission is by device memory. Queries
 * that arrive while others are on the GPU join the next wave; a query leaves
 * after its last slice with its exact top-k list. Requests whose scoring
 * scheme (matrix, alpha, beta) differs from the running ones wait until those
 * drain. While a server exists, use the database only through it.
 */
typedef struct sw_server sw_server;

typedef struct {
    uint32_t max_queue;        /* waiting requests beyond which submit fails SW_ERR_BUSY (4096) */
    uint32_t max_active;       /* query slots (64) */
    uint32_t max_qlen;         /* longest accepted query (8192) */
    uint32_t slices;           /* database slices per query (8) */
    uint64_t device_budget;    /* bytes for the slots (0 = max_active slots) */
} sw_server_opts;

typedef struct {
    double submit_ms;          /* times in ms since the server was created */
    double admit_ms;
    double done_ms;
} sw_latency;

typedef struct {
    uint64_t waves, completed, rejected;
    uint64_t cells;            /* DP cells of the completed queries */
    double busy_ms;            /* wall time spent in waves */
    uint32_t pending, active, max_active, slices;
    double gpu_ms;             /* device time of the waves (first to last command of each wave);
                                  busy_ms - gpu_ms is the host's share: launches, the
                                  wave-end synchronisation and bookkeeping */
} sw_server_stats;

/* Create a server (starts its scheduler thread). opts may be NULL. */
sw_status sw_server_create(sw_db* db, const sw_server_opts* opts, sw_server** out);
/* Queue one query (HOST buffers, copied before returning); receives a ticket. */
sw_status sw_server_submit(sw_server* srv, const uint8_t* query, uint32_t qlen,
                           const int8_t* matrix, int32_t alpha, int32_t beta, uint32_t top_k,
                           uint64_t* ticket);
/* Wait up to timeout_ms for a ticket: top_k results (HOST) and its timestamps.
 * SW_ERR_TIMEOUT if not done in time (the ticket stays valid); a finished
 * ticket is consumed. */
sw_status sw_server_wait(sw_server* srv, uint64_t ticket, uint32_t timeout_ms,
                         int32_t* top_scores, uint64_t* top_index, uint32_t* n_top,
                         sw_latency* lat);
/* Drop a ticket: a waiting request never runs, a running one leaves at the next wave. */
sw_status sw_server_cancel(sw_server* srv, uint64_t ticket);
sw_status sw_server_get_stats(sw_server* srv, sw_server_stats* out);
/* Stop the scheduler (outstanding requests are cancelled) and free the server. */
void sw_server_destroy(sw_server* srv);

/*
 * Score one query against caller-owned device sequences WITHOUT allocating
 * any device memory. The paper has no counterpart to this call; it exists for
 * callers that may not call cudaMalloc, for example a host application that
 * reserves all device memory up front through its own allocator and forbids
 * other allocations, or a serving loop that cannot afford the device-wide
 * synchronisation cudaMalloc can cause. It needs no database handle (loading
 * one allocates): the caller passes everything as DEVICE buffers.
 *
 *   d_query    : DEVICE, qlen codes;  d_matrix : DEVICE, alphabet * alphabet int8
 *   d_residues : DEVICE, the database sequences concatenated (codes < alphabet)
 *   d_offsets  : DEVICE, n_seqs + 1 uint64 offsets into d_residues
 *   max_len    : HOST value, the longest sequence in the set
 *   d_scores   : DEVICE, n_seqs int32, written in database order
 *   stream     : cudaStream_t as void*; the work is enqueued there
 *
 * For valid input the scores are identical to sw_search's on the same
 * sequences. Inputs the kernel cannot score are marked in the output instead
 * of failing the call (the host never reads the device buffers):
 *   -1  the sequence is longer than 2048 residues while qlen > 512 (the
 *       caller's max_len understated it);
 *   -2  the sequence holds a code >= alphabet, or the query does (then every
 *       score is -2). sw_search instead rejects such codes when the database
 *       is loaded.
 *
 * The working memory is one fixed device array of 33,554,688 bytes (32 MiB +
 * 256 B) inside the library, held by every GPU that loads the library until
 * the process exits. It bounds the input: when qlen > 512, every sequence must
 * be at most 2048 residues (a larger max_len is rejected with
 * SW_ERR_INVALID_ARG). Queries of at most 512 residues take sequences of any
 * length and use every SM; longer ones run on 128 blocks, one per row slot of
 * the array.
 *
 * Every call looks up the array's device address with cudaGetSymbolAddress
 * (with the caller's device current; nothing is cached, so a device reset is
 * harmless). With lazy module loading (the CUDA default) the first call on a
 * device is also when the library's module is loaded and the array and the
 * module's code take their device memory: a caller that will later give all
 * free memory to its own allocator should make one call before that, or run
 * with CUDA_MODULE_LOADING=EAGER. Make that first call before any stream
 * capture. All calls share the array and leave their contents in it: the work
 * counter is cleared at the start of every call, but calls whose work overlaps
 * on the GPU (different streams, or different host threads, at the same time)
 * race and give wrong scores. Serialise them, e.g. on one stream. The call
 * never calls cudaMalloc, cudaFree or any allocating routine.
 */
sw_status sw_search_noalloc(const uint8_t* d_query, uint32_t qlen, const int8_t* d_matrix,
                            uint32_t alphabet, int32_t alpha, int32_t beta,
                            const uint8_t* d_residues, const uint64_t* d_offsets, uint32_t n_seqs,
                            uint32_t max_len, int32_t* d_scores, void* stream);

/*
 * Traceback: one optimal local alignment of the query with each listed
 * database sequence (HOST buffers; the paper computes scores only and leaves
 * alignments to future work, Section IV.C). For each sequence:
 *
 *   score        the Smith-Waterman score of recurrence (1) (as sw_search);
 *   end cell     the first (query position, database position), in order of
 *                query then database position, where H reaches the score; the
 *                alignment ends by aligning those two residues;
 *   start cell   of the optimal alignments ending there, the latest start
 *                (largest query position, then largest database position);
 *   path         the three-state programme anchored at both cells, traced
 *                back from the end; H prefers an aligned pair, then a query
 *                residue against a gap, then a database residue against a gap,
 *                and a gap prefers extending to opening when both give its
 *                value. These rules make the alignment unique.
 *
 *   db_index   : HOST, n original database indices (any order, repeats allowed)
 *   out        : HOST, n records; ranges are 0-based and half-open; score 0
 *                gives empty ranges and no letters
 *   ops        : HOST, ops_cap chars; record k's letters are
 *                ops[out[k].ops_offset .. + out[k].ops_len): 'M' aligns a
 *                query residue with a database residue, 'I' is a query residue
 *                against a gap, 'D' a database residue against a gap
 *   ops_used   : HOST, receives the letters needed (also when ops_cap is too
 *                small, which fails with SW_ERR_INVALID_ARG and fills nothing
 *                else)
 *
 * Scores are computed in int32 whatever the penalties. Device memory: the box
 * between the start and end cells takes one byte per cell (batched within
 * 1 GiB; a larger single box takes its own size). Hits of at least 2^20 cells
 * (query length x sequence length) find their end and start cells on a whole
 * block of warps, on a second stream the handle creates on first use; the call
 * returns when both streams are done.
 */
typedef struct {
    int32_t score;
    uint32_t q_begin, q_end;    /* query residues [q_begin, q_end) */
    uint64_t db_index;          /* database sequence (original index) */
    uint32_t d_begin, d_end;    /* its residues [d_begin, d_end) */
    uint64_t ops_offset;        /* first letter of this alignment in ops */
    uint32_t ops_len;
} sw_alignment;

sw_status sw_align(sw_db* db, const uint8_t* query, uint32_t qlen, const int8_t* matrix,
                   int32_t alpha, int32_t beta, const uint64_t* db_index, uint32_t n,
                   sw_alignment* out, char* ops, uint64_t ops_cap, uint64_t* ops_used);

/*
 * The same for the hits of several queries in one call (all pairs aligned in
 * parallel): queries (HOST) concatenated with qoffsets[0..nq] as in
 * sw_search_batch; hit k aligns query hit_query[k] with db_index[k].
 */
sw_status sw_align_batch(sw_db* db, uint32_t nq, const uint8_t* queries, const uint64_t* qoffsets,
                         const int8_t* matrix, int32_t alpha, int32_t beta,
                         const uint32_t* hit_query, const uint64_t* db_index, uint32_t n,
                         sw_alignment* out, char* ops, uint64_t ops_cap, uint64_t* ops_used);

/*
 * Bounds-checked build (compiled with -DSW_DEBUG_BOUNDS, libswgb300_debug.so; a
 * stand-in for a memory checker): the kernels check their shared- and
 * global-memory indices, skip an access that would leave its buffer and record
 * the site of the first such access in the handle. This call waits for the
 * device, returns that site (0: none) and clears it. In the normal build it
 * always returns 0. Sites: 1-8 search kernels, 11-13 the block-wide kernels
 * (int32 rescoring, long alignment hits), 21-26 alignment.
 */
sw_status sw_db_debug_check(sw_db* db, uint32_t* site);

/* Message for the last non-OK status returned to this thread ("" if none). */
const char* sw_last_error(void);

/* Library version string. */
const char* sw_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SWGB300_SW_H */
