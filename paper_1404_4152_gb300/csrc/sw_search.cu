// Search orchestration: one query, or a batch, against a loaded database.
//
// Everything is enqueued on one stream in the order of the workflow of
// Section III (Fig. 2): the persistent wavefront kernel stages the query
// profile per pass (stage (i)) and aligns every database sequence (stage
// (ii)); pairs whose 16-bit lanes reached the saturation threshold are
// rescored exactly in int32 (the paper avoids this with 32-bit lanes,
// Section III); the top-k selection replaces the full sort of stage (iv).
//
// A batch packs two queries into the two 16-bit halves of every lane (their
// profile entries are then already packed), pairs queries of similar length,
// runs all pairs in one persistent launch whose work items are (database
// chunk, query pair), and is replayed from a captured CUDA graph when the same
// batch shape is searched again.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <numeric>
#include <vector>

#include "sw.h"
#include "sw_db.h"
#include "sw_internal.h"

using namespace swgb;

namespace {

constexpr int kTopkBlocks = 256;
constexpr uint64_t kRescoreScratch = 256ull << 20;
constexpr int kBlockRouteCounter = 4;  // d_counters word of the block route's work counter

const int kShortR[] = {8, 12, 16, 20, 24};

// The cost of one pass of 8 R query rows: the autotuner's time per row and residue, else
// alu_per_row ALU instructions per row plus about 8 per step.
double pass_cost(const sw_db* db, int mode, int R, double alu_per_row) {
    const double measured = db->tuned ? db->tuning.ns_per_row_residue[mode][(R - 8) / 4] : 0.0;
    return measured > 0 ? measured * kShortT * R : (alu_per_row * R + 8.0);
}

// The cost of an m-row query with R rows per thread: whole passes, except that the ring
// kernel with kRingLastR rows per thread ends with one shorter pass (ring_last_rows).
double rows_cost(const sw_db* db, int mode, uint32_t m, int R, double alu_per_row) {
    const uint32_t TR = (uint32_t)kShortT * R;
    if (mode == KernelChoice::kPairRing && R == kRingLastR) {
        const int last = ring_last_rows(m % TR);
        return (double)(m / TR) * pass_cost(db, mode, R, alu_per_row) +
               (last ? pass_cost(db, mode, last, alu_per_row) : 0.0);
    }
    return (double)((m + TR - 1) / TR) * pass_cost(db, mode, R, alu_per_row);
}

// The rows per thread of the least total cost over the items (padded rows included).
int choose_R(const sw_db* db, int mode, const std::vector<uint32_t>& lengths, double alu_per_row) {
    int bestR = 16;
    double best = 1e300;
    for (int i = 0; i < (int)(sizeof kShortR / sizeof kShortR[0]); ++i) {
        const int R = kShortR[i];
        const double measured = db->tuned ? db->tuning.ns_per_row_residue[mode][i] : 0.0;
        double cost = 0;
        for (uint32_t m : lengths) cost += rows_cost(db, mode, m, R, alu_per_row);
        if (measured <= 0 && R == 16) cost *= 0.97;
        if (cost < best) { best = cost; bestR = R; }
    }
    return bestR;
}

bool use_int32(const sw_db* db, int32_t alpha, int32_t beta) {
    return (db->flags & SW_DB_FLAG_FORCE_INT32) || (int64_t)alpha + beta > 32768;
}

// One query against pairs of database sequences: the score-profile ring
// unless the autotuner measured the int8 query profile faster on this GPU.
KernelChoice single_choice(const sw_db* db, uint32_t qlen, bool i32) {
    if (i32) return KernelChoice{KernelChoice::kInt32, 16};
    const KernelChoice qp{KernelChoice::kPairDb, choose_R(db, 0, {qlen}, 4.5)};
    if (db->flags & SW_DB_FLAG_QUERY_PROFILE) return qp;
    const KernelChoice ring{KernelChoice::kPairRing, choose_R(db, 3, {qlen}, 3.9)};
    if (!db->tuned) return ring;
    return rows_cost(db, KernelChoice::kPairDb, qlen, qp.R, 4.5) <
                   rows_cost(db, KernelChoice::kPairRing, qlen, ring.R, 3.9)
               ? qp
               : ring;
}

// Two halves per slot, each the longest unit plus the wavefront's slack.
uint64_t bstride_for(uint32_t max_len) {
    const uint64_t half = ((uint64_t)max_len + boundary_slack() + 3) & ~3ull;
    return 2 * half;
}

int occupancy_max(const std::vector<KernelChoice>& cs) {
    int m = 0;
    for (auto& c : cs) m = std::max(m, wavefront_occupancy(c, nullptr));
    return std::max(m, 1);
}

std::vector<KernelChoice> all_choices() {
    std::vector<KernelChoice> v;
    for (int R : kShortR) {
        v.push_back(KernelChoice{KernelChoice::kPairDb, R});
        v.push_back(KernelChoice{KernelChoice::kQueryPair, R});
        v.push_back(KernelChoice{KernelChoice::kPairRing, R});
    }
    v.push_back(KernelChoice{KernelChoice::kInt32, 16});
    return v;
}

cudaEvent_t take_event(sw_db* db) {
    if (!db->event_pool.empty()) {
        cudaEvent_t e = db->event_pool.back();
        db->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Brackets one phase with events when the handle is profiled.
// Also an NVTX range named after the phase on the host thread that enqueues it (for
// timeline tools; free when none is attached).
struct PhaseTimer {
    sw_db* db;
    int phase;
    cudaStream_t st;
    uint64_t cells;
    cudaEvent_t a = nullptr;
    bool open = true;
    PhaseTimer(sw_db* d, int p, cudaStream_t s, uint64_t c) : db(d), phase(p), st(s), cells(c) {
        static const char* const kNames[4] = {"sw.wavefront", "sw.rescore_int32", "sw.topk",
                                              "sw.batch"};
        nvtxRangePushA(kNames[p & 3]);
        if (db->flags & SW_DB_FLAG_PROFILE) {
            a = take_event(db);
            cudaEventRecord(a, st);
        }
    }
    void done() {
        if (open) {
            nvtxRangePop();
            open = false;
        }
        if (!a) return;
        cudaEvent_t b = take_event(db);
        cudaEventRecord(b, st);
        db->pending.push_back({phase, a, b, cells});
        a = nullptr;
    }
    ~PhaseTimer() {
        if (open) nvtxRangePop();
    }
};

}  // namespace

// Grow-only device buffer owned by the handle.
sw_status ensure(sw_db* db, DevBuf& b, size_t bytes, const char* what) {
    if (b.cap >= bytes && b.p) return SW_OK;
    if (b.p) {
        db_free(db, b.p, b.cap);
        b.p = nullptr;
        b.cap = 0;
    }
    size_t cap = std::max<size_t>(bytes, 256);
    cap = (cap + 255) & ~(size_t)255;
    void* p = nullptr;
    cudaError_t e = db_malloc(db, &p, cap);
    if (e != cudaSuccess) return cuda_fail(e, what);
    b.p = p;
    b.cap = cap;
    return SW_OK;
}

void set_block_route(sw_db* db, uint32_t opt_threshold) {
    uint64_t t = opt_threshold;
    if (t == 0)  // automatic: a pair unit (2 x L residues) longer than one warp's share of
                 // the search (total residues / (16 warps x SMs)) would finish after the rest
        t = std::max<uint64_t>(4ull * db->long_threshold,
                               db->total_residues / (32ull * (uint64_t)std::max(db->nsm, 1)));
    t = std::max<uint64_t>(t, db->long_threshold);
    db->block_threshold = (uint32_t)std::min<uint64_t>(t, 0xffffffffu);
    uint64_t n = 0;  // sequences above it: the first n sorted positions
    for (uint32_t L : db->seq_len) n += L > db->block_threshold;
    db->n_block_tiles = std::min<uint64_t>((n + kTileSeqs - 1) / kTileSeqs, db->n_long_tiles);
}

sw_status sw_db_prepare_search(sw_db* db) {
    sw_status st;
    {
        cudaError_t e;
        if ((e = cudaStreamCreateWithFlags(&db->blk_stream, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&db->blk_fork, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&db->blk_join, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(e, "block-wavefront stream");
    }
    if ((st = db_alloc(db, (void**)&db->d_counters, 256, "search counters"))) return st;
    if (cudaMemset(db->d_counters, 0, 256) != cudaSuccess)  // includes the error word
        return fail(SW_ERR_CUDA, "search counters: memset failed");
    const int warps = wavefront_block_threads() / 32;
    db->grid_short = db->nsm * occupancy_max(all_choices());
    if (db->n_long_tiles < db->n_tiles) {
        db->bstride_short = bstride_for(db->max_len_short);
        const uint64_t slots = (uint64_t)db->grid_short * warps * (32 / kShortT);
        if ((st = db_alloc(db, (void**)&db->d_bnd_short, slots * db->bstride_short * sizeof(uint2),
                           "boundary rows (short)")))
            return st;
    }
    if (db->n_long_tiles) {
        db->bstride_long = bstride_for(db->max_len_long);
        const uint64_t slots = (uint64_t)db->grid_short * warps * (32 / kLongT);
        if ((st = db_alloc(db, (void**)&db->d_bnd_long, slots * db->bstride_long * sizeof(uint2),
                           "boundary rows (long)")))
            return st;
    }
    // rescoring: one block per pair, as many per SM as fit (its score rings take most of
    // the shared memory), each with one scratch row (bstride entries), as many as
    // kRescoreScratch bytes allow
    db->bstride_rescore = bstride_for(std::max(4u, (db->max_len + 3u) & ~3u));
    {
        const uint64_t per_block = db->bstride_rescore * sizeof(uint2);
        const uint64_t fit = ((uint64_t)kRescoreScratch) / std::max<uint64_t>(per_block, 1);
        db->grid_rescore = (int)std::max<uint64_t>(
            1, std::min<uint64_t>(fit, (uint64_t)db->nsm * rescore_blocks_per_sm(db->alphabet)));
    }
    if ((st = db_alloc(db, (void**)&db->d_bnd_rescore,
                       (uint64_t)db->grid_rescore * db->bstride_rescore * sizeof(uint2),
                       "boundary rows (rescoring)")))
        return st;
    if ((st = db_alloc(db, (void**)&db->d_flags2, db->n_seqs * sizeof(uint2), "rescoring list")))
        return st;
    db->topk_nq = 1;
    if ((st = db_alloc(db, &db->d_topk, topk_scratch_bytes(1, SW_MAX_TOP_K, kTopkBlocks),
                       "top-k scratch")))
        return st;
    topk_scratch_carve(db->d_topk, 1, SW_MAX_TOP_K, kTopkBlocks, &db->topk);
    db->query_cap = 1u << 16;
    if ((st = db_alloc(db, (void**)&db->d_query, db->query_cap, "query staging")) ||
        (st = db_alloc(db, (void**)&db->d_matrix, SW_MAX_ALPHABET * SW_MAX_ALPHABET,
                       "matrix staging")) ||
        (st = db_alloc(db, (void**)&db->d_top_scores, SW_MAX_TOP_K * 4, "top-k scores")) ||
        (st = db_alloc(db, (void**)&db->d_top_index, SW_MAX_TOP_K * 8, "top-k indices")))
        return st;
    return SW_OK;
}

extern "C" sw_status sw_db_get_profile(sw_db* db, sw_profile* out) {
    clear_error();
    if (!db || !out) return fail(SW_ERR_INVALID_ARG, "sw_db_get_profile: NULL argument");
    for (auto& t : db->pending) {
        cudaError_t e = cudaEventSynchronize(t.b);
        if (e != cudaSuccess) return cuda_fail(e, "sw_db_get_profile");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t.a, t.b);
        db->prof_ms[t.phase] += ms;
        db->prof_calls[t.phase] += 1;
        db->prof_cells[t.phase] += t.cells;
        db->event_pool.push_back(t.a);
        db->event_pool.push_back(t.b);
    }
    db->pending.clear();
    out->launches = db->launches;
    for (int p = 0; p < 4; ++p) {
        out->calls[p] = db->prof_calls[p];
        out->cells[p] = db->prof_cells[p];
        out->ms[p] = db->prof_ms[p];
    }
    return SW_OK;
}

extern "C" sw_status sw_db_reset_profile(sw_db* db) {
    sw_profile tmp;
    sw_status st = sw_db_get_profile(db, &tmp);
    if (st) return st;
    db->launches = 0;
    for (int p = 0; p < 4; ++p) { db->prof_calls[p] = 0; db->prof_cells[p] = 0; db->prof_ms[p] = 0; }
    return SW_OK;
}

namespace {

WavefrontArgs base_args(sw_db* db, const int8_t* d_matrix, int32_t alpha, int32_t beta,
                        int32_t* d_scores, uint64_t stride, uint32_t units_per_tile) {
    WavefrontArgs a{};
    a.tile_data = db->d_tile_data;
    a.tile_off = db->d_tile_off;
    a.tile_len = db->d_tile_len;
    a.sorted_ids = db->d_sorted;
    a.matrix = d_matrix;
    a.alphabet = db->alphabet;
    a.alpha = alpha;
    a.beta = beta;
    a.scores = d_scores;
    a.score_stride = stride;
    // tiles [0, n_block_tiles) are the block wavefront's (fork_block_route)
    a.bin[0].first_unit = db->n_block_tiles * units_per_tile;
    a.bin[0].n_units = (db->n_long_tiles - db->n_block_tiles) * units_per_tile;
    a.bin[0].boundary = db->d_bnd_long;
    a.bin[0].bstride = db->bstride_long;
    a.bin[1].first_unit = db->n_long_tiles * units_per_tile;
    a.bin[1].n_units = (db->n_tiles - db->n_long_tiles) * units_per_tile;
    a.bin[1].boundary = db->d_bnd_short;
    a.bin[1].bstride = db->bstride_short;
    a.work_counter = db->d_counters + 0;
    a.flag_count = db->d_counters + 3;
    a.dbg = db->d_counters + kDebugWord;
    return a;
}

RescoreArgs rescore_args(sw_db* db, const int8_t* d_matrix, int32_t alpha, int32_t beta,
                         int32_t* d_scores, uint64_t stride) {
    RescoreArgs r{};
    r.tile_data = db->d_tile_data;
    r.tile_off = db->d_tile_off;
    r.tile_len = db->d_tile_len;
    r.sorted_ids = db->d_sorted;
    r.count = db->d_counters + 3;
    r.matrix = d_matrix;
    r.alphabet = db->alphabet;
    r.alpha = alpha;
    r.beta = beta;
    r.scores = d_scores;
    r.score_stride = stride;
    r.boundary = db->d_bnd_rescore;
    r.bstride = db->bstride_rescore;
    r.work_counter = db->d_counters + 2;
    r.dbg = db->d_counters + kDebugWord;
    return r;
}

// The sequences of the block route (the very long ones: whole tiles at the front of the
// sorted order) for nq queries: one block of 8 warps per (query, sequence) running the
// multi-warp wavefront of sw_blockwave.cuh in int32, on the handle's second stream beside
// the search kernel; join_block_route makes `stream` wait for it. r carries the query
// (single_qlen, or qoff / qlen per query row) and outputs.
sw_status fork_block_route(sw_db* db, RescoreArgs r, uint32_t nq, cudaStream_t stream,
                           bool* forked) {
    *forked = false;
    if (!db->n_block_tiles || nq == 0) return SW_OK;
    const uint64_t n = db->n_block_tiles * kTileSeqs;
    r.list = nullptr;
    r.count = nullptr;
    r.cap = 0;
    r.dense_n = (uint32_t)n;
    r.dense_count = (uint32_t)std::min<uint64_t>(n * nq, 0xffffffffu);
    r.work_counter = db->d_counters + kBlockRouteCounter;
    const int grid = (int)std::min<uint64_t>((uint64_t)db->grid_rescore, r.dense_count);
    cudaError_t e;
    if ((e = cudaEventRecord(db->blk_fork, stream)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(db->blk_stream, db->blk_fork, 0)) != cudaSuccess ||
        (e = launch_rescore(r, grid, db->blk_stream)) != cudaSuccess ||
        (e = cudaEventRecord(db->blk_join, db->blk_stream)) != cudaSuccess)
        return cuda_fail(e, "search: block-wavefront route");
    *forked = true;
    return SW_OK;
}

sw_status join_block_route(sw_db* db, bool forked, cudaStream_t stream) {
    if (!forked) return SW_OK;
    cudaError_t e = cudaStreamWaitEvent(stream, db->blk_join, 0);
    return e == cudaSuccess ? SW_OK : cuda_fail(e, "search: block-wavefront join");
}

int grid_for(const sw_db* db, const KernelChoice& kc) {
    const int occ = std::max(1, wavefront_occupancy(kc, nullptr));
    return std::max(1, std::min(db->grid_short, db->nsm * occ));
}

}  // namespace

// Enqueue one full single-query search on `stream`. Scores land in d_scores
// (original order).
sw_status enqueue_search(sw_db* db, const uint8_t* d_query, uint32_t qlen, const int8_t* d_matrix,
                         int32_t alpha, int32_t beta, uint32_t top_k, int32_t* d_scores,
                         int32_t* d_top_scores, uint64_t* d_top_index, cudaStream_t stream) {
    cudaError_t e;
    const bool i32 = use_int32(db, alpha, beta);
    if ((e = cudaMemsetAsync(db->d_counters, 0, 64, stream)) != cudaSuccess)
        return cuda_fail(e, "search: counter reset");
    const KernelChoice kc = single_choice(db, qlen, i32);
    {
        WavefrontArgs a = base_args(db, d_matrix, alpha, beta, d_scores, db->n_seqs,
                                    units_per_tile(kc));
        a.query = d_query;
        a.qlen = qlen;
        a.flag_list = db->d_flags2;
        a.flag_cap = (uint32_t)std::min<uint64_t>(db->n_seqs, 0xffffffffu);
        PhaseTimer pt(db, 0, stream, (uint64_t)qlen * db->total_residues);
        RescoreArgs rb = rescore_args(db, d_matrix, alpha, beta, d_scores, db->n_seqs);
        rb.query = d_query;
        rb.single_qlen = qlen;
        bool forked = false;
        sw_status st = fork_block_route(db, rb, 1, stream, &forked);
        if (st) return st;
        if ((e = launch_wavefront(kc, a, grid_for(db, kc), stream)) != cudaSuccess)
            return cuda_fail(e, "search: wavefront kernel");
        if ((st = join_block_route(db, forked, stream))) return st;
        pt.done();
        db->launches += 1 + (forked ? 1 : 0);
    }
    if (!i32) {
        RescoreArgs r = rescore_args(db, d_matrix, alpha, beta, d_scores, db->n_seqs);
        r.list = db->d_flags2;
        r.cap = (uint32_t)std::min<uint64_t>(db->n_seqs, 0xffffffffu);
        r.query = d_query;
        r.single_qlen = qlen;
        PhaseTimer pt(db, 1, stream, 0);
        if ((e = launch_rescore(r, db->grid_rescore, stream)) != cudaSuccess)
            return cuda_fail(e, "search: int32 rescoring kernel");
        pt.done();
        db->launches += 1;
    }
    if (top_k) {
        PhaseTimer pt(db, 2, stream, 0);
        if ((e = launch_topk(d_scores, db->n_seqs, db->n_seqs, 1, top_k, db->topk, d_top_scores,
                             d_top_index, stream)) != cudaSuccess)
            return cuda_fail(e, "search: top-k");
        pt.done();
        db->launches += topk_launch_count();
    }
    return SW_OK;
}

// ---------------------------------------------------------------------------
// batches
// ---------------------------------------------------------------------------

namespace {

// Pairs grouped by the rows per thread each runs best at; group g is pairs
// [group_first[g], group_first[g + 1]) with group_R[g] rows per thread.
constexpr int kMaxGroups = 5;   // one per rows-per-thread choice
constexpr int kGroupCounter0 = 16;  // the groups' work counters: d_counters[16 ..]

struct BatchPlan {
    std::vector<QueryPair> pairs;
    std::vector<QueryPair> singles;  // queries that run alone in the ring (len_b = 0)
    std::vector<uint64_t> qoff;
    std::vector<uint32_t> qlen;
    std::vector<int> group_R;
    std::vector<uint32_t> group_first;
    uint64_t cells = 0;
    uint32_t flag_cap = 0;
};

// Pair queries of similar length (longest first) and pick the kernel shape.
BatchPlan plan_batch(const sw_db* db, uint32_t nq, const uint64_t* qoffsets) {
    BatchPlan pl;
    pl.qoff.assign(qoffsets, qoffsets + nq);
    pl.qlen.resize(nq);
    for (uint32_t q = 0; q < nq; ++q) pl.qlen[q] = (uint32_t)(qoffsets[q + 1] - qoffsets[q]);
    std::vector<uint32_t> order(nq);
    std::iota(order.begin(), order.end(), 0u);
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t x, uint32_t y) { return pl.qlen[x] > pl.qlen[y]; });
    std::vector<uint32_t> item_len;
    for (uint32_t i = 0; i < nq; i += 2) {
        QueryPair p{};
        const uint32_t qa = order[i];
        p.off_a = pl.qoff[qa];
        p.len_a = pl.qlen[qa];
        p.q_a = qa;
        if (i + 1 < nq) {
            const uint32_t qb = order[i + 1];
            p.off_b = pl.qoff[qb];
            p.len_b = pl.qlen[qb];
            p.q_b = qb;
        } else {
            p.off_b = p.off_a;
            p.len_b = 0;
            p.q_b = 0xffffffffu;
        }
        // a pair runs its longer query's rows for both halves of the lanes; where that
        // costs more than the two queries alone in the score-profile ring (one query
        // against two sequences, 24 rows per lane and a short last pass), or where a
        // query has no partner, they run alone there
        const bool ring_ok = !(db->flags & SW_DB_FLAG_QUERY_PROFILE);
        if (ring_ok && (p.len_b == 0 ||
                        !pair_pays(db, p.len_a, p.len_b, KernelChoice{KernelChoice::kPairRing, kRingLastR}))) {
            QueryPair a = p;
            a.off_b = a.off_a;
            a.len_b = 0;
            a.q_b = 0xffffffffu;
            pl.singles.push_back(a);
            if (p.len_b) {
                QueryPair b{};
                b.off_a = b.off_b = p.off_b;
                b.len_a = p.len_b;
                b.q_a = p.q_b;
                b.q_b = 0xffffffffu;
                pl.singles.push_back(b);
            }
            continue;
        }
        pl.pairs.push_back(p);
        item_len.push_back(std::max(p.len_a, p.len_b));
    }
    // each pair takes the rows per thread of its least padded cost; pairs of one choice
    // run in one launch (longest first inside each, as sorted)
    std::vector<int> best_R(pl.pairs.size());
    for (size_t i = 0; i < pl.pairs.size(); ++i) best_R[i] = choose_R(db, 1, {item_len[i]}, 3.5);
    std::vector<QueryPair> grouped;
    pl.group_first.push_back(0);
    for (int R : kShortR) {
        for (size_t i = 0; i < pl.pairs.size(); ++i)
            if (best_R[i] == R) grouped.push_back(pl.pairs[i]);
        if (grouped.size() > pl.group_first.back()) {
            pl.group_R.push_back(R);
            pl.group_first.push_back((uint32_t)grouped.size());
        }
    }
    pl.pairs.swap(grouped);
    for (uint32_t q = 0; q < nq; ++q) pl.cells += (uint64_t)pl.qlen[q] * db->total_residues;
    pl.flag_cap = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(db->n_seqs, 1u << 20), 1u << 26);
    return pl;
}

sw_status upload_plan(sw_db* db, const BatchPlan& pl, cudaStream_t stream) {
    sw_status st;
    std::vector<QueryPair> items(pl.pairs);
    items.insert(items.end(), pl.singles.begin(), pl.singles.end());
    const size_t np = items.size(), nq = pl.qlen.size();
    if ((st = ensure(db, db->b_pairs, np * sizeof(QueryPair), "batch pairs")) ||
        (st = ensure(db, db->b_qoff, nq * 8, "batch query offsets")) ||
        (st = ensure(db, db->b_qlen, nq * 4, "batch query lengths")) ||
        (st = ensure(db, db->b_flags, (size_t)pl.flag_cap * sizeof(uint2), "batch rescoring list")) ||
        (st = ensure(db, db->b_topk, topk_scratch_bytes((uint32_t)nq, SW_MAX_TOP_K, kTopkBlocks),
                     "batch top-k scratch")))
        return st;
    cudaError_t e;
    // pageable sources: each copy has consumed its host data when the call returns
    if ((e = cudaMemcpyAsync(db->b_pairs.p, items.data(), np * sizeof(QueryPair),
                             cudaMemcpyHostToDevice, stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(db->b_qoff.p, pl.qoff.data(), nq * 8, cudaMemcpyHostToDevice,
                             stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(db->b_qlen.p, pl.qlen.data(), nq * 4, cudaMemcpyHostToDevice,
                             stream)) != cudaSuccess)
        return cuda_fail(e, "batch: plan upload");
    return SW_OK;
}

// The kernels of one batch (capturable: memsets and launches only).
sw_status launch_batch(sw_db* db, const BatchPlan& pl, const uint8_t* d_queries,
                       const int8_t* d_matrix, int32_t alpha, int32_t beta, uint32_t top_k,
                       int32_t* d_scores, int32_t* d_top_scores, uint64_t* d_top_index,
                       cudaStream_t stream) {
    cudaError_t e;
    const uint32_t nq = (uint32_t)pl.qlen.size();
    // the query-pair groups' counters, then the ring launch's
    static_assert(kGroupCounter0 + kMaxGroups + 1 <= kDebugWord, "counter words");
    if ((e = cudaMemsetAsync(db->d_counters, 0, (kGroupCounter0 + kMaxGroups + 1) * 4, stream)) !=
        cudaSuccess)
        return cuda_fail(e, "batch: counter reset");
    WavefrontArgs a = base_args(db, d_matrix, alpha, beta, d_scores, db->n_seqs, kTileSeqs);
    a.query = d_queries;
    a.flag_list = (uint2*)db->b_flags.p;
    a.flag_cap = pl.flag_cap;
    RescoreArgs rb = rescore_args(db, d_matrix, alpha, beta, d_scores, db->n_seqs);
    rb.query = d_queries;
    rb.qoff = (const uint64_t*)db->b_qoff.p;
    rb.qlen = (const uint32_t*)db->b_qlen.p;
    bool forked = false;
    sw_status st = fork_block_route(db, rb, nq, stream, &forked);
    if (st) return st;
    for (size_t g = 0; g < pl.group_R.size(); ++g) {  // one launch per rows-per-thread group
        const KernelChoice kc{KernelChoice::kQueryPair, pl.group_R[g]};
        a.pairs = (const QueryPair*)db->b_pairs.p + pl.group_first[g];
        a.n_pairs = pl.group_first[g + 1] - pl.group_first[g];
        a.work_counter = db->d_counters + kGroupCounter0 + g;
        if ((e = launch_wavefront(kc, a, grid_for(db, kc), stream)) != cudaSuccess)
            return cuda_fail(e, "batch: wavefront kernel");
    }
    if (!pl.singles.empty()) {  // the queries that run alone: one ring launch
        const KernelChoice kr{KernelChoice::kPairRing, kRingLastR};
        WavefrontArgs ar = base_args(db, d_matrix, alpha, beta, d_scores, db->n_seqs,
                                     units_per_tile(kr));
        ar.query = d_queries;
        ar.flag_list = (uint2*)db->b_flags.p;
        ar.flag_cap = pl.flag_cap;
        ar.pairs = (const QueryPair*)db->b_pairs.p + pl.pairs.size();
        ar.n_pairs = (uint32_t)pl.singles.size();
        ar.work_counter = db->d_counters + kGroupCounter0 + kMaxGroups;
        if ((e = launch_wavefront(kr, ar, grid_for(db, kr), stream)) != cudaSuccess)
            return cuda_fail(e, "batch: ring kernel");
    }
    if ((st = join_block_route(db, forked, stream))) return st;
    RescoreArgs r = rescore_args(db, d_matrix, alpha, beta, d_scores, db->n_seqs);
    r.list = (const uint2*)db->b_flags.p;
    r.cap = pl.flag_cap;
    r.query = d_queries;
    r.qoff = (const uint64_t*)db->b_qoff.p;
    r.qlen = (const uint32_t*)db->b_qlen.p;
    if ((e = launch_rescore(r, db->grid_rescore, stream)) != cudaSuccess)
        return cuda_fail(e, "batch: int32 rescoring kernel");
    if (top_k) {
        TopkScratch ts;
        topk_scratch_carve(db->b_topk.p, nq, SW_MAX_TOP_K, kTopkBlocks, &ts);
        if ((e = launch_topk(d_scores, db->n_seqs, db->n_seqs, nq, top_k, ts, d_top_scores,
                             d_top_index, stream)) != cudaSuccess)
            return cuda_fail(e, "batch: top-k");
    }
    return SW_OK;
}

// The plan's work items as uploaded: the pairs (grouped), then the queries run alone, each
// as the 64-bit words of its record (for an exact comparison).
std::vector<uint64_t> plan_items(const BatchPlan& pl) {
    std::vector<uint64_t> v;
    for (const auto* list : {&pl.pairs, &pl.singles})
        for (const QueryPair& p : *list) {
            const uint64_t* w = reinterpret_cast<const uint64_t*>(&p);
            v.insert(v.end(), w, w + sizeof(QueryPair) / 8);
        }
    return v;
}

// Graph replay key: everything a captured batch bakes in.
bool same_key(const BatchGraph& g, const BatchPlan& pl, const void* q, const void* m,
              int32_t alpha, int32_t beta, uint32_t k, const void* s, const void* ts,
              const void* ti, cudaStream_t st) {
    return g.exec && g.queries == q && g.matrix == m && g.alpha == alpha && g.beta == beta &&
           g.top_k == k && g.scores == s && g.top_s == ts && g.top_i == ti && g.stream == st &&
           g.qoff == pl.qoff && g.qlen == pl.qlen && g.group_R == pl.group_R &&
           g.group_first == pl.group_first && g.items == plan_items(pl);
}

}  // namespace

// Enqueue a batch on `stream`, replaying the captured graph when the batch
// shape and buffers match the previous call.
sw_status enqueue_batch(sw_db* db, uint32_t nq, const uint8_t* d_queries,
                        const uint64_t* qoffsets, const int8_t* d_matrix, int32_t alpha,
                        int32_t beta, uint32_t top_k, int32_t* d_scores, int32_t* d_top_scores,
                        uint64_t* d_top_index, cudaStream_t stream, BatchInfo* info) {
    if (use_int32(db, alpha, beta)) {
        // wide penalties or forced int32: one int32 search per query
        for (uint32_t q = 0; q < nq; ++q) {
            sw_status st = enqueue_search(
                db, d_queries + qoffsets[q], (uint32_t)(qoffsets[q + 1] - qoffsets[q]), d_matrix,
                alpha, beta, top_k, d_scores + (uint64_t)q * db->n_seqs,
                top_k ? d_top_scores + (uint64_t)q * top_k : nullptr,
                top_k ? d_top_index + (uint64_t)q * top_k : nullptr, stream);
            if (st) return st;
        }
        if (info) info->flag_cap = 0;
        return SW_OK;
    }
    BatchPlan pl = plan_batch(db, nq, qoffsets);
    sw_status st = upload_plan(db, pl, stream);
    if (st) return st;
    if (info) {
        info->cells = pl.cells;
        info->flag_cap = pl.flag_cap;
    }
    cudaError_t e;
    BatchGraph& g = db->graph;
    const bool hit = same_key(g, pl, d_queries, d_matrix, alpha, beta, top_k, d_scores,
                              d_top_scores, d_top_index, stream);
    if (!hit) {
        if (g.exec) {
            cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        if ((e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return cuda_fail(e, "batch: begin capture");
        st = launch_batch(db, pl, d_queries, d_matrix, alpha, beta, top_k, d_scores, d_top_scores,
                          d_top_index, stream);
        e = cudaStreamEndCapture(stream, &graph);
        if (st) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return cuda_fail(e, "batch: end capture");
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            g.exec = nullptr;
            return cuda_fail(e, "batch: graph instantiation");
        }
        g.queries = d_queries;
        g.matrix = d_matrix;
        g.alpha = alpha;
        g.beta = beta;
        g.top_k = top_k;
        g.scores = d_scores;
        g.top_s = d_top_scores;
        g.top_i = d_top_index;
        g.stream = stream;
        g.qoff = pl.qoff;
        g.qlen = pl.qlen;
        g.group_R = pl.group_R;
        g.group_first = pl.group_first;
        g.items = plan_items(pl);
        g.kernels = (uint32_t)pl.group_R.size() + 1 + (top_k ? topk_launch_count() : 0) +
                    (db->n_block_tiles ? 1 : 0) + (pl.singles.empty() ? 0 : 1);
    }
    PhaseTimer pt(db, 3, stream, pl.cells);
    if ((e = cudaGraphLaunch(g.exec, stream)) != cudaSuccess)
        return cuda_fail(e, "batch: graph launch");
    pt.done();
    db->launches += g.kernels;
    return SW_OK;
}

// Rows per thread of the query-pair kernel for pairs whose longer queries have these
// lengths (the server's waves).
int choose_pair_R(const sw_db* db, const std::vector<uint32_t>& lengths) {
    return choose_R(db, KernelChoice::kQueryPair, lengths, 3.5);
}

// Whether two queries (la >= lb rows) cost less as one pair in the query-pair kernel,
// which runs la rows for both, than one after the other in the kernel `alone`.
bool pair_pays(const sw_db* db, uint32_t la, uint32_t lb, swgb::KernelChoice alone) {
    const int R = choose_R(db, KernelChoice::kQueryPair, {la}, 3.5);
    const double pair = 2.0 * rows_cost(db, KernelChoice::kQueryPair, la, R, 3.5);
    const double apart = rows_cost(db, alone.mode, la, alone.R, 3.9) +
                         rows_cost(db, alone.mode, lb, alone.R, 3.9);
    return pair <= apart;
}

sw_status swgb::check_common(const sw_db* db, uint32_t qlen, int32_t alpha, int32_t beta,
                       uint32_t top_k, const char* fn) {
    if (!db) return fail(SW_ERR_INVALID_ARG, "%s: db is NULL", fn);
    if (qlen == 0) return fail(SW_ERR_INVALID_ARG, "%s: qlen must be >= 1", fn);
    if (alpha < 0 || beta < 0 || alpha > 32767 || beta > 32767)
        return fail(SW_ERR_INVALID_ARG, "%s: alpha and beta must lie in [0, 32767]", fn);
    if (top_k > SW_MAX_TOP_K)
        return fail(SW_ERR_INVALID_ARG, "%s: top_k %u exceeds %u", fn, top_k, SW_MAX_TOP_K);
    return SW_OK;
}

sw_status swgb::stage_query(sw_db* db, const uint8_t* query, uint32_t qlen, const int8_t* matrix) {
    cudaError_t e;
    if (qlen > db->query_cap) {
        void* p = nullptr;
        uint32_t cap = db->query_cap;
        while (cap < qlen) cap *= 2;
        if ((e = db_malloc(db, &p, cap)) != cudaSuccess) return cuda_fail(e, "query staging");
        for (auto& a : db->allocs)
            if (a.first == db->d_query) { db_free(db, a.first, a.second); a = {p, cap}; }
        db->d_query = (uint8_t*)p;
        db->query_cap = cap;
    }
    const size_t mbytes = (size_t)db->alphabet * db->alphabet;
    if ((e = cudaMemcpyAsync(db->d_query, query, qlen, cudaMemcpyHostToDevice, db->stream)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(db->d_matrix, matrix, mbytes, cudaMemcpyHostToDevice, db->stream)) !=
            cudaSuccess)
        return cuda_fail(e, "copy query/matrix to device");
    return SW_OK;
}

sw_status swgb::validate_host_query(const sw_db* db, const uint8_t* query, uint32_t qlen,
                              const int8_t* matrix, const char* fn) {
    if (!query || !matrix) return fail(SW_ERR_INVALID_ARG, "%s: query or matrix is NULL", fn);
    for (uint32_t i = 0; i < qlen; ++i)
        if (query[i] >= db->alphabet)
            return fail(SW_ERR_INVALID_ARG, "%s: query code %u at %u is not below alphabet %u", fn,
                        query[i], i, db->alphabet);
    return SW_OK;
}

namespace {

sw_status check_batch(const sw_db* db, uint32_t nq, const uint64_t* qoffsets, int32_t alpha,
                      int32_t beta, uint32_t top_k, const char* fn) {
    if (!db) return fail(SW_ERR_INVALID_ARG, "%s: db is NULL", fn);
    if (!qoffsets) return fail(SW_ERR_INVALID_ARG, "%s: NULL query offsets", fn);
    for (uint32_t q = 0; q < nq; ++q) {
        if (qoffsets[q + 1] <= qoffsets[q])
            return fail(SW_ERR_INVALID_ARG, "%s: query %u is empty or offsets not ascending", fn, q);
        if (qoffsets[q + 1] - qoffsets[q] > 0x7fffffffull)
            return fail(SW_ERR_INVALID_ARG, "%s: query %u is too long", fn, q);
    }
    return check_common(db, 1, alpha, beta, top_k, fn);
}

}  // namespace

extern "C" sw_status sw_search(sw_db* db, const uint8_t* query, uint32_t qlen,
                               const int8_t* matrix, int32_t alpha, int32_t beta, uint32_t top_k,
                               int32_t* scores, int32_t* top_scores, uint64_t* top_index,
                               uint32_t* n_top, sw_stats* stats) {
    clear_error();
    const auto t0 = std::chrono::steady_clock::now();
    sw_status st;
    if ((st = check_common(db, qlen, alpha, beta, top_k, "sw_search"))) return st;
    if ((st = validate_host_query(db, query, qlen, matrix, "sw_search"))) return st;
    if (top_k && (!top_scores || !top_index))
        return fail(SW_ERR_INVALID_ARG, "sw_search: top_k > 0 needs top_scores and top_index");
    DeviceScope scope(db->device);
    if ((st = stage_query(db, query, qlen, matrix))) return st;
    cudaError_t e;
    cudaEventRecord(db->ev_t0, db->stream);
    st = enqueue_search(db, db->d_query, qlen, db->d_matrix, alpha, beta, top_k, db->d_scores,
                        db->d_top_scores, db->d_top_index, db->stream);
    if (st) return st;
    cudaEventRecord(db->ev_t1, db->stream);
    const uint32_t kk = (uint32_t)std::min<uint64_t>(top_k, db->n_seqs);
    e = cudaSuccess;
    if (scores)
        e = cudaMemcpyAsync(scores, db->d_scores, db->n_seqs * 4, cudaMemcpyDeviceToHost,
                            db->stream);
    if (e == cudaSuccess && kk)
        e = cudaMemcpyAsync(top_scores, db->d_top_scores, kk * 4, cudaMemcpyDeviceToHost,
                            db->stream);
    if (e == cudaSuccess && kk)
        e = cudaMemcpyAsync(top_index, db->d_top_index, kk * 8, cudaMemcpyDeviceToHost,
                            db->stream);
    uint32_t nflag = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&nflag, db->d_counters + 3, 4, cudaMemcpyDeviceToHost, db->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(db->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sw_search");
    if (n_top) *n_top = kk;
    if (stats) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, db->ev_t0, db->ev_t1);
        stats->cells = (uint64_t)qlen * db->total_residues;
        stats->recomputed = nflag;
        stats->kernel_ms = ms;
        stats->total_ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                .count();
    }
    return SW_OK;
}

extern "C" sw_status sw_search_device(sw_db* db, const uint8_t* d_query, uint32_t qlen,
                                      const int8_t* d_matrix, int32_t alpha, int32_t beta,
                                      uint32_t top_k, int32_t* d_scores, int32_t* d_top_scores,
                                      uint64_t* d_top_index, void* stream) {
    clear_error();
    sw_status st;
    if ((st = check_common(db, qlen, alpha, beta, top_k, "sw_search_device"))) return st;
    if (!d_query || !d_matrix)
        return fail(SW_ERR_INVALID_ARG, "sw_search_device: query or matrix is NULL");
    if (top_k && (!d_top_scores || !d_top_index))
        return fail(SW_ERR_INVALID_ARG, "sw_search_device: top_k > 0 needs output buffers");
    DeviceScope scope(db->device);
    return enqueue_search(db, d_query, qlen, d_matrix, alpha, beta, top_k,
                          d_scores ? d_scores : db->d_scores, d_top_scores, d_top_index,
                          (cudaStream_t)stream);
}

extern "C" sw_status sw_search_batch_device(sw_db* db, uint32_t nq, const uint8_t* d_queries,
                                            const uint64_t* qoffsets, const int8_t* d_matrix,
                                            int32_t alpha, int32_t beta, uint32_t top_k,
                                            int32_t* d_scores, int32_t* d_top_scores,
                                            uint64_t* d_top_index, void* stream) {
    clear_error();
    sw_status st;
    if ((st = check_batch(db, nq, qoffsets, alpha, beta, top_k, "sw_search_batch_device")))
        return st;
    if (nq == 0) return SW_OK;
    if (!d_queries || !d_matrix || !d_scores)
        return fail(SW_ERR_INVALID_ARG, "sw_search_batch_device: NULL device buffer");
    if (top_k && (!d_top_scores || !d_top_index))
        return fail(SW_ERR_INVALID_ARG, "sw_search_batch_device: top_k > 0 needs output buffers");
    DeviceScope scope(db->device);
    return enqueue_batch(db, nq, d_queries, qoffsets, d_matrix, alpha, beta, top_k, d_scores,
                         d_top_scores, d_top_index, (cudaStream_t)stream, nullptr);
}

extern "C" sw_status sw_search_batch(sw_db* db, uint32_t nq, const uint8_t* const* queries,
                                     const uint32_t* qlens, const int8_t* matrix, int32_t alpha,
                                     int32_t beta, uint32_t top_k, int32_t* const* scores,
                                     int32_t* top_scores, uint64_t* top_index, uint32_t* n_top,
                                     sw_stats* stats) {
    clear_error();
    const auto t0 = std::chrono::steady_clock::now();
    if (!db) return fail(SW_ERR_INVALID_ARG, "sw_search_batch: db is NULL");
    if (nq == 0) return SW_OK;
    if (!queries || !qlens || !matrix)
        return fail(SW_ERR_INVALID_ARG, "sw_search_batch: NULL queries, lengths or matrix");
    if (top_k && (!top_scores || !top_index))
        return fail(SW_ERR_INVALID_ARG, "sw_search_batch: top_k > 0 needs top_scores and top_index");
    std::vector<uint64_t> off(nq + 1, 0);
    for (uint32_t q = 0; q < nq; ++q) {
        sw_status st;
        if ((st = check_common(db, qlens[q], alpha, beta, top_k, "sw_search_batch"))) return st;
        if ((st = validate_host_query(db, queries[q], qlens[q], matrix, "sw_search_batch")))
            return st;
        off[q + 1] = off[q] + qlens[q];
    }
    DeviceScope scope(db->device);
    sw_status st;
    const size_t kk1 = std::max(top_k, 1u);
    if ((st = ensure(db, db->b_queries, off[nq], "batch queries")) ||
        (st = ensure(db, db->b_scores, (size_t)nq * db->n_seqs * 4, "batch scores")) ||
        (st = ensure(db, db->b_top, (size_t)nq * kk1 * 16, "batch top-k")))
        return st;
    cudaError_t e;
    for (uint32_t q = 0; q < nq; ++q)
        if ((e = cudaMemcpyAsync((uint8_t*)db->b_queries.p + off[q], queries[q], qlens[q],
                                 cudaMemcpyHostToDevice, db->stream)) != cudaSuccess)
            return cuda_fail(e, "sw_search_batch: query upload");
    if ((e = cudaMemcpyAsync(db->d_matrix, matrix, (size_t)db->alphabet * db->alphabet,
                             cudaMemcpyHostToDevice, db->stream)) != cudaSuccess)
        return cuda_fail(e, "sw_search_batch: matrix upload");
    uint64_t* d_ti = (uint64_t*)db->b_top.p;
    int32_t* d_ts = (int32_t*)((char*)db->b_top.p + (size_t)nq * kk1 * 8);
    BatchInfo info{};
    cudaEventRecord(db->ev_t0, db->stream);
    if ((st = enqueue_batch(db, nq, (const uint8_t*)db->b_queries.p, off.data(), db->d_matrix,
                            alpha, beta, top_k, (int32_t*)db->b_scores.p, d_ts, d_ti, db->stream,
                            &info)))
        return st;
    cudaEventRecord(db->ev_t1, db->stream);
    uint32_t nflag = 0;
    if ((e = cudaMemcpyAsync(&nflag, db->d_counters + 3, 4, cudaMemcpyDeviceToHost, db->stream)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(db->stream)) != cudaSuccess)
        return cuda_fail(e, "sw_search_batch");
    if (info.flag_cap && nflag > info.flag_cap) {
        // more saturated pairs than the rescoring list holds: search again in int32
        const uint32_t keep = db->flags;
        db->flags |= SW_DB_FLAG_FORCE_INT32;
        st = enqueue_batch(db, nq, (const uint8_t*)db->b_queries.p, off.data(), db->d_matrix,
                           alpha, beta, top_k, (int32_t*)db->b_scores.p, d_ts, d_ti, db->stream,
                           nullptr);
        db->flags = keep;
        if (st) return st;
        if ((e = cudaStreamSynchronize(db->stream)) != cudaSuccess)
            return cuda_fail(e, "sw_search_batch: int32 retry");
    }
    const uint32_t kk = (uint32_t)std::min<uint64_t>(top_k, db->n_seqs);
    e = cudaSuccess;
    for (uint32_t q = 0; q < nq && e == cudaSuccess; ++q) {
        if (scores && scores[q])
            e = cudaMemcpyAsync(scores[q], (int32_t*)db->b_scores.p + (size_t)q * db->n_seqs,
                                db->n_seqs * 4, cudaMemcpyDeviceToHost, db->stream);
        if (e == cudaSuccess && kk) {
            e = cudaMemcpyAsync(top_scores + (size_t)q * top_k, d_ts + (size_t)q * top_k, kk * 4,
                                cudaMemcpyDeviceToHost, db->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(top_index + (size_t)q * top_k, d_ti + (size_t)q * top_k,
                                    kk * 8, cudaMemcpyDeviceToHost, db->stream);
        }
        if (n_top) n_top[q] = kk;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(db->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sw_search_batch: copy out");
    if (stats) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, db->ev_t0, db->ev_t1);
        uint64_t cells = 0;
        for (uint32_t q = 0; q < nq; ++q) cells += (uint64_t)qlens[q] * db->total_residues;
        stats->cells = cells;
        stats->recomputed = nflag;
        stats->kernel_ms = ms;
        stats->total_ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                .count();
    }
    return SW_OK;
}

extern "C" sw_status sw_db_debug_check(sw_db* db, uint32_t* site) {
    clear_error();
    if (!db || !site) return fail(SW_ERR_INVALID_ARG, "sw_db_debug_check: NULL argument");
    *site = 0;
    if (!kDebugBounds) return SW_OK;
    DeviceScope scope(db->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = cudaMemcpy(site, db->d_counters + kDebugWord, 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(db->d_counters + kDebugWord, 0, 4);
    if (e != cudaSuccess) return cuda_fail(e, "sw_db_debug_check");
    return SW_OK;
}
