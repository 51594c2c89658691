// Search orchestration: one query (or a batch) against a loaded database.
//
// Enqueued on one stream (the long-sequence kernel forks onto a side stream
// and joins back), in the order of the workflow of Section III (Fig. 2):
//   - the wavefront kernel over the long-sequence tiles (warp per pair),
//   - the wavefront kernel over the remaining tiles (8 lanes per pair),
//     both staging the query profile per pass (stage (i)) and aligning
//     (stage (ii)),
//   - int32 rescoring of any sequence whose 16-bit lanes reached the
//     saturation threshold (exactness; the paper avoids this with 32-bit
//     lanes, Section III),
//   - top-k (stage (iv)).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>

#include "sw.h"
#include "sw_db.h"
#include "sw_internal.h"

using namespace swgb;

namespace {

constexpr int kTopkBlocks = 256;
constexpr int kRescoreGrid = 64;

const int kShortR[] = {8, 12, 16, 20, 24};

// Rows padded to whole passes times the per-step work: 4.5 ALU operations per
// row plus about 8 per step.
KernelChoice choose_short(uint32_t qlen, bool int32) {
    if (int32) return KernelChoice{16, false};
    int bestR = 16;
    double best = 1e300;
    for (int R : kShortR) {
        const uint32_t TR = (uint32_t)kShortT * R;
        const double passes = (qlen + TR - 1) / TR;
        const double cost = passes * (4.5 * R + 8.0) * (R == 16 ? 0.97 : 1.0);
        if (cost < best) { best = cost; bestR = R; }
    }
    return KernelChoice{bestR, true};
}

KernelChoice rescore_choice() { return KernelChoice{16, false}; }

bool use_int32(const sw_db* db, int32_t alpha, int32_t beta) {
    return (db->flags & SW_DB_FLAG_FORCE_INT32) || (int64_t)alpha + beta > 32768;
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

}  // namespace

sw_status sw_db_prepare_search(sw_db* db) {
    sw_status st;
    if ((st = db_alloc(db, (void**)&db->d_counters, 256, "search counters"))) return st;

    // one persistent grid for every kernel variant; scratch rows per group slot
    std::vector<KernelChoice> all;
    for (int R : kShortR) all.push_back(KernelChoice{R, true});
    all.push_back(KernelChoice{16, false});
    const int warps = wavefront_block_threads() / 32;
    db->grid_short = db->nsm * occupancy_max(all);
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
    db->grid_rescore = std::min(kRescoreGrid, db->nsm * occupancy_max({rescore_choice()}));
    db->bstride_rescore = bstride_for(std::max(4u, (db->max_len + 3u) & ~3u));
    if ((st = db_alloc(db, (void**)&db->d_bnd_rescore,
                       (uint64_t)db->grid_rescore * warps * (32 / kLongT) * db->bstride_rescore *
                           sizeof(uint2),
                       "boundary rows (rescoring)")))
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

namespace {

WavefrontArgs base_args(sw_db* db, const uint8_t* d_query, uint32_t qlen, const int8_t* d_matrix,
                        int32_t alpha, int32_t beta, int32_t* d_scores) {
    WavefrontArgs a{};
    a.tile_data = db->d_tile_data;
    a.tile_off = db->d_tile_off;
    a.tile_len = db->d_tile_len;
    a.sorted_ids = db->d_sorted;
    a.query = d_query;
    a.qlen = qlen;
    a.matrix = d_matrix;
    a.alphabet = db->alphabet;
    a.alpha = alpha;
    a.beta = beta;
    a.scores = d_scores;
    a.flag_list = db->d_flags;
    a.flag_count = db->d_counters + 3;
    a.status = db->d_counters + 8;
    return a;
}

int grid_for(const sw_db* db, const KernelChoice& kc, int cap) {
    const int occ = std::max(1, wavefront_occupancy(kc, nullptr));
    return std::max(1, std::min(cap, db->nsm * occ));
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
struct PhaseTimer {
    sw_db* db;
    int phase;
    cudaStream_t st;
    uint64_t cells;
    cudaEvent_t a = nullptr;
    PhaseTimer(sw_db* d, int p, cudaStream_t s, uint64_t c) : db(d), phase(p), st(s), cells(c) {
        if (db->flags & SW_DB_FLAG_PROFILE) {
            a = take_event(db);
            cudaEventRecord(a, st);
        }
    }
    void done() {
        if (!a) return;
        cudaEvent_t b = take_event(db);
        cudaEventRecord(b, st);
        db->pending.push_back({phase, a, b, cells});
        a = nullptr;
    }
};

}  // namespace

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

// Enqueue one full search on `stream`. Scores land in d_scores (original order).
sw_status enqueue_search(sw_db* db, const uint8_t* d_query, uint32_t qlen, const int8_t* d_matrix,
                         int32_t alpha, int32_t beta, uint32_t top_k, int32_t* d_scores,
                         int32_t* d_top_scores, uint64_t* d_top_index, cudaStream_t stream) {
    cudaError_t e;
    const bool i32 = use_int32(db, alpha, beta);
    if ((e = cudaMemsetAsync(db->d_counters, 0, 64, stream)) != cudaSuccess)
        return cuda_fail(e, "search: counter reset");
    const uint64_t per_tile = i32 ? kTileSeqs : kTilePairs;  // units per tile
    {
        WavefrontArgs a = base_args(db, d_query, qlen, d_matrix, alpha, beta, d_scores);
        const KernelChoice kc = choose_short(qlen, i32);
        a.bin[0].first_unit = 0;
        a.bin[0].n_units = db->n_long_tiles * per_tile;
        a.bin[0].boundary = db->d_bnd_long;
        a.bin[0].bstride = db->bstride_long;
        a.bin[1].first_unit = db->n_long_tiles * per_tile;
        a.bin[1].n_units = (db->n_tiles - db->n_long_tiles) * per_tile;
        a.bin[1].boundary = db->d_bnd_short;
        a.bin[1].bstride = db->bstride_short;
        a.work_counter = db->d_counters + 0;
        PhaseTimer pt(db, 0, stream, (uint64_t)qlen * db->total_residues);
        if ((e = launch_wavefront(kc, a, grid_for(db, kc, db->grid_short), stream)) != cudaSuccess)
            return cuda_fail(e, "search: wavefront kernel");
        pt.done();
        db->launches += 1;
    }
    if (!i32) {
        WavefrontArgs a = base_args(db, d_query, qlen, d_matrix, alpha, beta, d_scores);
        a.bin[0].unit_list = db->d_flags;
        a.bin[0].unit_count = db->d_counters + 3;
        a.bin[0].boundary = db->d_bnd_rescore;
        a.bin[0].bstride = db->bstride_rescore;
        a.bin[1].n_units = 0;
        a.work_counter = db->d_counters + 2;
        PhaseTimer pt(db, 1, stream, 0);
        if ((e = launch_wavefront(rescore_choice(), a, db->grid_rescore, stream)) != cudaSuccess)
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

namespace {

sw_status check_common(const sw_db* db, uint32_t qlen, int32_t alpha, int32_t beta,
                       uint32_t top_k, const char* fn) {
    if (!db) return fail(SW_ERR_INVALID_ARG, "%s: db is NULL", fn);
    if (qlen == 0) return fail(SW_ERR_INVALID_ARG, "%s: qlen must be >= 1", fn);
    if (alpha < 0 || beta < 0 || alpha > 32767 || beta > 32767)
        return fail(SW_ERR_INVALID_ARG, "%s: alpha and beta must lie in [0, 32767]", fn);
    if (top_k > SW_MAX_TOP_K)
        return fail(SW_ERR_INVALID_ARG, "%s: top_k %u exceeds %u", fn, top_k, SW_MAX_TOP_K);
    return SW_OK;
}

struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        cudaSetDevice(dev);
    }
    ~DeviceScope() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

sw_status stage_query(sw_db* db, const uint8_t* query, uint32_t qlen, const int8_t* matrix) {
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

sw_status validate_host_query(const sw_db* db, const uint8_t* query, uint32_t qlen,
                              const int8_t* matrix, const char* fn) {
    if (!query || !matrix) return fail(SW_ERR_INVALID_ARG, "%s: query or matrix is NULL", fn);
    for (uint32_t i = 0; i < qlen; ++i)
        if (query[i] >= db->alphabet)
            return fail(SW_ERR_INVALID_ARG, "%s: query code %u at %u is not below alphabet %u", fn,
                        query[i], i, db->alphabet);
    return SW_OK;
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
    int32_t* d_ts = db->d_top_scores;
    uint64_t* d_ti = db->d_top_index;
    st = enqueue_search(db, db->d_query, qlen, db->d_matrix, alpha, beta, top_k, db->d_scores, d_ts,
                        d_ti, db->stream);
    if (st) return st;
    cudaEventRecord(db->ev_t1, db->stream);
    const uint32_t kk = (uint32_t)std::min<uint64_t>(top_k, db->n_seqs);
    e = cudaSuccess;
    if (scores)
        e = cudaMemcpyAsync(scores, db->d_scores, db->n_seqs * 4, cudaMemcpyDeviceToHost,
                            db->stream);
    if (e == cudaSuccess && kk)
        e = cudaMemcpyAsync(top_scores, d_ts, kk * 4, cudaMemcpyDeviceToHost, db->stream);
    if (e == cudaSuccess && kk)
        e = cudaMemcpyAsync(top_index, d_ti, kk * 8, cudaMemcpyDeviceToHost, db->stream);
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

extern "C" sw_status sw_search_batch(sw_db* db, uint32_t nq, const uint8_t* const* queries,
                                     const uint32_t* qlens, const int8_t* matrix, int32_t alpha,
                                     int32_t beta, uint32_t top_k, int32_t* const* scores,
                                     int32_t* top_scores, uint64_t* top_index, uint32_t* n_top,
                                     sw_stats* stats) {
    clear_error();
    if (!db) return fail(SW_ERR_INVALID_ARG, "sw_search_batch: db is NULL");
    if (nq == 0) return SW_OK;
    if (!queries || !qlens) return fail(SW_ERR_INVALID_ARG, "sw_search_batch: NULL queries");
    sw_stats total{};
    for (uint32_t q = 0; q < nq; ++q) {
        sw_stats s{};
        sw_status st = sw_search(db, queries[q], qlens[q], matrix, alpha, beta, top_k,
                                 scores ? scores[q] : nullptr,
                                 top_scores ? top_scores + (size_t)q * top_k : nullptr,
                                 top_index ? top_index + (size_t)q * top_k : nullptr,
                                 n_top ? n_top + q : nullptr, &s);
        if (st) return st;
        total.cells += s.cells;
        total.recomputed += s.recomputed;
        total.kernel_ms += s.kernel_ms;
        total.total_ms += s.total_ms;
    }
    if (stats) *stats = total;
    return SW_OK;
}
