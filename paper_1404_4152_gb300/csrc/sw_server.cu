// Continuous-batching search server over a database resident in HBM.
//
// The paper searches one query at a time (Section III). A server instead keeps
// the database on the device and takes queries as they arrive:
//  - the database is cut into S slices of about equal work (contiguous runs of
//    length-sorted chunks);
//  - a scheduler thread runs waves; one wave advances every admitted query by
//    one slice, in persistent launches whose work items are (query or query
//    pair, chunk of its slice) -- two queries at the same slice share the two
//    16-bit halves of the lanes when the pair costs less than the two alone;
//  - a query is admitted at a wave boundary when a slot is free: a slot is the
//    device memory a query needs (its score row and its codes), reserved up
//    front from the server's budget, so admission is by device memory;
//  - a query that finishes its last slice gets its top-k and leaves; its slot
//    is reused by the next waiting query in the following wave.
// Queries that arrive while others are on the GPU therefore join the next
// wave and their work overlaps with the older queries' remaining slices.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sw.h"
#include "sw_db.h"
#include "sw_internal.h"

using namespace swgb;

namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { kPending = 0, kActive = 1, kDone = 2, kCancelled = 3, kFailed = 4 };

struct Request {
    uint64_t ticket = 0;
    std::vector<uint8_t> query;
    std::vector<int8_t> matrix;
    int32_t alpha = 0, beta = 0;
    uint32_t top_k = 0;
    int state = kPending;
    int slot = -1;
    uint32_t next_slice = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    std::vector<int32_t> top_s;
    std::vector<uint64_t> top_i;
    uint32_t n_top = 0;
    sw_status status = SW_OK;
    std::string error;
};

}  // namespace

struct sw_server {
    sw_db* db = nullptr;
    uint32_t max_queue = 0, max_active = 0, max_qlen = 0, slices = 0;
    Clock::time_point t0;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> reqs;
    std::deque<std::shared_ptr<Request>> pending;
    std::vector<std::shared_ptr<Request>> active;
    std::vector<int> free_slots;
    std::vector<int8_t> scheme_matrix;  // scoring scheme of the active set
    int32_t scheme_alpha = 0, scheme_beta = 0;

    // device side
    cudaStream_t stream = nullptr;
    std::vector<std::pair<void*, size_t>> allocs;
    int32_t* d_scores = nullptr;   // max_active rows of n_seqs
    uint8_t* d_queries = nullptr;  // max_active x max_qlen
    int8_t* d_matrix = nullptr;
    QueryPair* d_pairs = nullptr;
    uint32_t* d_prefix = nullptr;
    uint32_t* d_chunk0 = nullptr;
    uint64_t* d_qoff = nullptr;
    uint32_t* d_qlen = nullptr;
    uint2* d_flags = nullptr;
    uint32_t flag_cap = 0;
    uint32_t* d_counters = nullptr;
    uint2* d_bnd = nullptr;
    uint64_t bstride = 0;
    int grid = 0;
    void* d_topk = nullptr;
    TopkScratch topk{};
    int32_t* d_top_s = nullptr;    // max_active x 1024
    uint64_t* d_top_i = nullptr;
    int32_t* h_top_s = nullptr;    // pinned
    uint64_t* h_top_i = nullptr;
    std::vector<uint32_t> slice_tile0;  // slices + 1 tile boundaries (multiples of 8)

    cudaEvent_t ev_wave0 = nullptr, ev_wave1 = nullptr;  // device time of one wave

    // statistics
    uint64_t waves = 0, completed = 0, rejected = 0, cells = 0;
    double busy_ms = 0, gpu_ms = 0;
};

namespace {

double now_ms(const sw_server* s) {
    return std::chrono::duration<double, std::milli>(Clock::now() - s->t0).count();
}

cudaError_t srv_alloc(sw_server* s, void** p, size_t bytes) {
    cudaError_t e = db_malloc(s->db, p, bytes ? bytes : 16);
    if (e == cudaSuccess) s->allocs.emplace_back(*p, bytes ? bytes : 16);
    return e;
}

void srv_release(sw_server* s) {
    for (auto& a : s->allocs) db_free(s->db, a.first, a.second);
    s->allocs.clear();
    if (s->h_top_s) cudaFreeHost(s->h_top_s);
    if (s->h_top_i) cudaFreeHost(s->h_top_i);
    if (s->ev_wave0) cudaEventDestroy(s->ev_wave0);
    if (s->ev_wave1) cudaEventDestroy(s->ev_wave1);
    if (s->stream) cudaStreamDestroy(s->stream);
}

// Kernel launch over per-item chunk ranges of bin 1 (items = query pairs).
sw_status launch_items(sw_server* s, KernelChoice kc, const std::vector<QueryPair>& items,
                       const std::vector<uint32_t>& chunk0, const std::vector<uint32_t>& nchunk,
                       int part) {
    sw_db* db = s->db;
    cudaError_t e;
    const uint32_t n = (uint32_t)items.size();
    if (n == 0) return SW_OK;
    std::vector<uint32_t> prefix(n + 1, 0);
    for (uint32_t i = 0; i < n; ++i) prefix[i + 1] = prefix[i] + nchunk[i];
    QueryPair* d_pairs = s->d_pairs + (size_t)part * s->max_active;
    uint32_t* d_prefix = s->d_prefix + (size_t)part * (s->max_active + 1);
    uint32_t* d_chunk0 = s->d_chunk0 + (size_t)part * s->max_active;
    uint32_t* counter = s->d_counters + 8 + part;
    if ((e = cudaMemcpyAsync(d_pairs, items.data(), n * sizeof(QueryPair), cudaMemcpyHostToDevice,
                             s->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_prefix, prefix.data(), (n + 1) * 4, cudaMemcpyHostToDevice,
                             s->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_chunk0, chunk0.data(), n * 4, cudaMemcpyHostToDevice,
                             s->stream)) != cudaSuccess)
        return cuda_fail(e, "server: wave upload");
    WavefrontArgs a{};
    a.dbg = db->d_counters + kDebugWord;
    a.tile_data = db->d_tile_data;
    a.tile_off = db->d_tile_off;
    a.tile_len = db->d_tile_len;
    a.sorted_ids = db->d_sorted;
    a.bin[1].first_unit = 0;
    a.bin[1].n_units = db->n_tiles * (units_per_tile(kc));
    a.bin[1].boundary = s->d_bnd;
    a.bin[1].bstride = s->bstride;
    a.query = s->d_queries;
    a.pairs = d_pairs;
    a.n_pairs = n;
    a.item_prefix = d_prefix;
    a.pair_chunk0 = d_chunk0;
    a.matrix = s->d_matrix;
    a.alphabet = db->alphabet;
    a.alpha = s->scheme_alpha;
    a.beta = s->scheme_beta;
    a.scores = s->d_scores;
    a.score_stride = db->n_seqs;
    a.flag_list = s->d_flags;
    a.flag_count = s->d_counters + 3;
    a.flag_cap = s->flag_cap;
    a.work_counter = counter;
    const int occ = std::max(1, wavefront_occupancy(kc, nullptr));
    const int grid = std::max(1, std::min(s->grid, db->nsm * occ));
    if ((e = launch_wavefront(kc, a, grid, s->stream)) != cudaSuccess)
        return cuda_fail(e, "server: wave kernel");
    db->launches += 1;
    return SW_OK;
}

// One wave: every active request advances by one slice. Requests at the same
// slice are paired (two queries per 16-bit lane pair) when their lengths are close
// enough for the pair to cost less than the two alone (the pair runs the longer
// one's rows for both); the others run alone in the mode that packs two database
// sequences instead.
sw_status run_wave(sw_server* s, std::vector<std::shared_ptr<Request>>& act, double* wave_gpu_ms) {
    sw_db* db = s->db;
    cudaError_t e;
    *wave_gpu_ms = 0;
    std::vector<std::shared_ptr<Request>> order = act;
    std::stable_sort(order.begin(), order.end(), [](const auto& x, const auto& y) {
        if (x->next_slice != y->next_slice) return x->next_slice < y->next_slice;
        return x->query.size() > y->query.size();
    });
    const bool i32 = (int64_t)s->scheme_alpha + s->scheme_beta > 32768;
    // lone queries: the ring with 24 rows per thread, whose short last pass fits any length
    const KernelChoice ks = i32 ? KernelChoice{KernelChoice::kInt32, 16}
                          : (db->flags & SW_DB_FLAG_QUERY_PROFILE)
                              ? KernelChoice{KernelChoice::kPairDb, 16}
                              : KernelChoice{KernelChoice::kPairRing, kRingLastR};
    auto one = [&](const Request& r) {
        QueryPair p{};
        p.off_a = p.off_b = (uint64_t)r.slot * s->max_qlen;
        p.len_a = (uint32_t)r.query.size();
        p.q_a = (uint32_t)r.slot;
        p.q_b = 0xffffffffu;
        return p;
    };
    // chunk ranges of a slice: 4-tile chunks (one sequence per unit), 8-tile chunks (pairs)
    auto range4 = [&](uint32_t sl, uint32_t* c0, uint32_t* n) {
        const uint32_t t0 = s->slice_tile0[sl], t1 = s->slice_tile0[sl + 1];
        *c0 = t0 / 4;
        *n = (t1 + 3) / 4 - t0 / 4;
    };
    auto range8 = [&](uint32_t sl, uint32_t* c0, uint32_t* n) {
        const uint32_t t0 = s->slice_tile0[sl], t1 = s->slice_tile0[sl + 1];
        *c0 = t0 / 8;
        *n = (t1 + 7) / 8 - t0 / 8;
    };
    if ((e = cudaEventRecord(s->ev_wave0, s->stream)) != cudaSuccess)
        return cuda_fail(e, "server: wave event");
    if ((e = cudaMemsetAsync(s->d_counters, 0, 64, s->stream)) != cudaSuccess)
        return cuda_fail(e, "server: counter reset");
    std::vector<QueryPair> pairs, singles;
    std::vector<uint32_t> pc0, pn, sc0, sn;
    for (size_t i = 0; i < order.size();) {
        const Request& ra = *order[i];
        uint32_t c0, n;
        if (i32) {
            singles.push_back(one(ra));
            range4(ra.next_slice, &c0, &n);
            sc0.push_back(c0);
            sn.push_back(n);
            i += 1;
        } else if (i + 1 < order.size() && order[i + 1]->next_slice == ra.next_slice &&
                   pair_pays(db, (uint32_t)ra.query.size(), (uint32_t)order[i + 1]->query.size(), ks)) {
            const Request& rb = *order[i + 1];
            QueryPair p = one(ra);
            p.off_b = (uint64_t)rb.slot * s->max_qlen;
            p.len_b = (uint32_t)rb.query.size();
            p.q_b = (uint32_t)rb.slot;
            pairs.push_back(p);
            range4(ra.next_slice, &c0, &n);
            pc0.push_back(c0);
            pn.push_back(n);
            i += 2;
        } else {
            singles.push_back(one(ra));
            range8(ra.next_slice, &c0, &n);
            sc0.push_back(c0);
            sn.push_back(n);
            i += 1;
        }
    }
    sw_status st;
    // paired queries: the rows per thread with the least padded cost for their lengths
    std::vector<uint32_t> plen;
    for (const QueryPair& p : pairs) plen.push_back(std::max(p.len_a, p.len_b));
    const int pair_R = pairs.empty() ? 16 : choose_pair_R(db, plen);
    if ((st = launch_items(s, KernelChoice{KernelChoice::kQueryPair, pair_R}, pairs, pc0, pn, 0)))
        return st;
    if ((st = launch_items(s, ks, singles, sc0, sn, 1))) return st;
    if (!i32) {
        RescoreArgs r{};
        r.dbg = db->d_counters + kDebugWord;
        r.tile_data = db->d_tile_data;
        r.tile_off = db->d_tile_off;
        r.tile_len = db->d_tile_len;
        r.sorted_ids = db->d_sorted;
        r.list = s->d_flags;
        r.count = s->d_counters + 3;
        r.cap = s->flag_cap;
        r.query = s->d_queries;
        r.qoff = s->d_qoff;
        r.qlen = s->d_qlen;
        r.matrix = s->d_matrix;
        r.alphabet = db->alphabet;
        r.alpha = s->scheme_alpha;
        r.beta = s->scheme_beta;
        r.scores = s->d_scores;
        r.score_stride = db->n_seqs;
        r.boundary = db->d_bnd_rescore;
        r.bstride = db->bstride_rescore;
        r.work_counter = s->d_counters + 2;
        if ((e = launch_rescore(r, db->grid_rescore, s->stream)) != cudaSuccess)
            return cuda_fail(e, "server: rescoring kernel");
        db->launches += 1;
    }
    // requests finishing this wave: top-k of their score row, copied to pinned memory
    for (auto& r : order) {
        if (r->next_slice + 1 != s->slices || r->top_k == 0) continue;
        int32_t* ts = s->d_top_s + (size_t)r->slot * SW_MAX_TOP_K;
        uint64_t* ti = s->d_top_i + (size_t)r->slot * SW_MAX_TOP_K;
        if ((e = launch_topk(s->d_scores + (size_t)r->slot * db->n_seqs, db->n_seqs, db->n_seqs, 1,
                             r->top_k, s->topk, ts, ti, s->stream)) != cudaSuccess)
            return cuda_fail(e, "server: top-k");
        db->launches += topk_launch_count();
        const uint32_t kk = (uint32_t)std::min<uint64_t>(r->top_k, db->n_seqs);
        if ((e = cudaMemcpyAsync(s->h_top_s + (size_t)r->slot * SW_MAX_TOP_K, ts, kk * 4,
                                 cudaMemcpyDeviceToHost, s->stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(s->h_top_i + (size_t)r->slot * SW_MAX_TOP_K, ti, kk * 8,
                                 cudaMemcpyDeviceToHost, s->stream)) != cudaSuccess)
            return cuda_fail(e, "server: result copy");
    }
    uint32_t nflag = 0;
    if ((e = cudaMemcpyAsync(&nflag, s->d_counters + 3, 4, cudaMemcpyDeviceToHost, s->stream)) !=
            cudaSuccess ||
        (e = cudaEventRecord(s->ev_wave1, s->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s->stream)) != cudaSuccess)
        return cuda_fail(e, "server: wave");
    float ms = 0;
    if (cudaEventElapsedTime(&ms, s->ev_wave0, s->ev_wave1) == cudaSuccess) *wave_gpu_ms = ms;
    if (nflag > s->flag_cap)
        return fail(SW_ERR_INTERNAL, "server: %u saturated pairs exceed the rescoring list (%u)",
                    nflag, s->flag_cap);
    return SW_OK;
}

void worker_loop(sw_server* s) {
    cudaSetDevice(s->db->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        s->cv_work.wait(lk, [&] { return s->stop || !s->pending.empty() || !s->active.empty(); });
        if (s->stop) break;
        // drop cancelled requests
        for (auto it = s->active.begin(); it != s->active.end();) {
            if ((*it)->state == kCancelled) {
                s->free_slots.push_back((*it)->slot);
                it = s->active.erase(it);
            } else {
                ++it;
            }
        }
        // admission: free slots, same scoring scheme as the active set
        while (!s->pending.empty() && !s->free_slots.empty()) {
            auto r = s->pending.front();
            if (r->state == kCancelled) {
                s->pending.pop_front();
                continue;
            }
            if (!s->active.empty() &&
                (r->matrix != s->scheme_matrix || r->alpha != s->scheme_alpha ||
                 r->beta != s->scheme_beta))
                break;
            s->pending.pop_front();
            if (s->active.empty()) {
                s->scheme_matrix = r->matrix;
                s->scheme_alpha = r->alpha;
                s->scheme_beta = r->beta;
                cudaMemcpyAsync(s->d_matrix, r->matrix.data(), r->matrix.size(),
                                cudaMemcpyHostToDevice, s->stream);
            }
            r->slot = s->free_slots.back();
            s->free_slots.pop_back();
            r->state = kActive;
            r->next_slice = 0;
            r->t_admit = now_ms(s);
            const uint64_t off = (uint64_t)r->slot * s->max_qlen;
            const uint32_t len = (uint32_t)r->query.size();
            cudaMemcpyAsync(s->d_queries + off, r->query.data(), len, cudaMemcpyHostToDevice,
                            s->stream);
            cudaMemcpyAsync(s->d_qoff + r->slot, &off, 8, cudaMemcpyHostToDevice, s->stream);
            cudaMemcpyAsync(s->d_qlen + r->slot, &len, 4, cudaMemcpyHostToDevice, s->stream);
            s->active.push_back(r);
        }
        if (s->active.empty()) continue;
        std::vector<std::shared_ptr<Request>> act = s->active;
        lk.unlock();
        const double tw0 = now_ms(s);
        double wave_gpu_ms = 0;
        const sw_status st = run_wave(s, act, &wave_gpu_ms);
        const std::string err = st ? std::string(sw_last_error()) : std::string();
        const double tw1 = now_ms(s);
        lk.lock();
        s->waves += 1;
        s->busy_ms += tw1 - tw0;
        s->gpu_ms += wave_gpu_ms;
        for (auto& r : act) {
            if (r->state == kCancelled) {  // cancelled during the wave
                s->free_slots.push_back(r->slot);
                continue;
            }
            if (r->state != kActive) continue;
            if (st) {
                r->state = kFailed;
                r->status = st;
                r->error = err;
            } else if (++r->next_slice < s->slices) {
                continue;
            } else {
                const uint32_t kk = (uint32_t)std::min<uint64_t>(r->top_k, s->db->n_seqs);
                r->top_s.assign(s->h_top_s + (size_t)r->slot * SW_MAX_TOP_K,
                                s->h_top_s + (size_t)r->slot * SW_MAX_TOP_K + kk);
                r->top_i.assign(s->h_top_i + (size_t)r->slot * SW_MAX_TOP_K,
                                s->h_top_i + (size_t)r->slot * SW_MAX_TOP_K + kk);
                r->n_top = kk;
                r->state = kDone;
                s->completed += 1;
                s->cells += (uint64_t)r->query.size() * s->db->total_residues;
            }
            r->t_done = now_ms(s);
            s->free_slots.push_back(r->slot);
        }
        s->active.erase(std::remove_if(s->active.begin(), s->active.end(),
                                       [](const auto& r) { return r->state != kActive; }),
                        s->active.end());
        s->cv_done.notify_all();
    }
}

}  // namespace

extern "C" sw_status sw_server_create(sw_db* db, const sw_server_opts* opts, sw_server** out) {
    clear_error();
    if (!db || !out) return fail(SW_ERR_INVALID_ARG, "sw_server_create: NULL argument");
    *out = nullptr;
    auto s = std::make_unique<sw_server>();
    s->db = db;
    s->max_queue = (opts && opts->max_queue) ? opts->max_queue : 4096;
    s->max_active = (opts && opts->max_active) ? opts->max_active : 64;
    s->max_qlen = (opts && opts->max_qlen) ? opts->max_qlen : 8192;
    s->slices = (opts && opts->slices) ? opts->slices : 8;
    const uint64_t budget = opts ? opts->device_budget : 0;
    s->t0 = Clock::now();
    cudaSetDevice(db->device);
    // admission by device memory: each slot is a score row plus the query codes
    const uint64_t slot_bytes = db->n_seqs * 4 + s->max_qlen + SW_MAX_TOP_K * 12 + 64;
    if (budget) {
        const uint64_t fit = budget / slot_bytes;
        if (fit == 0)
            return fail(SW_ERR_OOM, "sw_server_create: budget %llu holds no query slot (%llu bytes)",
                        (unsigned long long)budget, (unsigned long long)slot_bytes);
        s->max_active = (uint32_t)std::min<uint64_t>(s->max_active, fit);
    }
    // slices of about equal work (padded tile residues), cut at multiples of 8 tiles
    {
        const uint64_t groups = (db->n_tiles + 7) / 8;
        s->slices = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(s->slices, groups));
        std::vector<uint64_t> work(groups, 0);
        uint64_t total = 0;
        for (uint64_t t = 0; t < db->n_tiles; ++t) {
            work[t / 8] += (uint64_t)db->tile_len_host[t] * kTileSeqs;
            total += (uint64_t)db->tile_len_host[t] * kTileSeqs;
        }
        std::vector<uint32_t> b(1, 0);
        uint64_t acc = 0;
        uint32_t k = 1;
        for (uint64_t g = 0; g < groups && k < s->slices; ++g) {
            acc += work[g];
            if (acc * s->slices >= total * k) {
                if ((g + 1) * 8 < db->n_tiles) b.push_back((uint32_t)((g + 1) * 8));
                ++k;
            }
        }
        b.push_back((uint32_t)db->n_tiles);
        std::vector<uint32_t> u(1, 0);
        for (size_t i = 1; i < b.size(); ++i)
            if (b[i] > u.back()) u.push_back(b[i]);
        s->slice_tile0 = u;
        s->slices = (uint32_t)u.size() - 1;
    }
    cudaError_t e;
    const KernelChoice kqp{KernelChoice::kQueryPair, 16}, ki32{KernelChoice::kInt32, 16},
        kring{KernelChoice::kPairRing, kRingLastR};
    s->grid = db->nsm * std::max(1, std::max({wavefront_occupancy(kqp, nullptr),
                                              wavefront_occupancy(ki32, nullptr),
                                              wavefront_occupancy(kring, nullptr)}));
    s->bstride = 2ull * (((uint64_t)std::max(4u, (db->max_len + 3u) & ~3u) + boundary_slack() + 3) &
                         ~3ull);
    s->flag_cap = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(db->n_seqs, 1u << 20), 1u << 26);
    const uint64_t slots = (uint64_t)s->grid * (wavefront_block_threads() / 32) * (32 / kShortT);
    const uint32_t A = s->max_active;
    if ((e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreate(&s->ev_wave0)) != cudaSuccess ||
        (e = cudaEventCreate(&s->ev_wave1)) != cudaSuccess ||
        (e = srv_alloc(s.get(), (void**)&s->d_scores, (size_t)A * db->n_seqs * 4)) != cudaSuccess ||
        (e = srv_alloc(s.get(), (void**)&s->d_queries, (size_t)A * s->max_qlen)) != cudaSuccess ||
        (e = srv_alloc(s.get(), (void**)&s->d_matrix, SW_MAX_ALPHABET * SW_MAX_ALPHABET)) !=
            cudaSuccess ||
        (e = srv_alloc(s.get(), (void**)&s->d_pairs, (size_t)2 * A * sizeof(QueryPair))) !=
            cudaSuccess ||
        (e = srv_alloc(s.get(), (void**)&s->d_prefix, (size_t)2 * (A + 1) * 4)) != cudaSuccess ||
        (e = srv_alloc(s.get(), (void**)&s->d_chunk0, (size_t)2 * A * 4)) != cudaSuccess ||
        (e = srv_alloc(s.get(), (void**)&s->d_qoff, (size_t)A * 8)) != cudaSuccess ||
        (e = srv_alloc(s.get(), (void**)&s->d_qlen, (size_t)A * 4)) != cudaSuccess ||
        (e = srv_alloc(s.get(), (void**)&s->d_flags, (size_t)s->flag_cap * sizeof(uint2))) !=
            cudaSuccess ||
        (e = srv_alloc(s.get(), (void**)&s->d_counters, 256)) != cudaSuccess ||
        (e = srv_alloc(s.get(), (void**)&s->d_bnd, slots * s->bstride * sizeof(uint2))) !=
            cudaSuccess ||
        (e = srv_alloc(s.get(), &s->d_topk, topk_scratch_bytes(1, SW_MAX_TOP_K, 256))) !=
            cudaSuccess ||
        (e = srv_alloc(s.get(), (void**)&s->d_top_s, (size_t)A * SW_MAX_TOP_K * 4)) !=
            cudaSuccess ||
        (e = srv_alloc(s.get(), (void**)&s->d_top_i, (size_t)A * SW_MAX_TOP_K * 8)) !=
            cudaSuccess ||
        (e = cudaMallocHost((void**)&s->h_top_s, (size_t)A * SW_MAX_TOP_K * 4)) != cudaSuccess ||
        (e = cudaMallocHost((void**)&s->h_top_i, (size_t)A * SW_MAX_TOP_K * 8)) != cudaSuccess) {
        const sw_status st = cuda_fail(e, "sw_server_create");
        srv_release(s.get());
        return st;
    }
    topk_scratch_carve(s->d_topk, 1, SW_MAX_TOP_K, 256, &s->topk);
    for (int i = (int)A - 1; i >= 0; --i) s->free_slots.push_back(i);
    sw_server* raw = s.release();
    raw->worker = std::thread(worker_loop, raw);
    *out = raw;
    return SW_OK;
}

extern "C" sw_status sw_server_submit(sw_server* s, const uint8_t* query, uint32_t qlen,
                                      const int8_t* matrix, int32_t alpha, int32_t beta,
                                      uint32_t top_k, uint64_t* ticket) {
    clear_error();
    if (!s || !query || !matrix || !ticket)
        return fail(SW_ERR_INVALID_ARG, "sw_server_submit: NULL argument");
    if (qlen == 0 || qlen > s->max_qlen)
        return fail(SW_ERR_INVALID_ARG, "sw_server_submit: qlen %u outside 1..%u", qlen, s->max_qlen);
    if (alpha < 0 || beta < 0 || alpha > 32767 || beta > 32767)
        return fail(SW_ERR_INVALID_ARG, "sw_server_submit: alpha and beta must lie in [0, 32767]");
    if (top_k > SW_MAX_TOP_K) return fail(SW_ERR_INVALID_ARG, "sw_server_submit: top_k too large");
    const uint32_t A = s->db->alphabet;
    for (uint32_t i = 0; i < qlen; ++i)
        if (query[i] >= A)
            return fail(SW_ERR_INVALID_ARG, "sw_server_submit: query code %u at %u is not below %u",
                        query[i], i, A);
    auto r = std::make_shared<Request>();
    r->query.assign(query, query + qlen);
    r->matrix.assign(matrix, matrix + (size_t)A * A);
    r->alpha = alpha;
    r->beta = beta;
    r->top_k = top_k;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return fail(SW_ERR_BUSY, "sw_server_submit: server is shutting down");
    if (s->pending.size() >= s->max_queue) {
        s->rejected += 1;
        return fail(SW_ERR_BUSY, "sw_server_submit: queue full (%u waiting)", s->max_queue);
    }
    r->ticket = s->next_ticket++;
    r->t_submit = now_ms(s);
    s->reqs[r->ticket] = r;
    s->pending.push_back(r);
    *ticket = r->ticket;
    s->cv_work.notify_one();
    return SW_OK;
}

extern "C" sw_status sw_server_wait(sw_server* s, uint64_t ticket, uint32_t timeout_ms,
                                    int32_t* top_scores, uint64_t* top_index, uint32_t* n_top,
                                    sw_latency* lat) {
    clear_error();
    if (!s) return fail(SW_ERR_INVALID_ARG, "sw_server_wait: NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(SW_ERR_BUSY, "sw_server_wait: unknown ticket %llu",
                                         (unsigned long long)ticket);
    std::shared_ptr<Request> r = it->second;
    const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
        return r->state == kDone || r->state == kFailed || r->state == kCancelled;
    });
    if (!ok) return fail(SW_ERR_TIMEOUT, "sw_server_wait: ticket %llu not done after %u ms",
                         (unsigned long long)ticket, timeout_ms);
    s->reqs.erase(ticket);
    if (r->state == kCancelled) return fail(SW_ERR_INVALID_ARG, "sw_server_wait: ticket cancelled");
    if (r->state == kFailed) return fail(r->status, "%s", r->error.c_str());
    if (r->top_k && (!top_scores || !top_index))
        return fail(SW_ERR_INVALID_ARG, "sw_server_wait: output buffers are NULL");
    std::copy(r->top_s.begin(), r->top_s.end(), top_scores);
    std::copy(r->top_i.begin(), r->top_i.end(), top_index);
    if (n_top) *n_top = r->n_top;
    if (lat) {
        lat->submit_ms = r->t_submit;
        lat->admit_ms = r->t_admit;
        lat->done_ms = r->t_done;
    }
    return SW_OK;
}

extern "C" sw_status sw_server_cancel(sw_server* s, uint64_t ticket) {
    clear_error();
    if (!s) return fail(SW_ERR_INVALID_ARG, "sw_server_cancel: NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(SW_ERR_BUSY, "sw_server_cancel: unknown ticket");
    auto r = it->second;
    if (r->state == kPending || r->state == kActive) r->state = kCancelled;
    s->reqs.erase(it);
    s->cv_done.notify_all();
    return SW_OK;
}

extern "C" sw_status sw_server_get_stats(sw_server* s, sw_server_stats* out) {
    clear_error();
    if (!s || !out) return fail(SW_ERR_INVALID_ARG, "sw_server_get_stats: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    out->waves = s->waves;
    out->completed = s->completed;
    out->rejected = s->rejected;
    out->cells = s->cells;
    out->busy_ms = s->busy_ms;
    out->pending = (uint32_t)s->pending.size();
    out->active = (uint32_t)s->active.size();
    out->max_active = s->max_active;
    out->slices = s->slices;
    out->gpu_ms = s->gpu_ms;
    return SW_OK;
}

extern "C" void sw_server_destroy(sw_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (auto& r : s->pending) r->state = kCancelled;
        for (auto& r : s->active) r->state = kCancelled;
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->db->device);
    srv_release(s);
    delete s;
}
