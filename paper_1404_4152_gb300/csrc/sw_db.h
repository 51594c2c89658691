// The database handle and the host-side search plumbing shared by the
// library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <utility>
#include <vector>

#include "sw.h"
#include "sw_internal.h"

// Grow-only device buffer owned by a handle.
struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};

// The captured launch sequence of the last batch and what it baked in.
struct BatchGraph {
    cudaGraphExec_t exec = nullptr;
    const void* queries = nullptr;
    const void* matrix = nullptr;
    const void* scores = nullptr;
    const void* top_s = nullptr;
    const void* top_i = nullptr;
    int32_t alpha = 0, beta = 0;
    uint32_t top_k = 0;
    cudaStream_t stream = nullptr;
    std::vector<uint64_t> qoff;
    std::vector<uint32_t> qlen;
    std::vector<int> group_R;           // the launches: rows per thread and first pair
    std::vector<uint32_t> group_first;
    std::vector<uint64_t> items;        // the uploaded work items (pairs, then lone queries)
    uint32_t kernels = 0;
};

struct BatchInfo {
    uint64_t cells = 0;
    uint32_t flag_cap = 0;  // 0: the batch ran in int32 (no rescoring list)
};

struct sw_db {
    // identity
    int device = 0;
    uint32_t alphabet = 0;
    uint64_t n_seqs = 0;
    uint64_t total_residues = 0;
    uint32_t max_len = 0;
    uint32_t long_threshold = 3000;
    uint32_t block_threshold = 0;   // in effect (resolved from the option)
    uint64_t n_block_tiles = 0;     // tiles [0, n_block_tiles) go to the block wavefront
    cudaStream_t blk_stream = nullptr;  // the block wavefront beside the search kernel
    cudaEvent_t blk_fork = nullptr, blk_join = nullptr;
    uint64_t budget = 0;
    uint64_t dev_bytes = 0;
    uint32_t flags = 0;
    int nsm = 0;

    cudaStream_t stream = nullptr;  // the library's own stream (host-buffer calls)
    cudaEvent_t ev_t0 = nullptr, ev_t1 = nullptr;

    // length-sorted tiles (descending length); tiles [0, n_long_tiles) hold the
    // sequences above long_threshold
    uint64_t n_long = 0, n_tiles = 0, n_long_tiles = 0, tile_bytes = 0;
    uint32_t max_len_long = 0, max_len_short = 0;
    std::vector<uint32_t> tile_len_host;
    uint8_t* d_tile_data = nullptr;
    uint64_t* d_tile_off = nullptr;
    uint32_t* d_tile_len = nullptr;
    uint32_t* d_sorted = nullptr;  // sorted position -> original index
    std::vector<uint32_t> pos_of;  // host: original index -> sorted position
    std::vector<uint32_t> seq_len; // host: sequence lengths (original order)
    int32_t* d_scores = nullptr;   // internal score row (original order)
    uint2* d_flags2 = nullptr;     // (query row, sorted position) rescored in int32
    uint32_t* d_misc = nullptr;

    // search scratch
    uint32_t* d_counters = nullptr;  // 0: short work, 1: long work, 2: rescoring work, 3: flags
    uint2* d_bnd_short = nullptr;
    uint64_t bstride_short = 0;
    int grid_short = 0;
    uint2* d_bnd_long = nullptr;
    uint64_t bstride_long = 0;
    int grid_long = 0;
    uint2* d_bnd_rescore = nullptr;
    uint64_t bstride_rescore = 0;
    int grid_rescore = 0;
    void* d_topk = nullptr;
    swgb::TopkScratch topk{};
    uint32_t topk_nq = 0;
    uint8_t* d_query = nullptr;
    uint32_t query_cap = 0;
    int8_t* d_matrix = nullptr;
    int32_t* d_top_scores = nullptr;
    uint64_t* d_top_index = nullptr;
    void* h_pinned = nullptr;

    std::vector<std::pair<void*, size_t>> allocs;

    // batch buffers (grown on demand) and the captured batch graph
    DevBuf b_pairs, b_qoff, b_qlen, b_flags, b_topk, b_queries, b_scores, b_top;
    DevBuf a_rows, a_hits, a_dir, a_ops;  // sw_align scratch (grow-only)
    cudaStream_t a_stream = nullptr;      // sw_align: the long hits' kernel beside the others
    cudaEvent_t a_ev0 = nullptr, a_ev1 = nullptr;
    BatchGraph graph;

    // autotuning (sw_db_autotune)
    sw_tuning tuning{};
    bool tuned = false;

    // residues of the sequences in each bin (for cell counts)
    uint64_t residues_short = 0, residues_long = 0;

    // profiling (SW_DB_FLAG_PROFILE)
    struct Timed {
        int phase;
        cudaEvent_t a, b;
        uint64_t cells;
    };
    std::vector<Timed> pending;
    std::vector<cudaEvent_t> event_pool;
    uint64_t launches = 0;
    uint64_t prof_calls[4] = {0, 0, 0, 0};
    uint64_t prof_cells[4] = {0, 0, 0, 0};
    double prof_ms[4] = {0, 0, 0, 0};
};

namespace swgb {

// Shared by the search and alignment entry points (sw_search.cu).
sw_status check_common(const sw_db* db, uint32_t qlen, int32_t alpha, int32_t beta,
                       uint32_t top_k, const char* fn);
sw_status validate_host_query(const sw_db* db, const uint8_t* query, uint32_t qlen,
                              const int8_t* matrix, const char* fn);
sw_status stage_query(sw_db* db, const uint8_t* query, uint32_t qlen, const int8_t* matrix);
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

sw_status fail(sw_status st, const char* fmt, ...);
sw_status cuda_fail(cudaError_t e, const char* what);
void clear_error();
cudaError_t db_malloc(sw_db* db, void** p, size_t bytes);
void db_free(sw_db* db, void* p, size_t bytes);
sw_status db_alloc(sw_db* db, void** p, size_t bytes, const char* what);

}  // namespace swgb

// Rows per thread of the query-pair kernel for pairs whose longer queries have these
// lengths: the tuned (or estimated) cost of their padded rows (sw_search.cu).
int choose_pair_R(const sw_db* db, const std::vector<uint32_t>& lengths);
// Whether queries of la >= lb rows cost less paired in the query-pair kernel than each
// alone in the kernel `alone`.
bool pair_pays(const sw_db* db, uint32_t la, uint32_t lb, swgb::KernelChoice alone);
// Resolve the block-wavefront route from the option (0 = automatic, UINT32_MAX = never):
// the long tiles whose longest sequence exceeds the threshold (sw_search.cu).
void set_block_route(sw_db* db, uint32_t opt_threshold);
// Allocate the per-handle search scratch (boundary rows, counters, top-k).
sw_status sw_db_prepare_search(sw_db* db);
sw_status ensure(sw_db* db, DevBuf& b, size_t bytes, const char* what);
// Enqueue a whole single-query search / batch on a stream (sw_search.cu).
sw_status enqueue_search(sw_db* db, const uint8_t* d_query, uint32_t qlen, const int8_t* d_matrix,
                         int32_t alpha, int32_t beta, uint32_t top_k, int32_t* d_scores,
                         int32_t* d_top_scores, uint64_t* d_top_index, cudaStream_t stream);
sw_status enqueue_batch(sw_db* db, uint32_t nq, const uint8_t* d_queries,
                        const uint64_t* qoffsets, const int8_t* d_matrix, int32_t alpha,
                        int32_t beta, uint32_t top_k, int32_t* d_scores, int32_t* d_top_scores,
                        uint64_t* d_top_index, cudaStream_t stream, BatchInfo* info);
