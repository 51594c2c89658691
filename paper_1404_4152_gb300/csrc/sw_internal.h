// Internal declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace swgb {

// Bounds-checked build (-DSW_DEBUG_BOUNDS; compute-sanitizer is not available on every
// machine): sw_ok(cond, err, site) records the site of the first failed check in the
// handle's error word and returns false so the caller skips the access. In the normal
// build it is true and compiles away. Sites: 1-9 search kernels (query profile, ring,
// stage, matrix table, boundary read / write, database stream), 11-13 the block
// wavefront (rescoring, long alignment hits: scratch row, database codes, ring), 21-26
// alignment.
#ifdef SW_DEBUG_BOUNDS
constexpr bool kDebugBounds = true;
#else
constexpr bool kDebugBounds = false;
#endif
#ifdef __CUDACC__
__device__ __forceinline__ bool sw_ok(bool cond, uint32_t* err, uint32_t site) {
    if (kDebugBounds && !cond) {
        if (err) atomicCAS(err, 0u, site);
        return false;
    }
    return true;
}
#endif
constexpr int kDebugWord = 60;  // index of the error word in the handle's counters

// Residue code used for padding. Its profile row is all zeros, so padded
// cells score 0 against everything (the dummy residue of the sequence
// profile, Section III.B.1); codes from callers are always < 32.
constexpr uint32_t kPadCode = 32;
constexpr uint32_t kProfileRows = 33;  // codes 0..31 plus the pad code

// Database tiles: 8 sequences (4 pairs) of consecutive length-sorted
// positions, padded to a common length L (a multiple of 4). Tile bytes are
// laid out [L/4][4 pairs][4 columns][2 sequences]: the pair stream of pair g
// for columns 4c..4c+3 is the 8-byte word at ((c * 4 + g) * 8).
constexpr uint32_t kTileSeqs = 8;
constexpr uint32_t kTilePairs = 4;

// Lanes per unit and query rows per thread of the two bins: the long
// sequences get a warp per pair (kLongT x kLongR rows per pass), the rest
// 8 lanes per pair (R rows per thread, chosen per query).
constexpr int kShortT = 8;
constexpr int kLongT = 32;
constexpr int kLongR = 16;
constexpr int kTuneR = 5;  // rows-per-lane choices: 8, 12, 16, 20, 24

// The single-query ring kernel with 24 rows per thread runs floor(m / 192) whole passes
// of an m-row query and covers the rest (rem rows) with one pass of the fewest rows per
// thread among 8, 16 and 24 that holds them; 0 when nothing is left.
#ifdef __CUDACC__
__host__ __device__
#endif
constexpr int ring_last_rows(uint32_t rem) {
    return rem == 0 ? 0 : rem <= (uint32_t)kShortT * 8 ? 8 : rem <= (uint32_t)kShortT * 16 ? 16 : 24;
}
constexpr int kRingLastR = 24;  // the rows per thread of the kernel that does so

// One bin of units: pairs of sequences (single-query packed kernels) or
// single sequences (batched and int32 kernels) at sorted positions
// first_unit.., plus the bin's scratch rows.
struct BinArgs {
    uint64_t first_unit;            // first pair (or sequence) of the bin
    uint64_t n_units;
    uint2* boundary;                // per group slot: two halves of bstride/2 entries of (H, E)
    uint64_t bstride;               // a multiple of 8
};

// Two queries searched together in the two 16-bit halves of the lanes.
struct QueryPair {
    uint64_t off_a, off_b;          // offsets into the concatenated queries
    uint32_t len_a, len_b;          // len_b = 0: no second query
    uint32_t q_a, q_b;              // output rows (q_b = UINT32_MAX: none)
};

// Arguments of the search kernel (one launch = one query, or a batch of query
// pairs, against the database).
struct WavefrontArgs {
    // database
    const uint8_t* tile_data;
    const uint64_t* tile_off;       // per tile byte offset into tile_data
    const uint32_t* tile_len;       // per tile padded length
    const uint32_t* sorted_ids;     // sorted position -> original index (UINT32_MAX = empty)
    BinArgs bin[2];                 // 0: long sequences, 1: the rest
    // queries and scoring scheme
    const uint8_t* query;           // single query, or all queries concatenated
    uint32_t qlen;                  // single query length
    const QueryPair* pairs;         // batch: query pairs (NULL for a single query)
    uint32_t n_pairs;
    // serving waves: pair k covers bin-1 chunks pair_chunk0[k] .. + (item_prefix[k+1] -
    // item_prefix[k]); NULL = every pair covers both whole bins
    const uint32_t* item_prefix;    // n_pairs + 1
    const uint32_t* pair_chunk0;    // n_pairs
    const int8_t* matrix;
    uint32_t alphabet;
    int32_t alpha, beta;
    // outputs
    int32_t* scores;                // row q at scores + q * score_stride, original order
    uint64_t score_stride;
    uint2* flag_list;               // (query row, sorted position) to rescore in int32
    uint32_t* flag_count;
    uint32_t flag_cap;
    // scheduling
    uint32_t* work_counter;
    uint32_t* dbg;                  // error word of the bounds-checked build (may be NULL)
};

struct KernelChoice {
    // kPairRing: one query against pairs like kPairDb, with the score-profile ring
    enum Mode { kPairDb = 0, kQueryPair = 1, kInt32 = 2, kPairRing = 3 };
    Mode mode;    // what the two 16-bit halves hold (or int32 lanes)
    int R;        // query rows per thread in the short bin
};
constexpr int kModes = 4;

// Work units per database tile: pairs of sequences for the single-query
// packed kernels, sequences otherwise.
inline uint32_t units_per_tile(const KernelChoice& kc) {
    return kc.mode == KernelChoice::kPairDb || kc.mode == KernelChoice::kPairRing ? kTilePairs
                                                                                 : kTileSeqs;
}

// Arguments of the int32 rescoring kernel (a list of (query row, sorted position)).
struct RescoreArgs {
    const uint8_t* tile_data;
    const uint64_t* tile_off;
    const uint32_t* tile_len;
    const uint32_t* sorted_ids;
    const uint2* list;
    const uint32_t* count;
    uint32_t cap;
    const uint8_t* query;           // concatenated queries
    const uint64_t* qoff;           // per query row: offset and length (device); NULL: one
    const uint32_t* qlen;           //   query at offset 0 of length single_qlen
    uint32_t single_qlen;
    const int8_t* matrix;
    uint32_t alphabet;
    int32_t alpha, beta;
    int32_t* scores;
    uint64_t score_stride;
    uint2* boundary;                // per block: one row of bstride entries
    uint64_t bstride;
    uint32_t* work_counter;
    uint32_t* dbg;                  // error word of the bounds-checked build (may be NULL)
    // dense_n > 0: no list; entry e (< dense_count) is (query row e / dense_n, sorted
    // position e % dense_n) -- every query against the first dense_n sorted positions
    uint32_t dense_n;
    uint32_t dense_count;
};
cudaError_t launch_rescore(const RescoreArgs& a, int grid, cudaStream_t stream);
int rescore_blocks_per_sm(uint32_t alphabet);  // resident blocks per SM for this alphabet

// Entries past a unit's length that a boundary row half must hold (per half:
// length + boundary_slack(), rounded up to a multiple of 4).
uint32_t boundary_slack();

// Launch the search kernel (grid = number of persistent blocks).
cudaError_t launch_wavefront(const KernelChoice& kc, const WavefrontArgs& a, int grid,
                             cudaStream_t stream);
// Blocks per SM the kernel reaches (for sizing scratch), and its threads per block.
int wavefront_occupancy(const KernelChoice& kc, int* threads_per_block);
bool wavefront_supported(const KernelChoice& kc);
int wavefront_block_threads();
int wavefront_short_units_per_chunk();  // sequences per short-bin chunk (one-sequence modes)

// Tile layout: gather database residues into tiles (device side).
cudaError_t launch_build_tiles(const uint8_t* residues, const uint64_t* offsets,
                               const uint32_t* sorted_ids, uint64_t n_sorted,
                               const uint64_t* tile_off, const uint32_t* tile_len,
                               uint64_t n_tiles, uint8_t* tile_data, cudaStream_t stream);
cudaError_t launch_max_code(const uint8_t* residues, uint64_t n, uint32_t* out,
                            cudaStream_t stream);

// Top-k over nq score rows of length n (row q at scores + q * row_stride): one launch;
// each block selects its slice's top-k, the last block of a row merges them.
constexpr uint32_t kTopkCandidates = 8192;  // per row: blocks x k candidates at most
struct TopkScratch {
    int32_t* cand_score;   // nq * kTopkCandidates
    uint32_t* cand_index;  // nq * kTopkCandidates
    uint32_t* cand_count;  // nq * blocks
    uint32_t* done;        // nq: blocks of the row that have finished (cleared per launch)
    int blocks;            // most blocks per row
};
size_t topk_scratch_bytes(uint32_t nq, uint32_t kmax, int blocks);
void topk_scratch_carve(void* base, uint32_t nq, uint32_t kmax, int blocks, TopkScratch* s);
int topk_launch_count();  // kernels one launch_topk call enqueues
cudaError_t launch_topk(const int32_t* scores, uint64_t row_stride, uint64_t n, uint32_t nq,
                        uint32_t k, const TopkScratch& s, int32_t* top_scores,
                        uint64_t* top_index, cudaStream_t stream);

}  // namespace swgb
