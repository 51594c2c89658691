// Internal declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace swgb {

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

// One bin of units: pairs (packed 16-bit kernels) or sequences (int32), as
// sorted positions first_unit.. or an explicit list; plus its scratch rows.
struct BinArgs {
    uint64_t first_unit;            // first pair (or sequence) of the bin
    uint64_t n_units;               // pairs (PAIR kernels) or sequences (int32 kernels)
    const uint32_t* unit_list;      // optional: explicit sorted positions (int32 rescoring)
    const uint32_t* unit_count;     // device count for unit_list
    uint2* boundary;                // per group slot: two halves of bstride/2 entries of (H, E)
    uint64_t bstride;               // a multiple of 8
};

// Arguments of the search kernel (one launch = one query against the database).
struct WavefrontArgs {
    // database
    const uint8_t* tile_data;
    const uint64_t* tile_off;       // per tile byte offset into tile_data
    const uint32_t* tile_len;       // per tile padded length
    const uint32_t* sorted_ids;     // sorted position -> original index (UINT32_MAX = empty)
    BinArgs bin[2];                 // 0: long sequences (or a rescoring list), 1: the rest
    // query and scoring scheme
    const uint8_t* query;
    uint32_t qlen;
    const int8_t* matrix;
    uint32_t alphabet;
    int32_t alpha, beta;
    // outputs
    int32_t* scores;                // original order
    uint32_t* flag_list;            // sorted positions to rescore in int32
    uint32_t* flag_count;
    // scheduling
    uint32_t* work_counter;
    uint32_t* status;               // nonzero after an internal error
};

struct KernelChoice {
    int R;        // query rows per thread in the short bin
    bool pair;    // two sequences per group in packed 16-bit lanes; else one in int32
};

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

// Tile layout: gather database residues into tiles (device side).
cudaError_t launch_build_tiles(const uint8_t* residues, const uint64_t* offsets,
                               const uint32_t* sorted_ids, uint64_t n_sorted,
                               const uint64_t* tile_off, const uint32_t* tile_len,
                               uint64_t n_tiles, uint8_t* tile_data, cudaStream_t stream);
cudaError_t launch_max_code(const uint8_t* residues, uint64_t n, uint32_t* out,
                            cudaStream_t stream);

// Top-k over nq score rows of length n (row q at scores + q * row_stride).
struct TopkScratch {
    uint32_t* hist;        // nq * 2048
    uint32_t* state;       // nq * 8
    uint32_t* block_eq;    // nq * topk_blocks
    int32_t* cand_score;   // nq * kmax
    uint32_t* cand_index;  // nq * kmax (uint32 indices; n < 2^32)
    int blocks;
};
size_t topk_scratch_bytes(uint32_t nq, uint32_t kmax, int blocks);
void topk_scratch_carve(void* base, uint32_t nq, uint32_t kmax, int blocks, TopkScratch* s);
int topk_launch_count();  // kernels one launch_topk call enqueues
cudaError_t launch_topk(const int32_t* scores, uint64_t row_stride, uint64_t n, uint32_t nq,
                        uint32_t k, const TopkScratch& s, int32_t* top_scores,
                        uint64_t* top_index, cudaStream_t stream);

}  // namespace swgb
