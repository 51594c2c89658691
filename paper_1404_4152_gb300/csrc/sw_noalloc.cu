// sw_search_noalloc: scoring with no device allocation at all.
//
// Who needs it: callers that may not call cudaMalloc. Some host applications
// reserve the whole device memory up front through their own allocator and
// forbid any other allocation; in others cudaMalloc is too costly in the
// loop, because it can synchronise the device and stall unrelated streams.
// Such a caller hands in device buffers it already owns (query, matrix,
// database sequences, score output) and this entry point does the rest.
//
// The working memory the scoring kernel needs (its work counter and the
// per-warp rows that carry H and E between query passes) lives in one
// file-scope device array of fixed size, kNoAllocScratchBytes, which every
// GPU that loads the library keeps until the process exits. Host code never
// uses the array's name as an address: every call looks the address up with
// cudaGetSymbolAddress, with the caller's device current (after a device
// reset the module reloads at another address, so nothing is cached). With
// lazy module loading (the CUDA default) the first such lookup on a device
// loads the module, and that load is when the array and the module's code
// take their device memory; a caller that later hands all remaining memory to
// its own allocator makes one call first (or runs with
// CUDA_MODULE_LOADING=EAGER). Every call shares the array, so calls whose
// work overlaps on the GPU race with each other; the counter area is cleared
// at the start of each call, the rows are always written before they are read.
//
// The kernel is the int32 wavefront of the library's search kernel (a warp per
// sequence, 16 query rows per lane, the query profile staged per pass of 512
// rows), reading the caller's concatenated sequences directly. It marks the
// inputs it cannot score instead of failing the call (the host does not see
// the device buffers): a sequence longer than the fixed rows hold scores -1,
// and any code at or above the alphabet size (in the sequence, or anywhere in
// the query) gives -2.
#include <cuda_runtime.h>

#include <cstdint>

#include "sw.h"
#include "sw_db.h"

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kT = 32;                      // lanes per sequence
constexpr int kR = 16;                      // query rows per lane
constexpr int kRowsPerPass = kT * kR;       // 512
constexpr uint32_t kPad = 32;               // zero-score code
constexpr uint32_t kProfRows = 33;
constexpr int kGrid = 128;                  // persistent blocks that own a row slot
constexpr uint32_t kMaxLenMultiPass = 2048; // longest sequence when the query needs > 1 pass
constexpr size_t kCounterBytes = 256;
constexpr size_t kSlotEntries = 2ull * kMaxLenMultiPass;  // two halves of (H, E) rows
constexpr size_t kNoAllocScratchBytes =
    kCounterBytes + (size_t)kGrid * kWarps * kSlotEntries * sizeof(uint2);  // 32 MiB + 256 B

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct NoAllocArgs {
    const uint8_t* query;
    uint32_t qlen;
    const int8_t* matrix;
    uint32_t alphabet;
    int32_t alpha, beta;
    const uint8_t* residues;
    const uint64_t* offsets;
    uint32_t n_seqs;
    int32_t* scores;
    unsigned char* scratch;  // device address of g_noalloc_scratch
};

__device__ __forceinline__ int32_t sext_byte(uint32_t w, int b) {
    return (int32_t)(int8_t)(uint8_t)(w >> (8 * b));
}

__global__ void __launch_bounds__(kThreads) noalloc_score_kernel(const NoAllocArgs a) {
    __shared__ __align__(16) uint8_t prof[kProfRows * kRowsPerPass];
    __shared__ uint32_t s_chunk;
    __shared__ uint32_t s_bad_query;  // a query code >= alphabet was staged
    if (threadIdx.x == 0) s_bad_query = 0;
    uint32_t* counter = reinterpret_cast<uint32_t*>(a.scratch);
    uint2* rows = reinterpret_cast<uint2*>(a.scratch + kCounterBytes);

    const int warp = threadIdx.x >> 5, t = threadIdx.x & 31;
    const uint32_t P = (a.qlen + kRowsPerPass - 1) / kRowsPerPass;
    uint2* const bnd0 = rows + ((size_t)blockIdx.x * kWarps + warp) * kSlotEntries;
    const uint32_t A = a.alphabet;

    for (;;) {
        if (threadIdx.x == 0) s_chunk = atomicAdd(counter, 1u);
        __syncthreads();
        const uint64_t seq = (uint64_t)s_chunk * kWarps + warp;
        if ((uint64_t)s_chunk * kWarps >= a.n_seqs) break;
        const bool have = seq < a.n_seqs;
        uint64_t o = 0, n = 0;
        if (have) { o = a.offsets[seq]; n = a.offsets[seq + 1] - o; }
        // rows between passes hold at most kMaxLenMultiPass columns
        const bool too_long = P > 1 && n > kMaxLenMultiPass;
        const uint32_t L = (have && !too_long) ? (uint32_t)n : 0u;
        uint32_t Lw = L;
        for (int s = 16; s > 0; s >>= 1) Lw = max(Lw, __shfl_xor_sync(0xffffffffu, Lw, s));
        const uint32_t steps = Lw + kT - 1;
        int32_t best = 0;
        bool seq_bad = false;
        for (uint32_t p = 0; p < P; ++p) {
            __syncthreads();
            for (uint32_t idx = threadIdx.x; idx < kProfRows * (kRowsPerPass / 4); idx += kThreads) {
                const uint32_t r = idx / (kRowsPerPass / 4);
                const uint32_t k4 = (idx % (kRowsPerPass / 4)) * 4;
                uint32_t word = 0;
                for (int b = 0; b < 4; ++b) {
                    const uint32_t row = p * kRowsPerPass + k4 + b;
                    int v = 0;
                    if (row < a.qlen && r < A) {
                        const uint32_t qc = a.query[row];
                        if (qc < A) v = a.matrix[qc * A + r];
                        else if (r == 0) s_bad_query = 1;
                    }
                    word |= ((uint32_t)(uint8_t)(int8_t)v) << (8 * b);
                }
                reinterpret_cast<uint32_t*>(prof)[idx] = word;
            }
            __syncthreads();
            const uint2* bin = bnd0 + (p & 1) * kMaxLenMultiPass;
            uint2* bout = bnd0 + ((p + 1) & 1) * kMaxLenMultiPass;
            int32_t Hl[kR], Fr[kR];
            for (int r = 0; r < kR; ++r) { Hl[r] = 0; Fr[r] = 0; }
            int32_t hb_out = 0, eb_out = 0, hdiag0 = 0;
            bool bad_code = false;
            for (uint32_t s = 0; s < steps; ++s) {
                const int j = (int)s - t;
                int32_t h_in = (int32_t)__shfl_up_sync(0xffffffffu, (uint32_t)hb_out, 1);
                int32_t e_in = (int32_t)__shfl_up_sync(0xffffffffu, (uint32_t)eb_out, 1);
                const bool valid = j >= 0 && j < (int)L;
                if (t == 0) {
                    h_in = 0;
                    e_in = 0;
                    if (p > 0 && valid) { const uint2 v = bin[j]; h_in = (int32_t)v.x; e_in = (int32_t)v.y; }
                }
                uint32_t code = valid ? (uint32_t)a.residues[o + j] : kPad;
                if (valid && code >= A) {
                    bad_code = true;
                    code = kPad;
                }
                const uint4 w = *reinterpret_cast<const uint4*>(prof + code * kRowsPerPass + t * kR);
                const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
                int32_t diag = hdiag0, E = e_in;
                for (int r = 0; r < kR; ++r) {
                    const int32_t sc = sext_byte(ws[r >> 2], r & 3);
                    const int32_t H = max(max(diag + sc, 0), max(E, Fr[r]));
                    diag = Hl[r];
                    Hl[r] = H;
                    E = max(E - a.alpha, H - a.beta);
                    Fr[r] = max(Fr[r] - a.alpha, H - a.beta);
                    best = max(best, H);
                }
                hb_out = Hl[kR - 1];
                eb_out = E;
                hdiag0 = h_in;
                if (t == kT - 1 && p + 1 < P && valid) bout[j] = make_uint2((uint32_t)hb_out, (uint32_t)eb_out);
            }
            seq_bad |= bad_code;
        }
        for (int s = 16; s > 0; s >>= 1) best = max(best, (int32_t)__shfl_xor_sync(0xffffffffu, (uint32_t)best, s));
        seq_bad = __any_sync(0xffffffffu, seq_bad);
        if (have && t == 0) a.scores[seq] = too_long ? -1 : (seq_bad || s_bad_query) ? -2 : best;
        __syncthreads();
    }
}

}  // namespace

extern "C" sw_status sw_search_noalloc(const uint8_t* d_query, uint32_t qlen, const int8_t* d_matrix,
                                       uint32_t alphabet, int32_t alpha, int32_t beta,
                                       const uint8_t* d_residues, const uint64_t* d_offsets,
                                       uint32_t n_seqs, uint32_t max_len, int32_t* d_scores,
                                       void* stream) {
    using namespace swgb;
    clear_error();
    if (!d_query || !d_matrix || !d_offsets || !d_scores || (!d_residues && n_seqs))
        return fail(SW_ERR_INVALID_ARG, "sw_search_noalloc: NULL buffer");
    if (qlen == 0) return fail(SW_ERR_INVALID_ARG, "sw_search_noalloc: qlen must be >= 1");
    if (alphabet == 0 || alphabet > SW_MAX_ALPHABET)
        return fail(SW_ERR_INVALID_ARG, "sw_search_noalloc: alphabet must be 1..32");
    if (alpha < 0 || beta < 0 || alpha > 32767 || beta > 32767)
        return fail(SW_ERR_INVALID_ARG, "sw_search_noalloc: alpha and beta must lie in [0, 32767]");
    if (n_seqs == 0) return SW_OK;
    if (qlen > (uint32_t)kRowsPerPass && max_len > kMaxLenMultiPass)
        return fail(SW_ERR_INVALID_ARG,
                    "sw_search_noalloc: with a query longer than %d residues every sequence must "
                    "be at most %u residues (max_len = %u); the fixed scratch of %zu bytes holds "
                    "no more",
                    kRowsPerPass, kMaxLenMultiPass, max_len, kNoAllocScratchBytes);
    int dev = 0, nsm = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "sw_search_noalloc: cudaGetDevice");
    // looked up on every call: cheap once the module is loaded, and never stale
    void* p = nullptr;
    if ((e = cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess)
        return cuda_fail(e, "sw_search_noalloc: cudaGetSymbolAddress");
    unsigned char* scratch = (unsigned char*)p;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return cuda_fail(e, "sw_search_noalloc: SM count");
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, noalloc_score_kernel, kThreads,
                                                           0)) != cudaSuccess)
        return cuda_fail(e, "sw_search_noalloc: occupancy");
    // a query of one pass uses no rows: every SM gets blocks; otherwise one block per row slot
    int grid = nsm * (per_sm > 0 ? per_sm : 1);
    if (qlen > (uint32_t)kRowsPerPass && grid > kGrid) grid = kGrid;
    cudaStream_t st = (cudaStream_t)stream;
    if ((e = cudaMemsetAsync(scratch, 0, kCounterBytes, st)) != cudaSuccess)
        return cuda_fail(e, "sw_search_noalloc: clearing the work counter");
    NoAllocArgs a{d_query, qlen, d_matrix, alphabet, alpha, beta, d_residues, d_offsets,
                  n_seqs, d_scores, scratch};
    noalloc_score_kernel<<<grid, kThreads, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "sw_search_noalloc: launch");
    return SW_OK;
}
