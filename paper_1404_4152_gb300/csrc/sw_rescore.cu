// Exact int32 rescoring of (query, database sequence) pairs whose 16-bit
// lanes reached the saturation threshold, and int32 scoring of the very long
// database sequences (the block route of the search, dense entries).
//
// The paper keeps scores exact by computing in 32-bit lanes throughout
// (Section III); the packed 16-bit kernels here are exact below a threshold
// and hand every pair that reached it to this kernel, which evaluates
// recurrence (1) again in int32. Such pairs are the highest-scoring, hence
// long, ones, and often few, so a whole block works on one pair: the wavefront
// of warps over bands of query rows of sw_blockwave.cuh.
#include <cuda_runtime.h>
#include <cstdint>

#include "sw_blockwave.cuh"
#include "sw_internal.h"

namespace swgb {

namespace {

__global__ void __launch_bounds__(bw::kThreads) rescore_kernel(const RescoreArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    bw::setup(smem, a.matrix, a.alphabet);
    uint32_t* const entry_s = reinterpret_cast<uint32_t*>(smem + bw::kOffRed + 3 * 4 * bw::kWarps);
    uint2* const row7 = a.boundary + (uint64_t)blockIdx.x * a.bstride;  // warp 7 -> warp 0
    const uint32_t count = a.dense_n ? a.dense_count : min(*a.count, a.cap);
    for (;;) {
        __syncthreads();  // the previous pair is finished with the shared state
        if (threadIdx.x == 0) *entry_s = atomicAdd(a.work_counter, 1u);
        __syncthreads();
        const uint32_t e = *entry_s;
        if (e >= count) break;
        const uint2 ent = a.dense_n ? make_uint2(e / a.dense_n, e % a.dense_n) : a.list[e];
        const uint32_t q = ent.x;
        const uint64_t sp = ent.y;
        const uint8_t* qs = a.qoff ? a.query + a.qoff[q] : a.query;
        const uint32_t m = a.qoff ? a.qlen[q] : a.single_qlen;
        const uint64_t tile = sp / kTileSeqs;
        const uint32_t L = a.tile_len[tile];
        const uint64_t pbyte = ((sp >> 1) & (kTilePairs - 1)) * 8 + (sp & 1);
        const uint8_t* stream = a.tile_data + a.tile_off[tile] + pbyte;
        uint32_t* const dbg = a.dbg;
        auto code_at = [stream, pbyte, L, dbg](uint32_t j) -> uint32_t {
            if (!sw_ok((j >> 2) * 32 + (j & 3) * 2 + pbyte < (uint64_t)L * 8, dbg, 12)) return kPadCode;
            return stream[(size_t)(j >> 2) * 32 + (j & 3) * 2];
        };
        int32_t best = 0;
        uint32_t bi = 0, bj = 0;
        bw::block_programme<bw::kScore>(smem, a.alphabet, a.alpha, a.beta, row7, a.bstride, dbg, m, L,
                                        [qs](uint32_t i) -> uint32_t { return qs[i]; }, code_at, 0,
                                        best, bi, bj);
        if (threadIdx.x == 0) {
            const uint32_t id = a.sorted_ids[sp];
            if (id != 0xffffffffu) a.scores[(uint64_t)q * a.score_stride + id] = best;
        }
    }
}

}  // namespace

cudaError_t launch_rescore(const RescoreArgs& a, int grid, cudaStream_t stream) {
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    const uint32_t bytes = bw::smem_bytes(a.alphabet);
    cudaError_t e = cudaFuncSetAttribute(rescore_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes);
    if (e != cudaSuccess) return e;
    rescore_kernel<<<grid, bw::kThreads, bytes, stream>>>(a);
    return cudaGetLastError();
}

int rescore_blocks_per_sm(uint32_t alphabet) {
    const uint32_t bytes = bw::smem_bytes(alphabet);
    if (cudaFuncSetAttribute(rescore_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes) != cudaSuccess)
        return 1;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rescore_kernel, bw::kThreads, bytes) !=
        cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

}  // namespace swgb
