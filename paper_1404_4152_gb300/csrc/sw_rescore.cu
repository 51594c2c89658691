// Exact int32 rescoring of (query, database sequence) pairs whose 16-bit
// lanes reached the saturation threshold.
//
// The paper keeps scores exact by computing in 32-bit lanes throughout
// (Section III); the packed 16-bit kernels here are exact below a threshold
// and hand every pair that reached it to this kernel, which evaluates
// recurrence (1) again in int32. Such pairs are rare (under BLOSUM62 a score
// must pass ~32,700), so this kernel favours simplicity: a warp per pair, 16
// query rows per lane (512 rows per pass), the scoring matrix in shared
// memory and each lane's query codes for the pass in registers, so a score
// is one shared-memory load per cell. The (H, E) row between passes goes
// through the warp's scratch row, as in the search kernels; lane 0 loads the
// sequence codes and that row one 4-column block ahead.
#include <cuda_runtime.h>
#include <cstdint>

#include "sw_internal.h"
#include "sw_lanes.cuh"

namespace swgb {

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kT = 32;
constexpr int kR = 16;
constexpr int kRows = kT * kR;
constexpr int kM = kProfileRows;  // matrix staged as [33][33], pad row/column zero

__global__ void __launch_bounds__(kThreads) rescore_kernel(const RescoreArgs a) {
    __shared__ int32_t sM[kM * kM];
    for (uint32_t i = threadIdx.x; i < kM * kM; i += kThreads) {
        const uint32_t r = i / kM, c = i % kM;
        sM[i] = (r < a.alphabet && c < a.alphabet) ? (int32_t)a.matrix[r * a.alphabet + c] : 0;
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, t = threadIdx.x & 31;
    const uint64_t slot = (uint64_t)blockIdx.x * kWarps + warp;
    uint2* const bnd0 = a.boundary + slot * a.bstride;
    const uint64_t half = a.bstride / 2;
    const uint32_t count = min(*a.count, a.cap);

    for (;;) {
        uint32_t e = 0;
        if (t == 0) e = atomicAdd(a.work_counter, 1u);
        e = __shfl_sync(0xffffffffu, e, 0);
        if (e >= count) break;
        const uint2 ent = a.list[e];
        const uint32_t q = ent.x;
        const uint64_t sp = ent.y;
        const uint8_t* qs = a.qoff ? a.query + a.qoff[q] : a.query;
        const uint32_t m = a.qoff ? a.qlen[q] : a.single_qlen;
        const uint64_t tile = sp / kTileSeqs;
        const uint32_t L = a.tile_len[tile];
        const uint8_t* stream = a.tile_data + a.tile_off[tile] + ((sp >> 1) & (kTilePairs - 1)) * 8;
        const uint32_t P = (m + kRows - 1) / kRows;
        const uint32_t steps = (L + kT - 1 + 3) & ~3u;
        const uint32_t blocks_real = L / 4;  // 4-column blocks of the sequence (L is a multiple of 4)
        const uint32_t byte_sel = (uint32_t)(sp & 1);
        int32_t best = 0;
        for (uint32_t p = 0; p < P; ++p) {
            // this lane's query codes for the pass (pad code past the query end)
            uint32_t qc[kR];
#pragma unroll
            for (int l = 0; l < kR; ++l) {
                const uint32_t row = p * kRows + t * kR + l;
                uint32_t c = row < m ? (uint32_t)qs[row] : kPadCode;
                qc[l] = (c < a.alphabet ? c : kPadCode) * kM;
            }
            const uint2* bin = bnd0 + (p & 1) * half + kT;
            uint2* bout = bnd0 + ((p + 1) & 1) * half + kT;
            int32_t Hl[kR], Fr[kR];
#pragma unroll
            for (int l = 0; l < kR; ++l) { Hl[l] = 0; Fr[l] = 0; }
            int32_t hb_out = 0, eb_out = 0, hdiag0 = 0;
            uint32_t code_out = kPadCode;
            // lane 0's codes (a word of 4 columns x 2 sequences) and boundary entries,
            // loaded one 4-column block ahead
            const uint2 kPadW = make_uint2(0x20202020u, 0x20202020u);
            uint2 wq = kPadW;
            uint4 bq0 = make_uint4(0, 0, 0, 0), bq1 = make_uint4(0, 0, 0, 0);
            if (t == 0 && blocks_real > 0) {
                wq = *reinterpret_cast<const uint2*>(stream);
                if (p > 0) {
                    bq0 = reinterpret_cast<const uint4*>(bin)[0];
                    bq1 = reinterpret_cast<const uint4*>(bin)[1];
                }
            }
            for (uint32_t s0 = 0; s0 < steps; s0 += 4) {
                uint2 wn = kPadW;
                uint4 bn0 = make_uint4(0, 0, 0, 0), bn1 = make_uint4(0, 0, 0, 0);
                const uint32_t nb = (s0 >> 2) + 1;
                if (t == 0 && nb < blocks_real) {
                    wn = *reinterpret_cast<const uint2*>(stream + (size_t)nb * 32);
                    if (p > 0) {
                        bn0 = reinterpret_cast<const uint4*>(bin + s0 + 4)[0];
                        bn1 = reinterpret_cast<const uint4*>(bin + s0 + 4)[1];
                    }
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    int32_t h_in = (int32_t)__shfl_up_sync(0xffffffffu, (uint32_t)hb_out, 1);
                    int32_t e_in = (int32_t)__shfl_up_sync(0xffffffffu, (uint32_t)eb_out, 1);
                    uint32_t code = __shfl_up_sync(0xffffffffu, code_out, 1);
                    if (t == 0) {
                        const uint32_t w = (k < 2) ? wq.x : wq.y;
                        code = (w >> (16 * (k & 1) + 8 * byte_sel)) & 0xffu;
                        if (code > kPadCode) code = kPadCode;
                        const uint4& bq = (k < 2) ? bq0 : bq1;
                        h_in = (int32_t)((k & 1) ? bq.z : bq.x);
                        e_in = (int32_t)((k & 1) ? bq.w : bq.y);
                    }
                    code_out = code;
                    int32_t diag = hdiag0, E = e_in;
#pragma unroll
                    for (int l = 0; l < kR; ++l) {
                        const int32_t sc = sM[qc[l] + code];
                        const int32_t H = LaneS32::max3_relu(diag + sc, E, Fr[l]);
                        diag = Hl[l];
                        Hl[l] = H;
                        const int32_t hb = H - a.beta;
                        E = max(E - a.alpha, hb);
                        Fr[l] = max(Fr[l] - a.alpha, hb);
                        best = max(best, H);
                    }
                    hb_out = Hl[kR - 1];
                    eb_out = E;
                    hdiag0 = h_in;
                    if (t == kT - 1 && p + 1 < P)  // column s - 31, at entry kT + that >= 1
                        bout[(int)(s0 + k) - (kT - 1)] = make_uint2((uint32_t)hb_out, (uint32_t)eb_out);
                }
                wq = wn;
                bq0 = bn0;
                bq1 = bn1;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            best = max(best, (int32_t)__shfl_xor_sync(0xffffffffu, (uint32_t)best, o));
        if (t == 0) {
            const uint32_t id = a.sorted_ids[sp];
            if (id != 0xffffffffu) a.scores[(uint64_t)q * a.score_stride + id] = best;
        }
    }
}

}  // namespace

cudaError_t launch_rescore(const RescoreArgs& a, int grid, cudaStream_t stream) {
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    rescore_kernel<<<grid, kThreads, 0, stream>>>(a);
    return cudaGetLastError();
}

int rescore_block_threads() { return kThreads; }

}  // namespace swgb
