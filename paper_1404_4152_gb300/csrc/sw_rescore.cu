// Exact int32 rescoring of (query, database sequence) pairs whose 16-bit
// lanes reached the saturation threshold.
//
// The paper keeps scores exact by computing in 32-bit lanes throughout
// (Section III); the packed 16-bit kernels here are exact below a threshold
// and hand every pair that reached it to this kernel, which evaluates
// recurrence (1) again in int32. Such pairs are the highest-scoring, hence
// long, ones, and often few, so a whole block works on one pair: a wavefront
// of warps over bands of query rows.
//
// Each warp owns bands of kBand = 32 lanes x kR rows (bands w, w + 8, ...); in
// a band its lanes run the usual lane wavefront (lane t on column s - t at
// step s) with the scoring matrix in shared memory. Time is cut into
// super-steps of kC lane-steps separated by __syncthreads: at super-step k,
// warp w works on block g = k - 2w of its band sequence (band w + 8 (g / NBP),
// column block g % NBP), so warp w + 1 runs two blocks (at least 64 columns,
// more than the 31-column lane skew) behind warp w and reads the rows it
// needs from warp w's shared-memory ring of bottom rows. Warp 7 hands its
// bottom rows to warp 0's next band through a global scratch row; NBP >= 16
// column blocks per band keeps that row written before warp 0 reads it. No
// thread waits on another except at the block barriers.
#include <cuda_runtime.h>
#include <cstdint>

#include "sw_internal.h"
#include "sw_lanes.cuh"

namespace swgb {

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kT = 32;
constexpr int kR = 8;
constexpr int kBand = kT * kR;      // query rows per band
constexpr int kC = 64;              // lane-steps per super-step
constexpr int kRing = 4 * kC;       // bottom-row entries kept per warp
constexpr int kLag = 2;             // blocks between consecutive warps
constexpr int kMinNBP = 16;         // > kLag * (kWarps - 1) + 1
constexpr int kM = kProfileRows;    // matrix staged as [33][33], pad row/column zero

struct Smem {
    int32_t M[kM * kM];
    uint2 ring[kWarps][kRing];      // (H, E) of each warp's bottom row, by column
    uint2 top0[kC];                 // warp 0's top row for the current block
    uint8_t code[kWarps][kC];       // each warp's database codes for the current block
    int32_t best[kWarps];
    uint32_t entry;
};

__global__ void __launch_bounds__(kThreads) rescore_kernel(const RescoreArgs a) {
    __shared__ Smem sm;
    for (uint32_t i = threadIdx.x; i < kM * kM; i += kThreads) {
        const uint32_t r = i / kM, c = i % kM;
        sm.M[i] = (r < a.alphabet && c < a.alphabet) ? (int32_t)a.matrix[r * a.alphabet + c] : 0;
    }

    const int w = threadIdx.x >> 5, t = threadIdx.x & 31;
    uint2* const row7 = a.boundary + (uint64_t)blockIdx.x * a.bstride;  // warp 7 -> warp 0
    const uint32_t count = min(*a.count, a.cap);

    for (;;) {
        __syncthreads();  // the previous pair is finished with the shared state
        if (threadIdx.x == 0) sm.entry = atomicAdd(a.work_counter, 1u);
        __syncthreads();
        const uint32_t e = sm.entry;
        if (e >= count) break;
        const uint2 ent = a.list[e];
        const uint32_t q = ent.x;
        const uint64_t sp = ent.y;
        const uint8_t* qs = a.qoff ? a.query + a.qoff[q] : a.query;
        const uint32_t m = a.qoff ? a.qlen[q] : a.single_qlen;
        const uint64_t tile = sp / kTileSeqs;
        const uint32_t L = a.tile_len[tile];
        const uint8_t* stream =
            a.tile_data + a.tile_off[tile] + ((sp >> 1) & (kTilePairs - 1)) * 8 + (sp & 1);
        const uint32_t nband = (m + kBand - 1) / kBand;
        const uint32_t ns = (L + kT - 1 + kC - 1) / kC;  // blocks per band
        const uint32_t nbp = ns > (uint32_t)kMinNBP ? ns : (uint32_t)kMinNBP;
        const uint32_t rounds = (nband + kWarps - 1) / kWarps;
        const uint32_t K = kLag * (kWarps - 1) + nbp * rounds;

        int32_t best = 0;
        uint32_t qc[kR];
        int32_t Hl[kR], Fr[kR];
        int32_t hb_out = 0, eb_out = 0, hdiag0 = 0;
        uint32_t code_out = kPadCode;
        for (uint32_t k = 0; k < K; ++k) {
            const int64_t g = (int64_t)k - kLag * w;
            bool active = false;
            uint32_t round = 0, b = 0, band = 0;
            if (g >= 0) {
                round = (uint32_t)g / nbp;
                b = (uint32_t)g % nbp;
                band = (uint32_t)w + kWarps * round;
                active = band < nband && b < ns;
            }
            if (active) {
                if (b == 0) {  // a new band: this lane's query codes, empty rows
#pragma unroll
                    for (int l = 0; l < kR; ++l) {
                        const uint32_t row = band * kBand + t * kR + l;
                        const uint32_t c = row < m ? (uint32_t)qs[row] : kPadCode;
                        qc[l] = (c < a.alphabet ? c : kPadCode) * kM;
                        Hl[l] = 0;
                        Fr[l] = 0;
                    }
                    hb_out = eb_out = hdiag0 = 0;
                    code_out = kPadCode;
                }
                // lane 0's inputs for this block: database codes and, for warp 0 after
                // the first round, warp 7's bottom row of the band above
                const uint32_t c0 = b * kC;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint32_t j = c0 + (uint32_t)t + 32u * h;
                    uint32_t c = kPadCode;
                    if (j < L && sw_ok((j >> 2) * 32 + (j & 3) * 2 + ((sp >> 1) & (kTilePairs - 1)) * 8 +
                                           (sp & 1) < (uint64_t)L * 8, a.dbg, 12)) {
                        c = stream[(size_t)(j >> 2) * 32 + (j & 3) * 2];
                        if (c > kPadCode) c = kPadCode;
                    }
                    sm.code[w][t + 32 * h] = (uint8_t)c;
                    if (w == 0)
                        sm.top0[t + 32 * h] = (band > 0 && j < L && sw_ok(j < a.bstride, a.dbg, 11))
                                                  ? row7[j] : make_uint2(0, 0);
                }
                __syncwarp();
                const uint32_t ring_base = round * nbp * kC;  // ring index of column 0 in this round
                for (uint32_t s = 0; s < (uint32_t)kC; ++s) {
                    const uint32_t sigma = c0 + s;  // lane 0's column
                    int32_t h_in = (int32_t)__shfl_up_sync(0xffffffffu, (uint32_t)hb_out, 1);
                    int32_t e_in = (int32_t)__shfl_up_sync(0xffffffffu, (uint32_t)eb_out, 1);
                    uint32_t code = __shfl_up_sync(0xffffffffu, code_out, 1);
                    if (t == 0) {
                        code = sm.code[w][s];
                        uint2 top = make_uint2(0, 0);
                        if (w == 0)
                            top = sm.top0[s];
                        else if (sigma < L)
                            top = sm.ring[w - 1][(ring_base + sigma) % kRing];
                        h_in = (int32_t)top.x;
                        e_in = (int32_t)top.y;
                    }
                    code_out = code;
                    int32_t diag = hdiag0, E = e_in;
#pragma unroll
                    for (int l = 0; l < kR; ++l) {
                        int32_t sc = 0;
                        if (sw_ok(qc[l] + code < (uint32_t)(kM * kM), a.dbg, 13)) sc = sm.M[qc[l] + code];
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
                    const int64_t j = (int64_t)sigma - (kT - 1);  // lane 31's column
                    if (t == kT - 1 && j >= 0 && j < (int64_t)L && band + 1 < nband) {
                        const uint2 v = make_uint2((uint32_t)hb_out, (uint32_t)eb_out);
                        if (w + 1 < kWarps)
                            sm.ring[w][(ring_base + (uint32_t)j) % kRing] = v;
                        else if (sw_ok((uint64_t)j < a.bstride, a.dbg, 11))
                            row7[j] = v;
                    }
                }
            }
            __syncthreads();  // this block's rows are visible to the next warp
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            best = max(best, (int32_t)__shfl_xor_sync(0xffffffffu, (uint32_t)best, o));
        if (t == 0) sm.best[w] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t v = 0;
            for (int i = 0; i < kWarps; ++i) v = max(v, sm.best[i]);
            const uint32_t id = a.sorted_ids[sp];
            if (id != 0xffffffffu) a.scores[(uint64_t)q * a.score_stride + id] = v;
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
