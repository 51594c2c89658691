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
// step s). Time is cut into super-steps of kC lane-steps separated by
// __syncthreads: at super-step k, warp w works on block g = k - 2w of its band
// sequence (band w + 8 (g / NBP), column block g % NBP), so warp w + 1 runs two
// blocks (at least 64 columns, more than the 31-column lane skew) behind warp w
// and reads the rows it needs from warp w's shared-memory ring of bottom rows.
// Warp 7 hands its bottom rows to warp 0's next band through a global scratch
// row; NBP >= 16 column blocks per band keeps that row written before warp 0
// reads it. No thread waits on another except at the block barriers.
//
// Scores come from a per-warp score ring, the score profile of Section III.B.2
// built per block of columns: word [c][j mod kW] = fsbt(c, d_j) for every query
// code c and the kW most recent columns j. A lane reads the score of each of its
// rows with one conflict-free shared load at a fixed offset from a per-row
// address (the 32 lanes read 32 consecutive columns of rows a multiple of 32
// words apart). Lane 0's top inputs for the block are staged in shared memory
// and read by the lanes' shuffle (shfl_up_or_lds), so no lane takes a branch of
// its own inside the step loop.
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
constexpr int kC = 64;              // lane-steps per super-step (a multiple of 8)
constexpr int kRing = 4 * kC;       // bottom-row entries kept per warp
constexpr int kLag = 2;             // blocks between consecutive warps
constexpr int kMinNBP = 16;         // > kLag * (kWarps - 1) + 1
constexpr int kM = kProfileRows;    // matrix staged as [33][33], pad row/column zero
// score ring: columns c0 - 31 .. c0 + 63 are live during a block, so kW = 96 slots; a
// sub-block of 8 steps reads 8 consecutive slots from one base, so slots below kD are
// also kept at kW + slot; a code row is kRowWords words (a multiple of 32)
constexpr uint32_t kW = 96;
constexpr uint32_t kD = 8;
constexpr uint32_t kRowWords = 128;
static_assert(kW >= (uint32_t)(kT - 1 + kC) && kW + kD <= kRowWords && kRowWords % 32 == 0,
              "score ring");
static_assert(kW % 32 == 0, "a wrapped lane window must stay conflict-free");

// Dynamic shared memory, in bytes.
constexpr uint32_t kOffM = 0;
constexpr uint32_t kOffOut = (kM * kM * 4 + 15) & ~15u;               // uint2 [kWarps][kRing]
constexpr uint32_t kOffStage = kOffOut + kWarps * kRing * 8;          // uint2 [kWarps][kC]
constexpr uint32_t kOffBest = kOffStage + kWarps * kC * 8;            // int32 [kWarps] + entry
constexpr uint32_t kOffRing = kOffBest + 64;                          // int32 [kWarps][A+1][row]

__host__ __device__ constexpr uint32_t smem_bytes(uint32_t alphabet) {
    return kOffRing + kWarps * (alphabet + 1) * kRowWords * 4;
}

__global__ void __launch_bounds__(kThreads) rescore_kernel(const RescoreArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    int32_t* const M = reinterpret_cast<int32_t*>(smem + kOffM);
    int32_t* const best_w = reinterpret_cast<int32_t*>(smem + kOffBest);
    uint32_t* const entry_s = reinterpret_cast<uint32_t*>(smem + kOffBest + 32);
    const uint32_t A = a.alphabet;
    const uint32_t smem_s = (uint32_t)__cvta_generic_to_shared(smem);

    for (uint32_t i = threadIdx.x; i < kM * kM; i += kThreads) {
        const uint32_t r = i / kM, c = i % kM;
        M[i] = (r < A && c < A) ? (int32_t)a.matrix[r * A + c] : 0;
    }
    const int w = threadIdx.x >> 5, t = threadIdx.x & 31;
    // this warp's score ring: code row c at ring_w + c * kRowWords * 4; row A stays zero
    // (query rows past the query)
    const uint32_t ring_w = smem_s + kOffRing + (uint32_t)w * (A + 1) * kRowWords * 4;
    const uint32_t ring_lo = ring_w, ring_hi = ring_w + (A + 1) * kRowWords * 4;
    auto in_ring = [&](uint32_t addr) { return addr >= ring_lo && addr + 4 <= ring_hi; };
    for (uint32_t i = t; i < kRowWords; i += 32) sts_u32(ring_w + (A * kRowWords + i) * 4, 0u);
    const uint32_t stage_w = smem_s + kOffStage + (uint32_t)w * kC * 8;
    uint2* const stage_p = reinterpret_cast<uint2*>(smem + kOffStage) + w * kC;
    uint2* const out_ring = reinterpret_cast<uint2*>(smem + kOffOut);  // [kWarps][kRing]

    uint2* const row7 = a.boundary + (uint64_t)blockIdx.x * a.bstride;  // warp 7 -> warp 0
    const uint32_t count = min(*a.count, a.cap);
    const int32_t nalpha = -a.alpha, nbeta = -a.beta;

    for (;;) {
        __syncthreads();  // the previous pair is finished with the shared state
        if (threadIdx.x == 0) *entry_s = atomicAdd(a.work_counter, 1u);
        __syncthreads();
        const uint32_t e = *entry_s;
        if (e >= count) break;
        const uint2 ent = a.list[e];
        const uint32_t q = ent.x;
        const uint64_t sp = ent.y;
        const uint8_t* qs = a.qoff ? a.query + a.qoff[q] : a.query;
        const uint32_t m = a.qoff ? a.qlen[q] : a.single_qlen;
        const uint64_t tile = sp / kTileSeqs;
        const uint32_t L = a.tile_len[tile];
        const uint64_t pbyte = ((sp >> 1) & (kTilePairs - 1)) * 8 + (sp & 1);
        const uint8_t* stream = a.tile_data + a.tile_off[tile] + pbyte;
        const uint32_t nband = (m + kBand - 1) / kBand;
        const uint32_t ns = (L + kT - 1 + kC - 1) / kC;  // blocks per band
        const uint32_t nbp = ns > (uint32_t)kMinNBP ? ns : (uint32_t)kMinNBP;
        const uint32_t rounds = (nband + kWarps - 1) / kWarps;
        const uint32_t K = kLag * (kWarps - 1) + nbp * rounds;
        auto code_at = [&](uint32_t j) -> uint32_t {
            uint32_t c = kPadCode;
            if (j < L && sw_ok((j >> 2) * 32 + (j & 3) * 2 + pbyte < (uint64_t)L * 8, a.dbg, 12)) {
                c = stream[(size_t)(j >> 2) * 32 + (j & 3) * 2];
                if (c > kPadCode) c = kPadCode;
            }
            return c;
        };

        int32_t best = 0;
        uint32_t cur[kR];  // score-ring address of the code row of each of this lane's rows
        int32_t Hl[kR], Fr[kR];
        int32_t hb_out = 0, eb_out = 0, hdiag0 = 0;
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
                const uint32_t c0 = b * kC;                   // lane 0's first column
                const uint32_t ring_base = round * nbp * kC;  // bottom-ring index of column -31
                if (b == 0) {  // a new band: this lane's rows, empty state, zero columns < 0
#pragma unroll
                    for (int l = 0; l < kR; ++l) {
                        const uint32_t row = band * kBand + t * kR + l;
                        uint32_t c = row < m ? (uint32_t)qs[row] : A;
                        if (c > A) c = A;
                        cur[l] = ring_w + c * kRowWords * 4;  // slot added per sub-block
                        Hl[l] = 0;
                        Fr[l] = 0;
                    }
                    hb_out = eb_out = hdiag0 = 0;
                    // columns -31 .. -1 live in slots kW - 31 .. kW - 1
                    for (uint32_t i = t; i < A * (kT - 1); i += 32) {
                        const uint32_t c = i / (kT - 1), sl = kW - (kT - 1) + i % (kT - 1);
                        if (sw_ok(in_ring(ring_w + (c * kRowWords + sl) * 4), a.dbg, 13))
                            sts_u32(ring_w + (c * kRowWords + sl) * 4, 0u);
                    }
                }
                // build columns c0 + t and c0 + 32 + t of the score ring, stage thread 0's
                // top entries of columns c0 .. c0 + 63
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint32_t j = c0 + (uint32_t)t + 32u * h;
                    const uint32_t d = code_at(j);
                    const uint32_t sl = j % kW;
                    for (uint32_t c = 0; c < A; ++c) {
                        const uint32_t v = (uint32_t)M[c * kM + d];
                        const uint32_t at = ring_w + (c * kRowWords + sl) * 4;
                        if (sw_ok(in_ring(at), a.dbg, 13)) sts_u32(at, v);
                        if (sl < kD && sw_ok(in_ring(at + kW * 4), a.dbg, 13)) sts_u32(at + kW * 4, v);
                    }
                    uint2 top = make_uint2(0, 0);
                    if (j < L) {
                        if (w == 0) {
                            if (band > 0 && sw_ok(j + kT - 1 < a.bstride, a.dbg, 11)) top = row7[j + kT - 1];
                        } else {
                            top = out_ring[(w - 1) * kRing + (ring_base + j + kT - 1) % kRing];
                        }
                    }
                    stage_p[t + 32 * h] = top;
                }
                __syncwarp();  // this block's columns and top entries are visible
                // lane 31 hands its bottom row of column j = c0 + s - 31 on at index
                // ring_base + c0 + s (mod kRing: no wrap inside a block): to the next warp's
                // ring, or from warp 7 to the global row (entry j + 31) for the next band
                const bool put = t == kT - 1 && band + 1 < nband;
                uint2* const out = w + 1 < kWarps
                                       ? out_ring + w * kRing + (ring_base + c0) % kRing
                                       : row7 + c0;
                // slot of lane t's column at the block start
                uint32_t sl = (c0 + kW - (uint32_t)t) % kW;
#pragma unroll 1
                for (uint32_t sb = 0; sb < (uint32_t)kC; sb += 8) {
                    uint32_t addr[kR];
#pragma unroll
                    for (int l = 0; l < kR; ++l) addr[l] = cur[l] + sl * 4;
                    const uint32_t st_sb = stage_w + sb * 8;
                    uint2* const out_sb = out + sb;
#pragma unroll
                    for (int k8 = 0; k8 < 8; ++k8) {
                        const int32_t h_in = (int32_t)shfl_up_or_lds<kT>((uint32_t)hb_out, st_sb + k8 * 8);
                        const int32_t e_in = (int32_t)shfl_up_or_lds<kT>((uint32_t)eb_out, st_sb + k8 * 8 + 4);
                        int32_t diag = hdiag0, E = e_in;
#pragma unroll
                        for (int l = 0; l < kR; ++l) {
                            int32_t sc = 0;
                            if (sw_ok(in_ring(addr[l] + k8 * 4), a.dbg, 13))
                                sc = (int32_t)lds_u32(addr[l] + k8 * 4);
                            const int32_t x = diag + sc;                  // H[i-1][j-1] + fsbt
                            const int32_t H = LaneS32::max3_relu(x, E, Fr[l]);
                            diag = Hl[l];
                            Hl[l] = H;
                            const int32_t hb = H + nbeta;
                            E = LaneS32::addmax(E, nalpha, hb);
                            Fr[l] = LaneS32::addmax(Fr[l], nalpha, hb);
                            best = max(best, x);                          // max H = max(0, max x)
                        }
                        hb_out = Hl[kR - 1];
                        eb_out = E;
                        hdiag0 = h_in;
                        if (put && sw_ok(w + 1 < kWarps || c0 + sb + k8 < a.bstride, a.dbg, 11))
                            out_sb[k8] = make_uint2((uint32_t)hb_out, (uint32_t)eb_out);
                    }
                    sl = sl + 8 < kW ? sl + 8 : sl + 8 - kW;
                }
            }
            __syncthreads();  // this block's rows are visible to the next warp
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            best = max(best, (int32_t)__shfl_xor_sync(0xffffffffu, (uint32_t)best, o));
        if (t == 0) best_w[w] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t v = 0;
            for (int i = 0; i < kWarps; ++i) v = max(v, best_w[i]);
            const uint32_t id = a.sorted_ids[sp];
            if (id != 0xffffffffu) a.scores[(uint64_t)q * a.score_stride + id] = v;
        }
    }
}

}  // namespace

cudaError_t launch_rescore(const RescoreArgs& a, int grid, cudaStream_t stream) {
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    const uint32_t bytes = smem_bytes(a.alphabet);
    cudaError_t e = cudaFuncSetAttribute(rescore_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes);
    if (e != cudaSuccess) return e;
    rescore_kernel<<<grid, kThreads, bytes, stream>>>(a);
    return cudaGetLastError();
}

int rescore_block_threads() { return kThreads; }

int rescore_blocks_per_sm(uint32_t alphabet) {
    const uint32_t bytes = smem_bytes(alphabet);
    if (cudaFuncSetAttribute(rescore_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes) != cudaSuccess)
        return 1;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rescore_kernel, kThreads, bytes) !=
        cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

}  // namespace swgb
