// One int32 dynamic programme over a (query, database sequence) pair by a whole
// block: the wavefront of warps used by the rescoring kernel (every saturated pair)
// and by the alignment of long hits.
//
// Each warp owns bands of kBand = 32 lanes x kR rows (bands w, w + 8, ...); in
// a band its lanes run the lane wavefront (lane t on column s - t at step s).
// Time is cut into super-steps of kC lane-steps separated by __syncthreads: at
// super-step k, warp w works on block g = k - 2w of its band sequence (band
// w + 8 (g / NBP), column block g % NBP), so warp w + 1 runs two blocks (at
// least 64 columns, more than the 31-column lane skew) behind warp w and reads
// the rows it needs from warp w's shared-memory ring of bottom rows. Warp 7
// hands its bottom rows to warp 0's next band through a global scratch row;
// NBP >= 16 column blocks per band keeps that row written before warp 0 reads
// it. No thread waits on another except at the block barriers.
//
// Scores come from a per-warp score ring, the score profile of Section III.B.2
// built per block of columns: word [c][j mod kW] = fsbt(c, d_j) for every query
// code c and the kW most recent columns j. A lane reads the score of each of its
// rows with one conflict-free shared load at a fixed offset from a per-row
// address (the 32 lanes read 32 consecutive columns of rows a multiple of 32
// words apart). Lane 0's top inputs for the block are staged in shared memory
// and read by the lanes' shuffle (shfl_up_or_lds), so no lane takes a branch of
// its own inside the step loop.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "sw_internal.h"
#include "sw_lanes.cuh"

namespace swgb {
namespace bw {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kT = 32;
constexpr int kR = 8;
constexpr int kBand = kT * kR;      // query rows per band
constexpr int kC = 64;              // lane-steps per super-step (a multiple of 8)
constexpr int kRing = 4 * kC;       // bottom-row entries kept per warp
constexpr int kLag = 2;             // blocks between consecutive warps
constexpr int kMinNBP = 16;         // > kLag * (kWarps - 1) + 1
constexpr uint32_t kM = kProfileRows;  // matrix staged as [33][33], pad row/column zero
constexpr int32_t kNeg = -(1 << 29);   // minus infinity of the anchored programme
// score ring: columns c0 - 31 .. c0 + 63 are live during a block, so kW = 96 slots; a
// sub-block of 8 steps reads 8 consecutive slots from one base, so slots below kD are
// also kept at kW + slot; a code row is kRowWords words (a multiple of 32)
constexpr uint32_t kW = 96;
constexpr uint32_t kD = 8;
constexpr uint32_t kRowWords = 128;
static_assert(kW >= (uint32_t)(kT - 1 + kC) && kW + kD <= kRowWords && kRowWords % 32 == 0,
              "score ring");
static_assert(kW % 32 == 0, "a wrapped lane window must stay conflict-free");

// Dynamic shared memory of a block, in bytes.
constexpr uint32_t kOffM = 0;                                         // int32 [kM][kM]
constexpr uint32_t kOffOut = (kM * kM * 4 + 15) & ~15u;               // uint2 [kWarps][kRing]
constexpr uint32_t kOffStage = kOffOut + kWarps * kRing * 8;          // uint2 [kWarps][kC]
constexpr uint32_t kOffRed = kOffStage + kWarps * kC * 8;             // 3 words per warp + 1
constexpr uint32_t kOffRing = kOffRed + 128;                          // int32 [kWarps][A+1][row]

__host__ __device__ constexpr uint32_t smem_bytes(uint32_t alphabet) {
    return kOffRing + kWarps * (alphabet + 1) * kRowWords * 4;
}

// What the programme computes:
//  kScore:    recurrence (1); its maximum (the score).
//  kFirstMax: recurrence (1); its maximum and the first cell, in order of i then j,
//             that holds it.
//  kAnchored: the same gap model anchored at (0, 0) (no zero floor; minus infinity
//             outside the matrix); the first cell, in order of i then j, whose
//             aligned-pair value is S.
enum Mode { kScore = 0, kFirstMax = 1, kAnchored = 2 };

// Stage the matrix and zero every warp's row A of its score ring (query rows past
// the query); once per kernel, before the first programme (ends with a barrier).
__device__ __forceinline__ void setup(uint8_t* smem, const int8_t* matrix, uint32_t A) {
    int32_t* const M = reinterpret_cast<int32_t*>(smem + kOffM);
    for (uint32_t i = threadIdx.x; i < kM * kM; i += kThreads) {
        const uint32_t r = i / kM, c = i % kM;
        M[i] = (r < A && c < A) ? (int32_t)matrix[r * A + c] : 0;
    }
    const int w = threadIdx.x >> 5, t = threadIdx.x & 31;
    const uint32_t ring_w = (uint32_t)__cvta_generic_to_shared(smem) + kOffRing +
                            (uint32_t)w * (A + 1) * kRowWords * 4;
    for (uint32_t i = t; i < kRowWords; i += 32) sts_u32(ring_w + (A * kRowWords + i) * 4, 0u);
    __syncthreads();
}

// The programme over rows x cols (query codes qf(i), database codes df(j)), by every
// thread of the block; row7 is the block's global scratch row of bstride entries.
// Every thread returns the block's result (best, bi, bj; for kScore only best).
// Bounds-checked build: sites 11 (scratch row), 12 (database codes), 13 (ring).
template <int MODE, class QF, class DF>
__device__ void block_programme(uint8_t* smem, uint32_t A, int32_t alpha, int32_t beta,
                                uint2* row7, uint64_t bstride, uint32_t* dbg, uint32_t rows,
                                uint32_t cols, QF qf, DF df, int32_t S, int32_t& best_out,
                                uint32_t& bi_out, uint32_t& bj_out) {
    const int32_t border = MODE == kAnchored ? kNeg : 0;
    const int32_t* const M = reinterpret_cast<const int32_t*>(smem + kOffM);
    const int w = threadIdx.x >> 5, t = threadIdx.x & 31;
    const uint32_t smem_s = (uint32_t)__cvta_generic_to_shared(smem);
    const uint32_t ring_w = smem_s + kOffRing + (uint32_t)w * (A + 1) * kRowWords * 4;
    const uint32_t ring_hi = ring_w + (A + 1) * kRowWords * 4;
    auto in_ring = [&](uint32_t at) { return at >= ring_w && at + 4 <= ring_hi; };
    const uint32_t stage_w = smem_s + kOffStage + (uint32_t)w * kC * 8;
    uint2* const stage_p = reinterpret_cast<uint2*>(smem + kOffStage) + w * kC;
    uint2* const out_ring = reinterpret_cast<uint2*>(smem + kOffOut);  // [kWarps][kRing]
    const uint2 kBorder = make_uint2((uint32_t)border, (uint32_t)border);
    const int32_t nalpha = -alpha, nbeta = -beta;

    const uint32_t nband = (rows + kBand - 1) / kBand;
    const uint32_t ns = (cols + kT - 1 + kC - 1) / kC;  // blocks per band
    const uint32_t nbp = ns > (uint32_t)kMinNBP ? ns : (uint32_t)kMinNBP;
    const uint32_t rounds = (nband + kWarps - 1) / kWarps;
    const uint32_t K = kLag * (kWarps - 1) + nbp * rounds;

    int32_t best = MODE == kAnchored ? S : 0;
    uint32_t bi = 0xffffffffu, bj = 0xffffffffu;
    uint32_t cur[kR];  // score-ring address of the code row of each of this lane's rows
    int32_t Hl[kR], Fr[kR];
    int32_t hb_out = border, eb_out = border, hdiag0 = border;
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
                    uint32_t c = row < rows ? qf(row) : A;
                    if (c > A) c = A;
                    cur[l] = ring_w + c * kRowWords * 4;  // slot added per sub-block
                    Hl[l] = border;
                    Fr[l] = border;
                }
                hb_out = eb_out = hdiag0 = border;
                // columns -31 .. -1 live in slots kW - 31 .. kW - 1
                for (uint32_t i = t; i < A * (kT - 1); i += 32) {
                    const uint32_t c = i / (kT - 1), sl = kW - (kT - 1) + i % (kT - 1);
                    if (sw_ok(in_ring(ring_w + (c * kRowWords + sl) * 4), dbg, 13))
                        sts_u32(ring_w + (c * kRowWords + sl) * 4, 0u);
                }
            }
            // build columns c0 + t and c0 + 32 + t of the score ring, stage thread 0's
            // top entries of columns c0 .. c0 + 63
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t j = c0 + (uint32_t)t + 32u * h;
                uint32_t d = j < cols ? df(j) : kPadCode;
                if (d > kPadCode) d = kPadCode;
                const uint32_t sl = j % kW;
                for (uint32_t c = 0; c < A; ++c) {
                    const uint32_t v = (uint32_t)M[c * kM + d];
                    const uint32_t at = ring_w + (c * kRowWords + sl) * 4;
                    if (sw_ok(in_ring(at), dbg, 13)) sts_u32(at, v);
                    if (sl < kD && sw_ok(in_ring(at + kW * 4), dbg, 13)) sts_u32(at + kW * 4, v);
                }
                uint2 top = kBorder;
                if (j < cols) {
                    if (w == 0) {
                        if (band > 0 && sw_ok(j + kT - 1 < bstride, dbg, 11)) top = row7[j + kT - 1];
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
            uint2* const out = w + 1 < kWarps ? out_ring + w * kRing + (ring_base + c0) % kRing
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
                    const int64_t j = (int64_t)c0 + sb + k8 - t;
                    int32_t diag = hdiag0, E = e_in;
#pragma unroll
                    for (int l = 0; l < kR; ++l) {
                        int32_t sc = 0;
                        if (sw_ok(in_ring(addr[l] + k8 * 4), dbg, 13))
                            sc = (int32_t)lds_u32(addr[l] + k8 * 4);
                        if (MODE != kAnchored) {
                            const int32_t x = diag + sc;                  // H[i-1][j-1] + fsbt
                            const int32_t H = LaneS32::max3_relu(x, E, Fr[l]);
                            diag = Hl[l];
                            Hl[l] = H;
                            const int32_t hb = H + nbeta;
                            E = LaneS32::addmax(E, nalpha, hb);
                            Fr[l] = LaneS32::addmax(Fr[l], nalpha, hb);
                            if (MODE == kScore) {
                                best = max(best, x);                      // max H = max(0, max x)
                            } else {
                                const uint32_t i = band * kBand + (uint32_t)t * kR + l;
                                const bool valid = i < rows && j >= 0 && j < (int64_t)cols;
                                if (valid && (H > best || (H == best && (i < bi || (i == bi && (uint32_t)j < bj))))) {
                                    best = H;
                                    bi = i;
                                    bj = (uint32_t)j;
                                }
                            }
                        } else {
                            const uint32_t i = band * kBand + (uint32_t)t * kR + l;
                            const bool valid = i < rows && j >= 0 && j < (int64_t)cols;
                            const int32_t Mv = (i == 0 && j == 0) ? sc : max(diag + sc, kNeg);
                            int32_t H = max(Mv, max(E, Fr[l]));
                            if (valid && Mv == S && (i < bi || (i == bi && (uint32_t)j < bj))) {
                                bi = i;
                                bj = (uint32_t)j;
                            }
                            const int32_t hb = H + nbeta;
                            int32_t En = max(max(E + nalpha, hb), kNeg);
                            int32_t Fn = max(max(Fr[l] + nalpha, hb), kNeg);
                            if (!valid) {
                                H = kNeg;
                                En = kNeg;
                                Fn = kNeg;
                            }
                            diag = Hl[l];
                            Hl[l] = H;
                            E = En;
                            Fr[l] = Fn;
                        }
                    }
                    hb_out = Hl[kR - 1];
                    eb_out = E;
                    hdiag0 = h_in;
                    if (put && sw_ok(w + 1 < kWarps || c0 + sb + k8 < bstride, dbg, 11))
                        out_sb[k8] = make_uint2((uint32_t)hb_out, (uint32_t)eb_out);
                }
                sl = sl + 8 < kW ? sl + 8 : sl + 8 - kW;
            }
        }
        __syncthreads();  // this block's rows are visible to the next warp
    }
    // the block's result: the largest value, then the first cell in order of i then j
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int32_t ob = (int32_t)__shfl_xor_sync(0xffffffffu, (uint32_t)best, o);
        const uint32_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
        const uint32_t oj = __shfl_xor_sync(0xffffffffu, bj, o);
        if (ob > best || (ob == best && (oi < bi || (oi == bi && oj < bj)))) {
            best = ob;
            bi = oi;
            bj = oj;
        }
    }
    uint32_t* const red = reinterpret_cast<uint32_t*>(smem + kOffRed);
    if (t == 0) {
        red[3 * w] = (uint32_t)best;
        red[3 * w + 1] = bi;
        red[3 * w + 2] = bj;
    }
    __syncthreads();
    best = (int32_t)red[0];
    bi = red[1];
    bj = red[2];
    for (int v = 1; v < kWarps; ++v) {
        const int32_t ob = (int32_t)red[3 * v];
        const uint32_t oi = red[3 * v + 1], oj = red[3 * v + 2];
        if (ob > best || (ob == best && (oi < bi || (oi == bi && oj < bj)))) {
            best = ob;
            bi = oi;
            bj = oj;
        }
    }
    __syncthreads();  // the reduction words are free again
    best_out = best;
    bi_out = bi;
    bj_out = bj;
}

}  // namespace bw
}  // namespace swgb
