// Traceback: one optimal local alignment per requested database sequence.
//
// Section IV.C leaves the alignments themselves (not only their scores) to
// future work; a database search reports them for its top hits. Three
// dynamic programmes per (query, sequence) pair, in int32, each a lane
// wavefront of one warp (lane t on column s - t at step s, kR query rows per
// lane, passes of 32 kR rows with the bottom row kept in the warp's scratch,
// scores from the warp's score ring; a block is one warp, so the hits spread
// over every SM):
//
//  1. recurrence (1) with the score S and the end cell: the first (i, j), in
//     order of i then j, whose H equals S;
//  2. the same gap model run backwards from the end cell and anchored there
//     (no zero floor): the start cell is the first cell in that reversed order
//     whose aligned-pair value equals S, i.e. the latest start of an optimal
//     alignment ending at the end cell;
//  3. the three-state programme (M: a pair aligned, E: a query residue
//     against a gap, F: a database residue against a gap) over the box between
//     the two cells, anchored at both, writing for every cell which state
//     gives H (M, then E, then F on ties) and whether E and F extend (extension
//     preferred on ties) as one byte; lane 0 then walks the bytes back from M
//     at the end cell and writes the op string.
//
// Hits of at least kLongCells cells run programmes 1 and 2 in a second kernel,
// one block of 8 warps each (a wavefront of warps over bands of query rows), on
// a second stream beside the one-warp kernel.
//
// The end and start cells and the tie rules make the alignment unique, so it
// can be compared letter for letter.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "sw.h"
#include "sw_blockwave.cuh"
#include "sw_db.h"
#include "sw_internal.h"
#include "sw_lanes.cuh"

namespace swgb {

namespace {

constexpr int kWarps = 1;  // one warp per block: the hits spread over every SM
constexpr int kThreads = kWarps * 32;
constexpr int kBlocksPerSm = 12;
constexpr int kT = 32;
constexpr int kR = 12;
constexpr int kRows = kT * kR;
constexpr int kM = kProfileRows;
constexpr int32_t kNeg = -(1 << 29);  // minus infinity for the anchored programmes
// hits of this many cells go to the block kernel (measured on the top 10 hits of 20
// queries of 144..5,478 residues against 2 M sequences: 2^20 4.9 ms per batch, 2^21
// 7.1 ms, 2^22 11.6 ms)
constexpr uint64_t kLongCells = 1ull << 20;

struct AlignHit {
    uint64_t sp;        // sorted position of the sequence
    uint32_t n;         // its length
    uint32_t q_len;     // the query: length and offset in the concatenated queries
    uint64_t q_off;
    int32_t score;      // phase 0 outputs
    uint32_t ie, je, is, js;
    uint32_t ops_len;   // phase 1 output (0xffffffff: inconsistent bytes, see below)
    uint64_t dir_off;   // phase 1 inputs: offsets of its box bytes and of its ops
    uint64_t ops_off;
};

struct AlignArgs {
    const uint8_t* tile_data;
    const uint64_t* tile_off;
    const uint8_t* query;   // concatenated queries (AlignHit::q_off)
    const int8_t* matrix;
    uint32_t alphabet;
    int32_t alpha, beta;
    AlignHit* hits;
    uint32_t first, count;
    uint2* boundary;    // per warp: two halves of bstride / 2 entries
    uint64_t bstride;
    uint8_t* dir;
    char* ops;
    int phase;          // 0: score, end and start cells; 1: box programme and traceback
    uint64_t long_cells;        // phase 0: hits of at least this many cells go to the block
    const uint32_t* long_list;  //   kernel (their indices; 0 cells: none)
    uint32_t n_long;
    uint64_t long_row0;         // the block kernel's scratch rows start at this entry
    uint32_t* dbg;      // error word of the bounds-checked build
    uint64_t dir_cap;   // bytes of dir (checked)
};

__device__ __forceinline__ int32_t imax(int32_t a, int32_t b) { return a > b ? a : b; }

// The warp's score ring (the score profile of Section III.B.2 over a window of
// columns): word [c][j mod kW] = fsbt(c, d_j) for every query code c and the columns a
// 32-step block touches (its 32 and the 31 the lane skew reaches back); slots below kD
// are also kept at kW + slot so a sub-block of 8 steps reads 8 consecutive slots from one
// base. Code rows are kRowWords apart (a multiple of 32) and the 32 lanes read 32
// consecutive columns, so the loads are conflict-free. Row A is zero (rows past the query).
constexpr uint32_t kW = 64;
constexpr uint32_t kD = 8;
constexpr uint32_t kRowWords = 96;
static_assert(kW >= 2 * kT - 1 && kW + kD <= kRowWords && kRowWords % 32 == 0 && kW % 32 == 0,
              "score ring");

struct WarpSmem {
    uint32_t ring[kM * kRowWords];  // (A + 1) code rows used
    uint2 stage[kT];                // lane 0's top entries of the current block
};

// One dynamic programme over rows x cols by one warp. MODE 0: recurrence (1),
// tracking the first maximal cell; MODE 1: anchored at (0, 0), tracking the first
// cell whose aligned-pair value is S; MODE 2: anchored at (0, 0), writing each
// cell's traceback byte to dir[row * cols + col].
template <int MODE, class QF, class DF>
__device__ void run_dp(const AlignArgs& a, const int32_t* sM, WarpSmem& ws, uint2* bnd0,
                       uint64_t half, int t, uint32_t rows, uint32_t cols, QF qf, DF df, int32_t S,
                       int32_t& best, uint32_t& bi, uint32_t& bj, uint8_t* dir) {
    const int32_t border = MODE == 0 ? 0 : kNeg;
    const uint32_t A = a.alphabet;
    const uint32_t P = (rows + kRows - 1) / kRows;
    const uint32_t steps = cols + kT - 1;
    const uint32_t ring_s = (uint32_t)__cvta_generic_to_shared(ws.ring);
    const uint32_t stage_s = (uint32_t)__cvta_generic_to_shared(ws.stage);
    const uint32_t ring_hi = ring_s + (A + 1) * kRowWords * 4;
    auto in_ring = [&](uint32_t addr) { return addr >= ring_s && addr + 4 <= ring_hi; };
    for (uint32_t p = 0; p < P; ++p) {
        // score-ring address of each of this lane's rows at the slot of column -t
        uint32_t addr[kR];
        const uint32_t sl0 = (kW - (uint32_t)t) % kW;
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const uint32_t row = p * kRows + (uint32_t)t * kR + r;
            uint32_t c = row < rows ? qf(row) : A;
            if (c > A) c = A;
            addr[r] = ring_s + (c * kRowWords + sl0) * 4;
        }
        __syncwarp();  // the previous pass has finished reading the ring
        // columns -31 .. -1 score 0 (slots kW - 31 .. kW - 1)
        for (uint32_t i = t; i < A * (kT - 1); i += kT) {
            const uint32_t at = ring_s + ((i / (kT - 1)) * kRowWords + kW - (kT - 1) + i % (kT - 1)) * 4;
            if (sw_ok(in_ring(at), a.dbg, 26)) sts_u32(at, 0u);
        }
        int32_t Hl[kR], Fr[kR];
        uint32_t fx = 0;  // MODE 2: extension bit of Fr[r] in bit r
#pragma unroll
        for (int r = 0; r < kR; ++r) { Hl[r] = border; Fr[r] = border; }
        int32_t hb_out = border, eb_out = border, hdiag0 = border;
        uint32_t ex_out = 0;
        const uint2* bin = bnd0 + (p & 1) * half + kT;
        uint2* bout = bnd0 + ((p + 1) & 1) * half + kT;
        // lane t builds column s0 + t of each block of 32 steps and stages its top-row entry;
        // its code and entry are loaded one block ahead
        auto code_at = [&](uint32_t j) -> uint32_t {
            uint32_t c = j < cols ? df(j) : kPadCode;
            return c > kPadCode ? kPadCode : c;
        };
        const uint2 kBorder = make_uint2((uint32_t)border, MODE == 2 ? ((uint32_t)border << 1)
                                                                     : (uint32_t)border);
        auto top_at = [&](uint32_t j) -> uint2 {
            return (p > 0 && j < cols && sw_ok(kT + (uint64_t)j < half, a.dbg, 22)) ? bin[j] : kBorder;
        };
        uint32_t cnext = code_at(t);
        uint2 tnext = top_at(t);
        for (uint32_t s0 = 0; s0 < steps; s0 += kT) {
            __syncwarp();  // the previous block has finished with the slots and the stage
            {
                const uint32_t j = s0 + (uint32_t)t, d = cnext, sl = j % kW;
                for (uint32_t c = 0; c < A; ++c) {
                    const uint32_t at = ring_s + (c * kRowWords + sl) * 4;
                    const uint32_t v = (uint32_t)sM[c * kM + d];
                    if (sw_ok(in_ring(at), a.dbg, 26)) sts_u32(at, v);
                    if (sl < kD && sw_ok(in_ring(at + kW * 4), a.dbg, 26)) sts_u32(at + kW * 4, v);
                }
                ws.stage[t] = tnext;
                cnext = code_at(j + kT);
                tnext = top_at(j + kT);
            }
            __syncwarp();  // this block's columns and top entries are visible
            for (uint32_t sb = 0; sb < (uint32_t)kT && s0 + sb < steps; sb += 8) {
                const uint32_t st_sb = stage_s + sb * 8;
#pragma unroll
                for (int k8 = 0; k8 < 8; ++k8) {
                    const uint32_t s = s0 + sb + (uint32_t)k8;
                    const int32_t h_in = (int32_t)shfl_up_or_lds<kT>((uint32_t)hb_out, st_sb + k8 * 8);
                    const uint32_t pk = shfl_up_or_lds<kT>(
                        MODE == 2 ? ((uint32_t)eb_out << 1) | ex_out : (uint32_t)eb_out, st_sb + k8 * 8 + 4);
                    const int32_t e_in = MODE == 2 ? ((int32_t)pk >> 1) : (int32_t)pk;
                    uint32_t ex = MODE == 2 ? (pk & 1u) : 0u;
                    const int64_t j = (int64_t)s - t;
                    int32_t diag = hdiag0, E = e_in;
#pragma unroll
                    for (int r = 0; r < kR; ++r) {
                        const uint32_t i = p * kRows + (uint32_t)t * kR + r;
                        const bool valid = i < rows && j >= 0 && j < (int64_t)cols;
                        int32_t sc = 0;
                        if (sw_ok(in_ring(addr[r] + k8 * 4), a.dbg, 26)) sc = (int32_t)lds_u32(addr[r] + k8 * 4);
                        int32_t H, En, Fn;
                        if (MODE == 0) {
                            H = imax(imax(diag + sc, 0), imax(E, Fr[r]));
                            if (valid && (H > best || (H == best && (i < bi || (i == bi && (uint32_t)j < bj))))) {
                                best = H;
                                bi = i;
                                bj = (uint32_t)j;
                            }
                            const int32_t hb = H - a.beta;
                            En = imax(E - a.alpha, hb);
                            Fn = imax(Fr[r] - a.alpha, hb);
                        } else {
                            const int32_t Mv = (i == 0 && j == 0) ? sc : imax(diag + sc, kNeg);
                            const int32_t F = Fr[r];
                            H = imax(Mv, imax(E, F));
                            if (MODE == 1) {
                                if (valid && Mv == S && (i < bi || (i == bi && (uint32_t)j < bj))) {
                                    bi = i;
                                    bj = (uint32_t)j;
                                }
                            } else if (valid && sw_ok((uint64_t)i * cols + (uint64_t)j < (uint64_t)rows * cols,
                                                      a.dbg, 21)) {
                                const uint32_t hsel = (Mv >= E && Mv >= F) ? 0u : (E >= F ? 1u : 2u);
                                dir[(uint64_t)i * cols + (uint64_t)j] =
                                    (uint8_t)(hsel | (ex << 2) | (((fx >> r) & 1u) << 3));
                            }
                            const int32_t hb = H - a.beta;
                            const uint32_t exn = (E - a.alpha >= hb) ? 1u : 0u;
                            const uint32_t fxn = (F - a.alpha >= hb) ? 1u : 0u;
                            En = imax(imax(E - a.alpha, hb), kNeg);
                            Fn = imax(imax(F - a.alpha, hb), kNeg);
                            if (!valid) {
                                H = kNeg;
                                En = kNeg;
                                Fn = kNeg;
                            }
                            ex = valid ? exn : 0u;
                            if (MODE == 2) fx = (fx & ~(1u << r)) | ((valid ? fxn : 0u) << r);
                        }
                        diag = Hl[r];
                        Hl[r] = H;
                        E = En;
                        Fr[r] = Fn;
                    }
                    hb_out = Hl[kR - 1];
                    eb_out = E;
                    ex_out = ex;
                    hdiag0 = h_in;
                    if (t == kT - 1 && p + 1 < P && j >= 0 && j < (int64_t)cols &&
                        sw_ok(kT + (uint64_t)j < half, a.dbg, 23)) {
                        const uint32_t ev = MODE == 2 ? ((uint32_t)eb_out << 1) | ex_out : (uint32_t)eb_out;
                        bout[j] = make_uint2((uint32_t)hb_out, ev);
                    }
                }
                // next sub-block: 8 slots on, wrapping at kW (the lane's slot is kW - t + s)
                const uint32_t sl = (s0 + sb + kW - (uint32_t)t) % kW;
                const uint32_t delta = (sl + 8 < kW ? 8u : 8u - kW) * 4u;
#pragma unroll
                for (int r = 0; r < kR; ++r) addr[r] += delta;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Long hits: programmes 1 and 2 by a block of 8 warps (the wavefront of warps over
// bands of query rows of sw_blockwave.cuh), so the longest hits of a batch do not
// leave one warp working long after the rest of the GPU is done.
// ---------------------------------------------------------------------------
// Phase 0 (score, end and start cells) of the hits in a.long_list, one block each.
__global__ void __launch_bounds__(bw::kThreads) align_long_kernel(const AlignArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    bw::setup(smem, a.matrix, a.alphabet);
    uint2* const row7 = a.boundary + a.long_row0 + (uint64_t)blockIdx.x * a.bstride;
    for (uint32_t x = blockIdx.x; x < a.n_long; x += gridDim.x) {
        AlignHit& hit = a.hits[a.long_list[x]];
        const uint8_t* q = a.query + hit.q_off;
        const uint32_t qlen = hit.q_len;
        const uint64_t sp = hit.sp;
        const uint8_t* seq = a.tile_data + a.tile_off[sp / kTileSeqs] +
                             ((sp >> 1) & (kTilePairs - 1)) * 8 + (sp & 1);
        const uint32_t n = hit.n;
        uint32_t* const dbg = a.dbg;
        auto dcode = [seq, n, dbg](uint32_t j) -> uint32_t {
            return sw_ok(j < n, dbg, 25) ? seq[(size_t)(j >> 2) * 32 + (j & 3) * 2] : kPadCode;
        };
        int32_t best = 0;
        uint32_t bi = 0xffffffffu, bj = 0xffffffffu;
        bw::block_programme<bw::kFirstMax>(smem, a.alphabet, a.alpha, a.beta, row7, a.bstride, dbg,
                                           qlen, n, [q](uint32_t i) -> uint32_t { return q[i]; },
                                           dcode, 0, best, bi, bj);
        uint32_t is = 0, js = 0;
        if (best > 0) {
            const uint32_t ie = bi, je = bj;
            int32_t unused = 0;
            uint32_t ui = 0xffffffffu, uj = 0xffffffffu;
            bw::block_programme<bw::kAnchored>(
                smem, a.alphabet, a.alpha, a.beta, row7, a.bstride, dbg, ie + 1, je + 1,
                [q, ie](uint32_t u) -> uint32_t { return q[ie - u]; },
                [dcode, je](uint32_t v) -> uint32_t { return dcode(je - v); }, best, unused, ui, uj);
            is = ui <= ie ? ie - ui : 0;
            js = uj <= je ? je - uj : 0;
        }
        if (threadIdx.x == 0) {
            hit.score = best;
            hit.ie = best > 0 ? bi : 0;
            hit.je = best > 0 ? bj : 0;
            hit.is = is;
            hit.js = js;
        }
    }
}

__global__ void __launch_bounds__(kThreads) align_kernel(const AlignArgs a) {
    __shared__ int32_t sM[kM * kM];
    __shared__ WarpSmem wsm[kWarps];
    for (uint32_t i = threadIdx.x; i < kM * kM; i += kThreads) {
        const uint32_t r = i / kM, c = i % kM;
        sM[i] = (r < a.alphabet && c < a.alphabet) ? (int32_t)a.matrix[r * a.alphabet + c] : 0;
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, t = threadIdx.x & 31;
    const uint64_t slot = (uint64_t)blockIdx.x * kWarps + w;
    const uint64_t nwarps = (uint64_t)gridDim.x * kWarps;
    uint2* const bnd0 = a.boundary + slot * a.bstride;
    const uint64_t half = a.bstride / 2;
    for (uint64_t h = a.first + slot; h < (uint64_t)a.first + a.count; h += nwarps) {
        AlignHit& hit = a.hits[h];
        const uint8_t* q = a.query + hit.q_off;
        const uint32_t qlen = hit.q_len;
        const uint64_t sp = hit.sp;
        const uint8_t* seq = a.tile_data + a.tile_off[sp / kTileSeqs] +
                             ((sp >> 1) & (kTilePairs - 1)) * 8 + (sp & 1);
        const uint32_t n = hit.n;
        uint32_t* const dbg = a.dbg;
        auto dcode = [seq, n, dbg](uint32_t j) -> uint32_t {
            return sw_ok(j < n, dbg, 25) ? seq[(size_t)(j >> 2) * 32 + (j & 3) * 2] : kPadCode;
        };
        if (a.phase == 0) {
            if (a.long_cells && (uint64_t)qlen * n >= a.long_cells) continue;  // the block kernel's
            int32_t best = 0;
            uint32_t bi = 0xffffffffu, bj = 0xffffffffu;
            if (qlen && n)
                run_dp<0>(a, sM, wsm[w], bnd0, half, t, qlen, n, [q](uint32_t i) -> uint32_t { return q[i]; },
                          dcode, 0, best, bi, bj, nullptr);
            // first maximal cell over the warp
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
            uint32_t is = 0, js = 0;
            if (best > 0) {
                const uint32_t ie = bi, je = bj;
                int32_t unused = 0;
                uint32_t ui = 0xffffffffu, uj = 0xffffffffu;
                run_dp<1>(a, sM, wsm[w], bnd0, half, t, ie + 1, je + 1,
                          [q, ie](uint32_t u) -> uint32_t { return q[ie - u]; },
                          [dcode, je](uint32_t v) -> uint32_t { return dcode(je - v); }, best, unused,
                          ui, uj, nullptr);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const uint32_t oi = __shfl_xor_sync(0xffffffffu, ui, o);
                    const uint32_t oj = __shfl_xor_sync(0xffffffffu, uj, o);
                    if (oi < ui || (oi == ui && oj < uj)) {
                        ui = oi;
                        uj = oj;
                    }
                }
                // ui is always found (the optimal alignment starts somewhere); guard anyway
                is = ui <= ie ? ie - ui : 0;
                js = uj <= je ? je - uj : 0;
            }
            if (t == 0) {
                hit.score = best;
                hit.ie = best > 0 ? bi : 0;
                hit.je = best > 0 ? bj : 0;
                hit.is = is;
                hit.js = js;
            }
        } else {
            if (hit.score <= 0) {
                if (t == 0) hit.ops_len = 0;
                continue;
            }
            const uint32_t is = hit.is, js = hit.js;
            const uint32_t rows = hit.ie - is + 1, cols = hit.je - js + 1;
            if (!sw_ok(hit.dir_off + (uint64_t)rows * cols <= a.dir_cap, a.dbg, 24)) {
                if (t == 0) hit.ops_len = 0xffffffffu;
                continue;
            }
            uint8_t* dir = a.dir + hit.dir_off;
            int32_t unused = 0;
            uint32_t ui = 0, uj = 0;
            run_dp<2>(a, sM, wsm[w], bnd0, half, t, rows, cols,
                      [q, is](uint32_t u) -> uint32_t { return q[is + u]; },
                      [dcode, js](uint32_t v) -> uint32_t { return dcode(js + v); }, hit.score,
                      unused, ui, uj, dir);
            __syncwarp();
            if (t == 0) {
                // walk back from M at the end cell; letters come out reversed
                char* out = a.ops + hit.ops_off;
                const uint32_t cap = rows + cols;
                uint32_t u = rows - 1, v = cols - 1, len = 0, state = 0;
                bool ok = true;
                for (;;) {
                    if (len >= cap) { ok = false; break; }
                    const uint8_t b = dir[(uint64_t)u * cols + v];
                    if (state == 0) {
                        out[len++] = 'M';
                        if (u == 0 && v == 0) break;
                        if (u == 0 || v == 0) { ok = false; break; }
                        --u;
                        --v;
                        state = dir[(uint64_t)u * cols + v] & 3u;
                    } else if (state == 1) {
                        out[len++] = 'I';
                        if (u == 0) { ok = false; break; }
                        --u;
                        state = ((b >> 2) & 1u) ? 1u : (dir[(uint64_t)u * cols + v] & 3u);
                    } else {
                        out[len++] = 'D';
                        if (v == 0) { ok = false; break; }
                        --v;
                        state = ((b >> 3) & 1u) ? 2u : (dir[(uint64_t)u * cols + v] & 3u);
                    }
                    if (state > 2) { ok = false; break; }
                }
                if (ok) {
                    for (uint32_t k = 0; k < len / 2; ++k) {
                        const char c = out[k];
                        out[k] = out[len - 1 - k];
                        out[len - 1 - k] = c;
                    }
                }
                hit.ops_len = ok ? len : 0xffffffffu;
            }
        }
    }
}

}  // namespace

}  // namespace swgb

using namespace swgb;

namespace {

// Shared by sw_align and sw_align_batch: hits[k].q_off / q_len / sp / n are set, the
// queries and the matrix are on the device at d_queries / db->d_matrix.
sw_status align_hits(sw_db* db, const uint8_t* d_queries, int32_t alpha, int32_t beta,
                     std::vector<AlignHit>& hits, const uint64_t* db_index, sw_alignment* out,
                     char* ops, uint64_t ops_cap, uint64_t* ops_used) {
    sw_status st;
    const uint32_t n = (uint32_t)hits.size();
    // hits of at least kLongCells cells take phase 0 in the block kernel, one block each
    std::vector<uint32_t> long_list;
    for (uint32_t k = 0; k < n; ++k)
        if ((uint64_t)hits[k].q_len * hits[k].n >= kLongCells) long_list.push_back(k);
    const uint32_t n_long = (uint32_t)long_list.size();
    // scratch (grow-only buffers of the handle): per-warp rows (then one row per block of
    // the long hits' kernel), the hit table and the long list, and per batch the box bytes
    // and the op strings
    const uint64_t bstride = 2ull * (((uint64_t)db->max_len + kT + 8 + 3) & ~3ull);
    const uint64_t warp_bytes = bstride * sizeof(uint2);
    const int grid = (int)std::max<uint64_t>(
        1, std::min<uint64_t>({(uint64_t)db->nsm * kBlocksPerSm, (n + kWarps - 1) / kWarps,
                               (256ull << 20) / (warp_bytes * kWarps) + 1}));
    const int grid_long = (int)std::min<uint64_t>(n_long, (uint64_t)db->nsm * 2);
    const size_t hit_bytes = ((size_t)n * sizeof(AlignHit) + 15) & ~(size_t)15;
    if ((st = ensure(db, db->a_rows, ((size_t)grid * kWarps + grid_long) * warp_bytes,
                     "sw_align: scratch rows")) ||
        (st = ensure(db, db->a_hits, hit_bytes + (size_t)n * 4, "sw_align: hit table")))
        return st;
    if (n_long && !db->a_stream) {
        cudaError_t e0;
        if ((e0 = cudaStreamCreateWithFlags(&db->a_stream, cudaStreamNonBlocking)) != cudaSuccess ||
            (e0 = cudaEventCreateWithFlags(&db->a_ev0, cudaEventDisableTiming)) != cudaSuccess ||
            (e0 = cudaEventCreateWithFlags(&db->a_ev1, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(e0, "sw_align: second stream");
    }
    AlignHit* const d_hits = (AlignHit*)db->a_hits.p;
    uint32_t* const d_long = (uint32_t*)((uint8_t*)db->a_hits.p + hit_bytes);
    AlignArgs a{};
    a.tile_data = db->d_tile_data;
    a.tile_off = db->d_tile_off;
    a.query = d_queries;
    a.matrix = db->d_matrix;
    a.alphabet = db->alphabet;
    a.alpha = alpha;
    a.beta = beta;
    a.hits = d_hits;
    a.boundary = (uint2*)db->a_rows.p;
    a.bstride = bstride;
    a.dbg = db->d_counters + kDebugWord;
    cudaError_t e;
    // phase 0: scores, end and start cells of every hit; the long hits' block kernel runs
    // on the second stream beside the one-warp kernel
    if ((e = cudaMemcpyAsync(d_hits, hits.data(), n * sizeof(AlignHit), cudaMemcpyHostToDevice,
                             db->stream)) != cudaSuccess ||
        (n_long && (e = cudaMemcpyAsync(d_long, long_list.data(), (size_t)n_long * 4,
                                        cudaMemcpyHostToDevice, db->stream)) != cudaSuccess))
        return cuda_fail(e, "sw_align: upload");
    a.first = 0;
    a.count = n;
    a.phase = 0;
    a.long_cells = n_long ? kLongCells : 0;
    a.long_list = d_long;
    a.n_long = n_long;
    a.long_row0 = (uint64_t)grid * kWarps * bstride;
    if (n_long) {
        const uint32_t bytes = bw::smem_bytes(db->alphabet);
        if ((e = cudaEventRecord(db->a_ev0, db->stream)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(db->a_stream, db->a_ev0, 0)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(align_long_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)bytes)) != cudaSuccess)
            return cuda_fail(e, "sw_align: long hits");
        align_long_kernel<<<grid_long, bw::kThreads, bytes, db->a_stream>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess ||
            (e = cudaEventRecord(db->a_ev1, db->a_stream)) != cudaSuccess)
            return cuda_fail(e, "sw_align: long hits");
    }
    align_kernel<<<grid, kThreads, 0, db->stream>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (n_long && (e = cudaStreamWaitEvent(db->stream, db->a_ev1, 0)) != cudaSuccess) ||
        (e = cudaMemcpyAsync(hits.data(), d_hits, n * sizeof(AlignHit), cudaMemcpyDeviceToHost,
                             db->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(db->stream)) != cudaSuccess)
        return cuda_fail(e, "sw_align: score and end cells");

    // phase 1 in batches whose box bytes fit 1 GiB (a larger single box takes its size)
    auto box_of = [](const AlignHit& h) -> uint64_t {
        return h.score > 0 ? (uint64_t)(h.ie - h.is + 1) * (h.je - h.js + 1) : 0;
    };
    const uint64_t kDirBudget = 1ull << 30;
    uint64_t ops_total = 0;
    for (auto& h : hits) {
        h.ops_off = ops_total;
        if (h.score > 0) ops_total += (uint64_t)(h.ie - h.is + 1) + (h.je - h.js + 1);
    }
    std::vector<std::pair<uint32_t, uint32_t>> batches;
    uint64_t dir_need = 0;
    for (uint32_t b0 = 0; b0 < n;) {
        uint64_t used = 0;
        uint32_t b1 = b0;
        for (; b1 < n; ++b1) {
            const uint64_t box = (box_of(hits[b1]) + 15) & ~15ull;
            if (b1 > b0 && used + box > kDirBudget) break;
            hits[b1].dir_off = used;
            used += box;
        }
        batches.push_back({b0, b1});
        dir_need = std::max(dir_need, used);
        b0 = b1;
    }
    if ((st = ensure(db, db->a_dir, std::max<uint64_t>(dir_need, 256), "sw_align: traceback bytes")) ||
        (st = ensure(db, db->a_ops, std::max<uint64_t>(ops_total, 256), "sw_align: op strings")))
        return st;
    a.dir = (uint8_t*)db->a_dir.p;
    a.dir_cap = db->a_dir.cap;
    a.ops = (char*)db->a_ops.p;
    a.phase = 1;
    e = cudaMemcpyAsync(d_hits, hits.data(), n * sizeof(AlignHit), cudaMemcpyHostToDevice,
                        db->stream);
    for (size_t bi = 0; bi < batches.size() && e == cudaSuccess; ++bi) {
        a.first = batches[bi].first;
        a.count = batches[bi].second - batches[bi].first;
        align_kernel<<<grid, kThreads, 0, db->stream>>>(a);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hits.data(), d_hits, n * sizeof(AlignHit), cudaMemcpyDeviceToHost,
                            db->stream);
    std::vector<char> host_ops(ops_total);
    if (e == cudaSuccess && ops_total)
        e = cudaMemcpyAsync(host_ops.data(), db->a_ops.p, ops_total, cudaMemcpyDeviceToHost,
                            db->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(db->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sw_align: traceback");
    uint64_t total = 0;
    for (auto& h : hits) {
        if (h.ops_len == 0xffffffffu)
            return fail(SW_ERR_INTERNAL, "sw_align: traceback left its box");
        total += h.ops_len;
    }
    *ops_used = total;
    if (total > ops_cap || (total && !ops))
        return fail(SW_ERR_INVALID_ARG, "sw_align: ops buffer holds %llu letters, %llu needed",
                    (unsigned long long)ops_cap, (unsigned long long)total);
    uint64_t pos = 0;
    for (uint32_t k = 0; k < n; ++k) {
        const AlignHit& h = hits[k];
        sw_alignment& o = out[k];
        o.db_index = db_index[k];
        o.score = h.score;
        o.q_begin = h.score > 0 ? h.is : 0;
        o.q_end = h.score > 0 ? h.ie + 1 : 0;
        o.d_begin = h.score > 0 ? h.js : 0;
        o.d_end = h.score > 0 ? h.je + 1 : 0;
        o.ops_offset = pos;
        o.ops_len = h.ops_len;
        if (h.ops_len) std::memcpy(ops + pos, host_ops.data() + h.ops_off, h.ops_len);
        pos += h.ops_len;
    }
    return SW_OK;
}

sw_status make_hits(const sw_db* db, const uint64_t* db_index, uint32_t n, const char* fn,
                    std::vector<AlignHit>& hits) {
    hits.assign(n, AlignHit{});
    for (uint32_t k = 0; k < n; ++k) {
        if (db_index[k] >= db->n_seqs)
            return fail(SW_ERR_INVALID_ARG, "%s: db_index %llu out of range", fn,
                        (unsigned long long)db_index[k]);
        hits[k].sp = db->pos_of[db_index[k]];
        hits[k].n = db->seq_len[db_index[k]];
    }
    return SW_OK;
}

}  // namespace

extern "C" sw_status sw_align(sw_db* db, const uint8_t* query, uint32_t qlen, const int8_t* matrix,
                              int32_t alpha, int32_t beta, const uint64_t* db_index, uint32_t n,
                              sw_alignment* out, char* ops, uint64_t ops_cap, uint64_t* ops_used) {
    clear_error();
    sw_status st;
    if ((st = check_common(db, qlen, alpha, beta, 0, "sw_align"))) return st;
    if ((st = validate_host_query(db, query, qlen, matrix, "sw_align"))) return st;
    if (n && (!db_index || !out)) return fail(SW_ERR_INVALID_ARG, "sw_align: NULL db_index or out");
    if (!ops_used) return fail(SW_ERR_INVALID_ARG, "sw_align: NULL ops_used");
    *ops_used = 0;
    if (n == 0) return SW_OK;
    std::vector<AlignHit> hits;
    if ((st = make_hits(db, db_index, n, "sw_align", hits))) return st;
    for (auto& h : hits) {
        h.q_off = 0;
        h.q_len = qlen;
    }
    DeviceScope scope(db->device);
    if ((st = stage_query(db, query, qlen, matrix))) return st;
    return align_hits(db, db->d_query, alpha, beta, hits, db_index, out, ops, ops_cap, ops_used);
}

extern "C" sw_status sw_align_batch(sw_db* db, uint32_t nq, const uint8_t* queries,
                                    const uint64_t* qoffsets, const int8_t* matrix, int32_t alpha,
                                    int32_t beta, const uint32_t* hit_query, const uint64_t* db_index,
                                    uint32_t n, sw_alignment* out, char* ops, uint64_t ops_cap,
                                    uint64_t* ops_used) {
    clear_error();
    sw_status st;
    if ((st = check_common(db, 1, alpha, beta, 0, "sw_align_batch"))) return st;
    if (!qoffsets || !queries || !matrix)
        return fail(SW_ERR_INVALID_ARG, "sw_align_batch: NULL queries, offsets or matrix");
    if (n && (!db_index || !hit_query || !out))
        return fail(SW_ERR_INVALID_ARG, "sw_align_batch: NULL hit_query, db_index or out");
    if (!ops_used) return fail(SW_ERR_INVALID_ARG, "sw_align_batch: NULL ops_used");
    *ops_used = 0;
    for (uint32_t q = 0; q < nq; ++q)
        if (qoffsets[q + 1] <= qoffsets[q] || qoffsets[q + 1] - qoffsets[q] > 0x7fffffffull)
            return fail(SW_ERR_INVALID_ARG, "sw_align_batch: query %u is empty or offsets are bad", q);
    const uint64_t total = qoffsets[nq] - qoffsets[0];
    for (uint64_t i = 0; i < total; ++i)
        if (queries[qoffsets[0] + i] >= db->alphabet)
            return fail(SW_ERR_INVALID_ARG, "sw_align_batch: query code %u is not below alphabet %u",
                        queries[qoffsets[0] + i], db->alphabet);
    if (n == 0) return SW_OK;
    std::vector<AlignHit> hits;
    if ((st = make_hits(db, db_index, n, "sw_align_batch", hits))) return st;
    for (uint32_t k = 0; k < n; ++k) {
        if (hit_query[k] >= nq)
            return fail(SW_ERR_INVALID_ARG, "sw_align_batch: hit_query %u out of range", hit_query[k]);
        hits[k].q_off = qoffsets[hit_query[k]] - qoffsets[0];
        hits[k].q_len = (uint32_t)(qoffsets[hit_query[k] + 1] - qoffsets[hit_query[k]]);
    }
    DeviceScope scope(db->device);
    cudaError_t e;
    if ((st = ensure(db, db->b_queries, std::max<uint64_t>(total, 16), "sw_align_batch: queries")))
        return st;
    if ((e = cudaMemcpyAsync(db->b_queries.p, queries + qoffsets[0], total, cudaMemcpyHostToDevice,
                             db->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(db->d_matrix, matrix, (size_t)db->alphabet * db->alphabet,
                             cudaMemcpyHostToDevice, db->stream)) != cudaSuccess)
        return cuda_fail(e, "sw_align_batch: upload");
    return align_hits(db, (const uint8_t*)db->b_queries.p, alpha, beta, hits, db_index, out, ops,
                      ops_cap, ops_used);
}
