// Wavefront kernels for recurrence (1) of Section II.A (Smith-Waterman with
// affine gaps): the hot loop of a database search.
//
// Design (GB300-first; the paper's Xeon Phi kernels are prior art):
//  - A group of T consecutive lanes cooperates on one unit of work: two
//    alignments held in the two 16-bit halves of every register (packed
//    s16x2 arithmetic, the inter-sequence model of Section III.B with two
//    lanes per register), or one alignment in int32. The two alignments are
//    either one query against two length-sorted database sequences (a single
//    search) or two queries against one database sequence (a batch).
//  - Each thread holds R query rows (H and F of its rows live in registers,
//    the linear-space rows of Section III.A). The database sequence streams
//    through the group one column per step; thread t works on column s - t at
//    step s, so the group sweeps an anti-diagonal band (the minor-diagonal
//    pattern cited in Section I) and hands the bottom row's H and E, and the
//    residue codes of the column, to the next thread with warp shuffles.
//  - A pass covers T*R query rows. Between passes the bottom row is kept in a
//    global scratch row (the paper's tiled computation, Section IV.C; two
//    halves per group, read one / write the other) and the block stages the
//    next T*R rows of the query profile (Section III.B.2) in shared memory.
//  - The integer ALU pipe is the bottleneck: every max, fused add-max and
//    byte permute runs there (16x2 adds run on the FMA pipe). One cell pair
//    costs 3.5 ALU instructions: H as one three-way max with the zero floor,
//    E and F as one fused add-max each, and half of a three-way running max
//    (the diagonal add and H - beta run on the FMA pipe). The three-input and
//    fused forms occupy the ALU pipe two cycles per warp instruction, a plain
//    two-input max one. The int8 query-profile mode adds one permute per row
//    that merges the two database sequences' scores; two queries share the
//    database residue, so their profile entry is already the packed pair.
//  - The running maximum tracks x = H[i-1][j-1] + fsbt instead of H: E and F
//    only carry values strictly below an earlier H (by beta, or as a chain of
//    equal values ending at one), so the largest H of the matrix is
//    max(0, largest x). That keeps x live on the FMA pipe and leaves H a
//    single three-way max with the zero floor.
//  - Exactness: 16-bit lanes wrap, so a lane whose maximum reaches
//    thr16 = 32767 - max(0, max fsbt) is flagged and rescored in int32.
//    Below that threshold no intermediate can leave the 16-bit range
//    (H <= thr16 bounds H + fsbt; E, F >= -beta because H >= 0; E - alpha and
//    F - alpha >= -(alpha + beta) >= -32768 is required of the 16-bit path),
//    and the first cell whose H exceeds it does so through x (its E and F are
//    at most thr16 - beta), which is computed exactly, so the running maximum
//    of a lane that ever exceeded thr16 ends above it.
#include <cuda_runtime.h>
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "sw_internal.h"
#include "sw_lanes.cuh"

namespace swgb {

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
// Columns between consecutive threads of a group in process_chunk: thread t
// works on column s - kSkew * t at step s.
constexpr int kSkew = 2;

// fsbt(q[row], r) for one query row, 0 outside the query or the alphabet.
__device__ __forceinline__ int profile_score(const uint8_t* q, uint32_t qlen, const int8_t* matrix,
                                             uint32_t A, uint32_t row, uint32_t r) {
    if (row >= qlen || r >= A) return 0;
    const uint32_t qc = q[row];
    return qc < A ? (int)matrix[qc * A + r] : 0;
}

template <int R>
__device__ __forceinline__ void load_rows(const uint8_t* p, uint32_t (&w)[R / 4]) {
    if constexpr (R % 16 == 0) {
#pragma unroll
        for (int k = 0; k < R / 16; ++k) {
            const uint4 v = reinterpret_cast<const uint4*>(p)[k];
            w[4 * k] = v.x; w[4 * k + 1] = v.y; w[4 * k + 2] = v.z; w[4 * k + 3] = v.w;
        }
    } else if constexpr (R % 8 == 0) {
#pragma unroll
        for (int k = 0; k < R / 8; ++k) {
            const uint2 v = reinterpret_cast<const uint2*>(p)[k];
            w[2 * k] = v.x; w[2 * k + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int k = 0; k < R / 4; ++k) w[k] = reinterpret_cast<const uint32_t*>(p)[k];
    }
}

__device__ __forceinline__ uint32_t word_of(const uint4& v, int i) {
    return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// The query (or query pair) of one work item.
struct ItemQuery {
    const uint8_t* qa;
    const uint8_t* qb;
    uint32_t la, lb;  // lengths (lb = 0 when there is no second query)
    uint32_t ia, ib;  // output rows of the two queries (ib = UINT32_MAX: none)
};

// ---------------------------------------------------------------------------
// Modes: what the two halves of a lane hold, how the profile is laid out, and
// where results go.
// ---------------------------------------------------------------------------

// One query, two database sequences per group (16-bit halves = sequences).
// Profile: int8 prof[r][k] = fsbt(q[p*T*R + k], r); thread t reads R contiguous
// bytes at r * T*R + t * R; a permute merges the two sequences' scores.
struct ModePairDb {
    using Lane = LaneS16x2;
    static constexpr bool kPairStream = true;  // both sequences of the tile pair
    static constexpr bool kRing = false;
    template <int T, int R>
    struct Prof {
        static constexpr int TR = T * R;
        static constexpr size_t kBytes = (size_t)kProfileRows * TR;
        static __device__ __forceinline__ void stage(uint8_t* prof, const ItemQuery& iq,
                                                     const WavefrontArgs& a, uint32_t p) {
            for (uint32_t idx = threadIdx.x; idx < kProfileRows * (TR / 4); idx += kThreads) {
                const uint32_t r = idx / (TR / 4);
                const uint32_t k4 = (idx % (TR / 4)) * 4;
                uint32_t word = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int v = profile_score(iq.qa, iq.la, a.matrix, a.alphabet, p * TR + k4 + b, r);
                    word |= ((uint32_t)(uint8_t)(int8_t)v) << (8 * b);
                }
                reinterpret_cast<uint32_t*>(prof)[idx] = word;
            }
        }
    };
    template <int T, int R>
    struct Cols {
        uint32_t wa[R / 4], wb[R / 4];
        __device__ __forceinline__ void load(const uint8_t* prof, uint32_t code, int t) {
            const uint8_t* my = prof + t * R;
            load_rows<R>(my + (code & 0xffu) * (T * R), wa);
            load_rows<R>(my + (code >> 8) * (T * R), wb);
        }
        __device__ __forceinline__ uint32_t row(int l) const {
            const uint32_t b = (uint32_t)(l & 3);
            return prmt(wa[l / 4], wb[l / 4], b | ((8u | b) << 4) | ((4u + b) << 8) | ((12u + b) << 12));
        }
    };
};

// 32-bit profile words in 4-row chunks laid out [r][R/4][T][4 words]: thread t
// reads chunk c of code r at ((r * R/4 + c) * T + t) * 16, so the 8 lanes of a
// quarter-warp hit 8 different 16-byte bank groups whatever codes they use.
template <int T, int R>
__device__ __forceinline__ void load_chunks(const uint8_t* prof, uint32_t code, int t,
                                            uint4 (&w)[R / 4]) {
    const uint4* p = reinterpret_cast<const uint4*>(prof) + (size_t)code * (R / 4) * T + t;
#pragma unroll
    for (int c = 0; c < R / 4; ++c) w[c] = p[c * T];
}

// Two queries, one database sequence per group (16-bit halves = queries).
// Profile words hold both queries' scores for one (row, code).
struct ModeQueryPair {
    using Lane = LaneS16x2;
    static constexpr bool kPairStream = false;
    static constexpr bool kRing = false;
    template <int T, int R>
    struct Prof {
        static constexpr int TR = T * R;
        static constexpr size_t kBytes = (size_t)kProfileRows * TR * 4;
        static __device__ __forceinline__ void stage(uint8_t* prof, const ItemQuery& iq,
                                                     const WavefrontArgs& a, uint32_t p) {
            for (uint32_t idx = threadIdx.x; idx < kProfileRows * (TR / 4); idx += kThreads) {
                const uint32_t r = idx / (TR / 4), rem = idx % (TR / 4);
                const uint32_t c = rem / T, t = rem % T;
                const uint32_t row0 = p * TR + t * R + c * 4;
                uint32_t v[4];
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const uint32_t lo = (uint16_t)(int16_t)profile_score(iq.qa, iq.la, a.matrix,
                                                                         a.alphabet, row0 + b, r);
                    const uint32_t hi = (uint16_t)(int16_t)profile_score(iq.qb, iq.lb, a.matrix,
                                                                         a.alphabet, row0 + b, r);
                    v[b] = lo | (hi << 16);
                }
                reinterpret_cast<uint4*>(prof)[idx] = make_uint4(v[0], v[1], v[2], v[3]);
            }
        }
    };
    template <int T, int R>
    struct Cols {
        uint4 w[R / 4];
        __device__ __forceinline__ void load(const uint8_t* prof, uint32_t code, int t) {
            load_chunks<T, R>(prof, code, t, w);
        }
        __device__ __forceinline__ uint32_t row(int l) const { return word_of(w[l / 4], l % 4); }
    };
};

// One query, one database sequence per group, int32 lanes.
struct ModeInt32 {
    using Lane = LaneS32;
    static constexpr bool kPairStream = false;
    static constexpr bool kRing = false;
    template <int T, int R>
    struct Prof {
        static constexpr int TR = T * R;
        static constexpr size_t kBytes = (size_t)kProfileRows * TR * 4;
        static __device__ __forceinline__ void stage(uint8_t* prof, const ItemQuery& iq,
                                                     const WavefrontArgs& a, uint32_t p) {
            for (uint32_t idx = threadIdx.x; idx < kProfileRows * (TR / 4); idx += kThreads) {
                const uint32_t r = idx / (TR / 4), rem = idx % (TR / 4);
                const uint32_t c = rem / T, t = rem % T;
                const uint32_t row0 = p * TR + t * R + c * 4;
                int v[4];
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    v[b] = profile_score(iq.qa, iq.la, a.matrix, a.alphabet, row0 + b, r);
                reinterpret_cast<int4*>(prof)[idx] = make_int4(v[0], v[1], v[2], v[3]);
            }
        }
    };
    template <int T, int R>
    struct Cols {
        uint4 w[R / 4];
        __device__ __forceinline__ void load(const uint8_t* prof, uint32_t code, int t) {
            load_chunks<T, R>(prof, code, t, w);
        }
        __device__ __forceinline__ int32_t row(int l) const { return (int32_t)word_of(w[l / 4], l % 4); }
    };
};

// Aligns every unit of one chunk (kWarps warps x 32/T groups) against the
// item's query (pair). All warps of the block process the same chunk, pass by
// pass.
//
// Boundary rows: entry kSkew T + j of a slot half holds (H, E) of column j
// (entries below kSkew T take the fill steps' writes and are never read). Thread 0 reads them
// in aligned 4-column blocks; blocks at or past the unit's length L (a
// multiple of 4) read as zero, which is safe for the pad columns there: every
// value they produce stays at or below the largest real H.
template <class Mode, int T, int R>
__device__ __forceinline__ void process_chunk(const WavefrontArgs& a, const BinArgs& bin,
                                              uint64_t base, uint64_t n_units,
                                              const ItemQuery& iq, uint8_t* prof, int32_t thr16) {
    using Lane = typename Mode::Lane;
    using V = typename Lane::V;
    using Prof = typename Mode::template Prof<T, R>;
    constexpr int G = 32 / T;           // groups per warp
    constexpr int TR = T * R;           // query rows per pass
    constexpr bool kPair = Mode::kPairStream;
    constexpr uint32_t kPadPair = kPadCode | (kPadCode << 8);
    constexpr uint32_t kPadWord = kPadPair | (kPadPair << 16);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / T, t = lane % T;
    const uint32_t qmax = iq.la > iq.lb ? iq.la : iq.lb;
    const uint32_t P = (qmax + TR - 1) / TR;
    const uint64_t slot = ((uint64_t)blockIdx.x * kWarps + warp) * G + g;
    const uint64_t half = bin.bstride / 2;
    uint2* const bnd0 = bin.boundary + slot * bin.bstride;

    const V vbeta = Lane::splat(-a.beta);
    const V valpha = Lane::splat(-a.alpha);
    const V vzero = Lane::splat(0);

    // ---- locate this group's unit ----
    const uint64_t u = base + (uint64_t)warp * G + g;
    const bool have = u < n_units;
    uint64_t sp = 0;  // sorted position (the first sequence of the pair for kPair)
    uint32_t L = 0;
    const uint8_t* stream = a.tile_data;
    uint32_t half_sel = 0;  // one-sequence modes: which sequence of the pair stream
    if (have) {
        sp = kPair ? 2 * (bin.first_unit + u) : bin.first_unit + u;
        const uint64_t tile = sp / kTileSeqs;
        const uint32_t pslot = (uint32_t)((sp >> 1) & (kTilePairs - 1));
        L = a.tile_len[tile];
        stream = a.tile_data + a.tile_off[tile] + pslot * 8;
        half_sel = (uint32_t)(sp & 1);
    }
    uint32_t Lw = L;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) Lw = max(Lw, __shfl_xor_sync(0xffffffffu, Lw, o));
    const uint32_t steps = (Lw + kSkew * (T - 1) + 3) & ~3u;
    const uint32_t blocks_real = L / 4;  // 4-column blocks of this unit (L is a multiple of 4)

    V best = vzero;
    for (uint32_t p = 0; p < P; ++p) {
        __syncthreads();  // every warp is done with the previous pass's profile
        Prof::stage(prof, iq, a, p);
        __syncthreads();

        V Hl[R], Fr[R];
#pragma unroll
        for (int r = 0; r < R; ++r) { Hl[r] = vzero; Fr[r] = vzero; }
        // Thread t works on column s - 2t at step s, so the thread above produced
        // this thread's inputs (its bottom row H, E and the column's codes) two
        // steps earlier: the inputs of step s + 1 are shuffled at the start of
        // step s, and the two steps' dependence chains can overlap.
        V hb_out = vzero, eb_out = vzero, hdiag0 = vzero;  // this thread's last outputs
        uint32_t code_out = kPair ? kPadPair : kPadCode;
        V h_cur = vzero, e_cur = vzero;                     // inputs of the current step
        uint32_t code_cur = code_out;
        const uint2* const bnd_in = bnd0 + (p & 1) * half + kSkew * T;
        uint2* const bnd_out = bnd0 + ((p + 1) & 1) * half + kSkew * T;
        const bool read_bnd = p > 0;
        auto code_of = [&](const uint2& w, int k) -> uint32_t {
            const uint32_t v = (k < 2) ? w.x : w.y;
            return kPair ? ((v >> (16 * (k & 1))) & 0xffffu) : ((v >> (16 * (k & 1) + 8 * half_sel)) & 0xffu);
        };

        // thread 0's codes (4 columns per 8-byte word) and boundary values, one block ahead
        uint2 wq = make_uint2(kPadWord, kPadWord);
        uint4 bq0 = make_uint4(0, 0, 0, 0), bq1 = make_uint4(0, 0, 0, 0);
        if (t == 0 && blocks_real > 0) {
            wq = *reinterpret_cast<const uint2*>(stream);
            if (read_bnd && sw_ok(kSkew * T + 4 <= half, a.dbg, 6)) {
                bq0 = reinterpret_cast<const uint4*>(bnd_in)[0];
                bq1 = reinterpret_cast<const uint4*>(bnd_in)[1];
            }
        }
        if (t == 0) {  // column 0
            code_cur = code_of(wq, 0);
            h_cur = (V)bq0.x;
            e_cur = (V)bq0.y;
        }

        for (uint32_t s0 = 0; s0 < steps; s0 += 4) {
            uint2 wn = make_uint2(kPadWord, kPadWord);
            uint4 bn0 = make_uint4(0, 0, 0, 0), bn1 = make_uint4(0, 0, 0, 0);
            const uint32_t nb = (s0 >> 2) + 1;
            if (t == 0 && nb < blocks_real && sw_ok((uint64_t)nb * 4 < L, a.dbg, 8)) {
                wn = *reinterpret_cast<const uint2*>(stream + (size_t)nb * 32);
                if (read_bnd && sw_ok(kSkew * T + s0 + 8 <= half, a.dbg, 6)) {
                    bn0 = reinterpret_cast<const uint4*>(bnd_in + s0 + 4)[0];
                    bn1 = reinterpret_cast<const uint4*>(bnd_in + s0 + 4)[1];
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                // inputs of step s + 1: the thread above's outputs of step s - 1
                V h_nxt = (V)__shfl_up_sync(0xffffffffu, (uint32_t)hb_out, 1, T);
                V e_nxt = (V)__shfl_up_sync(0xffffffffu, (uint32_t)eb_out, 1, T);
                uint32_t code_nxt = __shfl_up_sync(0xffffffffu, code_out, 1, T);
                if (t == 0) {  // column s + 1
                    if (k < 3) {
                        code_nxt = code_of(wq, k + 1);
                        const uint4& bq = (k + 1 < 2) ? bq0 : bq1;
                        h_nxt = (V)(((k + 1) & 1) ? bq.z : bq.x);
                        e_nxt = (V)(((k + 1) & 1) ? bq.w : bq.y);
                    } else {
                        code_nxt = code_of(wn, 0);
                        h_nxt = (V)bn0.x;
                        e_nxt = (V)bn0.y;
                    }
                }
                typename Mode::template Cols<T, R> cs;
                if (!sw_ok((code_cur & 0xffu) < kProfileRows && (code_cur >> 8) < kProfileRows, a.dbg, 1))
                    code_cur = kPair ? kPadPair : kPadCode;
                cs.load(prof, code_cur, t);
                V diag = hdiag0;
                V E = e_cur;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const V sc = (V)cs.row(r);
                    const V x = Lane::vadd(diag, sc);              // H[i-1][j-1] + fsbt
                    const V H = Lane::max3_relu(x, E, Fr[r]);      // H[i][j]
                    diag = Hl[r];                                  // H[i][j-1]: diagonal of row i+1
                    Hl[r] = H;
                    const V hb = Lane::vadd(H, vbeta);             // H[i][j] - beta
                    E = Lane::addmax(E, valpha, hb);               // E[i+1][j]
                    Fr[r] = Lane::addmax(Fr[r], valpha, hb);       // F[i][j+1]
                    best = Lane::vmax(best, x);                    // max H = max(0, max x)
                }
                hb_out = Hl[R - 1];
                eb_out = E;
                code_out = code_cur;
                hdiag0 = h_cur;
                h_cur = h_nxt;
                e_cur = e_nxt;
                code_cur = code_nxt;
                if (t == T - 1 &&  // column s - 2 (T-1), at entry 2T + that >= 2
                    sw_ok((uint64_t)(kSkew * T + s0 + k - kSkew * (T - 1)) < half, a.dbg, 7))
                    bnd_out[(int)(s0 + k) - kSkew * (T - 1)] =
                        make_uint2((uint32_t)hb_out, (uint32_t)eb_out);
            }
            wq = wn;
            bq0 = bn0;
            bq1 = bn1;
        }
    }

    // ---- group maximum and results ----
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1)
        best = Lane::vmax(best, (V)__shfl_xor_sync(0xffffffffu, (uint32_t)best, o, T));
    if (!have || t != 0) return;
    if constexpr (std::is_same<Lane, LaneS32>::value) {
        const uint32_t id = a.sorted_ids[sp];
        if (id != 0xffffffffu) a.scores[(uint64_t)iq.ia * a.score_stride + id] = (int32_t)best;
    } else {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int32_t v = (int16_t)(h ? ((uint32_t)best >> 16) : ((uint32_t)best & 0xffffu));
        const uint64_t seq = kPair ? sp + h : sp;
        const uint32_t qi = kPair ? iq.ia : (h ? iq.ib : iq.ia);
        const uint32_t id = a.sorted_ids[seq];
        if (id == 0xffffffffu || qi == 0xffffffffu) continue;
        if (v >= thr16) {  // rescored in int32; -1 marks it until then
            const uint32_t k = atomicAdd(a.flag_count, 1u);
            if (k < a.flag_cap) a.flag_list[k] = make_uint2(qi, (uint32_t)seq);
            a.scores[(uint64_t)qi * a.score_stride + id] = -1;
        } else {
            a.scores[(uint64_t)qi * a.score_stride + id] = v;
        }
    }
    }
}

// ---------------------------------------------------------------------------
// Score-profile ring: one query, two database sequences per group
// ---------------------------------------------------------------------------
//
// The packed score of query row i against column j of a pair is
// (fsbt(q_i, dA_j), fsbt(q_i, dB_j)). ModePairDb merges the two int8 query
// profile entries with a byte permute for every cell pair. Here each warp
// keeps instead a ring of packed words (fsbt(c, dA_j), fsbt(c, dB_j)) for
// every query code c and a window of recent columns j of its pairs: the
// score profile of Section III.B.2, built on the fly per column rather than
// for whole sequences. A thread reads the packed score of each of its rows
// with one shared-memory load; the permutes drop from one per (row, column)
// to one per (code, column).
//
// Thread t of a group works on column s - S t at step s. With S = 2 its
// inputs (the thread above's bottom row) are ready two steps ahead and are
// shuffled one step early, so consecutive steps' dependence chains overlap.
//
// Ring layout, in 32-bit words per warp: code row c (0..A, row A all zeros
// for rows past the query) at c * RingGeom::kRowWords. S = 1: column j of
// group g in slot j mod W at word slot * G + g (G = 32 / T groups per warp).
// S = 2: the even and odd columns in two planes, column j in plane j & 1 at
// slot (j >> 1) mod W. A slot below D is also stored at W + slot, so a
// thread addresses the columns of one 8-step block from one base without a
// wrap. The T threads of a group read T columns of one parity (S = 2) or T
// consecutive columns (S = 1) at once; their slots differ mod 8 (T = 8: with
// g in the low bits the warp hits 32 distinct banks) or mod 32 (T = 32), and
// kRowWords is a multiple of 32, so the code of a row does not move its bank.
template <int S>
struct ModeRing {
    static constexpr bool kRing = true;
    static constexpr int kSkew = S;
};

constexpr int kRingBlock = 8;      // steps per block = columns built per block
constexpr int kStageWords = 18;    // per group: 8 boundary entries of (H, E), padded against conflicts
// fsbt by database code d: word [k][d] packs fsbt(4k .. 4k+3, d) as int8 (k < 8, d < 33), so
// threads loading word k for different codes d hit different banks
constexpr uint32_t kMtBytes = 8 * kProfileRows * 4;
constexpr uint32_t kRingOffset = kMtBytes + kWarps * 4 * kStageWords * 4;
// The two-column skew needs a larger window; it keeps two blocks per SM up to this alphabet.
constexpr uint32_t kRing2MaxAlphabet = 20;

template <int S>
__host__ __device__ constexpr int ring_row_words() { return S == 1 ? 96 : 160; }

template <int T, int S>
struct RingGeom {
    static constexpr int G = 32 / T;
    static constexpr uint32_t W = S == 1 ? 2 * T : (T == 8 ? 16 : 64);  // slots in the window
    static constexpr uint32_t D = kRingBlock / S;                        // slots stored twice
    static constexpr uint32_t kSlot = G * 4;                             // bytes between slots
    static constexpr uint32_t kPlane = (W + D) * G * 4;                  // bytes between planes
    static constexpr uint32_t kCodeBytes = ring_row_words<S>() * 4;
    static_assert(S * (W + D) * G <= (uint32_t)ring_row_words<S>() && ring_row_words<S>() % 32 == 0,
                  "ring row");
    // live window: the 8 columns built at a block start must not overwrite a column
    // still read in that block (the oldest is S (T - 1) columns behind)
    static_assert(S == 1 ? W >= T + kRingBlock - 1 : W >= T + 3, "ring window");
    static_assert((W % (T == 8 ? 8 : 32)) == 0, "bank pattern");
};

__host__ __device__ constexpr size_t ring_smem_bytes(uint32_t alphabet, int S) {
    return kRingOffset + (size_t)kWarps * (alphabet + 1) * (S == 1 ? ring_row_words<1>() : ring_row_words<2>()) * 4;
}

// Once per block: the matrix by database code, and every warp's all-zero row.
template <int S>
__device__ __forceinline__ void ring_setup(const WavefrontArgs& a, uint8_t* smem) {
    const uint32_t A = a.alphabet;
    for (uint32_t idx = threadIdx.x; idx < 8 * kProfileRows * 4; idx += kThreads) {
        const uint32_t k = idx / (kProfileRows * 4), d = (idx / 4) % kProfileRows;
        const uint32_t c = 4 * k + idx % 4;
        smem[idx] = (uint8_t)((c < A && d < A) ? a.matrix[c * A + d] : 0);
    }
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr uint32_t kRow = ring_row_words<S>();
    uint32_t* zero_row = reinterpret_cast<uint32_t*>(smem + kRingOffset) +
                         (size_t)warp * (A + 1) * kRow + A * kRow;
    for (uint32_t w = lane; w < kRow; w += 32) zero_row[w] = 0;
    __syncthreads();
}

// Passes p_first .. p_first + n_pass - 1 of the pair unit of one group against one
// query, R rows per thread, the first from query row row0 (as process_chunk for
// ModePairDb, with the score-profile ring instead of the int8 query profile); best
// collects the maximum.
template <int T, int R, int S>
__device__ __forceinline__ void ring_passes(const WavefrontArgs& a, const BinArgs& bin,
                                            uint64_t base, uint64_t n_units, const ItemQuery& iq,
                                            uint8_t* smem, uint32_t p_first, uint32_t n_pass,
                                            uint32_t row0_first, uint32_t& best) {
    using Lane = LaneS16x2;
    using V = uint32_t;
    using Geo = RingGeom<T, S>;
    constexpr int G = Geo::G;
    constexpr int TR = T * R;
    constexpr uint32_t W = Geo::W;
    constexpr uint32_t kSlot = Geo::kSlot;
    constexpr uint32_t kCodeBytes = Geo::kCodeBytes;
    constexpr uint32_t kSplit = T / kRingBlock;       // threads sharing one built column
    constexpr uint32_t kPadPair = kPadCode | (kPadCode << 8);
    constexpr uint32_t kAdvance = kRingBlock / S;     // slots per block

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / T, t = lane % T;
    const uint32_t A = a.alphabet;
    const uint64_t slot = ((uint64_t)blockIdx.x * kWarps + warp) * G + g;
    const uint64_t half = bin.bstride / 2;
    uint2* const bnd0 = bin.boundary + slot * bin.bstride;

    const uint32_t smem_s = (uint32_t)__cvta_generic_to_shared(smem);
    const uint32_t ring_s = smem_s + kRingOffset + (uint32_t)warp * (A + 1) * kCodeBytes + g * 4;
    const uint32_t stage_s = smem_s + kMtBytes + (uint32_t)(warp * 4 + g) * kStageWords * 4;
    // this warp's ring and this group's stage (checked in the bounds-checked build)
    const uint32_t ring_lo = ring_s - g * 4, ring_hi = ring_lo + (A + 1) * kCodeBytes;
    auto in_ring = [&](uint32_t addr) { return addr >= ring_lo && addr + 4 <= ring_hi; };
    const uint32_t* const mt = reinterpret_cast<const uint32_t*>(smem);

    const V vbeta = Lane::splat(-a.beta);
    const V valpha = Lane::splat(-a.alpha);
    const V vzero = 0;

    // ---- locate this group's unit (a pair of sequences) ----
    const uint64_t u = base + (uint64_t)warp * G + g;
    const bool have = u < n_units;
    uint64_t sp = 0;
    uint32_t L = 0;
    const uint8_t* stream = a.tile_data;
    if (have) {
        sp = 2 * (bin.first_unit + u);
        const uint64_t tile = sp / kTileSeqs;
        const uint32_t pslot = (uint32_t)((sp >> 1) & (kTilePairs - 1));
        L = a.tile_len[tile];
        stream = a.tile_data + a.tile_off[tile] + pslot * 8;
    }
    uint32_t Lw = L;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) Lw = max(Lw, __shfl_xor_sync(0xffffffffu, Lw, o));
    const uint32_t steps = (Lw + S * (T - 1) + kRingBlock - 1) & ~(uint32_t)(kRingBlock - 1);

    // what this thread builds: column (block start + bcol), codes bq, bq + kSplit, ...
    const uint32_t bcol = (uint32_t)t % kRingBlock;
    const uint32_t bq = (uint32_t)t / kRingBlock;
    const uint32_t bsel = bq | ((8u | bq) << 4) | ((4u + bq) << 8) | ((12u + bq) << 12);
    // ring byte offset of column j (code 0; the duplicate is + W * kSlot)
    auto col_off = [&](uint32_t j, bool& dup) -> uint32_t {
        if constexpr (S == 1) {
            const uint32_t js = j & (W - 1);
            dup = js < Geo::D;
            return js * kSlot;
        } else {
            const uint32_t js = (j >> 1) & (W - 1);
            dup = js < Geo::D;
            return (j & 1) * Geo::kPlane + js * kSlot;
        }
    };

    for (uint32_t p = p_first; p < p_first + n_pass; ++p) {
        constexpr int RR = R;
        const uint32_t row0 = row0_first + (p - p_first) * TR;
        // ring addresses of this thread's rows at the first block (slot of column -S t)
        uint32_t cur[RR];
        const uint32_t blk0 = (W - (uint32_t)t) & (W - 1);
#pragma unroll
        for (int r = 0; r < RR; ++r) {
            const uint32_t row = row0 + (uint32_t)t * RR + r;
            uint32_t c = A;
            if (row < iq.la) {
                const uint32_t qc = iq.qa[row];
                c = qc < A ? qc : A;
            }
            cur[r] = ring_s + c * kCodeBytes + blk0 * kSlot;
        }
        V Hl[RR], Fr[RR];
#pragma unroll
        for (int r = 0; r < RR; ++r) { Hl[r] = vzero; Fr[r] = vzero; }
        V hb_out = vzero, eb_out = vzero, hdiag0 = vzero;  // this thread's last outputs
        V h_cur = vzero, e_cur = vzero;                     // inputs of the current step (S = 2)
        const uint2* const bnd_in = bnd0 + (p & 1) * half + S * T;
        uint2* const bnd_out = bnd0 + ((p + 1) & 1) * half + S * T;
        const bool read_bnd = p > 0;
        // boundary entry of column bcol of the next block (threads below kRingBlock stage it)
        uint2 bnext = make_uint2(0, 0);
        if (t < kRingBlock && read_bnd && bcol < L && sw_ok(S * T + bcol < half, a.dbg, 6))
            bnext = bnd_in[bcol];
        if constexpr (S == 2) {
            if (t == 0) {  // column 0
                h_cur = bnext.x;
                e_cur = bnext.y;
            }
        }
        // the codes of the column this thread builds, loaded one block ahead
        auto codes_at = [&](uint32_t j) -> uint32_t {
            if (j < L && sw_ok((j >> 2) * 32 + ((sp >> 1) & (kTilePairs - 1)) * 8 + (j & 3) * 2 + 2 <=
                                   (uint64_t)L * 8, a.dbg, 8))
                return *reinterpret_cast<const uint16_t*>(stream + (size_t)(j >> 2) * 32 + (j & 3) * 2);
            return kPadPair;
        };
        uint32_t pc_next = codes_at(bcol);

        for (uint32_t s0 = 0; s0 < steps; s0 += kRingBlock) {
            __syncwarp();  // the slots rewritten below are no longer read
            {
                const uint32_t j = s0 + bcol;
                uint32_t pc = pc_next;
                pc_next = codes_at(j + kRingBlock);
                if (!sw_ok((pc & 0xffu) < kProfileRows && (pc >> 8) < kProfileRows, a.dbg, 5)) pc = kPadPair;
                const uint32_t* const ma = mt + (pc & 0xffu);
                const uint32_t* const mb = mt + (pc >> 8);
                bool dup;
                const uint32_t at0 = ring_s + col_off(j, dup);
                // the column's word for every code at ring address `at`; the 8 columns of a
                // block share dup, so the second copy is a branch the whole warp takes or skips
                auto build = [&](uint32_t at) {
                    if constexpr (kSplit == 1) {
                        if (A == 20) {  // the protein alphabet: five whole words, no per-code tests
#pragma unroll
                            for (int k = 0; k < 5; ++k) {
                                const uint32_t wa = ma[k * kProfileRows], wb = mb[k * kProfileRows];
#pragma unroll
                                for (int b = 0; b < 4; ++b) {
                                    const uint32_t c = 4u * k + b;
                                    const uint32_t v = prmt(wa, wb, b | ((8u | b) << 4) |
                                                                      ((4u + b) << 8) | ((12u + b) << 12));
                                    if (sw_ok(in_ring(at + c * kCodeBytes), a.dbg, 3))
                                        sts_u32(at + c * kCodeBytes, v);
                                }
                            }
                            return;
                        }
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            if (4u * k >= A) break;
                            const bool whole = 4u * k + 4 <= A;  // uniform: no per-code test
                            const uint32_t wa = ma[k * kProfileRows], wb = mb[k * kProfileRows];
#pragma unroll
                            for (int b = 0; b < 4; ++b) {
                                const uint32_t c = 4u * k + b;
                                if (whole || c < A) {
                                    const uint32_t v = prmt(wa, wb, b | ((8u | b) << 4) |
                                                                      ((4u + b) << 8) | ((12u + b) << 12));
                                    if (sw_ok(in_ring(at + c * kCodeBytes), a.dbg, 3))
                                        sts_u32(at + c * kCodeBytes, v);
                                }
                            }
                        }
                    } else {
                        static_assert(kSplit == 4, "codes per word");
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            if (4u * k >= A) break;
                            const uint32_t c = 4u * k + bq;
                            const uint32_t wa = ma[k * kProfileRows], wb = mb[k * kProfileRows];
                            if (c < A) {
                                const uint32_t v = prmt(wa, wb, bsel);
                                if (sw_ok(in_ring(at + c * kCodeBytes), a.dbg, 3))
                                    sts_u32(at + c * kCodeBytes, v);
                            }
                        }
                    }
                };
                build(at0);
                if (dup) build(at0 + W * kSlot);
            }
            if (s0 == 0 && t + 1 < T) {
                // columns -S(T-1) .. -1 score 0 at the start of a pass: slots W-T+1 .. W-1
                // (both planes for S = 2)
                const uint32_t at = ring_s + (W - T + 1 + (uint32_t)t) * kSlot;
                for (uint32_t c = 0; c < A; ++c) {
                    if (sw_ok(in_ring(at + c * kCodeBytes), a.dbg, 3)) sts_u32(at + c * kCodeBytes, 0u);
                    if constexpr (S == 2)
                        if (sw_ok(in_ring(at + c * kCodeBytes + Geo::kPlane), a.dbg, 3))
                            sts_u32(at + c * kCodeBytes + Geo::kPlane, 0u);
                }
            }
            if (t < kRingBlock) sts_u64(stage_s + (uint32_t)t * 8, bnext);
            __syncwarp();  // this block's columns and boundary entries are visible
            if (t < kRingBlock) {
                const uint32_t jn = s0 + kRingBlock + (uint32_t)t;
                bnext = (read_bnd && jn < L && sw_ok(S * T + jn < half, a.dbg, 6)) ? bnd_in[jn]
                                                                                 : make_uint2(0, 0);
            }
            uint2* const bo = bnd_out + (int)s0 - S * (T - 1);
#pragma unroll
            for (int k = 0; k < kRingBlock; ++k) {
                V h_in, e_in;
                if constexpr (S == 1) {
                    h_in = shfl_up_or_lds<T>(hb_out, stage_s + k * 8);
                    e_in = shfl_up_or_lds<T>(eb_out, stage_s + k * 8 + 4);
                } else {
                    // inputs of step s + 1: the thread above's outputs of step s - 1
                    V h_nxt, e_nxt;
                    if (k + 1 < kRingBlock) {
                        h_nxt = shfl_up_or_lds<T>(hb_out, stage_s + (k + 1) * 8);
                        e_nxt = shfl_up_or_lds<T>(eb_out, stage_s + (k + 1) * 8 + 4);
                    } else {  // column s + 1 opens the next block: thread 0 holds it
                        h_nxt = (V)__shfl_up_sync(0xffffffffu, (uint32_t)hb_out, 1, T);
                        e_nxt = (V)__shfl_up_sync(0xffffffffu, (uint32_t)eb_out, 1, T);
                        if (t == 0) {
                            h_nxt = bnext.x;
                            e_nxt = bnext.y;
                        }
                    }
                    h_in = h_cur;
                    e_in = e_cur;
                    h_cur = h_nxt;
                    e_cur = e_nxt;
                }
                const uint32_t koff = S == 1 ? k * kSlot : (k & 1) * Geo::kPlane + (k >> 1) * kSlot;
                // x = H[i-1][j-1] + fsbt of every row first (last row first, in place: the
                // row below has used the old H by then), then the H, E, F chain down the rows
#pragma unroll
                for (int r = RR - 1; r >= 0; --r) {
                    V sc = 0;
                    if (sw_ok(in_ring(cur[r] + koff), a.dbg, 2)) sc = lds_u32(cur[r] + koff);
                    Hl[r] = Lane::vadd(r > 0 ? Hl[r - 1] : hdiag0, sc);
                }
                V E = e_in;
#pragma unroll
                for (int r = 0; r < RR; ++r) {
                    const V x = Hl[r];
                    const V H = Lane::max3_relu(x, E, Fr[r]);      // H[i][j]
                    Hl[r] = H;
                    const V hb = Lane::vadd(H, vbeta);             // H[i][j] - beta
                    E = Lane::addmax(E, valpha, hb);               // E[i+1][j]
                    Fr[r] = Lane::addmax(Fr[r], valpha, hb);       // F[i][j+1]
                    best = Lane::vmax(best, x);                    // max H = max(0, max x)
                }
                hb_out = Hl[RR - 1];
                eb_out = E;
                hdiag0 = h_in;
                // two 32-bit stores: measured faster than one 64-bit store with 32 lanes per
                // group, and no slower with 8
                if (t == T - 1 && sw_ok((int64_t)(S * T) + (int64_t)(s0 + k) - S * (T - 1) >= 0 &&
                                            (uint64_t)(S * T + s0 + k - S * (T - 1)) < half,
                                        a.dbg, 7)) {
                    bo[k].x = (uint32_t)hb_out;
                    bo[k].y = (uint32_t)eb_out;
                }
            }
            // next block: slots advance by kAdvance, wrapping at W
            const uint32_t blk = ((s0 / S) - (uint32_t)t) & (W - 1);
            const uint32_t delta = (blk + kAdvance < W ? kAdvance : kAdvance - W) * kSlot;
#pragma unroll
            for (int r = 0; r < RR; ++r) cur[r] += delta;
        }
    }
}

// The last pass of fewer rows, compiled apart from the caller so that the whole-pass
// loop keeps its own register allocation and schedule.
template <int T, int R, int S>
__device__ __noinline__ void ring_last_pass(const WavefrontArgs& a, const BinArgs& bin,
                                            uint64_t base, uint64_t n_units, const ItemQuery& iq,
                                            uint8_t* smem, uint32_t p, uint32_t row0,
                                            uint32_t& best) {
    ring_passes<T, R, S>(a, bin, base, n_units, iq, smem, p, 1, row0, best);
}

// The pair unit of one group against one query in passes of T R rows; with 8 threads
// of 24 rows, the rows left after the whole passes take one pass of 8, 16 or 24 rows per
// thread (ring_last_rows: fewer padded rows).
template <int T, int R, int S>
__device__ __forceinline__ void process_chunk_ring(const WavefrontArgs& a, const BinArgs& bin,
                                                   uint64_t base, uint64_t n_units,
                                                   const ItemQuery& iq, uint8_t* smem,
                                                   int32_t thr16) {
    using Lane = LaneS16x2;
    using V = uint32_t;
    constexpr uint32_t TR = T * R;
    constexpr bool kShortLast = T == kShortT && R == kRingLastR;
    const uint32_t P = kShortLast ? iq.la / TR : (iq.la + TR - 1) / TR;
    const int last = kShortLast ? ring_last_rows(iq.la - P * TR) : 0;
    V best = 0;
    ring_passes<T, R, S>(a, bin, base, n_units, iq, smem, 0, P + (last == R), 0, best);
    if constexpr (kShortLast) {
        if (last == 8)
            ring_last_pass<T, 8, S>(a, bin, base, n_units, iq, smem, P, P * TR, best);
        else if (last == 16)
            ring_last_pass<T, 16, S>(a, bin, base, n_units, iq, smem, P, P * TR, best);
    }
    const int lane = threadIdx.x & 31;
    const int t = lane % T;
    const uint64_t u = base + (uint64_t)(threadIdx.x >> 5) * (32 / T) + lane / T;
    const bool have = u < n_units;
    const uint64_t sp = 2 * (bin.first_unit + u);

    // ---- group maximum and results ----
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1)
        best = Lane::vmax(best, (V)__shfl_xor_sync(0xffffffffu, (uint32_t)best, o, T));
    if (!have || t != 0) return;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int32_t v = (int16_t)(h ? ((uint32_t)best >> 16) : ((uint32_t)best & 0xffffu));
        const uint64_t seq = sp + h;
        const uint32_t id = a.sorted_ids[seq];
        if (id == 0xffffffffu) continue;
        if (v >= thr16) {  // rescored in int32; -1 marks it until then
            const uint32_t k = atomicAdd(a.flag_count, 1u);
            if (k < a.flag_cap) a.flag_list[k] = make_uint2(iq.ia, (uint32_t)seq);
            a.scores[(uint64_t)iq.ia * a.score_stride + id] = -1;
        } else {
            a.scores[(uint64_t)iq.ia * a.score_stride + id] = v;
        }
    }
}

template <class Mode, int T, int R>
__device__ __forceinline__ void run_chunk(const WavefrontArgs& a, const BinArgs& bin, uint64_t base,
                                          uint64_t n_units, const ItemQuery& iq, uint8_t* smem,
                                          int32_t thr16) {
    if constexpr (Mode::kRing)
        process_chunk_ring<T, R, Mode::kSkew>(a, bin, base, n_units, iq, smem, thr16);
    else
        process_chunk<Mode, T, R>(a, bin, base, n_units, iq, smem, thr16);
}

__device__ __forceinline__ ItemQuery item_query(const WavefrontArgs& a, uint32_t k) {
    ItemQuery iq;
    if (a.pairs) {
        const QueryPair qp = a.pairs[k];
        iq.qa = a.query + qp.off_a;
        iq.qb = a.query + qp.off_b;
        iq.la = qp.len_a;
        iq.lb = qp.len_b;
        iq.ia = qp.q_a;
        iq.ib = qp.q_b;
    } else {
        iq.qa = iq.qb = a.query;
        iq.la = a.qlen;
        iq.lb = 0;
        iq.ia = 0;
        iq.ib = 0xffffffffu;
    }
    return iq;
}

// Persistent search kernel. Work items are (chunk, query item) pairs, chunk
// major: chunks of bin 0 (the long sequences, a warp per unit: TL lanes x RL
// rows) first, then chunks of bin 1 (TS lanes per unit x RS rows), so the
// longest work starts first and one database chunk is reused across the
// query items from L2.
template <class Mode, int TS, int RS, int TL, int RL>
__global__ void __launch_bounds__(kThreads, 2) search_kernel(const WavefrontArgs a) {
    extern __shared__ __align__(16) uint8_t prof[];
    __shared__ uint32_t s_item;
    constexpr uint32_t UNITS_L = kWarps * (32 / TL);
    constexpr uint32_t UNITS_S = kWarps * (32 / TS);

    // 16-bit lanes are exact while every H stays at or below 32767 - max(0, max fsbt)
    __shared__ int s_smax;
    if (threadIdx.x == 0) s_smax = 0;
    __syncthreads();
    int mx = 0;
    for (uint32_t i = threadIdx.x; i < a.alphabet * a.alphabet; i += kThreads)
        mx = max(mx, (int)a.matrix[i]);
    atomicMax(&s_smax, mx);
    __syncthreads();
    const int32_t thr16 = 32767 - s_smax;
    if constexpr (Mode::kRing) ring_setup<Mode::kSkew>(a, prof);

    if (a.item_prefix) {
        // serving wave: each pair scans its own range of bin-1 chunks
        const uint32_t items = a.item_prefix[a.n_pairs];
        for (;;) {
            if (threadIdx.x == 0) s_item = atomicAdd(a.work_counter, 1u);
            __syncthreads();
            const uint32_t it = s_item;
            if (it >= items) break;
            uint32_t lo = 0, hi = a.n_pairs;
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (a.item_prefix[mid] <= it) lo = mid; else hi = mid;
            }
            const uint64_t chunk = (uint64_t)a.pair_chunk0[lo] + (it - a.item_prefix[lo]);
            run_chunk<Mode, TS, RS>(a, a.bin[1], chunk * UNITS_S, a.bin[1].n_units,
                                        item_query(a, lo), prof, thr16);
            __syncthreads();
        }
        return;
    }
    const uint32_t n_items_q = a.pairs ? a.n_pairs : 1u;
    const uint64_t chunks_long = (a.bin[0].n_units + UNITS_L - 1) / UNITS_L;
    const uint64_t chunks_short = (a.bin[1].n_units + UNITS_S - 1) / UNITS_S;
    const uint64_t items_long = chunks_long * n_items_q;
    const uint64_t items = items_long + chunks_short * n_items_q;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.work_counter, 1u);
        __syncthreads();
        const uint64_t it = s_item;
        if (it >= items) break;
        if (it < items_long) {
            const ItemQuery iq = item_query(a, (uint32_t)(it % n_items_q));
            run_chunk<Mode, TL, RL>(a, a.bin[0], (it / n_items_q) * UNITS_L, a.bin[0].n_units,
                                        iq, prof, thr16);
        } else {
            const uint64_t is = it - items_long;
            const ItemQuery iq = item_query(a, (uint32_t)(is % n_items_q));
            run_chunk<Mode, TS, RS>(a, a.bin[1], (is / n_items_q) * UNITS_S, a.bin[1].n_units,
                                        iq, prof, thr16);
        }
        __syncthreads();  // s_item is rewritten by the next iteration
    }
}

using KernelFn = void (*)(WavefrontArgs);

struct Entry {
    int mode;  // KernelChoice::Mode
    int R;
    KernelFn fn;
    size_t smem;
    int skew;  // ring entries: threads' column skew (1 or 2); 0 otherwise
};

template <class Mode, int R>
constexpr size_t smem_of() {
    return Mode::template Prof<kShortT, R>::kBytes > Mode::template Prof<kLongT, kLongR>::kBytes
               ? Mode::template Prof<kShortT, R>::kBytes
               : Mode::template Prof<kLongT, kLongR>::kBytes;
}

#define SWGB_ENTRY(M, MODE, R) \
    {M, R, search_kernel<MODE, kShortT, R, kLongT, kLongR>, smem_of<MODE, R>(), 0}
const Entry kEntries[] = {
    SWGB_ENTRY(0, ModePairDb, 8),     SWGB_ENTRY(0, ModePairDb, 12),
    SWGB_ENTRY(0, ModePairDb, 16),    SWGB_ENTRY(0, ModePairDb, 20),
    SWGB_ENTRY(0, ModePairDb, 24),    SWGB_ENTRY(1, ModeQueryPair, 8),
    SWGB_ENTRY(1, ModeQueryPair, 12), SWGB_ENTRY(1, ModeQueryPair, 16),
    SWGB_ENTRY(1, ModeQueryPair, 20), SWGB_ENTRY(1, ModeQueryPair, 24),
    SWGB_ENTRY(2, ModeInt32, 16),
#define SWGB_RING(S, R) {3, R, search_kernel<ModeRing<S>, kShortT, R, kLongT, kLongR>, 0, S}
    SWGB_RING(1, 8), SWGB_RING(1, 12), SWGB_RING(1, 16), SWGB_RING(1, 20), SWGB_RING(1, 24),
    SWGB_RING(2, 8), SWGB_RING(2, 12), SWGB_RING(2, 16), SWGB_RING(2, 20), SWGB_RING(2, 24),
#undef SWGB_RING
};
#undef SWGB_ENTRY

// Dynamic shared memory of one launch (the ring grows with the alphabet).
size_t entry_smem(const Entry& e, uint32_t alphabet) {
    return e.mode == 3 ? ring_smem_bytes(alphabet, e.skew) : e.smem;
}
// The largest alphabet an entry serves.
uint32_t entry_max_alphabet(const Entry& e) { return e.skew == 2 ? kRing2MaxAlphabet : 32; }

// The entry for a choice and alphabet: rings take the two-column skew when its
// window fits (alphabet <= kRing2MaxAlphabet), else the one-column skew.
const Entry* find_entry(const KernelChoice& kc, uint32_t alphabet) {
    const int skew = kc.mode != KernelChoice::kPairRing ? 0 : (alphabet <= kRing2MaxAlphabet ? 2 : 1);
    for (const Entry& e : kEntries)
        if (e.R == kc.R && e.mode == (int)kc.mode && e.skew == skew) return &e;
    return nullptr;
}

}  // namespace

bool wavefront_supported(const KernelChoice& kc) { return find_entry(kc, 32) != nullptr; }
int wavefront_block_threads() { return kThreads; }
int wavefront_short_units_per_chunk() { return kWarps * (32 / kShortT); }

int wavefront_occupancy(const KernelChoice& kc, int* threads_per_block) {
    if (threads_per_block) *threads_per_block = kThreads;
    // every entry the choice may launch, at the largest alphabet it serves
    int blocks = 0;
    for (uint32_t A : {kRing2MaxAlphabet, 32u}) {
        const Entry* e = find_entry(kc, A);
        if (!e) return 0;
        const size_t smem = entry_smem(*e, entry_max_alphabet(*e));
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(e->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess)
            return 0;
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, e->fn, kThreads, smem) != cudaSuccess)
            return 0;
        blocks = std::max(blocks, b);
    }
    return blocks;
}

cudaError_t launch_wavefront(const KernelChoice& kc, const WavefrontArgs& a, int grid,
                             cudaStream_t stream) {
    if (a.alphabet < 1 || a.alphabet > 32) return cudaErrorInvalidValue;
    const Entry* e = find_entry(kc, a.alphabet);
    if (!e) return cudaErrorInvalidValue;
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    const size_t smem = entry_smem(*e, a.alphabet);
    if (smem > 48 * 1024) {
        cudaError_t err = cudaFuncSetAttribute(e->fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)entry_smem(*e, entry_max_alphabet(*e)));
        if (err != cudaSuccess) return err;
    }
    e->fn<<<grid, kThreads, smem, stream>>>(a);
    return cudaGetLastError();
}

// Entries past a unit's length that a boundary row half must hold.
uint32_t boundary_slack() { return 2 * kLongT + 8; }

// ---------------------------------------------------------------------------
// Database layout kernels
// ---------------------------------------------------------------------------

namespace {

// One thread per (tile, 4-column block, pair): writes the pair's 8-byte word.
__global__ void build_tiles_kernel(const uint8_t* __restrict__ residues,
                                   const uint64_t* __restrict__ offsets,
                                   const uint32_t* __restrict__ sorted_ids, uint64_t n_sorted,
                                   const uint64_t* __restrict__ tile_off,
                                   const uint32_t* __restrict__ tile_len, uint64_t n_tiles,
                                   uint8_t* __restrict__ tile_data) {
    // grid-stride over tiles; each block handles one tile at a time
    for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const uint32_t L = tile_len[tile];
        const uint32_t words = (L / 4) * kTilePairs;
        uint8_t* out = tile_data + tile_off[tile];
        for (uint32_t w = threadIdx.x; w < words; w += blockDim.x) {
            const uint32_t c4 = w / kTilePairs, g = w % kTilePairs;
            uint8_t bytes[8];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint64_t sp = tile * kTileSeqs + 2 * g + h;
                uint64_t o = 0, n = 0;
                if (sp < n_sorted) {
                    const uint32_t id = sorted_ids[sp];
                    if (id != 0xffffffffu) { o = offsets[id]; n = offsets[id + 1] - o; }
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const uint64_t col = (uint64_t)c4 * 4 + c;
                    bytes[2 * c + h] = col < n ? residues[o + col] : (uint8_t)kPadCode;
                }
            }
            uint2 v;
            v.x = bytes[0] | (bytes[1] << 8) | (bytes[2] << 16) | ((uint32_t)bytes[3] << 24);
            v.y = bytes[4] | (bytes[5] << 8) | (bytes[6] << 16) | ((uint32_t)bytes[7] << 24);
            reinterpret_cast<uint2*>(out)[w] = v;
        }
    }
}

__global__ void max_code_kernel(const uint8_t* __restrict__ p, uint64_t n, uint32_t* out) {
    uint32_t m = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        m = max(m, (uint32_t)p[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

}  // namespace

cudaError_t launch_build_tiles(const uint8_t* residues, const uint64_t* offsets,
                               const uint32_t* sorted_ids, uint64_t n_sorted,
                               const uint64_t* tile_off, const uint32_t* tile_len,
                               uint64_t n_tiles, uint8_t* tile_data, cudaStream_t stream) {
    if (n_tiles == 0) return cudaSuccess;
    const int grid = (int)(n_tiles < 1048560ull ? n_tiles : 1048560ull);
    build_tiles_kernel<<<grid, 128, 0, stream>>>(residues, offsets, sorted_ids, n_sorted, tile_off,
                                                 tile_len, n_tiles, tile_data);
    return cudaGetLastError();
}

cudaError_t launch_max_code(const uint8_t* residues, uint64_t n, uint32_t* out,
                            cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    const uint64_t want = (n + 255) / 256;
    const int grid = (int)(want < 4096 ? want : 4096);
    max_code_kernel<<<grid, 256, 0, stream>>>(residues, n, out);
    return cudaGetLastError();
}

}  // namespace swgb
