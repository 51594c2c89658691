// Wavefront kernels for recurrence (1) of Section II.A (Smith-Waterman with
// affine gaps): the hot loop of a database search.
//
// Design (GB300-first; the paper's Xeon Phi kernels are prior art):
//  - A group of T consecutive lanes cooperates on one database "unit": a pair
//    of length-sorted sequences held in the two 16-bit halves of every
//    register (packed s16x2 arithmetic, the inter-sequence model of Section
//    III.B with two lanes per register), or one sequence in int32.
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
//  - The integer ALU pipe is the bottleneck (every max, fused add-max and
//    byte permute runs there; plain 16x2 adds run on the FMA pipe), so the
//    cell update is written to keep ALU work at 4.5 instructions per cell
//    pair: unpack the two int8 scores (prmt), H = max3(diag + s, E, F, 0)
//    with the add on the FMA pipe, E and F as fused add-max, and the running
//    maximum fused two rows at a time.
//  - Exactness: 16-bit lanes wrap, so a lane whose maximum reaches
//    thr16 = 32767 - max(0, max fsbt) is flagged and rescored by the int32
//    kernel. Below that threshold no intermediate can leave the 16-bit range
//    (H <= thr16 bounds H + fsbt; E, F >= -beta because H >= 0; E - alpha and
//    F - alpha >= -(alpha + beta) >= -32768 is required of the 16-bit path),
//    and the first cell that exceeds it is computed exactly, so the running
//    maximum of a lane that ever exceeded thr16 ends at or above it.
#include <cuda_runtime.h>
#include <cstdint>
#include <type_traits>

#include "sw_internal.h"

namespace swgb {

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}
// Packed pair of 16-bit lanes: low half = first sequence, high half = second.
struct LaneS16x2 {
    using V = uint32_t;
    static __device__ __forceinline__ V splat(int x) {
        const uint32_t u = (uint16_t)(int16_t)x;
        return u | (u << 16);
    }
    static __device__ __forceinline__ V vmax(V a, V b) {
        V d;
        asm("max.s16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
        return d;
    }
    static __device__ __forceinline__ V vadd(V a, V b) {
        V d;
        asm("add.s16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
        return d;
    }
    // max(a + b, c, 0) per lane
    static __device__ __forceinline__ V addmax_relu(V a, V b, V c) {
        return __viaddmax_s16x2_relu(a, b, c);
    }
    // max(a + b, c) per lane
    static __device__ __forceinline__ V addmax(V a, V b, V c) { return __viaddmax_s16x2(a, b, c); }
    // max(a, b, c, 0) per lane
    static __device__ __forceinline__ V max3_relu(V a, V b, V c) { return __vimax3_s16x2_relu(a, b, c); }
};

// One sequence in a 32-bit lane.
struct LaneS32 {
    using V = int32_t;
    static __device__ __forceinline__ V splat(int x) { return x; }
    static __device__ __forceinline__ V vmax(V a, V b) { return max(a, b); }
    static __device__ __forceinline__ V vadd(V a, V b) { return a + b; }
    static __device__ __forceinline__ V addmax_relu(V a, V b, V c) {
        return __viaddmax_s32_relu(a, b, c);
    }
    static __device__ __forceinline__ V addmax(V a, V b, V c) { return __viaddmax_s32(a, b, c); }
    static __device__ __forceinline__ V max3_relu(V a, V b, V c) { return __vimax3_s32_relu(a, b, c); }
};

// fsbt(q[row], r) for one query row, 0 outside the query or the alphabet.
__device__ __forceinline__ int profile_score(const WavefrontArgs& a, uint32_t row, uint32_t r) {
    if (row >= a.qlen || r >= a.alphabet) return 0;
    const uint32_t qc = a.query[row];
    return qc < a.alphabet ? (int)a.matrix[qc * a.alphabet + r] : 0;
}

// Query profile of one pass in shared memory: prof[r][k] = fsbt(q[p*T*R + k], r)
// as int8, r = 0..32 (32 = pad code, all zero). Thread t reads its R rows for
// one code as R contiguous bytes at r * T*R + t * R.
template <int T, int R, bool PAIR>
struct Profile {
    static constexpr int TR = T * R;
    static constexpr size_t kBytes = (size_t)kProfileRows * TR;

    static __device__ __forceinline__ void stage(uint8_t* prof, const WavefrontArgs& a, uint32_t p) {
        for (uint32_t idx = threadIdx.x; idx < kProfileRows * (TR / 4); idx += kThreads) {
            const uint32_t r = idx / (TR / 4);
            const uint32_t k4 = (idx % (TR / 4)) * 4;
            uint32_t word = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int v = profile_score(a, p * TR + k4 + b, r);
                word |= ((uint32_t)(uint8_t)(int8_t)v) << (8 * b);
            }
            reinterpret_cast<uint32_t*>(prof)[idx] = word;
        }
    }
};

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

// Substitution scores of one column for a thread's R rows, as lane words.
template <int T, int R, bool PAIR>
struct ColumnScores {
    using Lane = typename std::conditional<PAIR, LaneS16x2, LaneS32>::type;
    using V = typename Lane::V;
    uint32_t wa[R / 4], wb[PAIR ? R / 4 : 1];

    __device__ __forceinline__ void load(const uint8_t* prof, uint32_t ca, uint32_t cb, int t) {
        const uint8_t* my_rows = prof + t * R;
        load_rows<R>(my_rows + ca * (T * R), wa);
        if (PAIR) load_rows<R>(my_rows + cb * (T * R), reinterpret_cast<uint32_t(&)[R / 4]>(wb));
    }
    // row l: both sequences' int8 scores sign-extended into the two 16-bit
    // lanes (pair), or the int32 score
    __device__ __forceinline__ V row(int l) const {
        const uint32_t b = (uint32_t)(l & 3);
        if (PAIR) {
            return prmt(wa[l / 4], wb[l / 4], b | ((8u | b) << 4) | ((4u + b) << 8) | ((12u + b) << 12));
        } else {
            const uint32_t x = 8u | b;
            return (V)prmt(wa[l / 4], 0u, b | (x << 4) | (x << 8) | (x << 12));
        }
    }
};

// Aligns every unit of one chunk (kWarps warps x 32/T groups) against the
// whole query. All warps of the block process the same chunk, pass by pass.
//
// Boundary rows: entry T + j of a slot half holds (H, E) of column j (entries
// below T take the fill steps' writes and are never read). Thread 0 reads them
// in aligned 4-column blocks; blocks at or past the unit's length L (a
// multiple of 4) read as zero, which is safe for the pad columns there: every
// value they produce stays at or below the largest real H.
template <int T, int R, bool PAIR>
__device__ __forceinline__ void process_chunk(const WavefrontArgs& a, const BinArgs& bin,
                                              uint64_t base, uint64_t n_units, uint8_t* prof,
                                              int32_t thr16) {
    using Lane = typename std::conditional<PAIR, LaneS16x2, LaneS32>::type;
    using V = typename Lane::V;
    constexpr int G = 32 / T;           // groups per warp
    constexpr int TR = T * R;           // query rows per pass
    constexpr uint32_t kPadPair = kPadCode | (kPadCode << 8);
    constexpr uint32_t kPadWord = kPadPair | (kPadPair << 16);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / T, t = lane % T;
    const uint32_t P = (a.qlen + TR - 1) / TR;
    const uint64_t slot = ((uint64_t)blockIdx.x * kWarps + warp) * G + g;
    const uint64_t half = bin.bstride / 2;
    uint2* const bnd0 = bin.boundary + slot * bin.bstride;

    const V vbeta = Lane::splat(-a.beta);
    const V valpha = Lane::splat(-a.alpha);
    const V vzero = Lane::splat(0);

    // ---- locate this group's unit ----
    const uint64_t u = base + (uint64_t)warp * G + g;
    const bool have = u < n_units;
    uint64_t sp = 0;  // sorted position (first sequence of the pair)
    uint32_t L = 0;
    const uint8_t* stream = a.tile_data;
    uint32_t half_sel = 0;  // int32 lanes: which sequence of the pair stream
    if (have) {
        if (PAIR) sp = 2 * (bin.first_unit + u);
        else sp = bin.unit_list ? (uint64_t)bin.unit_list[u] : bin.first_unit + u;
        const uint64_t tile = sp / kTileSeqs;
        const uint32_t pslot = (uint32_t)((sp >> 1) & (kTilePairs - 1));
        L = a.tile_len[tile];
        stream = a.tile_data + a.tile_off[tile] + pslot * 8;
        half_sel = (uint32_t)(sp & 1);
    }
    uint32_t Lw = L;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) Lw = max(Lw, __shfl_xor_sync(0xffffffffu, Lw, o));
    const uint32_t steps = (Lw + T - 1 + 3) & ~3u;
    const uint32_t blocks_real = L / 4;  // 4-column blocks of this unit (L is a multiple of 4)

    V best = vzero;
    for (uint32_t p = 0; p < P; ++p) {
        __syncthreads();  // every warp is done with the previous pass's profile
        Profile<T, R, PAIR>::stage(prof, a, p);
        __syncthreads();

        V Hl[R], Fr[R];
#pragma unroll
        for (int r = 0; r < R; ++r) { Hl[r] = vzero; Fr[r] = vzero; }
        V hb_out = vzero, eb_out = vzero, hdiag0 = vzero;
        uint32_t code_out = PAIR ? kPadPair : kPadCode;
        const uint2* const bnd_in = bnd0 + (p & 1) * half + T;
        uint2* const bnd_out = bnd0 + ((p + 1) & 1) * half + T;
        const bool read_bnd = p > 0;

        // thread 0's codes (4 columns per 8-byte word) and boundary values, one block ahead
        uint2 wq = make_uint2(kPadWord, kPadWord);
        uint4 bq0 = make_uint4(0, 0, 0, 0), bq1 = make_uint4(0, 0, 0, 0);
        if (t == 0 && blocks_real > 0) {
            wq = *reinterpret_cast<const uint2*>(stream);
            if (read_bnd) {
                bq0 = reinterpret_cast<const uint4*>(bnd_in)[0];
                bq1 = reinterpret_cast<const uint4*>(bnd_in)[1];
            }
        }

        for (uint32_t s0 = 0; s0 < steps; s0 += 4) {
            uint2 wn = make_uint2(kPadWord, kPadWord);
            uint4 bn0 = make_uint4(0, 0, 0, 0), bn1 = make_uint4(0, 0, 0, 0);
            const uint32_t nb = (s0 >> 2) + 1;
            if (t == 0 && nb < blocks_real) {
                wn = *reinterpret_cast<const uint2*>(stream + (size_t)nb * 32);
                if (read_bnd) {
                    bn0 = reinterpret_cast<const uint4*>(bnd_in + s0 + 4)[0];
                    bn1 = reinterpret_cast<const uint4*>(bnd_in + s0 + 4)[1];
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                // inputs from the thread above: its previous step's bottom row and codes
                V h_in = (V)__shfl_up_sync(0xffffffffu, (uint32_t)hb_out, 1, T);
                V e_in = (V)__shfl_up_sync(0xffffffffu, (uint32_t)eb_out, 1, T);
                uint32_t code = __shfl_up_sync(0xffffffffu, code_out, 1, T);
                if (t == 0) {
                    const uint32_t w = (k < 2) ? wq.x : wq.y;
                    code = PAIR ? ((w >> (16 * (k & 1))) & 0xffffu)
                                : ((w >> (16 * (k & 1) + 8 * half_sel)) & 0xffu);
                    const uint4& bq = (k < 2) ? bq0 : bq1;
                    h_in = (V)((k & 1) ? bq.z : bq.x);
                    e_in = (V)((k & 1) ? bq.w : bq.y);
                }
                code_out = code;
                ColumnScores<T, R, PAIR> cs;
                cs.load(prof, PAIR ? (code & 0xffu) : code, code >> 8, t);
                V diag = hdiag0;
                V E = e_in;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const V sc = cs.row(r);
                    const V H = Lane::max3_relu(Lane::vadd(diag, sc), E, Fr[r]);  // H[i][j]
                    diag = Hl[r];                                  // H[i][j-1]: diagonal of row i+1
                    Hl[r] = H;
                    const V hb = Lane::vadd(H, vbeta);             // H[i][j] - beta
                    E = Lane::addmax(E, valpha, hb);               // E[i+1][j]
                    Fr[r] = Lane::addmax(Fr[r], valpha, hb);       // F[i][j+1]
                    best = Lane::vmax(best, H);
                }
                hb_out = Hl[R - 1];
                eb_out = E;
                hdiag0 = h_in;
                if (t == T - 1)  // column s - (T-1), at entry T + that >= 1
                    bnd_out[(int)(s0 + k) - (T - 1)] = make_uint2((uint32_t)hb_out, (uint32_t)eb_out);
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
    if (have && t == 0) {
        if (PAIR) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int32_t v = (int16_t)(h ? ((uint32_t)best >> 16) : ((uint32_t)best & 0xffffu));
                const uint32_t id = a.sorted_ids[sp + h];
                if (id == 0xffffffffu) continue;
                if (v >= thr16) {
                    const uint32_t k = atomicAdd(a.flag_count, 1u);
                    a.flag_list[k] = (uint32_t)(sp + h);
                } else {
                    a.scores[id] = v;
                }
            }
        } else {
            const uint32_t id = a.sorted_ids[sp];
            if (id != 0xffffffffu) a.scores[id] = (int32_t)best;
        }
    }
}

// Persistent search kernel over the two bins of a database. Chunks of bin 0
// (the long sequences, a warp per pair: TL lanes x RL rows) are handed out
// first, then chunks of bin 1 (TS lanes per pair x RS rows), so the longest
// work starts first. Bin 0 may instead be an explicit list of sorted
// positions (int32 rescoring).
template <int TS, int RS, int TL, int RL, bool PAIR>
__global__ void __launch_bounds__(kThreads) search_kernel(const WavefrontArgs a) {
    extern __shared__ __align__(16) uint8_t prof[];
    __shared__ uint32_t s_chunk, s_units;
    constexpr uint32_t UNITS_L = kWarps * (32 / TL);
    constexpr uint32_t UNITS_S = kWarps * (32 / TS);

    // 16-bit lanes are exact while every H stays at or below 32767 - max(0, max fsbt)
    __shared__ int s_smax;
    if (threadIdx.x == 0) s_smax = 0;
    __syncthreads();
    if (PAIR) {
        int mx = 0;
        for (uint32_t i = threadIdx.x; i < a.alphabet * a.alphabet; i += kThreads)
            mx = max(mx, (int)a.matrix[i]);
        atomicMax(&s_smax, mx);
        __syncthreads();
    }
    const int32_t thr16 = 32767 - s_smax;

    for (;;) {
        if (threadIdx.x == 0) {
            s_chunk = atomicAdd(a.work_counter, 1u);
            s_units = a.bin[0].unit_list ? *a.bin[0].unit_count : 0u;
        }
        __syncthreads();
        const uint64_t n_long = a.bin[0].unit_list ? (uint64_t)s_units : a.bin[0].n_units;
        const uint64_t chunks_long = (n_long + UNITS_L - 1) / UNITS_L;
        const uint64_t c = s_chunk;
        if (c < chunks_long) {
            process_chunk<TL, RL, PAIR>(a, a.bin[0], c * UNITS_L, n_long, prof, thr16);
        } else {
            const uint64_t base = (c - chunks_long) * UNITS_S;
            if (base >= a.bin[1].n_units) break;
            process_chunk<TS, RS, PAIR>(a, a.bin[1], base, a.bin[1].n_units, prof, thr16);
        }
        __syncthreads();  // s_chunk is rewritten by the next iteration
    }
}

using KernelFn = void (*)(WavefrontArgs);

struct Entry {
    int R;
    bool pair;
    KernelFn fn;
    size_t smem;
};

#define SWGB_ENTRY(R, P)                                                           \
    {R, P, search_kernel<kShortT, R, kLongT, kLongR, P>,                           \
     (Profile<kShortT, R, P>::kBytes > Profile<kLongT, kLongR, P>::kBytes         \
          ? Profile<kShortT, R, P>::kBytes                                         \
          : Profile<kLongT, kLongR, P>::kBytes)}
const Entry kEntries[] = {
    SWGB_ENTRY(8, true),  SWGB_ENTRY(12, true), SWGB_ENTRY(16, true),
    SWGB_ENTRY(20, true), SWGB_ENTRY(24, true), SWGB_ENTRY(16, false),
};
#undef SWGB_ENTRY

const Entry* find_entry(const KernelChoice& kc) {
    for (const Entry& e : kEntries)
        if (e.R == kc.R && e.pair == kc.pair) return &e;
    return nullptr;
}

}  // namespace

bool wavefront_supported(const KernelChoice& kc) { return find_entry(kc) != nullptr; }
int wavefront_block_threads() { return kThreads; }

int wavefront_occupancy(const KernelChoice& kc, int* threads_per_block) {
    const Entry* e = find_entry(kc);
    if (threads_per_block) *threads_per_block = kThreads;
    if (!e) return 0;
    if (e->smem > 48 * 1024 &&
        cudaFuncSetAttribute(e->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e->smem) !=
            cudaSuccess)
        return 0;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, e->fn, kThreads, e->smem) !=
        cudaSuccess)
        return 0;
    return blocks;
}

cudaError_t launch_wavefront(const KernelChoice& kc, const WavefrontArgs& a, int grid,
                             cudaStream_t stream) {
    const Entry* e = find_entry(kc);
    if (!e) return cudaErrorInvalidValue;
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    if (e->smem > 48 * 1024) {
        cudaError_t err =
            cudaFuncSetAttribute(e->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e->smem);
        if (err != cudaSuccess) return err;
    }
    e->fn<<<grid, kThreads, e->smem, stream>>>(a);
    return cudaGetLastError();
}

// Longest pad needed past a unit's last column by the boundary rows.
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
