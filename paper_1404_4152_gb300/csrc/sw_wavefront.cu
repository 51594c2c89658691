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
//    pattern cited in Section I) and hands the bottom row's H and E to the
//    next thread with a warp shuffle.
//  - A pass covers T*R query rows. Between passes the bottom row is kept in a
//    global scratch row (the paper's tiled computation, Section IV.C; two
//    halves per group, read one / write the other) and the block stages the
//    next T*R rows of the query profile (Section III.B.2) in shared memory.
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
    // substitution scores of row b of a 4-row int8 word, for both sequences,
    // sign-extended into the two 16-bit lanes
    static __device__ __forceinline__ V score(uint32_t wa, uint32_t wb, int b) {
        const uint32_t sel = (uint32_t)b | ((8u | b) << 4) | ((4u + b) << 8) | ((12u + b) << 12);
        return prmt(wa, wb, sel);
    }
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
    static __device__ __forceinline__ V score(uint32_t wa, uint32_t, int b) {
        const uint32_t s = 8u | b;
        return (V)prmt(wa, 0u, (uint32_t)b | (s << 4) | (s << 8) | (s << 12));
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

template <class Lane>
__device__ __forceinline__ typename Lane::V shfl_up_v(typename Lane::V v, int T) {
    return (typename Lane::V)__shfl_up_sync(0xffffffffu, (uint32_t)v, 1, T);
}

// Aligns every unit of one chunk (kWarps warps x 32/T groups) against the
// whole query. All warps of the block process the same chunk, pass by pass.
template <int T, int R, bool PAIR>
__device__ __forceinline__ void process_chunk(const WavefrontArgs& a, const BinArgs& bin,
                                              uint64_t base, uint64_t n_units, uint8_t* prof,
                                              int32_t thr16) {
    using Lane = typename std::conditional<PAIR, LaneS16x2, LaneS32>::type;
    using V = typename Lane::V;
    constexpr int G = 32 / T;           // groups per warp
    constexpr int TR = T * R;           // query rows per pass

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane / T, t = lane % T;
    const uint32_t P = (a.qlen + TR - 1) / TR;
    const uint64_t slot = ((uint64_t)blockIdx.x * kWarps + warp) * G + g;
    // two halves per slot: pass p reads half p&1 and writes the other one
    const uint64_t half = bin.bstride / 2;
    uint2* const bnd0 = bin.boundary + slot * bin.bstride;

    const V vbeta = Lane::splat(-a.beta);
    const V valpha = Lane::splat(-a.alpha);
    const V vzero = Lane::splat(0);
    const uint32_t A = a.alphabet;

    // ---- locate this group's unit ----
    const uint64_t u = base + (uint64_t)warp * G + g;
    const bool have = u < n_units;
    uint64_t sp = 0;  // sorted position (first sequence of the pair)
    uint32_t L = 0;
    const uint8_t* stream = a.tile_data;
    if (have) {
        if (PAIR) sp = 2 * (bin.first_unit + u);
        else sp = bin.unit_list ? (uint64_t)bin.unit_list[u] : bin.first_unit + u;
        const uint64_t tile = sp / kTileSeqs;
        const uint32_t pslot = (uint32_t)((sp >> 1) & (kTilePairs - 1));
        L = a.tile_len[tile];
        stream = a.tile_data + a.tile_off[tile] + pslot * 8 + (PAIR ? 0 : (sp & 1));
    }
    uint32_t Lw = L;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) Lw = max(Lw, __shfl_xor_sync(0xffffffffu, Lw, o));
    const uint32_t steps = (Lw + T - 1 + 3) & ~3u;

    V best = vzero;
    for (uint32_t p = 0; p < P; ++p) {
        __syncthreads();  // every warp is done with the previous pass's profile
        // stage query rows [p*TR, p*TR + TR) of the profile: prof[r][k] = fsbt(q[row], r)
        for (uint32_t idx = threadIdx.x; idx < kProfileRows * (TR / 4); idx += kThreads) {
            const uint32_t r = idx / (TR / 4);
            const uint32_t k4 = (idx % (TR / 4)) * 4;
            uint32_t word = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const uint32_t row = p * TR + k4 + b;
                int v = 0;
                if (row < a.qlen && r < A) {
                    const uint32_t qc = a.query[row];
                    if (qc < A) v = a.matrix[qc * A + r];
                }
                word |= ((uint32_t)(uint8_t)(int8_t)v) << (8 * b);
            }
            reinterpret_cast<uint32_t*>(prof)[idx] = word;
        }
        __syncthreads();

        V Hl[R], Fr[R];
#pragma unroll
        for (int r = 0; r < R; ++r) { Hl[r] = vzero; Fr[r] = vzero; }
        V hb_out = vzero, eb_out = vzero, hdiag0 = vzero;
        const bool read_bnd = (t == 0) && (p > 0);
        const bool write_bnd = (t == T - 1) && (p + 1 < P);
        const uint2* const bnd_in = bnd0 + (p & 1) * half;
        uint2* const bnd_out = bnd0 + ((p + 1) & 1) * half;
        const uint8_t* const my_rows = prof + t * R;

        // codes and boundary values for the current block of 4 steps
        uint32_t cq[4];
        uint2 bq[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int j = k - t;
            uint32_t c = PAIR ? (kPadCode | (kPadCode << 8)) : kPadCode;
            if (j >= 0 && j < (int)L) {
                const uint8_t* q = stream + (uint32_t)(j >> 2) * 32 + (j & 3) * 2;
                c = PAIR ? (uint32_t)*reinterpret_cast<const uint16_t*>(q) : (uint32_t)*q;
            }
            cq[k] = c;
            bq[k] = make_uint2(0u, 0u);
            if (read_bnd && j < (int)L) bq[k] = bnd_in[j];
        }

        for (uint32_t s0 = 0; s0 < steps; s0 += 4) {
            // prefetch the next block's codes and boundary row
            uint32_t cn[4];
            uint2 bn[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int j = (int)s0 + 4 + k - t;
                uint32_t c = PAIR ? (kPadCode | (kPadCode << 8)) : kPadCode;
                if (j >= 0 && j < (int)L) {
                    const uint8_t* q = stream + (uint32_t)(j >> 2) * 32 + (j & 3) * 2;
                    c = PAIR ? (uint32_t)*reinterpret_cast<const uint16_t*>(q) : (uint32_t)*q;
                }
                cn[k] = c;
                bn[k] = make_uint2(0u, 0u);
                if (read_bnd && j < (int)L) bn[k] = bnd_in[j];
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int j = (int)s0 + k - t;
                // top row input: H[i0-1][j] and E[i0][j] from the thread above
                V h_in = shfl_up_v<Lane>(hb_out, T);
                V e_in = shfl_up_v<Lane>(eb_out, T);
                if (t == 0) {
                    h_in = (V)bq[k].x;
                    e_in = (V)bq[k].y;
                }
                // substitution scores of this column for my R rows
                const uint32_t ca = PAIR ? (cq[k] & 0xffu) : cq[k];
                uint32_t wa[R / 4], wb[R / 4];
                load_rows<R>(my_rows + ca * TR, wa);
                if (PAIR) {
                    load_rows<R>(my_rows + (cq[k] >> 8) * TR, wb);
                } else {
#pragma unroll
                    for (int w = 0; w < R / 4; ++w) wb[w] = 0;
                }
                V diag = hdiag0;
                V E = e_in;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const V sc = Lane::score(wa[r / 4], wb[r / 4], r & 3);
                    const V ef = Lane::vmax(E, Fr[r]);
                    const V H = Lane::addmax_relu(diag, sc, ef);  // H[i][j]
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
                if (write_bnd && j >= 0 && j < (int)L)
                    bnd_out[j] = make_uint2((uint32_t)hb_out, (uint32_t)eb_out);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) { cq[k] = cn[k]; bq[k] = bn[k]; }
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
    extern __shared__ __align__(16) uint8_t prof[];  // [kProfileRows][rows per pass] int8
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
};

#define SWGB_ENTRY(R, P) {R, P, search_kernel<kShortT, R, kLongT, kLongR, P>}
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

size_t smem_bytes(const KernelChoice& kc) {
    const int rows = kShortT * kc.R > kLongT * kLongR ? kShortT * kc.R : kLongT * kLongR;
    return (size_t)kProfileRows * rows;
}

}  // namespace

bool wavefront_supported(const KernelChoice& kc) { return find_entry(kc) != nullptr; }
int wavefront_block_threads() { return kThreads; }

int wavefront_occupancy(const KernelChoice& kc, int* threads_per_block) {
    const Entry* e = find_entry(kc);
    if (threads_per_block) *threads_per_block = kThreads;
    if (!e) return 0;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, e->fn, kThreads, smem_bytes(kc)) !=
        cudaSuccess)
        return 0;
    return blocks;
}

cudaError_t launch_wavefront(const KernelChoice& kc, const WavefrontArgs& a, int grid,
                             cudaStream_t stream) {
    const Entry* e = find_entry(kc);
    if (!e) return cudaErrorInvalidValue;
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    e->fn<<<grid, kThreads, smem_bytes(kc), stream>>>(a);
    return cudaGetLastError();
}

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
