// Top-k of a search: stage (iv) of the workflow in Section III sorts all
// alignment scores in descending order; the library returns the best top_k,
// equal scores ordered by ascending database index, which makes the list
// unique.
//
// One launch per call (grid = blocks x rows). Every block takes a contiguous
// slice of its row and selects the slice's top-k exactly; the last block of the
// row to finish (a per-row counter) merges the blocks' candidates and sorts the
// result. The global top-k is contained in the union of the slices' top-k, and
// both selections break ties by index the same way, so the merge is exact.
//
// Selection of the top kk of M elements (non-negative int32 scores, in index
// order), by the whole block:
//   1. three histogram/select rounds over 11 + 11 + 10 bits of the score find the
//      kk-th largest score thr and how many scores must be taken at thr;
//   2. one ordered pass keeps every score > thr and the first of the scores ==
//      thr in index order, writing them in index order (a block-wide scan), so a
//      row's candidates, block after block, are again in index order.
// The merge runs the same selection over the candidates (held in shared
// memory), then sorts the kk survivors by (score desc, index asc) (bitonic).
#include <cuda_runtime.h>
#include <cstdint>

#include "sw_internal.h"

namespace swgb {

namespace {

constexpr int kBins = 2048;
constexpr int kThreads = 512;
constexpr int kWarpsT = kThreads / 32;
constexpr uint32_t kMaxK = 1024;
constexpr uint32_t kMinSlice = 1024;  // elements per block at least

__device__ __forceinline__ int digit_shift(int round) { return round == 0 ? 21 : (round == 1 ? 10 : 0); }
__device__ __forceinline__ uint32_t digit_mask(int round) { return round == 2 ? 0x3ffu : 0x7ffu; }
// bits above the digit of this round
__device__ __forceinline__ uint32_t high_mask(int round) {
    return round == 0 ? 0u : (round == 1 ? 0xffe00000u : 0xfffffc00u);
}

struct SelState {
    uint32_t prefix;  // the bits of thr found so far
    uint32_t krem;    // elements still to take at or below the prefix
};

struct TopkShared {
    uint32_t hist[kBins];
    uint32_t warp_cnt[2][kWarpsT];
    SelState st;
    uint32_t last;
};

// Block-wide: the top kk of M elements (score(i), index(i)), i in index order, by
// (score desc, index asc), written in index order to out_s / out_i. Every thread
// calls it; it begins and ends with a barrier.
template <class Score, class Index>
__device__ void block_select(Score score, Index index, uint32_t M, uint32_t kk, TopkShared& sh,
                             int32_t* out_s, uint32_t* out_i) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __syncthreads();
    if (tid == 0) sh.st = SelState{0u, kk};
    for (int round = 0; round < 3; ++round) {
        for (int i = tid; i < kBins; i += kThreads) sh.hist[i] = 0;
        __syncthreads();
        const uint32_t prefix = sh.st.prefix, hm = high_mask(round), dm = digit_mask(round);
        const int shft = digit_shift(round);
        // scores cluster in a few bins (the upper digits of small scores are all zero):
        // lanes of a warp that hit the same bin add their count with one atomic
        for (uint32_t t0 = 0; kk > 0 && t0 < M; t0 += kThreads) {
            const uint32_t i = t0 + tid;
            uint32_t bin = 0xffffffffu;
            if (i < M) {
                const uint32_t x = score(i);
                if ((x & hm) == prefix) bin = (x >> shft) & dm;
            }
            const unsigned same = __match_any_sync(0xffffffffu, bin);
            if (bin != 0xffffffffu && lane == __ffs(same) - 1) atomicAdd(&sh.hist[bin], __popc(same));
        }
        __syncthreads();
        if (warp == 0 && kk > 0) {
            // the digit holding the krem-th largest element: lane l sums bins
            // [nb - (l+1) per, nb - l per), lanes in descending order of bins
            const uint32_t krem = sh.st.krem;
            const int nb = round == 2 ? 1024 : kBins;
            const int per = nb / 32;
            const int hi = nb - lane * per;
            uint32_t sum = 0;
            for (int b = hi - per; b < hi; ++b) sum += sh.hist[b];
            uint32_t incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const uint32_t excl = incl - sum;
            if (excl < krem && incl >= krem) {  // exactly one lane
                uint32_t above = excl;
                int d = hi - 1;
                for (; d >= hi - per; --d) {
                    if (above + sh.hist[d] >= krem) break;
                    above += sh.hist[d];
                }
                sh.st.prefix = prefix | ((uint32_t)d << shft);
                sh.st.krem = krem - above;
            }
        }
        __syncthreads();
    }
    const uint32_t thr = sh.st.prefix;
    const uint32_t need = kk > 0 ? sh.st.krem : 0;  // scores == thr to take, first in index order
    // ordered pass: tiles of kThreads elements
    uint32_t base_sel = 0, base_eq = 0;
    for (uint32_t t0 = 0; kk > 0 && t0 < M; t0 += kThreads) {
        const uint32_t i = t0 + tid;
        const uint32_t x = i < M ? score(i) : 0u;
        const bool gt = i < M && x > thr;
        const bool eq = i < M && x == thr;
        const unsigned meq = __ballot_sync(0xffffffffu, eq);
        if (lane == 0) sh.warp_cnt[0][warp] = __popc(meq);
        __syncthreads();
        uint32_t eq_before = base_eq, eq_tile = 0;
        for (int w = 0; w < kWarpsT; ++w) {
            const uint32_t c = sh.warp_cnt[0][w];
            if (w < warp) eq_before += c;
            eq_tile += c;
        }
        eq_before += __popc(meq & ((1u << lane) - 1u));
        const bool sel = gt || (eq && eq_before < need);
        const unsigned msel = __ballot_sync(0xffffffffu, sel);
        if (lane == 0) sh.warp_cnt[1][warp] = __popc(msel);
        __syncthreads();
        uint32_t sel_before = base_sel, sel_tile = 0;
        for (int w = 0; w < kWarpsT; ++w) {
            const uint32_t c = sh.warp_cnt[1][w];
            if (w < warp) sel_before += c;
            sel_tile += c;
        }
        sel_before += __popc(msel & ((1u << lane) - 1u));
        if (sel && sel_before < kk) {
            out_s[sel_before] = (int32_t)x;
            out_i[sel_before] = index(i);
        }
        base_sel += sel_tile;
        base_eq += eq_tile;
        __syncthreads();  // warp_cnt is rewritten by the next tile
    }
    __syncthreads();
}

// grid = (blocks, rows). Dynamic shared memory: the row's candidates for the merge
// (kTopkCandidates scores and indices) and the sort keys.
__global__ void __launch_bounds__(kThreads) topk_kernel(const int32_t* __restrict__ scores,
                                                        uint64_t row_stride, uint64_t n,
                                                        uint32_t k, TopkScratch s,
                                                        int32_t* top_scores, uint64_t* top_index,
                                                        uint32_t k_out) {
    extern __shared__ __align__(16) uint8_t dyn[];
    __shared__ TopkShared sh;
    int32_t* const m_s = reinterpret_cast<int32_t*>(dyn);
    uint32_t* const m_i = reinterpret_cast<uint32_t*>(dyn + kTopkCandidates * 4);
    uint64_t* const key = reinterpret_cast<uint64_t*>(dyn + kTopkCandidates * 8);
    const uint32_t q = blockIdx.y, b = blockIdx.x, B = gridDim.x;
    const int tid = threadIdx.x;
    const int32_t* row = scores + (uint64_t)q * row_stride;

    // ---- this block's slice ----
    const uint64_t chunk = (n + B - 1) / B;
    const uint64_t b0 = (uint64_t)b * chunk;
    const uint64_t b1 = b0 + chunk < n ? b0 + chunk : n;
    const uint32_t M = b1 > b0 ? (uint32_t)(b1 - b0) : 0u;
    const uint32_t kk = M < k ? M : k;
    int32_t* const cs = s.cand_score + (uint64_t)q * kTopkCandidates + (uint64_t)b * k;
    uint32_t* const ci = s.cand_index + (uint64_t)q * kTopkCandidates + (uint64_t)b * k;
    block_select([&](uint32_t i) { return (uint32_t)row[b0 + i]; },
                 [&](uint32_t i) { return (uint32_t)(b0 + i); }, M, kk, sh, cs, ci);
    if (tid == 0) s.cand_count[(uint64_t)q * s.blocks + b] = kk;

    // ---- the last block of the row merges ----
    __threadfence();
    __syncthreads();
    if (tid == 0) sh.last = atomicAdd(&s.done[q], 1u) == B - 1;
    __syncthreads();
    if (!sh.last) return;
    __threadfence();
    // the candidates, block after block (index order), into shared memory
    uint32_t total = 0;
    for (uint32_t bb = 0; bb < B; ++bb) {
        const uint32_t c = *reinterpret_cast<volatile const uint32_t*>(&s.cand_count[(uint64_t)q * s.blocks + bb]);
        const volatile int32_t* src_s = s.cand_score + (uint64_t)q * kTopkCandidates + (uint64_t)bb * k;
        const volatile uint32_t* src_i = s.cand_index + (uint64_t)q * kTopkCandidates + (uint64_t)bb * k;
        for (uint32_t j = tid; j < c; j += kThreads) {
            m_s[total + j] = src_s[j];
            m_i[total + j] = src_i[j];
        }
        total += c;
    }
    const uint32_t kf = total < k ? total : k;  // = min(k, n)
    // the selection writes its kk survivors over the front of the same arrays only after
    // reading them all: select into the key area first
    int32_t* const f_s = reinterpret_cast<int32_t*>(key);
    uint32_t* const f_i = reinterpret_cast<uint32_t*>(key) + kMaxK;
    block_select([&](uint32_t i) { return (uint32_t)m_s[i]; }, [&](uint32_t i) { return m_i[i]; },
                 total, kf, sh, f_s, f_i);
    // sort the kf survivors: key = (score + 1) << 32 | ~index, descending (pads sort last)
    uint64_t mine[kMaxK / kThreads];
#pragma unroll
    for (int r = 0; r < (int)(kMaxK / kThreads); ++r) {
        const uint32_t i = tid + r * kThreads;
        mine[r] = i < kf ? (((uint64_t)((uint32_t)f_s[i] + 1u) << 32) | (uint64_t)(~f_i[i])) : 0ull;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < (int)(kMaxK / kThreads); ++r) key[tid + r * kThreads] = mine[r];
    __syncthreads();
    for (int size = 2; size <= (int)kMaxK; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < (int)kMaxK; i += kThreads) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool desc = (i & size) == 0;
                    const uint64_t x = key[i], y = key[j];
                    if (desc ? (x < y) : (x > y)) { key[i] = y; key[j] = x; }
                }
            }
            __syncthreads();
        }
    }
    for (uint32_t i = tid; i < kf; i += kThreads) {
        const uint64_t v = key[i];
        top_scores[(uint64_t)q * k_out + i] = (int32_t)((uint32_t)(v >> 32) - 1u);
        top_index[(uint64_t)q * k_out + i] = (uint64_t)(uint32_t)~(uint32_t)(v & 0xffffffffu);
    }
    if (tid == 0) s.done[q] = 0;  // ready for the next launch
}

constexpr size_t kDynBytes = (size_t)kTopkCandidates * 8 + (size_t)kMaxK * 8;

}  // namespace

size_t topk_scratch_bytes(uint32_t nq, uint32_t kmax, int blocks) {
    (void)kmax;
    return (size_t)nq * kTopkCandidates * 8 + (size_t)nq * blocks * 4 + (size_t)nq * 4 + 256;
}

void topk_scratch_carve(void* base, uint32_t nq, uint32_t kmax, int blocks, TopkScratch* s) {
    (void)kmax;
    char* p = (char*)base;
    s->cand_score = (int32_t*)p; p += (size_t)nq * kTopkCandidates * 4;
    s->cand_index = (uint32_t*)p; p += (size_t)nq * kTopkCandidates * 4;
    s->cand_count = (uint32_t*)p; p += (size_t)nq * blocks * 4;
    s->done = (uint32_t*)p;
    s->blocks = blocks;
}

int topk_launch_count() { return 1; }

cudaError_t launch_topk(const int32_t* scores, uint64_t row_stride, uint64_t n, uint32_t nq,
                        uint32_t k, const TopkScratch& s, int32_t* top_scores,
                        uint64_t* top_index, cudaStream_t stream) {
    if (k == 0 || n == 0 || nq == 0) return cudaSuccess;
    if (k > kMaxK) return cudaErrorInvalidValue;
    // blocks per row: every block's k candidates fit the row's candidate area, and every
    // block has at least kMinSlice elements
    uint64_t B = kTopkCandidates / k;
    const uint64_t by_n = (n + kMinSlice - 1) / kMinSlice;
    if (B > by_n) B = by_n;
    if (B > (uint64_t)s.blocks) B = (uint64_t)s.blocks;
    if (B < 1) B = 1;
    cudaError_t e = cudaFuncSetAttribute(topk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kDynBytes);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(s.done, 0, (size_t)nq * 4, stream)) != cudaSuccess) return e;
    topk_kernel<<<dim3((unsigned)B, nq), kThreads, kDynBytes, stream>>>(scores, row_stride, n, k, s,
                                                                        top_scores, top_index, k);
    return cudaGetLastError();
}

}  // namespace swgb
