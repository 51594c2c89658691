// Top-k of a search: stage (iv) of the workflow in Section III sorts all
// alignment scores in descending order; the library returns the best top_k,
// equal scores ordered by ascending database index, which makes the list
// unique.
//
// Exact radix select over the non-negative int32 scores, then a sort of the
// selected k:
//   1. three histogram/select rounds over 11 + 11 + 10 bits find the k-th
//      largest score thr and how many scores lie strictly above it;
//   2. one pass collects every score > thr (fewer than k of them) and counts
//      scores == thr per contiguous block; a second pass takes the first
//      (k - #above) scores == thr in index order;
//   3. one block sorts the k candidates by (score desc, index asc).
// Every row of a batch (one row per query) is handled in the same launches
// (grid.y = query).
#include <cuda_runtime.h>
#include <cstdint>

#include "sw_internal.h"

namespace swgb {

namespace {

constexpr int kBins = 2048;
constexpr int kHistThreads = 512;
constexpr int kGatherThreads = 256;

// state[q * 8 + ...]
enum { ST_PREFIX = 0, ST_KREM = 1, ST_ABOVE = 2, ST_NCAND = 3, ST_K = 4 };

__device__ __forceinline__ int digit_shift(int round) { return round == 0 ? 21 : (round == 1 ? 10 : 0); }
__device__ __forceinline__ uint32_t digit_mask(int round) { return round == 2 ? 0x3ffu : 0x7ffu; }
// bits above the digit of this round
__device__ __forceinline__ uint32_t high_mask(int round) {
    return round == 0 ? 0u : (round == 1 ? 0xffe00000u : 0xfffffc00u);
}

__global__ void topk_init(uint32_t* state, uint32_t* hist, uint64_t n, uint32_t k) {
    const uint32_t q = blockIdx.x;
    for (int i = threadIdx.x; i < kBins; i += blockDim.x) hist[(uint64_t)q * kBins + i] = 0;
    if (threadIdx.x == 0) {
        const uint32_t kk = (uint32_t)((uint64_t)k < n ? k : n);
        state[q * 8 + ST_PREFIX] = 0;
        state[q * 8 + ST_KREM] = kk;
        state[q * 8 + ST_ABOVE] = 0;
        state[q * 8 + ST_NCAND] = 0;
        state[q * 8 + ST_K] = kk;
    }
}

__global__ void topk_hist(const int32_t* __restrict__ scores, uint64_t row_stride, uint64_t n,
                          int round, const uint32_t* __restrict__ state, uint32_t* hist) {
    __shared__ uint32_t h[kBins];
    const uint32_t q = blockIdx.y;
    if (state[q * 8 + ST_K] == 0) return;
    for (int i = threadIdx.x; i < kBins; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const uint32_t prefix = state[q * 8 + ST_PREFIX];
    const uint32_t hm = high_mask(round), dm = digit_mask(round);
    const int sh = digit_shift(round);
    const int32_t* row = scores + (uint64_t)q * row_stride;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t x = (uint32_t)row[i];
        if ((x & hm) == prefix) atomicAdd(&h[(x >> sh) & dm], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kBins; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[(uint64_t)q * kBins + i], h[i]);
}

// One warp per query: pick the digit holding the k_rem-th largest element.
__global__ void topk_select(int round, uint32_t* state, uint32_t* hist) {
    const uint32_t q = blockIdx.x;
    const int lane = threadIdx.x;
    uint32_t* H = hist + (uint64_t)q * kBins;
    uint32_t* st = state + q * 8;
    const uint32_t krem = st[ST_KREM];
    if (st[ST_K] == 0) return;
    const int nb = round == 2 ? 1024 : kBins;
    const int per = nb / 32;
    // lane l owns bins [nb - (l+1)*per, nb - l*per) (descending order of lanes)
    const int hi = nb - lane * per;
    uint32_t sum = 0;
    for (int b = hi - per; b < hi; ++b) sum += H[b];
    // exclusive prefix over lanes (lane 0 = highest bins)
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const uint32_t excl = incl - sum;
    const bool mine = excl < krem && incl >= krem;
    const unsigned who = __ballot_sync(0xffffffffu, mine);
    if (mine) {
        uint32_t above = excl;
        int d = hi - 1;
        for (; d >= hi - per; --d) {
            if (above + H[d] >= krem) break;
            above += H[d];
        }
        st[ST_PREFIX] |= ((uint32_t)d) << digit_shift(round);
        st[ST_KREM] = krem - above;
        st[ST_ABOVE] += above;
    }
    (void)who;
    __syncwarp();
    // clear the histogram for the next round
    for (int b = lane; b < kBins; b += 32) H[b] = 0;
}

// Pass 1: collect scores > thr; count scores == thr per contiguous chunk.
__global__ void topk_gather_above(const int32_t* __restrict__ scores, uint64_t row_stride,
                                  uint64_t n, uint32_t* state, uint32_t* block_eq,
                                  int32_t* cand_score, uint32_t* cand_index, uint32_t kmax) {
    const uint32_t q = blockIdx.y;
    uint32_t* st = state + q * 8;
    if (st[ST_K] == 0) return;
    const uint32_t thr = st[ST_PREFIX];
    const uint64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const uint64_t b0 = (uint64_t)blockIdx.x * chunk;
    const uint64_t b1 = b0 + chunk < n ? b0 + chunk : n;
    const int32_t* row = scores + (uint64_t)q * row_stride;
    uint32_t eq = 0;
    for (uint64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        const uint32_t x = (uint32_t)row[i];
        if (x > thr) {
            const uint32_t c = atomicAdd(&st[ST_NCAND], 1u);
            cand_score[(uint64_t)q * kmax + c] = (int32_t)x;
            cand_index[(uint64_t)q * kmax + c] = (uint32_t)i;
        }
        eq += (x == thr);
    }
    __shared__ uint32_t red[kGatherThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) eq += __shfl_xor_sync(0xffffffffu, eq, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = eq;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int w = 0; w < kGatherThreads / 32; ++w) s += red[w];
        block_eq[(uint64_t)q * gridDim.x + blockIdx.x] = s;
    }
}

// Pass 2: the first k_rem scores == thr in index order.
__global__ void topk_gather_equal(const int32_t* __restrict__ scores, uint64_t row_stride,
                                  uint64_t n, const uint32_t* state, const uint32_t* block_eq,
                                  int32_t* cand_score, uint32_t* cand_index, uint32_t kmax) {
    const uint32_t q = blockIdx.y;
    const uint32_t* st = state + q * 8;
    if (st[ST_K] == 0) return;
    const uint32_t thr = st[ST_PREFIX];
    const uint32_t need = st[ST_KREM];
    const uint32_t above = st[ST_ABOVE];
    __shared__ uint32_t s_base;
    __shared__ uint32_t warp_cnt[kGatherThreads / 32];
    if (threadIdx.x == 0) {
        uint32_t b = 0;
        for (uint32_t i = 0; i < blockIdx.x; ++i) b += block_eq[(uint64_t)q * gridDim.x + i];
        s_base = b;
    }
    __syncthreads();
    uint32_t base = s_base;
    if (base >= need) return;
    const uint64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const uint64_t b0 = (uint64_t)blockIdx.x * chunk;
    const uint64_t b1 = b0 + chunk < n ? b0 + chunk : n;
    const int32_t* row = scores + (uint64_t)q * row_stride;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint64_t t0 = b0; t0 < b1; t0 += blockDim.x) {  // block-uniform loop
        const uint64_t i = t0 + threadIdx.x;
        const bool hit = i < b1 && (uint32_t)row[i] == thr;
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (lane == 0) warp_cnt[warp] = __popc(m);
        __syncthreads();
        uint32_t before = base;
        for (int w = 0; w < warp; ++w) before += warp_cnt[w];
        before += __popc(m & ((1u << lane) - 1u));
        if (hit && before < need) {
            cand_score[(uint64_t)q * kmax + above + before] = (int32_t)thr;
            cand_index[(uint64_t)q * kmax + above + before] = (uint32_t)i;
        }
        uint32_t tot = 0;
        for (int w = 0; w < kGatherThreads / 32; ++w) tot += warp_cnt[w];
        __syncthreads();
        base += tot;
        if (base >= need) break;
    }
}

// One block per query sorts the k candidates (bitonic, padded to 1024).
__global__ void topk_sort(const uint32_t* state, const int32_t* cand_score,
                          const uint32_t* cand_index, uint32_t kmax, int32_t* top_scores,
                          uint64_t* top_index, uint32_t k_out) {
    __shared__ uint64_t key[1024];
    const uint32_t q = blockIdx.x;
    const uint32_t k = state[q * 8 + ST_K];
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) {
        uint64_t v = 0;  // sorts last
        if ((uint32_t)i < k) {
            // descending score, ascending index: key = (score << 32) | ~index, sorted descending
            const uint32_t s = (uint32_t)cand_score[(uint64_t)q * kmax + i];
            const uint32_t idx = cand_index[(uint64_t)q * kmax + i];
            v = ((uint64_t)(s + 1u) << 32) | (uint64_t)(~idx);
        }
        key[i] = v;
    }
    __syncthreads();
    for (int size = 2; size <= 1024; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < 1024; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool desc = (i & size) == 0;
                    const uint64_t a = key[i], b = key[j];
                    if (desc ? (a < b) : (a > b)) { key[i] = b; key[j] = a; }
                }
            }
            __syncthreads();
        }
    }
    for (uint32_t i = threadIdx.x; i < k; i += blockDim.x) {
        const uint64_t v = key[i];
        top_scores[(uint64_t)q * k_out + i] = (int32_t)((uint32_t)(v >> 32) - 1u);
        top_index[(uint64_t)q * k_out + i] = (uint64_t)(uint32_t)~(uint32_t)(v & 0xffffffffu);
    }
}

}  // namespace

size_t topk_scratch_bytes(uint32_t nq, uint32_t kmax, int blocks) {
    const size_t a = (size_t)nq * kBins * 4;
    const size_t b = (size_t)nq * 8 * 4;
    const size_t c = (size_t)nq * blocks * 4;
    const size_t d = (size_t)nq * kmax * 4 * 2;
    return a + b + c + d + 256;
}

void topk_scratch_carve(void* base, uint32_t nq, uint32_t kmax, int blocks, TopkScratch* s) {
    char* p = (char*)base;
    s->hist = (uint32_t*)p; p += (size_t)nq * kBins * 4;
    s->state = (uint32_t*)p; p += (size_t)nq * 8 * 4;
    s->block_eq = (uint32_t*)p; p += (size_t)nq * blocks * 4;
    s->cand_score = (int32_t*)p; p += (size_t)nq * kmax * 4;
    s->cand_index = (uint32_t*)p;
    s->blocks = blocks;
}

int topk_launch_count() { return 1 + 3 * 2 + 3; }

cudaError_t launch_topk(const int32_t* scores, uint64_t row_stride, uint64_t n, uint32_t nq,
                        uint32_t k, const TopkScratch& s, int32_t* top_scores,
                        uint64_t* top_index, cudaStream_t stream) {
    if (k == 0 || n == 0 || nq == 0) return cudaSuccess;
    if (k > 1024) return cudaErrorInvalidValue;
    topk_init<<<nq, 256, 0, stream>>>(s.state, s.hist, n, k);
    const int hblocks = (int)((n + kHistThreads * 16 - 1) / (kHistThreads * 16));
    const dim3 hg(hblocks < 1 ? 1 : (hblocks > 1024 ? 1024 : hblocks), nq);
    for (int round = 0; round < 3; ++round) {
        topk_hist<<<hg, kHistThreads, 0, stream>>>(scores, row_stride, n, round, s.state, s.hist);
        topk_select<<<nq, 32, 0, stream>>>(round, s.state, s.hist);
    }
    const dim3 gg(s.blocks, nq);
    topk_gather_above<<<gg, kGatherThreads, 0, stream>>>(scores, row_stride, n, s.state,
                                                          s.block_eq, s.cand_score, s.cand_index,
                                                          1024);
    topk_gather_equal<<<gg, kGatherThreads, 0, stream>>>(scores, row_stride, n, s.state,
                                                          s.block_eq, s.cand_score, s.cand_index,
                                                          1024);
    topk_sort<<<nq, 1024, 0, stream>>>(s.state, s.cand_score, s.cand_index, 1024, top_scores,
                                       top_index, k);
    return cudaGetLastError();
}

}  // namespace swgb
