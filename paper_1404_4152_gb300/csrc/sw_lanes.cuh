// Device-side lane arithmetic shared by the search kernels: packed pairs of
// 16-bit lanes (two cells per 32-bit register) and plain int32 lanes, with
// the fused add-max forms the GPU executes in one instruction.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace swgb {

static __device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
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

// Shared-memory accesses by byte address (the state space known, no generic-address
// conversion).
static __device__ __forceinline__ uint32_t lds_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}
// The value of the thread above (shfl.up within segments of T threads); the
// first thread of a segment, which has none, loads it from shared memory.
template <int T>
static __device__ __forceinline__ uint32_t shfl_up_or_lds(uint32_t v, uint32_t addr) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "shfl.sync.up.b32 %0|p, %1, 1, %3, -1;\n\t"
        "@!p ld.shared.u32 %0, [%2];\n\t}"
        : "=r"(r)
        : "r"(v), "r"(addr), "n"((32 - T) << 8));
    return r;
}
static __device__ __forceinline__ void sts_u32(uint32_t addr, uint32_t v) {
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(addr), "r"(v));
}
static __device__ __forceinline__ void sts_u64(uint32_t addr, uint2 v) {
    asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(addr), "r"(v.x), "r"(v.y));
}

}  // namespace swgb
