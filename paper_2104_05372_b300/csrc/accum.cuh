// Warp-level Accum helpers: aggregation of equal keys before the atomic update.
#pragma once

#include "common.cuh"

namespace gpa {

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Sum of v over the lanes of `group` (a __match_any_sync mask containing this
// lane); every lane of the group gets the total. All 32 lanes must call it.
__device__ __forceinline__ float group_sum(float v, unsigned group) {
    float s = 0.f;
#pragma unroll 4
    for (int src = 0; src < 32; ++src) {
        const float t = __shfl_sync(0xffffffffu, v, src);
        if ((group >> src) & 1u) s += t;
    }
    return s;
}

__device__ __forceinline__ int group_sum(int v, unsigned group) {
    int s = 0;
#pragma unroll 4
    for (int src = 0; src < 32; ++src) {
        const int t = __shfl_sync(0xffffffffu, v, src);
        if ((group >> src) & 1u) s += t;
    }
    return s;
}

// Inclusive segmented scan over runs of equal keys in lane order (keys must
// form contiguous runs, as in a key-sorted sequence). The last lane of each run
// ends up with the run's total.
template <typename T>
__device__ __forceinline__ T run_scan(T v, int key) {
    const unsigned lane = lane_id();
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const T t = __shfl_up_sync(0xffffffffu, v, off);
        const int kk = __shfl_up_sync(0xffffffffu, key, off);
        if (lane >= (unsigned)off && kk == key) v += t;
    }
    return v;
}

__device__ __forceinline__ bool run_end(int key) {
    const int nxt = __shfl_down_sync(0xffffffffu, key, 1);
    return lane_id() == 31u || nxt != key;
}

}  // namespace gpa
