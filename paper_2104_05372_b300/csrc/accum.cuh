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

// First lane of this lane's run: the highest lane <= this one whose key differs
// from its left neighbour's (a run is a maximal stretch of adjacent equal keys;
// equal keys further apart are separate runs). All 32 lanes must call it.
__device__ __forceinline__ int run_head(int key) {
    const unsigned lane = lane_id();
    const int prev = __shfl_up_sync(0xffffffffu, key, 1);
    const unsigned starts = __ballot_sync(0xffffffffu, lane == 0u || prev != key);
    return 31 - __clz(starts & (0xffffffffu >> (31u - lane)));
}

// Inclusive scan of v within this lane's run [head, lane]; the last lane of
// each run ends up with the run's total. All 32 lanes must call it.
template <typename T>
__device__ __forceinline__ T run_scan_head(T v, int head) {
    const int lane = (int)lane_id();
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const T t = __shfl_up_sync(0xffffffffu, v, off);
        if (lane - off >= head) v += t;
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T run_scan(T v, int key) {
    return run_scan_head(v, run_head(key));
}

__device__ __forceinline__ bool run_end(int key) {
    const int nxt = __shfl_down_sync(0xffffffffu, key, 1);
    return lane_id() == 31u || nxt != key;
}

}  // namespace gpa
