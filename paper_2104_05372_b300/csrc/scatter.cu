// Index preparation (A7) and the generic Accum scatter (A6).
//
// Plan = stable sort of element ids by a data-derived key. Indices are checked
// here, where they are constructed from data (Sec. 6.3); invalid elements get
// the key n_keys and sort after every valid one. The sort is an LSD radix sort
// with 8-bit digits; each pass is stable: per-tile digit counts, one exclusive
// scan over (digit, tile), then one warp per tile writes its elements in order,
// ranking equal digits inside each 32-element step with __match_any_sync.
//
// accum_scatter_add: acc[idx[j]][c] += vals[j][c] (hist!(x.i) += v, Sec. 2.3.3;
// work-efficient and parallel at once, Sec. 6.1.2):
//   ATOMIC   one red.global.add per value;
//   WARPAGG  lanes of a warp with equal indices combine first (skewed keys);
//   SORT     key-sorted order from a plan, runs summed by a segmented warp scan.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "accum.cuh"
#include "common.cuh"
#include "plan_internal.cuh"
#include "trace.cuh"

namespace gpa {

constexpr int kSortTile = 4096;  // elements per radix tile (one warp writes it)

// keys from observations: key = camera if both indices are valid, else n_keys
__global__ void __launch_bounds__(256) plan_keys_obs_kernel(const int2* __restrict__ obs, int64_t n,
                                                            int n_keys, int n_aux, int32_t* __restrict__ key,
                                                            int32_t* __restrict__ id, int32_t* __restrict__ aux,
                                                            int32_t* __restrict__ status) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int2 o = __ldg(obs + j);
    const bool ok = o.x >= 0 && o.x < n_keys && o.y >= 0 && o.y < n_aux;
    if (!ok) report(status, GPA_ERR_INDEX);
    key[j] = ok ? o.x : n_keys;
    id[j] = (int32_t)j;
    aux[j] = o.y;
}

__global__ void __launch_bounds__(256) plan_keys_idx_kernel(const int32_t* __restrict__ idx, int64_t n,
                                                            int n_keys, int32_t* __restrict__ key,
                                                            int32_t* __restrict__ id, int32_t* __restrict__ aux,
                                                            int32_t* __restrict__ status) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int v = __ldg(idx + j);
    const bool ok = v >= 0 && v < n_keys;
    if (!ok) report(status, GPA_ERR_INDEX);
    key[j] = ok ? v : n_keys;
    id[j] = (int32_t)j;
    aux[j] = 0;
}

// per-tile digit histogram: cnt[digit * ntiles + tile]
__global__ void __launch_bounds__(256) radix_hist_kernel(const int32_t* __restrict__ key, int64_t n, int shift,
                                                         int64_t ntiles, int32_t* __restrict__ cnt) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t t0 = (int64_t)blockIdx.x * kSortTile;
    const int64_t t1 = min64(n, t0 + kSortTile);
    for (int64_t j = t0 + threadIdx.x; j < t1; j += 256) atomicAdd(&h[(key[j] >> shift) & 255], 1);
    __syncthreads();
    cnt[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}


// Offsets of the radix scatter: cnt [256][ntiles] (digit-major) becomes, in
// place, the exclusive prefix sum of the flattened array, computed in two
// parallel steps: digit totals, then one CTA per digit scanning its tiles
// with the totals of the smaller digits as base.
__global__ void __launch_bounds__(1024) digit_total_kernel(const int32_t* __restrict__ cnt, int64_t ntiles,
                                                           int32_t* __restrict__ tot) {
    __shared__ int32_t part[32];
    const int d = blockIdx.x;
    int32_t s = 0;
    for (int64_t t = threadIdx.x; t < ntiles; t += blockDim.x) s += cnt[(int64_t)d * ntiles + t];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        int32_t v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0;
        v = warp_sum(v);
        if (threadIdx.x == 0) tot[d] = v;
    }
}

__global__ void __launch_bounds__(1024) digit_scan_kernel(int32_t* __restrict__ cnt, int64_t ntiles,
                                                          const int32_t* __restrict__ tot) {
    __shared__ int32_t wsum[32];
    __shared__ int32_t carry;
    const int d = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        int32_t b = 0;
        for (int e = 0; e < d; ++e) b += tot[e];
        carry = b;
    }
    __syncthreads();
    int32_t* row = cnt + (int64_t)d * ntiles;
    for (int64_t t0 = 0; t0 < ntiles; t0 += blockDim.x) {  // uniform trip count
        const int64_t t = t0 + threadIdx.x;
        const int32_t v = t < ntiles ? row[t] : 0;
        int32_t x = v;  // inclusive scan within the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {  // scan of the warp sums
            int32_t w = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            wsum[lane] = w;  // inclusive
        }
        __syncthreads();
        const int32_t before = carry + (warp > 0 ? wsum[warp - 1] : 0);
        if (t < ntiles) row[t] = before + x - v;  // exclusive
        __syncthreads();
        if (threadIdx.x == 0) carry += wsum[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
}

// seg_off[k] = first position of key k in the sorted keys (n_keys + 1 entries;
// seg_off[n_keys] = number of valid elements, invalid keys being n_keys and
// sorted last): from the boundaries of the sorted runs, no atomics.
__global__ void __launch_bounds__(256) seg_offsets_kernel(const int32_t* __restrict__ key_s, int64_t n,
                                                          int n_keys, int32_t* __restrict__ seg_off) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j > n) return;
    const int prev = j == 0 ? -1 : key_s[j - 1];
    const int cur = j == n ? n_keys : key_s[j];
    for (int k = prev + 1; k <= cur; ++k) seg_off[k] = (int32_t)j;
}

// stable scatter of one tile by one warp
__global__ void __launch_bounds__(32) radix_scatter_kernel(const int32_t* __restrict__ kin,
                                                           const int32_t* __restrict__ iin, int64_t n, int shift,
                                                           int64_t ntiles, const int32_t* __restrict__ off,
                                                           int32_t* __restrict__ kout, int32_t* __restrict__ iout) {
    __shared__ int base[256];
    const int lane = threadIdx.x;
    for (int dgt = lane; dgt < 256; dgt += 32) base[dgt] = off[(int64_t)dgt * ntiles + blockIdx.x];
    __syncwarp();
    const int64_t t0 = (int64_t)blockIdx.x * kSortTile;
    const int64_t t1 = min64(n, t0 + kSortTile);
    const unsigned lt = (1u << lane) - 1u;
    constexpr int U = 4;  // iterations whose keys and ids are loaded together
    for (int64_t j0 = t0; j0 < t1; j0 += 32 * U) {
        int kk[U], ii[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t j = j0 + 32 * u + lane;
            kk[u] = j < t1 ? kin[j] : 0;
            ii[u] = j < t1 ? iin[j] : 0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t j = j0 + 32 * u + lane;
            const bool v = j < t1;
            const int dgt = v ? ((kk[u] >> shift) & 255) : 256 + lane;  // unique dummy digit
            const unsigned grp = __match_any_sync(0xffffffffu, dgt);
            const int rank = __popc(grp & lt);
            int pos = 0;
            if (v) pos = base[dgt] + rank;
            __syncwarp();
            if (v) {
                kout[pos] = kk[u];
                iout[pos] = ii[u];
                if (rank == 0) base[dgt] += __popc(grp);
            }
            __syncwarp();
        }
    }
}

__global__ void __launch_bounds__(256) plan_finish_kernel(const int32_t* __restrict__ ks,
                                                          const int32_t* __restrict__ is,
                                                          const int32_t* __restrict__ aux, int64_t n,
                                                          int32_t* __restrict__ perm, int32_t* __restrict__ key_sorted,
                                                          int32_t* __restrict__ aux_sorted) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int e = is[j];
    perm[j] = e;
    key_sorted[j] = ks[j];
    aux_sorted[j] = aux[e];
}

__global__ void plan_header_kernel(int64_t* __restrict__ hdr, int64_t n, int n_keys,
                                   const int32_t* __restrict__ seg_off) {
    hdr[0] = n;
    hdr[1] = n_keys;
    hdr[2] = seg_off[n_keys];
    hdr[3] = 0;
}

// ---- scatter -----------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) scatter_atomic_kernel(const int32_t* __restrict__ idx,
                                                             const T* __restrict__ vals, int64_t m, int w,
                                                             T* __restrict__ acc, int n_buckets,
                                                             int32_t* __restrict__ status) {
    const int64_t total = m * w;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        const int64_t j = e / w;
        const int c = (int)(e - j * w);
        const int b = __ldg(idx + j);
        if (b < 0 || b >= n_buckets) {
            if (c == 0) report(status, GPA_ERR_INDEX);
            continue;
        }
        atomicAdd(acc + (int64_t)b * w + c, __ldg(vals + e));
    }
}

template <typename T>
__global__ void __launch_bounds__(256) scatter_warpagg_kernel(const int32_t* __restrict__ idx,
                                                              const T* __restrict__ vals, int64_t m, int w,
                                                              T* __restrict__ acc, int n_buckets,
                                                              int32_t* __restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < m; base += stride) {
        const int64_t j = base + threadIdx.x;
        int b = j < m ? __ldg(idx + j) : -1;
        bool valid = j < m && b >= 0 && b < n_buckets;
        if (j < m && !valid) report(status, GPA_ERR_INDEX);
        const int key = valid ? b : -1 - lane;
        const unsigned grp = __match_any_sync(0xffffffffu, key);
        const bool multi = __any_sync(0xffffffffu, __popc(grp) > 1);
        const bool leader = valid && (__ffs(grp) - 1) == lane;
        for (int c = 0; c < w; ++c) {
            T v = valid ? __ldg(vals + j * w + c) : T(0);
            if (multi) v = group_sum(v, grp);
            if (leader) atomicAdd(acc + (int64_t)b * w + c, v);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) scatter_sorted_kernel(const int32_t* __restrict__ perm,
                                                             const int32_t* __restrict__ key_s,
                                                             const T* __restrict__ vals, int64_t m, int w,
                                                             T* __restrict__ acc, int n_buckets) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < m; base += stride) {
        const int64_t j = base + threadIdx.x;
        int b = j < m ? __ldg(key_s + j) : n_buckets;
        const int64_t e = (b >= 0 && b < n_buckets) ? (int64_t)__ldg(perm + j) : 0;
        if (e < 0 || e >= m) b = n_buckets;  // not a plan of these indices
        const bool valid = b >= 0 && b < n_buckets;  // invalid elements were reported by the plan
        const int key = valid ? b : -1 - lane;
        const bool last = run_end(key);
        const int head = run_head(key);
        for (int c = 0; c < w; ++c) {
            T v = valid ? __ldg(vals + e * w + c) : T(0);
            v = run_scan_head(v, head);
            if (valid && last) atomicAdd(acc + (int64_t)b * w + c, v);
        }
    }
}

// SMEM: every CTA accumulates into its own copy of acc in shared memory (shared
// atomics, no contention across the GPU), then adds each entry it touched into
// acc once. For few buckets: n_buckets * w <= kSmemEntries.
constexpr int kSmemEntries = 24576;  // 96 KB of float / int32: two CTAs per SM

template <typename T>
__global__ void __launch_bounds__(256) scatter_smem_kernel(const int32_t* __restrict__ idx,
                                                           const T* __restrict__ vals, int64_t m, int w,
                                                           T* __restrict__ acc, int n_buckets,
                                                           int32_t* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* priv = reinterpret_cast<T*>(smem_raw);
    const int ne = n_buckets * w;
    for (int e = threadIdx.x; e < ne; e += blockDim.x) priv[e] = T(0);
    __syncthreads();
    const int64_t total = m * w;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t e0 = 0;
    if (w == 1 && ((reinterpret_cast<uintptr_t>(idx) | reinterpret_cast<uintptr_t>(vals)) & 15) == 0) {
        // four elements per thread and step, 16-byte loads; four steps' loads
        // issued together so that eight are in flight per thread
        const int64_t m4 = m / 4;
        const int4* idx4 = reinterpret_cast<const int4*>(idx);
        const float4* val4 = reinterpret_cast<const float4*>(vals);
        auto add4 = [&](const int4 b4, const float4 raw) {
            const int bs[4] = {b4.x, b4.y, b4.z, b4.w};
            const float vf[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (bs[u] < 0 || bs[u] >= n_buckets) {
                    report(status, GPA_ERR_INDEX);
                    continue;
                }
                T v;
                memcpy(&v, &vf[u], sizeof(T));  // T is float or int32: the same 4 bytes
                atomicAdd(priv + bs[u], v);
            }
        };
        int64_t q = t0;
        for (; q + 3 * stride < m4; q += 4 * stride) {
            int4 b4[4];
            float4 raw[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                b4[h] = __ldg(idx4 + q + h * stride);
                raw[h] = __ldg(val4 + q + h * stride);
            }
#pragma unroll
            for (int h = 0; h < 4; ++h) add4(b4[h], raw[h]);
        }
        for (; q < m4; q += stride) add4(__ldg(idx4 + q), __ldg(val4 + q));
        e0 = m4 * 4;
    }
    for (int64_t e = e0 + t0; e < total; e += stride) {
        const int64_t j = w == 1 ? e : e / w;
        const int c = (int)(e - j * w);
        const int b = __ldg(idx + j);
        if (b < 0 || b >= n_buckets) {
            if (c == 0) report(status, GPA_ERR_INDEX);
            continue;
        }
        atomicAdd(priv + b * w + c, __ldg(vals + e));
    }
    __syncthreads();
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
        const T v = priv[e];
        if (v != T(0)) atomicAdd(acc + e, v);  // untouched entries add nothing
    }
}

// Complete reduction (one bucket, one value per element): per-thread sums, a
// warp tree, a block tree, one atomic per CTA.
template <typename T>
__global__ void __launch_bounds__(256) scatter_complete_kernel(const int32_t* __restrict__ idx,
                                                               const T* __restrict__ vals, int64_t m,
                                                               T* __restrict__ acc, int32_t* __restrict__ status) {
    T sum = T(0);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t j0 = 0;
    if (((reinterpret_cast<uintptr_t>(idx) | reinterpret_cast<uintptr_t>(vals)) & 15) == 0) {
        // four elements per thread and step, 16-byte loads; four steps' loads
        // issued together (eight in flight per thread), summed in step order
        const int64_t m4 = m / 4;
        const int4* idx4 = reinterpret_cast<const int4*>(idx);
        const float4* val4 = reinterpret_cast<const float4*>(vals);
        auto add4 = [&](const int4 b4, const float4 raw) {
            const int bs[4] = {b4.x, b4.y, b4.z, b4.w};
            const float vf[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (bs[u] != 0) {
                    report(status, GPA_ERR_INDEX);
                    continue;
                }
                T v;
                memcpy(&v, &vf[u], sizeof(T));
                sum += v;
            }
        };
        int64_t q = t0;
        for (; q + 3 * stride < m4; q += 4 * stride) {
            int4 b4[4];
            float4 raw[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                b4[h] = __ldg(idx4 + q + h * stride);
                raw[h] = __ldg(val4 + q + h * stride);
            }
#pragma unroll
            for (int h = 0; h < 4; ++h) add4(b4[h], raw[h]);
        }
        for (; q < m4; q += stride) add4(__ldg(idx4 + q), __ldg(val4 + q));
        j0 = m4 * 4;
    }
    for (int64_t j = j0 + t0; j < m; j += stride) {
        if (__ldg(idx + j) != 0) {
            report(status, GPA_ERR_INDEX);
            continue;
        }
        sum += __ldg(vals + j);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    __shared__ T part[8];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        T t = T(0);
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += part[i];
        atomicAdd(acc, t);
    }
}

// RUNS: equal indices are adjacent in input order (a regular segmented
// reduction, e.g. idx = j / L, or any grouped index): runs summed by a
// segmented warp scan, one atomic per run and warp, no plan. Correct for any
// index order; efficient when runs are long.
template <typename T>
__global__ void __launch_bounds__(256) scatter_runs_kernel(const int32_t* __restrict__ idx,
                                                           const T* __restrict__ vals, int64_t m, int w,
                                                           T* __restrict__ acc, int n_buckets,
                                                           int32_t* __restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < m; base += stride) {
        const int64_t j = base + threadIdx.x;
        const int b = j < m ? __ldg(idx + j) : -1;
        const bool valid = j < m && b >= 0 && b < n_buckets;
        if (j < m && !valid) report(status, GPA_ERR_INDEX);
        const int key = valid ? b : -1 - lane;
        const bool last = run_end(key);
        const int head = run_head(key);
        for (int c = 0; c < w; ++c) {
            T v = valid ? __ldg(vals + j * w + c) : T(0);
            v = run_scan_head(v, head);
            if (valid && last) atomicAdd(acc + (int64_t)b * w + c, v);
        }
    }
}

static unsigned grid_for(int64_t n) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + 255) / 256;
    const int64_t cap = (int64_t)sms * 8;
    return (unsigned)(want < cap ? want : cap);
}

// workspace: key_a, id_a, key_b, id_b, aux (n each), cnt (256 * ntiles), digit totals (256)
static size_t plan_ws_bytes(int64_t n) {
    const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    return 5 * plan_a256(sizeof(int32_t) * (size_t)n) + plan_a256(sizeof(int32_t) * 256 * (size_t)ntiles) +
           plan_a256(sizeof(int32_t) * 256) + 256;
}

static int build_plan(const int2* obs, const int32_t* idx, int64_t n, int n_keys, int n_aux, void* plan,
                      void* ws, int32_t* status, cudaStream_t s) {
    char* w = (char*)ws;
    const size_t vb = plan_a256(sizeof(int32_t) * (size_t)n);
    int32_t* ka = (int32_t*)(w);
    int32_t* ia = (int32_t*)(w + vb);
    int32_t* kb = (int32_t*)(w + 2 * vb);
    int32_t* ib = (int32_t*)(w + 3 * vb);
    int32_t* aux = (int32_t*)(w + 4 * vb);
    int32_t* cnt = (int32_t*)(w + 5 * vb);
    int32_t* tot = (int32_t*)(w + 5 * vb + plan_a256(sizeof(int32_t) * 256 * (size_t)((n + kSortTile - 1) / kSortTile)));
    const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    const unsigned g = (unsigned)((n + 255) / 256);
    if (obs)
        GPA_LAUNCH("plan_keys_obs", s, plan_keys_obs_kernel<<<g, 256, 0, s>>>(obs, n, n_keys, n_aux, ka, ia, aux, status));
    else
        GPA_LAUNCH("plan_keys_idx", s, plan_keys_idx_kernel<<<g, 256, 0, s>>>(idx, n, n_keys, ka, ia, aux, status));
    GPA_LAUNCH_CHECK();
    int bits = 1;
    while ((1ll << bits) <= (int64_t)n_keys) ++bits;  // keys in [0, n_keys]
    const int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        GPA_LAUNCH("radix_hist", s, radix_hist_kernel<<<(unsigned)ntiles, 256, 0, s>>>(ka, n, shift, ntiles, cnt));
        GPA_LAUNCH("digit_total", s, digit_total_kernel<<<256, 1024, 0, s>>>(cnt, ntiles, tot));
        GPA_LAUNCH("digit_scan", s, digit_scan_kernel<<<256, 1024, 0, s>>>(cnt, ntiles, tot));
        GPA_LAUNCH("radix_scatter", s, radix_scatter_kernel<<<(unsigned)ntiles, 32, 0, s>>>(ka, ia, n, shift, ntiles, cnt, kb, ib));
        GPA_LAUNCH_CHECK();
        int32_t* t = ka; ka = kb; kb = t;
        t = ia; ia = ib; ib = t;
    }
    PlanView pv = plan_view(plan, n, n_keys);
    GPA_LAUNCH("plan_finish", s, plan_finish_kernel<<<g, 256, 0, s>>>(ka, ia, aux, n, pv.perm, pv.key_sorted, pv.aux_sorted));
    GPA_LAUNCH("seg_offsets", s,
               seg_offsets_kernel<<<(unsigned)((n + 1 + 255) / 256), 256, 0, s>>>(pv.key_sorted, n, n_keys, pv.seg_off));
    GPA_LAUNCH("plan_header", s, plan_header_kernel<<<1, 1, 0, s>>>(pv.header, n, n_keys, pv.seg_off));
    GPA_LAUNCH_CHECK();
    return GPA_OK;
}

}  // namespace gpa

using namespace gpa;

extern "C" size_t gpa_plan_bytes(int64_t n_elems, int32_t n_keys) {
    if (n_elems < 1 || n_keys < 1) return 0;
    return plan_size(n_elems, n_keys);
}

extern "C" size_t gpa_plan_workspace_bytes(int64_t n_elems, int32_t n_keys) {
    if (n_elems < 1 || n_keys < 1) return 0;
    return plan_ws_bytes(n_elems);
}

static int plan_check(const void* in, int64_t n, int32_t n_keys, void* plan, size_t plan_bytes, void* ws,
                      size_t ws_bytes) {
    if (!in || !plan || !ws) return GPA_ERR_ARG;
    if (n < 1 || n > INT32_MAX || n_keys < 1 || n_keys >= INT32_MAX) return GPA_ERR_ARG;
    if ((((uintptr_t)plan) & 255) || (((uintptr_t)ws) & 255)) return GPA_ERR_ALIGN;
    if (plan_bytes < plan_size(n, n_keys) || ws_bytes < plan_ws_bytes(n)) return GPA_ERR_WORKSPACE;
    return GPA_OK;
}

extern "C" int gpa_obs_plan_build(const int32_t* obs, int64_t n_obs, int32_t n_cams, int32_t n_pts, void* plan,
                                  size_t plan_bytes, void* ws, size_t ws_bytes, int32_t* dev_status,
                                  gpa_stream_t stream) {
    int rc = plan_check(obs, n_obs, n_cams, plan, plan_bytes, ws, ws_bytes);
    if (rc) return rc;
    if (n_pts < 1) return GPA_ERR_ARG;
    if (((uintptr_t)obs) & 7) return GPA_ERR_ALIGN;
    return build_plan((const int2*)obs, nullptr, n_obs, n_cams, n_pts, plan, ws, dev_status, (cudaStream_t)stream);
}

extern "C" int gpa_index_plan_build(const int32_t* idx, int64_t m, int32_t n_keys, void* plan, size_t plan_bytes,
                                    void* ws, size_t ws_bytes, int32_t* dev_status, gpa_stream_t stream) {
    int rc = plan_check(idx, m, n_keys, plan, plan_bytes, ws, ws_bytes);
    if (rc) return rc;
    return build_plan(nullptr, idx, m, n_keys, 1, plan, ws, dev_status, (cudaStream_t)stream);
}

extern "C" int accum_scatter_add(const int32_t* idx, const void* vals, int64_t m, int32_t w, int32_t dtype,
                                 void* acc, int32_t n_buckets, int32_t strat, const void* plan,
                                 int32_t* dev_status, gpa_stream_t stream) {
    if (!idx || !vals || !acc) return GPA_ERR_ARG;
    if (m < 1 || m > INT32_MAX || w < 1 || w > 64 || n_buckets < 1) return GPA_ERR_ARG;
    if (dtype != 0 && dtype != 1) return GPA_ERR_ARG;
    if ((((uintptr_t)idx) | ((uintptr_t)vals) | ((uintptr_t)acc)) & 3) return GPA_ERR_ALIGN;
    const bool few = (int64_t)n_buckets * w <= kSmemEntries;
    if (strat == GPA_SCATTER_AUTO) strat = plan ? GPA_SCATTER_SORT : few ? GPA_SCATTER_SMEM : GPA_SCATTER_ATOMIC;
    cudaStream_t s = (cudaStream_t)stream;
    switch (strat) {
        case GPA_SCATTER_SMEM: {
            if (!few) return GPA_ERR_UNSUPPORTED;
            if (n_buckets == 1 && w == 1) {  // complete reduction
                const unsigned g = grid_for((m + 3) / 4);
                if (dtype == 0)
                    GPA_LAUNCH("scatter_complete", s,
                               scatter_complete_kernel<float><<<g, 256, 0, s>>>(idx, (const float*)vals, m,
                                                                                (float*)acc, dev_status));
                else
                    GPA_LAUNCH("scatter_complete", s,
                               scatter_complete_kernel<int><<<g, 256, 0, s>>>(idx, (const int*)vals, m, (int*)acc,
                                                                              dev_status));
                break;
            }
            const size_t smem = sizeof(float) * (size_t)n_buckets * w;
            // enough CTAs to fill the GPU, few enough that flushing stays small against the scatter
            int64_t per = (int64_t)n_buckets * w * 8;
            if (per < 4096) per = 4096;
            const int64_t want = (m * w + per - 1) / per;
            int dev = 0, sms = 148;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            int per_sm = (int)((200 * 1024) / (smem + 1024));  // CTAs that fit one SM's shared memory
            per_sm = per_sm < 1 ? 1 : per_sm > 8 ? 8 : per_sm;
            const unsigned cap = (unsigned)(sms * per_sm);
            const unsigned g = (unsigned)(want < 1 ? 1 : (want < cap ? want : cap));
            if (dtype == 0) {
                auto kern = scatter_smem_kernel<float>;
                if (smem > 48 * 1024 &&
                    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
                    return GPA_ERR_CUDA;
                GPA_LAUNCH("scatter_smem", s,
                           kern<<<g, 256, smem, s>>>(idx, (const float*)vals, m, w, (float*)acc, n_buckets,
                                                     dev_status));
            } else {
                auto kern = scatter_smem_kernel<int>;
                if (smem > 48 * 1024 &&
                    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
                    return GPA_ERR_CUDA;
                GPA_LAUNCH("scatter_smem", s,
                           kern<<<g, 256, smem, s>>>(idx, (const int*)vals, m, w, (int*)acc, n_buckets, dev_status));
            }
            break;
        }
        case GPA_SCATTER_RUNS: {
            const unsigned g = grid_for(m);
            if (dtype == 0)
                GPA_LAUNCH("scatter_runs", s,
                           scatter_runs_kernel<float><<<g, 256, 0, s>>>(idx, (const float*)vals, m, w, (float*)acc,
                                                                        n_buckets, dev_status));
            else
                GPA_LAUNCH("scatter_runs", s,
                           scatter_runs_kernel<int><<<g, 256, 0, s>>>(idx, (const int*)vals, m, w, (int*)acc,
                                                                      n_buckets, dev_status));
            break;
        }
        case GPA_SCATTER_ATOMIC: {
            const unsigned g = grid_for(m * w);
            if (dtype == 0)
                GPA_LAUNCH("scatter_atomic", s, scatter_atomic_kernel<float><<<g, 256, 0, s>>>(idx, (const float*)vals, m, w, (float*)acc, n_buckets,
                                                                dev_status));
            else
                GPA_LAUNCH("scatter_atomic", s, scatter_atomic_kernel<int><<<g, 256, 0, s>>>(idx, (const int*)vals, m, w, (int*)acc, n_buckets,
                                                              dev_status));
            break;
        }
        case GPA_SCATTER_WARPAGG: {
            const unsigned g = grid_for(m);
            if (dtype == 0)
                GPA_LAUNCH("scatter_warpagg", s, scatter_warpagg_kernel<float><<<g, 256, 0, s>>>(idx, (const float*)vals, m, w, (float*)acc,
                                                                 n_buckets, dev_status));
            else
                GPA_LAUNCH("scatter_warpagg", s, scatter_warpagg_kernel<int><<<g, 256, 0, s>>>(idx, (const int*)vals, m, w, (int*)acc, n_buckets,
                                                               dev_status));
            break;
        }
        case GPA_SCATTER_SORT: {
            if (!plan) return GPA_ERR_ARG;
            PlanView pv = plan_view(plan, m, n_buckets);
            const unsigned g = grid_for(m);
            if (dtype == 0)
                GPA_LAUNCH("scatter_sorted", s, scatter_sorted_kernel<float><<<g, 256, 0, s>>>(pv.perm, pv.key_sorted, (const float*)vals, m, w,
                                                                (float*)acc, n_buckets));
            else
                GPA_LAUNCH("scatter_sorted", s, scatter_sorted_kernel<int><<<g, 256, 0, s>>>(pv.perm, pv.key_sorted, (const int*)vals, m, w,
                                                              (int*)acc, n_buckets));
            break;
        }
        default:
            return GPA_ERR_ARG;
    }
    GPA_LAUNCH_CHECK();
    return GPA_OK;
}
