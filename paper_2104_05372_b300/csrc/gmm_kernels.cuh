// GMM FP32 kernel bodies shared by the per-call launches (gmm.cu) and the
// batched persistent kernels (gmm_batched.cu). Each __global__ kernel is a thin
// wrapper that passes its block index to the matching *_body device function.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "common.cuh"

namespace gpa {

// ---------------------------------------------------------------------------
// Configuration per padded dimension DP (16, 32, 64, 128)
// ---------------------------------------------------------------------------
template <int DP>
struct Fwd {
    static constexpr int NB = DP / 8;         // 8-row blocks of Q
    static constexpr int NWC = DP / 16;       // warps per component (pairs of row blocks)
    static constexpr int NS = 8 / NWC;        // components processed at once per CTA
    static constexpr int TP = 128;            // points per tile (4 per lane)
    static constexpr int XST = TP + 4;        // row stride of the transposed tile Xs[c][p]
    static constexpr int REC = DP * DP + DP + 4;  // staged record: Qt[c][r], b[r], cst, pad
    static constexpr int THREADS = 256;
    static constexpr size_t SMEM =
        sizeof(float) * (size_t)(DP * XST + 2 * NS * REC + 2 * NS * NWC * TP + 2 * NS * TP) + 64;
};

// Word offset of element c inside a point row of the backward tile: the two
// 16-byte halves of each 8-float chunk swap places when bit 2 of the chunk index
// is set, so that the chunks 8a.. read by the lanes of a warp spread over all
// 32 banks.
__host__ __device__ __forceinline__ int bwd_swz(int c) {
    const int a = c >> 3, h = (c >> 2) & 1;
    return (a << 3) + ((h ^ ((a >> 2) & 1)) << 2) + (c & 3);
}

template <int DP>
struct Bwd {
    static constexpr int NB = DP / 8;
    static constexpr int NOFF = NB * (NB - 1) / 2;     // strictly-lower 8x8 blocks
    static constexpr int NBLK = NB * (NB + 1) / 2;     // lower blocks incl. diagonal
    static constexpr int GC = DP == 16 ? 32 : DP == 32 ? 16 : DP == 64 ? 8 : 2;  // components per CTA
    static constexpr int NDIAG_T = GC * NB;            // threads on diagonal blocks
    static constexpr int NOFF_T = GC * NOFF;           // threads on off-diagonal blocks
    static constexpr int THREADS = ((NDIAG_T + NOFF_T + 31) / 32) * 32;
    static constexpr int TPB = 128;                    // points per tile
    static constexpr int XST = DP + 4;                 // row stride of Xs[p][c]
    // double-buffered: point tiles, raw log-joint and lse, and the cotangents r
    static constexpr size_t SMEM = sizeof(float) * (size_t)(2 * TPB * XST + 2 * GC * TPB + 2 * TPB + 2 * TPB * GC);
};

// ---------------------------------------------------------------------------
// A0: parameter expansion (one CTA per component)
// ---------------------------------------------------------------------------

template <int DP>
__device__ __forceinline__ void gmm_prep_kernel_body(const float* __restrict__ alpha,
                                                       const float* __restrict__ mu,
                                                       const float* __restrict__ q,
                                                       const float* __restrict__ l, int d, int k,
                                                       double gamma, int m, float* __restrict__ rec,
                                                       double* __restrict__ lpk,
                                                       double* __restrict__ scal, unsigned bx) {
    constexpr int REC = Fwd<DP>::REC;
    const int kk = bx;
    const int t = d * (d - 1) / 2;
    float* R = rec + (size_t)kk * REC;
    const float* qk = q + (size_t)kk * d;
    const float* lk = l + (size_t)kk * t;
    const float* muk = mu + (size_t)kk * d;
    // Q[r][c] from (q, l); zero above the diagonal and in the padding
    auto Qrc = [&](int r, int c) -> float {
        if (r >= d || c > r) return 0.f;
        return (c == r) ? expf(qk[r]) : lk[r * (r - 1) / 2 + c];
    };
    for (int e = threadIdx.x; e < DP * DP; e += blockDim.x) {
        const int c = e / DP, r = e % DP;
        R[e] = Qrc(r, c);  // transposed: Qt[c][r]
    }
    // b = Q mu: one warp per row, lanes over the row's columns (coalesced reads of l)
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int r = threadIdx.x >> 5; r < DP; r += nw) {
        double s = 0.0;
        if (r < d)
            for (int c = lane; c <= r; c += 32) s += (double)Qrc(r, c) * (double)muk[c];
        s = warp_sum(s);
        if (lane == 0) R[DP * DP + r] = (float)s;
    }
    // log-prior of this component and the constant alpha_k + sum_d q_kd
    const double nn = (double)(d + m + 1);
    double sq = 0.0, fro = 0.0, lg = 0.0;
    for (int r = threadIdx.x; r < d; r += blockDim.x) {
        const double qv = qk[r];
        sq += qv;
        fro += exp(2.0 * qv);
        lg += lgamma(0.5 * nn + 0.5 * (double)(-r));  // log Gamma_D(n/2) term j = r + 1
    }
    for (int j = threadIdx.x; j < t; j += blockDim.x) {
        const double lv = lk[j];
        fro += lv * lv;
    }
    // logsumexp(alpha) (used once, by component 0's block)
    double amax = -INFINITY;
    if (kk == 0)
        for (int i = threadIdx.x; i < k; i += blockDim.x) amax = fmax(amax, (double)alpha[i]);
    __shared__ double red[4][8];  // up to 256 threads
    sq = warp_sum(sq);
    fro = warp_sum(fro);
    lg = warp_sum(lg);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if (lane == 0) {
        red[0][threadIdx.x >> 5] = sq;
        red[1][threadIdx.x >> 5] = fro;
        red[2][threadIdx.x >> 5] = lg;
        red[3][threadIdx.x >> 5] = amax;
    }
    __syncthreads();
    double mx = -INFINITY;
    for (int w = 0; w < nw; ++w) mx = fmax(mx, red[3][w]);
    double ae = 0.0;
    if (kk == 0)
        for (int i = threadIdx.x; i < k; i += blockDim.x) ae += exp((double)alpha[i] - mx);
    ae = warp_sum(ae);
    __syncthreads();  // everyone has read red[3]
    if (lane == 0) red[3][threadIdx.x >> 5] = ae;
    __syncthreads();
    if (threadIdx.x == 0) {
        sq = 0.0;
        fro = 0.0;
        lg = 0.0;
        ae = 0.0;
        for (int w = 0; w < nw; ++w) {
            sq += red[0][w];
            fro += red[1][w];
            lg += red[2][w];
            ae += red[3][w];
        }
        R[DP * DP + DP] = (float)((double)alpha[kk] + sq);
        R[DP * DP + DP + 1] = 0.f;
        R[DP * DP + DP + 2] = 0.f;
        R[DP * DP + DP + 3] = 0.f;
        const double log_mvg = 0.25 * d * (d - 1) * log(3.14159265358979323846) + lg;
        const double cw = nn * d * log(gamma) - 0.5 * nn * d * log(2.0) - log_mvg;
        lpk[kk] = (double)m * sq - 0.5 * gamma * gamma * fro + cw;
        if (kk == 0) scal[0] = mx + log(ae);
    }
}

template <int DP>
__global__ void __launch_bounds__(128) gmm_prep_kernel(const float* __restrict__ alpha,
                                                       const float* __restrict__ mu,
                                                       const float* __restrict__ q,
                                                       const float* __restrict__ l, int d, int k,
                                                       double gamma, int m, float* __restrict__ rec,
                                                       double* __restrict__ lpk,
                                                       double* __restrict__ scal) {
    gmm_prep_kernel_body<DP>(alpha, mu, q, l, d, k, gamma, m, rec, lpk, scal, blockIdx.x);
}

// ---------------------------------------------------------------------------
// A1: forward log-joint and per-point logsumexp
// ---------------------------------------------------------------------------
// Z tile for one component: warp `wl` of the component owns row blocks rb0 = wl
// and rb1 = NB-1-wl (so every warp does the same work on the triangle), lane
// owns points 4*lane .. 4*lane+3. Row r needs c <= r only. The accumulators
// are packed float32 pairs along Q's rows: the operand pairs of Q come straight
// from the 16-byte loads and only the four point values need a broadcast per
// step, so 32 packed FMAs (each two float32 FMAs, rounded as the scalar
// instruction would) do the work of 64 scalar ones.
template <int DP>
__device__ __forceinline__ void fwd_gemm_packed(const float* __restrict__ Xs, const float* __restrict__ Q,
                                                int lane, int wl, float (&acc)[4][16]) {
    constexpr int NB = Fwd<DP>::NB, XST = Fwd<DP>::XST;
    const int rb0 = wl, rb1 = NB - 1 - wl;
    const int ce0 = 8 * (rb0 + 1), ce1 = 8 * (rb1 + 1);
    f2_t a2[4][8];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 8; ++i) a2[j][i] = 0ull;
    const float* xp = Xs + lane * 4;
    const float* qa = Q + rb0 * 8;
    const float* qb = Q + rb1 * 8;
    int c = 0;
#pragma unroll 2
    for (; c < ce0; ++c) {
        const float4 xv = *reinterpret_cast<const float4*>(xp + c * XST);
        const float4 a0 = *reinterpret_cast<const float4*>(qa + c * DP);
        const float4 a1 = *reinterpret_cast<const float4*>(qa + c * DP + 4);
        const float4 b0 = *reinterpret_cast<const float4*>(qb + c * DP);
        const float4 b1 = *reinterpret_cast<const float4*>(qb + c * DP + 4);
        const f2_t qs[8] = {f2_pack(a0.x, a0.y), f2_pack(a0.z, a0.w), f2_pack(a1.x, a1.y), f2_pack(a1.z, a1.w),
                            f2_pack(b0.x, b0.y), f2_pack(b0.z, b0.w), f2_pack(b1.x, b1.y), f2_pack(b1.z, b1.w)};
        const float xs[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const f2_t xb = f2_bcast(xs[j]);
#pragma unroll
            for (int i = 0; i < 8; ++i) a2[j][i] = f2_fma(xb, qs[i], a2[j][i]);
        }
    }
#pragma unroll 2
    for (; c < ce1; ++c) {
        const float4 xv = *reinterpret_cast<const float4*>(xp + c * XST);
        const float4 b0 = *reinterpret_cast<const float4*>(qb + c * DP);
        const float4 b1 = *reinterpret_cast<const float4*>(qb + c * DP + 4);
        const f2_t qs[4] = {f2_pack(b0.x, b0.y), f2_pack(b0.z, b0.w), f2_pack(b1.x, b1.y), f2_pack(b1.z, b1.w)};
        const float xs[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const f2_t xb = f2_bcast(xs[j]);
#pragma unroll
            for (int i = 0; i < 4; ++i) a2[j][4 + i] = f2_fma(xb, qs[i], a2[j][4 + i]);
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float2 v = f2_unpack(a2[j][i]);
            acc[j][2 * i] = v.x;
            acc[j][2 * i + 1] = v.y;
        }
}

// One CTA per tile of 128 points. x, lj, lse are chunk-local; the objective
// partial of this tile goes to part[tile0 + blockIdx.x].
template <int DP>
__device__ __forceinline__ void gmm_fwd_kernel_body(const float* __restrict__ x, int64_t n, int d, int k,
                   const float* __restrict__ rec, float* __restrict__ lj, int64_t lj_ld,
                   float* __restrict__ lse_out, double* __restrict__ part, int64_t tile0,
                   int32_t* __restrict__ status, unsigned bx) {
    using C = Fwd<DP>;
    constexpr int TP = C::TP, XST = C::XST, NS = C::NS, NWC = C::NWC, REC = C::REC;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* Xs = reinterpret_cast<float*>(smem_raw);     // [DP][XST]
    float* Qb = Xs + DP * XST;                           // [2][NS][REC]
    float* red = Qb + 2 * NS * REC;                      // [2][NS][NWC][TP]
    float* st = red + 2 * NS * NWC * TP;                 // [NS][TP][2]
    uint64_t* bar = reinterpret_cast<uint64_t*>(st + 2 * NS * TP);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int slot = warp / NWC, wl = warp % NWC;
    const int64_t p0 = (int64_t)bx * TP;
    const int nvalid = (int)min64(TP, n - p0);
    const int rounds = (k + NS - 1) / NS;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    // transposed, zero-padded point tile
    for (int e = tid; e < DP * XST; e += C::THREADS) Xs[e] = 0.f;
    __syncthreads();
    for (int e = tid; e < nvalid * d; e += C::THREADS) {
        const int p = e / d, c = e - p * d;
        Xs[c * XST + p] = __ldg(x + (p0 + p) * d + c);
    }
    auto issue = [&](int round) {
        const int buf = round & 1;
        int nb = 0;
        for (int s = 0; s < NS; ++s) nb += (round * NS + s < k) ? 1 : 0;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bar[buf], (uint32_t)(nb * REC * sizeof(float)));
        for (int s = 0; s < NS; ++s) {
            const int kk = round * NS + s;
            if (kk < k) bulk_g2s(Qb + (buf * NS + s) * REC, rec + (size_t)kk * REC, REC * sizeof(float), &bar[buf]);
        }
    };
    if (tid == 0) issue(0);

    // online logsumexp states: this thread owns pairs e = tid + 256*u of (slot, point)
    constexpr int NPAIR = (NS * TP + C::THREADS - 1) / C::THREADS;
    Lse ls[NPAIR];
#pragma unroll
    for (int u = 0; u < NPAIR; ++u) ls[u].init();

    bool ok = true;
    int last_issued = 0;  // highest round whose copies were issued (thread 0)
    for (int round = 0; round < rounds; ++round) {
        const int buf = round & 1;
        if (tid == 0 && round + 1 < rounds) {
            issue(round + 1);
            last_issued = round + 1;
        }
        ok = mbar_wait(&bar[buf], (round >> 1) & 1, status) && ok;
        ok = __syncthreads_and(ok);  // Xs ready (round 0); all threads agree on ok
        if (!ok) break;
        const int kk = round * NS + slot;
        float* redb = red + buf * NS * NWC * TP;
        if (kk < k) {
            const float* Q = Qb + (buf * NS + slot) * REC;
            float acc[4][16];
            fwd_gemm_packed<DP>(Xs, Q, lane, wl, acc);
            const int rb0 = wl, rb1 = C::NB - 1 - wl;
            float bv[16];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                bv[i] = Q[DP * DP + rb0 * 8 + i];
                bv[8 + i] = Q[DP * DP + rb1 * 8 + i];
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float s2 = 0.f;
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float z = acc[j][i] - bv[i];
                    s2 = fmaf(z, z, s2);
                }
                redb[(slot * NWC + wl) * TP + lane * 4 + j] = s2;
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < NPAIR; ++u) {
            const int e = tid + u * C::THREADS;
            if (e < NS * TP) {
                const int s = e / TP, p = e % TP;
                const int kc = round * NS + s;
                if (kc < k) {
                    float tot = 0.f;
#pragma unroll
                    for (int w = 0; w < NWC; ++w) tot += redb[(s * NWC + w) * TP + p];
                    const float sv = __ldg(rec + (size_t)kc * REC + DP * DP + DP) - 0.5f * tot;
                    if (p < nvalid) {
                        if (lj) lj[(int64_t)kc * lj_ld + p0 + p] = sv;
                        ls[u].add(sv);
                    }
                }
            }
        }
    }
    if (!ok && tid == 0) {
        // a wait gave up: let this CTA's copies in flight land (bounded) before exiting
        (void)mbar_wait(&bar[last_issued & 1], (last_issued >> 1) & 1, status);
        (void)mbar_wait(&bar[(last_issued + 1) & 1], ((last_issued - 1) >> 1) & 1, status);
    }
    // merge the slots' states per point; sum lse over the tile in float64
#pragma unroll
    for (int u = 0; u < NPAIR; ++u) {
        const int e = tid + u * C::THREADS;
        if (e < NS * TP) {
            st[2 * e] = ls[u].m;
            st[2 * e + 1] = ls[u].l;
        }
    }
    __syncthreads();
    double v = 0.0;
    if (tid < TP) {
        Lse a;
        a.init();
        for (int s = 0; s < NS; ++s) a.merge(st[2 * (s * TP + tid)], st[2 * (s * TP + tid) + 1]);
        if (tid < nvalid) {
            const float lv = a.value();
            if (lse_out) lse_out[p0 + tid] = lv;
            v = (double)lv;
        }
    }
    __shared__ double wsum[8];
    v = warp_sum(v);
    if (lane == 0) wsum[warp] = v;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += wsum[w];
        part[tile0 + bx] = ok ? s : NAN;
    }
}

template <int DP>
__global__ void __launch_bounds__(256, (DP <= 64 ? 2 : 1))
    gmm_fwd_kernel(const float* __restrict__ x, int64_t n, int d, int k,
                   const float* __restrict__ rec, float* __restrict__ lj, int64_t lj_ld,
                   float* __restrict__ lse_out, double* __restrict__ part, int64_t tile0,
                   int32_t* __restrict__ status) {
    gmm_fwd_kernel_body<DP>(x, n, d, k, rec, lj, lj_ld, lse_out, part, tile0, status, blockIdx.x);
}

// Sum of a given lse vector per 128-point tile (objective from a saved lse).
static __global__ void __launch_bounds__(128) gmm_lse_sum_kernel(const float* __restrict__ lse, int64_t n,
                                                          double* __restrict__ part) {
    const int64_t i = (int64_t)blockIdx.x * 128 + threadIdx.x;
    double v = i < n ? (double)lse[i] : 0.0;
    __shared__ double w[4];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) part[blockIdx.x] = w[0] + w[1] + w[2] + w[3];
}

// Objective = sum of tile partials (fixed order) + prior - N lse(alpha) - N D/2 log 2pi.
__device__ __forceinline__ void gmm_objective_finalize_kernel_body(
    const double* __restrict__ part, int64_t ntiles, const double* __restrict__ lpk, int k,
    const double* __restrict__ scal, int64_t n, int d, double* __restrict__ out, unsigned bx) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int64_t t = threadIdx.x; t < ntiles; t += 256) s += part[t];
    for (int64_t t = threadIdx.x; t < k; t += 256) s += lpk[t];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        *out = sh[0] - (double)n * scal[0] - 0.5 * (double)n * d * log(2.0 * 3.14159265358979323846);
}

static __global__ void __launch_bounds__(256) gmm_objective_finalize_kernel(
    const double* __restrict__ part, int64_t ntiles, const double* __restrict__ lpk, int k,
    const double* __restrict__ scal, int64_t n, int d, double* __restrict__ out) {
    gmm_objective_finalize_kernel_body(part, ntiles, lpk, k, scal, n, d, out, blockIdx.x);
}

// ---------------------------------------------------------------------------
// A2: backward Accum of R_k, m_k, S_k (lower 8x8 blocks) per component
// ---------------------------------------------------------------------------
// grid (component groups, point chunks). Diagonal-block threads fill warps of
// their own (they also accumulate m and R); off-diagonal threads fill the rest.
template <int DP>
__device__ __forceinline__ void gmm_bwd_kernel_body(const float* __restrict__ x, int64_t n, int d, int k,
                   const float* __restrict__ lj, int64_t lj_ld, const float* __restrict__ lse,
                   float seed, int64_t tiles_per_chunk, float* __restrict__ partS,
                   float* __restrict__ partM, unsigned bx, unsigned by) {
    using C = Bwd<DP>;
    constexpr int TPB = C::TPB, XST = C::XST, GC = C::GC, NB = C::NB, NBLK = C::NBLK;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* Xs = reinterpret_cast<float*>(smem_raw);  // [2][TPB][XST]
    float* rawlj = Xs + 2 * TPB * XST;                // [2][GC][TPB]
    float* rawlse = rawlj + 2 * GC * TPB;             // [2][TPB]
    float* rs = rawlse + 2 * TPB;                     // [2][TPB][GC]
    const int tid = threadIdx.x;
    const int kg0 = bx * GC;
    const int64_t ntiles = (n + TPB - 1) / TPB;
    const int64_t t_begin = (int64_t)by * tiles_per_chunk;
    const int64_t t_end = min64(ntiles, t_begin + tiles_per_chunk);

    // role of this thread
    const bool diag = tid < C::NDIAG_T;
    int kk, a, b;
    if (diag) {
        kk = tid / NB;
        a = b = tid % NB;
    } else {
        const int u = tid - C::NDIAG_T;
        kk = u / (C::NOFF > 0 ? C::NOFF : 1);
        int o = u - kk * C::NOFF;
        a = 1;
        while (o >= a) {
            o -= a;
            ++a;
        }
        b = o;
    }
    const bool active = (tid < C::NDIAG_T + C::NOFF_T) && (kg0 + kk < k);

    // Pipeline. The diagonal-block threads (whole warps, NDIAG_T of them) do
    // less arithmetic per point than the off-diagonal ones, so they also carry
    // the per-tile side work while the others accumulate: they copy the next
    // tile's log-joint and lse columns (cp.async, so their own wait covers
    // them) and turn them into the cotangents r. Every thread copies its share
    // of the next point tile. One block barrier per tile.
    constexpr int ND = C::NDIAG_T;
    auto issue_x = [&](int64_t t, int buf) {
        const int64_t p0 = t * TPB;
        const int nv = (int)min64(TPB, n - p0);
        float* X = Xs + buf * TPB * XST;
        for (int e = tid; e < nv * d; e += C::THREADS) {
            const int p = e / d, c = e - p * d;
            cp_async4(X + p * XST + bwd_swz(c), x + (p0 + p) * d + c);
        }
    };
    auto issue_lj = [&](int64_t t, int buf) {  // diagonal threads only
        const int64_t p0 = t * TPB;
        const int nv = (int)min64(TPB, n - p0);
        float* L = rawlj + buf * GC * TPB;
        for (int e = tid; e < GC * TPB; e += ND) {
            const int kc = e / TPB, p = e % TPB;
            if (p < nv && kg0 + kc < k) cp_async4(L + e, lj + (int64_t)(kg0 + kc) * lj_ld + p0 + p);
        }
        float* S = rawlse + buf * TPB;
        for (int p = tid; p < nv; p += ND) cp_async4(S + p, lse + p0 + p);
    };
    // cotangents r = seed exp(s - lse) of tile t from buffer buf; 0 on the ragged tail
    auto make_r = [&](int64_t t, int buf) {  // diagonal threads only
        const int64_t p0 = t * TPB;
        const int nv = (int)min64(TPB, n - p0);
        const float* L = rawlj + buf * GC * TPB;
        const float* S = rawlse + buf * TPB;
        float* R = rs + buf * TPB * GC;
        for (int e = tid; e < GC * TPB; e += ND) {
            const int kc = e / TPB, p = e % TPB;
            float r = 0.f;
            if (p < nv && kg0 + kc < k) r = seed * expf(L[e] - S[p]);
            R[p * GC + kc] = r;
        }
    };
    auto diag_sync = [] { asm volatile("bar.sync 2, %0;" ::"n"(ND) : "memory"); };

    for (int e = tid; e < 2 * TPB * XST; e += C::THREADS) Xs[e] = 0.f;
    __syncthreads();

    float acc[8][8];
    float macc[8];
    float racc = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        macc[i] = 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    }

    // prologue: tile t_begin in shared memory with its r, tile t_begin+1 in flight
    if (t_begin < t_end) {
        issue_x(t_begin, 0);
        if (diag) issue_lj(t_begin, 0);
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    if (diag && t_begin < t_end) make_r(t_begin, 0);
    if (t_begin + 1 < t_end) {
        issue_x(t_begin + 1, 1);
        if (diag) issue_lj(t_begin + 1, 1);
    }
    cp_async_commit();
    __syncthreads();

    for (int64_t t = t_begin; t < t_end; ++t) {
        const int buf = (int)((t - t_begin) & 1);
        if (active) {
            const float* Xb = Xs + buf * TPB * XST;
            const float* rb = rs + buf * TPB * GC;
            // halves of the chunks in swizzled order (see bwd_swz)
            const float* xa = Xb + 8 * a;
            const float* xb = Xb + 8 * b;
            const int ha = ((a >> 2) & 1) << 2, hb = ((b >> 2) & 1) << 2;
            if (diag) {
#pragma unroll 2
                for (int p = 0; p < TPB; ++p) {
                    const float4 a0 = *reinterpret_cast<const float4*>(xa + p * XST + ha);
                    const float4 a1 = *reinterpret_cast<const float4*>(xa + p * XST + (4 ^ ha));
                    const float rr = rb[p * GC + kk];
                    const float xv[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                    float ya[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) ya[i] = rr * xv[i];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        macc[i] += ya[i];
#pragma unroll
                        for (int j = 0; j <= i; ++j) acc[i][j] = fmaf(ya[i], xv[j], acc[i][j]);
                    }
                    racc += rr;
                }
            } else {
#pragma unroll 1
                for (int p = 0; p < TPB; ++p) {
                    const float4 b0 = *reinterpret_cast<const float4*>(xb + p * XST + hb);
                    const float4 b1 = *reinterpret_cast<const float4*>(xb + p * XST + (4 ^ hb));
                    const float rr = rb[p * GC + kk];
                    const float yv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float4 av = *reinterpret_cast<const float4*>(xa + p * XST + ((4 * h) ^ ha));
                        const float xv[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float ya = rr * xv[i];
#pragma unroll
                            for (int j = 0; j < 8; ++j) acc[4 * h + i][j] = fmaf(ya, yv[j], acc[4 * h + i][j]);
                        }
                    }
                }
            }
        }
        cp_async_wait_all();  // this thread's copies of tile t+1 have landed
        if (diag && t + 1 < t_end) {
            diag_sync();          // every diagonal thread's log-joint copies of tile t+1 are visible
            make_r(t + 1, buf ^ 1);
        }
        __syncthreads();      // tile t+1 and its r complete; nobody reads buffer `buf` any more
        if (t + 2 < t_end) {
            issue_x(t + 2, buf);
            if (diag) issue_lj(t + 2, buf);
        }
        cp_async_commit();
    }
    if (!active) return;
    const int kg = kg0 + kk;
    const int64_t base = ((int64_t)by * k + kg);
    float* S = partS + base * NBLK * 64 + (int64_t)(a * (a + 1) / 2 + b) * 64;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (!diag || j <= i) S[i * 8 + j] += acc[i][j];
    if (diag) {
        float* M = partM + base * (DP + 1);
#pragma unroll
        for (int i = 0; i < 8; ++i) M[8 * a + i] += macc[i];
        if (a == 0) M[DP] += racc;
    }
}

template <int DP>
__global__ void __launch_bounds__(Bwd<DP>::THREADS) __maxnreg__(DP == 64 ? 96 : 168)
    gmm_bwd_kernel(const float* __restrict__ x, int64_t n, int d, int k,
                   const float* __restrict__ lj, int64_t lj_ld, const float* __restrict__ lse,
                   float seed, int64_t tiles_per_chunk, float* __restrict__ partS,
                   float* __restrict__ partM) {
    gmm_bwd_kernel_body<DP>(x, n, d, k, lj, lj_ld, lse, seed, tiles_per_chunk, partS, partM, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// A3: finalize gradients per component (fixed-order sums over chunks)
// ---------------------------------------------------------------------------
template <int DP>
__device__ __forceinline__ void gmm_finalize_kernel_body(
    const float* __restrict__ alpha, const float* __restrict__ mu, const float* __restrict__ q,
    const float* __restrict__ l, int d, int k, int64_t n, double gamma, int m, double seed,
    const float* __restrict__ partS, const float* __restrict__ partM, int nchunks,
    const double* __restrict__ scal, float* __restrict__ d_alpha, float* __restrict__ d_mu,
    float* __restrict__ d_q, float* __restrict__ d_l, int centered, const double* __restrict__ exch,
    unsigned bx) {
    // centered: the partials hold sum r (x - mu)(x - mu)^T and sum r (x - mu)
    // (tensor-core path) instead of the raw moments S and m.
    // exch: when given, the sums come from an exchange vector (float64, already
    // combined over chunks and shards) instead of the chunk partials.
    constexpr int NBLK = Bwd<DP>::NBLK;
    constexpr int E = NBLK * 64 + DP + 1;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    double* Sd = reinterpret_cast<double*>(smem_raw);  // [NBLK*64]
    double* md = Sd + NBLK * 64;                         // [DP+1]
    double* vd = md + DP + 1;                            // [DP]  Q (m - R mu)
    double* mud = vd + DP;                               // [DP]
    float* Cf = reinterpret_cast<float*>(mud + DP);      // [DP][DP] symmetric
    float* Qf = Cf + DP * DP;                            // [DP][DP] lower
    const int kk = bx, tid = threadIdx.x;
    const int t = d * (d - 1) / 2;
    const float* qk = q + (size_t)kk * d;
    const float* lk = l + (size_t)kk * t;

    if (exch) {
        for (int e = tid; e < NBLK * 64; e += 256) Sd[e] = exch[(size_t)kk * E + e];
        for (int e = tid; e < DP + 1; e += 256) md[e] = exch[(size_t)kk * E + NBLK * 64 + e];
    } else {
        for (int e = tid; e < NBLK * 64; e += 256) {
            double s = 0.0;
            for (int c = 0; c < nchunks; ++c) s += partS[((int64_t)c * k + kk) * NBLK * 64 + e];
            Sd[e] = s;
        }
        for (int e = tid; e < DP + 1; e += 256) {
            double s = 0.0;
            for (int c = 0; c < nchunks; ++c) s += partM[((int64_t)c * k + kk) * (DP + 1) + e];
            md[e] = s;
        }
    }
    for (int e = tid; e < DP * DP; e += 256) {
        const int r = e / DP, c = e % DP;
        float v = 0.f;
        if (r < d && c <= r) v = (c == r) ? expf(qk[r]) : lk[r * (r - 1) / 2 + c];
        Qf[e] = v;
    }
    for (int e = tid; e < DP; e += 256) mud[e] = e < d ? (double)mu[(size_t)kk * d + e] : 0.0;
    __syncthreads();
    const double R = md[DP];
    for (int e = tid; e < DP * DP; e += 256) {
        const int a = e / DP, b = e % DP;
        if (b > a) continue;
        double c = 0.0;
        if (a < d) {
            const int A = a >> 3, B = b >> 3;
            const double S = Sd[(A * (A + 1) / 2 + B) * 64 + (a & 7) * 8 + (b & 7)];
            c = centered ? S : S - mud[a] * md[b] - md[a] * mud[b] + R * mud[a] * mud[b];
        }
        Cf[a * DP + b] = (float)c;
        Cf[b * DP + a] = (float)c;
    }
    for (int r = tid; r < DP; r += 256) {
        double v = 0.0;
        if (r < d)
            for (int j = 0; j <= r; ++j) v += (double)Qf[r * DP + j] * (centered ? md[j] : md[j] - R * mud[j]);
        vd[r] = v;
    }
    __syncthreads();
    // H = Q C on the lower triangle; dq from its diagonal, dl from the rest
    const int ne = d * (d + 1) / 2;
    for (int e = tid; e < ne; e += 256) {
        int r = (int)((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);
        while (r * (r + 1) / 2 > e) --r;
        while ((r + 1) * (r + 2) / 2 <= e) ++r;
        const int c = e - r * (r + 1) / 2;
        float h = 0.f;
        for (int j = 0; j <= r; ++j) h = fmaf(Qf[r * DP + j], Cf[j * DP + c], h);
        if (c == r) {
            const double ev = exp((double)qk[r]);
            d_q[(size_t)kk * d + r] += (float)(R - ev * (double)h + seed * ((double)m - gamma * gamma * ev * ev));
        } else {
            const int li = r * (r - 1) / 2 + c;
            d_l[(size_t)kk * t + li] += (float)(-(double)h - seed * gamma * gamma * (double)lk[li]);
        }
    }
    for (int c = tid; c < d; c += 256) {
        double s = 0.0;
        for (int r = c; r < d; ++r) s += (double)Qf[r * DP + c] * vd[r];
        d_mu[(size_t)kk * d + c] += (float)s;
    }
    if (tid == 0) d_alpha[kk] += (float)(R - seed * (double)n * exp((double)alpha[kk] - scal[0]));
}

template <int DP>
__global__ void __launch_bounds__(256) gmm_finalize_kernel(
    const float* __restrict__ alpha, const float* __restrict__ mu, const float* __restrict__ q,
    const float* __restrict__ l, int d, int k, int64_t n, double gamma, int m, double seed,
    const float* __restrict__ partS, const float* __restrict__ partM, int nchunks,
    const double* __restrict__ scal, float* __restrict__ d_alpha, float* __restrict__ d_mu,
    float* __restrict__ d_q, float* __restrict__ d_l, int centered, const double* __restrict__ exch) {
    gmm_finalize_kernel_body<DP>(alpha, mu, q, l, d, k, n, gamma, m, seed, partS, partM, nchunks, scal, d_alpha,
                                 d_mu, d_q, d_l, centered, exch, blockIdx.x);
}

// Exchange vector of one shard of points: per component the chunk partial sums
// [S blocks | m | R] combined in chunk order in float64, then the sum of the
// shard's per-point logsumexp (tile partials in tile order), added (+=) into
// exch. Sums of these vectors over shards are the Accum sums of all points
// (Sec. 2.3.2).
template <int DP>
__global__ void __launch_bounds__(256) gmm_exchange_kernel(const float* __restrict__ partS,
                                                           const float* __restrict__ partM, int nchunks, int k,
                                                           const double* __restrict__ fwd_part, int64_t ntiles,
                                                           double* __restrict__ exch) {
    // grid (k + 1, ceil(E / 256)): one entry per thread, its chunks summed in order
    constexpr int NS = Bwd<DP>::NBLK * 64, E = NS + DP + 1;
    const int kk = blockIdx.x;
    if (kk < k) {
        const int e = blockIdx.y * 256 + threadIdx.x;
        if (e < NS) {
            double s = 0.0;
            for (int c = 0; c < nchunks; ++c) s += partS[((int64_t)c * k + kk) * NS + e];
            exch[(size_t)kk * E + e] += s;
        } else if (e < E) {
            double s = 0.0;
            for (int c = 0; c < nchunks; ++c) s += partM[((int64_t)c * k + kk) * (DP + 1) + (e - NS)];
            exch[(size_t)kk * E + e] += s;
        }
        return;
    }
    if (blockIdx.y != 0) return;
    __shared__ double sh[256];
    double s = 0.0;
    for (int64_t t = threadIdx.x; t < ntiles; t += 256) s += fwd_part[t];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) exch[(size_t)k * E] += sh[0];
}


}  // namespace gpa
