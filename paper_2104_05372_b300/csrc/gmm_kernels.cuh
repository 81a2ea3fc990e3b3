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
// Configuration per padded dimension DP (16, 32, 64, 128; the batched form
// also has a class DP = 8 with kernels of its own, sharing only REC and NBLK)
// ---------------------------------------------------------------------------
template <int DP>
struct Fwd {
    static constexpr int NB = DP / 8;         // 8-row blocks of Q
    static constexpr int NWC = DP >= 16 ? DP / 16 : 1;  // warps per component (pairs of row blocks)
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

// Backward layouts. Every thread owns one full 8x8 block (a, b), a >= b, of one
// component's S (or, on the diagonal of the block-per-warp layout, two
// diagonal blocks); the m and R sums are spread over the threads as MP extra
// packed FMAs per point and block (see bwd_mtask). GC components per CTA.
//   D <= 32 (WB false): consecutive threads take consecutive blocks of a
//     component and run one instruction stream (diagonal blocks accumulated in
//     full, their upper halves dropped at the write-out).
//   D > 32 (WB true, blocks per warp): lane l of a warp takes component l % GC
//     of the CTA on slot l / GC of the warp's BPW = 32 / GC slots, so that the
//     lanes reading one chunk of a point row form a contiguous group and each
//     16-byte shared load serves BPW distinct addresses (one wavefront, given
//     distinct bank groups: see bwd_pos). The first NDW warps hold the diagonal
//     blocks, two per lane ((q, q) and (NB-1-q, NB-1-q)), and skip their upper
//     halves; the other NOW warps hold one off-diagonal block per lane. The 16
//     warps (4 per scheduler) carry equal work except the diagonal warps'
//     one-third extra, spread over different schedulers.
// GCX (sequential layout only): components per CTA other than the default,
// for the batched form's small component groups (instances with few
// components, where a default group would leave most threads idle).
template <int DP, int GCX = 0>
struct Bwd {
    static constexpr int NB = DP / 8;
    static constexpr int NBLK = NB * (NB + 1) / 2;     // lower blocks incl. diagonal
    static constexpr bool WB = DP >= 64;
    static_assert(GCX == 0 || !WB, "small component groups: sequential layout only");
    static constexpr int GC = GCX ? GCX : DP == 16 ? 42 : DP == 32 ? 25 : DP == 64 ? 16 : 4;  // components per CTA
    static constexpr int BPW = WB ? 32 / GC : 0;                 // slots per warp (lanes per slot = GC)
    static constexpr int NDW = WB ? (NB / 2) * GC / 32 : 0;      // warps on pairs of diagonal blocks
    static constexpr int NOW = WB ? (NBLK - NB) * GC / 32 : 0;   // warps on off-diagonal blocks
    static_assert(!WB || ((NB / 2) * GC % 32 == 0 && (NBLK - NB) * GC % 32 == 0), "whole warps of blocks");
    // m / R tasks per thread on the off-diagonal warps of the schedulers
    // without a diagonal warp (3 NB + 1 tasks over their threads)
    static constexpr int NLIGHT = WB ? ((NDW + NOW) / 4) * (4 - NDW) * BPW : 1;
    static constexpr int MTL = WB ? (3 * NB + 1 + NLIGHT - 1) / NLIGHT : 0;
    static_assert(!WB || (MTL <= 2 && NDW < 4 && (NDW + NOW) % 4 == 0), "task split");
    static constexpr int TPB = DP == 16 ? 32 : DP == 32 ? 64 : 128;  // points per tile
    static constexpr int MP = NB == 2 ? 3 : NB == 4 ? 2 : 1;  // m / R pairs per thread and block
    static constexpr int NACT = GC * NBLK;               // threads with a block (sequential layout)
    static constexpr int THREADS = WB ? 32 * (NDW + NOW) : ((NACT + 31) / 32) * 32;
    // resident CTAs per SM: as many threads per SM as the default group has
    static constexpr int MINB_DEF = DP == 16 ? 3 : DP == 32 ? 2 : 1;
    static constexpr int MINB = GCX ? MINB_DEF * (Bwd<DP>::THREADS / THREADS) : MINB_DEF;
    static constexpr int XST = DP + 4;  // row stride of the point tiles; floats DP, DP+1 hold 1.0
    // point-loop unroll of the per-call kernel and of the persistent batched
    // kernel, as far as the register budget of MINB resident CTAs allows
    static constexpr int UNROLL = DP == 128 ? 2 : DP == 64 ? 8 : 4;
    // (4 at DP <= 32 measured 3-7 % faster than 2 in the 512-instance batch,
    // in spite of a few spilled registers)
    static constexpr int UNROLL_BATCHED = DP == 128 ? 1 : DP <= 32 ? 4 : 2;
    // point tiles double-buffered; raw log-joint, lse and the cotangents r
    // triple-buffered
    static constexpr size_t SMEM = sizeof(float) * (size_t)(2 * TPB * XST + 3 * GC * TPB + 3 * TPB + 3 * TPB * GC);
};

// Float offset of coordinate c in a point row of the block-per-warp tile: the
// 16-byte half h of chunk a (coordinates 8a + 4h .. 8a + 4h + 3) sits in
// 16-byte slot h * NB + a, i.e. in bank group a mod 8 for both halves. A warp
// reads half h of its blocks' chunks in one instruction; chunks that differ
// mod 8 never share a bank.
template <int NB>
__host__ __device__ __forceinline__ int bwd_pos(int c) {
    return (((((c >> 2) & 1) * NB) + (c >> 3)) << 2) + (c & 3);
}

// Off-diagonal blocks of the 16 x 16 block triangle (D = 128) in warp order,
// (a << 4) | b: eight per warp, chosen (by a search over groupings) so that the
// distinct row chunks a of a warp differ mod 8, and so do its column chunks b.
__device__ __constant__ const unsigned char kOffBlocks16[120] = {
    0x32, 0x80, 0xa3, 0xa5, 0xa9, 0xe9, 0xf7, 0xfe,  0x81, 0x90, 0xb1, 0xb3, 0xc7, 0xd1, 0xd7, 0xfa,
    0x76, 0x82, 0x95, 0xb7, 0xc8, 0xc9, 0xd8, 0xeb,  0x20, 0x43, 0x51, 0xe3, 0xea, 0xed, 0xf1, 0xf3,
    0x61, 0x65, 0x73, 0x86, 0x98, 0xb8, 0xba, 0xda,  0x70, 0x72, 0x85, 0xb2, 0xb4, 0xc6, 0xcb, 0xd2,
    0x31, 0x52, 0xe5, 0xf2, 0xf5, 0xf8, 0xfb, 0xfc,  0x10, 0x40, 0x53, 0xa0, 0xb6, 0xe0, 0xf0, 0xf9,
    0x97, 0xa2, 0xb0, 0xc1, 0xd0, 0xd4, 0xd5, 0xdb,  0x21, 0x50, 0x60, 0x63, 0x93, 0xb5, 0xca, 0xf4,
    0x42, 0x74, 0x75, 0x96, 0xa7, 0xe2, 0xe6, 0xe8,  0x62, 0x64, 0xa6, 0xc2, 0xc4, 0xc5, 0xd3, 0xd9,
    0x41, 0x83, 0x84, 0x94, 0xa4, 0xe1, 0xe4, 0xfd,  0x54, 0x87, 0x92, 0xa8, 0xb9, 0xc3, 0xe7, 0xf6,
    0x30, 0x71, 0x91, 0xa1, 0xc0, 0xd6, 0xdc, 0xec};

// Off-diagonal block o (0 <= o < NB(NB-1)/2) of the block-per-warp layout.
template <int NB>
__device__ __forceinline__ void bwd_off_block(int o, int& a, int& b) {
    if constexpr (NB == 16) {
        const int v = kOffBlocks16[o];
        a = v >> 4;
        b = v & 15;
    } else {  // NB <= 8: every chunk index differs mod 8 anyway
        a = 1;
        b = o;
        while (b >= a) {
            b -= a;
            ++a;
        }
    }
}

// The m / R task of slot s of the thread on block (a, b): the natural
// coordinate index 2j of the pair (m_2j, m_2j+1) it accumulates, DP for R
// (operand: the constant 1.0 pair at the end of each tile row), or -1 (no task).
// Each of the 4 NB pairs of m and R goes to exactly one (block, slot) whose
// row or column chunk holds the pair:
//   NB >= 8: pair (c, 0) on (c, c); pair (c, s), s = 1..3, on the block of
//            chunks {c, c + s mod NB}; R on (4, 0);
//   NB == 4, NB == 2: the tables below.
template <int NB>
__host__ __device__ __forceinline__ int bwd_mtask(int a, int b, int s) {
    if constexpr (NB >= 8) {
        if (s != 0) return -1;
        if (a == b) return 8 * a;
        if (a == 4 && b == 0) return 8 * NB;
        const int s1 = a - b, s2 = NB - s1;
        if (s1 <= 3) return 8 * b + 2 * s1;
        if (s2 <= 3) return 8 * a + 2 * s2;
        return -1;
    } else if constexpr (NB == 4) {
        if (a == b) return s < 2 ? 8 * a + 2 * s : -1;
        const int blk = a * (a + 1) / 2 + b;  // (1,0)=1 (2,0)=3 (2,1)=4 (3,0)=6 (3,1)=7 (3,2)=8
        switch (blk) {
            case 1: return s == 0 ? 4 : s == 1 ? 32 : -1;
            case 3: return s == 0 ? 6 : s == 1 ? 22 : -1;
            case 4: return s == 0 ? 12 : -1;
            case 6: return s == 0 ? 28 : -1;
            case 7: return s == 0 ? 14 : s == 1 ? 30 : -1;
            case 8: return s == 0 ? 20 : -1;
            default: return -1;
        }
    } else {
        static_assert(NB == 2, "padded dimension 16, 32, 64 or 128");
        if (a == b) return s < 3 ? 8 * a + 2 * s : -1;
        return s == 0 ? 6 : s == 1 ? 14 : s == 2 ? 16 : -1;
    }
}

// ---------------------------------------------------------------------------
// A0: parameter expansion (one CTA per component)
// ---------------------------------------------------------------------------

template <int DP>
__device__ __forceinline__ void gmm_prep_kernel_body(const float* __restrict__ alpha,
                                                       const float* __restrict__ mu,
                                                       const float* __restrict__ q,
                                                       const float* __restrict__ l, int d, int k,
                                                       double gamma, int m, double cw, float* __restrict__ rec,
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
    // b = Q mu: one warp per row, lanes over the row's columns (coalesced reads
    // of l). Compensated float32 dot product (Dot2 of Ogita, Rump and Oishi:
    // exact products by FMA, TwoSum accumulation, pairs merged across lanes by
    // TwoSum), as accurate as a float64 sum before the final rounding to float.
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    auto two_sum_acc = [](float& hi, float& lo, float x) {
        const float t = __fadd_rn(hi, x);
        const float bb = __fsub_rn(t, hi);
        lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bb)), __fsub_rn(x, bb)));
        hi = t;
    };
    for (int r = threadIdx.x >> 5; r < DP; r += nw) {
        float hi = 0.f, lo = 0.f;
        if (r < d)
            for (int c = lane; c <= r; c += 32) {
                const float a = Qrc(r, c), b = muk[c];
                const float p = __fmul_rn(a, b);
                two_sum_acc(hi, lo, p);
                lo = __fadd_rn(lo, fmaf(a, b, -p));
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
            const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
            two_sum_acc(hi, lo, h2);
            lo = __fadd_rn(lo, l2);
        }
        if (lane == 0) R[DP * DP + r] = __fadd_rn(hi, lo);
    }
    // log-prior of this component and the constant alpha_k + sum_d q_kd
    double sq = 0.0, fro = 0.0;
    for (int r = threadIdx.x; r < d; r += blockDim.x) {
        const double qv = qk[r];
        sq += qv;
        fro += exp(2.0 * qv);
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
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if (lane == 0) {
        red[0][threadIdx.x >> 5] = sq;
        red[1][threadIdx.x >> 5] = fro;
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
        ae = 0.0;
        for (int w = 0; w < nw; ++w) {
            sq += red[0][w];
            fro += red[1][w];
            ae += red[3][w];
        }
        R[DP * DP + DP] = (float)((double)alpha[kk] + sq);
        R[DP * DP + DP + 1] = 0.f;
        R[DP * DP + DP + 2] = 0.f;
        R[DP * DP + DP + 3] = 0.f;
        lpk[kk] = (double)m * sq - 0.5 * gamma * gamma * fro + cw;  // cw: gmm_prior_const
        if (kk == 0) scal[0] = mx + log(ae);
    }
}

template <int DP>
__global__ void __launch_bounds__(128) gmm_prep_kernel(const float* __restrict__ alpha,
                                                       const float* __restrict__ mu,
                                                       const float* __restrict__ q,
                                                       const float* __restrict__ l, int d, int k,
                                                       double gamma, int m, double cw,
                                                       float* __restrict__ rec, double* __restrict__ lpk,
                                                       double* __restrict__ scal) {
    gmm_prep_kernel_body<DP>(alpha, mu, q, l, d, k, gamma, m, cw, rec, lpk, scal, blockIdx.x);
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
// instruction would) do the work of 64 scalar ones. The accumulators start at
// -b (the record's b = Q mu), so z = Q x - b comes out directly:
// z2[j][i] = (z_{r0}, z_{r0+1}) of point j for rows r0 = 8 rb0 + 2i (i < 4) and
// 8 rb1 + 2(i - 4) (i >= 4).
template <int DP>
__device__ __forceinline__ void fwd_gemm_packed(const float* __restrict__ Xs, const float* __restrict__ Q,
                                                int lane, int wl, float2 (&a2)[4][8]) {
    constexpr int NB = Fwd<DP>::NB, XST = Fwd<DP>::XST;
    const int rb0 = wl, rb1 = NB - 1 - wl;
    const int ce0 = 8 * (rb0 + 1), ce1 = 8 * (rb1 + 1);
    {
        const float4 b00 = *reinterpret_cast<const float4*>(Q + DP * DP + rb0 * 8);
        const float4 b01 = *reinterpret_cast<const float4*>(Q + DP * DP + rb0 * 8 + 4);
        const float4 b10 = *reinterpret_cast<const float4*>(Q + DP * DP + rb1 * 8);
        const float4 b11 = *reinterpret_cast<const float4*>(Q + DP * DP + rb1 * 8 + 4);
        const float2 nb[8] = {make_float2(-b00.x, -b00.y), make_float2(-b00.z, -b00.w), make_float2(-b01.x, -b01.y),
                              make_float2(-b01.z, -b01.w), make_float2(-b10.x, -b10.y), make_float2(-b10.z, -b10.w),
                              make_float2(-b11.x, -b11.y), make_float2(-b11.z, -b11.w)};
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int i = 0; i < 8; ++i) a2[j][i] = nb[i];
    }
    const float* xp = Xs + lane * 4;
    const float* qa = Q + rb0 * 8;
    const float* qb = Q + rb1 * 8;
    // one column c of both row blocks; row pairs of block 0 below i0 are skipped
    // (their Q entries in column c are zero: above the diagonal)
    auto step2 = [&](int c, int i0) {
        const float4 xv = *reinterpret_cast<const float4*>(xp + c * XST);
        const float4 a0 = *reinterpret_cast<const float4*>(qa + c * DP);
        const float4 a1 = *reinterpret_cast<const float4*>(qa + c * DP + 4);
        const float4 b0 = *reinterpret_cast<const float4*>(qb + c * DP);
        const float4 b1 = *reinterpret_cast<const float4*>(qb + c * DP + 4);
        const float2 qs[8] = {make_float2(a0.x, a0.y), make_float2(a0.z, a0.w), make_float2(a1.x, a1.y),
                              make_float2(a1.z, a1.w), make_float2(b0.x, b0.y), make_float2(b0.z, b0.w),
                              make_float2(b1.x, b1.y), make_float2(b1.z, b1.w)};
        const float xs[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float2 xb = make_float2(xs[j], xs[j]);
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (i >= 4 || i >= i0) a2[j][i] = __ffma2_rn(xb, qs[i], a2[j][i]);
        }
    };
    // one column c of row block 1 only, row pairs below i0 skipped
    auto step1 = [&](int c, int i0) {
        const float4 xv = *reinterpret_cast<const float4*>(xp + c * XST);
        const float4 b0 = *reinterpret_cast<const float4*>(qb + c * DP);
        const float4 b1 = *reinterpret_cast<const float4*>(qb + c * DP + 4);
        const float2 qs[4] = {make_float2(b0.x, b0.y), make_float2(b0.z, b0.w), make_float2(b1.x, b1.y),
                              make_float2(b1.z, b1.w)};
        const float xs[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float2 xb = make_float2(xs[j], xs[j]);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (i >= i0) a2[j][4 + i] = __ffma2_rn(xb, qs[i], a2[j][4 + i]);
        }
    };
    // columns left of block 0's diagonal: both blocks in full
#pragma unroll 2
    for (int c = 0; c < 8 * rb0; ++c) step2(c, 0);
    // block 0's diagonal columns 8 rb0 + t: row pairs i >= t / 2 only (row 8 rb0 + 2i + 1 >= c)
#pragma unroll
    for (int t = 0; t < 8; ++t) step2(8 * rb0 + t, t / 2);
    // columns between the diagonals: block 1 only
#pragma unroll 4
    for (int c = ce0; c < 8 * rb1; ++c) step1(c, 0);
#pragma unroll
    for (int t = 0; t < 8; ++t) step1(8 * rb1 + t, t / 2);
    (void)ce1;
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

    // per point: the slots' partial squared norms of round `rd` (in red buffer
    // rd & 1) into the log-joint and the online logsumexp
    auto finish_round = [&](int rd) {
        const float* redb = red + (rd & 1) * NS * NWC * TP;
#pragma unroll
        for (int u = 0; u < NPAIR; ++u) {
            const int e = tid + u * C::THREADS;
            if (e < NS * TP) {
                const int s = e / TP, p = e % TP;
                const int kc = rd * NS + s;
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
    };

    // One block barrier per round. Round r's contraction writes red buffer
    // r & 1 and reads records buffer r & 1; the log-joint of round r - 1 is
    // finished from red buffer (r - 1) & 1 in the same interval. The barrier
    // at the end of round r orders both before round r + 1 (which finishes
    // round r, and whose thread 0 refills records buffer r & 1 for round r + 2).
    __syncthreads();  // the point tile is complete
    bool ok = true;
    int last_issued = 0;  // highest round whose copies were issued (thread 0)
    int done = 0;         // rounds whose contraction completed on every thread
    for (int round = 0; round < rounds; ++round) {
        const int buf = round & 1;
        if (tid == 0 && round + 1 < rounds) {
            issue(round + 1);
            last_issued = round + 1;
        }
        ok = mbar_wait(&bar[buf], (round >> 1) & 1, status) && ok;
        const int kk = round * NS + slot;
        if (ok && kk < k) {
            float* redb = red + buf * NS * NWC * TP;
            const float* Q = Qb + (buf * NS + slot) * REC;
            float2 z2[4][8];
            fwd_gemm_packed<DP>(Xs, Q, lane, wl, z2);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
                for (int i = 0; i < 8; ++i) s2 = __ffma2_rn(z2[j][i], z2[j][i], s2);
                redb[(slot * NWC + wl) * TP + lane * 4 + j] = s2.x + s2.y;
            }
        }
        if (round > 0) finish_round(round - 1);
        // this thread's reads of the records in Qb[buf] (ordinary shared loads)
        // come before the bulk copy (async proxy) that refills the buffer after
        // the barrier
        fence_proxy_async_smem();
        ok = __syncthreads_and(ok);  // all threads agree on ok
        if (!ok) break;
        done = round + 1;
    }
    if (ok && done > 0) finish_round(done - 1);
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
// grid (component groups, point chunks). Each 8x8 block is accumulated in
// packed float32 pairs along its diagonals: with y = r x_a and pairs
// y2_i = (y_2i, y_2i+1),
//   D[i][j] += y2_i * (x_2j, x_2j+1)   -> (S[2i][2j],   S[2i+1][2j+1])
//   X[i][j] += y2_i * (x_2j+1, x_2j)   -> (S[2i][2j+1], S[2i+1][2j])
// where the swapped pairs are register moves of the loaded ones: no
// broadcasts, and every S entry sees the same float32 multiply and FMAs in the
// same point order as a scalar loop.
// UNROLL: point-loop unroll, registers permitting (the plain kernel takes 4
// for padded dimensions up to 64, the persistent batched kernel 2): the next
// points' shared loads overlap the FMAs.
template <int DP, int UNROLL = 1, int GCX = 0>
__device__ __forceinline__ void gmm_bwd_seq_body(const float* __restrict__ x, int64_t n, int d, int k,
                   const float* __restrict__ lj, int64_t lj_ld, const float* __restrict__ lse,
                   float seed, int64_t tiles_per_chunk, float* __restrict__ partS,
                   float* __restrict__ partM, unsigned bx, unsigned by) {
    using C = Bwd<DP, GCX>;
    constexpr int TPB = C::TPB, XST = C::XST, GC = C::GC, NB = C::NB, NBLK = C::NBLK, MP = C::MP;
    constexpr int NT = C::THREADS;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* Xs = reinterpret_cast<float*>(smem_raw);  // [2][TPB][XST]
    float* rawlj = Xs + 2 * TPB * XST;                // [3][GC][TPB]
    float* rawlse = rawlj + 3 * GC * TPB;             // [3][TPB]
    float* rs = rawlse + 3 * TPB;                     // [3][TPB][GC]
    const int tid = threadIdx.x;
    const int kg0 = bx * GC;
    const int64_t ntiles = (n + TPB - 1) / TPB;
    const int64_t t_begin = (int64_t)by * tiles_per_chunk;
    const int64_t t_end = min64(ntiles, t_begin + tiles_per_chunk);

    // role of this thread: component kk, block (a, b)
    const int kk = tid / NBLK;
    int a = 0, b = tid - kk * NBLK;
    while (b > a) {
        ++a;
        b -= a;
    }
    const bool active = (tid < C::NACT) && (kg0 + kk < k);
    int moff[MP];
#pragma unroll
    for (int s = 0; s < MP; ++s) {
        const int c = bwd_mtask<NB>(a, b, s);
        moff[s] = c < 0 ? DP : c == DP ? DP : bwd_swz(c);
    }

    // Pipeline, one block barrier per tile. At the top of tile t: the points
    // of t in X[t % 2] and their r in R[t % 3]; the points of t+1 and the
    // log-joint of t+2 in flight. 16-byte copies when the rows allow them.
    const bool v4 = (d % 4 == 0) && ((reinterpret_cast<uintptr_t>(x) & 15) == 0);
    auto issue_x = [&](int64_t t, int buf) {
        const int64_t p0 = t * TPB;
        const int nv = (int)min64(TPB, n - p0);
        float* X = Xs + buf * TPB * XST;
        if (v4) {
            const int q4 = d >> 2;
            for (int e = tid; e < nv * q4; e += NT) {
                const int p = e / q4, c = 4 * (e - p * q4);
                cp_async16(X + p * XST + bwd_swz(c), x + (p0 + p) * d + c);
            }
        } else {
            for (int e = tid; e < nv * d; e += NT) {
                const int p = e / d, c = e - p * d;
                cp_async4(X + p * XST + bwd_swz(c), x + (p0 + p) * d + c);
            }
        }
    };
    auto issue_lj = [&](int64_t t, int buf) {
        const int64_t p0 = t * TPB;
        const int nv = (int)min64(TPB, n - p0);
        float* L = rawlj + buf * GC * TPB;
        for (int e = tid; e < GC * TPB; e += NT) {
            const int kc = e / TPB, p = e % TPB;
            if (p < nv && kg0 + kc < k) cp_async4(L + e, lj + (int64_t)(kg0 + kc) * lj_ld + p0 + p);
        }
        float* S = rawlse + buf * TPB;
        for (int p = tid; p < nv; p += NT) cp_async4(S + p, lse + p0 + p);
    };
    // cotangents r = seed exp(s - lse) of tile t from buffer buf; 0 on the ragged tail
    auto make_r = [&](int64_t t, int buf) {
        const int64_t p0 = t * TPB;
        const int nv = (int)min64(TPB, n - p0);
        const float* L = rawlj + buf * GC * TPB;
        const float* S = rawlse + buf * TPB;
        float* R = rs + buf * TPB * GC;
        for (int e = tid; e < GC * TPB; e += NT) {
            const int kc = e / TPB, p = e % TPB;
            float r = 0.f;
            if (p < nv && kg0 + kc < k) r = seed * expf(L[e] - S[p]);
            R[p * GC + kc] = r;
        }
    };

    // zero tiles (padding coordinates and ragged rows stay finite), 1.0 at DP, DP+1
    for (int e = tid; e < 2 * TPB * XST; e += NT) {
        const int col = e % XST;
        Xs[e] = (col == DP || col == DP + 1) ? 1.f : 0.f;
    }
    __syncthreads();

    float2 accd[4][4], accx[4][4], macc[MP];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) accd[i][j] = accx[i][j] = make_float2(0.f, 0.f);
#pragma unroll
    for (int s = 0; s < MP; ++s) macc[s] = make_float2(0.f, 0.f);

    // prologue
    if (t_begin < t_end) {
        issue_x(t_begin, 0);
        issue_lj(t_begin, 0);
        if (t_begin + 1 < t_end) issue_lj(t_begin + 1, 1);
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    if (t_begin < t_end) make_r(t_begin, 0);
    if (t_begin + 1 < t_end) {
        make_r(t_begin + 1, 1);
        issue_x(t_begin + 1, 1);
        if (t_begin + 2 < t_end) issue_lj(t_begin + 2, 2);
    }
    cp_async_commit();
    __syncthreads();

    int b2 = 0, b3 = 0;  // (t - t_begin) mod 2, mod 3
    for (int64_t t = t_begin; t < t_end; ++t) {
        if (active) {
            const float* Xb = Xs + b2 * TPB * XST;
            const float* rb = rs + b3 * TPB * GC + kk;
            // halves of the chunks in swizzled order (see bwd_swz)
            const int ha = ((a >> 2) & 1) << 2, hb = ((b >> 2) & 1) << 2;
            const float* xa = Xb + 8 * a;
            const float* xb = Xb + 8 * b;
#pragma unroll UNROLL
            for (int p = 0; p < TPB; ++p) {
                const float rr = rb[p * GC];
                const float2 r2 = make_float2(rr, rr);
#pragma unroll
                for (int s = 0; s < MP; ++s)
                    macc[s] = __ffma2_rn(r2, *reinterpret_cast<const float2*>(Xb + p * XST + moff[s]), macc[s]);
                float2 y[4];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float4 av = *reinterpret_cast<const float4*>(xa + p * XST + ((4 * h) ^ ha));
                    y[2 * h] = __fmul2_rn(r2, make_float2(av.x, av.y));
                    y[2 * h + 1] = __fmul2_rn(r2, make_float2(av.z, av.w));
                }
#pragma unroll
                for (int g = 0; g < 2; ++g) {  // columns 4g .. 4g+3
                    const float4 bv = *reinterpret_cast<const float4*>(xb + p * XST + ((4 * g) ^ hb));
                    const float2 nb[2] = {make_float2(bv.x, bv.y), make_float2(bv.z, bv.w)};
                    const float2 sb[2] = {make_float2(bv.y, bv.x), make_float2(bv.w, bv.z)};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            accd[i][2 * g + j] = __ffma2_rn(y[i], nb[j], accd[i][2 * g + j]);
                            accx[i][2 * g + j] = __ffma2_rn(y[i], sb[j], accx[i][2 * g + j]);
                        }
                }
            }
        }
        const int n2 = b2 ^ 1, n3a = b3 == 2 ? 0 : b3 + 1, n3b = n3a == 2 ? 0 : n3a + 1;
        cp_async_wait_all();  // this thread's copies of x(t+1) and lj(t+2) have landed
        __syncthreads();      // x(t+1), lj(t+2) complete; nobody reads X[b2], R[b3] any more
        if (t + 2 < t_end) {
            make_r(t + 2, n3b);
            issue_x(t + 2, b2);
            if (t + 3 < t_end) issue_lj(t + 3, b3);
        }
        cp_async_commit();
        b2 = n2;
        b3 = n3a;
    }
    if (!active) return;
    const int kg = kg0 + kk;
    const int64_t base = ((int64_t)by * k + kg);
    float* S = partS + base * NBLK * 64 + (int64_t)(a * (a + 1) / 2 + b) * 64;
    const bool diag = a == b;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float2 dv = accd[i][j], xv = accx[i][j];
            // D: (2i, 2j), (2i+1, 2j+1); X: (2i, 2j+1), (2i+1, 2j)
            if (!diag || j <= i) {
                S[(2 * i) * 8 + 2 * j] += dv.x;
                S[(2 * i + 1) * 8 + 2 * j + 1] += dv.y;
                S[(2 * i + 1) * 8 + 2 * j] += xv.y;
            }
            if (!diag || j < i) S[(2 * i) * 8 + 2 * j + 1] += xv.x;
        }
    float* M = partM + base * (DP + 1);
#pragma unroll
    for (int s = 0; s < MP; ++s) {
        const int c = bwd_mtask<NB>(a, b, s);
        const float2 v = macc[s];
        if (c == DP) {
            M[DP] += v.x;
        } else if (c >= 0) {
            M[c] += v.x;
            M[c + 1] += v.y;
        }
    }
}

// Block-per-warp backward (D > 32): the same Accum sums as gmm_bwd_seq_body
// with every S entry, m pair and R receiving the same float32 operations in
// the same point order. Per point, a thread loads its row chunk (two 16-byte
// loads; two more for its second chunk), its component's r and the operands
// of its m / R tasks, then issues 4 packed multiplies and 32 packed FMAs per
// off-diagonal block, or 2 x (4 + 20) on its two diagonal blocks (upper
// halves skipped).
template <bool DIAG>
__device__ __forceinline__ void bwd_block_update(float2 r2, float4 a0, float4 a1, float4 b0, float4 b1,
                                                 float2 (&accd)[4][4], float2 (&accx)[4][4]) {
    float2 y[4];
    y[0] = __fmul2_rn(r2, make_float2(a0.x, a0.y));
    y[1] = __fmul2_rn(r2, make_float2(a0.z, a0.w));
    y[2] = __fmul2_rn(r2, make_float2(a1.x, a1.y));
    y[3] = __fmul2_rn(r2, make_float2(a1.z, a1.w));
    const float4 bq[2] = {b0, b1};
#pragma unroll
    for (int g = 0; g < 2; ++g) {  // columns 4g .. 4g+3
        const float4 bv = bq[g];
        const float2 nb[2] = {make_float2(bv.x, bv.y), make_float2(bv.z, bv.w)};
        const float2 sb[2] = {make_float2(bv.y, bv.x), make_float2(bv.w, bv.z)};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                if (DIAG && 2 * g + j > i) continue;  // pair column above the row pair
                accd[i][2 * g + j] = __ffma2_rn(y[i], nb[j], accd[i][2 * g + j]);
                accx[i][2 * g + j] = __ffma2_rn(y[i], sb[j], accx[i][2 * g + j]);
            }
    }
}

// Lower triangle (diagonal included) of the diagonal block of chunk v with
// row-scaled values y = r v (4 pairs) and v itself (a0, a1): the 10 pairs
// (S[2i][2j], S[2i+1][2j+1]), j <= i, through D(i, j), the 6 pairs
// (S[2i][2j+1], S[2i+1][2j]), j < i, through X(i, j), and the 4 entries
// S[2i+1][2i] as scalars h[i].
template <typename FD, typename FX>
__device__ __forceinline__ void bwd_tri_update(const float2 (&y)[4], float4 a0, float4 a1, FD&& D, FX&& X,
                                               float (&h)[4]) {
    const float v[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            D(i, j) = __ffma2_rn(y[i], make_float2(v[2 * j], v[2 * j + 1]), D(i, j));
            if (j < i) X(i, j) = __ffma2_rn(y[i], make_float2(v[2 * j + 1], v[2 * j]), X(i, j));
        }
        h[i] = fmaf(y[i].y, v[2 * i], h[i]);
    }
}

// One pass over a point tile. Off the diagonal (DIAG false): block (a, b)
// (pa*, pb* locate chunks a and b) into accd / accx, and MT m / R tasks, the
// pairs at moff[t] into macc[t]. On the diagonal: the lower triangles of blocks (a, a) and (b, b) in one
// set of 32 pairs -- block a in accd[i][j] (j <= i) and accx[i][j] (j < i),
// block b transposed into the other slots, accx[j][i] (j <= i) and accd[j][i]
// (j < i) -- plus the 8 scalars h; each block's m task is its chunk's first
// pair, i.e. the sum of y[0] (macc[0], macc[1]).
template <int DP, bool DIAG, int MT, int UNROLL>
__device__ __forceinline__ void bwd_wb_tile(const float* __restrict__ Xb, const float* __restrict__ rb, int pa0,
                                            int pb0, const int (&moff)[2], float2 (&accd)[4][4],
                                            float2 (&accx)[4][4], float (&h)[8], float2 (&macc)[2]) {
    using C = Bwd<DP>;
    constexpr int TPB = C::TPB, XST = C::XST, GC = C::GC, H1 = 4 * C::NB;  // second half of a chunk
#pragma unroll UNROLL
    for (int p = 0; p < TPB; ++p) {
        const float* row = Xb + p * XST;
        const float rr = rb[p * GC];
        const float2 r2 = make_float2(rr, rr);
        const float4 a0 = *reinterpret_cast<const float4*>(row + pa0);
        const float4 a1 = *reinterpret_cast<const float4*>(row + pa0 + H1);
        float2 y[4];
        y[0] = __fmul2_rn(r2, make_float2(a0.x, a0.y));
        y[1] = __fmul2_rn(r2, make_float2(a0.z, a0.w));
        y[2] = __fmul2_rn(r2, make_float2(a1.x, a1.y));
        y[3] = __fmul2_rn(r2, make_float2(a1.z, a1.w));
        if constexpr (DIAG) {
            float ha[4] = {h[0], h[1], h[2], h[3]};
            bwd_tri_update(y, a0, a1, [&](int i, int j) -> float2& { return accd[i][j]; },
                           [&](int i, int j) -> float2& { return accx[i][j]; }, ha);
            macc[0] = __fadd2_rn(macc[0], y[0]);
            const float4 b0 = *reinterpret_cast<const float4*>(row + pb0);
            const float4 b1 = *reinterpret_cast<const float4*>(row + pb0 + H1);
            float2 z[4];
            z[0] = __fmul2_rn(r2, make_float2(b0.x, b0.y));
            z[1] = __fmul2_rn(r2, make_float2(b0.z, b0.w));
            z[2] = __fmul2_rn(r2, make_float2(b1.x, b1.y));
            z[3] = __fmul2_rn(r2, make_float2(b1.z, b1.w));
            float hb[4] = {h[4], h[5], h[6], h[7]};
            bwd_tri_update(z, b0, b1, [&](int i, int j) -> float2& { return accx[j][i]; },
                           [&](int i, int j) -> float2& { return accd[j][i]; }, hb);
            macc[1] = __fadd2_rn(macc[1], z[0]);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                h[i] = ha[i];
                h[4 + i] = hb[i];
            }
        } else {
#pragma unroll
            for (int t = 0; t < MT; ++t)
                macc[t] = __ffma2_rn(r2, *reinterpret_cast<const float2*>(row + moff[t]), macc[t]);
            const float4 b0 = *reinterpret_cast<const float4*>(row + pb0);
            const float4 b1 = *reinterpret_cast<const float4*>(row + pb0 + H1);
            bwd_block_update<false>(r2, a0, a1, b0, b1, accd, accx);
        }
    }
}

// S block (a, b) of one component from its packed accumulators into the
// chunk's partial sums (+=); diagonal blocks keep their lower half.
__device__ __forceinline__ void bwd_store_block(float* __restrict__ S, bool diag, const float2 (&accd)[4][4],
                                                const float2 (&accx)[4][4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float2 dv = accd[i][j], xv = accx[i][j];
            // D: (2i, 2j), (2i+1, 2j+1); X: (2i, 2j+1), (2i+1, 2j)
            if (!diag || j <= i) {
                S[(2 * i) * 8 + 2 * j] += dv.x;
                S[(2 * i + 1) * 8 + 2 * j + 1] += dv.y;
                S[(2 * i + 1) * 8 + 2 * j] += xv.y;
            }
            if (!diag || j < i) S[(2 * i) * 8 + 2 * j + 1] += xv.x;
        }
}

template <int DP, int UNROLL = 1>
__device__ __forceinline__ void gmm_bwd_wb_body(const float* __restrict__ x, int64_t n, int d, int k,
                   const float* __restrict__ lj, int64_t lj_ld, const float* __restrict__ lse,
                   float seed, int64_t tiles_per_chunk, float* __restrict__ partS,
                   float* __restrict__ partM, unsigned bx, unsigned by) {
    using C = Bwd<DP>;
    constexpr int TPB = C::TPB, XST = C::XST, GC = C::GC, NB = C::NB, NBLK = C::NBLK;
    constexpr int NT = C::THREADS;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* Xs = reinterpret_cast<float*>(smem_raw);  // [2][TPB][XST]
    float* rawlj = Xs + 2 * TPB * XST;                // [3][GC][TPB]
    float* rawlse = rawlj + 3 * GC * TPB;             // [3][TPB]
    float* rs = rawlse + 3 * TPB;                     // [3][TPB][GC]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int kg0 = bx * GC;
    const int64_t ntiles = (n + TPB - 1) / TPB;
    const int64_t t_begin = (int64_t)by * tiles_per_chunk;
    const int64_t t_end = min64(ntiles, t_begin + tiles_per_chunk);

    // role of this thread: component kk of the CTA; diagonal blocks (a, a) and
    // (b, b) with b = NB - 1 - a, or off-diagonal block (a, b)
    const int kk = lane % GC, slot = lane / GC;
    const bool diag = warp < C::NDW;
    int a, b;
    if (diag) {
        a = warp * C::BPW + slot;
        b = NB - 1 - a;
    } else {
        bwd_off_block<NB>((warp - C::NDW) * C::BPW + slot, a, b);
    }
    const bool active = kg0 + kk < k;
    const int pa0 = bwd_pos<NB>(8 * a), pb0 = bwd_pos<NB>(8 * b);
    // m / R tasks. The diagonal threads sum the first pair (8c, 8c+1) of
    // their chunks c from their scaled row values (no load). The other 3 NB
    // pairs (8c + 2s, s = 1..3) and R (the constant 1.0 pair at DP) go to the
    // off-diagonal threads of warps on the schedulers without a diagonal warp
    // (warp w on scheduler w % 4), C::MTL tasks per thread, so that each
    // scheduler carries about the same packed FMAs per point.
    const bool light = !diag && (warp & 3) >= C::NDW;
    const int mtask0 = light ? ((warp >> 2) * (4 - C::NDW) + (warp & 3) - C::NDW) * C::BPW + slot : -1;
    int mco[2], moff[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int q = mtask0 < 0 || t >= C::MTL ? -1 : mtask0 * C::MTL + t;  // task id
        mco[t] = q < 0 || q > 3 * NB ? -1 : q == 3 * NB ? DP : 8 * (q / 3) + 2 * (q % 3 + 1);
        moff[t] = mco[t] < 0 || mco[t] == DP ? DP : bwd_pos<NB>(mco[t]);
    }

    // Pipeline, one block barrier per tile. At the top of tile t: the points
    // of t in X[t % 2] and their r in R[t % 3]; the points of t+1 and the
    // log-joint of t+2 in flight. 16-byte copies when the rows allow them.
    const bool v4 = (d % 4 == 0) && ((reinterpret_cast<uintptr_t>(x) & 15) == 0);
    auto issue_x = [&](int64_t t, int buf) {
        const int64_t p0 = t * TPB;
        const int nv = (int)min64(TPB, n - p0);
        float* X = Xs + buf * TPB * XST;
        if (v4 && d == DP) {  // full rows: constant divisor
            constexpr int Q4 = DP / 4;
            for (int e = tid; e < nv * Q4; e += NT) {
                const int p = e / Q4, c = 4 * (e - p * Q4);
                cp_async16(X + p * XST + bwd_pos<NB>(c), x + (p0 + p) * DP + c);
            }
        } else if (v4) {
            const int q4 = d >> 2;
            for (int e = tid; e < nv * q4; e += NT) {
                const int p = e / q4, c = 4 * (e - p * q4);
                cp_async16(X + p * XST + bwd_pos<NB>(c), x + (p0 + p) * d + c);
            }
        } else {
            for (int e = tid; e < nv * d; e += NT) {
                const int p = e / d, c = e - p * d;
                cp_async4(X + p * XST + bwd_pos<NB>(c), x + (p0 + p) * d + c);
            }
        }
    };
    auto issue_lj = [&](int64_t t, int buf) {
        const int64_t p0 = t * TPB;
        const int nv = (int)min64(TPB, n - p0);
        float* L = rawlj + buf * GC * TPB;
        for (int e = tid; e < GC * TPB; e += NT) {
            const int kc = e / TPB, p = e % TPB;
            if (p < nv && kg0 + kc < k) cp_async4(L + e, lj + (int64_t)(kg0 + kc) * lj_ld + p0 + p);
        }
        float* S = rawlse + buf * TPB;
        for (int p = tid; p < nv; p += NT) cp_async4(S + p, lse + p0 + p);
    };
    // cotangents r = seed exp(s - lse) of tile t from buffer buf; 0 on the ragged tail
    auto make_r = [&](int64_t t, int buf) {
        const int64_t p0 = t * TPB;
        const int nv = (int)min64(TPB, n - p0);
        const float* L = rawlj + buf * GC * TPB;
        const float* S = rawlse + buf * TPB;
        float* R = rs + buf * TPB * GC;
        for (int e = tid; e < GC * TPB; e += NT) {
            const int kc = e / TPB, p = e % TPB;
            float r = 0.f;
            if (p < nv && kg0 + kc < k) r = seed * expf(L[e] - S[p]);
            R[p * GC + kc] = r;
        }
    };

    // zero tiles (padding coordinates and ragged rows stay finite), 1.0 at DP, DP+1
    for (int e = tid; e < 2 * TPB * XST; e += NT) {
        const int col = e % XST;
        Xs[e] = (col == DP || col == DP + 1) ? 1.f : 0.f;
    }
    __syncthreads();

    float2 accd[4][4], accx[4][4], macc[2];
    float h[8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) accd[i][j] = accx[i][j] = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 8; ++i) h[i] = 0.f;
    macc[0] = macc[1] = make_float2(0.f, 0.f);

    // prologue
    if (t_begin < t_end) {
        issue_x(t_begin, 0);
        issue_lj(t_begin, 0);
        if (t_begin + 1 < t_end) issue_lj(t_begin + 1, 1);
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    if (t_begin < t_end) make_r(t_begin, 0);
    if (t_begin + 1 < t_end) {
        make_r(t_begin + 1, 1);
        issue_x(t_begin + 1, 1);
        if (t_begin + 2 < t_end) issue_lj(t_begin + 2, 2);
    }
    cp_async_commit();
    __syncthreads();

    int b2 = 0, b3 = 0;  // (t - t_begin) mod 2, mod 3
    for (int64_t t = t_begin; t < t_end; ++t) {
        const float* Xb = Xs + b2 * TPB * XST;
        const float* rb = rs + b3 * TPB * GC + kk;
        if (diag)  // warp-uniform
            bwd_wb_tile<DP, true, 0, UNROLL>(Xb, rb, pa0, pb0, moff, accd, accx, h, macc);
        else if (light)
            bwd_wb_tile<DP, false, C::MTL, UNROLL>(Xb, rb, pa0, pb0, moff, accd, accx, h, macc);
        else
            bwd_wb_tile<DP, false, 0, UNROLL>(Xb, rb, pa0, pb0, moff, accd, accx, h, macc);
        const int n2 = b2 ^ 1, n3a = b3 == 2 ? 0 : b3 + 1, n3b = n3a == 2 ? 0 : n3a + 1;
        cp_async_wait_all();  // this thread's copies of x(t+1) and lj(t+2) have landed
        __syncthreads();      // x(t+1), lj(t+2) complete; nobody reads X[b2], R[b3] any more
        if (t + 2 < t_end) {
            make_r(t + 2, n3b);
            issue_x(t + 2, b2);
            if (t + 3 < t_end) issue_lj(t + 3, b3);
        }
        cp_async_commit();
        b2 = n2;
        b3 = n3a;
    }
    if (!active) return;
    const int kg = kg0 + kk;
    const int64_t base = ((int64_t)by * k + kg);
    float* Sk = partS + base * NBLK * 64;
    float* M = partM + base * (DP + 1);
    if (diag) {
        // block (a, a): accd[i][j] (j <= i), accx[i][j] (j < i), h[0..3];
        // block (b, b): accx[j][i] (j <= i), accd[j][i] (j < i), h[4..7]
        float* Sa = Sk + (int64_t)(a * (a + 1) / 2 + a) * 64;
        float* Sb = Sk + (int64_t)(b * (b + 1) / 2 + b) * 64;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
#pragma unroll
            for (int j = 0; j <= i; ++j) {
                const float2 da = accd[i][j], db = accx[j][i];
                Sa[(2 * i) * 8 + 2 * j] += da.x;
                Sa[(2 * i + 1) * 8 + 2 * j + 1] += da.y;
                Sb[(2 * i) * 8 + 2 * j] += db.x;
                Sb[(2 * i + 1) * 8 + 2 * j + 1] += db.y;
                if (j < i) {
                    const float2 xa = accx[i][j], xb = accd[j][i];
                    Sa[(2 * i) * 8 + 2 * j + 1] += xa.x;
                    Sa[(2 * i + 1) * 8 + 2 * j] += xa.y;
                    Sb[(2 * i) * 8 + 2 * j + 1] += xb.x;
                    Sb[(2 * i + 1) * 8 + 2 * j] += xb.y;
                }
            }
            Sa[(2 * i + 1) * 8 + 2 * i] += h[i];
            Sb[(2 * i + 1) * 8 + 2 * i] += h[4 + i];
        }
        const int ma = bwd_mtask<NB>(a, a, 0), mb = bwd_mtask<NB>(b, b, 0);  // 8a, 8b
        M[ma] += macc[0].x;
        M[ma + 1] += macc[0].y;
        M[mb] += macc[1].x;
        M[mb + 1] += macc[1].y;
    } else {
        bwd_store_block(Sk + (int64_t)(a * (a + 1) / 2 + b) * 64, false, accd, accx);
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            if (mco[t] == DP) {
                M[DP] += macc[t].x;
            } else if (mco[t] >= 0) {
                M[mco[t]] += macc[t].x;
                M[mco[t] + 1] += macc[t].y;
            }
        }
    }
}

template <int DP, int UNROLL = 1, int GCX = 0>
__device__ __forceinline__ void gmm_bwd_kernel_body(const float* __restrict__ x, int64_t n, int d, int k,
                   const float* __restrict__ lj, int64_t lj_ld, const float* __restrict__ lse,
                   float seed, int64_t tiles_per_chunk, float* __restrict__ partS,
                   float* __restrict__ partM, unsigned bx, unsigned by) {
    if constexpr (Bwd<DP>::WB)
        gmm_bwd_wb_body<DP, UNROLL>(x, n, d, k, lj, lj_ld, lse, seed, tiles_per_chunk, partS, partM, bx, by);
    else
        gmm_bwd_seq_body<DP, UNROLL, GCX>(x, n, d, k, lj, lj_ld, lse, seed, tiles_per_chunk, partS, partM, bx,
                                          by);
}

template <int DP>
__global__ void __launch_bounds__(Bwd<DP>::THREADS, Bwd<DP>::MINB)
    gmm_bwd_kernel(const float* __restrict__ x, int64_t n, int d, int k,
                   const float* __restrict__ lj, int64_t lj_ld, const float* __restrict__ lse,
                   float seed, int64_t tiles_per_chunk, float* __restrict__ partS,
                   float* __restrict__ partM) {
    gmm_bwd_kernel_body<DP, Bwd<DP>::UNROLL>(x, n, d, k, lj, lj_ld, lse, seed, tiles_per_chunk, partS, partM,
                                                blockIdx.x, blockIdx.y);
}

// Sum over chunks c = 0 .. n-1 of p[c * stride] (float32 partials), in chunk
// order, as an unevaluated pair hi + lo of float32 (TwoSum, Knuth): about 48
// significant bits, as good as a float64 sum of float32 terms, but on the
// float32 pipe (this GPU issues float64 at a small fraction of that rate).
__device__ __forceinline__ double chunk_sum(const float* __restrict__ p, int64_t stride, int n) {
    float hi = 0.f, lo = 0.f;
    for (int c = 0; c < n; ++c) {
        const float x = p[(int64_t)c * stride];
        const float t = __fadd_rn(hi, x);
        const float bb = __fsub_rn(t, hi);
        lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bb)), __fsub_rn(x, bb)));
        hi = t;
    }
    return (double)hi + (double)lo;
}

// Row r and column c <= r of the e-th entry of a lower triangle stored by rows
// (e = r (r + 1) / 2 + c): float estimate of r, then exact integer fix-ups.
__device__ __forceinline__ void tri_index(int e, int& r, int& c) {
    r = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
    while (r * (r + 1) / 2 > e) --r;
    while ((r + 1) * (r + 2) / 2 <= e) ++r;
    c = e - r * (r + 1) / 2;
}

// ---------------------------------------------------------------------------
// A3: finalize gradients per component (fixed-order sums over chunks)
// ---------------------------------------------------------------------------
// Dynamic shared memory of gmm_finalize_kernel_body<DP>.
template <int DP>
constexpr size_t gmm_finalize_smem() {
    return sizeof(double) * ((DP / 8) * (DP / 8 + 1) / 2 * 64 + 3 * DP + 1) + sizeof(float) * (2 * DP * DP + 2 * DP) + 64;
}

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
    double* vd = md + DP + 1;                            // [DP]  v = m - R mu
    double* mud = vd + DP;                               // [DP]  mu
    float* Cf = reinterpret_cast<float*>(mud + DP);      // [DP][DP] symmetric
    float* Qf = Cf + DP * DP;                            // [DP][DP] lower
    float* vf = Qf + DP * DP;                            // [DP]  v in float32
    float* wf = vf + DP;                                 // [DP]  w = Q v
    const int kk = bx, tid = threadIdx.x;
    const int t = d * (d - 1) / 2;
    const float* qk = q + (size_t)kk * d;
    const float* lk = l + (size_t)kk * t;

    if (exch) {
        for (int e = tid; e < NBLK * 64; e += 256) Sd[e] = exch[(size_t)kk * E + e];
        for (int e = tid; e < DP + 1; e += 256) md[e] = exch[(size_t)kk * E + NBLK * 64 + e];
    } else {
        for (int e = tid; e < NBLK * 64; e += 256)
            Sd[e] = chunk_sum(partS + (int64_t)kk * NBLK * 64 + e, (int64_t)k * NBLK * 64, nchunks);
        for (int e = tid; e < DP + 1; e += 256)
            md[e] = chunk_sum(partM + (int64_t)kk * (DP + 1) + e, (int64_t)k * (DP + 1), nchunks);
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
    // v = m - R mu (raw moments) or m (centred sums): the cancelling
    // difference in float64, its result rounded once for the float32 products
    for (int j = tid; j < DP; j += 256) {
        vd[j] = centered ? md[j] : md[j] - R * mud[j];
        vf[j] = (float)vd[j];
    }
    __syncthreads();
    // C = S - mu v^T - m mu^T (= S - mu m^T - m mu^T + R mu mu^T), mirrored
    for (int e = tid; e < DP * (DP + 1) / 2; e += 256) {
        int a, b;
        tri_index(e, a, b);
        double c = 0.0;
        if (a < d) {
            const int A = a >> 3, B = b >> 3;
            const double S = Sd[(A * (A + 1) / 2 + B) * 64 + (a & 7) * 8 + (b & 7)];
            c = centered ? S : S - mud[a] * vd[b] - md[a] * mud[b];
        }
        Cf[a * DP + b] = (float)c;
        Cf[b * DP + a] = (float)c;
    }
    // w = Q v (float32: the operands are float32 values, no cancellation left)
    for (int r = tid; r < DP; r += 256) {
        float w = 0.f;
        if (r < d)
            for (int j = 0; j <= r; ++j) w = fmaf(Qf[r * DP + j], vf[j], w);
        wf[r] = w;
    }
    __syncthreads();
    // H = Q C on the lower triangle; dq from its diagonal, dl from the rest
    const int ne = d * (d + 1) / 2;
    const float sg2 = (float)(seed * gamma * gamma);
    for (int e = tid; e < ne; e += 256) {
        int r, c;
        tri_index(e, r, c);
        float h = 0.f;
        for (int j = 0; j <= r; ++j) h = fmaf(Qf[r * DP + j], Cf[j * DP + c], h);
        if (c == r) {
            const double ev = exp((double)qk[r]);
            d_q[(size_t)kk * d + r] += (float)(R - ev * (double)h + seed * ((double)m - gamma * gamma * ev * ev));
        } else {
            const int li = r * (r - 1) / 2 + c;
            d_l[(size_t)kk * t + li] += fmaf(-sg2, lk[li], -h);
        }
    }
    // d mu = Q^T w
    for (int c = tid; c < d; c += 256) {
        float s = 0.f;
        for (int r = c; r < d; ++r) s = fmaf(Qf[r * DP + c], wf[r], s);
        d_mu[(size_t)kk * d + c] += s;
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
// [S blocks | m | R] combined in chunk order (chunk_sum), then the sum of the
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
        if (e < NS)
            exch[(size_t)kk * E + e] += chunk_sum(partS + (int64_t)kk * NS + e, (int64_t)k * NS, nchunks);
        else if (e < E)
            exch[(size_t)kk * E + e] +=
                chunk_sum(partM + (int64_t)kk * (DP + 1) + (e - NS), (int64_t)k * (DP + 1), nchunks);
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
