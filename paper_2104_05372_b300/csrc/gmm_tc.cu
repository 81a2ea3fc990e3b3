// Gaussian mixture on the tensor cores (GPA_PREC_BF16_TC): the two dense
// contractions run as tcgen05 MMAs with BF16 operands in shared memory and FP32
// accumulators in tensor memory; logsumexp, exponentials and every sum over
// points stay FP32 / FP64 on the CUDA cores. Padded dimension 128 (64 < D <= 128).
//
// Forward (A1): Z = X Q_k^T per 128-point tile and component, with split-BF16
// operands: x = x_hi + x_lo and Q = Q_hi + Q_lo (each part BF16), and three MMAs
// per K step (hi*hi + lo*hi + hi*lo), which keeps about 16 bits of the FP32
// inputs -- a single BF16 pass leaves log-joint errors of ~0.4 at D = 128, i.e.
// ~40 % errors in the responsibilities exp(s - lse). Warp roles in a 192-thread
// CTA: warp 0 issues TMA loads (the point tile once, then each component's Q_k
// parts and its b_k / constant through a 2-stage ring), warp 1 owns the TMEM
// allocation and one of its lanes issues the MMAs (M=128 points, N=128 rows of
// Q_k, K=128 in 8 steps of 3) into a double-buffered accumulator, warps 2-5
// read the accumulator back (TMEM lane = point, one thread per point) and fold
// |z - b_k|^2 into the log-joint and an online logsumexp.
//
// Backward (A2): the Accum sums of a component, centred on its mean,
//   C_k = sum_i r_ik (x_i - mu_k)(x_i - mu_k)^T,  m'_k = sum_i r_ik (x_i - mu_k),
//   R_k = sum_i r_ik,
// with C_k = U_k^T U_k for U_k[p][a] = sqrt(r_pk) (x_p - mu_k)[a] (x read in
// FP32, U rounded once to BF16; r from the forward's log-joint). Eight
// producer warps build U_k^T (dimension-major, points contiguous) directly in
// the 128-byte-swizzled layout the MMA reads, one MMA thread accumulates
// C_k += U_k^T U_k (M=N=K=128, A and B the same tile) in TMEM for four
// components across every tile of a point chunk; the partial sums go to the
// same buffers the FP32 finalize reads (centred mode).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "common.cuh"
#include "gmm_internal.cuh"
#include "tc.cuh"
#include "trace.cuh"

namespace gpa {
namespace {

constexpr int TDP = 128;                       // padded dimension
constexpr int TM = 128;                        // points per tile
constexpr int REC = TDP * TDP + TDP + 4;       // FP32 prep record (b at TDP*TDP, cst after)
constexpr uint32_t ATOM = TM * 128;            // one 64-wide K slice of a 128-row operand: 16 KB
constexpr uint32_t TILE_BYTES = 2 * ATOM;      // 128 rows x 128 bf16
constexpr uint32_t IDESC = tc::idesc_bf16_f32(128, 128);

// ---- forward ------------------------------------------------------------------
constexpr int FQ = 2;                          // Q_k stages (hi and lo parts each)
constexpr uint32_t FB_BYTES = (TDP + 4) * 4;   // b_k, constant, pad
struct FwdSm {
    static constexpr uint32_t X = 0;                       // x_hi, x_lo tiles
    static constexpr uint32_t Q = X + 2 * TILE_BYTES;      // [FQ] x (Q_hi, Q_lo)
    static constexpr uint32_t B = Q + FQ * 2 * TILE_BYTES;
    static constexpr uint32_t RED = B + FQ * FB_BYTES;
    static constexpr uint32_t BAR = RED + 8 * 8;  // x_full, q_full[3], q_empty[3], acc_full[2], acc_empty[2]
    static constexpr uint32_t TMEMP = BAR + 16 * 8;
    static constexpr uint32_t FLAG = TMEMP + 8;
    static constexpr uint32_t END = FLAG + 8;
    static constexpr size_t SMEM = END + 1024;  // + alignment slack
};

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
    return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~(uintptr_t)1023);
}

__global__ void __launch_bounds__(192, 1)
    gmm_tc_fwd_kernel(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmxl,
                      const __grid_constant__ CUtensorMap tmq, const __grid_constant__ CUtensorMap tmql,
                      const float* __restrict__ rec, int64_t n, int64_t xrow0, int k, float* __restrict__ lj,
                      int64_t lj_ld, float* __restrict__ lse_out, double* __restrict__ part, int64_t tile0,
                      int32_t* __restrict__ status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = align1024(smem_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + FwdSm::BAR);
    uint64_t* x_full = bars;
    uint64_t* q_full = bars + 1;
    uint64_t* q_empty = bars + 1 + FQ;
    uint64_t* acc_full = bars + 1 + 2 * FQ;
    uint64_t* acc_empty = bars + 3 + 2 * FQ;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(sm + FwdSm::TMEMP);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + FwdSm::FLAG);
    double* red = reinterpret_cast<double*>(sm + FwdSm::RED);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t p0 = (int64_t)blockIdx.x * TM;

    if (threadIdx.x == 0) {
        mbar_init(x_full, 1);
        for (int s = 0; s < FQ; ++s) {
            mbar_init(&q_full[s], 1);
            mbar_init(&q_empty[s], 1 + 4);  // MMA commit + 4 epilogue warps (they read b_k)
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&acc_full[a], 1);
            mbar_init(&acc_empty[a], 4);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_holder, 256);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_holder;

    if (warp == 0) {
        if (lane == 0) {
            mbar_arrive_expect_tx(x_full, 2 * TILE_BYTES);
            tc::tma_load_2d(sm + FwdSm::X, &tmx, 0, (int)(xrow0 + p0), x_full);
            tc::tma_load_2d(sm + FwdSm::X + ATOM, &tmx, 64, (int)(xrow0 + p0), x_full);
            tc::tma_load_2d(sm + FwdSm::X + TILE_BYTES, &tmxl, 0, (int)(xrow0 + p0), x_full);
            tc::tma_load_2d(sm + FwdSm::X + TILE_BYTES + ATOM, &tmxl, 64, (int)(xrow0 + p0), x_full);
            for (int kk = 0; kk < k; ++kk) {
                const int s = kk % FQ;
                const uint32_t ph = (uint32_t)(kk / FQ) & 1u;
                if (!mbar_wait(&q_empty[s], ph ^ 1u, status)) {
                    *abort_flag = 1;
                    break;
                }
                mbar_arrive_expect_tx(&q_full[s], 2 * TILE_BYTES + FB_BYTES);
                uint8_t* qd = sm + FwdSm::Q + s * 2 * TILE_BYTES;
                tc::tma_load_2d(qd, &tmq, 0, kk * TDP, &q_full[s]);
                tc::tma_load_2d(qd + ATOM, &tmq, 64, kk * TDP, &q_full[s]);
                tc::tma_load_2d(qd + TILE_BYTES, &tmql, 0, kk * TDP, &q_full[s]);
                tc::tma_load_2d(qd + TILE_BYTES + ATOM, &tmql, 64, kk * TDP, &q_full[s]);
                bulk_g2s(sm + FwdSm::B + s * FB_BYTES, rec + (size_t)kk * REC + TDP * TDP, FB_BYTES, &q_full[s]);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            bool ok = mbar_wait(x_full, 0, status);
            for (int kk = 0; ok && kk < k; ++kk) {
                const int s = kk % FQ;
                const uint32_t ph = (uint32_t)(kk / FQ) & 1u;
                const int as = kk & 1;
                const uint32_t aph = (uint32_t)(kk >> 1) & 1u;
                if (!mbar_wait(&q_full[s], ph, status) || !mbar_wait(&acc_empty[as], aph ^ 1u, status)) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t xh = smem_u32(sm + FwdSm::X), xl = xh + TILE_BYTES;
                const uint32_t qh = smem_u32(sm + FwdSm::Q + s * 2 * TILE_BYTES), ql = qh + TILE_BYTES;
                const uint32_t dt = tmem + (uint32_t)(as * TDP);
#pragma unroll
                for (int j = 0; j < TDP / 16; ++j) {
                    const uint32_t off = (uint32_t)(j >> 2) * ATOM + (uint32_t)(j & 3) * 32u;
                    tc::mma_bf16(dt, tc::desc_sw128(xh + off), tc::desc_sw128(qh + off), IDESC, j > 0 ? 1u : 0u);
                    tc::mma_bf16(dt, tc::desc_sw128(xl + off), tc::desc_sw128(qh + off), IDESC, 1u);
                    tc::mma_bf16(dt, tc::desc_sw128(xh + off), tc::desc_sw128(ql + off), IDESC, 1u);
                }
                tc::mma_commit(&acc_full[as]);
                tc::mma_commit(&q_empty[s]);
            }
            if (!ok) *abort_flag = 1;
        }
        __syncwarp();
    } else {
        // epilogue: one thread per point (TMEM lane)
        const int qtr = warp & 3;
        const int row = qtr * 32 + lane;
        const bool valid = p0 + row < n;
        Lse st;
        st.init();
        for (int kk = 0; kk < k; ++kk) {
            const int s = kk % FQ;
            const int as = kk & 1;
            const uint32_t aph = (uint32_t)(kk >> 1) & 1u;
            if (!mbar_wait_warp(&acc_full[as], aph, status)) {
                *abort_flag = 1;
                break;
            }
            tc::fence_after_sync();
            const float* bb = reinterpret_cast<const float*>(sm + FwdSm::B + s * FB_BYTES);
            float s2 = 0.f;
#pragma unroll
            for (int ch = 0; ch < TDP / 32; ++ch) {
                float v[32];
                tc::tmem_ld32(tmem + ((uint32_t)(qtr * 32) << 16) + (uint32_t)(as * TDP + ch * 32), v);
                tc::tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 32; i += 4) {
                    const float4 b4 = *reinterpret_cast<const float4*>(bb + ch * 32 + i);
                    const float z0 = v[i] - b4.x, z1 = v[i + 1] - b4.y, z2 = v[i + 2] - b4.z, z3 = v[i + 3] - b4.w;
                    s2 = fmaf(z0, z0, s2);
                    s2 = fmaf(z1, z1, s2);
                    s2 = fmaf(z2, z2, s2);
                    s2 = fmaf(z3, z3, s2);
                }
            }
            const float cst = bb[TDP];
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) {
                tc::mbar_arrive(&acc_empty[as]);
                tc::mbar_arrive(&q_empty[s]);
            }
            const float sv = cst - 0.5f * s2;
            if (valid) {
                if (lj) lj[(int64_t)kk * lj_ld + p0 + row] = sv;
                st.add(sv);
            }
        }
        double v = 0.0;
        if (valid && !*abort_flag) {
            const float lv = st.value();
            if (lse_out) lse_out[p0 + row] = lv;
            v = (double)lv;
        }
        v = warp_sum(v);
        if (lane == 0) red[warp - 2] = v;
    }
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x == 64) part[tile0 + blockIdx.x] = *abort_flag ? NAN : red[0] + red[1] + red[2] + red[3];
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 256);
    }
}

// ---- backward -----------------------------------------------------------------
constexpr int BGC = 4;                          // components per CTA (4 x 128 TMEM columns)
constexpr int BPROD = 256;                      // producer threads (8 warps)
constexpr int BTHREADS = BPROD + 32;            // + the MMA warp
struct BwdSm {
    static constexpr uint32_t U = 0;                              // [BGC] tiles of 32 KB
    static constexpr uint32_t SR = U + BGC * TILE_BYTES;          // sqrt(r) [BGC][TM] float
    static constexpr uint32_t MU = SR + BGC * TM * 4;             // mu [BGC][TDP] float
    static constexpr uint32_t MRED = MU + BGC * TDP * 4;          // m' halves [BGC][TDP] float
    static constexpr uint32_t RRED = MRED + BGC * TDP * 4;        // R per warp [8][BGC] float
    static constexpr uint32_t BAR = RRED + 8 * BGC * 4;           // u_full[4], u_empty[4], done
    static constexpr uint32_t TMEMP = BAR + 16 * 8;
    static constexpr uint32_t FLAG = TMEMP + 8;  // abort flag, then the producers' decision slot
    static constexpr uint32_t END = FLAG + 8;
    static constexpr size_t SMEM = END + 1024;
};

__device__ __forceinline__ void producers_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(BPROD) : "memory");
}

__global__ void __launch_bounds__(BTHREADS, 1)
    gmm_tc_bwd_kernel(const float* __restrict__ x, int64_t n, int k, const float* __restrict__ mu,
                      int d, const float* __restrict__ lj, int64_t lj_ld, const float* __restrict__ lse,
                      float seed, int64_t tiles_per_chunk, float* __restrict__ partS, float* __restrict__ partM,
                      int nblk64, int32_t* __restrict__ status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = align1024(smem_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + BwdSm::BAR);
    uint64_t* u_full = bars;
    uint64_t* u_empty = bars + BGC;
    uint64_t* done = bars + 2 * BGC;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(sm + BwdSm::TMEMP);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + BwdSm::FLAG);
    float* sr = reinterpret_cast<float*>(sm + BwdSm::SR);
    float* mus = reinterpret_cast<float*>(sm + BwdSm::MU);
    float* mred = reinterpret_cast<float*>(sm + BwdSm::MRED);
    float* rred = reinterpret_cast<float*>(sm + BwdSm::RRED);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tid = threadIdx.x;
    const int kg0 = blockIdx.x * BGC;
    const int64_t ntiles = (n + TM - 1) / TM;
    const int64_t t_begin = (int64_t)blockIdx.y * tiles_per_chunk;
    const int64_t t_end = min64(ntiles, t_begin + tiles_per_chunk);

    if (tid == 0) {
        for (int c = 0; c < BGC; ++c) {
            mbar_init(&u_full[c], BPROD / 32);
            mbar_init(&u_empty[c], 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    for (int e = tid; e < BGC * TDP; e += BTHREADS) {
        const int c = e / TDP, a = e % TDP;
        mus[e] = (kg0 + c < k && a < d) ? mu[(size_t)(kg0 + c) * d + a] : 0.f;
    }
    if (warp == BPROD / 32) {
        tc::tmem_alloc(tmem_holder, 512);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_holder;

    if (warp == BPROD / 32) {
        // MMA issuer
        if (lane == 0) {
            bool ok = true;
            int it = 0;
            for (int64_t t = t_begin; ok && t < t_end; ++t, ++it) {
                for (int c = 0; c < BGC; ++c) {
                    if (!mbar_wait(&u_full[c], (uint32_t)it & 1u, status)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t ua = smem_u32(sm + BwdSm::U + c * TILE_BYTES);
#pragma unroll
                    for (int j = 0; j < TM / 16; ++j) {
                        const uint64_t dsc = tc::desc_sw128(ua + (uint32_t)(j >> 2) * ATOM + (uint32_t)(j & 3) * 32u);
                        tc::mma_bf16(tmem + (uint32_t)(c * TDP), dsc, dsc, IDESC, (it > 0 || j > 0) ? 1u : 0u);
                    }
                    tc::mma_commit(&u_empty[c]);
                }
            }
            if (!ok) *abort_flag = 1;
            tc::mma_commit(done);
        }
        __syncwarp();
    } else {
        // producers: thread owns dimension a and half of the tile's points
        const int a = tid & (TDP - 1);
        const int half = tid >> 7;
        float macc[BGC], racc[2] = {0.f, 0.f};
#pragma unroll
        for (int c = 0; c < BGC; ++c) macc[c] = 0.f;
        volatile int* decision = abort_flag + 1;  // written by thread 0 before a barrier, read after it
        int it = 0;
        for (int64_t t = t_begin; t < t_end; ++t, ++it) {
            const int64_t p0 = t * TM;
            // x values of this thread: points p0 + half*64 + 0..63, dimension a
            float xv[64];
#pragma unroll
            for (int j = 0; j < 64; ++j) {
                const int64_t p = p0 + half * 64 + j;
                xv[j] = (p < n && a < d) ? __ldg(x + p * d + a) : 0.f;
            }
            if (tid == 0) *decision = *abort_flag;
            producers_sync();  // previous tile's sqrt(r) no longer read; decision published
            if (*decision) break;  // uniform over all producer threads
            for (int e = tid; e < BGC * TM; e += BPROD) {
                const int c = e / TM, p = e % TM;
                float v = 0.f;
                if (p0 + p < n && kg0 + c < k)
                    v = expf(0.5f * (__ldg(lj + (int64_t)(kg0 + c) * lj_ld + p0 + p) - __ldg(lse + p0 + p)));
                sr[e] = v;
                racc[e / (BGC * TM / 2)] += v * v;
            }
            producers_sync();
#pragma unroll 1
            for (int c = 0; c < BGC; ++c) {
                if (!mbar_wait_warp(&u_empty[c], ((uint32_t)it & 1u) ^ 1u, status)) {
                    *abort_flag = 1;  // skip the work; the next decision point stops every warp
                    continue;
                }
                uint8_t* ut = sm + BwdSm::U + c * TILE_BYTES + half * ATOM;
                const float* src = sr + c * TM + half * 64;
                const float mc = mus[c * TDP + a];
                float mloc = 0.f;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    uint32_t w4[4];
#pragma unroll
                    for (int i = 0; i < 8; i += 2) {
                        const float s0 = src[j * 8 + i], s1 = src[j * 8 + i + 1];
                        const float u0 = s0 * (xv[j * 8 + i] - mc), u1 = s1 * (xv[j * 8 + i + 1] - mc);
                        mloc = fmaf(s0, u0, fmaf(s1, u1, mloc));
                        w4[i >> 1] = tc::pack_bf16x2(u0, u1);
                    }
                    *reinterpret_cast<uint4*>(ut + tc::sw128_offset((uint32_t)a, (uint32_t)j)) =
                        make_uint4(w4[0], w4[1], w4[2], w4[3]);
                }
                macc[c] += mloc;
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&u_full[c]);
            }
        }
        // m' halves
        if (half == 1)
            for (int c = 0; c < BGC; ++c) mred[c * TDP + a] = macc[c];
        // R: racc[0] holds component tid/128, racc[1] component 2 + tid/128
        {
            const float r0 = warp_sum(racc[0]), r1 = warp_sum(racc[1]);
            if (lane == 0) {
                const int cb = tid >> 7;
                rred[warp * BGC + cb] = r0;
                rred[warp * BGC + 2 + cb] = r1;
                rred[warp * BGC + 1 - cb] = 0.f;
                rred[warp * BGC + 3 - cb] = 0.f;
            }
        }
        producers_sync();
        const int64_t cbase = (int64_t)blockIdx.y * k;
        if (half == 0) {
            for (int c = 0; c < BGC; ++c) {
                const int kg = kg0 + c;
                if (kg >= k) break;
                float* M = partM + (cbase + kg) * (TDP + 1);
                M[a] += seed * (macc[c] + mred[c * TDP + a]);
                if (a == 0) {
                    float R = 0.f;
                    for (int w = 0; w < BPROD / 32; ++w) R += rred[w * BGC + c];
                    M[TDP] += seed * R;
                }
            }
        }
        // accumulators: warp w reads TMEM lanes of its quarter for components w/4 and w/4 + 2
        const bool fin = mbar_wait_warp(done, 0, status);
        if (!fin) *abort_flag = 1;
        tc::fence_after_sync();
        producers_sync();  // every warp has seen `done` (or given up) before reading the flag
        const int aborted = __shfl_sync(0xffffffffu, *abort_flag, 0);  // one value per warp
        if (!aborted && t_begin < t_end) {  // a CTA without tiles issued no MMA: TMEM holds nothing
            const int qtr = warp & 3;
            const int row = qtr * 32 + lane;  // dimension a of S
            for (int cc = 0; cc < 2; ++cc) {
                const int c = (warp >> 2) + 2 * cc;
                const int kg = kg0 + c;
                if (kg >= k) continue;
                float* S = partS + (cbase + kg) * (int64_t)nblk64;
#pragma unroll 1
                for (int ch = 0; ch < TDP / 32; ++ch) {
                    float v[32];
                    tc::tmem_ld32(tmem + ((uint32_t)(qtr * 32) << 16) + (uint32_t)(c * TDP + ch * 32), v);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const int b = ch * 32 + i;
                        if (b <= row) {
                            const int A = row >> 3, B = b >> 3;
                            S[(A * (A + 1) / 2 + B) * 64 + (row & 7) * 8 + (b & 7)] += seed * v[i];
                        }
                    }
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == BPROD / 32) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 512);
    }
}

// ---- conversions ----------------------------------------------------------------
// x [n][d] float -> x_hi + x_lo, each [n][128] bf16, zero padded
__global__ void __launch_bounds__(256) tc_convert_x_kernel(const float* __restrict__ x, int64_t n, int d,
                                                           __nv_bfloat16* __restrict__ xb,
                                                           __nv_bfloat16* __restrict__ xl) {
    const int64_t total = n * (TDP / 2);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        const int64_t i = e / (TDP / 2);
        const int c = (int)(e % (TDP / 2)) * 2;
        const float v0 = c < d ? __ldg(x + i * d + c) : 0.f;
        const float v1 = c + 1 < d ? __ldg(x + i * d + c + 1) : 0.f;
        const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
        reinterpret_cast<__nv_bfloat162*>(xb + i * TDP)[c / 2] = h;
        reinterpret_cast<__nv_bfloat162*>(xl + i * TDP)[c / 2] =
            __floats2bfloat162_rn(v0 - __low2float(h), v1 - __high2float(h));
    }
}

// prep record Qt[c][r] -> Q_hi + Q_lo, each qb[k][r][c] bf16
__global__ void __launch_bounds__(256) tc_convert_q_kernel(const float* __restrict__ rec, int k,
                                                           __nv_bfloat16* __restrict__ qb,
                                                           __nv_bfloat16* __restrict__ ql) {
    const int64_t total = (int64_t)k * TDP * TDP;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        const int64_t kk = e / (TDP * TDP);
        const int r = (int)((e / TDP) % TDP), c = (int)(e % TDP);
        const float v = rec[kk * REC + (int64_t)c * TDP + r];
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        qb[e] = h;
        ql[e] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

// ---- host ---------------------------------------------------------------------------
size_t a1024(size_t v) { return (v + 1023) & ~(size_t)1023; }

struct TcLayout {
    size_t off_xb, off_xl, off_qb, off_ql, fixed;
    int64_t npad;
};

TcLayout tc_layout(const GmmLayout& L, int64_t n, int k) {
    TcLayout T;
    T.npad = ((n + TM - 1) / TM) * TM;
    const size_t xbytes = a1024((size_t)T.npad * TDP * 2), qbytes = a1024((size_t)k * TDP * TDP * 2);
    T.off_xb = a1024(L.fixed);
    T.off_xl = T.off_xb + xbytes;
    T.off_qb = T.off_xl + xbytes;
    T.off_ql = T.off_qb + qbytes;
    T.fixed = T.off_ql + qbytes;
    return T;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            (void)cudaGetLastError();
    });
    return fn;
}

// 2-D bf16 tensor [rows][128], box 64 x box_rows, 128-byte swizzle.
bool make_map(CUtensorMap* m, const void* base, int64_t rows, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)TDP, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)TDP * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename K>
bool set_smem_tc(K kern, size_t bytes) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess;
}

int sm_count_tc() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

int convert_inputs(const GmmArgs& A, const GmmLayout& L, const TcLayout& T, char* ws, cudaStream_t s) {
    const unsigned g = (unsigned)sm_count_tc() * 8;
    GPA_LAUNCH("gmm_tc_convert_x", s,
               tc_convert_x_kernel<<<g, 256, 0, s>>>(A.x, A.n, A.d, (__nv_bfloat16*)(ws + T.off_xb),
                                                     (__nv_bfloat16*)(ws + T.off_xl)));
    GPA_LAUNCH("gmm_tc_convert_q", s,
               tc_convert_q_kernel<<<g, 256, 0, s>>>((const float*)(ws + L.off_rec), A.k,
                                                     (__nv_bfloat16*)(ws + T.off_qb),
                                                     (__nv_bfloat16*)(ws + T.off_ql)));
    return GPA_OK;
}

int launch_tc_fwd(const GmmArgs& A, const GmmLayout& L, const TcLayout& T, char* ws, int64_t row0, int64_t n_local,
                  float* lj, int64_t lj_ld, float* lse, cudaStream_t s) {
    CUtensorMap tmx, tmxl, tmq, tmql;
    if (!make_map(&tmx, ws + T.off_xb, A.n, TM) || !make_map(&tmxl, ws + T.off_xl, A.n, TM) ||
        !make_map(&tmq, ws + T.off_qb, (int64_t)A.k * TDP, TDP) ||
        !make_map(&tmql, ws + T.off_ql, (int64_t)A.k * TDP, TDP))
        return GPA_ERR_CUDA;
    if (!set_smem_tc(gmm_tc_fwd_kernel, FwdSm::SMEM)) return GPA_ERR_CUDA;
    const int64_t tiles = (n_local + TM - 1) / TM;
    GPA_LAUNCH("gmm_tc_fwd", s,
               gmm_tc_fwd_kernel<<<(unsigned)tiles, 192, FwdSm::SMEM, s>>>(
                   tmx, tmxl, tmq, tmql, (const float*)(ws + L.off_rec), n_local, row0, A.k, lj, lj_ld, lse,
                   (double*)(ws + L.off_fwd), row0 / TM, A.status));
    return GPA_OK;
}

int tc_bwd_chunks(int k, int64_t ntiles) {
    const int slots = sm_count_tc();  // one CTA per SM (all of TMEM)
    const int groups = (k + BGC - 1) / BGC;
    int best = 1;
    double best_eff = -1.0;
    for (int c = 1; c <= kGmmMaxChunks && c <= ntiles; ++c) {
        const int64_t total = (int64_t)groups * c;
        const int64_t waves = (total + slots - 1) / slots;
        const double eff = (double)total / (double)(waves * slots);
        if (eff > best_eff + 0.02 || (total < slots && eff > best_eff)) {
            best_eff = eff;
            best = c;
        }
    }
    return best;
}

int launch_tc_bwd(const GmmArgs& A, const GmmLayout& L, const TcLayout& T, char* ws, int64_t row0, int64_t n_local,
                  const float* lj, int64_t lj_ld, const float* lse, int nchunks, cudaStream_t s) {
    if (!set_smem_tc(gmm_tc_bwd_kernel, BwdSm::SMEM)) return GPA_ERR_CUDA;
    const int64_t ntiles = (n_local + TM - 1) / TM;
    const int64_t tpc = (ntiles + nchunks - 1) / nchunks;
    dim3 grid((A.k + BGC - 1) / BGC, nchunks);
    GPA_LAUNCH("gmm_tc_bwd", s,
               gmm_tc_bwd_kernel<<<grid, BTHREADS, BwdSm::SMEM, s>>>(
                   A.x + row0 * A.d, n_local, A.k, A.mu, A.d, lj, lj_ld, lse,
                   (float)A.seed, tpc, (float*)(ws + L.off_bS), (float*)(ws + L.off_bM),
                   gmm_bwd_partial_entries(TDP), A.status));
    return GPA_OK;
}

}  // namespace

bool gmm_tc_supported(int d) { return d > 64 && d <= 128; }

size_t gmm_tc_extra_bytes(int64_t n, int d, int k) {
    (void)d;
    const int64_t npad = ((n + TM - 1) / TM) * TM;
    return 2 * a1024((size_t)npad * TDP * 2) + 2 * a1024((size_t)k * TDP * TDP * 2) + 2048;
}

int gmm_tc_objective_run(const GmmArgs& A, const GmmLayout& L, char* ws, size_t ws_bytes, cudaStream_t s) {
    const TcLayout T = tc_layout(L, A.n, A.k);
    if (ws_bytes < T.fixed) return GPA_ERR_WORKSPACE;
    int rc = gmm_run_prep(A, L, ws, s);
    if (rc) return rc;
    if ((rc = convert_inputs(A, L, T, ws, s))) return rc;
    if ((rc = launch_tc_fwd(A, L, T, ws, 0, A.n, A.lj_out, A.n, A.lse_out, s))) return rc;
    return gmm_run_objective(A, L, ws, s);
}

int gmm_tc_vjp_run(const GmmArgs& A, const GmmLayout& L, char* ws, size_t ws_bytes, cudaStream_t s) {
    const TcLayout T = tc_layout(L, A.n, A.k);
    if (ws_bytes < T.fixed) return GPA_ERR_WORKSPACE;
    const int64_t ntiles = (A.n + TM - 1) / TM;
    const int nchunks = tc_bwd_chunks(A.k, ntiles);
    const int nent = gmm_bwd_partial_entries(TDP);
    if (cudaMemsetAsync(ws + L.off_bS, 0, sizeof(float) * (size_t)nchunks * A.k * nent, s) != cudaSuccess ||
        cudaMemsetAsync(ws + L.off_bM, 0, sizeof(float) * (size_t)nchunks * A.k * (TDP + 1), s) != cudaSuccess)
        return GPA_ERR_CUDA;
    int rc = gmm_run_prep(A, L, ws, s);
    if (rc) return rc;
    if ((rc = convert_inputs(A, L, T, ws, s))) return rc;
    if (A.lj_in) {
        if ((rc = launch_tc_bwd(A, L, T, ws, 0, A.n, A.lj_in, A.n, A.lse_in, nchunks, s))) return rc;
        if (A.out && (rc = gmm_run_lse_sum(A.lse_in, A.n, L, ws, s))) return rc;
    } else {
        // log-joint chunk after the tensor-core area, as large as the workspace allows
        const size_t avail = ws_bytes > T.fixed + 2048 ? ws_bytes - T.fixed - 2048 : 0;
        int64_t P = (int64_t)(avail / (sizeof(float) * (size_t)(A.k + 1)));
        P = (P / TM) * TM;
        if (P > T.npad) P = T.npad;
        if (P < TM) return GPA_ERR_WORKSPACE;
        float* lse = (float*)(ws + a1024(T.fixed));
        float* lj = (float*)(ws + a1024(T.fixed) + a1024(sizeof(float) * (size_t)P));
        for (int64_t c0 = 0; c0 < A.n; c0 += P) {
            const int64_t nl = min64(P, A.n - c0);
            // lj / lse are chunk-local: the forward writes them at p0 + row, p0 local
            if ((rc = launch_tc_fwd(A, L, T, ws, c0, nl, lj, P, lse, s))) return rc;
            if ((rc = launch_tc_bwd(A, L, T, ws, c0, nl, lj, P, lse, nchunks, s))) return rc;
        }
    }
    if ((rc = gmm_run_finalize(A, L, ws, nchunks, 1, s))) return rc;
    if (A.out) return gmm_run_objective(A, L, ws, s);
    return GPA_OK;
}

}  // namespace gpa
