// Gaussian mixture on the tensor cores (GPA_PREC_BF16_TC): the two dense
// contractions run as tcgen05 MMAs with BF16 operands in shared memory and FP32
// accumulators in tensor memory; logsumexp, exponentials and every sum over
// points stay FP32 / FP64 on the CUDA cores. Padded dimension TDP = 64
// (32 < D <= 64) or 128 (64 < D <= 128). Every MMA is M = N = 128: with TDP = 64
// two components share one 128-row operand (CPR = 128 / TDP components per
// block of rows).
//
// Forward (A1): Z = X Q_k^T per 128-point tile, with split-BF16 operands:
// x = x_hi + x_lo and Q = Q_hi + Q_lo (each part BF16), and three MMAs per K
// step (hi*hi + lo*hi + hi*lo), which keeps about 16 bits of the FP32 inputs --
// a single BF16 pass leaves log-joint errors of ~0.4 at D = 128, i.e. ~40 %
// errors in the responsibilities exp(s - lse). Warp roles in a 192-thread CTA:
// warp 0 issues TMA loads (the point tile once, then each round's Q rows and
// the b_k / constants through a ring of FQ stages: four at TDP = 64, two at
// TDP = 128, where shared memory holds no more), warp 1 owns the TMEM allocation
// and one of its lanes issues the MMAs (M=128 points, N=128 rows of CPR
// components, K=TDP in steps of 16, 3 passes each) into a double-buffered
// accumulator, warps 2-5 read the accumulator back (TMEM lane = point, one
// thread per point) and fold |z - b_k|^2 into the log-joint and an online
// logsumexp.
//
// Backward (A2): the Accum sums of a component, centred on its mean,
//   C_k = sum_i r_ik (x_i - mu_k)(x_i - mu_k)^T,  m'_k = sum_i r_ik (x_i - mu_k),
//   R_k = sum_i r_ik,
// with C_k = U_k^T U_k for U_k[p][a] = sqrt(r_pk) (x_p - mu_k)[a] (x read in
// FP32, U rounded once to BF16; r from the forward's log-joint). Sixteen
// producer warps build the 128-row blocks [U_k^T; ...] (CPR components stacked,
// points contiguous) directly in the 128-byte-swizzled layout the MMA reads; one
// MMA thread accumulates D += U^T U (A and B the same tile) in TMEM for four
// blocks across every tile of a point chunk, of which the diagonal TDP x TDP
// blocks are the C_k. The partial sums go to the same buffers the FP32 finalize
// reads (centred mode).
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

constexpr int TM = 128;                          // points per tile; rows of every MMA operand
constexpr uint32_t ATOM = TM * 128;              // one 64-wide K slice of a 128-row operand: 16 KB
constexpr uint32_t IDESC = tc::idesc_bf16_f32(128, 128);

template <int TDP>
struct Tc {
    static constexpr int NA = TDP / 64;                  // 64-wide K slices per row
    static constexpr int CPR = 128 / TDP;                // components per 128-row block
    static constexpr uint32_t TILE = NA * ATOM;          // a 128-row operand of K = TDP
    static constexpr int REC = TDP * TDP + TDP + 4;      // FP32 prep record (b at TDP*TDP, cst after)
    static constexpr uint32_t TAIL = (TDP + 4) * 4;      // b_k, constant, pad
};

// The dynamic shared array advanced to the next 1024-byte boundary (the
// 128-byte swizzle atoms need it). The offset is added to the shared array
// itself, so that the compiler keeps the pointer in the shared address space
// and accesses through it stay shared-memory instructions.
__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
    return p + ((1024u - (smem_u32(p) & 1023u)) & 1023u);
}

// ---- forward ------------------------------------------------------------------
template <int TDP>
struct FwdSm {
    using T = Tc<TDP>;
    // Q stages (hi and lo parts and the b_k tails each). A stage is refilled
    // only after the epilogue has read its tails, so the ring must cover the
    // epilogue's lag plus a TMA round trip: four stages where shared memory
    // allows (TDP = 64), two at TDP = 128.
    static constexpr int FQ = TDP == 64 ? 4 : 2;
    static constexpr uint32_t X = 0;                            // x_hi, x_lo tiles
    static constexpr uint32_t Q = X + 2 * T::TILE;              // [FQ] x (Q_hi, Q_lo)
    static constexpr uint32_t B = Q + FQ * 2 * T::TILE;         // [FQ][CPR] tails
    static constexpr uint32_t RED = B + FQ * T::CPR * T::TAIL;
    static constexpr uint32_t BAR = RED + 8 * 8;  // x_full, q_full[FQ], q_empty[FQ], acc_full[2], acc_empty[2]
    static_assert(1 + 2 * FQ + 4 <= 16, "barrier slots");
    static constexpr uint32_t TMEMP = BAR + 16 * 8;
    static constexpr uint32_t FLAG = TMEMP + 8;
    static constexpr uint32_t END = FLAG + 8;
    static constexpr size_t SMEM = END + 1024;  // + alignment slack
    static_assert(SMEM <= 227 * 1024, "forward shared memory");
};

template <int TDP>
__global__ void __launch_bounds__(192, 1)
    gmm_tc_fwd_kernel(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmxl,
                      const __grid_constant__ CUtensorMap tmq, const __grid_constant__ CUtensorMap tmql,
                      const float* __restrict__ rec, int64_t n, int64_t xrow0, int k, float* __restrict__ lj,
                      int64_t lj_ld, float* __restrict__ lse_out, double* __restrict__ part, int64_t tile0,
                      int32_t* __restrict__ status) {
    using T = Tc<TDP>;
    using S = FwdSm<TDP>;
    constexpr int FQ = S::FQ;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = align1024(smem_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + S::BAR);
    uint64_t* x_full = bars;
    uint64_t* q_full = bars + 1;
    uint64_t* q_empty = bars + 1 + FQ;
    uint64_t* acc_full = bars + 1 + 2 * FQ;
    uint64_t* acc_empty = bars + 3 + 2 * FQ;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(sm + S::TMEMP);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + S::FLAG);
    double* red = reinterpret_cast<double*>(sm + S::RED);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t p0 = (int64_t)blockIdx.x * TM;
    const int rounds = (k + T::CPR - 1) / T::CPR;

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
            mbar_arrive_expect_tx(x_full, 2 * T::TILE);
            for (int a = 0; a < T::NA; ++a) {
                tc::tma_load_2d(sm + S::X + a * ATOM, &tmx, 64 * a, (int)(xrow0 + p0), x_full);
                tc::tma_load_2d(sm + S::X + T::TILE + a * ATOM, &tmxl, 64 * a, (int)(xrow0 + p0), x_full);
            }
            for (int r = 0; r < rounds; ++r) {
                const int s = r % FQ;
                const uint32_t ph = (uint32_t)(r / FQ) & 1u;
                if (!mbar_wait(&q_empty[s], ph ^ 1u, status)) {
                    *abort_flag = 1;
                    break;
                }
                const int c0 = r * T::CPR;
                const int nc = min(T::CPR, k - c0);
                mbar_arrive_expect_tx(&q_full[s], 2 * T::TILE + nc * T::TAIL);
                uint8_t* qd = sm + S::Q + s * 2 * T::TILE;
                for (int a = 0; a < T::NA; ++a) {
                    tc::tma_load_2d(qd + a * ATOM, &tmq, 64 * a, r * TM, &q_full[s]);
                    tc::tma_load_2d(qd + T::TILE + a * ATOM, &tmql, 64 * a, r * TM, &q_full[s]);
                }
                for (int j = 0; j < nc; ++j)
                    bulk_g2s(sm + S::B + (s * T::CPR + j) * T::TAIL, rec + (size_t)(c0 + j) * T::REC + TDP * TDP,
                             T::TAIL, &q_full[s]);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            bool ok = mbar_wait(x_full, 0, status);
            for (int r = 0; ok && r < rounds; ++r) {
                const int s = r % FQ;
                const uint32_t ph = (uint32_t)(r / FQ) & 1u;
                const int as = r & 1;
                const uint32_t aph = (uint32_t)(r >> 1) & 1u;
                if (!mbar_wait(&q_full[s], ph, status) || !mbar_wait(&acc_empty[as], aph ^ 1u, status)) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t xh = smem_u32(sm + S::X), xl = xh + T::TILE;
                const uint32_t qh = smem_u32(sm + S::Q + s * 2 * T::TILE), ql = qh + T::TILE;
                const uint32_t dt = tmem + (uint32_t)(as * TM);
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
        for (int r = 0; r < rounds; ++r) {
            const int s = r % FQ;
            const int as = r & 1;
            const uint32_t aph = (uint32_t)(r >> 1) & 1u;
            if (!mbar_wait_warp(&acc_full[as], aph, status)) {
                *abort_flag = 1;
                break;
            }
            tc::fence_after_sync();
            float sv[Tc<TDP>::CPR], cst[Tc<TDP>::CPR];
            // |z - b|^2 per component: z - b and the squares as packed pairs into
            // four independent partial sums (no serial chain through one register)
            const float2 neg1 = make_float2(-1.f, -1.f);
#pragma unroll
            for (int j = 0; j < T::CPR; ++j) {
                const float* bb = reinterpret_cast<const float*>(sm + S::B + (s * T::CPR + j) * T::TAIL);
                float2 acc[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f),
                                 make_float2(0.f, 0.f)};
#pragma unroll
                for (int h = 0; h < TDP / 64; ++h) {  // 64 columns: two loads in flight, one wait
                    float v[2][32];
                    tc::tmem_ld64_wait(tmem + ((uint32_t)(qtr * 32) << 16) + (uint32_t)(as * TM + j * TDP + h * 64),
                                       v[0], v[1]);
#pragma unroll
                    for (int ch = 0; ch < 2; ++ch)
#pragma unroll
                        for (int i = 0; i < 32; i += 4) {
                            const float4 b4 = *reinterpret_cast<const float4*>(bb + h * 64 + ch * 32 + i);
                            const float2 z0 =
                                __ffma2_rn(make_float2(b4.x, b4.y), neg1, make_float2(v[ch][i], v[ch][i + 1]));
                            const float2 z1 =
                                __ffma2_rn(make_float2(b4.z, b4.w), neg1, make_float2(v[ch][i + 2], v[ch][i + 3]));
                            acc[(i >> 2) & 1] = __ffma2_rn(z0, z0, acc[(i >> 2) & 1]);
                            acc[2 + ((i >> 2) & 1)] = __ffma2_rn(z1, z1, acc[2 + ((i >> 2) & 1)]);
                        }
                }
                const float2 t = __fadd2_rn(__fadd2_rn(acc[0], acc[1]), __fadd2_rn(acc[2], acc[3]));
                sv[j] = t.x + t.y;
                cst[j] = bb[TDP];
            }
            // The stage's b_k tail was read through the generic proxy and the
            // producer refills it with a bulk copy (async proxy) once q_empty
            // completes: order the reads before that write.
            fence_proxy_async_smem();
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) {
                tc::mbar_arrive(&acc_empty[as]);
                tc::mbar_arrive(&q_empty[s]);
            }
#pragma unroll
            for (int j = 0; j < T::CPR; ++j) {
                const int kk = r * T::CPR + j;
                if (kk < k && valid) {
                    const float v = cst[j] - 0.5f * sv[j];
                    if (lj) lj[(int64_t)kk * lj_ld + p0 + row] = v;
                    st.add(v);
                }
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
constexpr int BSLOT = 4;                        // 128-row blocks per CTA (4 x 128 TMEM columns)
constexpr int BPROD = 512;                      // producer threads (16 warps, a quarter of the points each)
constexpr int BTHREADS = BPROD + 32;            // + the MMA warp
template <int TDP>
struct BwdSm {
    static constexpr int BGC = BSLOT * Tc<TDP>::CPR;                // components per CTA
    static constexpr int NUB = 4;                                   // U buffers (cycled over the 4 blocks)
    static constexpr uint32_t U = 0;                                // [NUB] tiles of 32 KB
    static constexpr uint32_t XS = U + NUB * 2 * ATOM;              // point tile [TM][d] float
    static constexpr uint32_t LJ = XS + TM * TDP * 4;               // log-joint [2][BGC][TM] float
    static constexpr uint32_t LS = LJ + 2 * BGC * TM * 4;           // lse [2][TM] float
    static constexpr uint32_t SR = LS + 2 * TM * 4;                 // sqrt(r) [BGC][TM] float
    static constexpr uint32_t MU = SR + BGC * TM * 4;               // mu [BSLOT][128] float
    static constexpr uint32_t MRED = MU + BSLOT * 128 * 4;          // m' of quarters 1..3 [3][BSLOT][128] float
    static constexpr uint32_t RSUM = MRED + 3 * BSLOT * 128 * 4;    // R per component [BGC] float
    static constexpr uint32_t BAR = RSUM + BGC * 4;                 // u_full[NUB], u_empty[NUB], done
    static constexpr uint32_t TMEMP = BAR + 16 * 8;
    static constexpr uint32_t FLAG = TMEMP + 8;  // abort flag, then the producers' decision slot
    static constexpr uint32_t END = FLAG + 8;
    static constexpr size_t SMEM = END + 1024;
    static_assert(SMEM <= 227 * 1024, "backward shared memory");
};

__device__ __forceinline__ void producers_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(BPROD) : "memory");
}

template <int TDP>
__global__ void __launch_bounds__(BTHREADS, 1)
    gmm_tc_bwd_kernel(const float* __restrict__ x, int64_t n, int k, const float* __restrict__ mu,
                      int d, const float* __restrict__ lj, int64_t lj_ld, const float* __restrict__ lse,
                      float seed, int64_t tiles_per_chunk, float* __restrict__ partS, float* __restrict__ partM,
                      int nblk64, int32_t* __restrict__ status) {
    using T = Tc<TDP>;
    using S = BwdSm<TDP>;
    constexpr int BGC = S::BGC, NUB = S::NUB;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = align1024(smem_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + S::BAR);
    uint64_t* u_full = bars;
    uint64_t* u_empty = bars + NUB;
    uint64_t* done = bars + 2 * NUB;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(sm + S::TMEMP);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + S::FLAG);
    float* xs = reinterpret_cast<float*>(sm + S::XS);
    float* ljs = reinterpret_cast<float*>(sm + S::LJ);
    float* lss = reinterpret_cast<float*>(sm + S::LS);
    float* sr = reinterpret_cast<float*>(sm + S::SR);
    float* mus = reinterpret_cast<float*>(sm + S::MU);
    float* mred = reinterpret_cast<float*>(sm + S::MRED);
    float* rsum = reinterpret_cast<float*>(sm + S::RSUM);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tid = threadIdx.x;
    const int kg0 = blockIdx.x * BGC;
    const int64_t ntiles = (n + TM - 1) / TM;
    const int64_t t_begin = (int64_t)blockIdx.y * tiles_per_chunk;
    const int64_t t_end = min64(ntiles, t_begin + tiles_per_chunk);

    if (tid == 0) {
        for (int c = 0; c < NUB; ++c) {
            mbar_init(&u_full[c], BPROD / 32);
            mbar_init(&u_empty[c], 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    // mean of the component owning row a' of block c
    for (int e = tid; e < BSLOT * 128; e += BTHREADS) {
        const int c = e / 128, ar = e % 128;
        const int kg = kg0 + c * T::CPR + ar / TDP, a = ar % TDP;
        mus[e] = (kg < k && a < d) ? mu[(size_t)kg * d + a] : 0.f;
    }
    for (int e = tid; e < BGC; e += BTHREADS) rsum[e] = 0.f;
    if (warp == BPROD / 32) {
        tc::tmem_alloc(tmem_holder, 512);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_holder;

    if (warp == BPROD / 32) {
        // MMA issuer: block c of tile `it` uses U buffer c % NUB, its use number
        // u = it * (BSLOT / NUB) + c / NUB giving the barrier phases
        if (lane == 0) {
            bool ok = true;
            int it = 0;
            for (int64_t t = t_begin; ok && t < t_end; ++t, ++it) {
                for (int c = 0; c < BSLOT; ++c) {
                    const int b = c % NUB;
                    const uint32_t use = (uint32_t)(it * (BSLOT / NUB) + c / NUB);
                    if (!mbar_wait(&u_full[b], use & 1u, status)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t ua = smem_u32(sm + S::U + b * 2 * ATOM);
#pragma unroll
                    for (int j = 0; j < TM / 16; ++j) {
                        const uint64_t dsc = tc::desc_sw128(ua + (uint32_t)(j >> 2) * ATOM + (uint32_t)(j & 3) * 32u);
                        tc::mma_bf16(tmem + (uint32_t)(c * 128), dsc, dsc, IDESC, (it > 0 || j > 0) ? 1u : 0u);
                    }
                    tc::mma_commit(&u_empty[b]);
                }
            }
            if (!ok) *abort_flag = 1;
            tc::mma_commit(done);
        }
        __syncwarp();
    } else {
        // producers: thread owns row a' of every block (component a'/TDP of the
        // block, dimension a'%TDP) and a quarter of the tile's points. Tile t+1
        // (points, log-joint, lse) is copied into shared memory while tile t is
        // built: the point tile has one buffer, free once every thread holds its
        // column of it in registers.
        const int ar = tid & 127;
        const int jr = ar / TDP, a = ar % TDP;
        const int qp = tid >> 7;  // points 32 qp .. 32 qp + 31 of the tile
        const bool vec = ((d & 3) == 0) && ((reinterpret_cast<uintptr_t>(x) & 15) == 0);
        auto issue = [&](int64_t t, int buf) {
            const int64_t p0 = t * TM;
            const int nv = (int)min64(TM, n - p0);
            float* X = xs;
            const float* src = x + p0 * d;
            if (vec) {
                for (int e = tid; e < nv * d / 4; e += BPROD) cp_async16(X + 4 * e, src + 4 * e);
            } else {
                for (int e = tid; e < nv * d; e += BPROD) cp_async4(X + e, src + e);
            }
            float* L = ljs + buf * BGC * TM;
            for (int e = tid; e < BGC * TM; e += BPROD) {
                const int c = e / TM, p = e % TM;
                if (p < nv && kg0 + c < k) cp_async4(L + e, lj + (int64_t)(kg0 + c) * lj_ld + p0 + p);
            }
            for (int p = tid; p < nv; p += BPROD) cp_async4(lss + buf * TM + p, lse + p0 + p);
        };
        float2 macc[BSLOT];  // m' of this thread's row per block, two partial sums
#pragma unroll
        for (int c = 0; c < BSLOT; ++c) macc[c] = make_float2(0.f, 0.f);
        float racc[BGC * TM / BPROD];
#pragma unroll
        for (int u = 0; u < BGC * TM / BPROD; ++u) racc[u] = 0.f;
        volatile int* decision = abort_flag + 1;  // written by thread 0 before a barrier, read after it
        if (t_begin < t_end) issue(t_begin, 0);
        cp_async_commit();
        int it = 0;
        for (int64_t t = t_begin; t < t_end; ++t, ++it) {
            const int buf = it & 1;
            const int64_t p0 = t * TM;
            cp_async_wait_all();  // this thread's copies of tile t have landed
            if (tid == 0) *decision = *abort_flag;
            // every thread's copies of tile t are visible, every thread is done with
            // tile t-1 (its sqrt(r) may be overwritten); decision published
            producers_sync();
            if (*decision) break;  // uniform over all producer threads
            const float* X = xs;
            const float* L = ljs + buf * BGC * TM;
            const float* Ls = lss + buf * TM;
#pragma unroll
            for (int u = 0; u < BGC * TM / BPROD; ++u) {
                const int e = tid + u * BPROD;
                const int c = e / TM, p = e % TM;
                float v = 0.f;
                if (p0 + p < n && kg0 + c < k) v = expf(0.5f * (L[e] - Ls[p]));
                sr[e] = v;
                racc[u] += v * v;
            }
            // x values of this thread: points p0 + 32 qp + 0..31, dimension a (0 past
            // the end), as pairs of consecutive points
            float2 xv[16];
            if (a < d && p0 + TM <= n) {  // a full tile: no per-point tests
                const float* xa = X + qp * 32 * d + a;
#pragma unroll
                for (int j = 0; j < 16; ++j) xv[j] = make_float2(xa[(2 * j) * d], xa[(2 * j + 1) * d]);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int p = qp * 32 + 2 * j;
                    xv[j] = make_float2((p0 + p < n && a < d) ? X[p * d + a] : 0.f,
                                        (p0 + p + 1 < n && a < d) ? X[(p + 1) * d + a] : 0.f);
                }
            }
            producers_sync();     // sqrt(r) of tile t complete, the point tile read by all
            if (t + 1 < t_end) issue(t + 1, buf ^ 1);  // log-joint buffer buf ^ 1 last read in tile t-1
            cp_async_commit();
#pragma unroll 1
            for (int c = 0; c < BSLOT; ++c) {
                const int b = c % NUB;
                const uint32_t use = (uint32_t)(it * (BSLOT / NUB) + c / NUB);
                // sqrt(r) of this block's 32 points and the mean, loaded before the
                // wait for the U buffer so that the wait covers their latency
                const float4* src = reinterpret_cast<const float4*>(sr + (c * T::CPR + jr) * TM + qp * 32);
                float4 sv4[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) sv4[q] = src[q];
                const float mcs = mus[c * 128 + ar];
                if (!mbar_wait_warp(&u_empty[b], (use & 1u) ^ 1u, status)) {
                    *abort_flag = 1;  // skip the work; the next decision point stops every warp
                    continue;
                }
                // points 32 qp .. +31 are chunks 4 (qp & 1) .. +3 of K atom qp >> 1
                uint8_t* ut = sm + S::U + b * 2 * ATOM + (qp >> 1) * ATOM;
                const float2 mc = make_float2(mcs, mcs);
                // u = sqrt(r) (x - mu) for two points per packed op; m' += sqrt(r) u in
                // four independent partial sums (no serial chain through the slot)
                float2 mq[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f),
                                make_float2(0.f, 0.f)};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float4 sa = sv4[2 * j], sb = sv4[2 * j + 1];
                    const float2 sp[4] = {make_float2(sa.x, sa.y), make_float2(sa.z, sa.w), make_float2(sb.x, sb.y),
                                          make_float2(sb.z, sb.w)};
                    uint32_t w4[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float2 u = __fmul2_rn(sp[i], __fadd2_rn(xv[4 * j + i], make_float2(-mc.x, -mc.y)));
                        mq[i] = __ffma2_rn(sp[i], u, mq[i]);
                        w4[i] = tc::pack_bf16x2(u.x, u.y);
                    }
                    *reinterpret_cast<uint4*>(ut + tc::sw128_offset((uint32_t)ar, (uint32_t)(4 * (qp & 1) + j))) =
                        make_uint4(w4[0], w4[1], w4[2], w4[3]);
                }
                macc[c] = __fadd2_rn(macc[c], __fadd2_rn(__fadd2_rn(mq[0], mq[1]), __fadd2_rn(mq[2], mq[3])));
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&u_full[b]);
            }
        }
        cp_async_wait_all();  // no copy may land after the block exits
        // m' of quarters 1..3 for quarter 0 to add
        if (qp > 0)
            for (int c = 0; c < BSLOT; ++c) mred[(qp - 1) * BSLOT * 128 + c * 128 + ar] = macc[c].x + macc[c].y;
        // R per component
#pragma unroll
        for (int u = 0; u < BGC * TM / BPROD; ++u) {
            const float rv = warp_sum(racc[u]);
            if (lane == 0) atomicAdd(&rsum[(tid + u * BPROD) / TM], rv);
        }
        producers_sync();
        const int64_t cbase = (int64_t)blockIdx.y * k;
        if (qp == 0) {
            for (int c = 0; c < BSLOT; ++c) {
                const int kg = kg0 + c * T::CPR + jr;
                if (kg >= k) continue;
                float* M = partM + (cbase + kg) * (TDP + 1);
                const float* mr = mred + c * 128 + ar;
                M[a] += seed * ((macc[c].x + macc[c].y) + mr[0] + mr[BSLOT * 128] + mr[2 * BSLOT * 128]);
                if (a == 0) M[TDP] += seed * rsum[c * T::CPR + jr];
            }
        }
        // accumulators: warp w reads TMEM lanes of its quarter w % 4 for block w / 4;
        // row a' = lane index, the component's columns are [jr*TDP, jr*TDP + TDP)
        const bool fin = mbar_wait_warp(done, 0, status);
        if (!fin) *abort_flag = 1;
        tc::fence_after_sync();
        producers_sync();  // every warp has seen `done` (or given up) before reading the flag
        const int aborted = __shfl_sync(0xffffffffu, *abort_flag, 0);  // one value per warp
        if (!aborted && t_begin < t_end) {  // a CTA without tiles issued no MMA: TMEM holds nothing
            const int qtr = warp & 3;
            const int row = qtr * 32 + lane;      // row a' of the block
            const int jw = row / TDP, aw = row % TDP;  // the same jw for the whole warp
            const int c = warp >> 2;
            const int kg = kg0 + c * T::CPR + jw;
            if (kg < k) {
                float* Sp = partS + (cbase + kg) * (int64_t)nblk64;
#pragma unroll 1
                for (int ch = 0; ch < TDP / 32; ++ch) {
                    float v[32];
                    tc::tmem_ld32_wait(tmem + ((uint32_t)(qtr * 32) << 16) + (uint32_t)(c * 128 + jw * TDP + ch * 32), v);
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const int b = ch * 32 + i;
                        if (b <= aw) {
                            const int A = aw >> 3, B = b >> 3;
                            Sp[(A * (A + 1) / 2 + B) * 64 + (aw & 7) * 8 + (b & 7)] += seed * v[i];
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
// x [n][d] float -> x_hi + x_lo, each [n][TDP] bf16, zero padded
template <int TDP>
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
template <int TDP>
__global__ void __launch_bounds__(256) tc_convert_q_kernel(const float* __restrict__ rec, int k,
                                                           __nv_bfloat16* __restrict__ qb,
                                                           __nv_bfloat16* __restrict__ ql) {
    const int64_t total = (int64_t)k * TDP * TDP;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        const int64_t kk = e / (TDP * TDP);
        const int r = (int)((e / TDP) % TDP), c = (int)(e % TDP);
        const float v = rec[kk * Tc<TDP>::REC + (int64_t)c * TDP + r];
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        qb[e] = h;
        ql[e] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

// ---- host ---------------------------------------------------------------------------
size_t a1024(size_t v) { return (v + 1023) & ~(size_t)1023; }

int tc_dp(int d) { return d <= 64 ? 64 : 128; }

struct TcLayout {
    size_t off_xb, off_xl, off_qb, off_ql, fixed;
    int64_t npad;
};

TcLayout tc_layout(const GmmLayout& L, int64_t n, int d, int k) {
    const int tdp = tc_dp(d);
    TcLayout T;
    T.npad = ((n + TM - 1) / TM) * TM;
    const size_t xbytes = a1024((size_t)T.npad * tdp * 2), qbytes = a1024((size_t)k * tdp * tdp * 2);
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

// 2-D bf16 tensor [rows][tdp], box 64 x 128 rows, 128-byte swizzle.
bool make_map(CUtensorMap* m, const void* base, int64_t rows, int tdp) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)tdp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)tdp * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)TM};
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

template <int TDP>
int convert_inputs(const GmmArgs& A, const GmmLayout& L, const TcLayout& T, char* ws, cudaStream_t s) {
    const unsigned g = (unsigned)sm_count_tc() * 8;
    GPA_LAUNCH("gmm_tc_convert_x", s,
               tc_convert_x_kernel<TDP><<<g, 256, 0, s>>>(A.x, A.n, A.d, (__nv_bfloat16*)(ws + T.off_xb),
                                                          (__nv_bfloat16*)(ws + T.off_xl)));
    GPA_LAUNCH("gmm_tc_convert_q", s,
               tc_convert_q_kernel<TDP><<<g, 256, 0, s>>>((const float*)(ws + L.off_rec), A.k,
                                                          (__nv_bfloat16*)(ws + T.off_qb),
                                                          (__nv_bfloat16*)(ws + T.off_ql)));
    return GPA_OK;
}

template <int TDP>
int launch_tc_fwd(const GmmArgs& A, const GmmLayout& L, const TcLayout& T, char* ws, int64_t row0, int64_t n_local,
                  float* lj, int64_t lj_ld, float* lse, cudaStream_t s) {
    CUtensorMap tmx, tmxl, tmq, tmql;
    if (!make_map(&tmx, ws + T.off_xb, A.n, TDP) || !make_map(&tmxl, ws + T.off_xl, A.n, TDP) ||
        !make_map(&tmq, ws + T.off_qb, (int64_t)A.k * TDP, TDP) ||
        !make_map(&tmql, ws + T.off_ql, (int64_t)A.k * TDP, TDP))
        return GPA_ERR_CUDA;
    auto kern = gmm_tc_fwd_kernel<TDP>;
    if (!set_smem_tc(kern, FwdSm<TDP>::SMEM)) return GPA_ERR_CUDA;
    const int64_t tiles = (n_local + TM - 1) / TM;
    GPA_LAUNCH("gmm_tc_fwd", s,
               kern<<<(unsigned)tiles, 192, FwdSm<TDP>::SMEM, s>>>(
                   tmx, tmxl, tmq, tmql, (const float*)(ws + L.off_rec), n_local, row0, A.k, lj, lj_ld, lse,
                   (double*)(ws + L.off_fwd), row0 / TM, A.status));
    return GPA_OK;
}

int tc_bwd_chunks(int k, int bgc, int64_t ntiles) {
    const int slots = sm_count_tc();  // one CTA per SM (all of TMEM)
    const int groups = (k + bgc - 1) / bgc;
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

template <int TDP>
int launch_tc_bwd(const GmmArgs& A, const GmmLayout& L, char* ws, int64_t row0, int64_t n_local, const float* lj,
                  int64_t lj_ld, const float* lse, int nchunks, cudaStream_t s) {
    auto kern = gmm_tc_bwd_kernel<TDP>;
    if (!set_smem_tc(kern, BwdSm<TDP>::SMEM)) return GPA_ERR_CUDA;
    const int64_t ntiles = (n_local + TM - 1) / TM;
    const int64_t tpc = (ntiles + nchunks - 1) / nchunks;
    dim3 grid((A.k + BwdSm<TDP>::BGC - 1) / BwdSm<TDP>::BGC, nchunks);
    GPA_LAUNCH("gmm_tc_bwd", s,
               kern<<<grid, BTHREADS, BwdSm<TDP>::SMEM, s>>>(
                   A.x + row0 * A.d, n_local, A.k, A.mu, A.d, lj, lj_ld, lse, (float)A.seed, tpc,
                   (float*)(ws + L.off_bS), (float*)(ws + L.off_bM), gmm_bwd_partial_entries(TDP), A.status));
    return GPA_OK;
}

template <int TDP>
int objective_run(const GmmArgs& A, const GmmLayout& L, char* ws, size_t ws_bytes, cudaStream_t s) {
    const TcLayout T = tc_layout(L, A.n, A.d, A.k);
    if (ws_bytes < T.fixed) return GPA_ERR_WORKSPACE;
    int rc = gmm_run_prep(A, L, ws, s);
    if (rc) return rc;
    if ((rc = convert_inputs<TDP>(A, L, T, ws, s))) return rc;
    if ((rc = launch_tc_fwd<TDP>(A, L, T, ws, 0, A.n, A.lj_out, A.n, A.lse_out, s))) return rc;
    return gmm_run_objective(A, L, ws, s);
}

template <int TDP>
int vjp_run(const GmmArgs& A, const GmmLayout& L, char* ws, size_t ws_bytes, cudaStream_t s) {
    const TcLayout T = tc_layout(L, A.n, A.d, A.k);
    if (ws_bytes < T.fixed) return GPA_ERR_WORKSPACE;
    const int64_t ntiles = (A.n + TM - 1) / TM;
    const int nchunks = tc_bwd_chunks(A.k, BwdSm<TDP>::BGC, ntiles);
    const int nent = gmm_bwd_partial_entries(TDP);
    if (cudaMemsetAsync(ws + L.off_bS, 0, sizeof(float) * (size_t)nchunks * A.k * nent, s) != cudaSuccess ||
        cudaMemsetAsync(ws + L.off_bM, 0, sizeof(float) * (size_t)nchunks * A.k * (TDP + 1), s) != cudaSuccess)
        return GPA_ERR_CUDA;
    int rc = gmm_run_prep(A, L, ws, s);
    if (rc) return rc;
    if ((rc = convert_inputs<TDP>(A, L, T, ws, s))) return rc;
    if (A.lj_in) {
        if ((rc = launch_tc_bwd<TDP>(A, L, ws, 0, A.n, A.lj_in, A.n, A.lse_in, nchunks, s))) return rc;
        if ((A.out || A.exch_out) && (rc = gmm_run_lse_sum(A.lse_in, A.n, L, ws, s))) return rc;
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
            if ((rc = launch_tc_fwd<TDP>(A, L, T, ws, c0, nl, lj, P, lse, s))) return rc;
            if ((rc = launch_tc_bwd<TDP>(A, L, ws, c0, nl, lj, P, lse, nchunks, s))) return rc;
        }
    }
    if (A.exch_out) return gmm_run_exchange(A, L, ws, nchunks, s);
    if ((rc = gmm_run_finalize(A, L, ws, nchunks, 1, s))) return rc;
    if (A.out) return gmm_run_objective(A, L, ws, s);
    return GPA_OK;
}

}  // namespace

bool gmm_tc_supported(int d) { return d > 32 && d <= 128; }

size_t gmm_tc_extra_bytes(int64_t n, int d, int k) {
    const int tdp = tc_dp(d);
    const int64_t npad = ((n + TM - 1) / TM) * TM;
    return 2 * a1024((size_t)npad * tdp * 2) + 2 * a1024((size_t)k * tdp * tdp * 2) + 2048;
}

int gmm_tc_objective_run(const GmmArgs& A, const GmmLayout& L, char* ws, size_t ws_bytes, cudaStream_t s) {
    return tc_dp(A.d) == 64 ? objective_run<64>(A, L, ws, ws_bytes, s) : objective_run<128>(A, L, ws, ws_bytes, s);
}

int gmm_tc_vjp_run(const GmmArgs& A, const GmmLayout& L, char* ws, size_t ws_bytes, cudaStream_t s) {
    return tc_dp(A.d) == 64 ? vjp_run<64>(A, L, ws, ws_bytes, s) : vjp_run<128>(A, L, ws, ws_bytes, s);
}

}  // namespace gpa
