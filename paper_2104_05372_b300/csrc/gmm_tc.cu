// Gaussian mixture on the tensor cores (GPA_PREC_BF16_TC): the two dense
// contractions run as tcgen05 MMAs with BF16 operands in shared memory and FP32
// accumulators in tensor memory; logsumexp, exponentials and every sum over
// points stay FP32 / FP64 on the CUDA cores. Padded dimension TDP = 64
// (32 < D <= 64) or 128 (64 < D <= 128).
//
// Forward (A1): z_ik = Q_k x_i - b_k for a 128-point tile against every
// component, as N = 256 MMAs over the nonzero blocks of the triangular Q_k with
// split-BF16 operands (gmm_tc_fwd_kernel). Backward (A2): the Accum sums of the
// reverse pass as the single contraction Y^T R over the points
// (gmm_tc_gram_kernel). Each kernel's comment gives its layout and warp roles.
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

template <int TDP>
struct Tc {
    static constexpr int REC = TDP * TDP + TDP + 4;      // FP32 prep record (b at TDP*TDP, cst after)
};

// The dynamic shared array advanced to the next 1024-byte boundary (the
// 128-byte swizzle atoms need it). The offset is added to the shared array
// itself, so that the compiler keeps the pointer in the shared address space
// and accesses through it stay shared-memory instructions.
__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
    return p + ((1024u - (smem_u32(p) & 1023u)) & 1023u);
}

// ---- forward ------------------------------------------------------------------
// Z = X Q_k^T per 128-point tile with split-BF16 operands: x = x_hi + x_lo and
// Q = Q_hi + Q_lo (each part BF16), three products per K step (x_hi Q_hi,
// x_lo Q_hi, x_hi Q_lo), which keeps about 16 bits of the FP32 inputs -- a
// single BF16 pass leaves log-joint errors of ~0.4 at D = 128, i.e. ~40 %
// errors in the responsibilities exp(s - lse).
//
// Q_k is lower triangular, so rows jG .. jG + G - 1 of z = Q_k x (one set)
// need only the first (j + 1) G columns of Q_k. A round takes CR = 256 / G
// components and runs NSET = TDP / G sets: set j stacks rows jG .. of each of
// the round's components into one 256-row MMA operand over K = 0 .. (j + 1) G
// - 1, so the zero blocks above the diagonal blocks are never multiplied. G =
// 16 at TDP = 128 (8 sets, 16 components per round, 9/16 of the dense MMA
// work), G = 32 at TDP = 64 (2 sets, 8 components, 3/4). Every MMA is M = 128
// and N = G nc (nc = the round's components: 256 but in a last, partial
// round), the widest single-CTA shape, so that the one issuing thread stays
// ahead of the tensor pipe.
//
// Pipeline stages are 32 KB operand atoms (256 rows x 64 columns, one TMA
// box), per set its NA_j = ceil((j + 1) G / 64) atoms of Q_hi, then of Q_lo.
// Set j accumulates in TMEM columns 256 (j % 2) .. (component c at 16 c), so
// the epilogue reads one set while the MMAs of the next run. The b_k tails of
// a round travel with its first stage into a ring of FT slots, which the
// epilogue releases; the Q stages are released by the MMAs.
//
// Warp roles (320 threads): warp 0 issues the TMA loads, one lane of warp 1
// the MMAs (warp 1 also owns the TMEM allocation), warps 2-9 read the
// accumulators back, one thread per point (TMEM lane) and half of the round's
// components, and fold |z - b_k|^2 into the log-joint and an online logsumexp.
template <int TDP, bool P = false>
struct FwdSm {
    static constexpr int NA = TDP / 64;                           // 64-wide column atoms of a Q row
    // rows of z per set: 16 (one MMA K step) at TDP = 128; at TDP = 64 sets of
    // 32 rows (two sets, 8 components per round) measured faster (2.39
    // against 2.78 ms at N = 2^20, K = 200): with sets of 16 rows the MMAs
    // of a set take less time than the epilogue's read of the previous one
    static constexpr int G = TDP == 64 ? 32 : 16;
    static constexpr int NSET = TDP / G;                          // sets per round
    static constexpr int CR = 256 / G;                            // components per round
    // column atoms of set j (its stages: these atoms of Q_hi, then of Q_lo)
    static constexpr __host__ __device__ int atoms(int j) { return ((j + 1) * G + 63) / 64; }
    // P: the persistent form (one CTA per SM over many tiles), which keeps two
    // x tiles at TDP = 64 (the next tile's loads while the current one is
    // multiplied) and so one Q stage fewer
    static constexpr int XB = P && TDP == 64 ? 2 : 1;              // x tile buffers
    static constexpr int FQ = TDP == 64 && !P ? 5 : 4;            // Q stages
    // tail slots (rounds): enough that the producer, FQ stages ahead of the
    // MMAs, never waits for the epilogue to finish a round
    static constexpr int FT = G >= 32 ? 4 : 3;
    static constexpr int EW = 8;                                  // epilogue warps
    static constexpr uint32_t XBYTES = 2 * NA * ATOM;             // x_hi, x_lo tiles (NA atoms each)
    static constexpr uint32_t STG = 2 * ATOM;                     // 256 rows x 128 bytes
    static constexpr uint32_t TAIL = (TDP + 4) * 4;               // b_k, constant, pad
    static constexpr uint32_t X = 0;                              // [XB] x tiles
    static constexpr uint32_t Q = X + XB * XBYTES;                // [FQ] stages
    static constexpr uint32_t B = Q + FQ * STG;                   // [FT][CR] tails
    static constexpr uint32_t RED = B + FT * CR * TAIL;           // warp sums of lse ([2][4] when P)
    static constexpr uint32_t MRG = RED + 8 * 8;                  // [128] (max, sum) of warps 6-9 ([2][128] when P)
    static constexpr uint32_t BAR = MRG + (P ? 2 : 1) * 128 * 8;  // x_full, q_full[FQ], q_empty[FQ], a_full[2],
                                                                  // a_empty[2], t_empty[FT]; when P also
                                                                  // x_empty, the second x_full / x_empty, m_full[2],
                                                                  // r_full[2]
    static_assert(2 * XB + 2 * FQ + 4 + FT + 4 <= 32, "barrier slots");
    static constexpr uint32_t TMEMP = BAR + 32 * 8;
    static constexpr uint32_t FLAG = TMEMP + 8;
    static constexpr uint32_t END = FLAG + 8;
    static constexpr size_t SMEM = END + 1024;
    static_assert(SMEM <= 227 * 1024, "forward shared memory");
    static_assert(Q % 1024 == 0 && STG % 1024 == 0 && XBYTES % 1024 == 0 && TAIL % 16 == 0,
                  "operand and copy alignment");
    static_assert(CR * G == 256 && (CR / 2) * G == 128 && NSET % 2 == 0,
                  "a round fills N = 256; each epilogue warp 128 columns");
};

// sum over CNT rows (columns off .. of a 64-column TMEM chunk) of (z - b)^2,
// z as raw FP32 bits from tcgen05.ld; off must fold to a constant where this
// is inlined (every caller's loop is unrolled), so v stays in registers
template <int CNT>
__device__ __forceinline__ float sumsq_rows(const uint32_t (&v)[64], int off, const float* __restrict__ b) {
    const float2 neg1 = make_float2(-1.f, -1.f);
    float2 acc[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
    for (int i = 0; i < CNT; i += 4) {
        const float4 b4 = *reinterpret_cast<const float4*>(b + i);
        const float2 z0 = __ffma2_rn(make_float2(b4.x, b4.y), neg1,
                                     make_float2(__uint_as_float(v[off + i]), __uint_as_float(v[off + i + 1])));
        const float2 z1 = __ffma2_rn(make_float2(b4.z, b4.w), neg1,
                                     make_float2(__uint_as_float(v[off + i + 2]), __uint_as_float(v[off + i + 3])));
        acc[(i >> 2) & 1] = __ffma2_rn(z0, z0, acc[(i >> 2) & 1]);
        acc[2 + ((i >> 2) & 1)] = __ffma2_rn(z1, z1, acc[2 + ((i >> 2) & 1)]);
    }
    const float2 t = __fadd2_rn(__fadd2_rn(acc[0], acc[1]), __fadd2_rn(acc[2], acc[3]));
    return t.x + t.y;
}

// ---- the forward's MMA issue -------------------------------------------------
// One thread issues every MMA of a CTA; its loop is straight-line code (the
// sets, atoms and K steps of a round unrolled at compile time) so that
// consecutive tcgen05.mma instructions are a few independent integer adds
// apart. Descriptors are handled as low words (start address >> 4: a K step
// of 32 bytes adds 2, an atom of 16 KB adds 1024; the field has 14 bits and
// operands stay below 256 KB, so a sum never carries into the next field)
// with one shared high word.
struct FwdIssue {
    uint64_t* q_full;
    uint64_t* q_empty;
    uint64_t* a_full;
    uint64_t* a_empty;
    int32_t* status;
    uint32_t tmem, xh, xl, q0, dhi, idesc;
    uint32_t s, ph;  // next Q stage slot and the parity of its fill
};

// The MMAs of one stage: NK K steps of its column atom. HI: x_hi and x_lo
// against Q_hi (two MMAs per step), else x_hi against Q_lo; `first` starts
// the set's accumulator.
template <int NK, bool HI>
__device__ __forceinline__ void fwd_stage_mmas(const FwdIssue& I, uint32_t d, uint32_t ah, uint32_t al, uint32_t bq,
                                               bool first) {
#pragma unroll
    for (int ks = 0; ks < NK; ++ks) {
        tc::mma_bf16_w(d, ah + 2u * ks, bq + 2u * ks, I.dhi, I.idesc, (first && ks == 0) ? 0u : 1u);
        if (HI) tc::mma_bf16_w(d, al + 2u * ks, bq + 2u * ks, I.dhi, I.idesc, 1u);
    }
}

template <bool HI>
__device__ __forceinline__ void fwd_stage_dispatch(const FwdIssue& I, int nk, uint32_t d, uint32_t ah, uint32_t al,
                                                   uint32_t bq, bool first) {
    switch (nk) {
        case 1: fwd_stage_mmas<1, HI>(I, d, ah, al, bq, first); break;
        case 2: fwd_stage_mmas<2, HI>(I, d, ah, al, bq, first); break;
        case 3: fwd_stage_mmas<3, HI>(I, d, ah, al, bq, first); break;
        default: fwd_stage_mmas<4, HI>(I, d, ah, al, bq, first); break;
    }
}

// Set J of a round (set number q of the CTA: TMEM half q % 2): its atoms of
// Q_hi, then of Q_lo, each one stage. False when a wait gave up.
template <class S, int J>
__device__ __forceinline__ bool fwd_set_mmas(FwdIssue& I, int q) {
    constexpr int NAJ = S::atoms(J), KS = (J + 1) * S::G / 16;
    const int b = q & 1;
    if (!mbar_wait(&I.a_empty[b], ((uint32_t)(q >> 1) & 1u) ^ 1u, I.status)) return false;
    const uint32_t d = I.tmem + 256u * (uint32_t)b;
#pragma unroll
    for (int lo = 0; lo < 2; ++lo)
#pragma unroll
        for (int at = 0; at < NAJ; ++at) {
            if (!mbar_wait(&I.q_full[I.s], I.ph, I.status)) return false;
            tc::fence_after_sync();
            const uint32_t bq = I.q0 + I.s * (S::STG >> 4);
            const uint32_t ah = I.xh + (uint32_t)at * (ATOM >> 4), al = I.xl + (uint32_t)at * (ATOM >> 4);
            const int nk = KS - 4 * at < 4 ? KS - 4 * at : 4;
            if (lo == 0)
                fwd_stage_dispatch<true>(I, nk, d, ah, al, bq, at == 0);
            else
                fwd_stage_dispatch<false>(I, nk, d, ah, al, bq, false);
            tc::mma_commit(&I.q_empty[I.s]);
            if (++I.s == (uint32_t)S::FQ) {
                I.s = 0;
                I.ph ^= 1u;
            }
        }
    tc::mma_commit(&I.a_full[b]);
    return true;
}

template <class S, int J, bool END = (J >= S::NSET)>
struct FwdSets {
    __device__ static __forceinline__ bool run(FwdIssue& I, int q) {
        return fwd_set_mmas<S, J>(I, q) && FwdSets<S, J + 1>::run(I, q + 1);
    }
};
template <class S, int J>
struct FwdSets<S, J, true> {
    __device__ static __forceinline__ bool run(FwdIssue&, int) { return true; }
};

template <int TDP>
__global__ void __launch_bounds__(64 + 32 * FwdSm<TDP>::EW, 1)
    gmm_tc_fwd_kernel(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmxl,
                      const __grid_constant__ CUtensorMap tmq, const __grid_constant__ CUtensorMap tmql,
                      const float* __restrict__ tails, int64_t n, int64_t xrow0, int k, int kq,
                      float* __restrict__ lj, int64_t lj_ld, float* __restrict__ lse_out, double* __restrict__ part,
                      int64_t tile0, const TcCatInst* __restrict__ cat, const int2* __restrict__ cat_tiles,
                      int32_t* __restrict__ status) {
    using S = FwdSm<TDP>;
    constexpr int FQ = S::FQ, FT = S::FT, NA = S::NA, G = S::G, NSET = S::NSET, CR = S::CR;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = align1024(smem_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + S::BAR);
    uint64_t* x_full = bars;
    uint64_t* q_full = bars + 1;
    uint64_t* q_empty = bars + 1 + FQ;
    uint64_t* a_full = bars + 1 + 2 * FQ;  // [2] accumulator halves of TMEM
    uint64_t* a_empty = a_full + 2;
    uint64_t* t_empty = a_full + 4;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(sm + S::TMEMP);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + S::FLAG);
    double* red = reinterpret_cast<double*>(sm + S::RED);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // this CTA's tile: tile blockIdx.x of the call, or, in a concatenated
    // class of the batched form, tile cat_tiles[blockIdx.x] of its instance
    // (its points from row xoff, its components from Q row block koff)
    int64_t p0 = (int64_t)blockIdx.x * TM, pidx = tile0 + blockIdx.x;
    int koff = 0;
    if (cat) {
        const int2 tt = cat_tiles[blockIdx.x];
        const TcCatInst& I = cat[tt.x];
        n = I.n;
        xrow0 = I.xoff;
        k = I.k;
        koff = I.koff;
        lj = I.lj;
        lj_ld = (I.n + TM - 1) / TM * TM;
        lse_out = I.lse;
        part = I.fwd;
        p0 = (int64_t)tt.y * TM;
        pidx = tt.y;
    }
    const int rounds = (k + CR - 1) / CR;

    if (threadIdx.x == 0) {
        mbar_init(x_full, 1);
        for (int s = 0; s < FQ; ++s) {
            mbar_init(&q_full[s], 1);
            mbar_init(&q_empty[s], 1);  // MMA commit
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&a_full[b], 1);
            mbar_init(&a_empty[b], S::EW);
        }
        for (int t = 0; t < FT; ++t) mbar_init(&t_empty[t], S::EW);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_holder, 512);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_holder;
    Lse st;  // epilogue threads: online logsumexp over the components they read
    st.init();

    if (warp == 0) {
        if (lane == 0) {
            mbar_arrive_expect_tx(x_full, 2 * NA * ATOM);
            for (int a = 0; a < NA; ++a) {
                tc::tma_load_2d(sm + S::X + a * ATOM, &tmx, 64 * a, (int)(xrow0 + p0), x_full);
                tc::tma_load_2d(sm + S::X + (NA + a) * ATOM, &tmxl, 64 * a, (int)(xrow0 + p0), x_full);
            }
            // per round and set j: the set's column atoms of Q_hi, then of
            // Q_lo; one 256-row box each (G rows of each of the round's
            // components; rows past the last one are never multiplied)
            uint32_t g = 0;
            bool ok = true;
            for (int r = 0; ok && r < rounds; ++r) {
                const int c0 = CR * r, nc = min(CR, k - c0), ts = r % FT;
                const uint32_t tph = (uint32_t)(r / FT) & 1u;
                for (int j = 0; ok && j < NSET; ++j) {
                    const int row = (j * kq + koff + c0) * G;
                    for (int lo = 0; ok && lo < 2; ++lo)
                        for (int at = 0; at < S::atoms(j); ++at, ++g) {
                            const int s = (int)(g % FQ);
                            const uint32_t ph = (g / FQ) & 1u;
                            const bool first = j == 0 && lo == 0 && at == 0;
                            if (!mbar_wait(&q_empty[s], ph ^ 1u, status) ||
                                (first && !mbar_wait(&t_empty[ts], tph ^ 1u, status))) {
                                ok = false;
                                break;
                            }
                            mbar_arrive_expect_tx(&q_full[s], S::STG + (first ? (uint32_t)nc * S::TAIL : 0u));
                            tc::tma_load_2d(sm + S::Q + s * S::STG, lo ? &tmql : &tmq, 64 * at, row, &q_full[s]);
                            if (first)
                                bulk_g2s(sm + S::B + ts * CR * S::TAIL, tails + (size_t)(koff + c0) * (TDP + 4),
                                         (uint32_t)nc * S::TAIL, &q_full[s]);
                        }
                }
            }
            if (!ok) *abort_flag = 1;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            bool ok = mbar_wait(x_full, 0, status);
            const uint64_t dx = tc::desc_sw128(smem_u32(sm + S::X)), dq = tc::desc_sw128(smem_u32(sm + S::Q));
            FwdIssue I{q_full, q_empty, a_full, a_empty, status, tmem, (uint32_t)dx,
                       (uint32_t)dx + (uint32_t)(NA * ATOM >> 4), (uint32_t)dq, (uint32_t)(dx >> 32), 0u, 0u, 0u};
            for (int r = 0; ok && r < rounds; ++r) {
                I.idesc = tc::idesc_bf16_f32(128, G * min(CR, k - CR * r));
                ok = FwdSets<S, 0>::run(I, r * NSET);
            }
            if (!ok) *abort_flag = 1;
        }
        __syncwarp();
    } else {
        // epilogue: one thread per point (TMEM lane). Warp w reads TMEM lanes
        // 32 (w % 4) ..; warps 2-5 take the first CR / 2 components of each
        // round, warps 6-9 the others: 128 columns per warp and set, read as
        // two 64-column chunks of 64 / G components each.
        constexpr int HC = CR / 2, PCH = 64 / G;  // components per warp, per chunk
        constexpr int TF = S::TAIL / 4;           // floats per tail
        const int qtr = warp & 3;
        const int jw = (warp - 2) >> 2;
        const int row = qtr * 32 + lane;
        const bool valid = p0 + row < n;
        const uint32_t tl = tmem + ((uint32_t)(qtr * 32) << 16) + (uint32_t)(128 * jw);
        for (int r = 0; r < rounds; ++r) {
            const int ts = r % FT;
            const float* bw = reinterpret_cast<const float*>(sm + S::B + (ts * CR + jw * HC) * S::TAIL);
            float sv[HC];
#pragma unroll
            for (int u = 0; u < HC; ++u) sv[u] = 0.f;
            uint32_t rv[2][64];
            // set by set: both chunks' loads issued together, one wait (the
            // two sets of TDP = 64 unrolled)
            constexpr int JU = NSET <= 2 ? NSET : 1;
#pragma unroll JU
            for (int j = 0; j < NSET; ++j) {
                const int q = r * NSET + j, b = q & 1;
                if (!mbar_wait_warp(&a_full[b], (uint32_t)(q >> 1) & 1u, status)) {
                    *abort_flag = 1;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t ta = tl + 256u * (uint32_t)b;
                const float* bj = bw + j * G;
                tc::tmem_ld64_issue(ta, rv[0]);
                tc::tmem_ld64_issue(ta + 64u, rv[1]);
                tc::tmem_ld64_tied_wait(rv[0]);
#pragma unroll
                for (int u = 0; u < PCH; ++u) sv[u] += sumsq_rows<G>(rv[0], u * G, bj + u * TF);
                tc::tmem_ld64_tied_wait(rv[1]);
#pragma unroll
                for (int u = 0; u < PCH; ++u) sv[PCH + u] += sumsq_rows<G>(rv[1], u * G, bj + (PCH + u) * TF);
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&a_empty[b]);
            }
            if (*abort_flag) break;
            // the round's tail slot goes back to the producer after its last
            // read (the constants)
            float cst[HC];
#pragma unroll
            for (int u = 0; u < HC; ++u) cst[u] = bw[u * TF + TDP];
            fence_proxy_async_smem();  // tails read through the generic proxy
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&t_empty[ts]);
#pragma unroll
            for (int u = 0; u < HC; ++u) {
                const int kk = CR * r + HC * jw + u;
                if (kk < k && valid) {
                    const float v = cst[u] - 0.5f * sv[u];
                    if (lj) lj[(int64_t)kk * lj_ld + p0 + row] = v;
                    st.add(v);
                }
            }
        }
        if (jw == 1) reinterpret_cast<float2*>(sm + S::MRG)[row] = make_float2(st.m, st.l);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp >= 2 && warp < 6) {  // each point's two partial logsumexps
        const int row = (warp & 3) * 32 + lane;
        const float2 o = reinterpret_cast<const float2*>(sm + S::MRG)[row];
        st.merge(o.x, o.y);
        double v = 0.0;
        if (p0 + row < n && !*abort_flag) {
            const float lv = st.value();
            if (lse_out) lse_out[p0 + row] = lv;
            v = (double)lv;
        }
        v = warp_sum(v);
        if (lane == 0) red[warp - 2] = v;
    }
    __syncthreads();
    if (threadIdx.x == 64) part[pidx] = *abort_flag ? NAN : red[0] + red[1] + red[2] + red[3];
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 512);
    }
}

// The forward of a concatenated class of the batched form, persistent: one
// CTA per SM takes the class's tiles w = blockIdx.x, blockIdx.x + gridDim.x,
// ... (tile cat_tiles[w] of its instance: its points from row xoff, its
// components from Q row block koff), so that the CTA start, tensor-memory
// allocation and pipeline fill and drain of gmm_tc_fwd_kernel are paid once per
// SM instead of once per tile (the class's tiles are short: about five rounds
// at its average K). The roles and the round structure are those of
// gmm_tc_fwd_kernel; in addition the MMA thread releases an x buffer after the
// last MMA of its tile, and at the end of a tile the two halves of each
// point's logsumexp merge through shared memory in two buffers by tile
// parity, each with its own barrier.
struct FwdItem {
    int64_t n, xrow0, p0, pidx, lj_ld;
    int k, koff;
    float* lj;
    float* lse_out;
    double* part;
};

template <int TDP>
__global__ void __launch_bounds__(64 + 32 * FwdSm<TDP, true>::EW, 1)
    gmm_tc_fwd_cat_kernel(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmxl,
                          const __grid_constant__ CUtensorMap tmq, const __grid_constant__ CUtensorMap tmql,
                          const float* __restrict__ tails, int kq, int n_items, const TcCatInst* __restrict__ cat,
                          const int2* __restrict__ cat_tiles, int32_t* __restrict__ status) {
    using S = FwdSm<TDP, true>;
    constexpr int FQ = S::FQ, FT = S::FT, NA = S::NA, G = S::G, NSET = S::NSET, CR = S::CR, XB = S::XB;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = align1024(smem_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + S::BAR);
    uint64_t* x_full = bars;                 // [XB]
    uint64_t* x_empty = bars + XB;           // [XB]
    uint64_t* q_full = bars + 2 * XB;        // [FQ]
    uint64_t* q_empty = q_full + FQ;         // [FQ]
    uint64_t* a_full = q_empty + FQ;         // [2] accumulator halves of TMEM
    uint64_t* a_empty = a_full + 2;          // [2]
    uint64_t* t_empty = a_full + 4;          // [FT]
    uint64_t* m_full = t_empty + FT;         // [2] per item parity: second halves of the logsumexps written
    uint64_t* r_full = m_full + 2;           // [2] per item parity: the tile's four warp sums written
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(sm + S::TMEMP);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + S::FLAG);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // persistent: CTA b takes items b, b + gridDim.x, ...
    auto item = [&](int w) {
        FwdItem it;
        const int2 tt = cat_tiles[w];
        const TcCatInst& I = cat[tt.x];
        it.n = I.n;
        it.xrow0 = I.xoff;
        it.k = I.k;
        it.koff = I.koff;
        it.lj = I.lj;
        it.lj_ld = (I.n + TM - 1) / TM * TM;
        it.lse_out = I.lse;
        it.part = I.fwd;
        it.p0 = (int64_t)tt.y * TM;
        it.pidx = tt.y;
        return it;
    };

    if (threadIdx.x == 0) {
        for (int b = 0; b < XB; ++b) {
            mbar_init(&x_full[b], 1);
            mbar_init(&x_empty[b], 1);  // MMA commit after the tile's last MMA
        }
        for (int s = 0; s < FQ; ++s) {
            mbar_init(&q_full[s], 1);
            mbar_init(&q_empty[s], 1);  // MMA commit
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&a_full[b], 1);
            mbar_init(&a_empty[b], S::EW);
            mbar_init(&m_full[b], S::EW / 2);
            mbar_init(&r_full[b], S::EW / 2);
        }
        for (int t = 0; t < FT; ++t) mbar_init(&t_empty[t], S::EW);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_holder, 512);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_holder;

    if (warp == 0) {
        if (lane == 0) {
            // per item: its x tile (into X buffer xt % XB, once the MMAs of the
            // item that used it are done), then per round and set j the set's
            // column atoms of Q_hi, then of Q_lo; one 256-row box each (G rows
            // of each of the round's components; rows past the last one are
            // never multiplied)
            uint32_t g = 0;
            int rr = 0;  // rounds issued (tail slots)
            bool ok = true;
            for (int w = blockIdx.x, xt = 0; ok && w < n_items; w += gridDim.x, ++xt) {
                const FwdItem it = item(w);
                const int xb = xt % XB;
                if (!mbar_wait(&x_empty[xb], ((uint32_t)(xt / XB) & 1u) ^ 1u, status)) {
                    ok = false;
                    break;
                }
                mbar_arrive_expect_tx(&x_full[xb], 2 * NA * ATOM);
                for (int a = 0; a < NA; ++a) {
                    tc::tma_load_2d(sm + S::X + xb * S::XBYTES + a * ATOM, &tmx, 64 * a, (int)(it.xrow0 + it.p0),
                                    &x_full[xb]);
                    tc::tma_load_2d(sm + S::X + xb * S::XBYTES + (NA + a) * ATOM, &tmxl, 64 * a,
                                    (int)(it.xrow0 + it.p0), &x_full[xb]);
                }
                const int rounds = (it.k + CR - 1) / CR;
                for (int r = 0; ok && r < rounds; ++r, ++rr) {
                    const int c0 = CR * r, nc = min(CR, it.k - c0), ts = rr % FT;
                    const uint32_t tph = (uint32_t)(rr / FT) & 1u;
                    for (int j = 0; ok && j < NSET; ++j) {
                        const int row = (j * kq + it.koff + c0) * G;
                        for (int lo = 0; ok && lo < 2; ++lo)
                            for (int at = 0; at < S::atoms(j); ++at, ++g) {
                                const int s = (int)(g % FQ);
                                const uint32_t ph = (g / FQ) & 1u;
                                const bool first = j == 0 && lo == 0 && at == 0;
                                if (!mbar_wait(&q_empty[s], ph ^ 1u, status) ||
                                    (first && !mbar_wait(&t_empty[ts], tph ^ 1u, status))) {
                                    ok = false;
                                    break;
                                }
                                mbar_arrive_expect_tx(&q_full[s], S::STG + (first ? (uint32_t)nc * S::TAIL : 0u));
                                tc::tma_load_2d(sm + S::Q + s * S::STG, lo ? &tmql : &tmq, 64 * at, row, &q_full[s]);
                                if (first)
                                    bulk_g2s(sm + S::B + ts * CR * S::TAIL,
                                             tails + (size_t)(it.koff + c0) * (TDP + 4), (uint32_t)nc * S::TAIL,
                                             &q_full[s]);
                            }
                    }
                }
            }
            if (!ok) *abort_flag = 1;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint64_t dx = tc::desc_sw128(smem_u32(sm + S::X)), dq = tc::desc_sw128(smem_u32(sm + S::Q));
            FwdIssue I{q_full, q_empty, a_full, a_empty, status, tmem, 0u, 0u, (uint32_t)dq, (uint32_t)(dx >> 32),
                       0u, 0u, 0u};
            bool ok = true;
            int q = 0;  // sets issued (TMEM halves)
            for (int w = blockIdx.x, xt = 0; ok && w < n_items; w += gridDim.x, ++xt) {
                const int kk = cat[cat_tiles[w].x].k;
                const int xb = xt % XB;
                if (!mbar_wait(&x_full[xb], (uint32_t)(xt / XB) & 1u, status)) {
                    ok = false;
                    break;
                }
                I.xh = (uint32_t)dx + (uint32_t)(xb * (S::XBYTES >> 4));
                I.xl = I.xh + (uint32_t)(NA * ATOM >> 4);
                const int rounds = (kk + CR - 1) / CR;
                for (int r = 0; ok && r < rounds; ++r, q += NSET) {
                    I.idesc = tc::idesc_bf16_f32(128, G * min(CR, kk - CR * r));
                    ok = FwdSets<S, 0>::run(I, q);
                }
                if (ok) tc::mma_commit(&x_empty[xb]);  // the item's MMAs have read its x tile
            }
            if (!ok) *abort_flag = 1;
        }
        __syncwarp();
    } else {
        // epilogue: one thread per point (TMEM lane). Warp w reads TMEM lanes
        // 32 (w % 4) ..; warps 2-5 take the first CR / 2 components of each
        // round, warps 6-9 the others: 128 columns per warp and set, read as
        // two 64-column chunks of 64 / G components each. At the end of an
        // item the two halves of each point's logsumexp merge through shared
        // memory (two buffers by item parity, each with a barrier).
        constexpr int HC = CR / 2, PCH = 64 / G;  // components per warp, per chunk
        constexpr int TF = S::TAIL / 4;           // floats per tail
        const int qtr = warp & 3;
        const int jw = (warp - 2) >> 2;
        const int row = qtr * 32 + lane;
        const uint32_t tl = tmem + ((uint32_t)(qtr * 32) << 16) + (uint32_t)(128 * jw);
        int q = 0, rr = 0;
        for (int w = blockIdx.x, ni = 0; w < n_items && !*abort_flag; w += gridDim.x, ++ni) {
            const FwdItem it = item(w);
            const bool valid = it.p0 + row < it.n;
            Lse st;  // online logsumexp over the components this thread reads
            st.init();
            const int rounds = (it.k + CR - 1) / CR;
            bool ok = true;
            for (int r = 0; ok && r < rounds; ++r, ++rr) {
                const int ts = rr % FT;
                const float* bw = reinterpret_cast<const float*>(sm + S::B + (ts * CR + jw * HC) * S::TAIL);
                float sv[HC];
#pragma unroll
                for (int u = 0; u < HC; ++u) sv[u] = 0.f;
                uint32_t rv[2][64];
                // set by set: both chunks' loads issued together, one wait (the
                // two sets of TDP = 64 unrolled)
                constexpr int JU = NSET <= 2 ? NSET : 1;
#pragma unroll JU
                for (int j = 0; j < NSET; ++j, ++q) {
                    const int b = q & 1;
                    if (!mbar_wait_warp(&a_full[b], (uint32_t)(q >> 1) & 1u, status)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t ta = tl + 256u * (uint32_t)b;
                    const float* bj = bw + j * G;
                    tc::tmem_ld64_issue(ta, rv[0]);
                    tc::tmem_ld64_issue(ta + 64u, rv[1]);
                    tc::tmem_ld64_tied_wait(rv[0]);
#pragma unroll
                    for (int u = 0; u < PCH; ++u) sv[u] += sumsq_rows<G>(rv[0], u * G, bj + u * TF);
                    tc::tmem_ld64_tied_wait(rv[1]);
#pragma unroll
                    for (int u = 0; u < PCH; ++u) sv[PCH + u] += sumsq_rows<G>(rv[1], u * G, bj + (PCH + u) * TF);
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&a_empty[b]);
                }
                if (!ok) break;
                // the round's tail slot goes back to the producer after its last
                // read (the constants)
                float cst[HC];
#pragma unroll
                for (int u = 0; u < HC; ++u) cst[u] = bw[u * TF + TDP];
                fence_proxy_async_smem();  // tails read through the generic proxy
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&t_empty[ts]);
#pragma unroll
                for (int u = 0; u < HC; ++u) {
                    const int kk = CR * r + HC * jw + u;
                    if (kk < it.k && valid) {
                        const float v = cst[u] - 0.5f * sv[u];
                        if (it.lj) it.lj[(int64_t)kk * it.lj_ld + it.p0 + row] = v;
                        st.add(v);
                    }
                }
            }
            if (!ok) {
                *abort_flag = 1;
                break;
            }
            // each point's two partial logsumexps, then the tile's sum of lse
            const int ib = ni & 1;
            const uint32_t iph = (uint32_t)(ni >> 1) & 1u;
            float2* mrg = reinterpret_cast<float2*>(sm + S::MRG) + ib * TM;
            double* red = reinterpret_cast<double*>(sm + S::RED) + ib * 4;
            if (jw == 1) {
                mrg[row] = make_float2(st.m, st.l);
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&m_full[ib]);
            } else {
                if (!mbar_wait_warp(&m_full[ib], iph, status)) {
                    *abort_flag = 1;
                    break;
                }
                const float2 o = mrg[row];
                st.merge(o.x, o.y);
                double v = 0.0;
                if (valid) {
                    const float lv = st.value();
                    if (it.lse_out) it.lse_out[it.p0 + row] = lv;
                    v = (double)lv;
                }
                v = warp_sum(v);
                if (lane == 0) {
                    red[warp - 2] = v;
                    tc::mbar_arrive(&r_full[ib]);
                }
                if (warp == 2 && lane == 0) {
                    if (!mbar_wait(&r_full[ib], iph, status)) {
                        *abort_flag = 1;
                    } else {
                        it.part[it.pidx] = red[0] + red[1] + red[2] + red[3];
                    }
                }
                __syncwarp();
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 512);
    }
}

// ---- backward -----------------------------------------------------------------
// The Accum sums of the reverse pass as one contraction over the points. With
// r_ik = seed exp(s_ik - lse_i) and, per point, the vector of products
//   y_i = [x_ia x_ib (a >= b), x_ia (a < d), 1]      (d(d+1)/2 + d + 1 entries),
// the sums S_k = sum_i r_ik x_i x_i^T (lower triangle), m_k = sum_i r_ik x_i and
// R_k = sum_i r_ik are the rows of  Y^T R  (Y: points x products, R: points x
// components), so a single BF16 MMA stream with FP32 accumulation computes all
// of them, each product exactly once (the triangle is not mirrored). Y is
// shared by every component and built on the CUDA cores per point tile; R is
// written once per call in BF16 (gmm_tc_r_kernel) and read by TMA.
//
// CTA: 256 product rows (two 128-row MMA blocks) x up to 256 components x a
// chunk of the points. Warps 0-15 build the Y tiles (64 points, K-major,
// 128-byte swizzle) and at the end copy the accumulators from tensor memory
// into the per-chunk partial sums; warp 16 loads the R tiles (TMA); one lane of
// warp 17 issues the MMAs (M = 128 products, N = components, K = 16 points).
constexpr int GTM = 64;                         // points per tile (4 MMA K steps)
constexpr int GMB = 2;                          // 128-row MMA blocks per CTA
constexpr int GPROD = 512;                      // producer threads
constexpr int GTHREADS = GPROD + 64;            // + TMA warp + MMA warp
constexpr int GKMAX = 256;                      // components per CTA (MMA N)
constexpr int GRB_POINTS = 1 << 18;             // points of R held at a time
constexpr uint32_t GYB = GMB * 128 * 128;       // one Y tile: 256 rows x 64 points bf16

// Transposed point tile (BF16): row c (a coordinate; row d = ones, d + 1 =
// zeros) holds the tile's 64 points in 128 bytes, the 16-byte group g of 8
// points at position g ^ (c & 7), so that a warp reading one group of 32
// different rows spreads over all banks.
__host__ __device__ __forceinline__ int gram_xpos(int c, int p) { return c * GTM + ((((p >> 3) ^ c) & 7) << 3) + (p & 7); }

template <int TDP>
struct GramSm {
    static constexpr int XR = TDP + 2;          // rows of a transposed point tile
    static constexpr int XS = 3;                // point-tile stages (copies run XS - 1 tiles ahead)
    // R-tile stages: the TMA runs RS - 1 tiles ahead of the MMAs, which covers
    // the latency of a 26-32 KB load from L2 / HBM
    static constexpr int RS = 3;
    static constexpr uint32_t Y = 0;                              // [2] Y tiles
    static constexpr uint32_t R = Y + 2 * GYB;                    // [RS] R tiles (<= 256 rows x 128 B)
    static constexpr uint32_t XT = R + RS * GKMAX * 128;          // [XS][XR][GTM] bf16
    static constexpr uint32_t BAR = XT + XS * XR * GTM * 2;  // y_full[2], y_empty[2], r_full[RS], r_empty[RS],
                                                             // x_full[XS], x_empty[XS], done
    static_assert(4 + 2 * RS + 2 * XS + 1 <= 24, "barrier slots");
    static constexpr uint32_t TMEMP = BAR + 24 * 8;
    static constexpr uint32_t FLAG = TMEMP + 8;                   // abort flag
    static constexpr uint32_t END = FLAG + 8;
    static constexpr size_t SMEM = END + 1024;
    static_assert(SMEM <= 227 * 1024, "gram shared memory");
};

// Two packed BF16 products, each rounded once to BF16.
__device__ __forceinline__ uint32_t bf16x2_mul(uint32_t a, uint32_t b) {
    const __nv_bfloat162 r =
        __hmul2(*reinterpret_cast<const __nv_bfloat162*>(&a), *reinterpret_cast<const __nv_bfloat162*>(&b));
    return *reinterpret_cast<const uint32_t*>(&r);
}

__device__ __forceinline__ void gram_producers_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(GPROD) : "memory");
}

// Product row i of y (0 <= i < np = d(d+1)/2 + d + 1; padding rows beyond):
// the two coordinates whose product it is (d = the constant 1, d + 1 = 0).
__device__ __forceinline__ void gram_row(int i, int d, int& u, int& v) {
    const int T = d * (d + 1) / 2;
    if (i < T) {
        int a = (int)((sqrtf(8.f * (float)i + 1.f) - 1.f) * 0.5f);
        while (a * (a + 1) / 2 > i) --a;
        while ((a + 1) * (a + 2) / 2 <= i) ++a;
        u = a;
        v = i - a * (a + 1) / 2;
    } else if (i < T + d) {
        u = i - T;
        v = d;
    } else if (i == T + d) {
        u = v = d;
    } else {
        u = v = d + 1;
    }
}

template <int TDP>
__global__ void __launch_bounds__(GTHREADS, 1)
    gmm_tc_gram_kernel(const __grid_constant__ CUtensorMap tmr, const __nv_bfloat16* __restrict__ xt_g, int64_t n, int d,
                       int k, int kn, int ngroups, int64_t tiles_per_chunk, float* __restrict__ partS,
                       float* __restrict__ partM, int nblk64, int rbox, const TcCatInst* __restrict__ cat,
                       const int4* __restrict__ cat_items, int32_t* __restrict__ status) {
    using S = GramSm<TDP>;
    constexpr int XS = S::XS;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = align1024(smem_raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + S::BAR);
    uint64_t* y_full = bars;
    uint64_t* y_empty = bars + 2;
    constexpr int RS = S::RS;
    uint64_t* r_full = bars + 4;
    uint64_t* r_empty = bars + 4 + RS;
    uint64_t* x_full = bars + 4 + 2 * RS;
    uint64_t* x_empty = bars + 4 + 2 * RS + XS;
    uint64_t* done = bars + 4 + 2 * RS + 2 * XS;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(sm + S::TMEMP);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + S::FLAG);
    __nv_bfloat16* xt = reinterpret_cast<__nv_bfloat16*>(sm + S::XT);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tid = threadIdx.x;
    // this CTA's work: (group blockIdx.x, chunk blockIdx.y) of the call, or, in
    // a concatenated class of the batched form, item cat_items[blockIdx.x] of
    // its instance (its points' R columns from xoff, its point tiles at xtoff)
    int bx = blockIdx.x, chunk = blockIdx.y;
    int64_t roff = 0;
    if (cat) {
        const int4 it = cat_items[blockIdx.x];
        const TcCatInst& I = cat[it.x];
        xt_g += I.xtoff;
        n = I.n;
        d = I.d;
        k = I.k;
        kn = I.kn;
        ngroups = I.ng;
        tiles_per_chunk = I.tpc;
        partS = I.bS;
        partM = I.bM;
        roff = I.xoff;
        bx = it.y;
        chunk = it.z;
    }
    const int g = bx % ngroups;           // product-row group
    const int kg0 = (bx / ngroups) * GKMAX;  // first component
    const int row0 = g * GMB * 128;
    const int64_t ntiles = (n + GTM - 1) / GTM;
    const int64_t t_begin = (int64_t)chunk * tiles_per_chunk;
    const int64_t t_end = min64(ntiles, t_begin + tiles_per_chunk);

    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(&y_full[b], GPROD / 32);
            mbar_init(&y_empty[b], 1);
        }
        for (int b = 0; b < RS; ++b) {
            mbar_init(&r_full[b], 1);
            mbar_init(&r_empty[b], 1);
        }
        for (int b = 0; b < XS; ++b) {
            mbar_init(&x_full[b], 1);
            mbar_init(&x_empty[b], GPROD / 32);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    // constant rows of the transposed point tiles: ones at row d, zeros at d + 1
    for (int e = tid; e < XS * GTM; e += GTHREADS) {
        const int b = e / GTM, p = e % GTM;
        xt[b * S::XR * GTM + d * GTM + p] = __float2bfloat16_rn(1.f);
        xt[b * S::XR * GTM + (d + 1) * GTM + p] = __float2bfloat16_rn(0.f);
    }
    if (warp == GPROD / 32 + 1) {
        tc::tmem_alloc(tmem_holder, 512);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_holder;
    const uint32_t rbytes = (uint32_t)kn * 128u;  // one R tile: kn components x 64 points bf16

    if (warp == GPROD / 32) {
        // per tile: the transposed point tile (one bulk copy of d rows x 64
        // points) and the R tile (TMA: components kg0 .. kg0 + kn - 1, zero rows
        // past K, 64 points)
        if (lane == 0) {
            const uint32_t xbytes = (uint32_t)d * GTM * 2u;
            int it = 0;
            for (int64_t t = t_begin; t < t_end; ++t, ++it) {
                const int xb = it % XS, b = it % RS;
                const uint32_t ux = (uint32_t)(it / XS), u = (uint32_t)(it / RS);
                if (!mbar_wait(&x_empty[xb], (ux & 1u) ^ 1u, status)) {
                    *abort_flag = 1;
                    break;
                }
                mbar_arrive_expect_tx(&x_full[xb], xbytes);
                bulk_g2s(xt + xb * S::XR * GTM, xt_g + t * (int64_t)d * GTM, xbytes, &x_full[xb]);
                if (!mbar_wait(&r_empty[b], (u & 1u) ^ 1u, status)) {
                    *abort_flag = 1;
                    break;
                }
                mbar_arrive_expect_tx(&r_full[b], rbytes);
                for (int j = 0; j < kn; j += rbox)  // boxes of rbox components (kn / rbox of them)
                    tc::tma_load_2d(sm + S::R + b * GKMAX * 128 + j * 128, &tmr, (int)(t * GTM + roff), kg0 + j,
                                    &r_full[b]);
            }
        }
        __syncwarp();
    } else if (warp == GPROD / 32 + 1) {
        // MMA issuer: D[mb] (tensor-memory columns 256 mb ..) += Y[mb] R^T
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_bf16_f32(128, kn);
            // descriptors as low words with one shared high word (as in the
            // forward): a K step of 32 bytes adds 2
            const uint64_t dy = tc::desc_sw128(smem_u32(sm + S::Y)), dr = tc::desc_sw128(smem_u32(sm + S::R));
            const uint32_t dhi = (uint32_t)(dy >> 32);
            bool ok = true;
            int it = 0;
            for (int64_t t = t_begin; ok && t < t_end; ++t, ++it) {
                const int b = it & 1, rb = it % RS;
                const uint32_t u = (uint32_t)(it >> 1), ur = (uint32_t)(it / RS);
                if (!mbar_wait(&y_full[b], u & 1u, status) || !mbar_wait(&r_full[rb], ur & 1u, status)) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t ya = (uint32_t)dy + (uint32_t)b * (GYB >> 4);
                const uint32_t ra = (uint32_t)dr + (uint32_t)rb * (GKMAX * 128 >> 4);
#pragma unroll
                for (int mb = 0; mb < GMB; ++mb)
#pragma unroll
                    for (int j = 0; j < GTM / 16; ++j)
                        tc::mma_bf16_w(tmem + (uint32_t)(mb * 256), ya + (uint32_t)(mb * (128 * 128 >> 4) + 2 * j),
                                       ra + 2u * j, dhi, idesc, (it > 0 || j > 0) ? 1u : 0u);
                tc::mma_commit(&y_empty[b]);
                tc::mma_commit(&r_empty[rb]);
            }
            if (!ok) *abort_flag = 1;
            tc::mma_commit(done);
        }
        __syncwarp();
    } else {
        // producers: thread = one product row (u, v) of one MMA block, points
        // 32 h .. 32 h + 31 of each tile; a warp takes 32 consecutive rows, so
        // its loads of x_u are broadcasts and its 32 rows x_v spread over all
        // banks. The coordinates are BF16; each product of two of them is
        // formed and rounded to BF16 by one packed multiply.
        const int lrow = tid & 255, h = tid >> 8;
        int u, v;
        gram_row(row0 + lrow, d, u, v);
        const int mb = lrow >> 7, r7 = lrow & 127;
        // this thread's read offsets in a point tile (groups 4h .. 4h + 3 of
        // rows u and v, 8 points each) and write offsets in a Y tile (the same
        // 16-byte chunks of its row)
        int ou[4], ov[4];
        uint32_t oy[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            ou[c] = gram_xpos(u, 8 * (4 * h + c));
            ov[c] = gram_xpos(v, 8 * (4 * h + c));
            oy[c] = (uint32_t)(mb * 128 * 128) + tc::sw128_offset((uint32_t)r7, (uint32_t)(4 * h + c));
        }
        int it = 0;
        for (int64_t t = t_begin; t < t_end; ++t, ++it) {
            const int b = it & 1, xb = it % XS;
            const uint32_t use = (uint32_t)(it >> 1), ux = (uint32_t)(it / XS);
            if (__shfl_sync(0xffffffffu, *abort_flag, 0)) break;  // a wait elsewhere gave up (waits are bounded anyway)
            if (!mbar_wait_warp(&x_full[xb], ux & 1u, status) ||
                !mbar_wait_warp(&y_empty[b], (use & 1u) ^ 1u, status)) {
                *abort_flag = 1;
                break;
            }
            const __nv_bfloat16* X = xt + xb * S::XR * GTM;
            uint8_t* yt = sm + S::Y + b * GYB;
#pragma unroll
            for (int c = 0; c < 4; ++c) {  // 8 points per 16-byte chunk of the Y row
                const uint4 a4 = *reinterpret_cast<const uint4*>(X + ou[c]);
                const uint4 b4 = *reinterpret_cast<const uint4*>(X + ov[c]);
                *reinterpret_cast<uint4*>(yt + oy[c]) =
                    make_uint4(bf16x2_mul(a4.x, b4.x), bf16x2_mul(a4.y, b4.y), bf16x2_mul(a4.z, b4.z),
                               bf16x2_mul(a4.w, b4.w));
            }
            fence_proxy_async_smem();  // the Y writes before the MMAs read them; the point-tile reads before its refill
            __syncwarp();
            if (lane == 0) {
                tc::mbar_arrive(&y_full[b]);
                tc::mbar_arrive(&x_empty[xb]);
            }
        }
        // accumulators: warp w reads the tensor-memory lanes of its quarter w % 4
        // (product rows 32 (w % 4) .. of block mb) for column chunks w / 4, +4, ...
        const bool fin = mbar_wait_warp(done, 0, status);
        if (!fin) *abort_flag = 1;
        tc::fence_after_sync();
        gram_producers_sync();  // every warp has seen `done` (or given up) before reading the flag
        const int aborted = __shfl_sync(0xffffffffu, *abort_flag, 0);
        if (!aborted && t_begin < t_end) {
            const int qtr = warp & 3;
            const int nch = GMB * (kn / 16);  // chunks of 16 columns over both blocks
            for (int cc = warp >> 2; cc < nch; cc += 4) {
                const int eb = cc / (kn / 16), c0 = (cc % (kn / 16)) * 16;
                float vals[16];
                tc::tmem_ld16_wait(tmem + ((uint32_t)(qtr * 32) << 16) + (uint32_t)(eb * 256 + c0), vals);
                int eu, ev;
                gram_row(row0 + eb * 128 + qtr * 32 + lane, d, eu, ev);
                if (ev > d) continue;  // padding row
                const int64_t cbase = (int64_t)chunk * k;
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int kk = kg0 + c0 + i;
                    if (kk >= k) break;
                    const float val = vals[i];
                    if (ev < d) {          // S entry (eu, ev), eu >= ev
                        const int A = eu >> 3, B = ev >> 3;
                        partS[(cbase + kk) * (int64_t)nblk64 + (A * (A + 1) / 2 + B) * 64 + (eu & 7) * 8 + (ev & 7)] +=
                            val;
                    } else if (eu < d) {   // m entry
                        partM[(cbase + kk) * (TDP + 1) + eu] += val;
                    } else {               // R
                        partM[(cbase + kk) * (TDP + 1) + TDP] += val;
                    }
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == GPROD / 32 + 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 512);
    }
}

// Point tiles for the gram kernel: tile t (points 64 t .. 64 t + 63, zero past
// n) as d rows of 64 BF16 values, row c holding coordinate c of the tile's
// points in the order of gram_xpos, so that one bulk copy brings a tile into
// shared memory in the layout the gram kernel reads. One CTA per tile.
// With XB (the forward's operands, TDP > 0): the same tile's rows also split
// into x_hi + x_lo (BF16, rows of TDP, zero padded) at rows xrow .. xrow + 63
// of xb / xl, from the one read of x.
template <int TDP = 0>
__device__ __forceinline__ void gmm_tc_xt_tile(const float* __restrict__ x, int64_t n, int d,
                                               __nv_bfloat16* __restrict__ xt, int64_t t,
                                               __nv_bfloat16* __restrict__ xb = nullptr,
                                               __nv_bfloat16* __restrict__ xl = nullptr, int64_t xrow = 0) {
    __shared__ float tile[GTM][129];
    const int64_t p0 = t * GTM;
    if (d % 4 == 0 && (reinterpret_cast<uintptr_t>(x) & 15) == 0) {  // 16-byte loads of the rows
        const int d4 = d / 4;
        for (int e = threadIdx.x; e < GTM * d4; e += blockDim.x) {
            const int p = e / d4, c = (e - p * d4) * 4;
            const float4 v = p0 + p < n ? __ldg(reinterpret_cast<const float4*>(x + (p0 + p) * d + c))
                                        : make_float4(0.f, 0.f, 0.f, 0.f);
            tile[p][c] = v.x;
            tile[p][c + 1] = v.y;
            tile[p][c + 2] = v.z;
            tile[p][c + 3] = v.w;
        }
    } else {
        for (int e = threadIdx.x; e < GTM * d; e += blockDim.x) {
            const int p = e / d, c = e - p * d;
            tile[p][c] = p0 + p < n ? __ldg(x + (p0 + p) * d + c) : 0.f;
        }
    }
    __syncthreads();
    // coordinate row c, 8-point group g: one 16-byte store
    __nv_bfloat16* out = xt + t * (int64_t)d * GTM;
    for (int e = threadIdx.x; e < d * (GTM / 8); e += blockDim.x) {
        const int c = e / (GTM / 8), g = e % (GTM / 8);
        uint4 w;
        w.x = tc::pack_bf16x2(tile[8 * g][c], tile[8 * g + 1][c]);
        w.y = tc::pack_bf16x2(tile[8 * g + 2][c], tile[8 * g + 3][c]);
        w.z = tc::pack_bf16x2(tile[8 * g + 4][c], tile[8 * g + 5][c]);
        w.w = tc::pack_bf16x2(tile[8 * g + 6][c], tile[8 * g + 7][c]);
        *reinterpret_cast<uint4*>(out + gram_xpos(c, 8 * g)) = w;
    }
    if constexpr (TDP > 0) {
        // point p, columns c .. c + 7: one 16-byte store each of x_hi and x_lo
        for (int e = threadIdx.x; e < GTM * (TDP / 8); e += blockDim.x) {
            const int p = e / (TDP / 8), c = (e % (TDP / 8)) * 8;
            uint32_t hw[4], lw[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float v0 = c + 2 * j < d ? tile[p][c + 2 * j] : 0.f;
                const float v1 = c + 2 * j + 1 < d ? tile[p][c + 2 * j + 1] : 0.f;
                const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
                const __nv_bfloat162 l = __floats2bfloat162_rn(v0 - __low2float(h), v1 - __high2float(h));
                hw[j] = *reinterpret_cast<const uint32_t*>(&h);
                lw[j] = *reinterpret_cast<const uint32_t*>(&l);
            }
            *reinterpret_cast<uint4*>(xb + (xrow + p) * TDP + c) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            *reinterpret_cast<uint4*>(xl + (xrow + p) * TDP + c) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
    }
}

// Point tiles and forward operands of one call from one read of x: CTA t makes
// point tile t and rows 64 t .. 64 t + 63 of x_hi, x_lo.
template <int TDP>
__global__ void __launch_bounds__(256) gmm_tc_xtb_kernel(const float* __restrict__ x, int64_t n, int d,
                                                         __nv_bfloat16* __restrict__ xt, __nv_bfloat16* __restrict__ xb,
                                                         __nv_bfloat16* __restrict__ xl) {
    gmm_tc_xt_tile<TDP>(x, n, d, xt, blockIdx.x, xb, xl, (int64_t)blockIdx.x * GTM);
}

// The same for every instance of a concatenated class: CTA t makes 64-point
// tile t of the concatenated rows, i.e. tile t - xoff / 64 of its instance,
// and those rows of x_hi, x_lo.
template <int TDP>
__global__ void __launch_bounds__(256) tc_cat_xt_kernel(const TcCatInst* __restrict__ cat,
                                                        const int* __restrict__ tile_inst, __nv_bfloat16* __restrict__ xt,
                                                        __nv_bfloat16* __restrict__ xb,
                                                        __nv_bfloat16* __restrict__ xl) {
    const TcCatInst& I = cat[tile_inst[blockIdx.x / 2]];
    gmm_tc_xt_tile<TDP>(I.x, I.n, I.d, xt + I.xtoff, (int64_t)blockIdx.x - I.xoff / GTM, xb, xl,
                        (int64_t)blockIdx.x * GTM);
}

// R of every instance of a concatenated class, [kr][np]: row c, column xoff + p
// holds seed exp(lj[c][p] - lse[p]) of the instance whose rows those are, for
// c < k and p < n; zero for its padding points and for rows k .. up to the
// next multiple of 16 (the width of its MMAs); rows beyond that are never
// read and not written. 8 points per thread (never across a 128-point tile).
__global__ void __launch_bounds__(256) tc_cat_r_kernel(const TcCatInst* __restrict__ cat,
                                                       const int* __restrict__ tile_inst, int64_t np, int kr,
                                                       __nv_bfloat16* __restrict__ rb) {
    const int64_t per_row = np / 8;
    const int64_t total = (int64_t)kr * per_row;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        const int c = (int)(e / per_row);
        const int64_t q0 = (e - (int64_t)c * per_row) * 8;
        const TcCatInst& I = cat[tile_inst[q0 / TM]];
        if (c >= (I.k + 15) / 16 * 16) continue;  // rows past the instance's MMA width are never read
        const int64_t p0 = q0 - I.xoff;
        const int64_t ld = (I.n + TM - 1) / TM * TM;  // log-joint rows padded to whole tiles
        float v[8];
        if (c < I.k && p0 + 8 <= I.n) {  // 16-byte loads: rows and lse start on tile boundaries
            const float4* l4 = reinterpret_cast<const float4*>(I.lj + (int64_t)c * ld + p0);
            const float4* s4 = reinterpret_cast<const float4*>(I.lse + p0);
            const float4 a0 = __ldcs(l4), a1 = __ldcs(l4 + 1), b0 = __ldg(s4), b1 = __ldg(s4 + 1);
            v[0] = I.seed * expf(a0.x - b0.x); v[1] = I.seed * expf(a0.y - b0.y);
            v[2] = I.seed * expf(a0.z - b0.z); v[3] = I.seed * expf(a0.w - b0.w);
            v[4] = I.seed * expf(a1.x - b1.x); v[5] = I.seed * expf(a1.y - b1.y);
            v[6] = I.seed * expf(a1.z - b1.z); v[7] = I.seed * expf(a1.w - b1.w);
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int64_t p = p0 + j;
                v[j] = (c < I.k && p < I.n) ? I.seed * expf(__ldg(I.lj + (int64_t)c * ld + p) - __ldg(I.lse + p)) : 0.f;
            }
        }
        *reinterpret_cast<uint4*>(rb + (int64_t)c * np + q0) =
            make_uint4(tc::pack_bf16x2(v[0], v[1]), tc::pack_bf16x2(v[2], v[3]), tc::pack_bf16x2(v[4], v[5]),
                       tc::pack_bf16x2(v[6], v[7]));
    }
}

// r[c][p] = seed exp(lj[c][p] - lse[p]) in BF16 for c < k, p < n; zero for the
// padding rows k <= c < kr and points n <= p < npad. 8 points per thread.
__global__ void __launch_bounds__(256) gmm_tc_r_kernel(const float* __restrict__ lj, int64_t lj_ld,
                                                       const float* __restrict__ lse, int64_t n, int k, int kr,
                                                       int64_t npad, float seed, __nv_bfloat16* __restrict__ rb) {
    const int64_t per_row = npad / 8;
    const int64_t total = (int64_t)kr * per_row;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // 16-byte loads where the rows allow them (p0 is a multiple of 8)
    const bool vec = ((reinterpret_cast<uintptr_t>(lj) | reinterpret_cast<uintptr_t>(lse)) & 15) == 0 && lj_ld % 4 == 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        const int c = (int)(e / per_row);
        const int64_t p0 = (e - (int64_t)c * per_row) * 8;
        float v[8];
        if (vec && c < k && p0 + 8 <= n) {
            const float4* l4 = reinterpret_cast<const float4*>(lj + (int64_t)c * lj_ld + p0);
            const float4* s4 = reinterpret_cast<const float4*>(lse + p0);
            const float4 a0 = __ldcs(l4), a1 = __ldcs(l4 + 1), b0 = __ldg(s4), b1 = __ldg(s4 + 1);
            v[0] = seed * expf(a0.x - b0.x); v[1] = seed * expf(a0.y - b0.y);
            v[2] = seed * expf(a0.z - b0.z); v[3] = seed * expf(a0.w - b0.w);
            v[4] = seed * expf(a1.x - b1.x); v[5] = seed * expf(a1.y - b1.y);
            v[6] = seed * expf(a1.z - b1.z); v[7] = seed * expf(a1.w - b1.w);
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int64_t p = p0 + j;
                v[j] = (c < k && p < n) ? seed * expf(__ldg(lj + (int64_t)c * lj_ld + p) - __ldg(lse + p)) : 0.f;
            }
        }
        *reinterpret_cast<uint4*>(rb + (int64_t)c * npad + p0) =
            make_uint4(tc::pack_bf16x2(v[0], v[1]), tc::pack_bf16x2(v[2], v[3]), tc::pack_bf16x2(v[4], v[5]),
                       tc::pack_bf16x2(v[6], v[7]));
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

// prep record Qt[c][r] -> Q_hi + Q_lo (bf16) in the forward's set-major
// layout, and the b_k tails. qb and ql each hold NSET parts [kq][G][TDP]: part
// j has rows jG .. jG + G - 1 of every Q_k, so that the rows of CR = 256 / G
// consecutive components form one 256-row TMA box. tails: [kq][TDP + 4] floats
// (b_k, the constant, padding), contiguous over the components so that a
// round's tails are one copy.
template <int TDP>
__global__ void __launch_bounds__(256) tc_convert_q_kernel(const float* __restrict__ rec, int kq,
                                                           __nv_bfloat16* __restrict__ qb,
                                                           __nv_bfloat16* __restrict__ ql,
                                                           float* __restrict__ tails) {
    constexpr int G = FwdSm<TDP>::G;
    const int64_t part = (int64_t)kq * G * TDP, total = part * FwdSm<TDP>::NSET;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        const int j = (int)(e / part);
        const int64_t f = e - j * part;
        const int64_t kk = f / (G * TDP);
        const int r = j * G + (int)((f / TDP) % G);
        const int c = (int)(f % TDP);
        const float v = rec[kk * Tc<TDP>::REC + (int64_t)c * TDP + r];
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        qb[e] = h;
        ql[e] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)kq * (TDP + 4); e += stride)
        tails[e] = rec[(e / (TDP + 4)) * Tc<TDP>::REC + TDP * TDP + e % (TDP + 4)];
}

// ---- host ---------------------------------------------------------------------------
size_t a1024(size_t v) { return (v + 1023) & ~(size_t)1023; }

int tc_dp(int d) { return d <= 64 ? 64 : 128; }

// BF16 rows of R: the components rounded up to a multiple of 16 (the MMA's N
// granularity); rows past K are zero.
int tc_r_rows(int k) { return (k + 15) / 16 * 16; }

// Points of R held in the workspace at a time.
int64_t tc_r_points(int64_t npad) { return npad < GRB_POINTS ? npad : (int64_t)GRB_POINTS; }

struct TcLayout {
    size_t off_xb, off_xl, off_qb, off_ql, off_tails, off_rb, off_xt, fixed;
    int64_t npad, rpoints;
};

TcLayout tc_layout(const GmmLayout& L, int64_t n, int d, int k) {
    const int tdp = tc_dp(d);
    TcLayout T;
    T.npad = ((n + TM - 1) / TM) * TM;
    T.rpoints = tc_r_points(T.npad);
    const size_t xbytes = a1024((size_t)T.npad * tdp * 2), qbytes = a1024((size_t)k * tdp * tdp * 2);
    T.off_xb = a1024(L.fixed);
    T.off_xl = T.off_xb + xbytes;
    T.off_qb = T.off_xl + xbytes;
    T.off_ql = T.off_qb + qbytes;
    T.off_tails = T.off_ql + qbytes;
    T.off_rb = T.off_tails + a1024((size_t)k * (tdp + 4) * 4);
    T.off_xt = T.off_rb + a1024((size_t)tc_r_rows(k) * T.rpoints * 2);
    T.fixed = T.off_xt + a1024((size_t)T.npad * d * 2);
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

// 2-D bf16 tensor [rows][tdp], box 64 x box_rows rows, 128-byte swizzle.
bool make_map(CUtensorMap* m, const void* base, int64_t rows, int tdp, int box_rows = TM) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)tdp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)tdp * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// R in BF16 [kr][npad_r], box 64 points x kn components, 128-byte swizzle;
// rows past kr read as zero.
bool make_map_r(CUtensorMap* m, const void* base, int64_t npad_r, int kr, int kn) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)npad_r, (cuuint64_t)kr};
    cuuint64_t strides[1] = {(cuuint64_t)npad_r * 2};
    cuuint32_t box[2] = {(cuuint32_t)GTM, (cuuint32_t)kn};
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

// The forward's operands x_hi, x_lo and Q_hi, Q_lo; with_xt: x_hi, x_lo come
// with the backward's transposed point tiles from one read of x.
template <int TDP>
int convert_inputs(const GmmArgs& A, const GmmLayout& L, const TcLayout& T, char* ws, cudaStream_t s,
                   bool with_xt = false) {
    // grid-stride kernels: one element pair (x) or element (Q) per thread and
    // step, the grid as large as the work up to 8 CTAs per SM
    const int64_t cap = (int64_t)sm_count_tc() * 8;
    const unsigned gx = (unsigned)min64(cap, (A.n * (TDP / 2) + 255) / 256);
    const unsigned gq = (unsigned)min64(cap, ((int64_t)A.k * TDP * TDP + 255) / 256);
    if (with_xt)
        GPA_LAUNCH("gmm_tc_xt", s,
                   gmm_tc_xtb_kernel<TDP><<<(unsigned)(T.npad / GTM), 256, 0, s>>>(
                       A.x, A.n, A.d, (__nv_bfloat16*)(ws + T.off_xt), (__nv_bfloat16*)(ws + T.off_xb),
                       (__nv_bfloat16*)(ws + T.off_xl)));
    else
        GPA_LAUNCH("gmm_tc_convert_x", s,
                   tc_convert_x_kernel<TDP><<<gx, 256, 0, s>>>(A.x, A.n, A.d, (__nv_bfloat16*)(ws + T.off_xb),
                                                               (__nv_bfloat16*)(ws + T.off_xl)));
    GPA_LAUNCH("gmm_tc_convert_q", s,
               tc_convert_q_kernel<TDP><<<gq, 256, 0, s>>>((const float*)(ws + L.off_rec), A.k,
                                                          (__nv_bfloat16*)(ws + T.off_qb),
                                                          (__nv_bfloat16*)(ws + T.off_ql),
                                                          (float*)(ws + T.off_tails)));
    return GPA_OK;
}

// Tensor maps of the forward's Q operands (hi, lo) in the set-major layout of
// tc_convert_q_kernel ([kq * TDP rows][TDP]), 256-row boxes.
template <int TDP>
bool make_q_maps(CUtensorMap (&m)[2], const void* qb, const void* ql, int64_t kq) {
    return make_map(&m[0], qb, kq * TDP, TDP, 256) && make_map(&m[1], ql, kq * TDP, TDP, 256);
}

template <int TDP>
int launch_tc_fwd(const GmmArgs& A, const GmmLayout& L, const TcLayout& T, char* ws, int64_t row0, int64_t n_local,
                  float* lj, int64_t lj_ld, float* lse, cudaStream_t s) {
    using S = FwdSm<TDP>;
    CUtensorMap tmx, tmxl, tq[2];
    if (!make_map(&tmx, ws + T.off_xb, A.n, TDP) || !make_map(&tmxl, ws + T.off_xl, A.n, TDP) ||
        !make_q_maps<TDP>(tq, ws + T.off_qb, ws + T.off_ql, A.k))
        return GPA_ERR_CUDA;
    const int64_t tiles = (n_local + TM - 1) / TM;
    auto kern = gmm_tc_fwd_kernel<TDP>;
    if (!set_smem_tc(kern, S::SMEM)) return GPA_ERR_CUDA;
    GPA_LAUNCH("gmm_tc_fwd", s,
               kern<<<(unsigned)tiles, 64 + 32 * S::EW, S::SMEM, s>>>(
                   tmx, tmxl, tq[0], tq[1], (const float*)(ws + T.off_tails), n_local, row0, A.k, A.k, lj, lj_ld,
                   lse, (double*)(ws + L.off_fwd), row0 / TM, nullptr, nullptr, A.status));
    return GPA_OK;
}

// Product rows of y (gram kernel): d(d+1)/2 + d + 1, in groups of 256.
int gram_groups(int d) { return (d * (d + 1) / 2 + d + 1 + GMB * 128 - 1) / (GMB * 128); }

// Point chunks of the gram grid: one wave of CTAs (one per SM: the kernel
// holds all of tensor memory) when that fills at least 85 % of the SMs, so
// that each CTA accumulates over as many tiles as possible before its
// write-out; otherwise the chunk count with the best wave efficiency.
int tc_bwd_chunks(int groups, int64_t ntiles) {
    const int slots = sm_count_tc();
    // at least kMinTiles point tiles per chunk: a CTA's set-up and write-out
    // of its partial sums cost about as much as that many tiles, and a small
    // problem spread over every SM would keep the others (the concurrent
    // instances of a batch) waiting for little work
    constexpr int64_t kMinTiles = 8;
    const int64_t cap = ntiles / kMinTiles > 1 ? ntiles / kMinTiles : 1;
    const int64_t one_wave = (int64_t)(slots / groups);
    if (one_wave >= 1 && groups * one_wave >= (int64_t)(0.85 * slots))
        return (int)min64(min64(one_wave, kGmmMaxChunks), cap);
    int best = 1;
    double best_eff = -1.0;
    for (int c = 1; c <= kGmmMaxChunks && c <= cap; ++c) {
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

// Reverse-pass sums of points row0 .. row0 + n_local - 1 (n_local <= the R
// capacity): R in BF16 from the log-joint chunk, then the gram kernel.
template <int TDP>
int launch_tc_bwd(const GmmArgs& A, const GmmLayout& L, const TcLayout& T, char* ws, int64_t row0, int64_t n_local,
                  const float* lj, int64_t lj_ld, const float* lse, int nchunks, cudaStream_t s) {
    const int kr = tc_r_rows(A.k), kn = kr < GKMAX ? kr : GKMAX;
    const int64_t npad_r = (n_local + GTM - 1) / GTM * GTM;
    __nv_bfloat16* rb = (__nv_bfloat16*)(ws + T.off_rb);
    const int64_t work = (int64_t)kr * (npad_r / 8);
    const int64_t want = (work + 255) / 256, cap = (int64_t)sm_count_tc() * 16;
    GPA_LAUNCH("gmm_tc_r", s,
               gmm_tc_r_kernel<<<(unsigned)(want < cap ? want : cap), 256, 0, s>>>(
                   lj, lj_ld, lse, n_local, A.k, kr, npad_r, (float)A.seed, rb));
    CUtensorMap tmr;
    if (!make_map_r(&tmr, rb, npad_r, kr, kn)) return GPA_ERR_CUDA;
    auto kern = gmm_tc_gram_kernel<TDP>;
    if (!set_smem_tc(kern, GramSm<TDP>::SMEM)) return GPA_ERR_CUDA;
    const int ng = gram_groups(A.d), nkg = (kr + GKMAX - 1) / GKMAX;
    const int64_t ntiles = (n_local + GTM - 1) / GTM;
    const int64_t tpc = (ntiles + nchunks - 1) / nchunks;
    dim3 grid((unsigned)(ng * nkg), (unsigned)nchunks);
    GPA_LAUNCH("gmm_tc_bwd", s,
               kern<<<grid, GTHREADS, GramSm<TDP>::SMEM, s>>>(tmr, (const __nv_bfloat16*)(ws + T.off_xt) + row0 * A.d, n_local,
                                                                A.d, A.k, kn, ng, tpc,
                                                         (float*)(ws + L.off_bS), (float*)(ws + L.off_bM),
                                                         gmm_bwd_partial_entries(TDP), kn, nullptr, nullptr,
                                                         A.status));
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

// point chunks of the gram grid for n points (the backward runs over at most
// rpoints at a time, with the same chunk grid each time)
template <int TDP>
int vjp_chunks(int64_t n, int d, int k, int64_t rpoints) {
    return tc_bwd_chunks(gram_groups(d) * ((tc_r_rows(k) + GKMAX - 1) / GKMAX),
                         (((n < rpoints ? n : rpoints) + GTM - 1) / GTM));
}

template <int TDP>
int vjp_run(const GmmArgs& A, const GmmLayout& L, char* ws, size_t ws_bytes, cudaStream_t s, int stages) {
    const TcLayout T = tc_layout(L, A.n, A.d, A.k);
    if (ws_bytes < T.fixed) return GPA_ERR_WORKSPACE;
    const int64_t RP = T.rpoints;  // points per backward launch (a multiple of 128)
    const int nchunks = vjp_chunks<TDP>(A.n, A.d, A.k, RP);
    int rc = GPA_OK;
    if ((stages & kGmmStagePrep) && (rc = gmm_run_prep(A, L, ws, s))) return rc;
    if (!(stages & kGmmStageCore)) return GPA_OK;
    const int nent = gmm_bwd_partial_entries(TDP);
    if (cudaMemsetAsync(ws + L.off_bS, 0, sizeof(float) * (size_t)nchunks * A.k * nent, s) != cudaSuccess ||
        cudaMemsetAsync(ws + L.off_bM, 0, sizeof(float) * (size_t)nchunks * A.k * (TDP + 1), s) != cudaSuccess)
        return GPA_ERR_CUDA;
    if ((rc = convert_inputs<TDP>(A, L, T, ws, s, true))) return rc;
    // the backward runs over at most RP points at a time (the R buffer), with
    // the same chunk grid each time so that the partial sums keep one order
    auto bwd_range = [&](int64_t c0, int64_t nl, const float* lj, int64_t lj_ld, const float* lse) {
        for (int64_t o = 0; o < nl; o += RP) {
            const int64_t m = min64(RP, nl - o);
            const int r = launch_tc_bwd<TDP>(A, L, T, ws, c0 + o, m, lj + o, lj_ld, lse + o, nchunks, s);
            if (r) return r;
        }
        return (int)GPA_OK;
    };
    if (A.lj_in) {
        if ((rc = bwd_range(0, A.n, A.lj_in, A.n, A.lse_in))) return rc;
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
            if ((rc = bwd_range(c0, nl, lj, P, lse))) return rc;
        }
    }
    if (!(stages & kGmmStageFinish)) return GPA_OK;
    if (A.exch_out) return gmm_run_exchange(A, L, ws, nchunks, s);
    if ((rc = gmm_run_finalize(A, L, ws, nchunks, 0, s))) return rc;  // raw moments, as the FP32 path
    if (A.out) return gmm_run_objective(A, L, ws, s);
    return GPA_OK;
}

// One concatenated class of the batched form: every stage one launch over all
// its instances' tiles, the forward persistent (prep before and finalize after
// run in the batched class kernels).
template <int TDP>
int cat_run(const TcCatClass& C, cudaStream_t s) {
    const int64_t cap = (int64_t)sm_count_tc() * 8;
    auto* xb = (__nv_bfloat16*)C.xb;
    auto* xl = (__nv_bfloat16*)C.xl;
    auto* qb = (__nv_bfloat16*)C.qb;
    auto* ql = (__nv_bfloat16*)C.ql;
    auto* rb = (__nv_bfloat16*)C.rb;
    GPA_LAUNCH("gmm_tc_convert_q", s,
               tc_convert_q_kernel<TDP><<<(unsigned)min64(cap, (C.kc * TDP * TDP + 255) / 256), 256, 0, s>>>(
                   C.rec, (int)C.kc, qb, ql, C.tails));
    GPA_LAUNCH("gmm_tc_xt", s,
               tc_cat_xt_kernel<TDP><<<(unsigned)(C.np / GTM), 256, 0, s>>>(C.inst, C.tile_inst,
                                                                          (__nv_bfloat16*)C.xt, xb, xl));
    CUtensorMap tmx, tmxl, tq[2], tmr;
    if (!make_map(&tmx, xb, C.np, TDP) || !make_map(&tmxl, xl, C.np, TDP) || !make_q_maps<TDP>(tq, qb, ql, C.kc) ||
        !make_map_r(&tmr, rb, C.np, (int)C.kr, 16))
        return GPA_ERR_CUDA;
    using SP = FwdSm<TDP, true>;
    auto kf = gmm_tc_fwd_cat_kernel<TDP>;
    if (!set_smem_tc(kf, SP::SMEM)) return GPA_ERR_CUDA;
    if (C.n_fwd > 0)
        GPA_LAUNCH("gmm_tc_fwd", s,
                   kf<<<(unsigned)min64(C.n_fwd, sm_count_tc()), 64 + 32 * SP::EW, SP::SMEM, s>>>(
                       tmx, tmxl, tq[0], tq[1], C.tails, (int)C.kc, C.n_fwd, C.inst, C.fwd_tiles, C.status));
    const int64_t rwork = C.kr * (C.np / 8);
    GPA_LAUNCH("gmm_tc_r", s,
               tc_cat_r_kernel<<<(unsigned)min64((int64_t)sm_count_tc() * 16, (rwork + 255) / 256), 256, 0, s>>>(
                   C.inst, C.tile_inst, C.np, (int)C.kr, rb));
    auto kg = gmm_tc_gram_kernel<TDP>;
    if (!set_smem_tc(kg, GramSm<TDP>::SMEM)) return GPA_ERR_CUDA;
    if (C.n_gram > 0)
        GPA_LAUNCH("gmm_tc_bwd", s,
                   kg<<<(unsigned)C.n_gram, GTHREADS, GramSm<TDP>::SMEM, s>>>(
                       tmr, (const __nv_bfloat16*)C.xt, 0, 0, 0, 16, 1, 1, nullptr, nullptr, gmm_bwd_partial_entries(TDP), 16, C.inst,
                       C.gram_items, C.status));
    return GPA_OK;
}

}  // namespace

int gmm_tc_cat_run(const TcCatClass& C, cudaStream_t s) {
    if (C.np % TM || C.np <= 0 || C.kc <= 0 || C.kr % 16 || C.kr <= 0) return GPA_ERR_ARG;
    return C.tdp == 64 ? cat_run<64>(C, s) : C.tdp == 128 ? cat_run<128>(C, s) : GPA_ERR_UNSUPPORTED;
}

int gmm_tc_cat_gram_groups(int d, int k) { return gram_groups(d) * ((tc_r_rows(k) + GKMAX - 1) / GKMAX); }

bool gmm_tc_supported(int d) { return d > 32 && d <= 128; }

size_t gmm_tc_extra_bytes(int64_t n, int d, int k) {
    const int tdp = tc_dp(d);
    const int64_t npad = ((n + TM - 1) / TM) * TM;
    return 2 * a1024((size_t)npad * tdp * 2) + 2 * a1024((size_t)k * tdp * tdp * 2) +
           a1024((size_t)k * (tdp + 4) * 4) + a1024((size_t)tc_r_rows(k) * tc_r_points(npad) * 2) +
           a1024((size_t)npad * d * 2) + 2048;
}

int gmm_tc_objective_run(const GmmArgs& A, const GmmLayout& L, char* ws, size_t ws_bytes, cudaStream_t s) {
    return tc_dp(A.d) == 64 ? objective_run<64>(A, L, ws, ws_bytes, s) : objective_run<128>(A, L, ws, ws_bytes, s);
}

int gmm_tc_vjp_run(const GmmArgs& A, const GmmLayout& L, char* ws, size_t ws_bytes, cudaStream_t s, int stages) {
    return tc_dp(A.d) == 64 ? vjp_run<64>(A, L, ws, ws_bytes, s, stages) : vjp_run<128>(A, L, ws, ws_bytes, s, stages);
}

int gmm_tc_bwd_nchunks(int64_t n, int d, int k) {
    const GmmLayout L = gmm_layout(n, d, k, 0);
    const TcLayout T = tc_layout(L, n, d, k);
    return tc_dp(d) == 64 ? vjp_chunks<64>(n, d, k, T.rpoints) : vjp_chunks<128>(n, d, k, T.rpoints);
}

}  // namespace gpa
