// Gaussian mixture with a Wishart prior: forward pass and reverse-mode gradient,
// FP32 on the CUDA cores (GPA_PREC_FP32).
//
// The program, per point i and component k (Q_k lower triangular):
//   s_ik = alpha_k + sum_d q_kd - |Q_k x_i - b_k|^2 / 2,   b_k = Q_k mu_k
//   f    = sum_i logsumexp_k s_ik - N logsumexp(alpha) - (N D/2) log 2pi + log-prior
// Forward (A1): one CTA per 128-point tile walks all K components; the
// contraction X Q_k^T is a register-blocked FP32 GEMM that skips the zero upper
// triangle of Q_k; the log-sum-exp over k is an online (max, sum) per point.
// Q_k (transposed, with b_k and the constant) is staged into shared memory by
// 1-D bulk (TMA) copies, double-buffered on mbarriers.
//
// Reverse (A2): grad f x = transpose (linearize f x) 1.0 (Sec. 5.2). With the
// cotangent of s_ik, r_ik = seed * exp(s_ik - lse_i), the reads of alpha_k,
// mu_k and Q_k inside the loop over points become accumulations into their
// cotangents (rule LetIndexingTranspose), regular segmented reductions indexed
// by k (Sec. 6.1.3). All of them follow from three Accum sums per component:
//   R_k = sum_i r_ik,  m_k = sum_i r_ik x_i,  S_k = sum_i r_ik x_i x_i^T,
// so the backward pass needs no recomputation of Q_k x_i: the forward pass's
// log-joint s_ik is stored (or recomputed chunk-wise under a memory budget) and
// the backward kernel is a symmetric rank-N update per component.
//
// Finalize (A3), per component, in a fixed order (deterministic):
//   C_k = S_k - mu m^T - m mu^T + R mu mu^T = sum_i r (x_i - mu)(x_i - mu)^T
//   H_k = Q_k C_k                (= sum_i r z_i (x_i - mu)^T, z = Q(x - mu))
//   d alpha_k += R_k - seed N softmax(alpha)_k
//   d mu_k    += Q_k^T Q_k (m_k - R_k mu_k)
//   d q_kr    += R_k - exp(q_kr) H_k[r][r] + seed (m - gamma^2 exp(2 q_kr))
//   d l_k(rc) += -H_k[r][c] - seed gamma^2 l_k(rc)
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "common.cuh"
#include "gmm_internal.cuh"
#include "gmm_kernels.cuh"
#include "trace.cuh"

namespace gpa {

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

int gmm_dp(int d) { return d <= 16 ? 16 : d <= 32 ? 32 : d <= 64 ? 64 : d <= 128 ? 128 : 0; }

template <int DP>
static int bwd_nblk() { return Bwd<DP>::NBLK; }

static int nblk_of(int dp) {
    switch (dp) {
        case 16: return Bwd<16>::NBLK;
        case 32: return Bwd<32>::NBLK;
        case 64: return Bwd<64>::NBLK;
        default: return Bwd<128>::NBLK;
    }
}
static int rec_of(int dp) { return dp * dp + dp + 4; }

GmmLayout gmm_layout(int64_t n, int d, int k, int64_t lj_points) {
    GmmLayout L{};
    L.dp = gmm_dp(d);
    L.ntiles = (n + 127) / 128;
    L.nchunk_max = kGmmMaxChunks;
    size_t off = 0;
    L.off_rec = off;  off = align256(off + sizeof(float) * (size_t)k * rec_of(L.dp));
    L.off_scal = off; off = align256(off + sizeof(double) * 8);
    L.off_lpk = off;  off = align256(off + sizeof(double) * (size_t)k);
    L.off_fwd = off;  off = align256(off + sizeof(double) * (size_t)L.ntiles);
    L.off_bS = off;   off = align256(off + sizeof(float) * (size_t)L.nchunk_max * k * nblk_of(L.dp) * 64);
    L.off_bM = off;   off = align256(off + sizeof(float) * (size_t)L.nchunk_max * k * (L.dp + 1));
    L.fixed = off;
    L.lj_points = lj_points;
    if (lj_points > 0) {
        L.off_lse = off; off = align256(off + sizeof(float) * (size_t)lj_points);
        L.off_lj = off;  off = align256(off + sizeof(float) * (size_t)lj_points * k);
    }
    L.total = off;
    return L;
}

int64_t gmm_lj_points_for(size_t ws_bytes, const GmmLayout& fixed, int64_t n, int k) {
    if (ws_bytes <= fixed.fixed + 1024) return 0;
    const size_t avail = ws_bytes - fixed.fixed - 1024;  // alignment slack
    int64_t p = (int64_t)(avail / (sizeof(float) * (size_t)(k + 1)));
    p = (p / 128) * 128;
    const int64_t nfull = ((n + 127) / 128) * 128;
    return p < nfull ? p : nfull;
}

template <typename K>
static bool set_smem(K kern, size_t bytes) {
    if (bytes <= 48 * 1024) return true;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) ==
           cudaSuccess;
}

static int num_sms() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

template <int DP>
static int launch_prep(const GmmArgs& A, const GmmLayout& L, char* ws, cudaStream_t s) {
    GPA_LAUNCH("gmm_prep", s,
               gmm_prep_kernel<DP><<<A.k, 128, 0, s>>>(A.alpha, A.mu, A.q, A.l, A.d, A.k, A.gamma, A.m,
                                                       gmm_prior_const(A.d, A.m, A.gamma),
                                                       (float*)(ws + L.off_rec), (double*)(ws + L.off_lpk),
                                                       (double*)(ws + L.off_scal)));
    return GPA_OK;
}

template <int DP>
static int launch_fwd(const GmmArgs& A, const GmmLayout& L, char* ws, const float* x, int64_t n_local,
                      int64_t tile0, float* lj, int64_t lj_ld, float* lse, int32_t* status,
                      cudaStream_t s) {
    using C = Fwd<DP>;
    auto kern = gmm_fwd_kernel<DP>;
    if (!set_smem(kern, C::SMEM)) return GPA_ERR_CUDA;
    const int64_t tiles = (n_local + C::TP - 1) / C::TP;
    GPA_LAUNCH("gmm_fwd", s,
               kern<<<(unsigned)tiles, C::THREADS, C::SMEM, s>>>(x, n_local, A.d, A.k,
                                                                (const float*)(ws + L.off_rec), lj, lj_ld, lse,
                                                                (double*)(ws + L.off_fwd), tile0, status));
    return GPA_OK;
}

// Chunk count for the backward grid: fill whole waves of resident CTAs.
template <int DP>
static int bwd_chunks(int k, int64_t ntiles) {
    using C = Bwd<DP>;
    int occ = 1;
    // the dynamic shared-memory limit must be raised before the query, or a
    // CTA above the 48 KB default reports no residency at all
    if (set_smem(gmm_bwd_kernel<DP>, C::SMEM))
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gmm_bwd_kernel<DP>, C::THREADS, C::SMEM);
    if (occ < 1) occ = 1;
    const int slots = num_sms() * occ;
    const int groups = (k + C::GC - 1) / C::GC;
    int best = 1;
    double best_eff = -1.0;
    for (int c = 1; c <= kGmmMaxChunks; ++c) {
        if (c > ntiles) break;
        const int64_t total = (int64_t)groups * c;
        const int64_t waves = (total + slots - 1) / slots;
        // work per CTA shrinks with c; efficiency = busy / (waves * slots)
        const double eff = (double)total / (double)(waves * slots);
        if (eff > best_eff + 0.02 || (total < slots && eff > best_eff)) {
            best_eff = eff;
            best = c;
        }
    }
    return best;
}

template <int DP>
static int launch_bwd(const GmmArgs& A, const GmmLayout& L, char* ws, const float* x, int64_t n_local,
                      const float* lj, int64_t lj_ld, const float* lse, int nchunks, cudaStream_t s) {
    using C = Bwd<DP>;
    auto kern = gmm_bwd_kernel<DP>;
    if (!set_smem(kern, C::SMEM)) return GPA_ERR_CUDA;
    const int64_t ntiles = (n_local + C::TPB - 1) / C::TPB;
    const int64_t tpc = (ntiles + nchunks - 1) / nchunks;
    dim3 grid((A.k + C::GC - 1) / C::GC, nchunks);
    GPA_LAUNCH("gmm_bwd", s,
               kern<<<grid, C::THREADS, C::SMEM, s>>>(x, n_local, A.d, A.k, lj, lj_ld, lse, (float)A.seed, tpc,
                                                      (float*)(ws + L.off_bS), (float*)(ws + L.off_bM)));
    return GPA_OK;
}

template <int DP>
static int launch_finalize(const GmmArgs& A, const GmmLayout& L, char* ws, int nchunks, cudaStream_t s,
                           int centered = 0) {
    const size_t smem = gmm_finalize_smem<DP>();
    auto kern = gmm_finalize_kernel<DP>;
    if (!set_smem(kern, smem)) return GPA_ERR_CUDA;
    GPA_LAUNCH("gmm_finalize", s,
               kern<<<A.k, 256, smem, s>>>(A.alpha, A.mu, A.q, A.l, A.d, A.k, A.n, A.gamma, A.m, A.seed,
                                           (const float*)(ws + L.off_bS), (const float*)(ws + L.off_bM), nchunks,
                                           (const double*)(ws + L.off_scal), A.d_alpha, A.d_mu, A.d_q, A.d_l,
                                           centered, A.exch_in));
    return GPA_OK;
}

template <int DP>
static int launch_exchange(const GmmArgs& A, const GmmLayout& L, char* ws, int nchunks, cudaStream_t s) {
    GPA_LAUNCH("gmm_exchange", s,
               gmm_exchange_kernel<DP><<<dim3(A.k + 1, (gmm_bwd_partial_entries(DP) + DP + 1 + 255) / 256), 256, 0,
                                         s>>>((const float*)(ws + L.off_bS),
                                                               (const float*)(ws + L.off_bM), nchunks, A.k,
                                                               (const double*)(ws + L.off_fwd), L.ntiles,
                                                               A.exch_out));
    return GPA_OK;
}

static int launch_objective(const GmmArgs& A, const GmmLayout& L, char* ws, cudaStream_t s) {
    GPA_LAUNCH("gmm_objective_finalize", s,
               gmm_objective_finalize_kernel<<<1, 256, 0, s>>>((const double*)(ws + L.off_fwd), L.ntiles,
                                                               (const double*)(ws + L.off_lpk), A.k,
                                                               (const double*)(ws + L.off_scal), A.n, A.d,
                                                               A.out));
    return GPA_OK;
}

template <int DP>
static int objective_impl(const GmmArgs& A, const GmmLayout& L, char* ws, cudaStream_t s) {
    int rc = launch_prep<DP>(A, L, ws, s);
    if (rc) return rc;
    rc = launch_fwd<DP>(A, L, ws, A.x, A.n, 0, A.lj_out, A.n, A.lse_out, A.status, s);
    if (rc) return rc;
    return launch_objective(A, L, ws, s);
}

template <int DP>
static int vjp_impl(const GmmArgs& A, const GmmLayout& L, char* ws, cudaStream_t s) {
    const int64_t ntiles_b = (A.n + Bwd<DP>::TPB - 1) / Bwd<DP>::TPB;
    const int nchunks = bwd_chunks<DP>(A.k, ntiles_b);
    if (cudaMemsetAsync(ws + L.off_bS, 0, sizeof(float) * (size_t)nchunks * A.k * Bwd<DP>::NBLK * 64, s) !=
            cudaSuccess ||
        cudaMemsetAsync(ws + L.off_bM, 0, sizeof(float) * (size_t)nchunks * A.k * (DP + 1), s) != cudaSuccess)
        return GPA_ERR_CUDA;
    int rc = launch_prep<DP>(A, L, ws, s);
    if (rc) return rc;
    if (A.lj_in) {
        rc = launch_bwd<DP>(A, L, ws, A.x, A.n, A.lj_in, A.n, A.lse_in, nchunks, s);
        if (rc) return rc;
        if (A.out || A.exch_out) {
            GPA_LAUNCH("gmm_lse_sum", s,
                       gmm_lse_sum_kernel<<<(unsigned)L.ntiles, 128, 0, s>>>(A.lse_in, A.n,
                                                                            (double*)(ws + L.off_fwd)));
        }
    } else {
        const int64_t P = L.lj_points;  // multiple of 128
        float* lj = (float*)(ws + L.off_lj);
        float* lse = (float*)(ws + L.off_lse);
        for (int64_t c0 = 0; c0 < A.n; c0 += P) {
            const int64_t nl = min64(P, A.n - c0);
            const float* xc = A.x + c0 * A.d;
            rc = launch_fwd<DP>(A, L, ws, xc, nl, c0 / 128, lj, P, lse, A.status, s);
            if (rc) return rc;
            // chunks of the backward grid stay the same across passes so that the
            // partial sums keep one fixed order
            rc = launch_bwd<DP>(A, L, ws, xc, nl, lj, P, lse, nchunks, s);
            if (rc) return rc;
        }
    }
    if (A.exch_out) return launch_exchange<DP>(A, L, ws, nchunks, s);
    rc = launch_finalize<DP>(A, L, ws, nchunks, s);
    if (rc) return rc;
    if (A.out) return launch_objective(A, L, ws, s);
    return GPA_OK;
}

// Stage launchers shared with the tensor-core path (dispatch on L.dp).
int gmm_run_prep(const GmmArgs& A, const GmmLayout& L, char* ws, cudaStream_t s) {
    switch (L.dp) {
        case 16: return launch_prep<16>(A, L, ws, s);
        case 32: return launch_prep<32>(A, L, ws, s);
        case 64: return launch_prep<64>(A, L, ws, s);
        case 128: return launch_prep<128>(A, L, ws, s);
    }
    return GPA_ERR_UNSUPPORTED;
}

int gmm_run_finalize(const GmmArgs& A, const GmmLayout& L, char* ws, int nchunks, int centered, cudaStream_t s) {
    switch (L.dp) {
        case 16: return launch_finalize<16>(A, L, ws, nchunks, s, centered);
        case 32: return launch_finalize<32>(A, L, ws, nchunks, s, centered);
        case 64: return launch_finalize<64>(A, L, ws, nchunks, s, centered);
        case 128: return launch_finalize<128>(A, L, ws, nchunks, s, centered);
    }
    return GPA_ERR_UNSUPPORTED;
}

int gmm_run_objective(const GmmArgs& A, const GmmLayout& L, char* ws, cudaStream_t s) {
    return launch_objective(A, L, ws, s);
}

int gmm_run_lse_sum(const float* lse, int64_t n, const GmmLayout& L, char* ws, cudaStream_t s) {
    GPA_LAUNCH("gmm_lse_sum",
               s, gmm_lse_sum_kernel<<<(unsigned)L.ntiles, 128, 0, s>>>(lse, n, (double*)(ws + L.off_fwd)));
    return GPA_OK;
}

int gmm_bwd_partial_entries(int dp) { return nblk_of(dp) * 64; }

int64_t gmm_exchange_len(int d, int k) {
    const int dp = gmm_dp(d);
    return (int64_t)k * (gmm_bwd_partial_entries(dp) + dp + 1) + 1;
}

int gmm_run_exchange(const GmmArgs& A, const GmmLayout& L, char* ws, int nchunks, cudaStream_t s) {
    switch (L.dp) {
        case 16: return launch_exchange<16>(A, L, ws, nchunks, s);
        case 32: return launch_exchange<32>(A, L, ws, nchunks, s);
        case 64: return launch_exchange<64>(A, L, ws, nchunks, s);
        case 128: return launch_exchange<128>(A, L, ws, nchunks, s);
    }
    return GPA_ERR_UNSUPPORTED;
}

// Finish the reverse pass from an exchange vector summed over shards: the
// gradient from its Accum sums, the objective from its sum of logsumexp.
static int finalize_from_exchange(const GmmArgs& A, const GmmLayout& L, char* ws, int centered, cudaStream_t s) {
    int rc = gmm_run_prep(A, L, ws, s);
    if (rc) return rc;
    if ((rc = gmm_run_finalize(A, L, ws, 1, centered, s))) return rc;
    if (!A.out) return GPA_OK;
    const int dp = gmm_dp(A.d);
    const int64_t E = gmm_bwd_partial_entries(dp) + dp + 1;
    GPA_LAUNCH("gmm_objective_finalize", s,
               gmm_objective_finalize_kernel<<<1, 256, 0, s>>>(A.exch_in + (size_t)A.k * E, 1,
                                                               (const double*)(ws + L.off_lpk), A.k,
                                                               (const double*)(ws + L.off_scal), A.n, A.d,
                                                               A.out));
    return GPA_OK;
}

int gmm_objective_run(const GmmArgs& A, const GmmLayout& L, char* ws, cudaStream_t s) {
    switch (L.dp) {
        case 16: return objective_impl<16>(A, L, ws, s);
        case 32: return objective_impl<32>(A, L, ws, s);
        case 64: return objective_impl<64>(A, L, ws, s);
        case 128: return objective_impl<128>(A, L, ws, s);
    }
    return GPA_ERR_UNSUPPORTED;
}

int gmm_vjp_run(const GmmArgs& A, const GmmLayout& L, char* ws, cudaStream_t s) {
    switch (L.dp) {
        case 16: return vjp_impl<16>(A, L, ws, s);
        case 32: return vjp_impl<32>(A, L, ws, s);
        case 64: return vjp_impl<64>(A, L, ws, s);
        case 128: return vjp_impl<128>(A, L, ws, s);
    }
    return GPA_ERR_UNSUPPORTED;
}

}  // namespace gpa

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
using namespace gpa;

static int gmm_check(const float* x, const float* alpha, const float* mu, const float* q, const float* l,
                     int64_t n, int32_t d, int32_t k, double gamma, int32_t prec) {
    if (!x || !alpha || !mu || !q || (d > 1 && !l)) return GPA_ERR_ARG;
    if (n < 1 || n > INT32_MAX || d < 1 || d > 128 || k < 1 || k > 4096) return GPA_ERR_ARG;
    if (!(gamma > 0.0)) return GPA_ERR_ARG;
    if (prec != GPA_PREC_FP32 && prec != GPA_PREC_BF16_TC) return GPA_ERR_ARG;
    if (prec == GPA_PREC_BF16_TC && !gmm_tc_supported(d)) return GPA_ERR_UNSUPPORTED;
    return GPA_OK;
}

extern "C" size_t gpa_gmm_workspace_bytes(int64_t n, int32_t d, int32_t k, int32_t prec,
                                          int64_t logjoint_points) {
    if (n < 1 || d < 1 || d > 128 || k < 1) return 0;
    int64_t P = logjoint_points <= 0 ? ((n + 127) / 128) * 128 : (logjoint_points / 128) * 128;
    if (P < 128) P = 128;
    const int64_t nfull = ((n + 127) / 128) * 128;
    if (P > nfull) P = nfull;
    size_t b = gmm_layout(n, d, k, P).total + 1024;
    if (prec == GPA_PREC_BF16_TC) b += gmm_tc_extra_bytes(n, d, k);
    return b;
}

extern "C" int gmm_objective(const float* x, const float* alpha, const float* mu, const float* q,
                             const float* l, int64_t n, int32_t d, int32_t k, double gamma, int32_t m,
                             int32_t prec, double* out, float* lse_out, float* logjoint_out, void* ws,
                             size_t ws_bytes, int32_t* dev_status, gpa_stream_t stream) {
    int rc = gmm_check(x, alpha, mu, q, l, n, d, k, gamma, prec);
    if (rc) return rc;
    if (!out || !ws) return GPA_ERR_ARG;
    if (((uintptr_t)ws) & 255) return GPA_ERR_ALIGN;
    GmmLayout L = gmm_layout(n, d, k, 0);
    if (ws_bytes < L.total) return GPA_ERR_WORKSPACE;
    GmmArgs A{};
    A.x = x; A.alpha = alpha; A.mu = mu; A.q = q; A.l = l; A.n = n; A.d = d; A.k = k;
    A.gamma = gamma; A.m = m; A.out = out; A.lse_out = lse_out; A.lj_out = logjoint_out;
    A.status = dev_status; A.seed = 1.0;
    if (prec == GPA_PREC_BF16_TC) return gmm_tc_objective_run(A, L, (char*)ws, ws_bytes, (cudaStream_t)stream);
    return gmm_objective_run(A, L, (char*)ws, (cudaStream_t)stream);
}

static int vjp_body(const float* x, const float* alpha, const float* mu, const float* q, const float* l,
                    int64_t n, int32_t d, int32_t k, double gamma, int32_t m, int32_t prec,
                    const float* logjoint_in, const float* lse_in, double seed, float* d_alpha, float* d_mu,
                    float* d_q, float* d_l, double* out, double* exch, void* ws, size_t ws_bytes,
                    int32_t* dev_status, gpa_stream_t stream) {
    if ((logjoint_in == nullptr) != (lse_in == nullptr)) return GPA_ERR_ARG;
    if (((uintptr_t)ws) & 255) return GPA_ERR_ALIGN;
    GmmLayout L = gmm_layout(n, d, k, 0);
    if (ws_bytes < L.total) return GPA_ERR_WORKSPACE;
    if (!logjoint_in && prec == GPA_PREC_FP32) {  // the tensor-core path sizes its own chunks
        const int64_t P = gmm_lj_points_for(ws_bytes, L, n, k);
        if (P < 128) return GPA_ERR_WORKSPACE;
        L = gmm_layout(n, d, k, P);
        if (ws_bytes < L.total) return GPA_ERR_WORKSPACE;
    }
    GmmArgs A{};
    A.x = x; A.alpha = alpha; A.mu = mu; A.q = q; A.l = l; A.n = n; A.d = d; A.k = k;
    A.gamma = gamma; A.m = m; A.out = out; A.lj_in = logjoint_in; A.lse_in = lse_in; A.seed = seed;
    A.d_alpha = d_alpha; A.d_mu = d_mu; A.d_q = d_q; A.d_l = d_l; A.status = dev_status; A.exch_out = exch;
    if (prec == GPA_PREC_BF16_TC) return gmm_tc_vjp_run(A, L, (char*)ws, ws_bytes, (cudaStream_t)stream);
    return gmm_vjp_run(A, L, (char*)ws, (cudaStream_t)stream);
}

extern "C" int gmm_vjp(const float* x, const float* alpha, const float* mu, const float* q, const float* l,
                       int64_t n, int32_t d, int32_t k, double gamma, int32_t m, int32_t prec,
                       const float* logjoint_in, const float* lse_in, double seed, float* d_alpha,
                       float* d_mu, float* d_q, float* d_l, double* out, void* ws, size_t ws_bytes,
                       int32_t* dev_status, gpa_stream_t stream) {
    int rc = gmm_check(x, alpha, mu, q, l, n, d, k, gamma, prec);
    if (rc) return rc;
    if (!d_alpha || !d_mu || !d_q || (d > 1 && !d_l) || !ws) return GPA_ERR_ARG;
    return vjp_body(x, alpha, mu, q, l, n, d, k, gamma, m, prec, logjoint_in, lse_in, seed, d_alpha, d_mu, d_q,
                    d_l, out, nullptr, ws, ws_bytes, dev_status, stream);
}

extern "C" int64_t gpa_gmm_exchange_len(int32_t d, int32_t k) {
    if (d < 1 || d > 128 || k < 1 || k > 4096) return 0;
    return gmm_exchange_len(d, k);
}

extern "C" int gmm_vjp_partial(const float* x, const float* alpha, const float* mu, const float* q,
                               const float* l, int64_t n, int32_t d, int32_t k, double gamma, int32_t m,
                               int32_t prec, const float* logjoint_in, const float* lse_in, double seed,
                               double* exch, void* ws, size_t ws_bytes, int32_t* dev_status,
                               gpa_stream_t stream) {
    int rc = gmm_check(x, alpha, mu, q, l, n, d, k, gamma, prec);
    if (rc) return rc;
    if (!exch || !ws) return GPA_ERR_ARG;
    if (((uintptr_t)exch) & 7) return GPA_ERR_ALIGN;
    return vjp_body(x, alpha, mu, q, l, n, d, k, gamma, m, prec, logjoint_in, lse_in, seed, nullptr, nullptr,
                    nullptr, nullptr, nullptr, exch, ws, ws_bytes, dev_status, stream);
}

extern "C" int gmm_vjp_finalize(const float* alpha, const float* mu, const float* q, const float* l,
                                int64_t n_total, int32_t d, int32_t k, double gamma, int32_t m, int32_t prec,
                                double seed, const double* exch, float* d_alpha, float* d_mu, float* d_q,
                                float* d_l, double* out, void* ws, size_t ws_bytes, int32_t* dev_status,
                                gpa_stream_t stream) {
    if (!alpha || !mu || !q || (d > 1 && !l) || !exch || !ws) return GPA_ERR_ARG;
    if (n_total < 1 || d < 1 || d > 128 || k < 1 || k > 4096 || !(gamma > 0.0)) return GPA_ERR_ARG;
    if (prec != GPA_PREC_FP32 && prec != GPA_PREC_BF16_TC) return GPA_ERR_ARG;
    if (prec == GPA_PREC_BF16_TC && !gmm_tc_supported(d)) return GPA_ERR_UNSUPPORTED;
    if (!d_alpha || !d_mu || !d_q || (d > 1 && !d_l)) return GPA_ERR_ARG;
    if ((((uintptr_t)ws) & 255) || (((uintptr_t)exch) & 7)) return GPA_ERR_ALIGN;
    const GmmLayout L = gmm_layout(1, d, k, 0);
    if (ws_bytes < L.off_fwd) return GPA_ERR_WORKSPACE;  // records, scalars, log-prior
    GmmArgs A{};
    A.alpha = alpha; A.mu = mu; A.q = q; A.l = l; A.n = n_total; A.d = d; A.k = k; A.gamma = gamma; A.m = m;
    A.seed = seed; A.out = out; A.d_alpha = d_alpha; A.d_mu = d_mu; A.d_q = d_q; A.d_l = d_l;
    A.status = dev_status; A.exch_in = exch;
    return finalize_from_exchange(A, L, (char*)ws, 0, (cudaStream_t)stream);  // raw moments from either path
}
