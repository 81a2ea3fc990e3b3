// Gaussian mixture: forward-mode directional derivative df(theta)[v]
// (linearize, Sec. 5.1), FP32 on the CUDA cores.
//
// The tangent travels with the value through every point and component:
//   z_ik  = Q_k x_i - b_k,                      b_k  = Q_k mu_k
//   zd_ik = Qd_k x_i - bd_k,                    bd_k = Qd_k mu_k + Q_k v_mu_k
//   s_ik  = cst_k - |z_ik|^2 / 2,               cst_k  = alpha_k + sum_d q_kd
//   sd_ik = cstd_k - z_ik . zd_ik,              cstd_k = v_alpha_k + sum_d v_q_kd
// with Qd_k the tangent of Q_k (exp(q_kr) v_q_kr on the diagonal, v_l below
// it). Per point, an online logsumexp carries the tangent along:
//   lse_i = logsumexp_k s_ik,   lsed_i = sum_k softmax_k(s_i.) sd_ik,
// and df = sum_i lsed_i - N sum_k softmax(alpha)_k v_alpha_k + (prior)'[v].
// Unlike the reverse pass, which reduces over points first (Accum sums), this
// pass produces the tangent of every per-point statistic, so the two meet
// only in <grad f, v> = df[v] (Sec. 5.2) and check one another.
//
// Kernel layout follows the forward pass (one CTA per 128-point tile, Q_k
// staged by 1-D bulk copies), with the tangent record Qd_k, bd_k, cstd_k
// staged next to each value record and a second triangular contraction.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "common.cuh"
#include "gmm_internal.cuh"
#include "gmm_kernels.cuh"
#include "trace.cuh"

namespace gpa {
namespace {

template <int DP>
struct Jvp {
    using F = Fwd<DP>;
    static constexpr int NWC = F::NWC, NS = F::NS, TP = F::TP, XST = F::XST, REC = F::REC;
    static constexpr int NBUF = DP == 128 ? 1 : 2;  // record buffers (one at DP = 128: shared memory)
    static constexpr int THREADS = 256;
    static constexpr size_t SMEM =
        sizeof(float) * (size_t)(DP * XST + NBUF * NS * 2 * REC + 2 * 2 * NS * NWC * TP + 3 * NS * TP) + 64;
    static_assert(SMEM <= 227 * 1024, "jvp shared memory");
};

// Online logsumexp with a tangent: l = sum e^(s - m), t = sum e^(s - m) sd.
struct LseT {
    float m, l, t;
    __device__ __forceinline__ void init() {
        m = -INFINITY;
        l = 0.f;
        t = 0.f;
    }
    __device__ __forceinline__ void add(float v, float vd) {
        if (v > m) {
            const float sc = m == -INFINITY ? 0.f : expf(m - v);
            l = l * sc + 1.f;
            t = t * sc + vd;
            m = v;
        } else {
            const float e = expf(v - m);
            l += e;
            t = fmaf(e, vd, t);
        }
    }
    __device__ __forceinline__ void merge(float m2, float l2, float t2) {
        if (m2 == -INFINITY) return;
        if (m == -INFINITY) {
            m = m2;
            l = l2;
            t = t2;
            return;
        }
        const float mx = fmaxf(m, m2);
        const float a = expf(m - mx), b = expf(m2 - mx);
        l = l * a + l2 * b;
        t = t * a + t2 * b;
        m = mx;
    }
};

// Tangent record of component k: Qd^T[c][r], bd[r], cstd, pad (the value
// record's layout); the log-prior's tangent; sum_k softmax(alpha)_k v_alpha_k.
template <int DP>
__global__ void __launch_bounds__(128) gmm_jvp_prep_kernel(
    const float* __restrict__ alpha, const float* __restrict__ mu, const float* __restrict__ q,
    const float* __restrict__ l, int d, int k, double gamma, int m, const float* __restrict__ v_alpha,
    const float* __restrict__ v_mu, const float* __restrict__ v_q, const float* __restrict__ v_l,
    float* __restrict__ recd, double* __restrict__ lpkd, double* __restrict__ scald) {
    constexpr int REC = Fwd<DP>::REC;
    const int kk = blockIdx.x;
    const int t = d * (d - 1) / 2;
    float* R = recd + (size_t)kk * REC;
    const float* qk = q + (size_t)kk * d;
    const float* lk = l + (size_t)kk * t;
    const float* muk = mu + (size_t)kk * d;
    const float* vqk = v_q + (size_t)kk * d;
    const float* vlk = v_l + (size_t)kk * t;
    const float* vmk = v_mu + (size_t)kk * d;
    auto Qrc = [&](int r, int c) -> float {
        if (r >= d || c > r) return 0.f;
        return (c == r) ? expf(qk[r]) : lk[r * (r - 1) / 2 + c];
    };
    auto Qdrc = [&](int r, int c) -> float {
        if (r >= d || c > r) return 0.f;
        return (c == r) ? expf(qk[r]) * vqk[r] : vlk[r * (r - 1) / 2 + c];
    };
    for (int e = threadIdx.x; e < DP * DP; e += blockDim.x) {
        const int c = e / DP, r = e % DP;
        R[e] = Qdrc(r, c);  // transposed: Qd^T[c][r]
    }
    for (int r = threadIdx.x; r < DP; r += blockDim.x) {
        double s = 0.0;
        if (r < d)
            for (int c = 0; c <= r; ++c) s += (double)Qdrc(r, c) * (double)muk[c] + (double)Qrc(r, c) * (double)vmk[c];
        R[DP * DP + r] = (float)s;
    }
    // sum_d v_q; prior tangent: m sum v_q - gamma^2 (sum exp(2q) v_q + sum l v_l)
    double sv = 0.0, pr = 0.0;
    for (int r = threadIdx.x; r < d; r += blockDim.x) {
        sv += vqk[r];
        pr += exp(2.0 * (double)qk[r]) * (double)vqk[r];
    }
    for (int j = threadIdx.x; j < t; j += blockDim.x) pr += (double)lk[j] * (double)vlk[j];
    __shared__ double red[2][4];
    sv = warp_sum(sv);
    pr = warp_sum(pr);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = sv;
        red[1][threadIdx.x >> 5] = pr;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        sv = red[0][0] + red[0][1] + red[0][2] + red[0][3];
        pr = red[1][0] + red[1][1] + red[1][2] + red[1][3];
        R[DP * DP + DP] = (float)((double)v_alpha[kk] + sv);
        R[DP * DP + DP + 1] = 0.f;
        R[DP * DP + DP + 2] = 0.f;
        R[DP * DP + DP + 3] = 0.f;
        lpkd[kk] = (double)m * sv - gamma * gamma * pr;
        if (kk == 0) {
            double mx = -INFINITY;
            for (int i = 0; i < k; ++i) mx = fmax(mx, (double)alpha[i]);
            double z = 0.0, w = 0.0;
            for (int i = 0; i < k; ++i) {
                const double e = exp((double)alpha[i] - mx);
                z += e;
                w += e * (double)v_alpha[i];
            }
            scald[0] = w / z;
        }
    }
}

// One CTA per 128-point tile; per round NS components, each staged as
// [value record | tangent record].
template <int DP>
__global__ void __launch_bounds__(256) gmm_jvp_kernel(const float* __restrict__ x, int64_t n, int d, int k,
                                                      const float* __restrict__ rec, const float* __restrict__ recd,
                                                      float* __restrict__ lse_dot_out, double* __restrict__ part,
                                                      double* __restrict__ partd, int32_t* __restrict__ status) {
    using C = Jvp<DP>;
    constexpr int TP = C::TP, XST = C::XST, NS = C::NS, NWC = C::NWC, REC = C::REC, NBUF = C::NBUF;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* Xs = reinterpret_cast<float*>(smem_raw);  // [DP][XST]
    float* Qb = Xs + DP * XST;                        // [NBUF][NS][2][REC]
    float* red = Qb + NBUF * NS * 2 * REC;            // [2 rounds][2 sums][NS][NWC][TP]
    float* st = red + 2 * 2 * NS * NWC * TP;          // [NS][TP][3]
    uint64_t* bar = reinterpret_cast<uint64_t*>(st + 3 * NS * TP);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int slot = warp / NWC, wl = warp % NWC;
    const int64_t p0 = (int64_t)blockIdx.x * TP;
    const int nvalid = (int)min64(TP, n - p0);
    const int rounds = (k + NS - 1) / NS;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    for (int e = tid; e < DP * XST; e += C::THREADS) Xs[e] = 0.f;
    __syncthreads();
    for (int e = tid; e < nvalid * d; e += C::THREADS) {
        const int p = e / d, c = e - p * d;
        Xs[c * XST + p] = __ldg(x + (p0 + p) * d + c);
    }
    // records of `round` into buffer round % NBUF, completion on bar[round % NBUF]
    auto issue = [&](int round) {
        const int buf = round % NBUF;
        int nb = 0;
        for (int s = 0; s < NS; ++s) nb += (round * NS + s < k) ? 1 : 0;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bar[buf], (uint32_t)(nb * 2 * REC * sizeof(float)));
        for (int s = 0; s < NS; ++s) {
            const int kk = round * NS + s;
            if (kk < k) {
                float* dst = Qb + (buf * NS + s) * 2 * REC;
                bulk_g2s(dst, rec + (size_t)kk * REC, REC * sizeof(float), &bar[buf]);
                bulk_g2s(dst + REC, recd + (size_t)kk * REC, REC * sizeof(float), &bar[buf]);
            }
        }
    };
    if (tid == 0) issue(0);

    constexpr int NPAIR = (NS * TP + C::THREADS - 1) / C::THREADS;
    LseT ls[NPAIR];
#pragma unroll
    for (int u = 0; u < NPAIR; ++u) ls[u].init();

    bool ok = true;
    int last_issued = 0;
    for (int round = 0; round < rounds; ++round) {
        const int buf = round % NBUF;
        const uint32_t phase = (uint32_t)(round / NBUF) & 1u;
        if (NBUF == 2 && tid == 0 && round + 1 < rounds) {
            issue(round + 1);
            last_issued = round + 1;
        }
        ok = mbar_wait(&bar[buf], phase, status) && ok;
        ok = __syncthreads_and(ok);  // Xs ready (round 0); all threads agree on ok
        if (!ok) break;
        const int kk = round * NS + slot;
        float* redb = red + (round & 1) * 2 * NS * NWC * TP;
        if (kk < k) {
            const float* Q = Qb + (buf * NS + slot) * 2 * REC;
            const float* Qd = Q + REC;
            float2 zb[4][8], zd[4][8];
            fwd_gemm_packed<DP>(Xs, Q, lane, wl, zb);   // Q x - b
            fwd_gemm_packed<DP>(Xs, Qd, lane, wl, zd);  // Q' x - b'
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float2 s2 = make_float2(0.f, 0.f), sd = make_float2(0.f, 0.f);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    s2 = __ffma2_rn(zb[j][i], zb[j][i], s2);
                    sd = __ffma2_rn(zb[j][i], zd[j][i], sd);
                }
                redb[(slot * NWC + wl) * TP + lane * 4 + j] = s2.x + s2.y;
                redb[NS * NWC * TP + (slot * NWC + wl) * TP + lane * 4 + j] = sd.x + sd.y;
            }
        }
        fence_proxy_async_smem();  // reads of the records before the bulk copy that refills them
        __syncthreads();           // partial sums complete; the records of this round are no longer read
        if (NBUF == 1 && tid == 0 && round + 1 < rounds) {
            issue(round + 1);
            last_issued = round + 1;
        }
#pragma unroll
        for (int u = 0; u < NPAIR; ++u) {
            const int e = tid + u * C::THREADS;
            if (e < NS * TP) {
                const int s = e / TP, p = e % TP;
                const int kc = round * NS + s;
                if (kc < k && p < nvalid) {
                    float t2 = 0.f, td = 0.f;
#pragma unroll
                    for (int w = 0; w < NWC; ++w) {
                        t2 += redb[(s * NWC + w) * TP + p];
                        td += redb[NS * NWC * TP + (s * NWC + w) * TP + p];
                    }
                    const float sv = __ldg(rec + (size_t)kc * REC + DP * DP + DP) - 0.5f * t2;
                    const float svd = __ldg(recd + (size_t)kc * REC + DP * DP + DP) - td;
                    ls[u].add(sv, svd);
                }
            }
        }
    }
    if (!ok && tid == 0) {
        // a wait gave up: let this CTA's copies in flight land (bounded) before exiting
        (void)mbar_wait(&bar[last_issued % NBUF], (uint32_t)(last_issued / NBUF) & 1u, status);
        if (NBUF == 2 && last_issued > 0)
            (void)mbar_wait(&bar[(last_issued - 1) % NBUF], (uint32_t)((last_issued - 1) / NBUF) & 1u, status);
    }
#pragma unroll
    for (int u = 0; u < NPAIR; ++u) {
        const int e = tid + u * C::THREADS;
        if (e < NS * TP) {
            st[3 * e] = ls[u].m;
            st[3 * e + 1] = ls[u].l;
            st[3 * e + 2] = ls[u].t;
        }
    }
    __syncthreads();
    double v = 0.0, vd = 0.0;
    if (tid < TP) {
        LseT a;
        a.init();
        for (int s = 0; s < NS; ++s) {
            const float* q3 = st + 3 * (s * TP + tid);
            a.merge(q3[0], q3[1], q3[2]);
        }
        if (tid < nvalid && ok) {
            const float ld = a.t / a.l;
            if (lse_dot_out) lse_dot_out[p0 + tid] = ld;
            v = (double)(a.m + logf(a.l));
            vd = (double)ld;
        }
    }
    __shared__ double wsum[2][8];
    v = warp_sum(v);
    vd = warp_sum(vd);
    if (lane == 0) {
        wsum[0][warp] = v;
        wsum[1][warp] = vd;
    }
    __syncthreads();
    if (tid == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < 8; ++w) {
            a += wsum[0][w];
            b += wsum[1][w];
        }
        part[blockIdx.x] = ok ? a : NAN;
        partd[blockIdx.x] = ok ? b : NAN;
    }
}

// df = sum of tile tangents + prior tangent - N sum softmax(alpha) v_alpha; f as the forward pass.
__global__ void __launch_bounds__(256) gmm_jvp_finalize_kernel(const double* __restrict__ part,
                                                               const double* __restrict__ partd, int64_t ntiles,
                                                               const double* __restrict__ lpk,
                                                               const double* __restrict__ lpkd, int k,
                                                               const double* __restrict__ scal,
                                                               const double* __restrict__ scald, int64_t n, int d,
                                                               double* __restrict__ df_out, double* __restrict__ f_out) {
    __shared__ double sh[2][256];
    double s = 0.0, sd = 0.0;
    for (int64_t t = threadIdx.x; t < ntiles; t += 256) {
        s += part[t];
        sd += partd[t];
    }
    for (int64_t t = threadIdx.x; t < k; t += 256) {
        s += lpk[t];
        sd += lpkd[t];
    }
    sh[0][threadIdx.x] = s;
    sh[1][threadIdx.x] = sd;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *df_out = sh[1][0] - (double)n * scald[0];
        if (f_out) *f_out = sh[0][0] - (double)n * scal[0] - 0.5 * (double)n * d * log(2.0 * 3.14159265358979323846);
    }
}

struct JvpLayout {
    GmmLayout L;  // value records, scalars, log-prior, tile sums (forward-pass offsets)
    size_t off_recd, off_lpkd, off_scald, off_partd, total;
};

size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

JvpLayout jvp_layout(int64_t n, int d, int k) {
    JvpLayout J{};
    const int dp = gmm_dp(d);
    const size_t rec = sizeof(float) * (size_t)k * (dp * dp + dp + 4);
    J.L.dp = dp;
    J.L.ntiles = (n + 127) / 128;
    size_t off = 0;
    J.L.off_rec = off;   off = a256(off + rec);
    J.L.off_scal = off;  off = a256(off + sizeof(double) * 8);
    J.L.off_lpk = off;   off = a256(off + sizeof(double) * (size_t)k);
    J.L.off_fwd = off;   off = a256(off + sizeof(double) * (size_t)J.L.ntiles);
    J.off_recd = off;    off = a256(off + rec);
    J.off_lpkd = off;    off = a256(off + sizeof(double) * (size_t)k);
    J.off_scald = off;   off = a256(off + sizeof(double) * 8);
    J.off_partd = off;   off = a256(off + sizeof(double) * (size_t)J.L.ntiles);
    J.total = off;
    return J;
}

template <int DP>
int jvp_run(const GmmArgs& A, const float* va, const float* vm, const float* vq, const float* vl, double* df,
            double* f, float* lse_dot, const JvpLayout& J, char* ws, cudaStream_t s) {
    using C = Jvp<DP>;
    int rc = gmm_run_prep(A, J.L, ws, s);
    if (rc) return rc;
    GPA_LAUNCH("gmm_jvp_prep", s,
               gmm_jvp_prep_kernel<DP><<<A.k, 128, 0, s>>>(A.alpha, A.mu, A.q, A.l, A.d, A.k, A.gamma, A.m, va, vm,
                                                           vq, vl, (float*)(ws + J.off_recd),
                                                           (double*)(ws + J.off_lpkd), (double*)(ws + J.off_scald)));
    auto kern = gmm_jvp_kernel<DP>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM) != cudaSuccess)
        return GPA_ERR_CUDA;
    GPA_LAUNCH("gmm_jvp", s,
               kern<<<(unsigned)J.L.ntiles, C::THREADS, C::SMEM, s>>>(
                   A.x, A.n, A.d, A.k, (const float*)(ws + J.L.off_rec), (const float*)(ws + J.off_recd), lse_dot,
                   (double*)(ws + J.L.off_fwd), (double*)(ws + J.off_partd), A.status));
    GPA_LAUNCH("gmm_jvp_finalize", s,
               gmm_jvp_finalize_kernel<<<1, 256, 0, s>>>(
                   (const double*)(ws + J.L.off_fwd), (const double*)(ws + J.off_partd), J.L.ntiles,
                   (const double*)(ws + J.L.off_lpk), (const double*)(ws + J.off_lpkd), A.k,
                   (const double*)(ws + J.L.off_scal), (const double*)(ws + J.off_scald), A.n, A.d, df, f));
    return GPA_OK;
}

}  // namespace
}  // namespace gpa

using namespace gpa;

extern "C" size_t gpa_gmm_jvp_workspace_bytes(int64_t n, int32_t d, int32_t k) {
    if (n < 1 || d < 1 || d > 128 || k < 1) return 0;
    return jvp_layout(n, d, k).total;
}

extern "C" int gmm_jvp(const float* x, const float* alpha, const float* mu, const float* q, const float* l,
                       int64_t n, int32_t d, int32_t k, double gamma, int32_t m, const float* v_alpha,
                       const float* v_mu, const float* v_q, const float* v_l, double* df_out, double* f_out,
                       float* lse_dot_out, void* ws, size_t ws_bytes, int32_t* dev_status, gpa_stream_t stream) {
    if (!x || !alpha || !mu || !q || (d > 1 && !l)) return GPA_ERR_ARG;
    if (!v_alpha || !v_mu || !v_q || (d > 1 && !v_l) || !df_out || !ws) return GPA_ERR_ARG;
    if (n < 1 || n > INT32_MAX || d < 1 || d > 128 || k < 1 || k > 4096 || !(gamma > 0.0)) return GPA_ERR_ARG;
    if (((uintptr_t)ws) & 255) return GPA_ERR_ALIGN;
    const JvpLayout J = jvp_layout(n, d, k);
    if (ws_bytes < J.total) return GPA_ERR_WORKSPACE;
    GmmArgs A{};
    A.x = x; A.alpha = alpha; A.mu = mu; A.q = q; A.l = l; A.n = n; A.d = d; A.k = k;
    A.gamma = gamma; A.m = m; A.status = dev_status; A.seed = 1.0;
    cudaStream_t s = (cudaStream_t)stream;
    switch (J.L.dp) {
        case 16: return jvp_run<16>(A, v_alpha, v_mu, v_q, v_l, df_out, f_out, lse_dot_out, J, (char*)ws, s);
        case 32: return jvp_run<32>(A, v_alpha, v_mu, v_q, v_l, df_out, f_out, lse_dot_out, J, (char*)ws, s);
        case 64: return jvp_run<64>(A, v_alpha, v_mu, v_q, v_l, df_out, f_out, lse_dot_out, J, (char*)ws, s);
        case 128: return jvp_run<128>(A, v_alpha, v_mu, v_q, v_l, df_out, f_out, lse_dot_out, J, (char*)ws, s);
    }
    return GPA_ERR_UNSUPPORTED;
}
