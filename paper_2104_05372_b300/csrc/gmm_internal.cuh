// Internal interface between the GMM C-ABI entry points and the FP32 and
// tensor-core implementations.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>
#include <stdint.h>

namespace gpa {

constexpr int kGmmMaxChunks = 64;  // point chunks of the backward grid (partials)

struct GmmArgs {
    const float *x, *alpha, *mu, *q, *l;
    int64_t n;
    int d, k;
    double gamma;
    int m;
    double seed;
    double* out;
    float* lse_out;
    float* lj_out;
    const float* lj_in;
    const float* lse_in;
    float *d_alpha, *d_mu, *d_q, *d_l;
    int32_t* status;
    double* exch_out;        // reverse pass: write the shard's exchange vector instead of finishing
    const double* exch_in;   // finish from a (summed) exchange vector
};

// Workspace layout (byte offsets, 256-byte aligned) of the FP32 path.
struct GmmLayout {
    int dp;              // padded dimension (16, 32, 64, 128)
    int64_t ntiles;      // 128-point tiles over N
    int nchunk_max;
    size_t off_rec;      // K staged records: Qt[DP][DP], b[DP], cst, pad (float)
    size_t off_scal;     // float64 scalars: [0] logsumexp(alpha)
    size_t off_lpk;      // float64 log-prior per component
    size_t off_fwd;      // float64 per-tile sums of lse
    size_t off_bS;       // float partial S blocks [chunk][K][NBLK][64]
    size_t off_bM;       // float partial m, R     [chunk][K][DP+1]
    size_t fixed;        // bytes before the log-joint area
    int64_t lj_points;   // points per log-joint chunk (0: none)
    size_t off_lse;      // float lse of the current chunk
    size_t off_lj;       // float log-joint [K][lj_points]
    size_t total;
};

int gmm_dp(int d);
GmmLayout gmm_layout(int64_t n, int d, int k, int64_t lj_points);
int64_t gmm_lj_points_for(size_t ws_bytes, const GmmLayout& fixed, int64_t n, int k);
int gmm_objective_run(const GmmArgs& A, const GmmLayout& L, char* ws, cudaStream_t s);
int gmm_vjp_run(const GmmArgs& A, const GmmLayout& L, char* ws, cudaStream_t s);

// Stages shared by both paths.
int gmm_run_prep(const GmmArgs& A, const GmmLayout& L, char* ws, cudaStream_t s);
int gmm_run_finalize(const GmmArgs& A, const GmmLayout& L, char* ws, int nchunks, int centered, cudaStream_t s);
int gmm_run_objective(const GmmArgs& A, const GmmLayout& L, char* ws, cudaStream_t s);
int gmm_run_lse_sum(const float* lse, int64_t n, const GmmLayout& L, char* ws, cudaStream_t s);
int gmm_bwd_partial_entries(int dp);  // floats of partial S per (chunk, component)
int64_t gmm_exchange_len(int d, int k);  // doubles of the exchange vector
int gmm_run_exchange(const GmmArgs& A, const GmmLayout& L, char* ws, int nchunks, cudaStream_t s);

// Tensor-core (tcgen05, BF16 operands, FP32 accumulate) path.
bool gmm_tc_supported(int d);
size_t gmm_tc_extra_bytes(int64_t n, int d, int k);
int gmm_tc_objective_run(const GmmArgs& A, const GmmLayout& L, char* ws, size_t ws_bytes, cudaStream_t s);
// Stages of a reverse pass: parameter expansion, the contractions, the
// finalize (gradient and objective). The batched form runs the first and last
// in its persistent kernels and asks the tensor-core path for the middle only.
enum : int { kGmmStagePrep = 1, kGmmStageCore = 2, kGmmStageFinish = 4, kGmmStagesAll = 7 };
int gmm_tc_vjp_run(const GmmArgs& A, const GmmLayout& L, char* ws, size_t ws_bytes, cudaStream_t s,
                   int stages = kGmmStagesAll);
int gmm_tc_bwd_nchunks(int64_t n, int d, int k);  // point chunks (partial sums) of the reverse pass

// Batched form, tensor-core instances of one padded dimension run together:
// their points, Q records, BF16 responsibilities and transposed point tiles
// live in concatenated buffers (each instance's points at a row offset that is
// a multiple of 128), and each stage is one launch over every instance's
// tiles. Device descriptors, built on the host by the batched plan.
struct TcCatInst {
    const float* x;              // [n][d] points
    float* lj;                   // [k][npad] log-joint (rows of n padded to whole 128-point tiles)
    float* lse;                  // [n] per-point logsumexp
    double* fwd;                 // [ceil(n / 128)] per-tile sums of lse
    float *bS, *bM;              // partial sums [nchunks][k][...] (zeroed by the caller)
    int64_t n, xoff, xtoff;      // points; first row in x / R; element offset of its point tiles
    int64_t tpc;                 // 64-point tiles per backward chunk
    int d, k, koff, kn, ng, nchunks;
    float seed;
};
struct TcCatClass {
    int tdp;
    int64_t np, kc, kr;          // rows of x / columns of R; components; rows of R
    const TcCatInst* inst;       // [instances]
    const int* tile_inst;        // [np / 128] instance of each 128-row tile
    const int2* fwd_tiles;       // [n_fwd] (instance, tile within it), longest first
    const int4* gram_items;      // [n_gram] (instance, product/component group, chunk, 0), longest first
    int n_fwd, n_gram;
    const float* rec;            // [kc] prep records
    float* tails;                // [kc][tdp + 4] b_k and constants
    void *xb, *xl, *qb, *ql, *rb;  // bf16 x_hi, x_lo [np][tdp]; Q_hi, Q_lo (kc * tdp * tdp each); R [kr][np]
    void* xt;                    // bf16 point tiles
    int32_t* status;
};
int gmm_tc_cat_run(const TcCatClass& C, cudaStream_t s);
int gmm_tc_cat_gram_groups(int d, int k);  // product x component groups of one instance

// The data-independent part of each component's Wishart log-prior, for
// n = d + m + 1 degrees of freedom: n d log(gamma) - (n d / 2) log 2 - log
// Gamma_d(n/2), with log Gamma_d(a) = d (d - 1) / 4 log(pi) + sum_{j<d}
// lgamma(a - j / 2). Computed once per call on the host in float64.
inline double gmm_prior_const(int d, int m, double gamma) {
    const double nn = (double)(d + m + 1);
    double lg = 0.0;
    for (int j = 0; j < d; ++j) lg += lgamma(0.5 * nn - 0.5 * (double)j);
    const double log_mvg = 0.25 * d * (d - 1) * log(3.14159265358979323846) + lg;
    return nn * d * log(gamma) - 0.5 * nn * d * log(2.0) - log_mvg;
}

}  // namespace gpa
