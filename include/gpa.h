/*
 * gpa.h -- C ABI of libgpa: forward passes and reverse-mode gradients of two
 * pointful array programs on one NVIDIA B300 (sm_103a), where the adjoint of
 * every gather is an associative accumulation (the Accum effect of
 * "Getting to the Point", arXiv 2104.05372, Sec. 2.3.2), so that the backward
 * pass stays parallel and work-efficient (Sec. 5.3.3, Sec. 6.1.2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Memory.   Every pointer argument is DEVICE memory owned by the caller, unless
 *           the argument's comment says otherwise. Arrays are dense, row-major,
 *           and flatten their index sets in row-major order (tuple index sets,
 *           Sec. 3.4). The library never allocates: scratch space is the
 *           caller's workspace `ws` of `ws_bytes` bytes (256-byte aligned), sized
 *           by the matching *_workspace_bytes query. Workspace contents need no
 *           initialisation and are meaningless after the call.
 * Streams.  Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *           stream) and returns immediately; results are valid once the stream
 *           has been synchronised.
 * Accum.    Gradient outputs (d_*) follow runAccum semantics: the call ADDS its
 *           contribution (+=) into buffers the caller initialised, typically to
 *           zero (Sec. 2.3.2, rule VarTranspose of Fig. "transpose"). Each
 *           element has one writer per call unless the strategy says atomics.
 * Errors.   Host-detectable problems (null pointer, size out of range,
 *           unsupported shape, workspace too small, misaligned pointer) return a
 *           nonzero gpa_status at once and enqueue nothing. Data-dependent
 *           problems found on the device (an index outside its index set, a
 *           bounded wait that ran out) are OR-ed into *dev_status (device int32,
 *           nullable; the caller zeroes it and reads it after synchronising);
 *           the offending element is skipped and the kernel never traps.
 *           GPA_ERR_CUDA reports a failed launch (cudaGetLastError).
 * Precision. Inputs and outputs are float32; objectives are float64 scalars.
 *           GPA_PREC_FP32 computes every product and sum in float32 (sums over
 *           points in float64 where stated); GPA_PREC_BF16_TC runs the dense
 *           contractions on the tensor cores with bfloat16 operands and float32
 *           accumulation (GMM only, for 32 < D <= 128; other D return
 *           GPA_ERR_UNSUPPORTED).
 */
#ifndef GPA_H
#define GPA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* gpa_stream_t; /* same type as cudaStream_t */

#if defined(__GNUC__)
#define GPA_API __attribute__((visibility("default")))
#else
#define GPA_API
#endif

typedef enum {
    GPA_OK = 0,
    GPA_ERR_ARG = 1,         /* null pointer, non-positive or too-large size */
    GPA_ERR_INDEX = 2,       /* (device) an index outside its index set */
    GPA_ERR_CUDA = 3,        /* a CUDA launch or runtime call failed */
    GPA_ERR_WORKSPACE = 4,   /* ws_bytes smaller than the query asked for */
    GPA_ERR_TIMEOUT = 5,     /* (device) a bounded wait gave up */
    GPA_ERR_UNSUPPORTED = 6, /* shape / precision / strategy not provided */
    GPA_ERR_ALIGN = 7        /* a pointer lacks the stated alignment */
} gpa_status;

typedef enum { GPA_PREC_FP32 = 0, GPA_PREC_BF16_TC = 1 } gpa_prec;

typedef enum {
    GPA_SCATTER_AUTO = 0,    /* SORT when a plan is given, else SMEM when the buckets fit, else ATOMIC */
    GPA_SCATTER_ATOMIC = 1,  /* one red.global.add per element */
    GPA_SCATTER_WARPAGG = 2, /* lanes of a warp with equal keys combine first */
    GPA_SCATTER_SORT = 3,    /* key-sorted order from a plan, segmented warp sums */
    GPA_SCATTER_SMEM = 4,    /* accum_scatter_add only: per-CTA copy of the buckets in shared
                                memory (n_buckets * w <= 24576), one global add per touched
                                entry; one bucket of width 1 is a complete reduction (trees) */
    GPA_SCATTER_RUNS = 5     /* accum_scatter_add only: equal indices adjacent in input order
                                (regular segmented, e.g. idx = j / L): segmented warp sums, no
                                plan; correct for any order */
} gpa_scatter;

/* Human-readable name of a gpa_status value (static string, never NULL). */
GPA_API const char* gpa_status_string(int status);

/* Library version as 10000*major + 100*minor + patch. */
GPA_API int gpa_version(void);

/* ========================================================================= */
/* Gaussian mixture with a Wishart prior                                     */
/* ========================================================================= */
/*
 * Parameters (K components in D dimensions, T = D(D-1)/2):
 *   alpha [K]      log-weights
 *   mu    [K][D]   means
 *   q     [K][D]   log-diagonal of the inverse-Cholesky factor Q_k
 *   l     [K][T]   strict-lower entries of Q_k, row-major packing:
 *                  Q_k[r][c] = l[k][r(r-1)/2 + c] for r > c, Q_k[r][r] = exp(q[k][r])
 *   x     [N][D]   points
 * Objective (log posterior, float64):
 *   f = sum_i logsumexp_k( alpha_k + sum_d q_kd - |Q_k (x_i - mu_k)|^2 / 2 )
 *       - N logsumexp(alpha) - (N D / 2) log(2 pi)
 *       + sum_k [ m sum_d q_kd - (gamma^2 / 2)(sum_d exp(2 q_kd) + sum_t l_kt^2) ]
 *       + K [ n D log(gamma) - (n D / 2) log 2 - log Gamma_D(n / 2) ],  n = D + m + 1,
 *   i.e. the mixture log-likelihood plus a Wishart(n, gamma^-2 I) log-prior on
 *   each precision matrix Q_k^T Q_k.
 * The log-joint s[k][i] = alpha_k + sum_d q_kd - |Q_k (x_i - mu_k)|^2 / 2 and
 * lse[i] = logsumexp_k s[k][i] are the per-point statistics the gradient needs.
 * Supported shapes: 1 <= D <= 128, 1 <= K <= 4096, 1 <= N <= 2^31 - 1.
 * Alignment: every pointer 4-byte aligned.
 */

/* Bytes of workspace needed by gmm_objective / gmm_vjp for this shape.
 * logjoint_points: how many points' log-joint columns (K floats each) the
 * workspace must hold for gmm_vjp when it recomputes the log-joint itself
 * (logjoint_in == NULL). 0 means "all N" (one pass); smaller values bound the
 * memory and make gmm_vjp run the forward pass in chunks of that many points
 * (rounded down to a multiple of 128, at least 128). gmm_objective needs no
 * log-joint space. */
GPA_API size_t gpa_gmm_workspace_bytes(int64_t n, int32_t d, int32_t k, int32_t prec,
                               int64_t logjoint_points);

/*
 * Forward pass: *out = f (device float64). Optionally writes lse_out [N]
 * (device float32, nullable) and logjoint_out [K][N] (device float32,
 * nullable; component-major so that each component's column is contiguous).
 * Sums over points are taken in float64 per 128-point tile and combined in a
 * fixed order (run-to-run deterministic).
 */
GPA_API int gmm_objective(const float* x, const float* alpha, const float* mu, const float* q,
                  const float* l, int64_t n, int32_t d, int32_t k, double gamma, int32_t m,
                  int32_t prec, double* out, float* lse_out, float* logjoint_out, void* ws,
                  size_t ws_bytes, int32_t* dev_status, gpa_stream_t stream);

/*
 * Reverse pass: seed * grad f, added (+=) into d_alpha [K], d_mu [K][D],
 * d_q [K][D], d_l [K][T] (grad f x = transpose (linearize f x) 1.0, Sec. 5.2;
 * seed = 1 gives the gradient). Optionally writes *out = f (nullable).
 * If logjoint_in [K][N] and lse_in [N] (both from gmm_objective on the same
 * inputs) are given, they are reused; if both are NULL the log-joint is
 * recomputed in the workspace, in chunks as large as the workspace allows.
 * Giving exactly one of them is GPA_ERR_ARG.
 * The reads of alpha_k, mu_k, Q_k inside the loop over points become
 * regular segmented reductions indexed by the component (Sec. 6.1.3),
 * accumulated per (component group, point chunk) and combined in a fixed order
 * (run-to-run deterministic).
 */
GPA_API int gmm_vjp(const float* x, const float* alpha, const float* mu, const float* q, const float* l,
            int64_t n, int32_t d, int32_t k, double gamma, int32_t m, int32_t prec,
            const float* logjoint_in, const float* lse_in, double seed, float* d_alpha,
            float* d_mu, float* d_q, float* d_l, double* out, void* ws, size_t ws_bytes,
            int32_t* dev_status, gpa_stream_t stream);

/*
 * Forward-mode directional derivative (linearize, Sec. 5.1):
 * *df_out = df(theta)[v] = d/de f(theta + e v) at e = 0 for the direction
 * v = (v_alpha [K], v_mu [K][D], v_q [K][D], v_l [K][T]) (device float32, the
 * parameters' layouts). The tangents ride along the forward pass point by
 * point: z_ik and its tangent Qd_k (x_i - mu_k) - Q_k v_mu_k, s_ik and its
 * tangent, and an online logsumexp over k with its tangent. Optional outputs:
 * *f_out = f (device float64, nullable) and lse_dot_out [N] (device float32,
 * nullable) = the tangent of logsumexp_k s_ik per point. FP32 arithmetic, sums
 * over points in float64 per 128-point tile in a fixed order.
 * <grad f, v> (gmm_vjp) equals df[v] (Sec. 5.2) up to rounding.
 */
GPA_API size_t gpa_gmm_jvp_workspace_bytes(int64_t n, int32_t d, int32_t k); /* 0 on bad arguments */
GPA_API int gmm_jvp(const float* x, const float* alpha, const float* mu, const float* q, const float* l,
                    int64_t n, int32_t d, int32_t k, double gamma, int32_t m, const float* v_alpha,
                    const float* v_mu, const float* v_q, const float* v_l, double* df_out, double* f_out,
                    float* lse_dot_out, void* ws, size_t ws_bytes, int32_t* dev_status,
                    gpa_stream_t stream);

/* ------------------------------------------------------------------------- */
/* Data-parallel GMM gradient: points sharded over ranks                      */
/* ------------------------------------------------------------------------- */
/*
 * The Accum sums of the reverse pass are associative (Sec. 2.3.2: partial sums
 * over any partition of the points combine by addition), so the gradient over
 * points split across ranks is: each rank runs gmm_vjp_partial on its shard,
 * the ranks add their exchange vectors (one all-reduce, sum), and each rank
 * runs gmm_vjp_finalize on the sum. Parameters are replicated; per-point
 * statistics never leave their rank.
 *
 * Exchange vector: float64, gpa_gmm_exchange_len(d, k) entries; per component
 * the sums [S (lower 8x8 blocks of the padded dimension) | m | R] of the
 * reverse pass (raw moments, S = sum r x x^T, m = sum r x, R = sum r, for both
 * precisions; every rank must use the same prec), then the sum over the
 * shard's points of logsumexp_k s_ik. Its layout is internal; only its length
 * and its additivity are part of the interface.
 */
GPA_API int64_t gpa_gmm_exchange_len(int32_t d, int32_t k); /* 0 on bad arguments */

/* Shard half: arguments as gmm_vjp for this rank's n points (logjoint_in /
 * lse_in of the shard, or both NULL); adds (+=) the shard's exchange vector
 * into exch (device, 8-byte aligned, zeroed by the caller), so that successive
 * calls over chunks of the points accumulate them. seed scales every term as
 * in gmm_vjp. Workspace: gpa_gmm_workspace_bytes(n, d, k, prec, .) of the
 * shard (or chunk). */
GPA_API int gmm_vjp_partial(const float* x, const float* alpha, const float* mu, const float* q,
                            const float* l, int64_t n, int32_t d, int32_t k, double gamma, int32_t m,
                            int32_t prec, const float* logjoint_in, const float* lse_in, double seed,
                            double* exch, void* ws, size_t ws_bytes, int32_t* dev_status,
                            gpa_stream_t stream);

/* Combine half: exch = the sum over all shards of their exchange vectors (same
 * seed and prec on every rank), n_total = the sum of the shards' n. Adds (+=)
 * seed * grad f of the whole data set to d_alpha, d_mu, d_q, d_l and writes
 * *out = f (nullable), exactly as one gmm_vjp over all points would (up to
 * the order of the float64 sums). Any workspace that serves gmm_vjp_partial
 * for the same d, k serves this call. */
GPA_API int gmm_vjp_finalize(const float* alpha, const float* mu, const float* q, const float* l,
                             int64_t n_total, int32_t d, int32_t k, double gamma, int32_t m, int32_t prec,
                             double seed, const double* exch, float* d_alpha, float* d_mu, float* d_q,
                             float* d_l, double* out, void* ws, size_t ws_bytes, int32_t* dev_status,
                             gpa_stream_t stream);

/* ------------------------------------------------------------------------- */
/* GMM from host memory                                                       */
/* ------------------------------------------------------------------------- */
/* Objective and seed * gradient of a mixture whose points and parameters are
 * in HOST memory, the results written to HOST memory: the end-to-end form of
 * gmm_vjp. x [n][d], alpha, mu, q, l as in gmm_vjp but host pointers, best
 * page-locked (cudaHostAlloc / cudaHostRegister) so that the copies run
 * asynchronously; pageable memory works with slower, blocking copies. The
 * parameters are copied in on `stream`; the points go to the device in chunks
 * of chunk_points (a multiple of 128; 0 = 2^19; the first chunk a quarter of
 * that) through two staging buffers in ws, each chunk's copy issued on a
 * library stream (one per device, made on first use) so that it overlaps the
 * reverse pass on the previous chunk (gmm_vjp_partial on `stream`); the
 * chunks' exchange vectors add up in ws and gmm_vjp_finalize finishes them.
 * d_alpha, d_mu, d_q, d_l (host, d_l ignored for d = 1) receive seed * grad f
 * (WRITTEN, not added) and *out (host, nullable) the objective, by copies on
 * `stream`: they hold the results once `stream` has completed the call's work
 * (synchronize it before reading them). Device memory: ws only, of
 * gpa_gmm_vjp_host_workspace_bytes(n, d, k, prec, chunk_points) bytes (two
 * chunks of points, the parameters, gradients, exchange vector and a chunk's
 * gmm_vjp workspace), 256-byte aligned. Calls on one device share the library
 * stream: concurrent calls from several host threads are ordered by it.
 * Errors as gmm_vjp. */
GPA_API size_t gpa_gmm_vjp_host_workspace_bytes(int64_t n, int32_t d, int32_t k, int32_t prec,
                                                int64_t chunk_points); /* 0 on bad arguments */
GPA_API int gmm_vjp_host(const float* x, const float* alpha, const float* mu, const float* q, const float* l,
                         int64_t n, int32_t d, int32_t k, double gamma, int32_t m, int32_t prec, double seed,
                         float* d_alpha, float* d_mu, float* d_q, float* d_l, double* out, int64_t chunk_points,
                         void* ws, size_t ws_bytes, int32_t* dev_status, gpa_stream_t stream);

/* ------------------------------------------------------------------------- */
/* Batched GMM: many instances of uneven N, D, K in persistent kernels        */
/* ------------------------------------------------------------------------- */
/* One mixture instance (all pointers device memory; layouts as for gmm_vjp). */
typedef struct {
    const float *x, *alpha, *mu, *q, *l;
    float *d_alpha, *d_mu, *d_q, *d_l; /* += seed * gradient */
    double* out;                       /* objective f, nullable */
    int64_t n;
    int32_t d, k;
    double gamma;
    int32_t m;
    double seed;
    int32_t prec; /* GPA_PREC_FP32, or GPA_PREC_BF16_TC for 32 < d <= 128 (the tensor-core
                     path; see gmm_batched_vjp) */
} gpa_gmm_instance;

/* Workspace for gmm_batched_prepare / gmm_batched_vjp over these instances
 * (host array). chunk_points: points per backward work item (>= 64; larger
 * values mean fewer partial sums, smaller values more parallelism). 0 on bad
 * arguments. */
GPA_API size_t gpa_gmm_batched_workspace_bytes(const gpa_gmm_instance* inst, int32_t n_inst,
                                               int64_t chunk_points);

/* Build the work lists (one item per (instance, component) for parameter
 * expansion and finalize, per (instance, 128-point tile) for the forward pass,
 * per (instance, component group, point chunk) for the backward Accum; forward
 * and backward lists in longest-first order) and copy them with the instance
 * descriptors into ws. Synchronises `stream` before returning. Call it once per
 * set of instances (pointers, shapes, seeds, precisions), before gmm_batched_vjp.
 * With tensor-core instances it also makes, once per device, the library's own
 * streams and events over which gmm_batched_vjp spreads them. */
GPA_API int gmm_batched_prepare(const gpa_gmm_instance* inst, int32_t n_inst, int64_t chunk_points,
                                void* ws, size_t ws_bytes, gpa_stream_t stream);

/* Objective and seed * gradient of every prepared instance: per padded
 * dimension class (D <= 8, 16, 32, 64, 128) up to five persistent kernels
 * (prep, forward, backward in default and small component groups, finalize)
 * whose CTAs pull work items from an atomic counter (flattened loops, Sec.
 * 6.1.1), plus two memsets. Enqueues device work only, so the call can be captured in a
 * CUDA graph and replayed while the inputs live at the same addresses.
 * ctas_per_sm caps resident CTAs per SM (0 = as many as fit). `inst`,
 * n_inst, chunk_points must equal the gmm_batched_prepare arguments. FP32
 * CUDA-core arithmetic, deterministic like gmm_vjp. Instances with prec =
 * GPA_PREC_BF16_TC run the contractions of the tensor-core path of gmm_vjp
 * instead (their prep and finalize run in the class's persistent kernels):
 * those of one padded dimension (64 or 128) as one concatenated class, each
 * stage one launch over all their tiles, when their BF16 responsibilities
 * (rows: the largest K rounded up to 16; columns: the sum of their n rounded
 * up to 128) fit 8 GiB; otherwise instance by instance, spread over 8 library
 * streams forked from `stream` with events and joined back into it
 * (capturable in the same graph), each in a workspace region of its own
 * (gmm_vjp's tensor-core workspace for its n, d, k). */
GPA_API int gmm_batched_vjp(const gpa_gmm_instance* inst, int32_t n_inst, int64_t chunk_points,
                            int32_t ctas_per_sm, void* ws, size_t ws_bytes, int32_t* dev_status,
                            gpa_stream_t stream);

/* Per-class settings of the batched form. The classes are the padded
 * dimensions 8 (D <= 8), 16, 32, 64 and 128, index 0..4. For each class:
 *   chunk_points  points per backward work item (>= 64);
 *   ctas_per_sm   resident persistent CTAs per SM of its forward and backward
 *                 kernels (0 = as many as fit);
 *   small_groups  1: an FP32 instance whose component count K fills the
 *                 class's small component group (10 components at D <= 16, 6 at
 *                 D <= 32) with fewer idle threads than the default group (42,
 *                 25) takes its backward work items in that group size; 0: the
 *                 default groups only. Ignored for the other classes.
 * gmm_batched_prepare / gmm_batched_vjp / gpa_gmm_batched_workspace_bytes
 * are the _opts calls with every class set to (chunk_points, ctas_per_sm, 0).
 * The results do not depend on the settings beyond the order of the float32
 * sums of the backward (which the settings fix, so every run with the same
 * settings gives the same bits). */
#define GPA_BATCH_CLASSES 5
typedef struct {
    int64_t chunk_points[GPA_BATCH_CLASSES];
    int32_t ctas_per_sm[GPA_BATCH_CLASSES];
    int32_t small_groups[GPA_BATCH_CLASSES];
} gpa_batched_opts;

/* As gpa_gmm_batched_workspace_bytes, gmm_batched_prepare, gmm_batched_vjp
 * with per-class settings (host struct, read during the call; the same
 * settings for all three). GPA_ERR_ARG (0 bytes) for a null opts, a
 * chunk_points below 64 or a negative ctas_per_sm. */
GPA_API size_t gpa_gmm_batched_workspace_bytes_opts(const gpa_gmm_instance* inst, int32_t n_inst,
                                                    const gpa_batched_opts* opts);
GPA_API int gmm_batched_prepare_opts(const gpa_gmm_instance* inst, int32_t n_inst, const gpa_batched_opts* opts,
                                     void* ws, size_t ws_bytes, gpa_stream_t stream);
GPA_API int gmm_batched_vjp_opts(const gpa_gmm_instance* inst, int32_t n_inst, const gpa_batched_opts* opts,
                                 void* ws, size_t ws_bytes, int32_t* dev_status, gpa_stream_t stream);

/* ========================================================================= */
/* Camera reprojection (bundle adjustment residual)                          */
/* ========================================================================= */
/*
 * cams [C][11]  camera j = [w(3) Rodrigues rotation, c(3) centre, f focal,
 *                pp(2) principal point, kappa(2) radial distortion]
 * pts  [P][3]   3-D points
 * obs  [M][2]   int32 (camera index, point index) per observation
 * tgt  [M][2]   observed 2-D positions
 * Per observation: u = X - c, Y = R(w) u, p = (Y_0, Y_1) / Y_2, rho = |p|^2,
 * L = 1 + kappa_0 rho + kappa_1 rho^2, res = f L p + pp - tgt.
 * R(w) = exp([w]x) (rotation by |w| about w/|w|); the rotation of each camera
 * is expanded once per call in float64 and its last row carried as a float32
 * hi/lo pair so that Y_2 keeps its relative accuracy for points close to the
 * image plane.
 * Supported: 1 <= C, P <= 2^31 - 1, 1 <= M <= 2^31 - 1. Alignment: obs 8-byte,
 * tgt / res / w 8-byte, others 4-byte.
 */

/* Workspace for reproj_residual / reproj_vjp / reproj_residual_vjp / reproj_jvp:
 * the expanded cameras, and for the VJPs the points copied into 16-byte rows
 * and the padded point accumulators. */
GPA_API size_t gpa_reproj_workspace_bytes(int32_t n_cams, int32_t n_pts, int64_t n_obs);

/* res [M][2] = projection - target. Observations whose indices fall outside
 * their index sets get NaN residuals and set GPA_ERR_INDEX. */
GPA_API int reproj_residual(const float* cams, const float* pts, const int32_t* obs, const float* tgt,
                    int32_t n_cams, int32_t n_pts, int64_t n_obs, float* res, void* ws,
                    size_t ws_bytes, int32_t* dev_status, gpa_stream_t stream);

/* Order of the per-observation arrays (w, tgt, res) of the SORT strategy:
 * GPA_OBS_INPUT: row j belongs to observation j (obs[j]);
 * GPA_OBS_PLAN:  row i belongs to the observation at position i of the plan's
 *                camera-sorted order (plan perm[i]). The kernels then read and
 *                write these arrays contiguously instead of through the
 *                permutation, e.g. for a least-squares loop that keeps its
 *                targets permuted once and its residuals in plan order. */
typedef enum { GPA_OBS_INPUT = 0, GPA_OBS_PLAN = 1 } gpa_obs_order;

/* reproj_residual computed in the camera-sorted order of a plan built from obs
 * by gpa_obs_plan_build (each camera's record is read once per run of its
 * observations instead of once per observation); with obs_order
 * GPA_OBS_INPUT, res is written in input order and every entry equals
 * reproj_residual's bit for bit; with GPA_OBS_PLAN, tgt and res are in plan
 * order. obs is checked (non-null, 8-byte aligned) but not read: the plan
 * carries the indices. Invalid indices: NaN rows and GPA_ERR_INDEX, as above. */
GPA_API int reproj_residual_sorted(const float* cams, const float* pts, const int32_t* obs, const float* tgt,
                    int32_t n_cams, int32_t n_pts, int64_t n_obs, float* res, const void* plan, int32_t obs_order,
                    void* ws, size_t ws_bytes, int32_t* dev_status, gpa_stream_t stream);

/*
 * VJP of the residual with cotangent w [M][2]: d_cams[c] += J_cam^T w_j and
 * d_pts[p] += J_pt^T w_j over all observations j with obs[j] = (c, p): the
 * transpose of the gathers cams.(obs.j.0), pts.(obs.j.1) is an irregular
 * segmented reduction (histogram pattern, Sec. 6.1.3; LetIndexingTranspose,
 * Fig. "transpose"). strat selects how the Accum is carried out; SORT needs
 * `plan` from gpa_obs_plan_build on the same obs (nullable otherwise).
 * obs_order (gpa_obs_order): the order of w; GPA_OBS_PLAN needs SORT.
 * Atomic strategies give float32 sums whose rounding depends on the order.
 */
GPA_API int reproj_vjp(const float* cams, const float* pts, const int32_t* obs, const float* w,
               int32_t n_cams, int32_t n_pts, int64_t n_obs, float* d_cams, float* d_pts,
               int32_t strat, const void* plan, int32_t obs_order, void* ws, size_t ws_bytes,
               int32_t* dev_status, gpa_stream_t stream);

/*
 * Gauss-Newton normal equations of the residual, the blocks of J^T J and J^T r
 * for J = d res / d(cams, pts) (each observation's 2 x 14 Jacobian rows, from the
 * reverse pass with unit cotangents):
 *   U [C][66]  += sum over the camera's observations of J_c^T J_c (11 x 11,
 *                 upper triangle packed by rows: (a, b), a <= b)
 *   V [P][6]   += sum over the point's observations of J_p^T J_p (3 x 3, same packing)
 *   W [M][w_ld] = J_c^T J_p of each observation in columns 0..32 (11 x 3
 *                 row-major; nullable); columns 33..w_ld-1 are set to 0.
 *                 33 <= w_ld <= 64. w_order 0: row j holds observation j;
 *                 w_order 1 (SORT only): row i holds the observation at
 *                 position i of the plan's camera-sorted order (plan perm[i]),
 *                 so that rows are written in order. With w_ld a multiple of 8
 *                 and W 32-byte aligned every row is written as whole 32-byte
 *                 sectors, which matters under SORT with w_order 0, where rows
 *                 land in camera order: a partly written sector costs a
 *                 read-modify-write in DRAM.
 *   g_cams [C][11] += J_c^T r,  g_pts [P][3] += J_p^T r,  res [M][2] = r (nullable)
 * The camera and point blocks are Accum reductions like the VJP's, with a
 * 66 + 11 and a 6 + 3 float payload. strat: SORT (camera-sorted runs from
 * `plan`, gpa_obs_plan_build on the same obs) or ATOMIC (input order); AUTO
 * picks SORT when a plan is given. Out-of-range observations get NaN in W and
 * res and set GPA_ERR_INDEX. Workspace: gpa_reproj_gn_workspace_bytes. Sums in
 * float32, order-dependent. The paper has no counterpart of this call; it is
 * the consumer of the VJP that a least-squares solver needs.
 */
GPA_API size_t gpa_reproj_gn_workspace_bytes(int32_t n_cams, int32_t n_pts, int64_t n_obs);
GPA_API int reproj_normal_eqs(const float* cams, const float* pts, const int32_t* obs, const float* tgt,
                              int32_t n_cams, int32_t n_pts, int64_t n_obs, float* U, float* V, float* W,
                              int32_t w_ld, int32_t w_order, float* g_cams, float* g_pts, float* res, int32_t strat,
                              const void* plan, void* ws, size_t ws_bytes, int32_t* dev_status,
                              gpa_stream_t stream);

/* JVP of the residual (forward mode, linearize, Sec. 5.1): jv [M][2] =
 * J_cam(j) v_cams[c] + J_pt(j) v_pts[p] for each observation j = (c, p), with
 * tangents v_cams [C][11] and v_pts [P][3] laid out like cams and pts.
 * Out-of-range observations get NaN and set GPA_ERR_INDEX. Workspace as for
 * reproj_residual. */
GPA_API int reproj_jvp(const float* cams, const float* pts, const int32_t* obs, const float* v_cams,
                       const float* v_pts, int32_t n_cams, int32_t n_pts, int64_t n_obs, float* jv, void* ws,
                       size_t ws_bytes, int32_t* dev_status, gpa_stream_t stream);

/* Fused residual + VJP in one pass over the observations: res as
 * reproj_residual, then d_cams / d_pts += J^T (wscale * res) (the Gauss-Newton
 * gradient of wscale * |res|^2 / 2 when wscale = 1). obs_order: the order of
 * tgt and res (GPA_OBS_PLAN needs SORT). */
GPA_API int reproj_residual_vjp(const float* cams, const float* pts, const int32_t* obs,
                        const float* tgt, int32_t n_cams, int32_t n_pts, int64_t n_obs,
                        float wscale, float* res, float* d_cams, float* d_pts, int32_t strat,
                        const void* plan, int32_t obs_order, void* ws, size_t ws_bytes, int32_t* dev_status,
                        gpa_stream_t stream);

/*
 * Same result as reproj_vjp, for callers that cannot give the library a
 * workspace: code whose device memory is owned by another allocator (a host
 * framework's caching pool, a plugin or extension host) that forbids or cannot
 * afford a cudaMalloc on its call path, or code whose device-memory budget is
 * fixed at start-up. The paper has no counterpart; it is an interface choice.
 * The only scratch, the expanded cameras, lives in a fixed array in device
 * memory owned by the library (GPA_NOALLOC_MAX_CAMS cameras, 2 MiB on every
 * GPU that loads the library, held until the process exits); the call itself
 * allocates nothing. More cameras than that return GPA_ERR_WORKSPACE and
 * enqueue nothing. Each call looks up the array's address in the calling
 * thread's current device context (a host-side lookup), so the array is found
 * again after cudaDeviceReset or in another context; the first call in a
 * context loads the library's device code there, so make that first call
 * before any stream capture. Every call shares the array and it keeps the last
 * call's contents (each call rewrites the records it reads before reading
 * them): calls that overlap on the GPU, on any streams, race. The points are
 * gathered in place and d_pts is updated with one atomic per coordinate (no
 * padded rows). Arguments, strategies and Accum (+=) semantics are those of
 * reproj_vjp.
 */
#define GPA_NOALLOC_MAX_CAMS 16384
GPA_API int reproj_vjp_noalloc(const float* cams, const float* pts, const int32_t* obs, const float* w,
                               int32_t n_cams, int32_t n_pts, int64_t n_obs, float* d_cams, float* d_pts,
                               int32_t strat, const void* plan, int32_t* dev_status, gpa_stream_t stream);

/* ========================================================================= */
/* Index preparation and the generic Accum scatter                           */
/* ========================================================================= */
/*
 * An index plan: the stable sort of element ids by a data-derived key
 * (keys from `obs` column 0, i.e. the camera, for the reprojection; the
 * scatter indices for accum_scatter_add). Index validity is checked here, where
 * indices are made from data (Sec. 6.3): elements whose key is outside
 * [0, n_keys) (or, for observations, whose point is outside [0, n_pts)) set
 * GPA_ERR_INDEX and are placed after all valid elements.
 * Plan layout (in `plan`, 256-byte aligned, size from the query):
 *   int64 header[4] = {n_elems, n_keys, n_valid (written on device), reserved}
 *   int32 perm[n_elems]         element ids in key order (stable)
 *   int32 key_sorted[n_elems]   keys in that order (n_keys for invalid ones)
 *   int32 aux_sorted[n_elems]   second index in that order (point ids; 0 for scatter)
 *   int32 seg_off[n_keys + 1]   start of each key's run; seg_off[n_keys] = n_valid
 * The integer contents are bit-exact with a stable counting sort.
 */
GPA_API size_t gpa_plan_bytes(int64_t n_elems, int32_t n_keys);
GPA_API size_t gpa_plan_workspace_bytes(int64_t n_elems, int32_t n_keys);

/* Plan over observations keyed by camera (obs [M][2]); checks both indices. */
GPA_API int gpa_obs_plan_build(const int32_t* obs, int64_t n_obs, int32_t n_cams, int32_t n_pts,
                       void* plan, size_t plan_bytes, void* ws, size_t ws_bytes,
                       int32_t* dev_status, gpa_stream_t stream);

/* Plan over plain indices idx [M] with n_keys buckets. */
GPA_API int gpa_index_plan_build(const int32_t* idx, int64_t m, int32_t n_keys, void* plan,
                         size_t plan_bytes, void* ws, size_t ws_bytes, int32_t* dev_status,
                         gpa_stream_t stream);

/*
 * acc[idx[j]][c] += vals[j][c] for j < m, c < w (hist!(x.i) += v, Sec. 2.3.3,
 * Sec. 6.1.2). dtype 0 = float32 values and accumulator, 1 = int32 (exact,
 * wrapping on overflow). Indices outside [0, n_buckets) set GPA_ERR_INDEX and
 * are skipped. SORT needs `plan` from gpa_index_plan_build on the same idx.
 * The strategies follow the reduction patterns of Sec. 6.1.3: complete (one
 * bucket: SMEM's tree), regular segmented (RUNS), irregular (ATOMIC, WARPAGG,
 * SORT; SMEM when the buckets are few). SMEM with more than 24576 entries is
 * GPA_ERR_UNSUPPORTED. 1 <= w <= 64. Alignment: 4-byte.
 */
GPA_API int accum_scatter_add(const int32_t* idx, const void* vals, int64_t m, int32_t w, int32_t dtype,
                      void* acc, int32_t n_buckets, int32_t strat, const void* plan,
                      int32_t* dev_status, gpa_stream_t stream);

/* ========================================================================= */
/* Diagnostics                                                               */
/* ========================================================================= */
/*
 * Check that this device's bounded waits give up as the error convention
 * above states: launches one CTA whose 64 threads wait, with the library's
 * per-thread wait and with its warp-uniform wait, on a shared-memory mbarrier
 * that expects one arrival that never comes. Each wait gives up after limit_ns
 * nanoseconds of the device's global timer (1 <= limit_ns <= 1e9; the
 * library's own waits use 1e9), ORs GPA_ERR_TIMEOUT into *dev_status and adds 1
 * to *gave_up (device int32, zeroed by the caller; 64 after the launch
 * completes). No copy engine, tensor memory or other kernel is involved, and
 * the device stays usable afterwards. The paper has no counterpart; it makes
 * the library's failure path testable without a fault.
 */
GPA_API int gpa_check_bounded_wait(int64_t limit_ns, int32_t* dev_status, int32_t* gave_up,
                                   gpa_stream_t stream);

/* ========================================================================= */
/* Tracing                                                                   */
/* ========================================================================= */
/* Enable (1) or disable (0) per-launch timing: while enabled, every kernel the
 * library launches is bracketed by two CUDA events on its stream (events are
 * created once and reused; no device memory is allocated). Process-wide. */
GPA_API void gpa_trace_enable(int on);

/* Resolve the recorded launches (waits for the last one) and return the length
 * of the text "name launches total_ms\n" (one line per kernel name). If buf
 * (host memory) holds more than that many bytes, the text is copied into it
 * NUL-terminated and the records are forgotten; otherwise (buf NULL or too
 * short) nothing is copied and the records are kept. */
GPA_API int gpa_trace_summary(char* buf, size_t len);

#ifdef __cplusplus
}
#endif
#endif /* GPA_H */
