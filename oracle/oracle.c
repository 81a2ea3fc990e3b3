/*
 * FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously-correct definitions of what the hot path computes.
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may load
 * this file; the product (the CUDA library) never links or calls it, and the two
 * share no code. Inputs are the same float32 / int32 arrays the GPU path sees,
 * widened to double on read.
 *
 * Passages followed (arXiv 2104.05372, "Getting to the Point"):
 *  - Accum (Sec. 2.3.2): write-only additive updates, associative, so a loop of
 *    updates may be split into partial sums that are combined afterwards. The
 *    OpenMP loops below do exactly that: thread-private accumulators over a
 *    partition of the points / observations, combined once at the end.
 *  - Reference indexing and histogram (Sec. 2.3.3, Sec. 6.1.2): acc!(idx) += v.
 *  - linearize (Sec. 5.1): forward mode, primal plus tangent.
 *  - transpose and grad (Sec. 5.2, Fig. "transpose"): grad f x = transpose
 *    (linearize f x) 1.0; the transpose of an indexed read y.v is an
 *    accumulation into r!v (rule LetIndexingTranspose).
 *
 * The two programs themselves are not in the paper; they are stated as
 * mathematics by the benchmark workload, and this file writes that mathematics
 * out:
 *   GMM:  Q_k lower triangular, Q_k[r][r] = exp(q_kr), Q_k[r][c] = l_k[r(r-1)/2+c]
 *         (r > c); precision = Q_k^T Q_k.
 *         f = sum_i logsumexp_k(alpha_k + sum_d q_kd - 0.5 |Q_k (x_i - mu_k)|^2)
 *             - N logsumexp(alpha) - (N D / 2) log(2 pi)
 *             + sum_k [ m sum_d q_kd - (gamma^2/2)(sum_d exp(2 q_kd) + sum_t l_kt^2) ]
 *             + K c_W,
 *         c_W = n D log(gamma) - (n D / 2) log 2 - log Gamma_D(n/2), n = D + m + 1
 *         (the log-density of a Wishart(n, gamma^-2 I) prior on each precision).
 *   Reprojection: camera [w(3), c(3), f, pp(2), kappa(2)], point X:
 *         u = X - c; Y = R(w) u (Rodrigues); p = Y_xy / Y_z; rho = |p|^2;
 *         L = 1 + k1 rho + k2 rho^2; res = f L p + pp - t.
 *
 * Parity status of each function is stated beside it; every function here is
 * pinned by a CPU test against something other than itself.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* GMM                                                                       */
/* ------------------------------------------------------------------------- */

/* Dense lower-triangular Q_k (d x d, row-major) from (q, l). */
static void gmm_expand_q(const float* q, const float* l, int d, int k, double* Q) {
    const int t = d * (d - 1) / 2;
    for (int kk = 0; kk < k; ++kk) {
        double* Qk = Q + (size_t)kk * d * d;
        for (int r = 0; r < d; ++r)
            for (int c = 0; c < d; ++c) {
                double v = 0.0;
                if (c == r) v = exp((double)q[kk * d + r]);
                else if (c < r) v = (double)l[(size_t)kk * t + r * (r - 1) / 2 + c];
                Qk[r * d + c] = v;
            }
    }
}

static double logsumexp(const double* v, int n) {
    double mx = v[0];
    for (int i = 1; i < n; ++i) if (v[i] > mx) mx = v[i];
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += exp(v[i] - mx);
    return mx + log(s);
}

/* log of the multivariate gamma function Gamma_D(a). */
static double log_mvgamma(int dd, double a) {
    double s = 0.25 * dd * (dd - 1) * log(M_PI);
    for (int j = 1; j <= dd; ++j) s += lgamma(a + 0.5 * (1 - j));
    return s;
}

/* Wishart prior part of the objective: sum over components plus K constants. */
static double gmm_log_prior(const float* q, const float* l, int d, int k, double gamma, int m) {
    const int t = d * (d - 1) / 2;
    const double n = (double)(d + m + 1);
    const double cw = n * d * log(gamma) - 0.5 * n * d * log(2.0) - log_mvgamma(d, 0.5 * n);
    double lp = 0.0;
    for (int kk = 0; kk < k; ++kk) {
        double sq = 0.0, fro = 0.0;
        for (int r = 0; r < d; ++r) {
            double qv = q[kk * d + r];
            sq += qv;
            fro += exp(2.0 * qv);
        }
        for (int j = 0; j < t; ++j) {
            double lv = l[(size_t)kk * t + j];
            fro += lv * lv;
        }
        lp += m * sq - 0.5 * gamma * gamma * fro + cw;
    }
    return lp;
}

/* s[kk] = alpha_k + sum_d q_kd - 0.5 |Q_k (x_i - mu_k)|^2 for every component;
 * also returns xc (k x d) and z (k x d) when the buffers are given. */
static void gmm_point(const float* xi, const float* alpha, const float* mu, const float* q,
                      const double* Q, int d, int k, double* s, double* xc_all, double* z_all,
                      double* tmp) {
    for (int kk = 0; kk < k; ++kk) {
        double* xc = xc_all ? xc_all + (size_t)kk * d : tmp;
        double* z = z_all ? z_all + (size_t)kk * d : tmp + d;
        for (int c = 0; c < d; ++c) xc[c] = (double)xi[c] - (double)mu[kk * d + c];
        const double* Qk = Q + (size_t)kk * d * d;
        double nz = 0.0;
        for (int r = 0; r < d; ++r) {
            double acc = 0.0;
            for (int c = 0; c <= r; ++c) acc += Qk[r * d + c] * xc[c];
            z[r] = acc;
            nz += acc * acc;
        }
        double ld = 0.0;
        for (int r = 0; r < d; ++r) ld += q[kk * d + r];
        s[kk] = (double)alpha[kk] + ld - 0.5 * nz;
    }
}

static double alpha_lse(const float* alpha, int k) {
    double* a = (double*)malloc(sizeof(double) * k);
    for (int i = 0; i < k; ++i) a[i] = alpha[i];
    double r = logsumexp(a, k);
    free(a);
    return r;
}

/* Objective f (parity pinned: scipy Gaussian + Wishart log-densities, tests). */
double oracle_gmm_objective(const float* x, const float* alpha, const float* mu, const float* q,
                            const float* l, int64_t n, int d, int k, double gamma, int m,
                            double* lse_out) {
    double* Q = (double*)malloc(sizeof(double) * (size_t)k * d * d);
    gmm_expand_q(q, l, d, k, Q);
    double ll = 0.0;
#pragma omp parallel reduction(+ : ll)
    {
        double* s = (double*)malloc(sizeof(double) * k);
        double* tmp = (double*)malloc(sizeof(double) * 2 * d);
#pragma omp for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            gmm_point(x + (size_t)i * d, alpha, mu, q, Q, d, k, s, NULL, NULL, tmp);
            double lse = logsumexp(s, k);
            if (lse_out) lse_out[i] = lse;
            ll += lse;
        }
        free(s);
        free(tmp);
    }
    free(Q);
    ll -= (double)n * alpha_lse(alpha, k) + 0.5 * (double)n * d * log(2.0 * M_PI);
    return ll + gmm_log_prior(q, l, d, k, gamma, m);
}

/* Per-point log-joint s_ik and logsumexp for a list of point indices. */
void oracle_gmm_logjoint_at(const float* x, const float* alpha, const float* mu, const float* q,
                            const float* l, int d, int k, const int64_t* idx, int64_t n_idx,
                            double* s_out /* n_idx x k, nullable */, double* lse_out /* n_idx */) {
    double* Q = (double*)malloc(sizeof(double) * (size_t)k * d * d);
    gmm_expand_q(q, l, d, k, Q);
#pragma omp parallel
    {
        double* s = (double*)malloc(sizeof(double) * k);
        double* tmp = (double*)malloc(sizeof(double) * 2 * d);
#pragma omp for schedule(static)
        for (int64_t j = 0; j < n_idx; ++j) {
            gmm_point(x + (size_t)idx[j] * d, alpha, mu, q, Q, d, k, s, NULL, NULL, tmp);
            if (s_out) memcpy(s_out + (size_t)j * k, s, sizeof(double) * k);
            lse_out[j] = logsumexp(s, k);
        }
        free(s);
        free(tmp);
    }
    free(Q);
}

/*
 * seed * gradient of f (parity pinned: central finite differences of the
 * objective, tests). Reverse mode as linearize-then-transpose (Sec. 5.2): per
 * point the cotangent of s_ik is r_ik = seed * softmax_k(s_i.)_k; reads of
 * alpha_k, mu_k and Q_k inside the loop over points turn into accumulations
 * into their cotangent slots (LetIndexingTranspose), kept thread-private and
 * combined at the end (Accum, Sec. 2.3.2).
 */
/*
 * The Accum half of the gradient over the n points given: the cotangent
 * accumulations A_k = sum_i r_ik, MU_k = -sum_i Q_k^T zbar_ik and
 * QB_k = sum_i zbar_ik (x_i - mu_k)^T (lower triangle, zbar = -r z), with
 * r_ik = seed * softmax_k(s_i.)_k. Returns sum_i logsumexp_k s_ik. These sums
 * are additive over any partition of the points (Sec. 2.3.2), which is what
 * the data-parallel form relies on.
 */
double oracle_gmm_accum(const float* x, const float* alpha, const float* mu, const float* q,
                        const float* l, int64_t n, int d, int k, double seed,
                        double* A, double* MU, double* QB) {
    double* Q = (double*)malloc(sizeof(double) * (size_t)k * d * d);
    gmm_expand_q(q, l, d, k, Q);
    memset(A, 0, sizeof(double) * (size_t)k);
    memset(MU, 0, sizeof(double) * (size_t)k * d);
    memset(QB, 0, sizeof(double) * (size_t)k * d * d);
    double ll = 0.0;
#pragma omp parallel reduction(+ : ll)
    {
        double* a_p = (double*)calloc((size_t)k, sizeof(double));
        double* mu_p = (double*)calloc((size_t)k * d, sizeof(double));
        double* qb_p = (double*)calloc((size_t)k * d * d, sizeof(double));
        double* s = (double*)malloc(sizeof(double) * k);
        double* xc = (double*)malloc(sizeof(double) * (size_t)k * d);
        double* z = (double*)malloc(sizeof(double) * (size_t)k * d);
        double* zbar = (double*)malloc(sizeof(double) * d);
#pragma omp for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            gmm_point(x + (size_t)i * d, alpha, mu, q, Q, d, k, s, xc, z, NULL);
            const double lse = logsumexp(s, k);
            ll += lse;
            for (int kk = 0; kk < k; ++kk) {
                const double r = seed * exp(s[kk] - lse);   /* cotangent of s_ik */
                a_p[kk] += r;                                /* s = alpha_k + ...  */
                const double* xck = xc + (size_t)kk * d;
                const double* zk = z + (size_t)kk * d;
                for (int rr = 0; rr < d; ++rr) zbar[rr] = -r * zk[rr]; /* s = ... - |z|^2/2 */
                double* qb = qb_p + (size_t)kk * d * d;
                const double* Qk = Q + (size_t)kk * d * d;
                for (int rr = 0; rr < d; ++rr)               /* z = Q xc: Qbar += zbar xc^T */
                    for (int c = 0; c <= rr; ++c) qb[rr * d + c] += zbar[rr] * xck[c];
                for (int c = 0; c < d; ++c) {                /* xcbar = Q^T zbar; xc = x - mu */
                    double xb = 0.0;
                    for (int rr = c; rr < d; ++rr) xb += Qk[rr * d + c] * zbar[rr];
                    mu_p[(size_t)kk * d + c] -= xb;
                }
            }
        }
#pragma omp critical
        {
            for (int kk = 0; kk < k; ++kk) A[kk] += a_p[kk];
            for (size_t j = 0; j < (size_t)k * d; ++j) MU[j] += mu_p[j];
            for (size_t j = 0; j < (size_t)k * d * d; ++j) QB[j] += qb_p[j];
        }
        free(a_p); free(mu_p); free(qb_p); free(s); free(xc); free(z); free(zbar);
    }
    free(Q);
    return ll;
}

/*
 * The rest of the gradient from Accum sums taken over all n_total points: the
 * cotangents of the terms outside the loop over points (-N logsumexp(alpha)
 * and the prior) and the chain through Q_k = (exp(q_k) on the diagonal, l_k
 * below it). Returns f, given sum_lse = sum_i logsumexp_k s_ik.
 */
double oracle_gmm_finish(const float* alpha, const float* q, const float* l, int64_t n_total, int d, int k,
                         double gamma, int m, double seed, const double* A, const double* MU,
                         const double* QB, double sum_lse, double* d_alpha, double* d_mu, double* d_q,
                         double* d_l) {
    const int t = d * (d - 1) / 2;
    /* -N logsumexp(alpha): cotangent -seed N softmax(alpha). */
    const double la = alpha_lse(alpha, k);
    for (int kk = 0; kk < k; ++kk) d_alpha[kk] = A[kk] - seed * (double)n_total * exp((double)alpha[kk] - la);
    for (int kk = 0; kk < k; ++kk) {
        for (int r = 0; r < d; ++r) {
            const double qv = q[kk * d + r];
            const double e = exp(qv);
            /* sum_d q_kd in s (weight A_k), Q[r][r] = exp(q), prior m q - gamma^2 exp(2q)/2 */
            d_q[kk * d + r] = A[kk] + QB[(size_t)kk * d * d + r * d + r] * e +
                              seed * ((double)m - gamma * gamma * e * e);
            d_mu[kk * d + r] = MU[(size_t)kk * d + r];
        }
        for (int r = 1; r < d; ++r)
            for (int c = 0; c < r; ++c) {
                const size_t j = (size_t)kk * t + r * (r - 1) / 2 + c;
                d_l[j] = QB[(size_t)kk * d * d + r * d + c] - seed * gamma * gamma * (double)l[j];
            }
    }
    const double ll = sum_lse - ((double)n_total * la + 0.5 * (double)n_total * d * log(2.0 * M_PI));
    return ll + gmm_log_prior(q, l, d, k, gamma, m);
}

double oracle_gmm_grad(const float* x, const float* alpha, const float* mu, const float* q,
                       const float* l, int64_t n, int d, int k, double gamma, int m, double seed,
                       double* d_alpha, double* d_mu, double* d_q, double* d_l) {
    double* A = (double*)malloc(sizeof(double) * (size_t)k);
    double* MU = (double*)malloc(sizeof(double) * (size_t)k * d);
    double* QB = (double*)malloc(sizeof(double) * (size_t)k * d * d);
    const double sum_lse = oracle_gmm_accum(x, alpha, mu, q, l, n, d, k, seed, A, MU, QB);
    const double f = oracle_gmm_finish(alpha, q, l, n, d, k, gamma, m, seed, A, MU, QB, sum_lse, d_alpha, d_mu,
                                       d_q, d_l);
    free(A); free(MU); free(QB);
    return f;
}

/*
 * Directional derivative df(theta)[v] by forward mode (linearize, Sec. 5.1)
 * (parity pinned: central finite differences along v, tests). Returns df; the
 * objective goes to *f_out and the per-point tangent of logsumexp_k s_ik to
 * lse_dot_out when given.
 */
double oracle_gmm_jvp(const float* x, const float* alpha, const float* mu, const float* q,
                      const float* l, int64_t n, int d, int k, double gamma, int m,
                      const double* v_alpha, const double* v_mu, const double* v_q,
                      const double* v_l, double* f_out, double* lse_dot_out /* n, nullable */) {
    const int t = d * (d - 1) / 2;
    double* Q = (double*)malloc(sizeof(double) * (size_t)k * d * d);
    double* QD = (double*)calloc((size_t)k * d * d, sizeof(double)); /* tangent of Q */
    gmm_expand_q(q, l, d, k, Q);
    for (int kk = 0; kk < k; ++kk)
        for (int r = 0; r < d; ++r) {
            QD[(size_t)kk * d * d + r * d + r] = exp((double)q[kk * d + r]) * v_q[kk * d + r];
            for (int c = 0; c < r; ++c)
                QD[(size_t)kk * d * d + r * d + c] = v_l[(size_t)kk * t + r * (r - 1) / 2 + c];
        }
    double tot = 0.0, ll = 0.0;
#pragma omp parallel reduction(+ : tot, ll)
    {
        double* s = (double*)malloc(sizeof(double) * k);
        double* sd = (double*)malloc(sizeof(double) * k);
        double* xc = (double*)malloc(sizeof(double) * d);
#pragma omp for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            const float* xi = x + (size_t)i * d;
            for (int kk = 0; kk < k; ++kk) {
                for (int c = 0; c < d; ++c) xc[c] = (double)xi[c] - (double)mu[kk * d + c];
                const double* Qk = Q + (size_t)kk * d * d;
                const double* QDk = QD + (size_t)kk * d * d;
                double nz = 0.0, zzd = 0.0, ld = 0.0, ldd = 0.0;
                for (int r = 0; r < d; ++r) {
                    double z = 0.0, zd = 0.0;
                    for (int c = 0; c <= r; ++c) {
                        z += Qk[r * d + c] * xc[c];
                        zd += QDk[r * d + c] * xc[c] - Qk[r * d + c] * v_mu[kk * d + c];
                    }
                    nz += z * z;
                    zzd += z * zd;
                    ld += q[kk * d + r];
                    ldd += v_q[kk * d + r];
                }
                s[kk] = (double)alpha[kk] + ld - 0.5 * nz;
                sd[kk] = v_alpha[kk] + ldd - zzd;
            }
            const double lse = logsumexp(s, k);
            ll += lse;
            double dd = 0.0;
            for (int kk = 0; kk < k; ++kk) dd += exp(s[kk] - lse) * sd[kk];
            if (lse_dot_out) lse_dot_out[i] = dd; /* tangent of logsumexp_k s_ik */
            tot += dd;
        }
        free(s); free(sd); free(xc);
    }
    const double la = alpha_lse(alpha, k);
    for (int kk = 0; kk < k; ++kk) tot -= (double)n * exp((double)alpha[kk] - la) * v_alpha[kk];
    for (int kk = 0; kk < k; ++kk) {
        for (int r = 0; r < d; ++r) {
            const double qv = q[kk * d + r];
            tot += ((double)m - gamma * gamma * exp(2.0 * qv)) * v_q[kk * d + r];
        }
        for (int j = 0; j < t; ++j)
            tot -= gamma * gamma * (double)l[(size_t)kk * t + j] * v_l[(size_t)kk * t + j];
    }
    if (f_out) {
        ll -= (double)n * la + 0.5 * (double)n * d * log(2.0 * M_PI);
        *f_out = ll + gmm_log_prior(q, l, d, k, gamma, m);
    }
    free(Q); free(QD);
    return tot;
}

/* ------------------------------------------------------------------------- */
/* Reprojection                                                              */
/* ------------------------------------------------------------------------- */

/* Forward-mode numbers with 14 tangent slots: 11 camera parameters, 3 point
 * coordinates (linearize, Sec. 5.1, carried out numerically). */
#define NT 14
typedef struct { double v; double d[NT]; } dual;

static dual dc(double v) { dual r; r.v = v; memset(r.d, 0, sizeof r.d); return r; }
static dual dvar(double v, int i) { dual r = dc(v); if (i >= 0) r.d[i] = 1.0; return r; }
static dual dadd(dual a, dual b) { dual r; r.v = a.v + b.v; for (int i = 0; i < NT; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
static dual dsub(dual a, dual b) { dual r; r.v = a.v - b.v; for (int i = 0; i < NT; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
static dual dmul(dual a, dual b) { dual r; r.v = a.v * b.v; for (int i = 0; i < NT; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
static dual ddiv(dual a, dual b) {
    dual r; r.v = a.v / b.v;
    for (int i = 0; i < NT; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
    return r;
}
static dual dsqrt_(dual a) { dual r; r.v = sqrt(a.v); for (int i = 0; i < NT; ++i) r.d[i] = a.d[i] / (2.0 * r.v); return r; }
static dual dsin_(dual a) { dual r; r.v = sin(a.v); const double c = cos(a.v); for (int i = 0; i < NT; ++i) r.d[i] = c * a.d[i]; return r; }
static dual dcos_(dual a) { dual r; r.v = cos(a.v); const double s = -sin(a.v); for (int i = 0; i < NT; ++i) r.d[i] = s * a.d[i]; return r; }

/* Projected 2-D position f L p + pp of point X seen by camera cam. */
static void project(const dual* cam, const dual* X, dual* out) {
    const dual* w = cam;
    dual u[3];
    for (int j = 0; j < 3; ++j) u[j] = dsub(X[j], cam[3 + j]);
    dual th2 = dadd(dadd(dmul(w[0], w[0]), dmul(w[1], w[1])), dmul(w[2], w[2]));
    dual Y[3];
    if (th2.v > 1e-16) { /* theta > 1e-8: Rodrigues' rotation formula */
        dual th = dsqrt_(th2);
        dual kx = ddiv(w[0], th), ky = ddiv(w[1], th), kz = ddiv(w[2], th);
        dual ct = dcos_(th), st = dsin_(th);
        dual omc = dsub(dc(1.0), ct);
        dual kxu[3] = {dsub(dmul(ky, u[2]), dmul(kz, u[1])), dsub(dmul(kz, u[0]), dmul(kx, u[2])),
                       dsub(dmul(kx, u[1]), dmul(ky, u[0]))};
        dual kdu = dadd(dadd(dmul(kx, u[0]), dmul(ky, u[1])), dmul(kz, u[2]));
        dual kk[3] = {kx, ky, kz};
        for (int j = 0; j < 3; ++j)
            Y[j] = dadd(dadd(dmul(u[j], ct), dmul(kxu[j], st)), dmul(kk[j], dmul(kdu, omc)));
    } else { /* first order: u + w x u */
        dual wxu[3] = {dsub(dmul(w[1], u[2]), dmul(w[2], u[1])), dsub(dmul(w[2], u[0]), dmul(w[0], u[2])),
                       dsub(dmul(w[0], u[1]), dmul(w[1], u[0]))};
        for (int j = 0; j < 3; ++j) Y[j] = dadd(u[j], wxu[j]);
    }
    dual p0 = ddiv(Y[0], Y[2]), p1 = ddiv(Y[1], Y[2]);
    dual rho = dadd(dmul(p0, p0), dmul(p1, p1));
    dual L = dadd(dadd(dc(1.0), dmul(cam[9], rho)), dmul(cam[10], dmul(rho, rho)));
    dual fl = dmul(cam[6], L);
    out[0] = dadd(dmul(fl, p0), cam[7]);
    out[1] = dadd(dmul(fl, p1), cam[8]);
}

/* Jacobian J (2 x 14) and value of the projection of observation j. */
static void obs_jacobian(const float* cams, const float* pts, int32_t ci, int32_t pi, double* val,
                         double J[2][NT]) {
    dual cam[11], X[3], out[2];
    for (int a = 0; a < 11; ++a) cam[a] = dvar(cams[(size_t)ci * 11 + a], a);
    for (int b = 0; b < 3; ++b) X[b] = dvar(pts[(size_t)pi * 3 + b], 11 + b);
    project(cam, X, out);
    for (int o = 0; o < 2; ++o) {
        val[o] = out[o].v;
        for (int a = 0; a < NT; ++a) J[o][a] = out[o].d[a];
    }
}

static int obs_ok(const int32_t* obs, int64_t j, int32_t nc, int32_t np_) {
    const int32_t ci = obs[2 * j], pi = obs[2 * j + 1];
    return ci >= 0 && ci < nc && pi >= 0 && pi < np_;
}

/* res_j = proj_j - t_j (parity pinned: scipy rotation, worked example, tests).
 * Observations with an out-of-range index get NaN; returns their count. */
int64_t oracle_reproj_residual(const float* cams, const float* pts, const int32_t* obs,
                               const float* tgt, int32_t n_cams, int32_t n_pts, int64_t n_obs,
                               double* res) {
    int64_t bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t j = 0; j < n_obs; ++j) {
        if (!obs_ok(obs, j, n_cams, n_pts)) { res[2 * j] = res[2 * j + 1] = NAN; ++bad; continue; }
        double val[2], J[2][NT];
        obs_jacobian(cams, pts, obs[2 * j], obs[2 * j + 1], val, J);
        res[2 * j] = val[0] - (double)tgt[2 * j];
        res[2 * j + 1] = val[1] - (double)tgt[2 * j + 1];
    }
    return bad;
}

/*
 * VJP of the residual: d_cams[c] += J_cam^T w_j, d_pts[p] += J_pt^T w_j over all
 * observations (the transpose of the gathers cams.(obs.j.0), pts.(obs.j.1) is an
 * Accum into the sliced references, LetIndexingTranspose, Sec. 5.2 / 5.3.3).
 * Outputs are overwritten (not accumulated). Parity pinned: dot-product test
 * against oracle_reproj_jvp, whose Jacobian columns are checked by central
 * differences. Returns the number of skipped (out-of-range) observations.
 */
int64_t oracle_reproj_vjp(const float* cams, const float* pts, const int32_t* obs, const float* w,
                          int32_t n_cams, int32_t n_pts, int64_t n_obs, double* d_cams,
                          double* d_pts) {
    memset(d_cams, 0, sizeof(double) * (size_t)n_cams * 11);
    memset(d_pts, 0, sizeof(double) * (size_t)n_pts * 3);
    int64_t bad = 0;
#pragma omp parallel reduction(+ : bad)
    {
        double* dc_p = (double*)calloc((size_t)n_cams * 11, sizeof(double));
        double* dp_p = (double*)calloc((size_t)n_pts * 3, sizeof(double));
#pragma omp for schedule(static)
        for (int64_t j = 0; j < n_obs; ++j) {
            if (!obs_ok(obs, j, n_cams, n_pts)) { ++bad; continue; }
            const int32_t ci = obs[2 * j], pi = obs[2 * j + 1];
            double val[2], J[2][NT];
            obs_jacobian(cams, pts, ci, pi, val, J);
            const double w0 = w[2 * j], w1 = w[2 * j + 1];
            for (int a = 0; a < 11; ++a) dc_p[(size_t)ci * 11 + a] += J[0][a] * w0 + J[1][a] * w1;
            for (int b = 0; b < 3; ++b) dp_p[(size_t)pi * 3 + b] += J[0][11 + b] * w0 + J[1][11 + b] * w1;
        }
#pragma omp critical
        {
            for (size_t i = 0; i < (size_t)n_cams * 11; ++i) d_cams[i] += dc_p[i];
            for (size_t i = 0; i < (size_t)n_pts * 3; ++i) d_pts[i] += dp_p[i];
        }
        free(dc_p);
        free(dp_p);
    }
    return bad;
}

/* JVP of the residual: jv_j = J_cam v_cams[c] + J_pt v_pts[p] (linearize). */
int64_t oracle_reproj_jvp(const float* cams, const float* pts, const int32_t* obs,
                          int32_t n_cams, int32_t n_pts, int64_t n_obs, const double* v_cams,
                          const double* v_pts, double* jv) {
    int64_t bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t j = 0; j < n_obs; ++j) {
        if (!obs_ok(obs, j, n_cams, n_pts)) { jv[2 * j] = jv[2 * j + 1] = NAN; ++bad; continue; }
        const int32_t ci = obs[2 * j], pi = obs[2 * j + 1];
        double val[2], J[2][NT];
        obs_jacobian(cams, pts, ci, pi, val, J);
        for (int o = 0; o < 2; ++o) {
            double s = 0.0;
            for (int a = 0; a < 11; ++a) s += J[o][a] * v_cams[(size_t)ci * 11 + a];
            for (int b = 0; b < 3; ++b) s += J[o][11 + b] * v_pts[(size_t)pi * 3 + b];
            jv[2 * j + o] = s;
        }
    }
    return bad;
}

/*
 * Gauss-Newton normal equations of the reprojection (J = d res / d(cams, pts)):
 *   U[c] = sum_{j: cam c} J_c^T J_c   (11 x 11, upper triangle packed by rows: 66)
 *   V[p] = sum_{j: point p} J_p^T J_p (3 x 3, upper triangle packed by rows: 6)
 *   W[j] = J_c^T J_p of observation j (11 x 3 row-major, nullable)
 *   g_cams[c] = sum J_c^T r_j, g_pts[p] = sum J_p^T r_j, res[j] = r_j (nullable)
 * with J_c, J_p the 2 x 11 and 2 x 3 blocks of observation j's Jacobian: the
 * block rows of J^T J, each an Accum into the camera's or the point's slot.
 * Outputs are overwritten. Parity pinned: (J^T J) v = J^T (J v) through
 * oracle_reproj_jvp / oracle_reproj_vjp, and a dense J^T J on tiny inputs
 * (tests). Returns the number of skipped (out-of-range) observations.
 */
int64_t oracle_reproj_normal_eqs(const float* cams, const float* pts, const int32_t* obs, const float* tgt,
                                 int32_t n_cams, int32_t n_pts, int64_t n_obs, double* U, double* V,
                                 double* W, double* g_cams, double* g_pts, double* res) {
    double* Jb = (double*)malloc(sizeof(double) * (size_t)n_obs * 2 * NT);
    double* rb = (double*)malloc(sizeof(double) * (size_t)n_obs * 2);
    int64_t bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t j = 0; j < n_obs; ++j) {
        if (!obs_ok(obs, j, n_cams, n_pts)) { ++bad; continue; }
        double val[2], J[2][NT];
        obs_jacobian(cams, pts, obs[2 * j], obs[2 * j + 1], val, J);
        for (int o = 0; o < 2; ++o) {
            rb[2 * j + o] = val[o] - (double)tgt[2 * j + o];
            for (int a = 0; a < NT; ++a) Jb[(size_t)j * 2 * NT + o * NT + a] = J[o][a];
        }
    }
    memset(U, 0, sizeof(double) * (size_t)n_cams * 66);
    memset(V, 0, sizeof(double) * (size_t)n_pts * 6);
    memset(g_cams, 0, sizeof(double) * (size_t)n_cams * 11);
    memset(g_pts, 0, sizeof(double) * (size_t)n_pts * 3);
    for (int64_t j = 0; j < n_obs; ++j) {
        if (!obs_ok(obs, j, n_cams, n_pts)) {
            if (res) res[2 * j] = res[2 * j + 1] = NAN;
            if (W) for (int e = 0; e < 33; ++e) W[(size_t)j * 33 + e] = NAN;
            continue;
        }
        const int32_t ci = obs[2 * j], pi = obs[2 * j + 1];
        const double* J0 = Jb + (size_t)j * 2 * NT;
        const double* J1 = J0 + NT;
        const double r0 = rb[2 * j], r1 = rb[2 * j + 1];
        int e = 0;
        for (int a = 0; a < 11; ++a)
            for (int b = a; b < 11; ++b, ++e) U[(size_t)ci * 66 + e] += J0[a] * J0[b] + J1[a] * J1[b];
        e = 0;
        for (int a = 0; a < 3; ++a)
            for (int b = a; b < 3; ++b, ++e) V[(size_t)pi * 6 + e] += J0[11 + a] * J0[11 + b] + J1[11 + a] * J1[11 + b];
        if (W)
            for (int a = 0; a < 11; ++a)
                for (int b = 0; b < 3; ++b) W[(size_t)j * 33 + a * 3 + b] = J0[a] * J0[11 + b] + J1[a] * J1[11 + b];
        for (int a = 0; a < 11; ++a) g_cams[(size_t)ci * 11 + a] += J0[a] * r0 + J1[a] * r1;
        for (int b = 0; b < 3; ++b) g_pts[(size_t)pi * 3 + b] += J0[11 + b] * r0 + J1[11 + b] * r1;
        if (res) { res[2 * j] = r0; res[2 * j + 1] = r1; }
    }
    free(Jb);
    free(rb);
    return bad;
}

/* Per-observation Jacobian rows (M x 2 x 14), for tests on small inputs. */
void oracle_reproj_jacobian(const float* cams, const float* pts, const int32_t* obs, int64_t n_obs,
                            double* jac) {
    for (int64_t j = 0; j < n_obs; ++j) {
        double val[2], J[2][NT];
        obs_jacobian(cams, pts, obs[2 * j], obs[2 * j + 1], val, J);
        for (int o = 0; o < 2; ++o)
            for (int a = 0; a < NT; ++a) jac[(size_t)j * 2 * NT + o * NT + a] = J[o][a];
    }
}

/* ------------------------------------------------------------------------- */
/* Accum scatter and index preparation                                       */
/* ------------------------------------------------------------------------- */

/* acc[idx[j], :] += vals[j, :] for float values, sequentially in j (the plain
 * meaning of hist!(x.i) += v, Sec. 2.3.3 / 6.1.2). acc is overwritten from zero.
 * Out-of-range indices are skipped; returns their count. */
int64_t oracle_scatter_add_f64(const int32_t* idx, const float* vals, int64_t m, int w,
                               int32_t n_buckets, double* acc) {
    memset(acc, 0, sizeof(double) * (size_t)n_buckets * w);
    int64_t bad = 0;
    for (int64_t j = 0; j < m; ++j) {
        const int32_t b = idx[j];
        if (b < 0 || b >= n_buckets) { ++bad; continue; }
        for (int c = 0; c < w; ++c) acc[(size_t)b * w + c] += (double)vals[(size_t)j * w + c];
    }
    return bad;
}

/* Same for int32 values, accumulated in int64 (exact). */
int64_t oracle_scatter_add_i64(const int32_t* idx, const int32_t* vals, int64_t m, int w,
                               int32_t n_buckets, int64_t* acc) {
    memset(acc, 0, sizeof(int64_t) * (size_t)n_buckets * w);
    int64_t bad = 0;
    for (int64_t j = 0; j < m; ++j) {
        const int32_t b = idx[j];
        if (b < 0 || b >= n_buckets) { ++bad; continue; }
        for (int c = 0; c < w; ++c) acc[(size_t)b * w + c] += (int64_t)vals[(size_t)j * w + c];
    }
    return bad;
}

/*
 * Stable sort of element ids by key (counting sort): perm lists, for key 0,
 * 1, ..., the ids j with that key in increasing j; seg_off[b] is where key b's
 * run starts (seg_off[n_keys] = number of valid keys). Index validity is checked
 * where the index is made from data (Sec. 6.3): returns the number of keys out
 * of [0, n_keys), which are left out of perm.
 */
int64_t oracle_stable_sort_by_key(const int32_t* keys, int64_t m, int32_t n_keys, int32_t* perm,
                                  int64_t* seg_off) {
    int64_t* cnt = (int64_t*)calloc((size_t)n_keys + 1, sizeof(int64_t));
    int64_t bad = 0;
    for (int64_t j = 0; j < m; ++j) {
        const int32_t b = keys[j];
        if (b < 0 || b >= n_keys) { ++bad; continue; }
        cnt[b + 1]++;
    }
    for (int32_t b = 0; b < n_keys; ++b) cnt[b + 1] += cnt[b];
    memcpy(seg_off, cnt, sizeof(int64_t) * ((size_t)n_keys + 1));
    for (int64_t j = 0; j < m; ++j) {
        const int32_t b = keys[j];
        if (b < 0 || b >= n_keys) continue;
        perm[cnt[b]++] = (int32_t)j;
    }
    free(cnt);
    return bad;
}
