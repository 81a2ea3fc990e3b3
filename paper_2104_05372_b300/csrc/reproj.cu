// Camera reprojection residual and its VJP with Accum scatter into per-camera
// and per-point cotangents (bundle-adjustment objective), FP32 on CUDA cores.
//
// Per observation j with (c, p) = obs[j]:
//   u = X_p - c_c, Y = R(w_c) u, p = Y_xy / Y_z, rho = |p|^2,
//   L = 1 + k1 rho + k2 rho^2, res_j = f L p + pp - t_j.
// The rotation of each camera is expanded once per call in float64 (A4's
// parameter expansion): R as a float32 hi/lo pair, plus the Jacobian factor
// J_r(w) = I - (1-cos t)/t^2 [w]x + (t - sin t)/t^3 [w]x^2 (t = |w|), for which
// d(R u)/dw = -[R u]x J_r^T. Y_z is evaluated with error-free transformations
// (u exact as a hi/lo pair, products via FMA, sums via TwoSum), so points close
// to the image plane keep the accuracy of the float64 oracle.
//
// VJP (A5): the reads cams.(obs.j.0), pts.(obs.j.1) transpose to accumulations
// into d_cams!(obs.j.0) and d_pts!(obs.j.1) (LetIndexingTranspose) -- an
// irregular segmented reduction (histogram pattern, Sec. 6.1.3). Strategies:
//   ATOMIC  one red.global.add per value, observations in their own order;
//   WARPAGG lanes of a warp with the same camera / point combine first;
//   SORT    observations in camera-sorted order from a plan: runs of equal
//           cameras are summed with a segmented warp scan, one atomic per run.
// No observation stores its Jacobian: the projection is recomputed from the
// gathered parameters (only non-linear steps keep their inputs, Sec. 5.3.2).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "accum.cuh"
#include "common.cuh"
#include "plan_internal.cuh"
#include "trace.cuh"

namespace gpa {

constexpr int kCamRec = 32;  // floats per expanded camera: one 128-byte line
// layout: [0..8] R hi (row-major), [9..11] R lo of the depth row, [12..14] c, [15] f,
//         [16..17] pp, [18..19] kappa, [20..28] J_r (row-major), [29..31] pad.
// The residual reads the first 20 floats only.
constexpr int kCamResid = 20;

// Rodrigues coefficients as power series in x = theta^2 (the Taylor series of
// sin and cos), summed by Horner's rule with constant coefficients:
//   f1 = sin t / t         = sum_n (-1)^n x^n / (2n+1)!
//   f2 = (1 - cos t) / t^2 = sum_n (-1)^n x^n / (2n+2)!
//   g  = (t - sin t) / t^3 = sum_n (-1)^n x^n / (2n+3)!
// Terms n = 0 .. kSeriesTerms; for x <= kSeriesMaxTh2 the first omitted term
// is below 1e-17, and the float64 sums are within 4e-16 of the exact values
// (checked against 120-digit arithmetic over [0, 16]).
constexpr int kSeriesTerms = 16;
constexpr double kSeriesMaxTh2 = 16.0;

__host__ __device__ constexpr double inv_factorial(int k) {
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= (double)i;
    return 1.0 / f;
}

// sum_{n=0}^{kSeriesTerms} (-1)^n x^n / (2n + off)!
template <int OFF, typename T>
__device__ __forceinline__ T rodrigues_series(T x) {
    constexpr int N = kSeriesTerms;
    T t = (T)((N & 1 ? -1.0 : 1.0) * inv_factorial(2 * N + OFF));
#pragma unroll
    for (int n = N - 1; n >= 0; --n) t = fma(t, x, (T)((n & 1 ? -1.0 : 1.0) * inv_factorial(2 * n + OFF)));
    return t;
}

// The record o of the camera with parameters c. The rotation is formed in
// float64 (its last row is stored as a float32 hi/lo pair); the right
// Jacobian J_r = I - A [w]x + B [w]x^2, stored in float32, is formed in float32.
__device__ __forceinline__ void cam_expand_one(const float (&c)[11], float (&o)[kCamRec]) {
    const double w0 = c[0], w1 = c[1], w2 = c[2];
    const double th2 = w0 * w0 + w1 * w1 + w2 * w2;
    double R[9];
    float A, B;
    if (th2 <= kSeriesMaxTh2) {
        // R = I + f1 [w]x + f2 [w]x^2 with [w]x^2 = w w^T - theta^2 I
        const double f1 = rodrigues_series<1>(th2), f2 = rodrigues_series<2>(th2);
        const double d = 1.0 - f2 * th2;  // cos theta
        R[0] = fma(f2, w0 * w0, d);          R[1] = fma(f2, w0 * w1, -f1 * w2); R[2] = fma(f2, w0 * w2, f1 * w1);
        R[3] = fma(f2, w1 * w0, f1 * w2);    R[4] = fma(f2, w1 * w1, d);        R[5] = fma(f2, w1 * w2, -f1 * w0);
        R[6] = fma(f2, w2 * w0, -f1 * w1);   R[7] = fma(f2, w2 * w1, f1 * w0);  R[8] = fma(f2, w2 * w2, d);
        A = (float)f2;
        B = rodrigues_series<3>((float)th2);
    } else {  // theta > 4: unit axis k, sin and cos of theta
        const double th = sqrt(th2);
        const double k0 = w0 / th, k1 = w1 / th, k2 = w2 / th;
        double st, ct;
        sincos(th, &st, &ct);
        const double omc = 1.0 - ct;
        R[0] = ct + omc * k0 * k0;      R[1] = -st * k2 + omc * k0 * k1; R[2] = st * k1 + omc * k0 * k2;
        R[3] = st * k2 + omc * k1 * k0; R[4] = ct + omc * k1 * k1;      R[5] = -st * k0 + omc * k1 * k2;
        R[6] = -st * k1 + omc * k2 * k0; R[7] = st * k0 + omc * k2 * k1; R[8] = ct + omc * k2 * k2;
        A = (float)(omc / th2);
        B = (float)((th - st) / (th2 * th));
    }
    // [w]x and [w]x^2 = w w^T - theta^2 I in float32
    const float v[3] = {c[0], c[1], c[2]};
    const float x2 = (float)th2;
    const float W[9] = {0.f, -v[2], v[1], v[2], 0.f, -v[0], -v[1], v[0], 0.f};
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float hi = (float)R[i];
        o[i] = hi;
        if (i >= 6) o[9 + (i - 6)] = (float)(R[i] - (double)hi);
        const int r = i / 3, q = i % 3;
        const float W2 = v[r] * v[q] - (r == q ? x2 : 0.f);
        o[20 + i] = fmaf(B, W2, fmaf(-A, W[i], r == q ? 1.f : 0.f));
    }
    o[12] = c[3]; o[13] = c[4]; o[14] = c[5];
    o[15] = c[6]; o[16] = c[7]; o[17] = c[8];
    o[18] = c[9]; o[19] = c[10];
    o[29] = 0.f; o[30] = 0.f; o[31] = 0.f;
}

// One warp per block: a camera's expansion is a chain of dependent float64
// operations, which this GPU issues at a low rate, so the cameras are spread
// over as many SMs as possible.
constexpr int kCamPerBlock = 32;

// Cameras cam0 .. cam0 + 31 by one warp, lane = camera. Parameters and
// records pass through shared memory (sm: 32 x 33 floats) so that both move
// as contiguous rows: a thread storing its own 128-byte record would touch 32
// lines per store instruction.
__device__ __forceinline__ void cam_expand_warp(const float* __restrict__ cams, int n_cams, int cam0,
                                                float* __restrict__ rec, float* sm) {
    const int lane = threadIdx.x & 31;
    const int nv = min(32, n_cams - cam0);
    for (int i = lane; i < nv * 11; i += 32) sm[i] = __ldg(cams + (size_t)cam0 * 11 + i);
    __syncwarp();
    float c[11], o[kCamRec];
#pragma unroll
    for (int j = 0; j < 11; ++j) c[j] = lane < nv ? sm[lane * 11 + j] : 0.f;
    __syncwarp();
    cam_expand_one(c, o);
#pragma unroll
    for (int j = 0; j < kCamRec; ++j) sm[lane * (kCamRec + 1) + j] = o[j];
    __syncwarp();
    for (int i = 0; i < nv; ++i) rec[(size_t)(cam0 + i) * kCamRec + lane] = sm[i * (kCamRec + 1) + lane];
}

__global__ void __launch_bounds__(32) cam_expand_kernel(const float* __restrict__ cams, int n_cams,
                                                        float* __restrict__ rec) {
    __shared__ float sm[32 * (kCamRec + 1)];
    cam_expand_warp(cams, n_cams, blockIdx.x * kCamPerBlock, rec, sm);
}

// Per-call preparation of the VJP: the first ncb blocks expand the cameras
// (kCamPerBlock each, by their first warp), the others copy the points into
// 16-byte rows (x, y, z, 0), so that a gathered point is one 16-byte load, and
// zero the padded point accumulators (when acc is given).
__global__ void __launch_bounds__(128) vjp_prep_kernel(const float* __restrict__ cams, int n_cams,
                                                       float* __restrict__ rec, int ncb,
                                                       const float* __restrict__ pts, int n_pts,
                                                       float4* __restrict__ pts4, float4* __restrict__ acc) {
    __shared__ float sm[32 * (kCamRec + 1)];
    if ((int)blockIdx.x < ncb) {
        if (threadIdx.x < kCamPerBlock) cam_expand_warp(cams, n_cams, blockIdx.x * kCamPerBlock, rec, sm);
        return;
    }
    const int64_t stride = (int64_t)(gridDim.x - ncb) * blockDim.x;
    for (int64_t p = (int64_t)(blockIdx.x - ncb) * blockDim.x + threadIdx.x; p < n_pts; p += stride) {
        const float* X = pts + p * 3;
        pts4[p] = make_float4(__ldg(X), __ldg(X + 1), __ldg(X + 2), 0.f);
        if (acc) acc[p] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// ---- error-free transformations ---------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// The first NF floats of camera ci's record (128-byte aligned) in 32-byte loads:
// one sector per lane per load instruction (16-byte loads would fetch every
// sector of a gathered record twice).
template <int NF>
__device__ __forceinline__ void load_cam(const float* __restrict__ rec, int ci, float (&cam)[kCamRec]) {
    const float* p = rec + (size_t)ci * kCamRec;
#pragma unroll
    for (int i = 0; i < (NF + 7) / 8; ++i)
        asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=f"(cam[8 * i]), "=f"(cam[8 * i + 1]), "=f"(cam[8 * i + 2]), "=f"(cam[8 * i + 3]),
              "=f"(cam[8 * i + 4]), "=f"(cam[8 * i + 5]), "=f"(cam[8 * i + 6]), "=f"(cam[8 * i + 7])
            : "l"(p + 8 * i));
}

// Point pi of a [P][3] array: one float2 and one float load when the array is
// 8-byte aligned (which half is 8-byte aligned follows the parity of pi),
// three float loads otherwise.
__device__ __forceinline__ void load_point(const float* __restrict__ pts, int pi, bool al8, float& X0, float& X1,
                                           float& X2) {
    const float* X = pts + (size_t)pi * 3;
    if (!al8) {
        X0 = __ldg(X);
        X1 = __ldg(X + 1);
        X2 = __ldg(X + 2);
    } else if ((pi & 1) == 0) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(X));
        X0 = v.x;
        X1 = v.y;
        X2 = __ldg(X + 2);
    } else {
        X0 = __ldg(X);
        const float2 v = __ldg(reinterpret_cast<const float2*>(X + 1));
        X1 = v.x;
        X2 = v.y;
    }
}

// Point pi from the padded copy (one 16-byte load) when there is one.
__device__ __forceinline__ void load_point_any(const float4* __restrict__ pts4, const float* __restrict__ pts, int pi,
                                               bool al8, float& X0, float& X1, float& X2) {
    if (pts4) {
        const float4 v = __ldg(pts4 + pi);
        X0 = v.x;
        X1 = v.y;
        X2 = v.z;
    } else {
        load_point(pts, pi, al8, X0, X1, X2);
    }
}

// d_pts[pi] += g directly: float2 + float atomics when d_pts is 8-byte aligned.
__device__ __forceinline__ void red_add_point(float* __restrict__ d_pts, int pi, const float (&g)[3], bool al8) {
    float* dp = d_pts + (size_t)pi * 3;
    if (!al8) {
        atomicAdd(dp, g[0]);
        atomicAdd(dp + 1, g[1]);
        atomicAdd(dp + 2, g[2]);
    } else if ((pi & 1) == 0) {
        atomicAdd(reinterpret_cast<float2*>(dp), make_float2(g[0], g[1]));
        atomicAdd(dp + 2, g[2]);
    } else {
        atomicAdd(dp, g[0]);
        atomicAdd(reinterpret_cast<float2*>(dp + 1), make_float2(g[1], g[2]));
    }
}

struct Proj {
    float Y[3];   // rotated point (Y[2] compensated)
    float p[2];   // normalised image coordinates
    float rho, L;
    float out[2]; // f L p + pp
};

// Projection of point X by the expanded camera rc (a register copy of the record).
__device__ __forceinline__ Proj project(const float* __restrict__ rc, float X0, float X1, float X2) {
    Proj P;
    float u[3], ue[3];
    two_sum(X0, -rc[12], u[0], ue[0]);
    two_sum(X1, -rc[13], u[1], ue[1]);
    two_sum(X2, -rc[14], u[2], ue[2]);
    float Rh[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) Rh[i] = rc[i];
    P.Y[0] = fmaf(Rh[0], u[0], fmaf(Rh[1], u[1], Rh[2] * u[2]));
    P.Y[1] = fmaf(Rh[3], u[0], fmaf(Rh[4], u[1], Rh[5] * u[2]));
    {
        float pr[3], pe[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            pr[j] = __fmul_rn(Rh[6 + j], u[j]);
            pe[j] = fmaf(Rh[6 + j], u[j], -pr[j]);
        }
        float s1, t1, s2, t2;
        two_sum(pr[0], pr[1], s1, t1);
        two_sum(s1, pr[2], s2, t2);
        float corr = t1 + t2 + pe[0] + pe[1] + pe[2];
#pragma unroll
        for (int j = 0; j < 3; ++j) corr = fmaf(rc[9 + j], u[j], fmaf(Rh[6 + j], ue[j], corr));
        P.Y[2] = s2 + corr;
    }
    P.p[0] = P.Y[0] / P.Y[2];
    P.p[1] = P.Y[1] / P.Y[2];
    P.rho = P.p[0] * P.p[0] + P.p[1] * P.p[1];
    const float k1 = rc[18], k2 = rc[19], f = rc[15];
    P.L = 1.f + k1 * P.rho + k2 * P.rho * P.rho;
    P.out[0] = f * P.L * P.p[0] + rc[16];
    P.out[1] = f * P.L * P.p[1] + rc[17];
    return P;
}

// Cotangents of the 11 camera parameters and 3 point coordinates for a
// cotangent (w0, w1) of the projection.
__device__ __forceinline__ void project_vjp(const float* __restrict__ rc, const Proj& P, float w0, float w1,
                                            float (&gc)[11], float (&gp)[3]) {
    const float f = rc[15], k1 = rc[18], k2 = rc[19];
    const float pw = P.p[0] * w0 + P.p[1] * w1;
    const float dL = f * pw;
    const float drho = dL * (k1 + 2.f * k2 * P.rho);
    const float fl = f * P.L;
    const float dp0 = fl * w0 + 2.f * drho * P.p[0];
    const float dp1 = fl * w1 + 2.f * drho * P.p[1];
    const float inv = 1.f / P.Y[2];
    const float yb0 = dp0 * inv, yb1 = dp1 * inv;
    const float yb2 = -(dp0 * P.p[0] + dp1 * P.p[1]) * inv;
    // d X = R^T ybar
    float dX[3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
        dX[j] = rc[j] * yb0 + rc[3 + j] * yb1 + rc[6 + j] * yb2;
    // d w = J_r (Y x ybar)
    const float cx = P.Y[1] * yb2 - P.Y[2] * yb1;
    const float cy = P.Y[2] * yb0 - P.Y[0] * yb2;
    const float cz = P.Y[0] * yb1 - P.Y[1] * yb0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
        gc[i] = rc[20 + 3 * i] * cx + rc[21 + 3 * i] * cy + rc[22 + 3 * i] * cz;
    gc[3] = -dX[0]; gc[4] = -dX[1]; gc[5] = -dX[2];
    gc[6] = P.L * pw;
    gc[7] = w0; gc[8] = w1;
    gc[9] = dL * P.rho;
    gc[10] = dL * P.rho * P.rho;
    gp[0] = dX[0]; gp[1] = dX[1]; gp[2] = dX[2];
}

// Tangent of the projection for tangents (vc[0..10]) of the camera and (vx) of
// the point (linearize, Sec. 5.1): Ydot = R (Xdot - cdot) + (J_r^T wdot) x Y,
// pdot = (Ydot_xy - p Ydot_z) / Y_z, rhodot = 2 p.pdot,
// Ldot = k1dot rho + k1 rhodot + k2dot rho^2 + 2 k2 rho rhodot,
// out_dot = fdot L p + f Ldot p + f L pdot + ppdot.
__device__ __forceinline__ void project_jvp(const float* __restrict__ rc, const Proj& P, const float (&vc)[11],
                                            const float (&vx)[3], float (&jv)[2]) {
    const float f = rc[15], k1 = rc[18], k2 = rc[19];
    float v[3];  // J_r^T wdot
#pragma unroll
    for (int a = 0; a < 3; ++a) v[a] = rc[20 + a] * vc[0] + rc[23 + a] * vc[1] + rc[26 + a] * vc[2];
    const float du[3] = {vx[0] - vc[3], vx[1] - vc[4], vx[2] - vc[5]};
    float Yd[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) Yd[i] = rc[3 * i] * du[0] + rc[3 * i + 1] * du[1] + rc[3 * i + 2] * du[2];
    Yd[0] += v[1] * P.Y[2] - v[2] * P.Y[1];
    Yd[1] += v[2] * P.Y[0] - v[0] * P.Y[2];
    Yd[2] += v[0] * P.Y[1] - v[1] * P.Y[0];
    const float inv = 1.f / P.Y[2];
    const float pd0 = (Yd[0] - P.p[0] * Yd[2]) * inv, pd1 = (Yd[1] - P.p[1] * Yd[2]) * inv;
    const float rhod = 2.f * (P.p[0] * pd0 + P.p[1] * pd1);
    const float Ld = vc[9] * P.rho + k1 * rhod + vc[10] * P.rho * P.rho + 2.f * k2 * P.rho * rhod;
    const float fL = f * P.L, c0 = vc[6] * P.L + f * Ld;
    jv[0] = c0 * P.p[0] + fL * pd0 + vc[7];
    jv[1] = c0 * P.p[1] + fL * pd1 + vc[8];
}

__global__ void __launch_bounds__(256) reproj_jvp_kernel(const float* __restrict__ rec, const float* __restrict__ pts,
                                                         const int2* __restrict__ obs, const float* __restrict__ v_cams,
                                                         const float* __restrict__ v_pts, int n_cams, int n_pts,
                                                         int64_t n_obs, float2* __restrict__ jv_out,
                                                         int32_t* __restrict__ status, int pts8) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_obs; j += stride) {
        const int2 o = __ldg(obs + j);
        if (o.x < 0 || o.x >= n_cams || o.y < 0 || o.y >= n_pts) {
            jv_out[j] = make_float2(NAN, NAN);
            report(status, GPA_ERR_INDEX);
            continue;
        }
        float rc[kCamRec];
        load_cam<kCamRec>(rec, o.x, rc);
        float X0, X1, X2;
        load_point(pts, o.y, pts8, X0, X1, X2);
        const Proj P = project(rc, X0, X1, X2);
        float vc[11], vx[3], jv[2];
#pragma unroll
        for (int i = 0; i < 11; ++i) vc[i] = __ldg(v_cams + (size_t)o.x * 11 + i);
#pragma unroll
        for (int i = 0; i < 3; ++i) vx[i] = __ldg(v_pts + (size_t)o.y * 3 + i);
        project_jvp(rc, P, vc, vx, jv);
        jv_out[j] = make_float2(jv[0], jv[1]);
    }
}

__global__ void __launch_bounds__(256) reproj_residual_kernel(
    const float* __restrict__ rec, const float* __restrict__ pts, const int2* __restrict__ obs,
    const float2* __restrict__ tgt, int n_cams, int n_pts, int64_t n_obs, float2* __restrict__ res,
    int32_t* __restrict__ status, int pts8) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_obs; j += stride) {
        const int2 o = __ldg(obs + j);
        if (o.x < 0 || o.x >= n_cams || o.y < 0 || o.y >= n_pts) {
            res[j] = make_float2(NAN, NAN);
            report(status, GPA_ERR_INDEX);
            continue;
        }
        float rc[kCamRec];
        load_cam<kCamResid>(rec, o.x, rc);
        float X0, X1, X2;
        load_point(pts, o.y, pts8, X0, X1, X2);
        const Proj P = project(rc, X0, X1, X2);
        const float2 t = __ldg(tgt + j);
        res[j] = make_float2(P.out[0] - t.x, P.out[1] - t.y);
    }
}

// VJP over observations; FUSED also writes res and uses w = wscale * res.
template <int STRAT, bool FUSED>
__global__ void __launch_bounds__(256) reproj_vjp_kernel(
    const float* __restrict__ rec, const float* __restrict__ pts, const float4* __restrict__ pts4,
    const int2* __restrict__ obs,
    const float2* __restrict__ wv, const float2* __restrict__ tgt, float wscale, int n_cams, int n_pts,
    int64_t n_obs, float* __restrict__ d_cams, float* __restrict__ d_pts,
    float4* __restrict__ d_pts4, float2* __restrict__ res, int32_t* __restrict__ status, int pts8, int dpts8) {
    static_assert(STRAT == GPA_SCATTER_ATOMIC || STRAT == GPA_SCATTER_WARPAGG, "SORT has its own kernel");
    // point cotangents: into the 16-byte padded accumulators d_pts4 (one vector
    // atomic per observation) when given, else straight into d_pts
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    // trip count is uniform over the block so that every lane reaches the shuffles
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n_obs; base += stride) {
        const int64_t pos = base + threadIdx.x;
        bool valid = pos < n_obs;
        int64_t e = pos;  // element id
        int ci = -1, pi = -1;
        if (valid) {
            const int2 o = __ldg(obs + pos);
            ci = o.x;
            pi = o.y;
            if (ci < 0 || ci >= n_cams || pi < 0 || pi >= n_pts) {
                if (FUSED) res[e] = make_float2(NAN, NAN);
                report(status, GPA_ERR_INDEX);
                valid = false;
            }
        }
        float gc[11], gp[3];
#pragma unroll
        for (int i = 0; i < 11; ++i) gc[i] = 0.f;
        gp[0] = gp[1] = gp[2] = 0.f;
        if (valid) {
            float rc[kCamRec];
            load_cam<kCamRec>(rec, ci, rc);
            float X0, X1, X2;
            load_point_any(pts4, pts, pi, pts8, X0, X1, X2);
            const Proj P = project(rc, X0, X1, X2);
            float w0, w1;
            if (FUSED) {
                const float2 t = __ldg(tgt + e);
                const float r0 = P.out[0] - t.x, r1 = P.out[1] - t.y;
                res[e] = make_float2(r0, r1);
                w0 = wscale * r0;
                w1 = wscale * r1;
            } else {
                const float2 w = __ldg(wv + e);
                w0 = w.x;
                w1 = w.y;
            }
            project_vjp(rc, P, w0, w1, gc, gp);
        }
        if (STRAT == GPA_SCATTER_ATOMIC) {
            if (valid) {
                float* dc = d_cams + (size_t)ci * 11;
#pragma unroll
                for (int i = 0; i < 11; ++i) red_add(dc + i, gc[i]);
                if (d_pts4)
                    atomicAdd(d_pts4 + pi, make_float4(gp[0], gp[1], gp[2], 0.f));
                else
                    red_add_point(d_pts, pi, gp, dpts8);
            }
        } else if (STRAT == GPA_SCATTER_WARPAGG) {
            const int ck = valid ? ci : -1 - lane;
            const unsigned gcm = __match_any_sync(0xffffffffu, ck);
            if (__any_sync(0xffffffffu, __popc(gcm) > 1)) {
#pragma unroll
                for (int i = 0; i < 11; ++i) gc[i] = group_sum(gc[i], gcm);
            }
            if (valid && (__ffs(gcm) - 1) == lane) {
                float* dc = d_cams + (size_t)ci * 11;
#pragma unroll
                for (int i = 0; i < 11; ++i) red_add(dc + i, gc[i]);
            }
            const int pk = valid ? pi : -1 - lane;
            const unsigned gpm = __match_any_sync(0xffffffffu, pk);
            if (__any_sync(0xffffffffu, __popc(gpm) > 1)) {
#pragma unroll
                for (int i = 0; i < 3; ++i) gp[i] = group_sum(gp[i], gpm);
            }
            if (valid && (__ffs(gpm) - 1) == lane) {
                if (d_pts4)
                    atomicAdd(d_pts4 + pi, make_float4(gp[0], gp[1], gp[2], 0.f));
                else
                    red_add_point(d_pts, pi, gp, dpts8);
            }
        }
    }
}

// SORT strategy: observations in the plan's camera-sorted order, kOpt
// consecutive ones per thread. A thread keeps its camera's expanded record and
// its partial camera cotangent in registers while the camera repeats (a camera
// owns about M / C consecutive observations), adds a finished run with 11
// atomics when its camera changes, and at the end of its chunk the lanes of a
// warp merge their last runs (cameras are non-decreasing across lanes) with one
// segmented scan, whose last lane per camera adds the sum. Point cotangents go
// out per observation (points are in random order).
constexpr int kOpt = 8;

// Inclusive scan of v over runs of equal keys in lane order, 11 values at once
// (the run head is computed once).
__device__ __forceinline__ void seg_scan11(float (&v)[11], int key) {
    const int head = run_head(key);
#pragma unroll
    for (int i = 0; i < 11; ++i) v[i] = run_scan_head(v[i], head);
}

// VJP = false (with FUSED): the residual alone, in camera-sorted order.
// PORD: the per-observation arrays (w, tgt, res) are indexed by plan position
// (row i belongs to observation perm[i]) instead of by observation: they are
// read and written contiguously and the permutation is not read at all.
template <bool FUSED, bool VJP = true, bool PORD = false>
__global__ void __launch_bounds__(256) reproj_vjp_sorted_kernel(
    const float* __restrict__ rec, const float* __restrict__ pts, const float4* __restrict__ pts4,
    const float2* __restrict__ wv,
    const float2* __restrict__ tgt, float wscale, int n_cams, int n_pts, int64_t n_obs,
    const int32_t* __restrict__ perm, const int32_t* __restrict__ key_s, const int32_t* __restrict__ aux_s,
    float* __restrict__ d_cams, float* __restrict__ d_pts, float4* __restrict__ d_pts4, float2* __restrict__ res,
    int32_t* __restrict__ status, int pts8, int dpts8) {
    const int lane = threadIdx.x & 31;
    const int64_t chunk = (int64_t)blockDim.x * kOpt;
    // trip count is uniform over the block so that every lane reaches the shuffles
    for (int64_t base = (int64_t)blockIdx.x * chunk; base < n_obs; base += (int64_t)gridDim.x * chunk) {
        const int64_t pos0 = base + (int64_t)threadIdx.x * kOpt;
        int ev[kOpt], cv[kOpt], pv[kOpt];
        if (pos0 + kOpt <= n_obs) {  // plan arrays are 256-byte aligned, pos0 a multiple of 8
#pragma unroll
            for (int h = 0; h < kOpt / 4; ++h) {
                const int4 e4 = PORD ? make_int4(0, 0, 0, 0) : __ldg(reinterpret_cast<const int4*>(perm + pos0) + h);
                const int4 c4 = __ldg(reinterpret_cast<const int4*>(key_s + pos0) + h);
                const int4 p4 = __ldg(reinterpret_cast<const int4*>(aux_s + pos0) + h);
                ev[4 * h] = e4.x; ev[4 * h + 1] = e4.y; ev[4 * h + 2] = e4.z; ev[4 * h + 3] = e4.w;
                cv[4 * h] = c4.x; cv[4 * h + 1] = c4.y; cv[4 * h + 2] = c4.z; cv[4 * h + 3] = c4.w;
                pv[4 * h] = p4.x; pv[4 * h + 1] = p4.y; pv[4 * h + 2] = p4.z; pv[4 * h + 3] = p4.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < kOpt; ++i) {
                const bool in = pos0 + i < n_obs;
                ev[i] = !in ? -1 : PORD ? 0 : __ldg(perm + pos0 + i);
                cv[i] = in ? __ldg(key_s + pos0 + i) : -1;
                pv[i] = in ? __ldg(aux_s + pos0 + i) : -1;
            }
        }
        // the random gathers of every observation of the thread first (points,
        // cotangents or targets), so that they are in flight together
        float xq[kOpt][3];
        float2 wq[kOpt];
#pragma unroll
        for (int i = 0; i < kOpt; ++i) {
            const bool ok = pos0 + i < n_obs && ev[i] >= 0 && ev[i] < n_obs && pv[i] >= 0 && pv[i] < n_pts;
            xq[i][0] = xq[i][1] = xq[i][2] = 0.f;
            wq[i] = make_float2(0.f, 0.f);
            if (ok) {
                load_point_any(pts4, pts, pv[i], pts8, xq[i][0], xq[i][1], xq[i][2]);
                wq[i] = __ldg((FUSED ? tgt : wv) + (PORD ? pos0 + i : (int64_t)ev[i]));
            }
        }
        float gc[11];
#pragma unroll
        for (int i = 0; i < 11; ++i) gc[i] = 0.f;
        int cur = -1, rcam = -1;
        float rc[kCamRec];
#pragma unroll
        for (int i = 0; i < kOpt; ++i) {
            if (pos0 + i >= n_obs) break;
            const int ci = cv[i], pi = pv[i];
            const int64_t e = PORD ? pos0 + i : (int64_t)ev[i];  // row of the per-observation arrays
            const bool e_ok = e >= 0 && e < n_obs;
            if (!e_ok || ci < 0 || ci >= n_cams || pi < 0 || pi >= n_pts) {
                if (FUSED && e_ok) res[e] = make_float2(NAN, NAN);
                report(status, GPA_ERR_INDEX);
                continue;
            }
            if (VJP && ci != cur) {
                if (cur >= 0) {
                    float* dc = d_cams + (size_t)cur * 11;
#pragma unroll
                    for (int j = 0; j < 11; ++j) {
                        red_add(dc + j, gc[j]);
                        gc[j] = 0.f;
                    }
                }
                cur = ci;
            }
            if (ci != rcam) {
                load_cam<VJP ? kCamRec : kCamResid>(rec, ci, rc);
                rcam = ci;
            }
            const Proj P = project(rc, xq[i][0], xq[i][1], xq[i][2]);
            float w0, w1;
            if (FUSED) {
                const float2 t = wq[i];
                const float r0 = P.out[0] - t.x, r1 = P.out[1] - t.y;
                res[e] = make_float2(r0, r1);
                w0 = wscale * r0;
                w1 = wscale * r1;
            } else {
                w0 = wq[i].x;
                w1 = wq[i].y;
            }
            if constexpr (VJP) {
                float gl[11], gp[3];
                project_vjp(rc, P, w0, w1, gl, gp);
#pragma unroll
                for (int j = 0; j < 11; ++j) gc[j] += gl[j];
                if (d_pts4)
                    atomicAdd(d_pts4 + pi, make_float4(gp[0], gp[1], gp[2], 0.f));
                else
                    red_add_point(d_pts, pi, gp, dpts8);
            }
        }
        if constexpr (VJP) {
            const int ck = cur >= 0 ? cur : -1 - lane;
            seg_scan11(gc, ck);
            const bool last = run_end(ck);  // a shuffle: every lane evaluates it
            if (cur >= 0 && last) {
                float* dc = d_cams + (size_t)cur * 11;
#pragma unroll
                for (int j = 0; j < 11; ++j) red_add(dc + j, gc[j]);
            }
        }
    }
}

// Gauss-Newton normal equations (J = d res / d(cams, pts), rows from
// project_vjp with unit cotangents): per camera U += J_c^T J_c (66, upper
// triangle by rows) and g_cams += J_c^T r, per point V += J_p^T J_p (6) and
// g_pts += J_p^T r, per observation W = J_c^T J_p (33) and res. A thread takes
// kGnOpt consecutive observations (camera-sorted from a plan, or in input
// order), keeps its camera's 77 sums in registers while the camera repeats and
// adds them when it changes; the lanes of a warp merge their last runs with one
// segmented scan. The point's 9 sums go out as three 16-byte atomics into
// padded accumulators (pacc, [P][3] float4: V[0..5], g[0..2], pad).
constexpr int kGnOpt = 4;

template <bool SORTED>
__global__ void __launch_bounds__(128) reproj_gn_kernel(
    const float* __restrict__ rec, const float* __restrict__ pts, const int2* __restrict__ obs,
    const float2* __restrict__ tgt, int n_cams, int n_pts, int64_t n_obs, const int32_t* __restrict__ perm,
    const int32_t* __restrict__ key_s, const int32_t* __restrict__ aux_s, float* __restrict__ U,
    float* __restrict__ W, int w_ld, int w_plan, float* __restrict__ g_cams, float4* __restrict__ pacc,
    float2* __restrict__ res, int32_t* __restrict__ status, int pts8) {
    // w_plan (SORTED only): W row of the observation at plan position pos is
    // row pos, so a warp fills one contiguous range of rows over its kGnOpt
    // iterations; otherwise row e (input order)
    const int lane = threadIdx.x & 31;
    __shared__ float wstage[4 * 32 * 33];  // per warp: 32 rows of W, one per lane
    const int64_t chunk = (int64_t)blockDim.x * kGnOpt;
    for (int64_t base = (int64_t)blockIdx.x * chunk; base < n_obs; base += (int64_t)gridDim.x * chunk) {
        const int64_t pos0 = base + (int64_t)threadIdx.x * kGnOpt;
        int ev[kGnOpt], cv[kGnOpt], pv[kGnOpt];
#pragma unroll
        for (int i = 0; i < kGnOpt; ++i) {
            const int64_t pos = pos0 + i;
            if (pos >= n_obs) {
                ev[i] = cv[i] = pv[i] = -1;
            } else if (SORTED) {
                ev[i] = __ldg(perm + pos);
                cv[i] = __ldg(key_s + pos);
                pv[i] = __ldg(aux_s + pos);
            } else {
                const int2 o = __ldg(obs + pos);
                ev[i] = (int)pos;
                cv[i] = o.x;
                pv[i] = o.y;
            }
        }
        float ua[66], ga[11];
#pragma unroll
        for (int a = 0; a < 66; ++a) ua[a] = 0.f;
#pragma unroll
        for (int a = 0; a < 11; ++a) ga[a] = 0.f;
        int cur = -1, rcam = -1;
        float rc[kCamRec];
        float* stage = wstage + (threadIdx.x >> 5) * 32 * 33;  // this warp's W rows
#pragma unroll
        for (int i = 0; i < kGnOpt; ++i) {
            // no early exits: every lane reaches the warp's W store below
            const int e = ev[i], ci = cv[i], pi = pv[i];
            const bool active = pos0 + i < n_obs;
            const bool e_ok = active && e >= 0 && e < n_obs;
            const bool valid = e_ok && ci >= 0 && ci < n_cams && pi >= 0 && pi < n_pts;
            if (active && !valid) {
                if (e_ok && res) res[e] = make_float2(NAN, NAN);
                report(status, GPA_ERR_INDEX);
            }
            if (valid) {
                if (ci != cur) {
                    if (cur >= 0) {
#pragma unroll
                        for (int a = 0; a < 66; ++a) {
                            red_add(U + (size_t)cur * 66 + a, ua[a]);
                            ua[a] = 0.f;
                        }
#pragma unroll
                        for (int a = 0; a < 11; ++a) {
                            red_add(g_cams + (size_t)cur * 11 + a, ga[a]);
                            ga[a] = 0.f;
                        }
                    }
                    cur = ci;
                }
                if (ci != rcam) {
                    load_cam<kCamRec>(rec, ci, rc);
                    rcam = ci;
                }
                float X0, X1, X2;
                load_point(pts, pi, pts8, X0, X1, X2);
                const Proj P = project(rc, X0, X1, X2);
                const float2 t = __ldg(tgt + e);
                const float r0 = P.out[0] - t.x, r1 = P.out[1] - t.y;
                if (res) res[e] = make_float2(r0, r1);
                float j0c[11], j0p[3], j1c[11], j1p[3];
                project_vjp(rc, P, 1.f, 0.f, j0c, j0p);
                project_vjp(rc, P, 0.f, 1.f, j1c, j1p);
                int q = 0;
#pragma unroll
                for (int a = 0; a < 11; ++a) {
                    ga[a] = fmaf(j0c[a], r0, fmaf(j1c[a], r1, ga[a]));
#pragma unroll
                    for (int b = a; b < 11; ++b, ++q) ua[q] = fmaf(j0c[a], j0c[b], fmaf(j1c[a], j1c[b], ua[q]));
                }
                if (W) {
#pragma unroll
                    for (int a = 0; a < 11; ++a)
#pragma unroll
                        for (int b = 0; b < 3; ++b)
                            stage[lane * 33 + a * 3 + b] = fmaf(j0c[a], j0p[b], j1c[a] * j1p[b]);
                }
                float v[9];
                q = 0;
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = a; b < 3; ++b, ++q) v[q] = fmaf(j0p[a], j0p[b], j1p[a] * j1p[b]);
#pragma unroll
                for (int a = 0; a < 3; ++a) v[6 + a] = fmaf(j0p[a], r0, j1p[a] * r1);
                float4* pa = pacc + (size_t)pi * 3;
                atomicAdd(pa, make_float4(v[0], v[1], v[2], v[3]));
                atomicAdd(pa + 1, make_float4(v[4], v[5], v[6], v[7]));
                atomicAdd(pa + 2, make_float4(v[8], 0.f, 0.f, 0.f));
            }
            if (W) {
                // the warp writes its 32 rows, each as contiguous stores (NaN rows
                // for bad indices), padding columns 33 .. w_ld-1 as zeros: with
                // w_ld a multiple of 8 on a 32-byte aligned W every row is whole
                // 32-byte sectors, so rows landing in random order (camera-sorted
                // runs) never leave a sector partly written
                const bool by_pos = SORTED && w_plan;
                const int mode = valid ? 1 : ((by_pos ? active : e_ok) ? 2 : 0);
                const int wrow = by_pos ? (int)(pos0 + i) : e;
                __syncwarp();
                for (int rr = 0; rr < 32; ++rr) {
                    const int mr = __shfl_sync(0xffffffffu, mode, rr);
                    const int er = __shfl_sync(0xffffffffu, wrow, rr);
                    if (mr) {  // streaming stores: W passes through L2 once and should not evict
                               // the sectors of tgt and res that neighbouring observations reuse
                        float* Wr = W + (size_t)er * w_ld;
                        __stcs(Wr + lane, mr == 1 ? stage[rr * 33 + lane] : NAN);
                        const int c2 = 32 + lane;
                        if (c2 < w_ld) __stcs(Wr + c2, c2 == 32 ? (mr == 1 ? stage[rr * 33 + 32] : NAN) : 0.f);
                    }
                }
                __syncwarp();
            }
        }
        const int ck = cur >= 0 ? cur : -1 - lane;
        const int head = run_head(ck);
        const bool last = run_end(ck);  // shuffles: every lane evaluates them
#pragma unroll
        for (int a = 0; a < 66; ++a) ua[a] = run_scan_head(ua[a], head);
#pragma unroll
        for (int a = 0; a < 11; ++a) ga[a] = run_scan_head(ga[a], head);
        if (cur >= 0 && last) {
#pragma unroll
            for (int a = 0; a < 66; ++a) red_add(U + (size_t)cur * 66 + a, ua[a]);
#pragma unroll
            for (int a = 0; a < 11; ++a) red_add(g_cams + (size_t)cur * 11 + a, ga[a]);
        }
    }
}

// V[p] += pacc[p] (first 6), g_pts[p] += pacc[p] (next 3).
__global__ void __launch_bounds__(256) gn_points_add_kernel(const float4* __restrict__ pacc, int n_pts,
                                                            float* __restrict__ V, float* __restrict__ g_pts) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pts; p += stride) {
        const float4 a = pacc[3 * p], b = pacc[3 * p + 1], c = pacc[3 * p + 2];
        float* v = V + p * 6;
        v[0] += a.x; v[1] += a.y; v[2] += a.z; v[3] += a.w; v[4] += b.x; v[5] += b.y;
        float* g = g_pts + p * 3;
        g[0] += b.z; g[1] += b.w; g[2] += c.x;
    }
}

// d_pts[p] += acc[p].xyz (the padded accumulators of one VJP call).
__global__ void __launch_bounds__(256) pts4_add_kernel(const float4* __restrict__ acc, int n_pts,
                                                       float* __restrict__ d_pts) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pts; p += stride) {
        const float4 v = acc[p];
        float* dp = d_pts + p * 3;
        dp[0] += v.x;
        dp[1] += v.y;
        dp[2] += v.z;
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static int sm_count() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

static unsigned obs_grid(int64_t n_obs) {
    const int64_t want = (n_obs + 255) / 256;
    const int64_t cap = (int64_t)sm_count() * 8;
    return (unsigned)(want < cap ? want : cap);
}

static int expand_cams(const float* cams, int n_cams, float* rec, cudaStream_t s) {
    GPA_LAUNCH("cam_expand", s,
               cam_expand_kernel<<<(n_cams + kCamPerBlock - 1) / kCamPerBlock, kCamPerBlock, 0, s>>>(cams, n_cams,
                                                                                                       rec));
    return GPA_OK;
}

static bool al_dev(const void* p, uintptr_t a) { return (((uintptr_t)p) & (a - 1)) == 0; }

template <int STRAT, bool FUSED>
static int launch_vjp(const float* rec, const float* pts, const float4* pts4, const int32_t* obs, const float* w, const float* tgt,
                      float wscale, int n_cams, int n_pts, int64_t n_obs, const PlanView& pv, float* d_cams,
                      float* d_pts, float4* d_pts4, float* res, int32_t* status, cudaStream_t s) {
    GPA_LAUNCH(FUSED ? "reproj_residual_vjp" : "reproj_vjp", s,
               reproj_vjp_kernel<STRAT, FUSED><<<obs_grid(n_obs), 256, 0, s>>>(
                   rec, pts, pts4, (const int2*)obs, (const float2*)w, (const float2*)tgt, wscale, n_cams, n_pts,
                   n_obs, d_cams, d_pts, d_pts4, (float2*)res, status, al_dev(pts, 8) ? 1 : 0,
                   al_dev(d_pts, 8) ? 1 : 0));
    return GPA_OK;
}

template <bool FUSED>
static int launch_vjp_sorted(const float* rec, const float* pts, const float4* pts4, const float* w, const float* tgt, float wscale,
                             int n_cams, int n_pts, int64_t n_obs, const PlanView& pv, float* d_cams, float* d_pts,
                             float4* d_pts4, float* res, int32_t* status, cudaStream_t s, int obs_order = 0) {
    const int64_t want = (n_obs + 256 * kOpt - 1) / (256 * kOpt), cap = (int64_t)sm_count() * 8;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    if (obs_order)
        GPA_LAUNCH(FUSED ? "reproj_residual_vjp" : "reproj_vjp", s,
                   (reproj_vjp_sorted_kernel<FUSED, true, true><<<grid, 256, 0, s>>>(
                       rec, pts, pts4, (const float2*)w, (const float2*)tgt, wscale, n_cams, n_pts, n_obs, pv.perm,
                       pv.key_sorted, pv.aux_sorted, d_cams, d_pts, d_pts4, (float2*)res, status,
                       al_dev(pts, 8) ? 1 : 0, al_dev(d_pts, 8) ? 1 : 0)));
    else
        GPA_LAUNCH(FUSED ? "reproj_residual_vjp" : "reproj_vjp", s,
                   reproj_vjp_sorted_kernel<FUSED><<<grid, 256, 0, s>>>(
                       rec, pts, pts4, (const float2*)w, (const float2*)tgt, wscale, n_cams, n_pts, n_obs, pv.perm,
                       pv.key_sorted, pv.aux_sorted, d_cams, d_pts, d_pts4, (float2*)res, status,
                       al_dev(pts, 8) ? 1 : 0, al_dev(d_pts, 8) ? 1 : 0));
    return GPA_OK;
}

// pts4: the points in 16-byte rows; d_pts4: padded point accumulators, added
// into d_pts after the scatter. Both in the workspace, written by
// vjp_prep_kernel before this call.
template <bool FUSED>
static int dispatch_vjp(int strat, const float* rec, const float* pts, const float4* pts4, const int32_t* obs,
                        const float* w,
                        const float* tgt, float wscale, int n_cams, int n_pts, int64_t n_obs,
                        const PlanView& pv, float* d_cams, float* d_pts, float4* d_pts4, float* res,
                        int32_t* status, cudaStream_t s, int obs_order = 0) {
    int rc = GPA_ERR_ARG;
    switch (strat) {
        case GPA_SCATTER_ATOMIC:
            rc = launch_vjp<GPA_SCATTER_ATOMIC, FUSED>(rec, pts, pts4, obs, w, tgt, wscale, n_cams, n_pts, n_obs, pv,
                                                      d_cams, d_pts, d_pts4, res, status, s);
            break;
        case GPA_SCATTER_WARPAGG:
            rc = launch_vjp<GPA_SCATTER_WARPAGG, FUSED>(rec, pts, pts4, obs, w, tgt, wscale, n_cams, n_pts, n_obs, pv,
                                                       d_cams, d_pts, d_pts4, res, status, s);
            break;
        case GPA_SCATTER_SORT:
            rc = launch_vjp_sorted<FUSED>(rec, pts, pts4, w, tgt, wscale, n_cams, n_pts, n_obs, pv, d_cams, d_pts, d_pts4,
                                          res, status, s, obs_order);
            break;
    }
    if (rc || !d_pts4) return rc;
    const int64_t want = (n_pts + 255) / 256, cap = (int64_t)sm_count() * 8;
    GPA_LAUNCH("reproj_pts_add", s,
               pts4_add_kernel<<<(unsigned)(want < cap ? want : cap), 256, 0, s>>>(d_pts4, n_pts, d_pts));
    return GPA_OK;
}

}  // namespace gpa

using namespace gpa;

static bool al(const void* p, uintptr_t a) { return (((uintptr_t)p) & (a - 1)) == 0; }

// Workspace: expanded cameras, then the padded point accumulators of the VJP,
// then the points in 16-byte rows.
static size_t cam_area(int32_t n_cams) { return (sizeof(float) * (size_t)n_cams * kCamRec + 255) & ~(size_t)255; }
static size_t pt4_area(int32_t n_pts) { return (sizeof(float4) * (size_t)n_pts + 255) & ~(size_t)255; }

extern "C" size_t gpa_reproj_workspace_bytes(int32_t n_cams, int32_t n_pts, int64_t n_obs) {
    (void)n_obs;
    if (n_cams < 1 || n_pts < 1) return 0;
    return cam_area(n_cams) + 2 * pt4_area(n_pts);
}

static float4* pts_acc(void* ws, int32_t n_cams) { return (float4*)((char*)ws + cam_area(n_cams)); }
static float4* pts_pad(void* ws, int32_t n_cams, int32_t n_pts) {
    return (float4*)((char*)ws + cam_area(n_cams) + pt4_area(n_pts));
}

// Camera expansion, padded point copy and zeroed point accumulators in one launch.
static int vjp_prep(const float* cams, int n_cams, float* rec, const float* pts, int n_pts, float4* pts4,
                    float4* acc, cudaStream_t s) {
    const int ncb = (n_cams + kCamPerBlock - 1) / kCamPerBlock;
    const int64_t want = ((int64_t)n_pts + 127) / 128, cap = (int64_t)sm_count() * 16;
    const int npb = (int)(want < cap ? want : cap);
    GPA_LAUNCH("reproj_vjp_prep", s,
               vjp_prep_kernel<<<(unsigned)(ncb + npb), 128, 0, s>>>(cams, n_cams, rec, ncb, pts, n_pts, pts4, acc));
    return GPA_OK;
}

static int reproj_check(const float* cams, const float* pts, const int32_t* obs, int32_t n_cams,
                        int32_t n_pts, int64_t n_obs, void* ws, size_t ws_bytes) {
    if (!cams || !pts || !obs || !ws) return GPA_ERR_ARG;
    if (n_cams < 1 || n_pts < 1 || n_obs < 1 || n_obs > INT32_MAX) return GPA_ERR_ARG;
    if (!al(obs, 8) || !al(cams, 4) || !al(pts, 4) || !al(ws, 256)) return GPA_ERR_ALIGN;
    if (ws_bytes < gpa_reproj_workspace_bytes(n_cams, n_pts, n_obs)) return GPA_ERR_WORKSPACE;
    return GPA_OK;
}

extern "C" int reproj_residual(const float* cams, const float* pts, const int32_t* obs, const float* tgt,
                               int32_t n_cams, int32_t n_pts, int64_t n_obs, float* res, void* ws,
                               size_t ws_bytes, int32_t* dev_status, gpa_stream_t stream) {
    int rc = reproj_check(cams, pts, obs, n_cams, n_pts, n_obs, ws, ws_bytes);
    if (rc) return rc;
    if (!tgt || !res) return GPA_ERR_ARG;
    if (!al(tgt, 8) || !al(res, 8)) return GPA_ERR_ALIGN;
    cudaStream_t s = (cudaStream_t)stream;
    float* rec = (float*)ws;
    rc = expand_cams(cams, n_cams, rec, s);
    if (rc) return rc;
    GPA_LAUNCH("reproj_residual", s,
               reproj_residual_kernel<<<obs_grid(n_obs), 256, 0, s>>>(rec, pts, (const int2*)obs,
                                                                      (const float2*)tgt, n_cams, n_pts, n_obs,
                                                                      (float2*)res, dev_status, al(pts, 8) ? 1 : 0));
    return GPA_OK;
}

extern "C" int reproj_residual_sorted(const float* cams, const float* pts, const int32_t* obs, const float* tgt,
                                      int32_t n_cams, int32_t n_pts, int64_t n_obs, float* res, const void* plan,
                                      int32_t obs_order, void* ws, size_t ws_bytes, int32_t* dev_status,
                                      gpa_stream_t stream) {
    int rc = reproj_check(cams, pts, obs, n_cams, n_pts, n_obs, ws, ws_bytes);
    if (rc) return rc;
    if (!tgt || !res || !plan || (obs_order != 0 && obs_order != 1)) return GPA_ERR_ARG;
    if (!al(tgt, 8) || !al(res, 8)) return GPA_ERR_ALIGN;
    cudaStream_t s = (cudaStream_t)stream;
    float* rec = (float*)ws;
    float4* pts4 = pts_pad(ws, n_cams, n_pts);
    rc = vjp_prep(cams, n_cams, rec, pts, n_pts, pts4, nullptr, s);
    if (rc) return rc;
    const PlanView pv = plan_view(plan, n_obs, n_cams);
    const int64_t want = (n_obs + 256 * kOpt - 1) / (256 * kOpt), cap = (int64_t)sm_count() * 8;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    if (obs_order)
        GPA_LAUNCH("reproj_residual_sorted", s,
                   (reproj_vjp_sorted_kernel<true, false, true><<<grid, 256, 0, s>>>(
                       rec, pts, pts4, nullptr, (const float2*)tgt, 1.f, n_cams, n_pts, n_obs, pv.perm, pv.key_sorted,
                       pv.aux_sorted, nullptr, nullptr, nullptr, (float2*)res, dev_status, al_dev(pts, 8) ? 1 : 0, 0)));
    else
        GPA_LAUNCH("reproj_residual_sorted", s,
                   (reproj_vjp_sorted_kernel<true, false><<<grid, 256, 0, s>>>(
                       rec, pts, pts4, nullptr, (const float2*)tgt, 1.f, n_cams, n_pts, n_obs, pv.perm, pv.key_sorted,
                       pv.aux_sorted, nullptr, nullptr, nullptr, (float2*)res, dev_status, al_dev(pts, 8) ? 1 : 0, 0)));
    return GPA_OK;
}

static int resolve_strat(int strat, const void* plan) {
    if (strat == GPA_SCATTER_AUTO) return plan ? GPA_SCATTER_SORT : GPA_SCATTER_ATOMIC;
    return strat;
}

extern "C" int reproj_vjp(const float* cams, const float* pts, const int32_t* obs, const float* w,
                          int32_t n_cams, int32_t n_pts, int64_t n_obs, float* d_cams, float* d_pts,
                          int32_t strat, const void* plan, int32_t obs_order, void* ws, size_t ws_bytes,
                          int32_t* dev_status, gpa_stream_t stream) {
    int rc = reproj_check(cams, pts, obs, n_cams, n_pts, n_obs, ws, ws_bytes);
    if (rc) return rc;
    if (!w || !d_cams || !d_pts) return GPA_ERR_ARG;
    if (!al(w, 8)) return GPA_ERR_ALIGN;
    strat = resolve_strat(strat, plan);
    if (strat < GPA_SCATTER_ATOMIC || strat > GPA_SCATTER_SORT) return GPA_ERR_ARG;
    if (obs_order != 0 && (obs_order != 1 || strat != GPA_SCATTER_SORT)) return GPA_ERR_ARG;
    PlanView pv{};
    if (strat == GPA_SCATTER_SORT) {
        if (!plan) return GPA_ERR_ARG;
        pv = plan_view(plan, n_obs, n_cams);
    }
    cudaStream_t s = (cudaStream_t)stream;
    float* rec = (float*)ws;
    float4* acc = pts_acc(ws, n_cams);
    float4* pts4 = pts_pad(ws, n_cams, n_pts);
    rc = vjp_prep(cams, n_cams, rec, pts, n_pts, pts4, acc, s);
    if (rc) return rc;
    return dispatch_vjp<false>(strat, rec, pts, pts4, obs, w, nullptr, 1.f, n_cams, n_pts, n_obs, pv, d_cams, d_pts,
                               acc, nullptr, dev_status, s, obs_order);
}

extern "C" int reproj_jvp(const float* cams, const float* pts, const int32_t* obs, const float* v_cams,
                          const float* v_pts, int32_t n_cams, int32_t n_pts, int64_t n_obs, float* jv, void* ws,
                          size_t ws_bytes, int32_t* dev_status, gpa_stream_t stream) {
    int rc = reproj_check(cams, pts, obs, n_cams, n_pts, n_obs, ws, ws_bytes);
    if (rc) return rc;
    if (!v_cams || !v_pts || !jv) return GPA_ERR_ARG;
    if (!al(jv, 8) || !al(v_cams, 4) || !al(v_pts, 4)) return GPA_ERR_ALIGN;
    cudaStream_t s = (cudaStream_t)stream;
    float* rec = (float*)ws;
    rc = expand_cams(cams, n_cams, rec, s);
    if (rc) return rc;
    GPA_LAUNCH("reproj_jvp", s,
               reproj_jvp_kernel<<<obs_grid(n_obs), 256, 0, s>>>(rec, pts, (const int2*)obs, v_cams, v_pts, n_cams,
                                                                 n_pts, n_obs, (float2*)jv, dev_status,
                                                                 al(pts, 8) ? 1 : 0));
    return GPA_OK;
}

extern "C" int reproj_residual_vjp(const float* cams, const float* pts, const int32_t* obs, const float* tgt,
                                   int32_t n_cams, int32_t n_pts, int64_t n_obs, float wscale, float* res,
                                   float* d_cams, float* d_pts, int32_t strat, const void* plan, int32_t obs_order,
                                   void* ws, size_t ws_bytes, int32_t* dev_status, gpa_stream_t stream) {
    int rc = reproj_check(cams, pts, obs, n_cams, n_pts, n_obs, ws, ws_bytes);
    if (rc) return rc;
    if (!tgt || !res || !d_cams || !d_pts) return GPA_ERR_ARG;
    if (!al(tgt, 8) || !al(res, 8)) return GPA_ERR_ALIGN;
    strat = resolve_strat(strat, plan);
    if (strat < GPA_SCATTER_ATOMIC || strat > GPA_SCATTER_SORT) return GPA_ERR_ARG;
    if (obs_order != 0 && (obs_order != 1 || strat != GPA_SCATTER_SORT)) return GPA_ERR_ARG;
    PlanView pv{};
    if (strat == GPA_SCATTER_SORT) {
        if (!plan) return GPA_ERR_ARG;
        pv = plan_view(plan, n_obs, n_cams);
    }
    cudaStream_t s = (cudaStream_t)stream;
    float* rec = (float*)ws;
    float4* acc = pts_acc(ws, n_cams);
    float4* pts4 = pts_pad(ws, n_cams, n_pts);
    rc = vjp_prep(cams, n_cams, rec, pts, n_pts, pts4, acc, s);
    if (rc) return rc;
    return dispatch_vjp<true>(strat, rec, pts, pts4, obs, nullptr, tgt, wscale, n_cams, n_pts, n_obs, pv, d_cams,
                              d_pts, acc, res, dev_status, s, obs_order);
}

extern "C" size_t gpa_reproj_gn_workspace_bytes(int32_t n_cams, int32_t n_pts, int64_t n_obs) {
    (void)n_obs;
    if (n_cams < 1 || n_pts < 1) return 0;
    return cam_area(n_cams) + ((sizeof(float4) * 3 * (size_t)n_pts + 255) & ~(size_t)255);
}

extern "C" int reproj_normal_eqs(const float* cams, const float* pts, const int32_t* obs, const float* tgt,
                                 int32_t n_cams, int32_t n_pts, int64_t n_obs, float* U, float* V, float* W,
                                 int32_t w_ld, int32_t w_order, float* g_cams, float* g_pts, float* res,
                                 int32_t strat, const void* plan, void* ws, size_t ws_bytes, int32_t* dev_status,
                                 gpa_stream_t stream) {
    if (!cams || !pts || !obs || !tgt || !U || !V || !g_cams || !g_pts || !ws) return GPA_ERR_ARG;
    if (W && (w_ld < 33 || w_ld > 64)) return GPA_ERR_ARG;
    if (w_order != 0 && w_order != 1) return GPA_ERR_ARG;
    if (n_cams < 1 || n_pts < 1 || n_obs < 1 || n_obs > INT32_MAX) return GPA_ERR_ARG;
    if (!al(obs, 8) || !al(tgt, 8) || (res && !al(res, 8)) || !al(ws, 256)) return GPA_ERR_ALIGN;
    if (!al(cams, 4) || !al(pts, 4) || !al(U, 4) || !al(V, 4) || (W && !al(W, 4)) || !al(g_cams, 4) ||
        !al(g_pts, 4))
        return GPA_ERR_ALIGN;
    if (ws_bytes < gpa_reproj_gn_workspace_bytes(n_cams, n_pts, n_obs)) return GPA_ERR_WORKSPACE;
    strat = resolve_strat(strat, plan);
    if (strat != GPA_SCATTER_ATOMIC && strat != GPA_SCATTER_SORT) return GPA_ERR_UNSUPPORTED;
    if (w_order == 1 && strat != GPA_SCATTER_SORT) return GPA_ERR_ARG;  // plan order needs the plan
    PlanView pv{};
    if (strat == GPA_SCATTER_SORT) {
        if (!plan) return GPA_ERR_ARG;
        pv = plan_view(plan, n_obs, n_cams);
    }
    cudaStream_t s = (cudaStream_t)stream;
    float* rec = (float*)ws;
    float4* pacc = pts_acc(ws, n_cams);
    int rc = expand_cams(cams, n_cams, rec, s);
    if (rc) return rc;
    if (cudaMemsetAsync(pacc, 0, sizeof(float4) * 3 * (size_t)n_pts, s) != cudaSuccess) return GPA_ERR_CUDA;
    const int64_t want = (n_obs + 128 * kGnOpt - 1) / (128 * kGnOpt), cap = (int64_t)sm_count() * 12;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    const int p8 = al(pts, 8) ? 1 : 0;
    if (strat == GPA_SCATTER_SORT)
        GPA_LAUNCH("reproj_normal_eqs", s,
                   reproj_gn_kernel<true><<<grid, 128, 0, s>>>(rec, pts, (const int2*)obs, (const float2*)tgt,
                                                               n_cams, n_pts, n_obs, pv.perm, pv.key_sorted,
                                                               pv.aux_sorted, U, W, w_ld, w_order, g_cams, pacc,
                                                               (float2*)res, dev_status, p8));
    else
        GPA_LAUNCH("reproj_normal_eqs", s,
                   reproj_gn_kernel<false><<<grid, 128, 0, s>>>(rec, pts, (const int2*)obs, (const float2*)tgt,
                                                                n_cams, n_pts, n_obs, nullptr, nullptr, nullptr, U,
                                                                W, w_ld, 0, g_cams, pacc, (float2*)res, dev_status,
                                                                p8));
    const int64_t pw = (n_pts + 255) / 256, pc = (int64_t)sm_count() * 8;
    GPA_LAUNCH("reproj_gn_points", s,
               gn_points_add_kernel<<<(unsigned)(pw < pc ? pw : pc), 256, 0, s>>>(pacc, n_pts, V, g_pts));
    return GPA_OK;
}

// ---------------------------------------------------------------------------
// reproj_vjp_noalloc: reproj_vjp whose only scratch (the expanded cameras) lives
// in a fixed array in device memory that the library owns, for callers that
// cannot hand the library a workspace.
// ---------------------------------------------------------------------------
namespace gpa {
// Largest camera count the built-in scratch holds (32 floats per camera,
// 2 MiB per GPU that loads the library, kept until the process exits).
constexpr int kNoAllocMaxCams = GPA_NOALLOC_MAX_CAMS;
static_assert(kNoAllocMaxCams * kCamRec * sizeof(float) == (2u << 20), "scratch size stated in gpa.h");
static __device__ __align__(256) float g_cam_scratch[kNoAllocMaxCams * kCamRec];

// Device address of g_cam_scratch in the current device's context. In host
// code the array's name only stands in for the symbol, so its address has to be
// looked up, with the device current. The lookup is repeated on every call (a
// host-side table lookup once the module is loaded): an address cached per
// device ordinal would go stale after cudaDeviceReset or in another context of
// the same device, where the module is loaded again at another address.
static int cam_scratch_address(float** out) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_cam_scratch) != cudaSuccess || p == nullptr) {
        (void)cudaGetLastError();
        return GPA_ERR_CUDA;
    }
    *out = static_cast<float*>(p);
    return GPA_OK;
}
}  // namespace gpa

extern "C" int reproj_vjp_noalloc(const float* cams, const float* pts, const int32_t* obs, const float* w,
                                  int32_t n_cams, int32_t n_pts, int64_t n_obs, float* d_cams, float* d_pts,
                                  int32_t strat, const void* plan, int32_t* dev_status, gpa_stream_t stream) {
    if (!cams || !pts || !obs || !w || !d_cams || !d_pts) return GPA_ERR_ARG;
    if (n_cams < 1 || n_pts < 1 || n_obs < 1 || n_obs > INT32_MAX) return GPA_ERR_ARG;
    if (n_cams > kNoAllocMaxCams) return GPA_ERR_WORKSPACE;  // more cameras than the built-in scratch holds
    if (!al(obs, 8) || !al(w, 8) || !al(cams, 4) || !al(pts, 4)) return GPA_ERR_ALIGN;
    strat = resolve_strat(strat, plan);
    if (strat < GPA_SCATTER_ATOMIC || strat > GPA_SCATTER_SORT) return GPA_ERR_ARG;
    PlanView pv{};
    if (strat == GPA_SCATTER_SORT) {
        if (!plan) return GPA_ERR_ARG;
        pv = plan_view(plan, n_obs, n_cams);
    }
    float* rec = nullptr;
    int rc = cam_scratch_address(&rec);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // every record the VJP reads is rewritten here first: nothing needs clearing
    rc = expand_cams(cams, n_cams, rec, s);
    if (rc) return rc;
    // no 16-byte point rows and no padded accumulators (they would need scratch
    // per point): the kernels gather the points directly and add into d_pts
    return dispatch_vjp<false>(strat, rec, pts, nullptr, obs, w, nullptr, 1.f, n_cams, n_pts, n_obs, pv, d_cams, d_pts,
                               nullptr, nullptr, dev_status, s);
}
