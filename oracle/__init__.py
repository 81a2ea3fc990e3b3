"""FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Thin ctypes wrappers around ``oracle.c`` (plain C, double precision, OpenMP
partitions for Accum-style sums). Only the tests, ``__graft_entry__.smoke()``
and the benchmark's CPU-baseline leg may import this package. It shares no code
with the CUDA library and never calls it.

Pins (what each function is checked against in ``tests/test_oracle_*.py``):
  gmm_objective  scipy multivariate-normal and Wishart log-densities, mixture
                 log-likelihood via scipy logsumexp, diagonal closed form
  gmm_grad       central finite differences of gmm_objective; jvp dot test
  gmm_jvp        central finite differences along random directions
  reproj_*       scipy Rotation for the rotation, a hand-worked projection,
                 central differences of the Jacobian, identity camera,
                 small-angle continuity, dot-product test <Jv, w> = <v, J^T w>
  scatter_add_*  numpy bincount / add.at, brute-force tiny histograms
  stable_sort    numpy argsort(kind="stable")
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-std=gnu11"]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
            f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
            i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
            i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
            vp = C.c_void_p
            I64, I32, D = C.c_int64, C.c_int, C.c_double
            lib.oracle_num_threads.restype = C.c_int
            lib.oracle_gmm_objective.argtypes = [f32p] * 5 + [I64, I32, I32, D, I32, vp]
            lib.oracle_gmm_objective.restype = D
            lib.oracle_gmm_logjoint_at.argtypes = [f32p] * 5 + [I32, I32, i64p, I64, vp, f64p]
            lib.oracle_gmm_grad.argtypes = [f32p] * 5 + [I64, I32, I32, D, I32, D] + [f64p] * 4
            lib.oracle_gmm_accum.argtypes = [f32p] * 5 + [I64, I32, I32, D] + [f64p] * 3
            lib.oracle_gmm_accum.restype = D
            lib.oracle_gmm_finish.argtypes = [f32p] * 3 + [I64, I32, I32, D, I32, D] + [f64p] * 3 + [D] + \
                [f64p] * 4
            lib.oracle_gmm_finish.restype = D
            lib.oracle_gmm_grad.restype = D
            lib.oracle_gmm_jvp.argtypes = [f32p] * 5 + [I64, I32, I32, D, I32] + [f64p] * 4 + [vp, vp]
            lib.oracle_gmm_jvp.restype = D
            lib.oracle_reproj_residual.argtypes = [f32p, f32p, i32p, f32p, I32, I32, I64, f64p]
            lib.oracle_reproj_residual.restype = I64
            lib.oracle_reproj_vjp.argtypes = [f32p, f32p, i32p, f32p, I32, I32, I64, f64p, f64p]
            lib.oracle_reproj_vjp.restype = I64
            lib.oracle_reproj_jvp.argtypes = [f32p, f32p, i32p, I32, I32, I64, f64p, f64p, f64p]
            lib.oracle_reproj_jvp.restype = I64
            lib.oracle_reproj_jacobian.argtypes = [f32p, f32p, i32p, I64, f64p]
            lib.oracle_reproj_normal_eqs.argtypes = [f32p, f32p, i32p, f32p, I32, I32, I64] + [vp] * 6
            lib.oracle_reproj_normal_eqs.restype = I64
            lib.oracle_scatter_add_f64.argtypes = [i32p, f32p, I64, I32, I32, f64p]
            lib.oracle_scatter_add_f64.restype = I64
            lib.oracle_scatter_add_i64.argtypes = [i32p, i32p, I64, I32, I32, i64p]
            lib.oracle_scatter_add_i64.restype = I64
            lib.oracle_stable_sort_by_key.argtypes = [i32p, I64, I32, i32p, i64p]
            lib.oracle_stable_sort_by_key.restype = I64
            _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _gmm_args(g):
    return (_c(g.x, np.float32), _c(g.alpha, np.float32), _c(g.mu, np.float32),
            _c(g.q, np.float32), _c(g.l, np.float32))


def gmm_objective(g, want_lse: bool = False):
    """f and (optionally) lse_i for a ``synth.GMMInputs``."""
    lib = _load()
    lse = np.empty(g.n, np.float64) if want_lse else None
    f = lib.oracle_gmm_objective(*_gmm_args(g), g.n, g.d, g.k, g.gamma, g.m,
                                 lse.ctypes.data if want_lse else None)
    return (f, lse) if want_lse else f


def gmm_logjoint_at(g, idx):
    """(s[idx, :], lse[idx]) for a list of point indices."""
    lib = _load()
    idx = _c(idx, np.int64)
    s = np.empty((idx.size, g.k), np.float64)
    lse = np.empty(idx.size, np.float64)
    lib.oracle_gmm_logjoint_at(*_gmm_args(g), g.d, g.k, idx, idx.size, s.ctypes.data, lse)
    return s, lse


def gmm_grad(g, seed: float = 1.0):
    """(f, d_alpha, d_mu, d_q, d_l): seed times the gradient of f."""
    lib = _load()
    t = g.d * (g.d - 1) // 2
    da = np.empty(g.k); dm = np.empty((g.k, g.d)); dq = np.empty((g.k, g.d)); dl = np.empty((g.k, t))
    f = lib.oracle_gmm_grad(*_gmm_args(g), g.n, g.d, g.k, g.gamma, g.m, float(seed), da, dm, dq, dl)
    return f, da, dm, dq, dl


def gmm_accum(g, seed: float = 1.0):
    """Accum sums of the gradient over the points of g, packed into one float64
    vector [A (K) | MU (K*D) | QB (K*D*D) | sum of logsumexp]: additive over any
    partition of the points."""
    lib = _load()
    a = np.empty(g.k); mu = np.empty((g.k, g.d)); qb = np.empty((g.k, g.d, g.d))
    sl = lib.oracle_gmm_accum(*_gmm_args(g), g.n, g.d, g.k, float(seed), a, mu, qb)
    return np.concatenate([a, mu.ravel(), qb.ravel(), [sl]])


def gmm_finish(g, n_total: int, sums, seed: float = 1.0):
    """(f, d_alpha, d_mu, d_q, d_l) from Accum sums (gmm_accum's layout) over
    n_total points; only the parameters of g are read."""
    lib = _load()
    k, d = g.k, g.d
    t = d * (d - 1) // 2
    sums = np.ascontiguousarray(sums, np.float64)
    a = sums[:k].copy(); mu = sums[k:k + k * d].copy(); qb = sums[k + k * d:k + k * d + k * d * d].copy()
    da = np.empty(k); dm = np.empty((k, d)); dq = np.empty((k, d)); dl = np.empty((k, t))
    f = lib.oracle_gmm_finish(_c(g.alpha, np.float32), _c(g.q, np.float32), _c(g.l, np.float32), int(n_total), d, k,
                              g.gamma, g.m, float(seed), a, mu, qb, float(sums[-1]), da, dm, dq, dl)
    return f, da, dm, dq, dl


def gmm_jvp(g, va, vm, vq, vl, want_lse_dot: bool = False):
    """(df[v], f), and the per-point tangent of logsumexp_k s_ik when asked."""
    lib = _load()
    fo = C.c_double()
    ld = np.empty(g.n, np.float64) if want_lse_dot else None
    df = lib.oracle_gmm_jvp(*_gmm_args(g), g.n, g.d, g.k, g.gamma, g.m, _c(va, np.float64),
                            _c(vm, np.float64), _c(vq, np.float64), _c(vl, np.float64),
                            C.addressof(fo), None if ld is None else ld.ctypes.data)
    return (df, fo.value, ld) if want_lse_dot else (df, fo.value)


def reproj_residual(r):
    lib = _load()
    res = np.empty((r.n_obs, 2), np.float64)
    bad = lib.oracle_reproj_residual(_c(r.cams, np.float32), _c(r.pts, np.float32),
                                     _c(r.obs, np.int32), _c(r.tgt, np.float32), r.n_cams,
                                     r.n_pts, r.n_obs, res)
    return res, int(bad)


def reproj_vjp(r, w=None):
    lib = _load()
    w = r.w if w is None else w
    dcm = np.empty((r.n_cams, 11), np.float64)
    dpt = np.empty((r.n_pts, 3), np.float64)
    bad = lib.oracle_reproj_vjp(_c(r.cams, np.float32), _c(r.pts, np.float32), _c(r.obs, np.int32),
                                _c(w, np.float32), r.n_cams, r.n_pts, r.n_obs, dcm, dpt)
    return dcm, dpt, int(bad)


def reproj_jvp(r, v_cams, v_pts):
    lib = _load()
    jv = np.empty((r.n_obs, 2), np.float64)
    bad = lib.oracle_reproj_jvp(_c(r.cams, np.float32), _c(r.pts, np.float32), _c(r.obs, np.int32),
                                r.n_cams, r.n_pts, r.n_obs, _c(v_cams, np.float64),
                                _c(v_pts, np.float64), jv)
    return jv, int(bad)


def reproj_jacobian(r):
    lib = _load()
    jac = np.empty((r.n_obs, 2, 14), np.float64)
    lib.oracle_reproj_jacobian(_c(r.cams, np.float32), _c(r.pts, np.float32), _c(r.obs, np.int32),
                               r.n_obs, jac)
    return jac


def reproj_normal_eqs(r, want_w: bool = True):
    """Gauss-Newton blocks (U [C][66], V [P][6], W [M][33] or None, g_cams [C][11],
    g_pts [P][3], res [M][2], skipped count); U and V are upper triangles packed
    by rows."""
    lib = _load()
    U = np.empty((r.n_cams, 66)); V = np.empty((r.n_pts, 6))
    W = np.empty((r.n_obs, 33)) if want_w else None
    gc = np.empty((r.n_cams, 11)); gp = np.empty((r.n_pts, 3)); res = np.empty((r.n_obs, 2))
    bad = lib.oracle_reproj_normal_eqs(_c(r.cams, np.float32), _c(r.pts, np.float32), _c(r.obs, np.int32),
                                       _c(r.tgt, np.float32), r.n_cams, r.n_pts, r.n_obs, U.ctypes.data,
                                       V.ctypes.data, None if W is None else W.ctypes.data, gc.ctypes.data,
                                       gp.ctypes.data, res.ctypes.data)
    return U, V, W, gc, gp, res, int(bad)


def scatter_add(idx, vals, n_buckets: int):
    """acc (float64 for float32 values, int64 for int32 values) and the skipped count."""
    lib = _load()
    idx = _c(idx, np.int32)
    m = idx.shape[0]
    w = 1 if vals.ndim == 1 else vals.shape[1]
    if vals.dtype == np.float32:
        acc = np.empty((n_buckets, w), np.float64)
        bad = lib.oracle_scatter_add_f64(idx, _c(vals, np.float32), m, w, n_buckets, acc)
    elif vals.dtype == np.int32:
        acc = np.empty((n_buckets, w), np.int64)
        bad = lib.oracle_scatter_add_i64(idx, _c(vals, np.int32), m, w, n_buckets, acc)
    else:
        raise TypeError(vals.dtype)
    return acc, int(bad)


def stable_sort_by_key(keys, n_keys: int):
    """(perm, seg_off, n_bad) of a stable counting sort by key."""
    lib = _load()
    keys = _c(keys, np.int32)
    perm = np.full(keys.shape[0], -1, np.int32)
    seg = np.empty(n_keys + 1, np.int64)
    bad = lib.oracle_stable_sort_by_key(keys, keys.shape[0], n_keys, perm, seg)
    return perm[: seg[-1]], seg, int(bad)
