"""Seeded synthetic inputs for the two programs and the Accum scatter.

This module only draws random numbers. It holds none of the arithmetic of the
method: no objective, no projection, no derivative. Both the FP64 oracle and the
CUDA path take their inputs from here, so the two sides see bit-identical
float32 / int32 arrays.

Every array comes from its own numpy ``Generator`` seeded with
``SeedSequence([seed, stream_id])``, so adding an array never changes another.

Workloads (value distributions as the benchmark configurations state them):

* GMM: x ~ N(0,1), means ~ N(0,1), log-weights ~ N(0,1), log-diagonal of the
  inverse-Cholesky factor ~ U(-0.5, 0.5), strict-lower entries ~ N(0, 0.1^2),
  Wishart gamma = 1, m = 0.
* Reprojection: camera = [rotation(3) ~ N(0,0.1^2), centre(3) ~ N(0,1),
  focal ~ U(500,1500), principal point(2) ~ N(0,1), radial(2) ~ N(0,(1e-3)^2)];
  points ~ N(0,1) + (0,0,5); observations uniform-random (camera, point) int32
  pairs; targets ~ N(0,1); cotangents w ~ N(0,1).
* Batched GMM: N log-uniform in [1e3, 2e5], D uniform over {8,16,32,64},
  K log-uniform in [4,128]; integers drawn as round(exp(U(ln a, ln b))) clamped.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

CAM_PARAMS = 11  # [rot(3), centre(3), focal, principal point(2), radial(2)]

# stream ids: one per array so that arrays are independent of each other
_S_X, _S_ALPHA, _S_MU, _S_Q, _S_L = 1, 2, 3, 4, 5
_S_ROT, _S_CEN, _S_F, _S_PP, _S_K, _S_PTS, _S_OBS_C, _S_OBS_P, _S_TGT, _S_W = range(10, 20)
_S_IDX, _S_VALS = 30, 31
_S_TAN = 40
_S_BATCH = 50


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([int(seed) & 0xFFFFFFFF, stream]))


@dataclass
class GMMInputs:
    x: np.ndarray       # (N, D) float32, row-major
    alpha: np.ndarray   # (K,) float32 log-weights
    mu: np.ndarray      # (K, D) float32 means
    q: np.ndarray       # (K, D) float32 log-diagonal of the inverse-Cholesky factor
    l: np.ndarray       # (K, D(D-1)/2) float32 strict-lower entries, row-major packing
    gamma: float = 1.0
    m: int = 0

    @property
    def n(self) -> int:
        return self.x.shape[0]

    @property
    def d(self) -> int:
        return self.x.shape[1]

    @property
    def k(self) -> int:
        return self.alpha.shape[0]


def gmm_inputs(n: int, d: int, k: int, seed: int = 0, gamma: float = 1.0, m: int = 0) -> GMMInputs:
    """The GMM workload: shapes (N, D, K) with the configuration's distributions."""
    t = d * (d - 1) // 2
    x = _rng(seed, _S_X).standard_normal((n, d), dtype=np.float32)
    alpha = _rng(seed, _S_ALPHA).standard_normal(k).astype(np.float32)
    mu = _rng(seed, _S_MU).standard_normal((k, d)).astype(np.float32)
    q = _rng(seed, _S_Q).uniform(-0.5, 0.5, (k, d)).astype(np.float32)
    l = (0.1 * _rng(seed, _S_L).standard_normal((k, t))).astype(np.float32)
    return GMMInputs(np.ascontiguousarray(x), alpha, mu, q, l, float(gamma), int(m))


def gmm_tangents(d: int, k: int, seed: int = 0):
    """Random tangent / cotangent directions for (alpha, mu, q, l): float64."""
    r = _rng(seed, _S_TAN)
    t = d * (d - 1) // 2
    return (r.standard_normal(k), r.standard_normal((k, d)), r.standard_normal((k, d)),
            r.standard_normal((k, t)))


@dataclass
class ReprojInputs:
    cams: np.ndarray   # (C, 11) float32
    pts: np.ndarray    # (P, 3) float32
    obs: np.ndarray    # (M, 2) int32 (camera, point)
    tgt: np.ndarray    # (M, 2) float32
    w: np.ndarray      # (M, 2) float32 cotangent of the residual

    @property
    def n_cams(self) -> int:
        return self.cams.shape[0]

    @property
    def n_pts(self) -> int:
        return self.pts.shape[0]

    @property
    def n_obs(self) -> int:
        return self.obs.shape[0]


def reproj_inputs(n_cams: int, n_pts: int, n_obs: int, seed: int = 0) -> ReprojInputs:
    """The bundle-adjustment workload with the configuration's distributions."""
    cams = np.empty((n_cams, CAM_PARAMS), np.float32)
    cams[:, 0:3] = 0.1 * _rng(seed, _S_ROT).standard_normal((n_cams, 3))
    cams[:, 3:6] = _rng(seed, _S_CEN).standard_normal((n_cams, 3))
    cams[:, 6] = _rng(seed, _S_F).uniform(500.0, 1500.0, n_cams)
    cams[:, 7:9] = _rng(seed, _S_PP).standard_normal((n_cams, 2))
    cams[:, 9:11] = 1e-3 * _rng(seed, _S_K).standard_normal((n_cams, 2))
    pts = _rng(seed, _S_PTS).standard_normal((n_pts, 3)).astype(np.float32)
    pts[:, 2] += np.float32(5.0)
    obs = np.empty((n_obs, 2), np.int32)
    obs[:, 0] = _rng(seed, _S_OBS_C).integers(0, n_cams, n_obs, dtype=np.int32)
    obs[:, 1] = _rng(seed, _S_OBS_P).integers(0, n_pts, n_obs, dtype=np.int32)
    tgt = _rng(seed, _S_TGT).standard_normal((n_obs, 2), dtype=np.float32)
    w = _rng(seed, _S_W).standard_normal((n_obs, 2), dtype=np.float32)
    return ReprojInputs(cams, pts, obs, tgt, w)


def reproj_tangents(n_cams: int, n_pts: int, seed: int = 0):
    """Random tangent directions (float64) for cameras and points."""
    r = _rng(seed, _S_TAN)
    return r.standard_normal((n_cams, CAM_PARAMS)), r.standard_normal((n_pts, 3))


def scatter_inputs(m: int, w: int, n_buckets: int, dtype: str = "f32", seed: int = 0,
                   skew: float = 0.0):
    """Indices and values for acc[idx[j], :] += vals[j, :].

    ``skew`` > 0 draws bucket ids from a Zipf-like law (heavy contention on a few
    buckets); 0 draws them uniformly.
    """
    r = _rng(seed, _S_IDX)
    if skew > 0.0:
        ranks = np.arange(1, n_buckets + 1, dtype=np.float64)
        p = ranks ** (-skew)
        p /= p.sum()
        idx = r.choice(n_buckets, size=m, p=p).astype(np.int32)
    else:
        idx = r.integers(0, n_buckets, m, dtype=np.int32)
    rv = _rng(seed, _S_VALS)
    if dtype == "f32":
        vals = rv.standard_normal((m, w), dtype=np.float32)
    elif dtype == "i32":
        vals = rv.integers(-1000, 1000, (m, w), dtype=np.int32)
    else:
        raise ValueError(dtype)
    return idx, vals


def _log_uniform_int(r: np.random.Generator, a: int, b: int, size: int) -> np.ndarray:
    v = np.rint(np.exp(r.uniform(math.log(a), math.log(b), size)))
    return np.clip(v, a, b).astype(np.int64)


def batched_shapes(n_inst: int = 512, seed: int = 0, n_range=(1000, 200000),
                   d_set=(8, 16, 32, 64), k_range=(4, 128)):
    """(N, D, K) per instance for the batched workload."""
    r = _rng(seed, _S_BATCH)
    ns = _log_uniform_int(r, n_range[0], n_range[1], n_inst)
    ds = r.choice(np.asarray(d_set, np.int64), n_inst)
    ks = _log_uniform_int(r, k_range[0], k_range[1], n_inst)
    return [(int(n), int(d), int(k)) for n, d, k in zip(ns, ds, ks)]


def batched_inputs(shapes, seed: int = 0):
    """One GMMInputs per instance; instance i is seeded with seed ^ (i + 1) << 16."""
    return [gmm_inputs(n, d, k, seed=(seed ^ ((i + 1) << 16))) for i, (n, d, k) in enumerate(shapes)]
