"""Central differences of the FP64 oracle objective on sampled gradient
coordinates at full size (test helper; calls only the oracle).

A coordinate of component k (alpha_k, mu_k, q_k, l_k) moves only column k of
the log-joint s_ik, so f(theta + h e_j) - f(theta) needs no full pass:
  sum_i logsumexp_j s'_ij - sum_i lse_i = sum_i log1p(p_ik expm1(s'_ik - s_ik)),
with p_ik = exp(s_ik - lse_i) from the oracle's exact lse, while the terms
-N logsumexp(alpha) and the Wishart prior change in closed form. Each
difference therefore costs three recomputations of one column (O(N D^2)).
The steps are taken in float32 (the parameters' type) and the quotient
divides by the steps actually taken.
"""
import dataclasses

import numpy as np
from scipy.special import logsumexp

import oracle

BLOCKS = ("alpha", "mu", "q", "l")
STEPS = {"alpha": 2.0 ** -10, "mu": 2.0 ** -10, "q": 2.0 ** -10, "l": 2.0 ** -12}


def fd_coordinates(g, lse_ref, grads, per_block=16, seed=64):
    """Compare grads (alpha, mu, q, l; float64 arrays) with central differences
    of the oracle objective on `per_block` random coordinates per block.
    Returns a list of (block, k, j, got, fd, err) with
    err = |got - fd| / max(|fd|, rms of the block)."""
    every = np.arange(g.n, dtype=np.int64)
    n, gam2 = float(g.n), g.gamma ** 2
    t = g.d * (g.d - 1) // 2

    def column(al, m_, q_, l_):
        g1 = dataclasses.replace(g, alpha=np.array([al], np.float32), mu=m_[None].copy(), q=q_[None].copy(),
                                 l=l_[None].copy())
        return oracle.gmm_logjoint_at(g1, every)[0][:, 0]

    rng = np.random.default_rng(seed)
    out = []
    for block in BLOCKS:
        h = STEPS[block]
        gb = grads[BLOCKS.index(block)]
        rms = float(np.sqrt(np.mean(np.asarray(gb, np.float64) ** 2)))
        for _ in range(per_block):
            k = int(rng.integers(g.k))
            j = int(rng.integers({"alpha": 1, "mu": g.d, "q": g.d, "l": t}[block]))
            base = {"alpha": g.alpha[k:k + 1].copy(), "mu": g.mu[k].copy(), "q": g.q[k].copy(), "l": g.l[k].copy()}
            s0 = column(base["alpha"][0], base["mu"], base["q"], base["l"])
            p = np.exp(s0 - lse_ref)
            d = {}
            for sign in (1, -1):
                pv = {b: v.copy() for b, v in base.items()}
                pv[block][j] = np.float32(np.float64(base[block][j]) + sign * h)
                s1 = column(pv["alpha"][0], pv["mu"], pv["q"], pv["l"])
                dll = float(np.sum(np.log1p(p * np.expm1(s1 - s0))))
                if block == "alpha":
                    al1 = g.alpha.astype(np.float64).copy()
                    al1[k] = pv["alpha"][0]
                    dll -= n * (logsumexp(al1) - logsumexp(g.alpha.astype(np.float64)))
                elif block == "q":
                    q0, q1 = np.float64(base["q"][j]), np.float64(pv["q"][j])
                    dll += g.m * (q1 - q0) - 0.5 * gam2 * (np.exp(2 * q1) - np.exp(2 * q0))
                elif block == "l":
                    l0, l1 = np.float64(base["l"][j]), np.float64(pv["l"][j])
                    dll -= 0.5 * gam2 * (l1 * l1 - l0 * l0)
                d[sign] = (dll, np.float64(pv[block][j]))
            fd = (d[1][0] - d[-1][0]) / (d[1][1] - d[-1][1])
            got = float(gb[k] if block == "alpha" else gb[k, j])
            out.append((block, k, j, got, float(fd), abs(got - fd) / max(abs(fd), rms)))
    return out


def per_block_errors(rows):
    """Per block: the worst coordinate error and the normwise error of the
    sampled coordinates, ||got - fd|| / ||fd||."""
    res = {}
    for block in BLOCKS:
        r = [x for x in rows if x[0] == block]
        got = np.array([x[3] for x in r])
        fd = np.array([x[4] for x in r])
        res[block] = {"max": max(x[5] for x in r),
                      "normwise": float(np.linalg.norm(got - fd) / max(np.linalg.norm(fd), 1e-300))}
    return res
