"""Seeded synthetic inputs for the exact ddKS path.

This module only draws numbers: it holds none of the statistic's arithmetic,
so both the CUDA path and the CPU oracle can take their inputs from it.  All
draws use numpy's PCG64 (``np.random.default_rng(seed)``); the arrays it
returns are the authoritative bytes (float32 inputs are drawn in float64 and
cast once).

The shapes and distributions stand in for the paper's synthetic datasets
(Sec. 4.1: Gaussian samples, Gaussian mixtures, uniform/Beta marginals); no
dataset item of the paper is reproduced.
"""
from __future__ import annotations

import math

import numpy as np


def gaussian_pair(seed=0, n_p=200, n_t=200, d=3, shift=0.2, dtype=np.float32):
    """P ~ N(0, I_d), T ~ N(shift * 1, I_d) from one generator (P drawn first)."""
    rng = np.random.default_rng(seed)
    P = rng.standard_normal((n_p, d))
    T = rng.standard_normal((n_t, d)) + shift
    return P.astype(dtype), T.astype(dtype)


def correlated_pair_with_ties(seed=0, n_p=20000, n_t=20000, d=4, rho=0.5, dup_frac=0.01,
                              dtype=np.float32):
    """P ~ N(0, I_d); T has standard normal marginals with corr(x0, x1) = rho.

    Then round(dup_frac * n_t) rows of T (chosen without replacement) are
    overwritten by exact copies of as many randomly chosen P rows, so that
    equal points across the two samples exercise the tie convention.
    """
    rng = np.random.default_rng(seed)
    P = rng.standard_normal((n_p, d))
    Z = rng.standard_normal((n_t, d))
    T = Z.copy()
    T[:, 1] = rho * Z[:, 0] + math.sqrt(1.0 - rho * rho) * Z[:, 1]
    P = P.astype(dtype)
    T = T.astype(dtype)
    n_dup = int(round(dup_frac * n_t))
    if n_dup > 0:
        rows_t = rng.choice(n_t, size=n_dup, replace=False)
        rows_p = rng.choice(n_p, size=n_dup, replace=False)
        T[rows_t] = P[rows_p]
    return P, T


def uniform_beta_pair(seed=0, n_p=4096, n_t=4096, d=12, beta_dim=5, dtype=np.float64):
    """P ~ U[0,1]^d; T the same except coordinate beta_dim ~ Beta(2, 2)."""
    rng = np.random.default_rng(seed)
    P = rng.random((n_p, d))
    T = rng.random((n_t, d))
    T[:, beta_dim] = rng.beta(2.0, 2.0, size=n_t)
    return P.astype(dtype), T.astype(dtype)


def mixture_means(rng, d, k=3, scale=1.0):
    """k component means, each +-scale (random sign) on one random axis."""
    means = np.zeros((k, d))
    for c in range(k):
        axis = int(rng.integers(0, d))
        means[c, axis] = scale if rng.random() < 0.5 else -scale
    return means


def mixture_sample(rng, n, means, sigma=0.5):
    """n points from the equal-weight isotropic Gaussian mixture with these means."""
    k, d = means.shape
    comp = rng.integers(0, k, size=n)
    return means[comp] + sigma * rng.standard_normal((n, d))


def mixture_pair(seed=0, n_p=2000, n_t=2000, d=3, shift=0.0, sigma=0.5, dtype=np.float32):
    """P and T from the same 3-component mixture; T shifted by shift * 1."""
    rng = np.random.default_rng(seed)
    means = mixture_means(rng, d)
    P = mixture_sample(rng, n_p, means, sigma)
    T = mixture_sample(rng, n_t, means, sigma) + shift
    return P.astype(dtype), T.astype(dtype)


def dvu_pair(seed=0, n_p=100, n_t=100, d=1000, dtype=np.float32):
    """Diagonal versus uniform (Sec. 4.1): P uniform on the diagonal of the
    unit cube (every coordinate of a point equal to one U[0,1] draw), T
    uniform in [0,1]^d."""
    rng = np.random.default_rng(seed)
    u = rng.random(n_p)
    P = np.repeat(u[:, None], d, axis=1)
    T = rng.random((n_t, d))
    return P.astype(dtype), T.astype(dtype)


def dvu_null_pair(seed=0, n_p=50, n_t=50, d=3, dtype=np.float32):
    """Both samples from the diagonal distribution of DVU (the null case of
    the type I study of Sec. 3)."""
    rng = np.random.default_rng(seed)
    u = rng.random(n_p)
    v = rng.random(n_t)
    P = np.repeat(u[:, None], d, axis=1)
    T = np.repeat(v[:, None], d, axis=1)
    return P.astype(dtype), T.astype(dtype)


def log_uniform_int(rng, lo, hi, size=None):
    """Integers log-uniform in [lo, hi]."""
    v = np.exp(rng.uniform(math.log(lo), math.log(hi + 1), size=size))
    return np.clip(np.floor(v).astype(np.int64), lo, hi)


def uneven_problems(seed=0, count=256, n_lo=64, n_hi=8192, dims=tuple(range(2, 9)),
                    dtype=np.float32):
    """count two-sample problems: NP, NT independently log-uniform in [n_lo, n_hi],
    d uniform over dims, mixture data with a random shift in [0, 0.3]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n_p = int(log_uniform_int(rng, n_lo, n_hi))
        n_t = int(log_uniform_int(rng, n_lo, n_hi))
        d = int(dims[int(rng.integers(0, len(dims)))])
        means = mixture_means(rng, d)
        shift = float(rng.uniform(0.0, 0.3))
        P = mixture_sample(rng, n_p, means).astype(dtype)
        T = (mixture_sample(rng, n_t, means) + shift).astype(dtype)
        out.append((P, T))
    return out


def serving_requests(seed=0, count=2000, rate_hz=200.0, n_lo=100, n_hi=50000,
                     dims=(2, 3, 4, 6, 8), dtype=np.float32):
    """Poisson arrivals: returns a list of (arrival_s, P, T)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(count):
        t += float(rng.exponential(1.0 / rate_hz))
        n_p = int(log_uniform_int(rng, n_lo, n_hi))
        n_t = int(log_uniform_int(rng, n_lo, n_hi))
        d = int(dims[int(rng.integers(0, len(dims)))])
        means = mixture_means(rng, d)
        shift = float(rng.uniform(0.0, 0.3))
        P = mixture_sample(rng, n_p, means).astype(dtype)
        T = (mixture_sample(rng, n_t, means) + shift).astype(dtype)
        out.append((t, P, T))
    return out


def random_pair(seed, n_p, n_t, d, kind="normal", dtype=np.float32):
    """Small test inputs with a chosen value structure.

    kind: "normal" (continuous), "int" (small integers, many ties),
    "const" (all coordinates equal), "shifted" (T strictly above P).
    """
    rng = np.random.default_rng(seed)
    if kind == "normal":
        P = rng.standard_normal((n_p, d))
        T = rng.standard_normal((n_t, d)) + 0.3
    elif kind == "int":
        P = rng.integers(-3, 4, size=(n_p, d)).astype(np.float64)
        T = rng.integers(-2, 5, size=(n_t, d)).astype(np.float64)
    elif kind == "const":
        P = np.full((n_p, d), 1.5)
        T = np.full((n_t, d), 1.5)
    elif kind == "shifted":
        P = rng.random((n_p, d))
        T = rng.random((n_t, d)) + 2.0
    else:
        raise ValueError(kind)
    return P.astype(dtype), T.astype(dtype)


CONFIGS = {
    "cfg1_d3_200x200_f32": lambda: gaussian_pair(seed=0),
    "cfg2_d4_20000x20000_f32_ties": lambda: correlated_pair_with_ties(seed=0),
    "cfg3_d12_4096x4096_f64": lambda: uniform_beta_pair(seed=0),
    "cfg4_d3_2000x2000_mixture_null": lambda: mixture_pair(seed=0, shift=0.0),
    "cfg4_d3_2000x2000_mixture_alt": lambda: mixture_pair(seed=0, shift=0.2),
}
