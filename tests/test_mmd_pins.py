"""CPU pins of the MMD loss gradient (Sec. "Forward Mode", Listing mmd) on the
oracle alone: the shift formula dL/dtheta_k = (p_+ - p_-)^T K (p - q) for a
Gaussian kernel on basis indices equals central finite differences of the
loss computed from the oracle's exact output distributions."""
import math

import numpy as np

import oracle
import workloads as W


def kernel(n, sigma):
    x = np.arange(1 << n, dtype=float)
    return np.exp(-(x[:, None] - x[None, :]) ** 2 / (2 * sigma * sigma))


def dist(n, gates, params):
    psi = oracle.apply_circuit(oracle.zero_state(n), n, gates, params)
    return np.abs(psi) ** 2


def mmd(p, q, K):
    return p @ K @ p - 2 * p @ K @ q + q @ K @ q


def test_shift_formula_equals_finite_differences():
    n = 4
    gates, params = W.variational(n, 2, "ring", seed=8)
    rs = np.random.default_rng(1)
    q = rs.random(1 << n)
    q /= q.sum()
    for sigma in (0.5, 2.0, 5.0):
        K = kernel(n, sigma)
        p = dist(n, gates, params)
        h = 1e-5
        for k in range(len(params)):
            pp, pm = np.array(params, float), np.array(params, float)
            pp[k] += math.pi / 2
            pm[k] -= math.pi / 2
            shift = (dist(n, gates, pp) - dist(n, gates, pm)) @ K @ (p - q)
            fp, fm = np.array(params, float), np.array(params, float)
            fp[k] += h
            fm[k] -= h
            fd = (mmd(dist(n, gates, fp), q, K) - mmd(dist(n, gates, fm), q, K)) / (2 * h)
            assert abs(shift - fd) < 1e-7, (sigma, k, shift, fd)
