"""Planted robust-PCA instances, following the synthetic set-up of Section 3 of the paper.

An m x n rank-r matrix L* = P Q^T is drawn with P, Q having i.i.d. standard normal
entries.  The support of S* is drawn uniformly without replacement, with exactly
round(alpha * m * n) positions, and its values are i.i.d. uniform on
[-c E|L*_ij|, c E|L*_ij|].  E|L*_ij| is read as the empirical mean of |L*| over the drawn
instance (the expectation has no closed form for r > 1).  D = L* + S*.

All randomness comes from one numpy ``Generator(PCG64(seed))`` in a fixed order
(P, Q, support, values), so a seed fixes every byte of D.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class PlantedInstance:
    m: int
    n: int
    r: int
    alpha: float
    c: float
    seed: int
    P: np.ndarray          # m x r, N(0,1)
    Q: np.ndarray          # n x r, N(0,1)
    D: np.ndarray          # m x n float64, row-major: L* + S*
    support: np.ndarray    # int64 linear indices i*n + j of supp(S*), ascending
    values: np.ndarray     # float64 values of S* at ``support``
    mean_abs_L: float      # the E|L*_ij| used for the value range
    mu: float              # incoherence of L* (assumption A1)

    @property
    def L(self) -> np.ndarray:
        """The planted low-rank matrix L* = P Q^T (formed on demand)."""
        return self.P @ self.Q.T

    @property
    def S(self) -> np.ndarray:
        """The planted sparse matrix S* as a dense array (formed on demand)."""
        S = np.zeros(self.m * self.n)
        S[self.support] = self.values
        return S.reshape(self.m, self.n)

    def params(self) -> dict:
        return paper_parameters(self.mu, self.m, self.n, self.r, self.alpha)


def incoherence(P: np.ndarray, Q: np.ndarray) -> float:
    """mu of L = P Q^T per assumption A1: the smallest mu with
    max_i ||e_i^T U||^2 <= mu r / m and max_j ||e_j^T V||^2 <= mu r / n, where U and V
    are orthonormal bases of the column spaces of P and Q (these span the singular
    subspaces of L when P and Q have full column rank)."""
    m, r = P.shape
    n = Q.shape[0]
    U, _ = np.linalg.qr(P)
    V, _ = np.linalg.qr(Q)
    mu_u = m / r * float(np.max(np.sum(U * U, axis=1)))
    mu_v = n / r * float(np.max(np.sum(V * V, axis=1)))
    return max(mu_u, mu_v)


def paper_parameters(mu: float, m: int, n: int, r: int, alpha: float) -> dict:
    """Parameter choices of the synthetic experiments (Section 3): the algorithms are
    given 1.1 mu, beta = 1.1 mu r / (2 sqrt(mn)), beta_init = 1.1 mu r / sqrt(mn), and
    gamma = 0.5 for alpha < 0.55, else 0.65."""
    mu_in = 1.1 * mu
    root = math.sqrt(m * n)
    return {
        "beta": mu_in * r / (2.0 * root),
        "beta_init": mu_in * r / root,
        "gamma": 0.5 if alpha < 0.55 else 0.65,
        "mu": mu_in,
    }


def planted_instance(m: int, n: int, r: int, alpha: float, c: float, seed: int) -> PlantedInstance:
    rng = np.random.Generator(np.random.PCG64(seed))
    P = rng.standard_normal((m, r))
    Q = rng.standard_normal((n, r))
    D = P @ Q.T
    mean_abs = float(np.mean(np.abs(D)))
    k = int(round(alpha * m * n))
    support = rng.choice(m * n, size=k, replace=False).astype(np.int64)
    values = rng.uniform(-c * mean_abs, c * mean_abs, size=k)
    order = np.argsort(support, kind="stable")
    support = support[order]
    values = values[order]
    flat = D.reshape(-1)
    flat[support] += values
    return PlantedInstance(m=m, n=n, r=r, alpha=alpha, c=c, seed=seed, P=P, Q=Q, D=D,
                           support=support, values=values, mean_abs_L=mean_abs,
                           mu=incoherence(P, Q))
