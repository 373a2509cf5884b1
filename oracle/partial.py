"""Plain FP64 CPU oracle of AccAltProj with partially observed entries.

TEST INFRASTRUCTURE, like oracle/accaltproj.py: only the test suite, ``__graft_entry__.smoke()``
and the CPU legs of ``bench.py`` may import it; it shares no code with the CUDA path.

The paper solves the fully observed problem and names robust PCA from a subset of the
entries as the next question in its closing section, without an algorithm.  The reading
taken here (not the paper's text) extends each step of Algorithms 1-3 by the sampling
operator P_Obs (keep the observed entries, zero the rest) and the sampling fraction
p = |Obs| / (m n): the L-update becomes a step of size 1/p along the observed residual
before the tangent-space projection and the truncation, as in matrix completion:

  Algorithm 3:  Y = P_Obs(D) / p;  zeta_{-1} = beta_init sigma_1(Y);
                S_{-1} = T_{zeta_{-1}}(P_Obs(D));  L_0 = H_r(P_Obs(D - S_{-1}) / p);
                zeta_0 = beta sigma_1(P_Obs(D - S_{-1}) / p);  S_0 = T_{zeta_0}(P_Obs(D - L_0)).
  Algorithm 1:  Z_k = L_k + P_Obs(D - L_k - S_k) / p;
                L_{k+1} = H_r(P_T~k Z_k) by the QR + 2r x 2r SVD route of Section 2.1;
                zeta_{k+1} = beta (sigma_{r+1} + gamma^{k+1} sigma_1) of P_T~k Z_k;
                S_{k+1} = T_{zeta_{k+1}}(P_Obs(D - L_{k+1})).
  Stopping:     err_k = ||P_Obs(D - L_k - S_k)||_F / ||P_Obs(D)||_F < tol.

With every entry observed (p = 1) each line is the fully observed step of accaltproj.py
(Z_k = L_k + (D - L_k - S_k) = D - S_k up to rounding).  The unobserved values of D never
enter: every use of D goes through P_Obs.
"""
from __future__ import annotations

import numpy as np

from . import accaltproj as O


def sample(D: np.ndarray, observed: np.ndarray) -> np.ndarray:
    """P_Obs(D): the observed entries of D, zero elsewhere."""
    return np.where(observed, D, 0.0)


def initialize(D, observed, r, beta_init, beta):
    """Algorithm 3 on the sampled matrix (see the module docstring)."""
    p = float(np.mean(observed))
    Dobs = sample(D, observed)
    sigma1 = float(O.truncated_svd(Dobs / p, 1)[1][0])
    zeta_m1 = beta_init * sigma1
    S_m1 = O.hard_threshold(Dobs, zeta_m1)
    U0, s0, V0 = O.truncated_svd(sample(D - S_m1, observed) / p, r)
    zeta0 = beta * float(s0[0])
    L0 = (U0 * s0) @ V0.T
    S0 = O.hard_threshold(sample(D - L0, observed), zeta0)
    return {"U": U0, "sigma": s0, "V": V0, "zeta": zeta0, "S": S0, "p": p, "sigma1_D": sigma1}


def relative_error(D, observed, L, S):
    """err_k = ||P_Obs(D - L - S)||_F / ||P_Obs(D)||_F."""
    return float(np.linalg.norm(sample(D - L - S, observed)) / np.linalg.norm(sample(D, observed)))


def step(D, observed, U, sigma, V, zeta, k, r, beta, gamma, mu, do_trim=True):
    """One pass of the loop from L_k = U diag(sigma) V^T and zeta_k: S_k, err_k, Trim,
    L_{k+1} and zeta_{k+1}."""
    p = float(np.mean(observed))
    L = (U * sigma) @ V.T
    S = O.hard_threshold(sample(D - L, observed), zeta)
    err = relative_error(D, observed, L, S)
    Ut, Vt = O.trimmed_bases(U, V, mu, r, do_trim)
    Z = L + sample(D - L - S, observed) / p
    U1, s1, V1, sM = O.tangent_truncated_svd(Z, Ut, Vt, r)
    zeta1 = O.next_threshold(beta, gamma, k + 1, sM, r)
    return {"S": S, "err": err, "Ut": Ut, "Vt": Vt, "ZV": Z @ Vt, "ZtU": Z.T @ Ut, "U": U1, "sigma": s1, "V": V1,
            "sigma_M": sM, "zeta": zeta1}


def accaltproj_partial(D, observed, r, beta, gamma, tol, mu, beta_init=None, do_trim=True, max_iter=100):
    """Algorithm 1 with the initialisation of Algorithm 3, on the observed entries only."""
    if beta_init is None:
        beta_init = 2.0 * beta
    init = initialize(D, observed, r, beta_init, beta)
    U, sigma, V, zeta, S = init["U"], init["sigma"], init["V"], init["zeta"], init["S"]
    hist = {"err": [], "zeta": [zeta]}
    k = 0
    while True:
        L = (U * sigma) @ V.T
        err = relative_error(D, observed, L, S)
        hist["err"].append(err)
        if err < tol or k >= max_iter:
            break
        st = step(D, observed, U, sigma, V, zeta, k, r, beta, gamma, mu, do_trim)
        U, sigma, V, zeta = st["U"], st["sigma"], st["V"], st["zeta"]
        hist["zeta"].append(zeta)
        L = (U * sigma) @ V.T
        S = O.hard_threshold(sample(D - L, observed), zeta)
        k += 1
    return {"U": U, "sigma": sigma, "V": V, "S": S, "L": L, "iters": k, "err": err, "zeta": zeta, "init": init,
            "history": hist}
