"""Plain FP64 CPU oracle of AccAltProj (Cai, Cai & Wei, "Accelerated Alternating
Projections for Robust PCA", arXiv 1711.05519).

TEST INFRASTRUCTURE.  This module exists to check the CUDA library against the paper.  Only
the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  It shares no code with the CUDA path: it uses numpy / scipy in float64, one
library call per mathematical step, with no blocking, fusion or reordering beyond what
the paper states, so it can be checked against the paper by eye.

Notation follows the paper: D = L + S is m x n, r the target rank, L_k = U_k Sigma_k V_k^T
the current low-rank estimate, S_k the sparse estimate, zeta_k the threshold, beta and
gamma the threshold parameters, mu the incoherence level used by Trim.

Readings of the paper taken where it is silent or garbled (each also listed in the
design notes of the repository):
  * Trim (Algorithm 2) caps the rows of U at sqrt(mu r / m) and the rows of V at
    sqrt(mu r / n), as assumption A1 does for a rectangular matrix; the algorithm box uses
    one constant sqrt(mu r / n) because it is written for m = n.
  * The second QR of Section 2.1 is taken of (I - V~V~^T)(D - S_k)^T U~ (the transpose is
    implied by the shapes for rectangular D).
  * The threshold keeps |Z_ij| > zeta strictly, Eq. (10).
  * zeta_0 = beta sigma_1(D - S_{-1}) carries no sigma_{r+1} term (Algorithm 3); from k = 0
    on, zeta_{k+1} = beta (sigma_{r+1} + gamma^{k+1} sigma_1) of P_T~k(D - S_k)
    (Algorithm 1).  The simplified form zeta_{k+1} = beta gamma^{k+1} sigma_1 is offered as
    ``zeta_mode="simple"``.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse.linalg as sla

# Sizes up to which the oracle takes a dense LAPACK SVD instead of ARPACK.
DENSE_SVD_LIMIT = 1500


# --------------------------------------------------------------------------------------
# Operators of Section 2.1
# --------------------------------------------------------------------------------------

def tangent_project(Z: np.ndarray, U: np.ndarray, V: np.ndarray) -> np.ndarray:
    """Eq. (6): P_T Z = U U^T Z + Z V V^T - U U^T Z V V^T, for orthonormal U (m x r) and
    V (n x r) spanning the tangent space of Eq. (5)."""
    UUtZ = U @ (U.T @ Z)
    ZVVt = (Z @ V) @ V.T
    return UUtZ + ZVVt - (UUtZ @ V) @ V.T


def complement_project(Z: np.ndarray, U: np.ndarray, V: np.ndarray) -> np.ndarray:
    """Eq. (7): (I - P_T) Z = (I - U U^T) Z (I - V V^T)."""
    left = Z - U @ (U.T @ Z)
    return left - (left @ V) @ V.T


def best_rank_r(Z: np.ndarray, r: int) -> np.ndarray:
    """Eq. (8): H_r(Z), the SVD of Z with all but the r largest singular values zeroed."""
    Qm, lam, Pt = np.linalg.svd(Z, full_matrices=False)
    return (Qm[:, :r] * lam[:r]) @ Pt[:r]


def hard_threshold(Z: np.ndarray, zeta: float) -> np.ndarray:
    """Eq. (10): [T_zeta Z]_ij = Z_ij if |Z_ij| > zeta, else 0."""
    return np.where(np.abs(Z) > zeta, Z, 0.0)


def relative_error(D: np.ndarray, L: np.ndarray, S: np.ndarray) -> float:
    """Eq. (11): err_k = ||D - L_k - S_k||_F / ||D||_F."""
    return float(np.linalg.norm(D - L - S) / np.linalg.norm(D))


def trim(U: np.ndarray, V: np.ndarray, mu: float, r: int):
    """Algorithm 2 (Trim): scale row i of U by min(1, c_U / ||U^(i)||) and row j of V by
    min(1, c_V / ||V^(j)||), with c_U = sqrt(mu r / m) and c_V = sqrt(mu r / n).  Returns the
    trimmed factors A and B (L~ = A Sigma B^T)."""
    m, n = U.shape[0], V.shape[0]
    c_u = math.sqrt(mu * r / m)
    c_v = math.sqrt(mu * r / n)
    A = np.empty_like(U)
    for i in range(m):
        norm = np.linalg.norm(U[i])
        A[i] = U[i] * (min(1.0, c_u / norm) if norm > 0 else 1.0)
    B = np.empty_like(V)
    for j in range(n):
        norm = np.linalg.norm(V[j])
        B[j] = V[j] * (min(1.0, c_v / norm) if norm > 0 else 1.0)
    return A, B


def trimmed_bases(U: np.ndarray, V: np.ndarray, mu: float, r: int, do_trim: bool = True):
    """U~_k and V~_k of Section 2.1: orthonormal bases of the column spaces of the trimmed
    factors, taken by a QR decomposition (the footnote to Eq. (5)).  Without trim they
    are U_k and V_k themselves."""
    if not do_trim:
        return U, V
    A, B = trim(U, V, mu, r)
    Ut, _ = np.linalg.qr(A)
    Vt, _ = np.linalg.qr(B)
    return Ut, Vt


def tangent_truncated_svd(Z: np.ndarray, Ut: np.ndarray, Vt: np.ndarray, r: int):
    """H_r(P_T~ Z) by the route of Section 2.1: QR of (I - U~U~^T) Z V~ and of
    (I - V~V~^T) Z^T U~, the 2r x 2r matrix M = [[U~^T Z V~, R2^T], [R1, 0]], its SVD, and
    Eq. (9) for the new factors.

    Returns (U_new, sigma_new, V_new, sigma_M) where sigma_M holds all 2r singular values
    of M, which are those of P_T~ Z."""
    ZV = Z @ Vt
    ZtU = Z.T @ Ut
    C = Ut.T @ ZV
    Q1, R1 = np.linalg.qr(ZV - Ut @ C)
    Q2, R2 = np.linalg.qr(ZtU - Vt @ C.T)
    M = np.block([[C, R2.T], [R1, np.zeros((r, r))]])
    UM, sM, VMt = np.linalg.svd(M)
    U_new = np.hstack([Ut, Q1]) @ UM[:, :r]
    V_new = np.hstack([Vt, Q2]) @ VMt.T[:, :r]
    return U_new, sM[:r].copy(), V_new, sM


def next_threshold(beta: float, gamma: float, k_next: int, sigma_M: np.ndarray, r: int,
                   zeta_mode: str = "paper") -> float:
    """Algorithm 1: zeta_{k+1} = beta (sigma_{r+1} + gamma^{k+1} sigma_1), singular values
    of P_T~k(D - S_k).  ``zeta_mode="simple"`` drops the sigma_{r+1} term."""
    if zeta_mode == "paper":
        return float(beta * (sigma_M[r] + gamma ** k_next * sigma_M[0]))
    if zeta_mode == "simple":
        return float(beta * gamma ** k_next * sigma_M[0])
    raise ValueError(zeta_mode)


# --------------------------------------------------------------------------------------
# Initialisation, Algorithm 3
# --------------------------------------------------------------------------------------

def truncated_svd(X: np.ndarray, k: int, seed: int = 0):
    """Top-k singular triplets, descending.  Dense LAPACK for small matrices, ARPACK with
    tolerance 0 (machine precision) and a fixed start vector otherwise."""
    if min(X.shape) <= DENSE_SVD_LIMIT:
        U, s, Vt = np.linalg.svd(X, full_matrices=False)
        return U[:, :k], s[:k], Vt[:k].T
    v0 = np.random.Generator(np.random.PCG64(seed)).standard_normal(min(X.shape))
    U, s, Vt = sla.svds(X, k=k, tol=0, v0=v0, solver="arpack")
    order = np.argsort(s)[::-1]
    return U[:, order], s[order], Vt[order].T


def initialize(D: np.ndarray, r: int, beta_init: float, beta: float) -> dict:
    """Algorithm 3, two steps of AltProj:
    zeta_{-1} = beta_init sigma_1(D); S_{-1} = T(D); L_0 = H_r(D - S_{-1});
    zeta_0 = beta sigma_1(D - S_{-1}); S_0 = T_{zeta_0}(D - L_0)."""
    sigma1_D = float(truncated_svd(D, 1)[1][0])
    zeta_m1 = beta_init * sigma1_D
    S_m1 = hard_threshold(D, zeta_m1)
    U0, s0, V0 = truncated_svd(D - S_m1, r)
    zeta0 = beta * float(s0[0])
    L0 = (U0 * s0) @ V0.T
    S0 = hard_threshold(D - L0, zeta0)
    return {"U": U0, "sigma": s0, "V": V0, "zeta": zeta0, "S": S0, "sigma1_D": sigma1_D,
            "zeta_init": zeta_m1, "S_init": S_m1}


# --------------------------------------------------------------------------------------
# Algorithm 1
# --------------------------------------------------------------------------------------

def step(D: np.ndarray, U: np.ndarray, sigma: np.ndarray, V: np.ndarray, zeta: float, k: int,
         r: int, beta: float, gamma: float, mu: float, do_trim: bool = True,
         zeta_mode: str = "paper") -> dict:
    """One pass of the while-loop of Algorithm 1 starting from L_k = U diag(sigma) V^T and
    zeta_k: S_k = T_{zeta_k}(D - L_k) and err_k (the loop test), then Trim, L_{k+1} and
    zeta_{k+1}.  Used by the tests to check one GPU iteration from the GPU's own state."""
    L = (U * sigma) @ V.T
    S = hard_threshold(D - L, zeta)
    err = relative_error(D, L, S)
    Ut, Vt = trimmed_bases(U, V, mu, r, do_trim)
    Z = D - S
    U1, s1, V1, sM = tangent_truncated_svd(Z, Ut, Vt, r)
    zeta1 = next_threshold(beta, gamma, k + 1, sM, r, zeta_mode)
    return {"S": S, "err": err, "Ut": Ut, "Vt": Vt, "ZV": Z @ Vt, "ZtU": Z.T @ Ut,
            "U": U1, "sigma": s1, "V": V1, "sigma_M": sM, "zeta": zeta1}


def accaltproj(D: np.ndarray, r: int, beta: float, gamma: float, tol: float, mu: float,
               beta_init: float | None = None, do_trim: bool = True, max_iter: int = 100,
               zeta_mode: str = "paper", record_support: bool = False) -> dict:
    """Algorithm 1 with the initialisation of Algorithm 3.  The loop stops when
    err_k < tol or after ``max_iter`` iterations (Section 3 uses 100).

    Returns the final factors, S, and per-iteration histories of err_k, zeta_k, the
    singular values of M_k and nnz(S_k) (and the supports when ``record_support``)."""
    if beta_init is None:
        beta_init = 2.0 * beta
    init = initialize(D, r, beta_init, beta)
    U, sigma, V, zeta, S = init["U"], init["sigma"], init["V"], init["zeta"], init["S"]
    hist = {"err": [], "zeta": [zeta], "sigma_M": [], "nnz": [], "support": []}
    k = 0
    while True:
        L = (U * sigma) @ V.T
        err = relative_error(D, L, S)
        hist["err"].append(err)
        hist["nnz"].append(int(np.count_nonzero(S)))
        if record_support:
            hist["support"].append(np.flatnonzero(S))
        if err < tol or k >= max_iter:
            break
        Ut, Vt = trimmed_bases(U, V, mu, r, do_trim)
        U, sigma, V, sM = tangent_truncated_svd(D - S, Ut, Vt, r)
        zeta = next_threshold(beta, gamma, k + 1, sM, r, zeta_mode)
        hist["sigma_M"].append(sM)
        hist["zeta"].append(zeta)
        L = (U * sigma) @ V.T
        S = hard_threshold(D - L, zeta)
        k += 1
    return {"U": U, "sigma": sigma, "V": V, "S": S, "L": L, "iters": k, "err": err,
            "zeta": zeta, "init": init, "history": hist}
