"""Comparison helpers for the GPU-versus-oracle parity tests."""
import numpy as np


def support_mismatch(gpu_idx, D, L_ref, zeta_ref, band_rel=1e-6, band_abs_rel_D=0.0):
    """Indices where the GPU support differs from supp(T_zeta(D - L_ref)), and whether
    every one of them lies within the tie band | |R_ij| - zeta | <= band_rel*zeta +
    band_abs_rel_D*max(|D_ij|, |L_ij|) computed from the oracle's R."""
    R = (D - L_ref).reshape(-1)
    ref = np.flatnonzero(np.abs(R) > zeta_ref)
    diff = np.setxor1d(np.asarray(gpu_idx), ref)
    if diff.size == 0:
        return diff, True
    band = band_rel * zeta_ref + band_abs_rel_D * np.maximum(np.abs(D.reshape(-1)[diff]), np.abs(L_ref.reshape(-1)[diff]))
    ok = bool(np.all(np.abs(np.abs(R[diff]) - zeta_ref) <= band))
    return diff, ok


def rel_fro(A, B):
    return float(np.linalg.norm(A - B) / np.linalg.norm(B))


def factored_rel_err(U, sig, V, P, Q):
    """||U diag(sig) V^T - P Q^T||_F / ||P Q^T||_F from thin QR factors (no m x n array):
    X Y^T with X = [U diag(sig), -P], Y = [V, Q] has the norm of R_X R_Y^T, which the QR
    gives to rounding level (a difference of squared norms would stop at ~1e-8)."""
    rx = np.linalg.qr(np.hstack([U * sig, -P]), mode="r")
    ry = np.linalg.qr(np.hstack([V, Q]), mode="r")
    rp = np.linalg.qr(P, mode="r")
    rq = np.linalg.qr(Q, mode="r")
    return float(np.linalg.norm(rx @ ry.T) / np.linalg.norm(rp @ rq.T))
