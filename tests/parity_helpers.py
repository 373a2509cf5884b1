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
