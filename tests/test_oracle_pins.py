"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: a worked example the
paper prints, the defining properties of an orthogonal projector, a dense LAPACK SVD of an
explicitly formed matrix (brute force on tiny inputs), the Eckart-Young identity, or the
guarantees of Theorems 1 and 2 on planted instances.  ``test_pins_catch_planted_mistakes``
plants plausible mistakes in copies of the oracle's functions and checks that the pins
fail on each of them.
"""
import math
import os

import numpy as np
import pytest

import synth
from oracle import accaltproj as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _orth(rng, m, r):
    return np.linalg.qr(rng.standard_normal((m, r)))[0]


def _read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *nums = line.split()
            vals[key] = np.array([float(x) for x in nums])
    return vals


# ---------------------------------------------------------------------------------------
# Worked example printed in the paper
# ---------------------------------------------------------------------------------------

def test_tight_example_of_projection_norm_lemma():
    g = _read_golden("pt_norm_tight_example.txt")
    U = g["U"].reshape(2, 1)
    V = g["V"].reshape(2, 1)
    Z = g["Z"].reshape(2, 2)
    PZ = O.tangent_project(Z, U, V)
    ratio = np.linalg.norm(PZ, 2) / np.linalg.norm(Z, 2)
    assert ratio == pytest.approx(g["ratio"][0], rel=1e-14)
    # By hand: U U^T Z keeps row 1, Z V V^T keeps column 1, their overlap is Z_11.
    assert np.allclose(PZ, [[1.0, math.sqrt(2)], [math.sqrt(2), 0.0]], atol=1e-15)
    # The bound itself on random symmetric inputs in the symmetric setting.
    rng = np.random.default_rng(5)
    for _ in range(50):
        n, r = rng.integers(2, 12), 1
        r = int(rng.integers(1, n))
        Uq = _orth(rng, n, r)
        X = rng.standard_normal((n, n))
        X = X + X.T
        assert np.linalg.norm(O.tangent_project(X, Uq, Uq), 2) <= math.sqrt(4 / 3) * np.linalg.norm(X, 2) * (1 + 1e-12)


# ---------------------------------------------------------------------------------------
# P_T is the orthogonal projector onto T = {U A^T + B V^T}: Eqs. (5)-(7)
# ---------------------------------------------------------------------------------------

def _check_projector(project, complement, rng, m, n, r):
    U, V = _orth(rng, m, r), _orth(rng, n, r)
    Z = rng.standard_normal((m, n))
    # Elements of T (Eq. (5)) are fixed.
    A, B = rng.standard_normal((n, r)), rng.standard_normal((m, r))
    T_elem = U @ A.T + B @ V.T
    ok = np.allclose(project(T_elem, U, V), T_elem, atol=1e-12)
    # Elements of the orthogonal complement are annihilated.
    X = rng.standard_normal((m, n))
    perp = X - U @ (U.T @ X)
    perp = perp - (perp @ V) @ V.T
    ok &= np.allclose(project(perp, U, V), 0.0, atol=1e-12)
    # Idempotence, orthogonality of the two parts, and they sum to Z.
    PZ = project(Z, U, V)
    ok &= np.allclose(project(PZ, U, V), PZ, atol=1e-12)
    QZ = complement(Z, U, V)
    ok &= abs(np.sum(PZ * QZ)) < 1e-10 * np.sum(Z * Z)
    ok &= np.allclose(PZ + QZ, Z, atol=1e-12)
    # rank(P_T Z) <= 2r.
    s = np.linalg.svd(PZ, compute_uv=False)
    ok &= (min(m, n) <= 2 * r) or s[2 * r] < 1e-10 * s[0]
    return bool(ok)


@pytest.mark.parametrize("m,n,r", [(7, 7, 1), (12, 9, 2), (9, 13, 3), (30, 20, 4), (40, 64, 5)])
def test_tangent_projection_is_orthogonal_projector(m, n, r):
    rng = np.random.default_rng(m * 100 + n + r)
    for _ in range(5):
        assert _check_projector(O.tangent_project, O.complement_project, rng, m, n, r)


# ---------------------------------------------------------------------------------------
# H_r: Eq. (8) and the QR + 2r x 2r SVD route of Section 2.1
# ---------------------------------------------------------------------------------------

def test_best_rank_r_eckart_young():
    rng = np.random.default_rng(1)
    for _ in range(20):
        m, n = rng.integers(3, 40, size=2)
        r = int(rng.integers(1, min(m, n)))
        Z = rng.standard_normal((m, n))
        H = O.best_rank_r(Z, r)
        s = np.linalg.svd(Z, compute_uv=False)
        assert np.linalg.matrix_rank(H, tol=1e-9 * s[0]) <= r
        assert np.linalg.norm(Z - H) ** 2 == pytest.approx(np.sum(s[r:] ** 2), rel=1e-9, abs=1e-12)
        # A rank-r matrix is its own best rank-r approximation.
        L = rng.standard_normal((m, r)) @ rng.standard_normal((r, n))
        assert np.allclose(O.best_rank_r(L, r), L, atol=1e-10)


def _check_qr_route(route, rng, m, n, r):
    """Brute force: the QR route must equal a dense SVD truncation of the explicitly
    formed P_T Z (Eq. (6)), and the spectrum of M must be that of P_T Z."""
    U, V = _orth(rng, m, r), _orth(rng, n, r)
    Z = rng.standard_normal((m, n)) + 3.0 * _orth(rng, m, r) @ rng.standard_normal((r, n))
    PZ = U @ (U.T @ Z) + (Z @ V) @ V.T - U @ (U.T @ Z @ V) @ V.T
    Qd, ld, Pd = np.linalg.svd(PZ, full_matrices=False)
    if ld[r - 1] - ld[r] < 1e-6 * ld[0]:
        return True  # H_r not unique; skip this draw
    H_dense = (Qd[:, :r] * ld[:r]) @ Pd[:r]
    Un, sn, Vn, sM = route(Z, U, V, r)
    ok = np.allclose((Un * sn) @ Vn.T, H_dense, atol=1e-10 * ld[0])
    ok &= np.allclose(sM, ld[: 2 * r], rtol=1e-10, atol=1e-12 * ld[0])
    ok &= np.allclose(Un.T @ Un, np.eye(r), atol=1e-10) and np.allclose(Vn.T @ Vn, np.eye(r), atol=1e-10)
    return bool(ok)


def test_qr_route_equals_dense_truncated_svd_of_projection():
    rng = np.random.default_rng(2)
    checked = 0
    for _ in range(60):
        r = int(rng.integers(1, 6))
        m = int(rng.integers(2 * r + 1, 64))
        n = int(rng.integers(2 * r + 1, 64))
        assert _check_qr_route(O.tangent_truncated_svd, rng, m, n, r)
        checked += 1
    assert checked == 60


# ---------------------------------------------------------------------------------------
# Threshold (Eq. (10)), trim (Algorithm 2), zeta schedule (Algorithm 1)
# ---------------------------------------------------------------------------------------

def test_hard_threshold_is_strict():
    zeta = 0.75
    Z = np.array([[0.75, -0.75, 0.7500000000000001, -0.7500000000000001],
                  [0.0, 0.5, -2.0, 3.0]])
    T = O.hard_threshold(Z, zeta)
    assert np.array_equal(T, [[0.0, 0.0, 0.7500000000000001, -0.7500000000000001],
                              [0.0, 0.0, -2.0, 3.0]])


def test_trim_caps_row_norms_exactly():
    rng = np.random.default_rng(3)
    m, n, r, mu = 50, 30, 3, 1.5
    U = _orth(rng, m, r)
    V = _orth(rng, n, r)
    U[0] *= 10.0  # force rows above the cap (trim does not need orthonormal input)
    V[1] *= 10.0
    A, B = O.trim(U, V, mu, r)
    cu, cv = math.sqrt(mu * r / m), math.sqrt(mu * r / n)
    for X, Y, c in ((U, A, cu), (V, B, cv)):
        nx = np.linalg.norm(X, axis=1)
        ny = np.linalg.norm(Y, axis=1)
        big = nx > c
        assert big.any() and (~big).any()
        assert np.allclose(ny[big], c, rtol=1e-14)
        assert np.array_equal(Y[~big], X[~big])
        # Rows keep their direction.
        assert np.allclose(Y[big] / ny[big, None], X[big] / nx[big, None], atol=1e-14)
    Ut, Vt = O.trimmed_bases(U, V, mu, r)
    assert np.allclose(Ut.T @ Ut, np.eye(r), atol=1e-13)
    assert np.allclose(Ut @ (Ut.T @ A), A, atol=1e-13)  # same column space as A
    assert np.allclose(Vt @ (Vt.T @ B), B, atol=1e-13)


def test_threshold_schedule_closed_form():
    s = np.array([10.0, 4.0, 2.0, 1.0])
    assert O.next_threshold(0.1, 0.5, 3, s, 2) == pytest.approx(0.1 * (2.0 + 0.125 * 10.0))
    assert O.next_threshold(0.1, 0.5, 3, s, 2, "simple") == pytest.approx(0.1 * 0.125 * 10.0)


# ---------------------------------------------------------------------------------------
# Whole method on planted instances: Theorems 1 and 2, Section 3
# ---------------------------------------------------------------------------------------

@pytest.fixture(scope="module")
def config1_run():
    inst = synth.planted_instance(500, 500, 5, 0.1, 1.0, 0)
    p = inst.params()
    res = O.accaltproj(inst.D, 5, p["beta"], p["gamma"], 1e-10, p["mu"], beta_init=p["beta_init"],
                       record_support=True)
    return inst, p, res


def test_planted_recovery_config1(config1_run):
    inst, p, res = config1_run
    assert res["err"] < 1e-10
    L = inst.L
    assert np.linalg.norm(res["L"] - L) / np.linalg.norm(L) < 1e-9
    # S is recovered on the planted support.
    assert np.linalg.norm(res["S"] - inst.S) / np.linalg.norm(inst.S) < 1e-8


def test_support_stays_inside_planted_support(config1_run):
    """Theorem 1: supp(S_k) is a subset of Omega at every k."""
    inst, _, res = config1_run
    omega = inst.support
    for supp in res["history"]["support"]:
        assert np.isin(supp, omega).all()


def test_linear_convergence_rate(config1_run):
    """Theorem 1: the error decays like gamma^k.  The fitted slope of log err_k over the
    converging iterations is at most log(gamma) plus slack."""
    _, p, res = config1_run
    err = np.array(res["history"]["err"])
    tail = err[err < 1e-2]
    k = np.arange(len(tail))
    slope = np.polyfit(k, np.log(tail), 1)[0]
    assert slope <= math.log(p["gamma"]) + 0.3
    assert len(err) - 1 == res["iters"] <= 100


def test_initialisation_meets_theorem2_bounds(config1_run):
    """Theorem 2: ||L - L_0||_2 <= 8 alpha mu r sigma_1^L, ||S - S_0||_inf <= mu r / n sigma_1^L
    and supp(S_0) inside Omega (mu here is the instance's own incoherence)."""
    inst, p, res = config1_run
    init = res["init"]
    L = inst.L
    s1L = np.linalg.norm(L, 2)
    L0 = (init["U"] * init["sigma"]) @ init["V"].T
    mu, r, n, alpha = inst.mu, inst.r, inst.n, inst.alpha
    assert np.linalg.norm(L - L0, 2) <= 8 * alpha * mu * r * s1L
    assert np.max(np.abs(inst.S - init["S"])) <= mu * r / n * s1L
    assert np.isin(np.flatnonzero(init["S"]), inst.support).all()
    # sigma_1(D) matches a dense SVD.
    assert init["sigma1_D"] == pytest.approx(np.linalg.norm(inst.D, 2), rel=1e-12)


def _schedule_tracks_gamma_power(res, inst, p, tol=0.02):
    """On a planted instance sigma_1(P_T(D - S_k)) settles at sigma_1(L*) within the first
    iterations and sigma_{r+1}(P_T(D - S_k)) is negligible beside gamma^{k+1} sigma_1, so the
    schedule of Algorithm 1 started from zeta_0 = beta sigma_1(D - S_{-1}) (Algorithm 3) must
    follow zeta_k = beta gamma^k sigma_1(L*) at every k, which is the gamma^k rate of Theorem 1.
    sigma_1(L*) comes from a dense SVD of the planted matrix, not from the oracle."""
    s1L = np.linalg.norm(inst.L, 2)
    z = np.asarray(res["history"]["zeta"])
    c = z / (p["beta"] * p["gamma"] ** np.arange(len(z)) * s1L)
    return bool(len(z) > 10 and np.all(np.abs(c - 1.0) < tol))


def test_threshold_schedule_tracks_gamma_power(config1_run):
    inst, p, res = config1_run
    assert _schedule_tracks_gamma_power(res, inst, p)
    # zeta_0 of Algorithm 3 against a dense spectral norm of D - S_{-1}
    init = res["init"]
    assert init["zeta"] == pytest.approx(p["beta"] * np.linalg.norm(inst.D - init["S_init"], 2), rel=1e-12)
    # zeta_{k+1} / zeta_k = gamma from the first step on (k + 1 in the exponent, not k)
    z = np.asarray(res["history"]["zeta"])
    assert np.allclose(z[1:] / z[:-1], p["gamma"], rtol=0.01)


def test_iterates_obey_theorem1_l2_bound(config1_run):
    """Theorem 1's L bound, ||L - L_k||_2 <= 8 alpha mu r gamma^k sigma_1^L, along the path."""
    inst, p, res = config1_run
    # Re-run the path step by step with the oracle's own step() to get every L_k.
    L = inst.L
    s1L = np.linalg.norm(L, 2)
    init = res["init"]
    U, s, V, zeta = init["U"], init["sigma"], init["V"], init["zeta"]
    for k in range(res["iters"]):
        Lk = (U * s) @ V.T
        bound = 8 * inst.alpha * inst.mu * inst.r * p["gamma"] ** k * s1L
        assert np.linalg.norm(L - Lk, 2) <= bound + 1e-9 * s1L
        st = O.step(inst.D, U, s, V, zeta, k, 5, p["beta"], p["gamma"], p["mu"])
        U, s, V, zeta = st["U"], st["sigma"], st["V"], st["zeta"]
    assert np.linalg.norm((U * s) @ V.T - res["L"]) < 1e-8 * s1L


def test_rectangular_and_no_trim_recover():
    inst = synth.planted_instance(300, 180, 3, 0.1, 1.0, 4)
    p = inst.params()
    for do_trim in (True, False):
        res = O.accaltproj(inst.D, 3, p["beta"], p["gamma"], 1e-9, p["mu"], beta_init=p["beta_init"],
                           do_trim=do_trim)
        assert res["err"] < 1e-9
        assert np.linalg.norm(res["L"] - inst.L) / np.linalg.norm(inst.L) < 1e-7


@pytest.mark.slow
def test_phase_transition_table2_endpoints():
    """Table 2, c = 1, n = 2500, r = 5: recovery (||L_k - L||_F/||L||_F <= 1e-4, tol 1e-6)
    succeeds in 10/10 trials at alpha = 0.3 and fails in 10/10 at alpha = 0.75.  Two trials
    of each endpoint are run here."""
    for alpha, expect in ((0.3, True), (0.75, False)):
        for seed in (11, 12):
            inst = synth.planted_instance(2500, 2500, 5, alpha, 1.0, seed)
            p = inst.params()
            res = O.accaltproj(inst.D, 5, p["beta"], p["gamma"], 1e-6, p["mu"], beta_init=p["beta_init"])
            ok = np.linalg.norm(res["L"] - inst.L) / np.linalg.norm(inst.L) <= 1e-4
            assert ok == expect, (alpha, seed)


# ---------------------------------------------------------------------------------------
# The pins are sensitive: plant plausible mistakes in copies of the oracle's functions.
# ---------------------------------------------------------------------------------------

def _proj_dropped_term(Z, U, V):
    return U @ (U.T @ Z) + (Z @ V) @ V.T


def _proj_wrong_sign(Z, U, V):
    UUtZ = U @ (U.T @ Z)
    return UUtZ + (Z @ V) @ V.T + (UUtZ @ V) @ V.T


def _proj_swapped(Z, U, V):
    return U @ (U.T @ Z) + (Z @ V) @ V.T - U @ (U.T @ Z) @ U @ U.T if Z.shape[0] == Z.shape[1] else Z * 0


def _route_dropped_R2(Z, Ut, Vt, r):
    ZV, ZtU = Z @ Vt, Z.T @ Ut
    C = Ut.T @ ZV
    Q1, R1 = np.linalg.qr(ZV - Ut @ C)
    Q2, R2 = np.linalg.qr(ZtU - Vt @ C.T)
    M = np.block([[C, np.zeros((r, r))], [R1, np.zeros((r, r))]])
    UM, sM, VMt = np.linalg.svd(M)
    return np.hstack([Ut, Q1]) @ UM[:, :r], sM[:r], np.hstack([Vt, Q2]) @ VMt.T[:, :r], sM


def _route_transposed_C(Z, Ut, Vt, r):
    ZV, ZtU = Z @ Vt, Z.T @ Ut
    C = Ut.T @ ZV
    Q1, R1 = np.linalg.qr(ZV - Ut @ C)
    Q2, R2 = np.linalg.qr(ZtU - Vt @ C.T)
    M = np.block([[C.T, R2.T], [R1, np.zeros((r, r))]])
    UM, sM, VMt = np.linalg.svd(M)
    return np.hstack([Ut, Q1]) @ UM[:, :r], sM[:r], np.hstack([Vt, Q2]) @ VMt.T[:, :r], sM


def _route_no_projection(Z, Ut, Vt, r):
    ZV, ZtU = Z @ Vt, Z.T @ Ut
    C = Ut.T @ ZV
    Q1, R1 = np.linalg.qr(ZV)
    Q2, R2 = np.linalg.qr(ZtU - Vt @ C.T)
    M = np.block([[C, R2.T], [R1, np.zeros((r, r))]])
    UM, sM, VMt = np.linalg.svd(M)
    return np.hstack([Ut, Q1]) @ UM[:, :r], sM[:r], np.hstack([Vt, Q2]) @ VMt.T[:, :r], sM


def test_pins_catch_planted_mistakes(monkeypatch):
    # the threshold exponent: gamma^k in place of gamma^{k+1} (Algorithm 1)
    inst = synth.planted_instance(500, 500, 5, 0.1, 1.0, 0)
    p = inst.params()
    good = O.next_threshold
    monkeypatch.setattr(O, "next_threshold",
                        lambda beta, gamma, k_next, sM, r, zeta_mode="paper": good(beta, gamma, k_next - 1, sM, r,
                                                                                   zeta_mode))
    bad = O.accaltproj(inst.D, 5, p["beta"], p["gamma"], 1e-10, p["mu"], beta_init=p["beta_init"])
    assert not _schedule_tracks_gamma_power(bad, inst, p)
    monkeypatch.setattr(O, "next_threshold", good)
    rng = np.random.default_rng(9)
    for bad in (_proj_dropped_term, _proj_wrong_sign, _proj_swapped):
        assert not all(_check_projector(bad, O.complement_project, rng, 12, 12, 2) for _ in range(3))
    for bad in (_route_dropped_R2, _route_transposed_C, _route_no_projection):
        assert not all(_check_qr_route(bad, rng, 20, 16, 3) for _ in range(5))
    # The correct versions pass the same checks.
    assert all(_check_projector(O.tangent_project, O.complement_project, rng, 12, 12, 2) for _ in range(3))
    assert all(_check_qr_route(O.tangent_truncated_svd, rng, 20, 16, 3) for _ in range(5))
