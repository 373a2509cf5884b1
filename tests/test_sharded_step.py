"""Row-band sharding of one iteration of Algorithm 1 on CPU ranks (gloo, world size 2).

Rank p holds a band of rows of D and of U; V, sigma and zeta are replicated.  The only
exchanges are sums: the pass's partial Y2 = sum_p Z_p^T U~_p (n x r words), the Gram
matrices of the trimmed U and of W1 and C = U~^T Y1 (3 r^2 words), and the residual and
support totals (2 words).  Everything else (Trim of V, V~, W2, the Cholesky factors, the
2r x 2r SVD and zeta_{k+1}) is replicated, and U_{k+1} stays distributed.  The test checks
that the sharded step gives the unsharded oracle step (oracle/accaltproj.py), to rounding,
and that the exchanged partials are the unsharded products.  The sharded arithmetic here is
plain numpy on the oracle's definitions (Section 2.1, Eqs. (5)-(11), Algorithm 2); the GPU
library runs one instance per GPU."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _allreduce(x):
    import torch
    import torch.distributed as dist

    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
    dist.all_reduce(t)
    return t.numpy()


def _chol_t(G):
    """R (upper, R^T R = G) and T = R^-1: the QR of Section 2.1 with Q = X T implicit."""
    R = np.linalg.cholesky(G).T
    return R, np.linalg.inv(R)


def sharded_step(D_p, rows, m, U_p, sigma, V, zeta, k, r, beta, gamma, mu):
    """One iteration from L_k on the band `rows` of D; returns this rank's rows of U_{k+1},
    the replicated sigma_{k+1}, V_{k+1}, zeta_{k+1}, and the exchanged sums."""
    from oracle import accaltproj as O

    n = V.shape[0]
    # Trim (Algorithm 2): rows of U capped at sqrt(mu r / m) (the global m), V replicated
    cap_u, cap_v = np.sqrt(mu * r / m), np.sqrt(mu * r / n)
    A_p = U_p * np.minimum(1.0, cap_u / np.maximum(np.linalg.norm(U_p, axis=1), 1e-300))[:, None]
    B = V * np.minimum(1.0, cap_v / np.maximum(np.linalg.norm(V, axis=1), 1e-300))[:, None]
    # orthonormal bases: U~ = A~ T_u with the Gram matrix of A~ summed over the ranks
    G_u = _allreduce(A_p.T @ A_p)
    _, T_u = _chol_t(G_u)
    _, T_v = _chol_t(B.T @ B)
    Ut_p, Vt = A_p @ T_u, B @ T_v
    # the fused pass on the band: S_k, residual, Y1 rows (local), Y2 partial (summed)
    L_p = (U_p * sigma) @ V.T
    S_p = O.hard_threshold(D_p - L_p, zeta)
    Z_p = D_p - S_p
    tot = _allreduce(np.array([np.sum((D_p - L_p - S_p) ** 2), np.count_nonzero(S_p), np.sum(D_p ** 2)]))
    Y1_p = Z_p @ Vt
    Y2 = _allreduce(Z_p.T @ Ut_p)
    # projections and the Gram matrices of Section 2.1
    C = _allreduce(Ut_p.T @ Y1_p)
    W1_p = Y1_p - Ut_p @ C
    W2 = Y2 - Vt @ C.T
    G1 = _allreduce(W1_p.T @ W1_p)
    R1, T1 = _chol_t(G1)
    R2, T2 = _chol_t(W2.T @ W2)
    M = np.block([[C, R2.T], [R1, np.zeros((r, r))]])
    UM, sM, VMt = np.linalg.svd(M)
    VM = VMt.T
    U1_p = Ut_p @ UM[:r, :r] + W1_p @ (T1 @ UM[r:, :r])  # Eq. (9), Q1 = W1 T1 implicit
    V1 = Vt @ VM[:r, :r] + W2 @ (T2 @ VM[r:, :r])
    zeta1 = O.next_threshold(beta, gamma, k + 1, sM, r)
    return {"U": U1_p, "sigma": sM[:r].copy(), "V": V1, "zeta": zeta1, "err": np.sqrt(tot[0] / tot[2]),
            "nnz": tot[1], "Y2": Y2, "C": C, "G1": G1}


def _worker(rank, world, port, case, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import synth
    from oracle import accaltproj as O

    dist.init_process_group("gloo", rank=rank, world_size=world)
    m, n, r, alpha, seed, k = case
    inst = synth.planted_instance(m, n, r, alpha, 1.0, seed)
    p = inst.params()
    ini = O.initialize(inst.D, r, p["beta_init"], p["beta"])
    U, s, V, zeta = ini["U"], ini["sigma"], ini["V"], ini["zeta"]
    for kk in range(k):  # the unsharded trajectory to iterate k, replicated
        st = O.step(inst.D, U, s, V, zeta, kk, r, p["beta"], p["gamma"], p["mu"])
        U, s, V, zeta = st["U"], st["sigma"], st["V"], st["zeta"]
    bands = np.array_split(np.arange(m), world)
    rows = bands[rank]
    res = sharded_step(inst.D[rows], rows, m, U[rows], s, V, zeta, k, r, p["beta"], p["gamma"], p["mu"])
    out[rank] = {"rows": rows, **res}
    dist.destroy_process_group()


@pytest.mark.parametrize("case", [(300, 260, 4, 0.1, 71, 3), (257, 301, 3, 0.15, 72, 5)])
def test_row_band_step_equals_the_unsharded_step(case):
    import synth
    from oracle import accaltproj as O

    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(rk, 2, port, case, out)) for rk in range(2)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(120)
    assert all(pr.exitcode == 0 for pr in procs)
    m, n, r, alpha, seed, k = case
    inst = synth.planted_instance(m, n, r, alpha, 1.0, seed)
    p = inst.params()
    ini = O.initialize(inst.D, r, p["beta_init"], p["beta"])
    U, s, V, zeta = ini["U"], ini["sigma"], ini["V"], ini["zeta"]
    for kk in range(k):
        st = O.step(inst.D, U, s, V, zeta, kk, r, p["beta"], p["gamma"], p["mu"])
        U, s, V, zeta = st["U"], st["sigma"], st["V"], st["zeta"]
    ref = O.step(inst.D, U, s, V, zeta, k, r, p["beta"], p["gamma"], p["mu"])
    a, b = out[0], out[1]
    # replicated results agree between the ranks exactly, and with the oracle to rounding
    assert np.array_equal(a["sigma"], b["sigma"]) and a["zeta"] == b["zeta"] and np.array_equal(a["V"], b["V"])
    U1 = np.zeros((m, r))
    U1[a["rows"]], U1[b["rows"]] = a["U"], b["U"]
    L_sh = (U1 * a["sigma"]) @ a["V"].T
    L_ref = (ref["U"] * ref["sigma"]) @ ref["V"].T
    assert np.linalg.norm(L_sh - L_ref) < 1e-12 * np.linalg.norm(L_ref)
    assert a["zeta"] == pytest.approx(ref["zeta"], rel=1e-12)
    # the exchanged sums are the unsharded products
    Ut, Vt = O.trimmed_bases(U, V, p["mu"], r)
    Lk = (U * s) @ V.T
    Z = inst.D - O.hard_threshold(inst.D - Lk, zeta)
    assert np.allclose(np.abs(a["Y2"]), np.abs(Z.T @ Ut), rtol=0, atol=1e-10 * np.abs(Z.T @ Ut).max())
    assert a["nnz"] == np.count_nonzero(O.hard_threshold(inst.D - Lk, zeta))
    assert a["err"] == pytest.approx(O.relative_error(inst.D, Lk, O.hard_threshold(inst.D - Lk, zeta)), rel=1e-12)
