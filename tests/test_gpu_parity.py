"""GPU versus FP64-oracle parity through the C ABI (needs a GB300 and the built library).

Tolerances (relative Frobenius error of L against the oracle at the same iteration count):
1e-10 in FP64 mode and 1e-5 in FP32 mode.  Supports must agree exactly except for entries
whose residual lies within the tie band around the threshold (1e-6 zeta_k, plus the FP32
rounding of R_ij, 1e-6 max(|D_ij|, |L_ij|), in FP32 mode).
"""
import numpy as np
import pytest
import torch

import synth
from oracle import accaltproj as O
from parity_helpers import rel_fro, support_mismatch

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1711_05519_gb300")


def _solver(p, prec, tol, **kw):
    return P.Solver(p["beta"], p["gamma"], tol, precision=prec, beta_init=p["beta_init"], mu_trim=p["mu"], **kw)


def _gpu_run(inst, prec, tol, r=None, **kw):
    p = inst.params()
    r = r or inst.r
    dt = torch.float64 if prec == "fp64" else torch.float32
    D = torch.from_numpy(inst.D).to("cuda", dt)
    with _solver(p, prec, tol, **kw) as s:
        s.init(D, r)
        kinds = s.pass_kind()
        code, stats = s.run()
        U, sig, V = (t.cpu().numpy() for t in s.lowrank())
        idx, val = (t.cpu().numpy() for t in s.sparse())
    Dh = D.double().cpu().numpy()
    return {"code": code, "stats": stats, "L": (U * sig) @ V.T, "U": U, "sig": sig, "V": V, "idx": idx,
            "val": val, "D": Dh, "kinds": kinds}


def _oracle_same_k(D, inst, k, r=None, **kw):
    p = inst.params()
    return O.accaltproj(D, r or inst.r, p["beta"], p["gamma"], 0.0, p["mu"], beta_init=p["beta_init"], max_iter=k,
                        **kw)


def test_fp64_config1_end_to_end():
    """500 x 500, r = 5, alpha = 0.1, c = 1, seed 0, stop at 1e-10."""
    inst = synth.planted_instance(500, 500, 5, 0.1, 1.0, 0)
    g = _gpu_run(inst, "fp64", 1e-10)
    assert g["code"] == P.OK
    k = g["stats"][-1]["k"]
    assert g["stats"][-1]["err"] < 1e-10
    full = O.accaltproj(inst.D, 5, inst.params()["beta"], inst.params()["gamma"], 1e-10, inst.params()["mu"],
                        beta_init=inst.params()["beta_init"])
    assert abs(full["iters"] - k) <= 1
    ref = _oracle_same_k(inst.D, inst, k)
    assert rel_fro(g["L"], ref["L"]) < 1e-10
    diff, ok = support_mismatch(g["idx"], inst.D, ref["L"], ref["zeta"])
    assert ok, diff
    assert rel_fro(g["L"], inst.L) < 1e-9
    # per-iteration error history agrees
    errs = np.array([s["err"] for s in g["stats"]])
    assert np.allclose(errs, ref["history"]["err"], rtol=1e-6, atol=1e-14)


def test_fp64_init_matches_algorithm3():
    inst = synth.planted_instance(300, 260, 4, 0.1, 1.0, 3)
    p = inst.params()
    D = torch.from_numpy(inst.D).cuda()
    with _solver(p, "fp64", 1e-10) as s:
        s.init(D, 4)
        U, sig, V = (t.cpu().numpy() for t in s.lowrank())
        idx, _ = (t.cpu().numpy() for t in s.sparse())
        _, st = s.iterate(1)
    ref = O.initialize(inst.D, 4, p["beta_init"], p["beta"])
    L0 = (ref["U"] * ref["sigma"]) @ ref["V"].T
    assert rel_fro((U * sig) @ V.T, L0) < 1e-10
    assert st[0]["zeta"] == pytest.approx(ref["zeta"], rel=1e-12)
    diff, ok = support_mismatch(idx, inst.D, L0, ref["zeta"])
    assert ok, diff


def test_fp64_one_step_from_gpu_state():
    """The oracle takes the GPU's own state after k passes and performs pass k; the GPU's
    S_k, err_k, L_{k+1} and spectrum of M_k must match it."""
    inst = synth.planted_instance(400, 350, 5, 0.15, 1.0, 5)
    p = inst.params()
    D = torch.from_numpy(inst.D).cuda()
    with _solver(p, "fp64", 0.0) as s:
        s.init(D, 5)
        for k in range(0, 12):
            U, sig, V = (t.cpu().numpy() for t in s.lowrank())
            idx, val = (t.cpu().numpy() for t in s.sparse())
            _, st = s.iterate(1)
            U1, sig1, V1 = (t.cpu().numpy() for t in s.lowrank())
            o = O.step(inst.D, U, sig, V, st[0]["zeta"], k, 5, p["beta"], p["gamma"], p["mu"])
            assert st[0]["k"] == k
            assert st[0]["err"] == pytest.approx(o["err"], rel=1e-9)
            diff, ok = support_mismatch(idx, inst.D, (U * sig) @ V.T, st[0]["zeta"])
            assert ok, (k, diff)
            assert st[0]["nnz"] == len(idx)
            assert st[0]["sigma1"] == pytest.approx(o["sigma_M"][0], rel=1e-11)
            assert st[0]["sigma_r1"] == pytest.approx(o["sigma_M"][5], rel=1e-9, abs=1e-12 * o["sigma_M"][0])
            assert rel_fro((U1 * sig1) @ V1.T, (o["U"] * o["sigma"]) @ o["V"].T) < 1e-11


def test_fp32_config1_matches_oracle():
    inst = synth.planted_instance(500, 500, 5, 0.1, 1.0, 0)
    g = _gpu_run(inst, "fp32", 1e-5)
    k = g["stats"][-1]["k"]
    assert g["stats"][-1]["err"] < 1e-5
    ref = _oracle_same_k(g["D"], inst, k)
    assert rel_fro(g["L"], ref["L"]) < 1e-5
    diff, ok = support_mismatch(g["idx"], g["D"], ref["L"], ref["zeta"], band_abs_rel_D=1e-6)
    assert ok, diff


@pytest.mark.parametrize("m,n,r", [(384, 320, 7), (256, 512, 8), (256, 384, 9), (384, 320, 10), (300, 512, 12),
                                   (512, 448, 16)])
def test_fp32_tensor_pass_ranks_7_to_16(m, n, r):
    # r = 7, 8: initialisation pass in the rank-16 image layout, iteration pass in the rank-8
    # one (two image sets); r >= 9: both passes in the rank-16 layout (3 stages, N32 Y
    # accumulators, 10 column tiles per CTA at most)
    inst = synth.planted_instance(m, n, r, 0.08, 1.0, m + n + r)
    g = _gpu_run(inst, "fp32", 1e-5)
    assert g["kinds"] == ("tensor", "tensor")
    assert g["stats"][-1]["err"] < 1e-5
    ref = _oracle_same_k(g["D"], inst, g["stats"][-1]["k"])
    assert rel_fro(g["L"], ref["L"]) < 1e-5
    diff, ok = support_mismatch(g["idx"], g["D"], ref["L"], ref["zeta"], band_abs_rel_D=1e-6)
    assert ok, diff


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("m,n,r", [(333, 217, 3), (129, 515, 2), (600, 97, 1), (257, 263, 7)])
def test_ragged_shapes(prec, m, n, r):
    inst = synth.planted_instance(m, n, r, 0.08, 1.0, m + n)
    tol = 1e-10 if prec == "fp64" else 1e-5
    g = _gpu_run(inst, prec, tol)
    k = g["stats"][-1]["k"]
    assert g["stats"][-1]["err"] < tol
    ref = _oracle_same_k(g["D"], inst, k)
    assert rel_fro(g["L"], ref["L"]) < (1e-10 if prec == "fp64" else 1e-5)
    diff, ok = support_mismatch(g["idx"], g["D"], ref["L"], ref["zeta"],
                                band_abs_rel_D=0.0 if prec == "fp64" else 1e-6)
    assert ok, diff


def test_large_rank_no_trim_and_simple_threshold():
    inst = synth.planted_instance(220, 200, 16, 0.05, 1.0, 2)
    for kw in ({"trim": False}, {"zeta_mode": "simple"}):
        g = _gpu_run(inst, "fp64", 1e-9, **kw)
        k = g["stats"][-1]["k"]
        okw = {"do_trim": kw.get("trim", True), "zeta_mode": kw.get("zeta_mode", "paper")}
        ref = _oracle_same_k(inst.D, inst, k, **okw)
        assert rel_fro(g["L"], ref["L"]) < 1e-9
        assert g["stats"][-1]["err"] < 1e-9


def test_invalid_arguments_and_capacity():
    inst = synth.planted_instance(64, 64, 2, 0.1, 1.0, 1)
    p = inst.params()
    D = torch.from_numpy(inst.D).cuda()
    with _solver(p, "fp64", 1e-8) as s:
        for r in (0, 17, 33):
            with pytest.raises(P.RpcaError) as e:
                s.init(D, r)
            assert e.value.code == P.INVALID_ARG
        with pytest.raises(P.RpcaError) as e:
            s.iterate(1)
        assert e.value.code == P.STATE
        s.init(D, 2)
        s.run()
        import ctypes
        nnz = ctypes.c_int64(0)
        code = P.lib().rpca_get_sparse(s._ctx, None, None, 0, ctypes.byref(nnz))
        assert code == P.CAPACITY and nnz.value > 0


def test_nan_in_D_is_reported():
    inst = synth.planted_instance(64, 80, 2, 0.1, 1.0, 1)
    Dn = inst.D.copy()
    Dn[3, 7] = np.nan
    p = inst.params()
    with _solver(p, "fp32", 1e-6, init_max_passes=3) as s:
        with pytest.raises(P.RpcaError) as e:
            s.init(torch.from_numpy(Dn).float().cuda(), 2)
            s.run()
        assert e.value.code == P.NUMERICAL


def test_solve_device_and_host_entry_points():
    inst = synth.planted_instance(300, 280, 3, 0.1, 1.0, 8)
    p = inst.params()
    D = torch.from_numpy(inst.D).float()
    out_d = P.solve(D.cuda(), 3, p["beta"], p["gamma"], 1e-5)
    out_h = P.solve_host(D.pin_memory(), 3, p["beta"], p["gamma"], 1e-5, s_cap=300 * 280)
    assert out_d["status"] == P.OK and out_h["status"] == P.OK
    assert out_d["iters"] == out_h["iters"] and out_d["err"] < 1e-5
    Ld = (out_d["U"].cpu().numpy() * out_d["sigma"].cpu().numpy()) @ out_d["V"].cpu().numpy().T
    Lh = (out_h["U"].numpy() * out_h["sigma"].numpy()) @ out_h["V"].numpy().T
    assert np.array_equal(Ld, Lh)
    assert np.array_equal(out_d["idx"].cpu().numpy(), out_h["idx"][: out_h["nnz"]].numpy())
    assert rel_fro(Ld, inst.L) < 1e-4


def test_host_entry_point_keeps_and_regrows_its_buffers():
    # rpca_solve_host keeps its device buffers between calls: a larger problem regrows them,
    # a smaller one reuses them, and after the release the next call allocates again; each
    # result equals the device entry point's on the same input
    cases = [(300, 250, 3, 31), (420, 380, 5, 32), (300, 250, 3, 31)]
    for i, (m, n, r, seed) in enumerate(cases):
        inst = synth.planted_instance(m, n, r, 0.1, 1.0, seed)
        p = inst.params()
        D = torch.from_numpy(inst.D).float()
        out_d = P.solve(D.cuda(), r, p["beta"], p["gamma"], 1e-5)
        out_h = P.solve_host(D.pin_memory(), r, p["beta"], p["gamma"], 1e-5, s_cap=m * n)
        assert out_h["status"] == out_d["status"] == P.OK
        Ld = (out_d["U"].cpu().numpy() * out_d["sigma"].cpu().numpy()) @ out_d["V"].cpu().numpy().T
        Lh = (out_h["U"].numpy() * out_h["sigma"].numpy()) @ out_h["V"].numpy().T
        assert np.array_equal(Ld, Lh), i
        assert np.array_equal(out_d["idx"].cpu().numpy(), out_h["idx"][: out_h["nnz"]].numpy()), i
        if i == 1:
            P.solve_host_release()



@pytest.mark.parametrize("prec", ["fp32", "fp64", "bf16_split"])
def test_resume_from_factor_checkpoint(prec):
    # a solve interrupted after ck iterations (its process "fails": the context is dropped) and
    # resumed in a new context from the factors and (k, zeta_k, flags) alone ends where the
    # uninterrupted solve ends; the BF16_SPLIT checkpoint is taken after its passes switched
    # to hi + lo
    inst = synth.planted_instance(500, 440, 5, 0.1, 1.0, 41)
    p = inst.params()
    D = torch.from_numpy(inst.D).to("cuda", torch.float64 if prec == "fp64" else torch.float32)
    tol = 1e-10 if prec == "fp64" else 1e-5
    ck = 8 if prec == "bf16_split" else 5
    with _solver(p, prec, tol) as s:
        s.init(D, 5)
        code0, st0 = s.run()
        L0 = [t.cpu().numpy() for t in s.lowrank()]
    with _solver(p, prec, tol) as s:
        s.init(D, 5)
        s.iterate(ck)
        ckpt = [t.clone() for t in s.lowrank()] + list(s.state())
    assert ckpt[3] == ck
    assert ckpt[5] == (P.rpca.STATE_READS_LO if prec == "bf16_split" else 0)
    with _solver(p, prec, tol) as s:
        s.init(D, 5)
        s.set_lowrank(*ckpt)
        assert s.state() == tuple(ckpt[3:])
        code1, st1 = s.run()
        L1 = [t.cpu().numpy() for t in s.lowrank()]
    assert code0 == code1 == P.OK
    assert st1[0]["k"] == ck and st1[-1]["k"] == st0[-1]["k"]
    # same iterates up to rounding (Trim and the bases are recomputed from the checkpoint); in
    # single precision the two runs' iterates differ by ~1e-7 relative, which moves err_k by
    # up to ~1e-8 absolute
    assert [x["err"] for x in st1] == pytest.approx([x["err"] for x in st0[ck:]], rel=1e-3,
                                                    abs=0.0 if prec == "fp64" else 1e-7)
    A, B = [(U * s) @ V.T for U, s, V in (L0, L1)]
    assert rel_fro(B, A) < (1e-9 if prec == "fp64" else 1e-5)


def test_bounded_waits_report_timeout_and_leave_the_context_usable():
    mbar_status, grid_status = P.selftest_waits()
    assert mbar_status == P.TIMEOUT and grid_status == P.TIMEOUT
    inst = synth.planted_instance(200, 180, 3, 0.1, 1.0, 2)
    g = _gpu_run(inst, "fp32", 1e-5)
    assert g["code"] == P.OK


@pytest.mark.parametrize("prec,ltol", [("fp64", 1e-10), ("fp32", 1e-5)])
@pytest.mark.parametrize("m,n,r,seed", [(300, 260, 4, 51), (420, 400, 6, 52)])
def test_rank_deficient_projection_keeps_the_solve_valid(prec, ltol, m, n, r, seed):
    """alpha = 0: D = L* is exactly of rank r, the initialisation finds its column space, and
    (I - U~U~^T) Z V~ vanishes up to rounding, so the QR of Section 2.1 meets a zero R1 (a
    direction lost to rounding; the library drops it as a zero row of R1).  The iteration
    (tol 0, six steps) must stay at L* and agree with the oracle, whose QR completes the
    basis in its own way (only L is compared)."""
    inst = synth.planted_instance(m, n, r, 0.0, 1.0, seed)
    p = inst.params()
    D = torch.from_numpy(inst.D).to("cuda", torch.float64 if prec == "fp64" else torch.float32)
    with _solver(p, prec, 0.0, max_iter=6) as s:
        s.init(D, r)
        code, stats = s.run()
        U, sig, V = (t.cpu().numpy() for t in s.lowrank())
    assert code == P.NOT_CONVERGED and stats[-1]["k"] == 6
    assert all(np.isfinite([x["err"] for x in stats])) and np.isfinite(U).all() and np.isfinite(V).all()
    L = (U * sig) @ V.T
    assert rel_fro(L, inst.L) < ltol
    ref = _oracle_same_k(D.double().cpu().numpy(), inst, 6)
    assert rel_fro(L, ref["L"]) < ltol
