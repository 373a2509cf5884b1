"""Robust PCA from a subset of the entries on the GPU (an entry of D that is NaN is
unobserved) against the FP64 oracle of oracle/partial.py at the same iteration count:
relative Frobenius error of L 1e-10 in FP64 and 1e-5 in FP32, supports equal outside the tie
band, and every support entry observed."""
import numpy as np
import pytest
import torch

import synth
from oracle import partial as OP
from parity_helpers import factored_rel_err, rel_fro, support_mismatch

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1711_05519_gb300")


def _case(m, n, r, alpha, p_obs, seed):
    inst = synth.planted_instance(m, n, r, alpha, 1.0, seed)
    obs = np.random.default_rng(seed + 100).random((m, n)) < p_obs
    Dn = inst.D.copy()
    Dn[~obs] = np.nan
    return inst, obs, Dn


@pytest.mark.parametrize("prec,tol,ltol,kind", [("fp64", 1e-10, 1e-10, "simt"), ("fp32", 1e-5, 1e-5, "tensor"),
                                                ("fp32", 1e-5, 1e-5, "simt")])
def test_partial_observation_matches_oracle(prec, tol, ltol, kind):
    r = 4
    inst, obs, Dn = _case(500, 460, r, 0.05, 0.6, 31)
    p = inst.params()
    D = torch.from_numpy(Dn).to("cuda", torch.float64 if prec == "fp64" else torch.float32)
    with P.Solver(p["beta"], p["gamma"], tol, precision=prec, beta_init=p["beta_init"], mu_trim=p["mu"],
                  observed="nan", pass_kind=kind) as s:
        s.init(D, r)
        assert s.pass_kind()[0] == kind
        code, stats = s.run()
        U, sig, V = (t.double().cpu().numpy() for t in s.lowrank())
        idx, _ = (t.cpu().numpy() for t in s.sparse())
    assert code == P.OK and stats[-1]["err"] < tol
    k = stats[-1]["k"]
    Dh = D.double().cpu().numpy()  # the values the GPU read, NaN where unobserved
    full = OP.accaltproj_partial(Dh, obs, r, p["beta"], p["gamma"], tol, p["mu"], beta_init=p["beta_init"])
    assert abs(full["iters"] - k) <= 1
    ref = OP.accaltproj_partial(Dh, obs, r, p["beta"], p["gamma"], 0.0, p["mu"], beta_init=p["beta_init"], max_iter=k)
    L = (U * sig) @ V.T
    assert rel_fro(L, ref["L"]) < ltol
    # err_k carries the absolute error of L relative to ||D|| (1e-6 in FP32)
    assert np.allclose([x["err"] for x in stats], ref["history"]["err"], rtol=1e-6 if prec == "fp64" else 1e-3,
                       atol=1e-12 if prec == "fp64" else 2e-6)
    assert obs.reshape(-1)[idx].all()
    diff, ok = support_mismatch(idx, Dh, ref["L"], ref["zeta"], band_abs_rel_D=0.0 if prec == "fp64" else 1e-6)
    assert ok, diff[:10]
    # exact recovery of the planted L* from 60% of the entries
    assert factored_rel_err(U, sig, V, inst.P, inst.Q) < 10 * ltol


def test_partial_observation_one_step_at_larger_size():
    """2000 x 2000, r = 5, 50% observed, FP32 tensor-core pass: one iteration from the GPU's
    own state against the oracle's step from the same state."""
    r = 5
    inst, obs, Dn = _case(2000, 2000, r, 0.05, 0.5, 32)
    p = inst.params()
    D = torch.from_numpy(Dn).to("cuda", torch.float32)
    Dh = D.double().cpu().numpy()
    with P.Solver(p["beta"], p["gamma"], 1e-5, precision="fp32", beta_init=p["beta_init"], mu_trim=p["mu"],
                  observed="nan") as s:
        s.init(D, r)
        s.iterate(4)
        U, sig, V = (t.double().cpu().numpy() for t in s.lowrank())
        k, zeta, _ = s.state()
        _, st = s.iterate(1)
        U1, s1, V1 = (t.double().cpu().numpy() for t in s.lowrank())
    o = OP.step(Dh, obs, U, sig, V, zeta, k, r, p["beta"], p["gamma"], p["mu"])
    assert st[0]["err"] == pytest.approx(o["err"], rel=1e-5)
    assert st[0]["sigma1"] == pytest.approx(o["sigma_M"][0], rel=1e-5)
    assert rel_fro((U1 * s1) @ V1.T, (o["U"] * o["sigma"]) @ o["V"].T) < 1e-5
    assert st[0]["zeta"] == pytest.approx(zeta, rel=1e-12)
