"""Parity at the full sizes of the synthetic workloads, through the solver calls the
benchmark times (tensor-core pass).

  2nd workload: m = n = 10^4, r = 5, alpha = 0.1, c = 1, FP32, tol 1e-5.
  3rd workload: m = n = 2*10^4, r = 10, alpha = 0.2, c = 3, D stored as bf16 hi + lo
                (BF16_SPLIT), tol 1e-5.

The FP64 oracle cannot run the whole solve at these sizes in test time, so it checks one
iteration taken from the GPU's own state (S_k, err_k, the spectrum of M_k and L_{k+1}),
and the rest is checked through properties that hold at any size: err_k < tol, linear
decay, L within 1e-5 of the planted L* (which the FP64 oracle recovers to 1e-10 on the
500 x 500 workload), and supp(S_k) inside the planted support (Theorem 1).
Tolerances: FP32 (and bf16 hi + lo once it reads lo): 1e-5 relative for err_k, sigma_1 of
M_k and L_{k+1}; supports exact outside the FP32 tie band.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import accaltproj as O
from parity_helpers import factored_rel_err, rel_fro, support_mismatch

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1711_05519_gb300")


def _check_one_step(s, D64, inst, p, k, r, D_pass=None, support=True):
    """Pass k from the GPU's state against the oracle's step from the same state.  D_pass is
    the D the pass reads (default D64); the sparse output is extracted from D64 and compared
    entry by entry when `support` is set."""
    D_pass = D64 if D_pass is None else D_pass
    U, sig, V = (t.double().cpu().numpy() for t in s.lowrank())
    if support:
        idx, _ = (t.cpu().numpy() for t in s.sparse())
    _, st = s.iterate(1)
    U1, sig1, V1 = (t.double().cpu().numpy() for t in s.lowrank())
    o = O.step(D_pass, U, sig, V, st[0]["zeta"], k, r, p["beta"], p["gamma"], p["mu"])
    assert st[0]["k"] == k
    assert st[0]["err"] == pytest.approx(o["err"], rel=1e-5)
    # entries inside the tie band around zeta_k: the only ones on which the pass (tensor-core
    # rebuild of L), the extraction (FP32 rebuild) and the oracle (FP64) may disagree
    L = (U * sig) @ V.T
    band = 1e-6 * st[0]["zeta"] + 1e-6 * np.maximum(np.abs(D_pass), np.abs(L))
    n_band = int(np.count_nonzero(np.abs(np.abs(D_pass - L) - st[0]["zeta"]) <= band))
    del L, band
    assert abs(st[0]["nnz"] - int(np.count_nonzero(o["S"]))) <= n_band
    if support:
        diff, ok = support_mismatch(idx, D64, (U * sig) @ V.T, st[0]["zeta"], band_abs_rel_D=1e-6)
        assert ok, (k, diff[:10])
        assert abs(st[0]["nnz"] - len(idx)) <= n_band
    assert st[0]["sigma1"] == pytest.approx(o["sigma_M"][0], rel=1e-5)
    assert st[0]["sigma_r1"] == pytest.approx(o["sigma_M"][r], rel=1e-4, abs=1e-6 * o["sigma_M"][0])
    L1 = (U1 * sig1) @ V1.T
    assert rel_fro(L1, (o["U"] * o["sigma"]) @ o["V"].T) < 1e-5
    return st[0]


def _solve_checks(s, inst, errs, r, sample=None):
    errs = np.asarray(errs)
    assert errs[-1] < 1e-5
    # linear decay once the iteration has started to contract
    k0 = int(np.argmax(errs < 0.1))
    assert np.all(errs[k0 + 1:] < 0.7 * errs[k0:-1])
    U, sig, V = (t.double().cpu().numpy() for t in s.lowrank())
    assert factored_rel_err(U, sig, V, inst.P, inst.Q) < 1e-5
    idx, _ = (t.cpu().numpy() for t in s.sparse())
    if sample is not None:
        idx = np.random.default_rng(1).choice(idx, size=min(sample, idx.size), replace=False)
    pos = np.searchsorted(inst.support, idx)  # the planted support is sorted
    assert np.all(inst.support[np.minimum(pos, inst.support.size - 1)] == idx)


def test_fp32_10000_r5():
    inst = synth.planted_instance(10000, 10000, 5, 0.1, 1.0, 0)
    p = inst.params()
    D = torch.from_numpy(inst.D.astype(np.float32)).cuda()
    D64 = D.double().cpu().numpy()
    with P.Solver(p["beta"], p["gamma"], 1e-5, precision="fp32", beta_init=p["beta_init"], mu_trim=p["mu"]) as s:
        s.init(D, 5)
        assert s.pass_kind() == ("tensor", "tensor")
        _, st = s.iterate(6)
        errs = [x["err"] for x in st]
        errs.append(_check_one_step(s, D64, inst, p, 6, 5)["err"])
        code, st = s.run()
        errs += [x["err"] for x in st]
        assert code == P.OK
        _solve_checks(s, inst, errs, 5)


def test_bf16_split_20000_r10():
    inst = synth.planted_instance(20000, 20000, 10, 0.2, 3.0, 0)
    p = inst.params()
    D = torch.from_numpy(inst.D.astype(np.float32)).cuda()
    D64 = D.double().cpu().numpy()
    with P.Solver(p["beta"], p["gamma"], 1e-5, precision="bf16_split", beta_init=p["beta_init"],
                  mu_trim=p["mu"]) as s:
        s.init(D, 10)
        assert s.pass_kind() == ("tensor", "tensor")
        _, st = s.iterate(9)
        errs = [x["err"] for x in st]
        assert errs[-1] < 1e-2  # the passes read hi + lo from here on
        # the D these passes read: hi = bf16(D), lo = bf16(D - hi), both round-to-nearest-even
        hi = D.bfloat16()
        lo = (D - hi.float()).bfloat16()
        D_hl = (hi.double() + lo.double()).cpu().numpy()
        del hi, lo
        errs.append(_check_one_step(s, D64, inst, p, 9, 10, D_pass=D_hl, support=False)["err"])
        code, st = s.run()
        errs += [x["err"] for x in st]
        assert code == P.OK
        _solve_checks(s, inst, errs, 10, sample=1_000_000)
