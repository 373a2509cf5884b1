"""Pins of the soft-gate reference pass (CPU): hard limit equals Eq. (10) and the main
oracle's step, the gate value at the threshold, and autograd against finite differences."""
import numpy as np
import pytest
import torch

import synth
from oracle import accaltproj as O
from oracle import learned as OL


def _setup(m=60, n=50, r=3, seed=0):
    inst = synth.planted_instance(m, n, r, 0.1, 1.0, seed)
    p = inst.params()
    ini = O.initialize(inst.D, r, p["beta_init"], p["beta"])
    U, s, V = ini["U"], ini["sigma"], ini["V"]
    Ut, Vt = O.trimmed_bases(U, V, p["mu"], r)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x))
    return inst, p, t(inst.D), t(U * s), t(V), t(Ut), t(Vt), ini["zeta"], (U, s, V)


def test_hard_limit_matches_oracle_step():
    inst, p, D, W, V, Ut, Vt, zeta, (U, s, Vn) = _setup()
    Y1, Y2, res2, nnz = OL.soft_pass(D, W, V, Ut, Vt, zeta, 0.0)
    st = O.step(inst.D, U, s, Vn, zeta, 0, 3, p["beta"], p["gamma"], p["mu"])
    assert np.allclose(Y1.numpy(), st["ZV"], rtol=1e-12, atol=1e-10)
    assert np.allclose(Y2.numpy(), st["ZtU"], rtol=1e-12, atol=1e-10)
    assert nnz == np.count_nonzero(st["S"])
    assert np.sqrt(float(res2)) / np.linalg.norm(inst.D) == pytest.approx(st["err"], rel=1e-12)
    # small tau approaches the hard threshold
    Y1s, _, _, _ = OL.soft_pass(D, W, V, Ut, Vt, zeta, 1e-6)
    assert np.allclose(Y1s.numpy(), st["ZV"], rtol=1e-6, atol=1e-6 * np.abs(st["ZV"]).max())


def test_gate_is_one_half_at_threshold():
    D = torch.tensor([[2.0, -2.0, 0.5]], dtype=torch.float64)
    W = torch.zeros(1, 1, dtype=torch.float64)
    V = torch.zeros(3, 1, dtype=torch.float64)
    I1 = torch.ones(1, 1, dtype=torch.float64)
    Vt = torch.eye(3, 1, dtype=torch.float64)
    Y1, Y2, res2, nnz = OL.soft_pass(D, W, V, I1, Vt, 2.0, 0.1)
    # Z = D - R g with R = D and g = 1/2 at |R| = zeta
    assert float(Y1[0, 0]) == pytest.approx(1.0)
    assert nnz == 0


def test_autograd_matches_central_differences():
    inst, p, D, W, V, Ut, Vt, zeta, _ = _setup(seed=3)
    rng = np.random.default_rng(0)
    Y1b = torch.from_numpy(rng.standard_normal(tuple(W.shape)))
    Y2b = torch.from_numpy(rng.standard_normal(tuple(V.shape)))
    resb = 0.7
    tau = 0.1
    gW, gV, gUt, gVt, gz = OL.soft_pass_vjp(D, W, V, Ut, Vt, zeta, tau, Y1b, Y2b, resb)

    def J(W, V, Ut, Vt, z):
        Y1, Y2, res2, _ = OL.soft_pass(D, W, V, Ut, Vt, z, tau)
        return float((Y1b * Y1).sum() + (Y2b * Y2).sum() + resb * res2)

    h = 1e-6
    for name, base, g in (("W", W, gW), ("V", V, gV), ("Ut", Ut, gUt), ("Vt", Vt, gVt)):
        d = torch.from_numpy(rng.standard_normal(tuple(base.shape)))
        args = {"W": W, "V": V, "Ut": Ut, "Vt": Vt}
        plus = dict(args, **{name: base + h * d})
        minus = dict(args, **{name: base - h * d})
        fd = (J(plus["W"], plus["V"], plus["Ut"], plus["Vt"], zeta) - J(minus["W"], minus["V"], minus["Ut"], minus["Vt"], zeta)) / (2 * h)
        assert float((g * d).sum()) == pytest.approx(fd, rel=1e-6, abs=1e-8)
    hz = 1e-7 * zeta
    fdz = (J(W, V, Ut, Vt, zeta + hz) - J(W, V, Ut, Vt, zeta - hz)) / (2 * hz)
    assert gz == pytest.approx(fdz, rel=1e-6, abs=1e-8)


# ---------------------------------------------------------------------------------------
# Threshold network and training loss of the learned schedule
# ---------------------------------------------------------------------------------------

def _theta(rng, out_scale=0.3):
    th = torch.from_numpy(rng.uniform(-0.4, 0.4, 1313))
    th[1280:1312] *= out_scale / 0.4
    return th


def test_schedule_network_reduces_to_the_paper_rule():
    rng = np.random.default_rng(0)
    th = _theta(rng)
    s = torch.from_numpy(rng.standard_normal((9, 6)))
    plain = torch.from_numpy(rng.uniform(0.1, 2.0, 9))
    # zero output layer: g = 0 and the schedule is Algorithm 1's own
    z = th.clone()
    z[1280:] = 0.0
    assert torch.equal(OL.learned_zeta(z, s, plain), plain)
    # a saturated output is clamped to a factor of 4 either way
    big = z.clone()
    big[1312] = 50.0
    assert torch.allclose(OL.learned_zeta(big, s, plain), 4.0 * plain, rtol=1e-15)
    big[1312] = -50.0
    assert torch.allclose(OL.learned_zeta(big, s, plain), plain / 4.0, rtol=1e-15)
    # the packing: output = w3 . h2 + b3 with h2 from a hand-evaluated first unit path
    W1, b1, W2, b2, w3, b3 = OL.unpack_schedule(th)
    h1 = np.tanh(W1.numpy() @ s[0].numpy() + b1.numpy())
    h2 = np.tanh(W2.numpy() @ h1 + b2.numpy())
    assert float(OL.schedule_net(th, s[:1])[0]) == pytest.approx(float(w3.numpy() @ h2 + float(b3)), rel=1e-14)


def test_schedule_network_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    th = _theta(rng).requires_grad_(True)
    s = torch.from_numpy(rng.standard_normal((7, 6)))
    plain = torch.from_numpy(rng.uniform(0.1, 2.0, 7))
    zb = torch.from_numpy(rng.standard_normal(7))
    (zb * OL.learned_zeta(th, s, plain)).sum().backward()
    d = torch.from_numpy(rng.standard_normal(1313))
    h = 1e-6
    f = lambda t: float((zb * OL.learned_zeta(t, s, plain)).sum())
    fd = (f(th.detach() + h * d) - f(th.detach() - h * d)) / (2 * h)
    assert float((th.grad * d).sum()) == pytest.approx(fd, rel=1e-7)


def test_projection_loss_is_the_tangent_projection_error():
    rng = np.random.default_rng(2)
    m, n, r, rp = 30, 24, 3, 2
    Ut = np.linalg.qr(rng.standard_normal((m, r)))[0]
    Vt = np.linalg.qr(rng.standard_normal((n, r)))[0]
    Z = rng.standard_normal((m, n))
    P, Q = rng.standard_normal((m, rp)), rng.standard_normal((n, rp))
    t = torch.from_numpy
    got = OL.projection_loss(t(Z @ Vt), t(Z.T @ Ut), t(Ut), t(Vt), t(P), t(Q))
    want = np.linalg.norm(O.tangent_project(Z, Ut, Vt) - P @ Q.T) ** 2 / np.linalg.norm(P @ Q.T) ** 2
    assert float(got) == pytest.approx(want, rel=1e-12)
    # gradient in Y1, Y2 against central differences
    Y1 = t(Z @ Vt).requires_grad_(True)
    Y2 = t(Z.T @ Ut).requires_grad_(True)
    OL.projection_loss(Y1, Y2, t(Ut), t(Vt), t(P), t(Q)).backward()
    d1, d2 = t(rng.standard_normal((m, r))), t(rng.standard_normal((n, r)))
    f = lambda a, b: float(OL.projection_loss(a, b, t(Ut), t(Vt), t(P), t(Q)))
    h = 1e-6
    fd = (f(Y1.detach() + h * d1, Y2.detach() + h * d2) - f(Y1.detach() - h * d1, Y2.detach() - h * d2)) / (2 * h)
    assert float((Y1.grad * d1).sum() + (Y2.grad * d2).sum()) == pytest.approx(fd, rel=1e-7)
