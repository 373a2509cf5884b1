"""The learned threshold schedule on the library (GPU): the network kernels (forward and the
hand-written backward), the training loss kernel and the device-side LEARNED iteration,
each against the FP64 CPU references of oracle/learned.py."""
import numpy as np
import pytest
import torch

import synth
from oracle import learned as OL

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1711_05519_gb300")
from paper_1711_05519_gb300 import learned as PL  # noqa: E402


def _theta(seed, out_scale=0.3):
    th = PL.init_theta(seed)
    g = torch.Generator(device="cpu").manual_seed(seed)
    th[1280:1312] = (out_scale * (2 * torch.rand(32, generator=g) - 1)).cuda()
    th[1312] = 0.05
    return th


def _instance(m, n, r, alpha, seed, dtype=torch.float32):
    inst = synth.planted_instance(m, n, r, alpha, 1.0, seed)
    p = inst.params()
    return {"D": torch.from_numpy(inst.D).to("cuda", dtype), "r": r, "beta": p["beta"], "gamma": p["gamma"],
            "mu": p["mu"], "P": torch.from_numpy(inst.P).cuda(), "Q": torch.from_numpy(inst.Q).cuda()}


def test_schedule_kernels_match_fp64_reference():
    rng = np.random.default_rng(0)
    th = _theta(1, out_scale=0.6)
    n = 13
    s = rng.standard_normal((n, 6)).astype(np.float32)
    s[:, 0] *= 3.0
    s[-1] = 40.0  # drives the output into the clamp
    feats = torch.from_numpy(s).cuda()
    plain = torch.from_numpy(rng.uniform(0.05, 3.0, n)).cuda()
    zb = torch.from_numpy(rng.standard_normal(n)).cuda()
    zeta, g = PL.schedule_forward(th, feats, plain)
    grad = PL.schedule_backward(th, feats, plain, zb)
    th64 = th.double().cpu().requires_grad_(True)
    ref = OL.learned_zeta(th64, torch.from_numpy(s).double(), plain.cpu())
    (zb.cpu() * ref).sum().backward()
    assert np.allclose(zeta.cpu().numpy(), ref.detach().numpy(), rtol=2e-6, atol=0)
    gref = th64.grad.numpy()
    assert np.linalg.norm(grad.double().cpu().numpy() - gref) < 2e-5 * np.linalg.norm(gref)
    # a saturated output contributes nothing through the clamp, and the threshold is the
    # paper's times 4
    sat = th.clone()
    sat[1312] = 50.0
    zs, gs = PL.schedule_forward(sat, feats, plain)
    assert torch.equal(gs.cpu(), torch.full((n,), float(np.float32(np.log(4.0)))))
    assert np.allclose(zs.cpu().numpy(), 4.0 * plain.cpu().numpy(), rtol=1e-6)
    assert float(PL.schedule_backward(sat, feats, plain, zb).abs().max()) == 0.0


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_projection_loss_kernel_matches_reference(dtype):
    rng = np.random.default_rng(2)
    m, n, r, R, rp = 300, 260, 3, 4, 3
    Ut = np.linalg.qr(rng.standard_normal((m, r)))[0]
    Vt = np.linalg.qr(rng.standard_normal((n, r)))[0]
    Z = rng.standard_normal((m, n))
    Pm, Qm = rng.standard_normal((m, rp)), rng.standard_normal((n, rp))
    pad = lambda X: np.hstack([X, np.zeros((X.shape[0], R - r))])
    cu = lambda X: torch.from_numpy(np.ascontiguousarray(pad(X))).to("cuda", dtype)
    Y1, Y2, Utg, Vtg = cu(Z @ Vt), cu(Z.T @ Ut), cu(Ut), cu(Vt)
    loss, Y1b, Y2b = PL.projection_loss(Y1, Y2, Utg, Vtg, torch.from_numpy(Pm).cuda(), torch.from_numpy(Qm).cuda(), r)
    # the reference sees exactly the values the kernel read
    t = [x.double().cpu()[:, :r].clone() for x in (Y1, Y2, Utg, Vtg)]
    t[0].requires_grad_(True)
    t[1].requires_grad_(True)
    ref = OL.projection_loss(*t, torch.from_numpy(Pm), torch.from_numpy(Qm))
    ref.backward()
    assert float(loss) == pytest.approx(float(ref), rel=1e-10)
    tol = 1e-9 if dtype == torch.float64 else 1e-5
    for got, want in ((Y1b, t[0].grad), (Y2b, t[1].grad)):
        got = got.double().cpu()
        assert float((got[:, :r] - want).norm() / want.norm()) < tol
        assert float(got[:, r:].abs().max()) == 0.0


def test_learned_iteration_applies_the_network_on_the_device():
    x = _instance(600, 560, 3, 0.15, 11)
    th = _theta(3)
    ops, stats = PL.unrolled_trace(x, th, 9)
    assert len(stats) == 9
    feats = torch.tensor([st["features"] for st in stats], dtype=torch.float32)
    plain = torch.tensor([st["zeta_next_plain"] for st in stats], dtype=torch.float64)
    zref = OL.learned_zeta(th.double().cpu(), feats.double(), plain).numpy()
    znext = np.array([st["zeta"] for st in stats[1:]])
    assert np.allclose(znext, zref[:-1], rtol=2e-6, atol=0)
    # the kernel used in training reproduces the thresholds the iteration used, bit for bit
    zk, _ = PL.schedule_forward(th, feats.cuda(), plain.cuda())
    assert np.array_equal(zk.cpu().numpy()[:-1], znext)
    # the recorded statistics are the ones the network is defined on
    for k, st in enumerate(stats):
        f = np.array(st["features"])
        assert f[0] == pytest.approx(np.log(st["sigma1"]), rel=1e-6)
        assert f[2] == pytest.approx(np.log(st["err"]), rel=1e-6)
        assert f[4] == pytest.approx((k + 1) / 9, rel=1e-6)
        assert f[5] == pytest.approx(np.log(st["zeta"] / st["sigma1"]), rel=1e-5, abs=1e-6)
        assert f[3] == pytest.approx(st["support_changes"] / (600 * 560), rel=1e-6, abs=1e-9)
    assert stats[0]["support_changes"] == 0 and max(st["support_changes"] for st in stats[1:]) > 0


def test_support_change_count_of_the_pass():
    # the pass's count of support changes against the symmetric difference of the supports
    # extracted before consecutive iterations (pass and extraction may differ only inside the
    # FP32 tie band, a handful of entries)
    x = _instance(500, 480, 4, 0.1, 12)
    th = _theta(4)
    with PL._solver(x, 0.0, 8) as s:
        s.set_schedule(th, 8)
        s.init(x["D"], 4)
        prev, seen = None, 0
        for k in range(6):
            idx = set(s.sparse()[0].cpu().numpy().tolist())
            _, st = s.iterate(1)
            if prev is not None:
                assert abs(st[0]["support_changes"] - len(idx ^ prev)) <= 4
                seen = max(seen, len(idx ^ prev))
            prev = idx
    assert seen > 100  # the supports did move between these iterations


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_zero_output_layer_reproduces_the_paper_schedule(prec):
    dt = torch.float64 if prec == "fp64" else torch.float32
    x = _instance(400, 380, 3, 0.1, 13, dt)
    th = PL.init_theta(5)  # output layer zero: g = 0
    c0, st0, f0 = PL.solve(x, None, tol=1e-5 if prec == "fp32" else 1e-10, precision=prec)
    c1, st1, f1 = PL.solve(x, th, tol=1e-5 if prec == "fp32" else 1e-10, precision=prec)
    assert c0 == c1 == P.OK
    assert [s["err"] for s in st0] == [s["err"] for s in st1]
    assert [s["zeta"] for s in st0] == [s["zeta"] for s in st1]


def test_training_gradient_matches_central_differences():
    """The gradient of the training objective (network -> soft pass -> loss, all by the
    library's backward kernels) against central differences of the forward kernels, with the
    unrolled trajectory held fixed, FP64 passes."""
    x = _instance(200, 200, 3, 0.1, 7, torch.float64)
    th = _theta(6)
    trace = PL.unrolled_trace(x, th, 6, precision="fp64")
    leaf = th.clone().requires_grad_(True)
    J, _, _ = PL.unrolled_loss(x, leaf, 6, 0.05, trace=trace)
    J.backward()
    g = leaf.grad.double()
    d = g / g.norm()
    h = 1e-2  # FP32 parameters: a step well above their rounding
    Jp = float(PL.unrolled_loss(x, (th.double() + h * d).float(), 6, 0.05, trace=trace)[0])
    Jm = float(PL.unrolled_loss(x, (th.double() - h * d).float(), 6, 0.05, trace=trace)[0])
    fd = (Jp - Jm) / (2 * h)
    assert float(g.norm()) == pytest.approx(fd, rel=2e-2)
