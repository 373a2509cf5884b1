"""GPU checks of the soft-gate pass and its hand-written adjoint (rpca_learn_pass,
rpca_learn_pass_adjoint) against the FP64 CPU reference (torch autograd) and against
central finite differences, and of the learned schedule itself."""
import numpy as np
import pytest
import torch

import synth
from oracle import accaltproj as O
from oracle import learned as OL

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1711_05519_gb300")
from paper_1711_05519_gb300 import learned as PL  # noqa: E402


def _case(m=200, n=180, r=3, seed=0, dtype=torch.float64):
    inst = synth.planted_instance(m, n, r, 0.1, 1.0, seed)
    p = inst.params()
    ini = O.initialize(inst.D, r, p["beta_init"], p["beta"])
    U, s, V = ini["U"], ini["sigma"], ini["V"]
    Ut, Vt = O.trimmed_bases(U, V, p["mu"], r)
    cpu = [torch.from_numpy(np.ascontiguousarray(x)) for x in (inst.D, U * s, V, Ut, Vt)]
    gpu = [x.to("cuda", dtype).contiguous() for x in cpu]
    # a threshold inside the bulk of |R| so that many gates are active
    Rabs = np.abs(inst.D - (U * s) @ V.T)
    zeta = float(np.quantile(Rabs, 0.9))
    return cpu, gpu, zeta


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("tau", [0.0, 0.05])
def test_forward_matches_reference(dtype, tau):
    cpu, gpu, zeta = _case(dtype=dtype)
    zt = torch.tensor(zeta, dtype=torch.float64, device="cuda")
    Y1, Y2, stats = PL.learn_pass(*gpu, zt, tau)
    # the reference sees exactly the values the GPU read
    ref = OL.soft_pass(*[g.double().cpu() for g in gpu], zeta, tau)
    tol = 1e-11 if dtype == torch.float64 else 2e-5
    for got, want in ((Y1, ref[0]), (Y2, ref[1])):
        got = got.double().cpu()
        assert float((got - want).norm() / want.norm()) < tol
    assert float(stats[0]) == pytest.approx(float(ref[2]), rel=(1e-11 if dtype == torch.float64 else 1e-4))
    if dtype == torch.float64:
        assert int(stats[1]) == ref[3]


def test_support_masks_count_changes():
    cpu, gpu, zeta = _case()
    m, n = gpu[0].shape
    words = (n + 31) // 32
    ma = torch.zeros(m * words, dtype=torch.int32, device="cuda")
    mb = torch.zeros_like(ma)
    PL.learn_pass(*gpu, torch.tensor(zeta, dtype=torch.float64, device="cuda"), 0.0, None, ma)
    _, _, st = PL.learn_pass(*gpu, torch.tensor(0.7 * zeta, dtype=torch.float64, device="cuda"), 0.0, ma, mb)
    R = (cpu[0] - cpu[1] @ cpu[2].T).abs()
    changed = int(((R > zeta) ^ (R > 0.7 * zeta)).sum())
    assert int(st[2]) == changed > 0
    bits = mb.cpu().numpy().view(np.uint32).reshape(m, words)
    dense = np.unpackbits(bits.view(np.uint8), bitorder="little").reshape(m, words * 32)[:, :n].astype(bool)
    assert np.array_equal(dense, (R > 0.7 * zeta).numpy())


def test_adjoint_matches_fp64_autograd_reference():
    cpu, gpu, zeta = _case(seed=4)
    rng = np.random.default_rng(1)
    Y1b = torch.from_numpy(rng.standard_normal(tuple(cpu[1].shape)))
    Y2b = torch.from_numpy(rng.standard_normal(tuple(cpu[2].shape)))
    tau, resb = 0.05, 0.3
    zt = torch.tensor(zeta, dtype=torch.float64, device="cuda")
    Utb, Vtb, Wb, Vb, zb = PL.learn_pass_adjoint(*gpu, zt, tau, Y1b.cuda(), Y2b.cuda(), resb)
    gW, gV, gUt, gVt, gz = OL.soft_pass_vjp(*cpu, zeta, tau, Y1b, Y2b, resb)
    for got, want in ((Wb, gW), (Vb, gV), (Utb, gUt), (Vtb, gVt)):
        assert float((got.cpu() - want).norm() / want.norm()) < 1e-9
    assert float(zb) == pytest.approx(gz, rel=1e-9)


def test_adjoint_matches_central_differences():
    """Directional derivatives of J = <Y1b, Y1> + <Y2b, Y2> + resb res2 at m = n = 200,
    FP64, by central differences of the GPU forward pass, along directions of unit norm
    mixing the adjoint's own direction with a random one."""
    cpu, gpu, zeta = _case(m=200, n=200, r=3, seed=7)
    D, W, V, Ut, Vt = gpu
    rng = np.random.default_rng(2)
    Y1b = torch.from_numpy(rng.standard_normal(tuple(W.shape))).cuda()
    Y2b = torch.from_numpy(rng.standard_normal(tuple(V.shape))).cuda()
    tau, resb = 0.05, 0.3

    def J(W_, V_, Ut_, Vt_, z):
        Y1, Y2, st = PL.learn_pass(D, W_, V_, Ut_, Vt_, torch.tensor(z, dtype=torch.float64, device="cuda"), tau)
        return float((Y1b * Y1).sum() + (Y2b * Y2).sum() + resb * st[0])

    Utb, Vtb, Wb, Vb, zb = PL.learn_pass_adjoint(D, W, V, Ut, Vt, torch.tensor(zeta, dtype=torch.float64,
                                                 device="cuda"), tau, Y1b, Y2b, resb)
    base = {"W": W, "V": V, "Ut": Ut, "Vt": Vt}
    for name, g in (("W", Wb), ("V", Vb), ("Ut", Utb), ("Vt", Vtb)):
        rnd = torch.from_numpy(rng.standard_normal(tuple(base[name].shape))).cuda()
        d = g / g.norm() + 0.5 * rnd / rnd.norm()
        h = 1e-5 * float(base[name].norm())
        plus = dict(base, **{name: base[name] + h * d})
        minus = dict(base, **{name: base[name] - h * d})
        fd = (J(plus["W"], plus["V"], plus["Ut"], plus["Vt"], zeta) -
              J(minus["W"], minus["V"], minus["Ut"], minus["Vt"], zeta)) / (2 * h)
        assert float((g * d).sum()) == pytest.approx(fd, rel=1e-5), name
    hz = 1e-6 * zeta
    fdz = (J(W, V, Ut, Vt, zeta + hz) - J(W, V, Ut, Vt, zeta - hz)) / (2 * hz)
    assert float(zb) == pytest.approx(fdz, rel=1e-5)


def test_autograd_function_backpropagates_to_zeta():
    cpu, gpu, zeta = _case(seed=9)
    z = torch.tensor(zeta, dtype=torch.float64, device="cuda", requires_grad=True)
    Y1, Y2, res2 = PL.LearnPass.apply(*gpu, z, 0.05)
    (Y1.sum() + 2 * Y2.sum() + res2).backward()
    zc = torch.tensor(zeta, dtype=torch.float64, requires_grad=True)
    r1, r2, rr, _ = OL.soft_pass(*cpu, zc, 0.05)
    (r1.sum() + 2 * r2.sum() + rr).backward()
    assert float(z.grad) == pytest.approx(float(zc.grad), rel=1e-9)
