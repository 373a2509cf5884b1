"""FP64 CPU reference of the soft-gate pass used to train a learned threshold schedule.

TEST INFRASTRUCTURE: only the tests may import this module.  Plain PyTorch CPU ops in
float64 with autograd give the reference values and gradients of the library's
rpca_learn_pass / rpca_learn_pass_adjoint.

The pass is the m x n part of one AccAltProj iteration (Section 2.1) with the hard
threshold of Eq. (10) replaced by the gate g(R; zeta) = sigmoid((|R| - zeta) / (tau zeta))
(tau = 0: the hard threshold itself):
    L = W V^T, R = D - L, S = R g, Z = D - S, Y1 = Z V~, Y2 = Z^T U~,
    res2 = ||D - L - S||_F^2, nnz = |{|R| > zeta}|.
"""
import torch


def soft_pass(D, W, V, Ut, Vt, zeta, tau):
    L = W @ V.T
    R = D - L
    if tau > 0:
        g = torch.sigmoid((R.abs() - zeta) / (tau * zeta))
    else:
        g = (R.abs() > zeta).to(D.dtype)
    S = R * g
    Z = D - S
    return Z @ Vt, Z.T @ Ut, ((R - S) ** 2).sum(), int((R.abs() > zeta).sum())


def soft_pass_vjp(D, W, V, Ut, Vt, zeta, tau, Y1b, Y2b, resb):
    """Cotangents of (W, V, U~, V~, zeta) for J = <Y1b, Y1> + <Y2b, Y2> + resb * res2, by
    torch autograd in float64."""
    W, V, Ut, Vt = (x.detach().clone().requires_grad_(True) for x in (W, V, Ut, Vt))
    z = torch.tensor(float(zeta), dtype=torch.float64, requires_grad=True)
    Y1, Y2, res2, _ = soft_pass(D, W, V, Ut, Vt, z, tau)
    J = (Y1b * Y1).sum() + (Y2b * Y2).sum() + resb * res2
    J.backward()
    return W.grad, V.grad, Ut.grad, Vt.grad, float(z.grad)
