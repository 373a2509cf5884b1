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


# ---------------------------------------------------------------------------------------
# Threshold network of the learned schedule and its training loss (FP64 references)
# ---------------------------------------------------------------------------------------
LOG4 = 1.3862943611198906


def unpack_schedule(theta):
    """Packed parameters -> (W1 32x6, b1, W2 32x32, b2, w3, b3), the layout of the library."""
    o = [0, 192, 224, 1248, 1280, 1312, 1313]
    W1 = theta[o[0]:o[1]].reshape(32, 6)
    W2 = theta[o[2]:o[3]].reshape(32, 32)
    return W1, theta[o[1]:o[2]], W2, theta[o[3]:o[4]], theta[o[4]:o[5]], theta[o[5]]


def schedule_net(theta, s):
    """g(s) = w3 . tanh(W2 tanh(W1 s + b1) + b2) + b3 for rows s of an n x 6 array."""
    W1, b1, W2, b2, w3, b3 = unpack_schedule(theta)
    h1 = torch.tanh(s @ W1.T + b1)
    h2 = torch.tanh(h1 @ W2.T + b2)
    return h2 @ w3 + b3


def learned_zeta(theta, s, plain):
    """zeta = zeta^plain exp(clamp(g(s), -log 4, log 4))."""
    return plain * torch.exp(torch.clamp(schedule_net(theta, s), -LOG4, LOG4))


def projection_loss(Y1, Y2, Ut, Vt, P, Q):
    """||F G^T - P Q^T||_F^2 / ||P Q^T||_F^2 with F = [U~, Y1 - U~ U~^T Y1], G = [Y2, V~]:
    for Y1 = Z V~ and Y2 = Z^T U~ (orthonormal U~, V~), F G^T is P_T Z of Eq. (6).  Dense
    m x n products; small sizes only."""
    C = Ut.T @ Y1
    F = torch.cat([Ut, Y1 - Ut @ C], 1)
    G = torch.cat([Y2, Vt], 1)
    Ls = P @ Q.T
    return ((F @ G.T - Ls) ** 2).sum() / (Ls ** 2).sum()
