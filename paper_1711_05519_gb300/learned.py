"""Learned threshold schedule for an unrolled AccAltProj.

A small network g_theta maps per-iteration statistics to a multiplier of the paper's
threshold (Algorithm 1):

    zeta_{k+1} = beta (sigma_{r+1} + gamma^{k+1} sigma_1) * exp(clamp(g_theta(s_k), -log 4, log 4))

with s_k = [log sigma_1, log(sigma_{r+1}/sigma_1), log err_k, fraction of the support that
changed, k/K, log(zeta_k/sigma_1)].  The plain schedule is g = 0 (the output layer starts at
zero, so an untrained network reproduces it).

Training unrolls K iterations.  The m x n work of each iteration is the library's pass with
the soft gate g(R; zeta) = sigmoid((|R| - zeta)/(tau zeta)) (rpca_learn_pass) and its
hand-written adjoint (rpca_learn_pass_adjoint) behind `LearnPass`, a torch.autograd.Function.
The loss of iteration k is the relative distance of the tangent-space projection
P_T(D - S_k(zeta_k)) to the planted L*, computed from the pass products alone (the
projection has rank <= 2r); the factors between iterations are checkpointed and detached,
so each zeta_k is judged by the projection it produces (truncated back-propagation of
depth one).  The O((m + n) r) algebra of the unrolled iterations (trim, QR, 2r x 2r SVD,
loss) uses torch tensor ops on the GPU; every m x n step runs in the library's kernels.
"""
from __future__ import annotations

import ctypes
import math

import torch

from .rpca import CUDA_ERR, RpcaError, _check, lib

LOG4 = math.log(4.0)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dtype_code(t):
    return {torch.float32: 1, torch.float64: 0}[t.dtype]


def _bind():
    L = lib()
    if getattr(L, "_learn_bound", False):
        return L
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    L.rpca_learn_pass.argtypes = [vp, i64, i64, i64, i32, i32, vp, vp, vp, vp, vp, dbl, vp, vp, vp, vp, vp, vp]
    L.rpca_learn_pass.restype = i32
    L.rpca_learn_pass_adjoint.argtypes = [vp, i64, i64, i64, i32, i32, vp, vp, vp, vp, vp, dbl, vp, vp, dbl, vp, vp,
                                          vp, vp, vp, vp]
    L.rpca_learn_pass_adjoint.restype = i32
    L._learn_bound = True
    return L


def learn_pass(D, W, V, Ut, Vt, zeta, tau, mask_old=None, mask_new=None):
    """Forward pass (no autograd): returns Y1, Y2 and stats [res2, hard nnz, changes]."""
    L = _bind()
    m, n = D.shape
    R = W.shape[1]
    Y1 = torch.empty(m, R, dtype=D.dtype, device=D.device)
    Y2 = torch.empty(n, R, dtype=D.dtype, device=D.device)
    stats = torch.empty(4, dtype=torch.float64, device=D.device)
    _check(L.rpca_learn_pass(_ptr(D), m, n, D.stride(0), _dtype_code(D), R, _ptr(W), _ptr(V), _ptr(Ut), _ptr(Vt),
                             _ptr(zeta), float(tau), _ptr(Y1), _ptr(Y2), _ptr(stats), _ptr(mask_old), _ptr(mask_new),
                             _stream()), "rpca_learn_pass")
    return Y1, Y2, stats


def learn_pass_adjoint(D, W, V, Ut, Vt, zeta, tau, Y1b, Y2b, resb):
    L = _bind()
    m, n = D.shape
    R = W.shape[1]
    Utb, Wb = (torch.empty(m, R, dtype=D.dtype, device=D.device) for _ in range(2))
    Vtb, Vb = (torch.empty(n, R, dtype=D.dtype, device=D.device) for _ in range(2))
    zb = torch.empty((), dtype=torch.float64, device=D.device)
    Y1c, Y2c = Y1b.contiguous(), Y2b.contiguous()  # keep the copies alive until the kernel is enqueued
    _check(L.rpca_learn_pass_adjoint(_ptr(D), m, n, D.stride(0), _dtype_code(D), R, _ptr(W), _ptr(V), _ptr(Ut),
                                     _ptr(Vt), _ptr(zeta), float(tau), _ptr(Y1c), _ptr(Y2c), float(resb), _ptr(Utb),
                                     _ptr(Vtb), _ptr(Wb), _ptr(Vb), _ptr(zb), _stream()), "rpca_learn_pass_adjoint")
    return Utb, Vtb, Wb, Vb, zb


class LearnPass(torch.autograd.Function):
    """(D, W, V, U~, V~, zeta) -> (Y1 = Z V~, Y2 = Z^T U~, res2), Z = D - R sigmoid(...)."""

    @staticmethod
    def forward(ctx, D, W, V, Ut, Vt, zeta, tau):
        W, V, Ut, Vt = (x.contiguous() for x in (W, V, Ut, Vt))
        zeta_d = zeta.detach().to(torch.float64).reshape(()).contiguous()
        Y1, Y2, stats = learn_pass(D, W, V, Ut, Vt, zeta_d, tau)
        ctx.save_for_backward(D, W, V, Ut, Vt, zeta_d)
        ctx.tau = tau
        ctx.zeta_shape = zeta.shape
        ctx.zeta_dtype = zeta.dtype
        return Y1, Y2, stats[0].clone()

    @staticmethod
    def backward(ctx, gY1, gY2, gres):
        D, W, V, Ut, Vt, zeta = ctx.saved_tensors
        if gY1 is None:
            gY1 = torch.zeros_like(W[:, :1].expand(-1, W.shape[1]))
        if gY2 is None:
            gY2 = torch.zeros_like(V[:, :1].expand(-1, V.shape[1]))
        resb = float(gres) if gres is not None else 0.0
        Utb, Vtb, Wb, Vb, zb = learn_pass_adjoint(D, W, V, Ut, Vt, zeta, ctx.tau, gY1.to(D.dtype), gY2.to(D.dtype),
                                                  resb)
        return None, Wb, Vb, Utb, Vtb, zb.to(ctx.zeta_dtype).reshape(ctx.zeta_shape), None


class ThresholdMLP(torch.nn.Module):
    """6 -> 32 -> 32 -> 1 (tanh); the output layer starts at zero (plain schedule)."""

    def __init__(self, hidden: int = 32):
        super().__init__()
        self.net = torch.nn.Sequential(torch.nn.Linear(6, hidden), torch.nn.Tanh(), torch.nn.Linear(hidden, hidden),
                                       torch.nn.Tanh(), torch.nn.Linear(hidden, 1))
        torch.nn.init.zeros_(self.net[-1].weight)
        torch.nn.init.zeros_(self.net[-1].bias)

    def forward(self, s):
        return torch.clamp(self.net(s), -LOG4, LOG4).squeeze(-1)


# ---------------------------------------------------------------------------------------
# O((m + n) r) algebra of one iteration (Section 2.1), torch ops, FP64
# ---------------------------------------------------------------------------------------

def trimmed_bases(U, V, mu, r, trim=True):
    """Trim (Algorithm 2) and orthonormal bases of the trimmed factors."""
    if not trim:
        return U, V
    m, n = U.shape[0], V.shape[0]
    cu, cv = math.sqrt(mu * r / m), math.sqrt(mu * r / n)
    A = U * torch.clamp(cu / U.norm(dim=1, keepdim=True).clamp_min(1e-300), max=1.0)
    B = V * torch.clamp(cv / V.norm(dim=1, keepdim=True).clamp_min(1e-300), max=1.0)
    return torch.linalg.qr(A)[0], torch.linalg.qr(B)[0]


def tangent_update(Y1, Y2, Ut, Vt, r):
    """H_r(P_T Z) from Y1 = Z V~, Y2 = Z^T U~ by the QR + 2r x 2r SVD route."""
    C = Ut.T @ Y1
    Q1, R1 = torch.linalg.qr(Y1 - Ut @ C)
    Q2, R2 = torch.linalg.qr(Y2 - Vt @ C.T)
    Z0 = torch.zeros(r, r, dtype=Y1.dtype, device=Y1.device)
    M = torch.cat([torch.cat([C, R2.T], 1), torch.cat([R1, Z0], 1)], 0)
    UM, s, VMt = torch.linalg.svd(M)
    U = torch.cat([Ut, Q1], 1) @ UM[:, :r]
    V = torch.cat([Vt, Q2], 1) @ VMt.T[:, :r]
    return U, s[:r], V, s


def projection_loss(Y1, Y2, Ut, Vt, P, Q, normL2):
    """||P_T Z - L*||_F^2 / ||L*||_F^2 with P_T Z = [U~, Y1 - U~C] [Y2, V~]^T (Eq. (6))
    and L* = P Q^T, from small Gram products only."""
    C = Ut.T @ Y1
    F = torch.cat([Ut, Y1 - Ut @ C], 1)
    G = torch.cat([Y2, Vt], 1)
    ff = F.T @ F
    gg = G.T @ G
    cross = (F.T @ P) @ (Q.T @ G)
    return (torch.trace(ff @ gg) - 2.0 * torch.trace(cross) + normL2) / normL2


class Unrolled:
    """K iterations of AccAltProj from the library's initialisation, with the plain or a
    learned threshold schedule."""

    def __init__(self, D, r, beta, gamma, mu, K=12, tau=0.05, pass_dtype=torch.float32, trim=True):
        self.D = D.to(pass_dtype).contiguous()
        self.r, self.beta, self.gamma, self.mu, self.K, self.tau = r, beta, gamma, mu, K, tau
        self.trim = trim
        from .rpca import Solver

        with Solver(beta, gamma, 0.0, precision="fp64" if pass_dtype == torch.float64 else "fp32",
                    beta_init=2 * beta, mu_trim=mu) as s:
            s.init(self.D, r)
            U, sig, V = s.lowrank()
        self.U0, self.s0, self.V0 = U, sig, V
        m, n = D.shape
        self.words = (n + 31) // 32
        self.mask = [torch.zeros(m * self.words, dtype=torch.int32, device=D.device) for _ in range(2)]
        self.normD = float(torch.linalg.norm(self.D.double()))
        self.R = _padded(r)

    def _pad(self, X):
        if X.shape[1] == self.R:
            return X.to(self.D.dtype).contiguous()
        return torch.nn.functional.pad(X, (0, self.R - X.shape[1])).to(self.D.dtype).contiguous()

    def run(self, mlp=None, P=None, Q=None, hard=False, tol=None, max_iter=None):
        """Runs K iterations (or, with `tol`, until err_k < tol, at most `max_iter`).
        Returns (losses per iteration, final relative error, final factors); with `tol` the
        number of passes run is in self.passes."""
        r = self.r
        K = self.K if tol is None else (max_iter or 100)
        U, s, V = self.U0, self.s0, self.V0
        zeta = torch.tensor(self.beta * float(s[0]), dtype=torch.float64, device=self.D.device)
        normL2 = None
        if P is not None:
            normL2 = torch.trace((P.T @ P) @ (Q.T @ Q))
        losses = []
        err = 1.0
        prev_mask = None
        tau = 0.0 if hard else self.tau
        for k in range(K):
            Ut, Vt = trimmed_bases(U, V, self.mu, r, self.trim)
            W = U * s
            cur = self.mask[k % 2]
            Y1, Y2, stats = learn_pass(self.D, self._pad(W), self._pad(V), self._pad(Ut), self._pad(Vt),
                                       zeta.detach().reshape(()).contiguous(), 0.0, prev_mask, cur)
            err = math.sqrt(max(float(stats[0]), 0.0)) / self.normD
            self.passes = k + 1
            if tol is not None and err < tol:
                break
            change = float(stats[2]) / (self.D.shape[0] * self.D.shape[1]) if prev_mask is not None else 0.0
            prev_mask = cur
            if normL2 is not None and not hard:
                Y1s, Y2s, _ = LearnPass.apply(self.D, self._pad(W), self._pad(V), self._pad(Ut), self._pad(Vt),
                                              zeta, tau)
                losses.append(projection_loss(Y1s[:, :r].double(), Y2s[:, :r].double(), Ut, Vt, P, Q, normL2))
            U, s, V, sM = tangent_update(Y1[:, :r].double(), Y2[:, :r].double(), Ut, Vt, r)
            plain = self.beta * (sM[r] + self.gamma ** (k + 1) * sM[0])
            if mlp is None:
                zeta = plain.detach()
            else:
                feats = torch.stack([torch.log(sM[0]), torch.log(sM[r].clamp_min(1e-300) / sM[0]),
                                     torch.log(torch.tensor(max(err, 1e-300), dtype=torch.float64, device=sM.device)),
                                     torch.tensor(change, dtype=torch.float64, device=sM.device),
                                     torch.tensor((k + 1) / self.K, dtype=torch.float64, device=sM.device),
                                     torch.log(zeta.detach() / sM[0])]).float().detach()
                zeta = plain.detach() * torch.exp(mlp(feats[None])[0].double())
        return losses, err, (U, s, V)


def save_mlp(mlp: "ThresholdMLP", path: str) -> None:
    import numpy as np

    np.savez(path, **{k: v.detach().cpu().numpy() for k, v in mlp.state_dict().items()})


def load_mlp(path: str, device="cuda") -> "ThresholdMLP":
    import numpy as np

    mlp = ThresholdMLP()
    data = np.load(path)
    mlp.load_state_dict({k: torch.from_numpy(data[k]) for k in data.files})
    return mlp.to(device)


def _padded(r: int) -> int:
    for R in (1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 14, 16):
        if R >= r:
            return R
    raise ValueError(r)


def final_error(factors, P, Q):
    U, s, V = factors
    W = U * s
    normL2 = torch.trace((P.T @ P) @ (Q.T @ Q))
    d2 = torch.trace((W.T @ W) @ (V.T @ V)) - 2 * torch.trace((W.T @ P) @ (Q.T @ V)) + normL2
    return float(torch.sqrt(d2.clamp_min(0) / normL2))


def train(instances, K=12, steps=100, lr=1e-2, tau=0.05, seed=0, log=None):
    """Trains a ThresholdMLP on planted instances: list of dicts with D (CUDA), r, beta,
    gamma, mu, P, Q (CUDA FP64)."""
    torch.manual_seed(seed)
    dev = instances[0]["D"].device
    mlp = ThresholdMLP().to(dev)
    opt = torch.optim.Adam(mlp.parameters(), lr=lr)
    runners = [Unrolled(x["D"], x["r"], x["beta"], x["gamma"], x["mu"], K=K, tau=tau) for x in instances]
    for step in range(steps):
        x = instances[step % len(instances)]
        run = runners[step % len(instances)]
        losses, _, _ = run.run(mlp=mlp, P=x["P"], Q=x["Q"])
        loss = torch.stack([torch.log(l.clamp_min(1e-300)) for l in losses]).mean()
        opt.zero_grad()
        loss.backward()
        opt.step()
        if log is not None:
            log.append(float(loss.detach()))
    return mlp
