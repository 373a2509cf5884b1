"""Learned threshold schedule for AccAltProj, trained and run through the library.

A small network g_theta (6 -> 32 -> 32 -> 1, tanh, FP32) maps per-iteration statistics to a
multiplier of the paper's threshold (Algorithm 1):

    zeta_{k+1} = beta (sigma_{r+1} + gamma^{k+1} sigma_1) * exp(clamp(g_theta(s_k), -log 4, log 4))

with s_k = [log sigma_1, log(sigma_{r+1}/sigma_1), log err_k, fraction of the support that
changed since pass k - 1, (k+1)/K, log(zeta_k/sigma_1)].  The plain schedule is g = 0 (a zero
output layer), so an untrained network reproduces it.  The network is evaluated on the device
inside the library's iteration (zeta mode "learned"); nothing of it runs in Python.

Training unrolls K iterations of the library's own iteration in that mode.  For each
iteration k >= 1 it recomputes zeta_k from the recorded statistics s_{k-1} (ScheduleZeta,
rpca_schedule_forward / rpca_schedule_backward), evaluates the m x n pass at the recorded
operands with the soft gate g(R; zeta) = sigmoid((|R| - zeta)/(tau zeta)) (LearnPass,
rpca_learn_pass / rpca_learn_pass_adjoint) and the loss ||P_T(D - S_k(zeta_k)) - L*||_F^2 /
||L*||_F^2 from the pass products (ProjectionLoss, rpca_projection_loss).  The operands of
each iteration are checkpointed (O((m + n) r) per iteration, never an m x n array) and held
fixed, so each zeta_k is judged by the projection it produces (back-propagation truncated to
one iteration).  The objective is the mean of log loss_k; Adam (rpca_adam_step) updates the
parameters.  Every step of the forward and backward computation is a kernel of the library;
torch supplies device memory, streams and the autograd bookkeeping.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from .rpca import SCHEDULE_PARAMS, Solver, _check, lib

LOG4 = math.log(4.0)
HIDDEN, INPUTS = 32, 6


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


# ---------------------------------------------------------------------------------------
# The soft-gated pass and its adjoint
# ---------------------------------------------------------------------------------------

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
            gY1 = torch.zeros_like(W)
        if gY2 is None:
            gY2 = torch.zeros_like(V)
        resb = float(gres) if gres is not None else 0.0
        Utb, Vtb, Wb, Vb, zb = learn_pass_adjoint(D, W, V, Ut, Vt, zeta, ctx.tau, gY1.to(D.dtype), gY2.to(D.dtype),
                                                  resb)
        return None, Wb, Vb, Utb, Vtb, zb.to(ctx.zeta_dtype).reshape(ctx.zeta_shape), None


# ---------------------------------------------------------------------------------------
# The threshold network and the training loss
# ---------------------------------------------------------------------------------------

def schedule_forward(theta, feats, plain):
    """zeta_i = plain_i exp(clamp(g(feats_i))) and the clamped g, by the library's kernel."""
    n = feats.shape[0]
    zeta = torch.empty(n, dtype=torch.float64, device=feats.device)
    g = torch.empty(n, dtype=torch.float32, device=feats.device)
    feats, plain = feats.contiguous(), plain.contiguous()
    _check(lib().rpca_schedule_forward(_ptr(theta), _ptr(feats), _ptr(plain), n, _ptr(zeta), _ptr(g), _stream()),
           "rpca_schedule_forward")
    return zeta, g


def schedule_backward(theta, feats, plain, zeta_bar):
    grad = torch.empty(SCHEDULE_PARAMS, dtype=torch.float32, device=feats.device)
    feats, plain, zeta_bar = feats.contiguous(), plain.contiguous(), zeta_bar.contiguous()
    _check(lib().rpca_schedule_backward(_ptr(theta), _ptr(feats), _ptr(plain), _ptr(zeta_bar), feats.shape[0],
                                        _ptr(grad), _stream()), "rpca_schedule_backward")
    return grad


class ScheduleZeta(torch.autograd.Function):
    """(theta, s (n x 6 float32), zeta^plain (n float64)) -> zeta (n float64)."""

    @staticmethod
    def forward(ctx, theta, feats, plain):
        theta = theta.contiguous()
        zeta, _ = schedule_forward(theta, feats, plain)
        ctx.save_for_backward(theta, feats, plain)
        return zeta

    @staticmethod
    def backward(ctx, zeta_bar):
        theta, feats, plain = ctx.saved_tensors
        return schedule_backward(theta, feats, plain, zeta_bar.to(torch.float64)), None, None


def projection_loss(Y1, Y2, Ut, Vt, P, Q, r):
    """loss_k (device float64 scalar) and its gradients with respect to Y1, Y2."""
    m, R = Y1.shape
    n = Y2.shape[0]
    loss = torch.empty((), dtype=torch.float64, device=Y1.device)
    Y1b, Y2b = torch.empty_like(Y1), torch.empty_like(Y2)
    work = torch.empty(2 * r * (m + n), dtype=torch.float64, device=Y1.device)
    args = [x.contiguous() for x in (Y1, Y2, Ut, Vt)]
    P, Q = P.contiguous(), Q.contiguous()
    _check(lib().rpca_projection_loss(*(_ptr(x) for x in args), m, n, R, r, _dtype_code(Y1), _ptr(P), _ptr(Q),
                                      P.shape[1], _ptr(loss), _ptr(Y1b), _ptr(Y2b), _ptr(work), _stream()),
           "rpca_projection_loss")
    return loss, Y1b, Y2b


class ProjectionLoss(torch.autograd.Function):
    """(Y1, Y2; U~, V~, P, Q held fixed) -> ||P_T Z - P Q^T||_F^2 / ||P Q^T||_F^2."""

    @staticmethod
    def forward(ctx, Y1, Y2, Ut, Vt, P, Q, r):
        loss, Y1b, Y2b = projection_loss(Y1, Y2, Ut, Vt, P, Q, r)
        ctx.save_for_backward(Y1b, Y2b)
        return loss

    @staticmethod
    def backward(ctx, gloss):
        Y1b, Y2b = ctx.saved_tensors
        return Y1b * gloss.to(Y1b.dtype), Y2b * gloss.to(Y2b.dtype), None, None, None, None, None


# ---------------------------------------------------------------------------------------
# Parameters, training and evaluation
# ---------------------------------------------------------------------------------------

def init_theta(seed=0, device="cuda"):
    """Packed parameters (see include/rpca.h): hidden layers drawn like torch.nn.Linear's
    default (uniform +-1/sqrt(fan_in)), output layer zero (the plain schedule)."""
    rng = np.random.default_rng(seed)
    th = np.zeros(SCHEDULE_PARAMS, dtype=np.float32)
    o = 0
    for rows, cols in ((HIDDEN, INPUTS), (HIDDEN, HIDDEN)):
        b = 1.0 / math.sqrt(cols)
        th[o:o + rows * cols] = rng.uniform(-b, b, rows * cols)
        o += rows * cols
        th[o:o + rows] = rng.uniform(-b, b, rows)
        o += rows
    return torch.from_numpy(th).to(device)


def save_theta(theta, path):
    np.savez(path, theta=theta.detach().cpu().numpy().astype(np.float32))


def load_theta(path, device="cuda"):
    return torch.from_numpy(np.load(path)["theta"].astype(np.float32)).to(device)


def _solver(x, tol, max_iter, zeta_mode="learned", precision="fp32"):
    return Solver(x["beta"], x["gamma"], tol, precision=precision, zeta_mode=zeta_mode, beta_init=2 * x["beta"],
                  mu_trim=x["mu"], max_iter=max_iter)


def unrolled_trace(x, theta, K, precision="fp32"):
    """Runs K iterations of the library in zeta mode "learned" on instance x and returns, per
    iteration k, the operands (W, V, U~, V~) of pass k and its statistics record."""
    ops, stats = [], []
    with _solver(x, 0.0, K, precision=precision) as s:
        s.set_schedule(theta, K)
        s.init(x["D"], x["r"])
        for _ in range(K):
            ops.append(s.pass_operands())
            _, st = s.iterate(1)
            if not st:
                ops.pop()
                break
            stats.extend(st)
    return ops, stats


def unrolled_loss(x, theta, K, tau, trace=None):
    """Objective of one training instance: mean over k = 1 .. K-1 of log loss_k (a tensor
    attached to theta through the library's backward kernels).  `trace` (operands and
    statistics of an unrolled_trace) holds the trajectory fixed; by default it is run with
    the current parameters."""
    ops, stats = trace if trace is not None else unrolled_trace(x, theta.detach(), K)
    dev = x["D"].device
    feats = torch.tensor([st["features"] for st in stats[:-1]], dtype=torch.float32, device=dev)
    plain = torch.tensor([st["zeta_next_plain"] for st in stats[:-1]], dtype=torch.float64, device=dev)
    zetas = ScheduleZeta.apply(theta, feats, plain)
    losses = []
    for k in range(1, len(ops)):
        W, V, Ut, Vt = ops[k]
        Y1, Y2, _ = LearnPass.apply(x["D"], W, V, Ut, Vt, zetas[k - 1], tau)
        losses.append(ProjectionLoss.apply(Y1, Y2, Ut, Vt, x["P"], x["Q"], x["r"]))
    return torch.stack(losses).log().mean(), zetas, stats


class Adam:
    """Adam on the packed parameters, by the library's rpca_adam_step."""

    def __init__(self, theta, lr=1e-2, betas=(0.9, 0.999), eps=1e-8):
        self.theta, self.lr, self.betas, self.eps = theta, lr, betas, eps
        self.m1 = torch.zeros_like(theta)
        self.m2 = torch.zeros_like(theta)
        self.t = 0

    def step(self, grad):
        self.t += 1
        grad = grad.contiguous()
        _check(lib().rpca_adam_step(_ptr(self.theta), _ptr(grad), _ptr(self.m1), _ptr(self.m2), self.theta.numel(),
                                    self.t, self.lr, self.betas[0], self.betas[1], self.eps, _stream()),
               "rpca_adam_step")


def train(instances, K=12, steps=100, lr=1e-2, tau=0.05, seed=0, log=None):
    """Trains the schedule on planted instances: list of dicts with D (CUDA float32), r,
    beta, gamma, mu, P, Q (CUDA float64, L* = P Q^T).  Returns the packed parameters."""
    theta = init_theta(seed, device=instances[0]["D"].device)
    opt = Adam(theta, lr=lr)
    for step in range(steps):
        x = instances[step % len(instances)]
        leaf = theta.detach().clone().requires_grad_(True)
        J, _, _ = unrolled_loss(x, leaf, K, tau)
        J.backward()
        opt.step(leaf.grad)
        if log is not None:
            log.append(float(J.detach()))
    return theta


def solve(x, theta=None, tol=1e-5, K=12, max_iter=100, precision="fp32"):
    """Solves instance x to tol through the library, with the learned schedule (theta) or the
    paper's (theta None).  Returns (status, per-pass statistics, factors)."""
    with _solver(x, tol, max_iter, zeta_mode="learned" if theta is not None else "paper", precision=precision) as s:
        if theta is not None:
            s.set_schedule(theta, K)
        s.init(x["D"], x["r"])
        code, stats = s.run()
        return code, stats, s.lowrank()
