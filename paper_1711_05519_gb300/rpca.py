"""Python binding of the C ABI in include/rpca.h (ctypes; argument marshalling only).

Every step of the method runs in the CUDA library ``librpca.so``; this module only passes
device pointers, sizes and the current torch CUDA stream across the ABI.  There is no
CPU path: if the library is missing, loading it raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librpca.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "rpca.h")

OK, INVALID_ARG, CUDA_ERR, NUMERICAL, CAPACITY, NOT_CONVERGED, TIMEOUT, STATE = range(8)
DTYPE_F64, DTYPE_F32 = 0, 1
PREC = {"fp64": 0, "fp32": 1, "bf16": 2, "bf16_split": 3}
ZETA = {"paper": 0, "simple": 1, "external": 2, "learned": 3}
SCHEDULE_PARAMS = 1313
PASS_KIND = {"auto": 0, "simt": 1, "tensor": 2}
OBSERVED = {"all": 0, "nan": 1}
STATE_READS_LO = 1


class RpcaError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} ({code})")


class Params(ctypes.Structure):
    _fields_ = [
        ("beta", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("tol", ctypes.c_double),
        ("beta_init", ctypes.c_double),
        ("mu_trim", ctypes.c_double),
        ("max_iter", ctypes.c_int),
        ("trim", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("zeta_mode", ctypes.c_int),
        ("init_max_passes", ctypes.c_int),
        ("init_tol", ctypes.c_double),
        ("pass_kind", ctypes.c_int),
        ("split_switch", ctypes.c_double),
        ("observed", ctypes.c_int),
    ]


class IterStats(ctypes.Structure):
    _fields_ = [
        ("k", ctypes.c_int),
        ("err", ctypes.c_double),
        ("zeta", ctypes.c_double),
        ("sigma1", ctypes.c_double),
        ("sigma_r1", ctypes.c_double),
        ("nnz", ctypes.c_int64),
        ("zeta_next_plain", ctypes.c_double),
        ("g", ctypes.c_double),
        ("features", ctypes.c_double * 6),
        ("support_changes", ctypes.c_int64),
    ]


_lib = None


def lib() -> ctypes.CDLL:
    """Loads librpca.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1711_05519_gb300.build.build()")
    import torch.cuda  # noqa: F401  (loads the CUDA runtime the library links against)

    L = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    pi64, pint, pdbl = ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    L.rpca_status_string.restype = ctypes.c_char_p
    L.rpca_status_string.argtypes = [i32]
    L.rpca_params_default.argtypes = [ctypes.POINTER(Params)]
    L.rpca_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Params), vp]
    L.rpca_destroy.argtypes = [vp]
    L.rpca_destroy.restype = None
    L.rpca_solve_host_release.argtypes = []
    L.rpca_solve_host_release.restype = None
    L.rpca_set_lowrank.argtypes = [vp, vp, vp, vp, i32, dbl, i32]
    L.rpca_get_state.argtypes = [vp, pint, ctypes.POINTER(dbl), pint]
    L.rpca_init.argtypes = [vp, vp, i64, i64, i64, i32, i32]
    L.rpca_iterate.argtypes = [vp, i32, ctypes.POINTER(IterStats), pint]
    L.rpca_set_zeta.argtypes = [vp, dbl]
    L.rpca_get_lowrank.argtypes = [vp, vp, vp, vp]
    L.rpca_get_sparse.argtypes = [vp, vp, vp, i64, pi64]
    L.rpca_set_profiling.argtypes = [vp, i32]
    L.rpca_get_profile.argtypes = [vp, pdbl, pi64, pdbl, pi64]
    L.rpca_get_pass_kind.argtypes = [vp, pint, pint]
    L.rpca_get_sparse_noalloc.argtypes = [vp, i64, i64, i64, i32, vp, vp, vp, dbl, vp, vp, i64, pi64, vp]
    L.rpca_set_schedule.argtypes = [vp, vp, i32]
    L.rpca_get_pass_operands.argtypes = [vp, vp, vp, vp, vp, pint]
    L.rpca_schedule_forward.argtypes = [vp, vp, vp, i32, vp, vp, vp]
    L.rpca_schedule_backward.argtypes = [vp, vp, vp, vp, i32, vp, vp]
    L.rpca_adam_step.argtypes = [vp, vp, vp, vp, i32, i32, dbl, dbl, dbl, dbl, vp]
    L.rpca_projection_loss.argtypes = [vp, vp, vp, vp, i64, i64, i32, i32, i32, vp, vp, i32, vp, vp, vp, vp, vp]
    solve_args = [vp, i64, i64, i32, dbl, dbl, dbl, vp, vp, vp, vp, vp, i64, pi64, pint, pdbl]
    L.rpca_solve.argtypes = solve_args
    L.rpca_solve_host.argtypes = solve_args
    for name in ("rpca_params_default", "rpca_create", "rpca_init", "rpca_iterate", "rpca_set_zeta",
                 "rpca_get_lowrank", "rpca_get_sparse", "rpca_solve", "rpca_solve_host", "rpca_set_profiling",
                 "rpca_get_profile", "rpca_get_sparse_noalloc", "rpca_get_pass_kind", "rpca_set_schedule",
                 "rpca_get_pass_operands", "rpca_schedule_forward", "rpca_schedule_backward", "rpca_adam_step",
                 "rpca_projection_loss"):
        getattr(L, name).restype = i32
    _lib = L
    return L


def status_string(code: int) -> str:
    return lib().rpca_status_string(code).decode()


def header_functions() -> list[str]:
    """Names of the functions declared in include/rpca.h."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rpca_[a-z_]+)\s*\(", text)))


def _check(code: int, where: str, allow=(OK,)) -> int:
    if code not in allow:
        raise RpcaError(code, where)
    return code


def _stream_ptr(stream) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Solver:
    """One AccAltProj solve on the current CUDA device (a context of the C ABI)."""

    def __init__(self, beta: float, gamma: float, tol: float, precision: str = "fp32", trim: bool = True,
                 zeta_mode: str = "paper", max_iter: int = 100, beta_init: float = 0.0, mu_trim: float = 0.0,
                 init_max_passes: int = 0, init_tol: float = 0.0, pass_kind: str = "auto",
                 split_switch: float = 0.0, observed: str = "all", stream=None):
        L = lib()
        p = Params()
        L.rpca_params_default(ctypes.byref(p))
        p.beta, p.gamma, p.tol = beta, gamma, tol
        p.beta_init, p.mu_trim = beta_init, mu_trim
        p.max_iter, p.trim = max_iter, int(bool(trim))
        p.precision, p.zeta_mode = PREC[precision], ZETA[zeta_mode]
        p.init_max_passes, p.init_tol = init_max_passes, init_tol
        p.pass_kind = PASS_KIND[pass_kind]
        p.split_switch = split_switch
        p.observed = OBSERVED[observed]
        self.params = p
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._ctx = ctypes.c_void_p()
        _check(L.rpca_create(ctypes.byref(self._ctx), ctypes.byref(p), _stream_ptr(self.stream)), "rpca_create")
        self._D = None
        self.m = self.n = self.r = 0

    def close(self):
        if self._ctx:
            lib().rpca_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def init(self, D: torch.Tensor, r: int) -> None:
        """Algorithm 3 on D (2-D CUDA tensor, float32 or float64, unit column stride)."""
        if not (D.is_cuda and D.dim() == 2 and D.stride(1) == 1):
            raise ValueError("D must be a 2-D CUDA tensor with unit column stride")
        dt = {torch.float32: DTYPE_F32, torch.float64: DTYPE_F64}.get(D.dtype)
        if dt is None:
            raise ValueError("D must be float32 or float64")
        self._D = D  # the context borrows D
        self.m, self.n = D.shape
        self.r = r
        _check(lib().rpca_init(self._ctx, ctypes.c_void_p(D.data_ptr()), self.m, self.n, D.stride(0), dt, r),
               "rpca_init")

    def iterate(self, n_iters: int) -> tuple[int, list[dict]]:
        buf = (IterStats * max(n_iters, 1))()
        done = ctypes.c_int(0)
        code = lib().rpca_iterate(self._ctx, n_iters, buf, ctypes.byref(done))
        _check(code, "rpca_iterate", allow=(OK, NOT_CONVERGED))
        stats = [{"k": s.k, "err": s.err, "zeta": s.zeta, "sigma1": s.sigma1, "sigma_r1": s.sigma_r1,
                  "nnz": s.nnz, "zeta_next_plain": s.zeta_next_plain, "g": s.g, "features": list(s.features),
                  "support_changes": s.support_changes} for s in buf[: done.value]]
        return code, stats

    def run(self, max_passes: int | None = None) -> tuple[int, list[dict]]:
        """Iterates until err_k < tol or the iteration cap."""
        return self.iterate(max_passes if max_passes is not None else self.params.max_iter + 1)

    def pass_kind(self) -> tuple[str, str]:
        it, ini = ctypes.c_int(0), ctypes.c_int(0)
        _check(lib().rpca_get_pass_kind(self._ctx, ctypes.byref(it), ctypes.byref(ini)), "rpca_get_pass_kind")
        names = {1: "simt", 2: "tensor"}
        return names[it.value], names[ini.value]

    def set_profiling(self, on: bool, every: int = 1) -> None:
        """Events around every launch (every = 1) or around every `every`-th fused pass only."""
        if every < 1:
            raise ValueError("every must be >= 1")
        _check(lib().rpca_set_profiling(self._ctx, int(every) if on else 0), "rpca_set_profiling")

    def profile(self) -> dict:
        pm, om = ctypes.c_double(0), ctypes.c_double(0)
        pn, on = ctypes.c_int64(0), ctypes.c_int64(0)
        _check(lib().rpca_get_profile(self._ctx, ctypes.byref(pm), ctypes.byref(pn), ctypes.byref(om),
                                      ctypes.byref(on)), "rpca_get_profile")
        return {"pass_ms": pm.value, "pass_launches": pn.value, "other_ms": om.value, "other_launches": on.value}

    def set_zeta(self, zeta: float) -> None:
        _check(lib().rpca_set_zeta(self._ctx, zeta), "rpca_set_zeta")

    def set_schedule(self, theta: torch.Tensor, depth: int) -> None:
        """zeta_mode "learned": network parameters (CUDA float32, SCHEDULE_PARAMS values) and
        the unrolled depth K."""
        if not (theta.is_cuda and theta.dtype == torch.float32 and theta.numel() == SCHEDULE_PARAMS):
            raise ValueError("theta must be a CUDA float32 tensor of SCHEDULE_PARAMS values")
        self._theta = theta.contiguous()
        _check(lib().rpca_set_schedule(self._ctx, ctypes.c_void_p(self._theta.data_ptr()), int(depth)),
               "rpca_set_schedule")

    def pass_operands(self):
        """(W, V, U~, V~) the next pass reads, copies in the working precision, padded width."""
        dev = self._D.device
        dt = torch.float64 if self.params.precision == PREC["fp64"] else torch.float32
        R = _padded_rank(self.r)
        W, Ut = (torch.empty(self.m, R, dtype=dt, device=dev) for _ in range(2))
        V, Vt = (torch.empty(self.n, R, dtype=dt, device=dev) for _ in range(2))
        w = ctypes.c_int(0)
        _check(lib().rpca_get_pass_operands(self._ctx, ctypes.c_void_p(W.data_ptr()), ctypes.c_void_p(V.data_ptr()),
                                            ctypes.c_void_p(Ut.data_ptr()), ctypes.c_void_p(Vt.data_ptr()),
                                            ctypes.byref(w)), "rpca_get_pass_operands")
        assert w.value == R
        return W, V, Ut, Vt

    def lowrank(self):
        dev = self._D.device
        U = torch.empty(self.m, self.r, dtype=torch.float64, device=dev)
        s = torch.empty(self.r, dtype=torch.float64, device=dev)
        V = torch.empty(self.n, self.r, dtype=torch.float64, device=dev)
        _check(lib().rpca_get_lowrank(self._ctx, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(s.data_ptr()),
                                      ctypes.c_void_p(V.data_ptr())), "rpca_get_lowrank")
        return U, s, V

    def state(self) -> tuple[int, float, int]:
        """(k, zeta_k, flags): index of the iterate held, the threshold of the next pass and
        the RPCA_STATE_* bits (1: a BF16_SPLIT solve reads hi + lo)."""
        k, z, f = ctypes.c_int(0), ctypes.c_double(0), ctypes.c_int(0)
        _check(lib().rpca_get_state(self._ctx, ctypes.byref(k), ctypes.byref(z), ctypes.byref(f)), "rpca_get_state")
        return k.value, z.value, f.value

    def set_lowrank(self, U: torch.Tensor, sigma: torch.Tensor, V: torch.Tensor, k: int, zeta: float,
                    flags: int = 0) -> None:
        """Resumes from a factor checkpoint (lowrank() and state() of an earlier context on
        the same D); call after init()."""
        dev = self._D.device
        U, sigma, V = (t.to(dev, torch.float64).contiguous() for t in (U, sigma, V))
        _check(lib().rpca_set_lowrank(self._ctx, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(sigma.data_ptr()),
                                      ctypes.c_void_p(V.data_ptr()), int(k), float(zeta), int(flags)),
               "rpca_set_lowrank")

    def sparse(self, cap: int | None = None):
        """supp(S_k) as ascending linear indices i*n + j, and the values S_ij.  With `cap` (for
        example the support count of the last iteration's statistics) one call fills buffers
        of that size; without it, or if the support is larger, a first call sizes them."""
        nnz = ctypes.c_int64(0)
        if cap is None:
            code = lib().rpca_get_sparse(self._ctx, None, None, 0, ctypes.byref(nnz))
            _check(code, "rpca_get_sparse", allow=(OK, CAPACITY))
            cap = nnz.value
        dev = self._D.device
        idx = torch.empty(max(cap, 1), dtype=torch.int64, device=dev)
        val = torch.empty(max(cap, 1), dtype=torch.float64, device=dev)
        code = lib().rpca_get_sparse(self._ctx, ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(val.data_ptr()),
                                     cap, ctypes.byref(nnz))
        if code == CAPACITY:
            return self.sparse(None)
        _check(code, "rpca_get_sparse")
        return idx[: nnz.value], val[: nnz.value]


def _padded_rank(r: int) -> int:
    for R in (1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 14, 16):
        if R >= r:
            return R
    raise ValueError(r)


def solve(D: torch.Tensor, r: int, beta: float, gamma: float, tol: float, s_cap: int | None = None) -> dict:
    """rpca_solve on a float32 CUDA tensor (contiguous)."""
    if not (D.is_cuda and D.dtype == torch.float32 and D.is_contiguous()):
        raise ValueError("D must be a contiguous float32 CUDA tensor")
    m, n = D.shape
    dev = D.device
    cap = m * n if s_cap is None else s_cap
    U = torch.empty(m, r, dtype=torch.float64, device=dev)
    s = torch.empty(r, dtype=torch.float64, device=dev)
    V = torch.empty(n, r, dtype=torch.float64, device=dev)
    idx = torch.empty(max(cap, 1), dtype=torch.int64, device=dev)
    val = torch.empty(max(cap, 1), dtype=torch.float64, device=dev)
    nnz, iters, err = ctypes.c_int64(0), ctypes.c_int(0), ctypes.c_double(0)
    code = lib().rpca_solve(ctypes.c_void_p(D.data_ptr()), m, n, r, beta, gamma, tol,
                            ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(s.data_ptr()),
                            ctypes.c_void_p(V.data_ptr()), ctypes.c_void_p(idx.data_ptr()),
                            ctypes.c_void_p(val.data_ptr()), cap, ctypes.byref(nnz), ctypes.byref(iters),
                            ctypes.byref(err))
    _check(code, "rpca_solve", allow=(OK, NOT_CONVERGED))
    return {"status": code, "U": U, "sigma": s, "V": V, "idx": idx[: nnz.value], "val": val[: nnz.value],
            "iters": iters.value, "err": err.value}


def solve_host(D: torch.Tensor, r: int, beta: float, gamma: float, tol: float, s_cap: int,
               out: dict | None = None) -> dict:
    """rpca_solve_host on a float32 CPU tensor (ideally pinned); outputs are CPU tensors
    (pass ``out`` from a previous call to reuse them).  The library keeps its device buffers
    between calls; solve_host_release() frees them."""
    if D.is_cuda or D.dtype != torch.float32 or not D.is_contiguous():
        raise ValueError("D must be a contiguous float32 CPU tensor")
    m, n = D.shape
    if out is None:
        out = {"U": torch.empty(m, r, dtype=torch.float64, pin_memory=True),
               "sigma": torch.empty(r, dtype=torch.float64, pin_memory=True),
               "V": torch.empty(n, r, dtype=torch.float64, pin_memory=True),
               "idx": torch.empty(max(s_cap, 1), dtype=torch.int64, pin_memory=True),
               "val": torch.empty(max(s_cap, 1), dtype=torch.float64, pin_memory=True)}
    nnz, iters, err = ctypes.c_int64(0), ctypes.c_int(0), ctypes.c_double(0)
    code = lib().rpca_solve_host(ctypes.c_void_p(D.data_ptr()), m, n, r, beta, gamma, tol,
                                 ctypes.c_void_p(out["U"].data_ptr()), ctypes.c_void_p(out["sigma"].data_ptr()),
                                 ctypes.c_void_p(out["V"].data_ptr()), ctypes.c_void_p(out["idx"].data_ptr()),
                                 ctypes.c_void_p(out["val"].data_ptr()), s_cap, ctypes.byref(nnz),
                                 ctypes.byref(iters), ctypes.byref(err))
    _check(code, "rpca_solve_host", allow=(OK, NOT_CONVERGED))
    out.update(status=code, nnz=nnz.value, iters=iters.value, err=err.value)
    return out


def selftest_waits() -> tuple[int, int]:
    """Status codes recorded by the bounded-wait self-test kernels (TIMEOUT expected)."""
    a, b = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().rpca_selftest_waits(ctypes.byref(a), ctypes.byref(b)), "rpca_selftest_waits")
    return a.value, b.value


def solve_host_release() -> None:
    """Frees the device buffers and context that rpca_solve_host keeps between calls."""
    lib().rpca_solve_host_release()
