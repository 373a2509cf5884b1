"""rpca_get_sparse_noalloc, the support extraction that allocates no device memory, against
rpca_get_sparse (GPU).  It is meant for callers that may not allocate device memory
themselves (memory owned by another framework's caching pool, or a fixed device-memory
budget set at start-up).  This file is collected last so that a run stopping at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

import synth
from parity_helpers import support_mismatch

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1711_05519_gb300")


def _noalloc(D, U, s, V, zeta, cap, null_outputs=False):
    m, n = D.shape
    r = U.shape[1]
    idx = torch.empty(max(cap, 1), dtype=torch.int64, device="cuda")
    val = torch.empty(max(cap, 1), dtype=torch.float64, device="cuda")
    nnz = ctypes.c_int64(-1)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    out_i = None if null_outputs else ctypes.c_void_p(idx.data_ptr())
    out_v = None if null_outputs else ctypes.c_void_p(val.data_ptr())
    code = P.lib().rpca_get_sparse_noalloc(ctypes.c_void_p(D.data_ptr()), m, n, D.stride(0), r,
                                           ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(s.data_ptr()),
                                           ctypes.c_void_p(V.data_ptr()), zeta, out_i, out_v, cap,
                                           ctypes.byref(nnz), stream)
    return code, nnz.value, idx[: max(nnz.value, 0)].cpu().numpy(), val[: max(nnz.value, 0)].cpu().numpy()


def _padded(D64, pad, dtype):
    """D as a strided view of a wider buffer: leading dimension n + pad."""
    m, n = D64.shape
    buf = torch.zeros(m, n + pad, dtype=dtype, device="cuda")
    buf[:, :n] = torch.from_numpy(D64).to(dtype)
    return buf[:, :n]


@pytest.mark.parametrize("r,pad", [(4, 0), (1, 0), (16, 0), (4, 24)])
def test_noalloc_extraction_matches_get_sparse(r, pad):
    m, n = 700, 520
    inst = synth.planted_instance(m, n, r, 0.1, 1.0, 21)
    p = inst.params()
    D = _padded(inst.D, pad, torch.float32)
    assert D.stride(0) == n + pad
    with P.Solver(p["beta"], p["gamma"], 1e-5, precision="fp32", beta_init=p["beta_init"], mu_trim=p["mu"]) as s:
        s.init(D, r)
        s.iterate(6)
        _, zeta, _ = s.state()
        U, sig, V = s.lowrank()
        idx_ref, val_ref = (t.cpu().numpy() for t in s.sparse())
    assert len(idx_ref) > 0
    for _ in range(2):  # two calls in a row share the static scratch
        code, nnz, idx, val = _noalloc(D, U, sig, V, zeta, m * n)
        assert code == P.OK and nnz == len(idx_ref)
        assert np.array_equal(idx, idx_ref)
        assert np.array_equal(val, val_ref)
    # too small an output buffer: capacity error with the required size
    code, nnz, _, _ = _noalloc(D, U, sig, V, zeta, 1)
    assert code == P.CAPACITY and nnz == len(idx_ref)
    # a threshold above every |R_ij|: empty support, written through NULL buffers of capacity 0
    code, nnz, _, _ = _noalloc(D, U, sig, V, 1e30, 0, null_outputs=True)
    assert code == P.OK and nnz == 0
    # and the scratch holds no trace of that call for the next one
    code, nnz, idx, _ = _noalloc(D, U, sig, V, zeta, m * n)
    assert code == P.OK and np.array_equal(idx, idx_ref)


def test_noalloc_from_fp64_factors_thresholds_in_fp32():
    # factors from an FP64 context: the entry point rebuilds L and thresholds in FP32 (as
    # documented), so its support is the FP64 one except for entries inside the FP32 tie band
    m, n, r = 640, 500, 5
    inst = synth.planted_instance(m, n, r, 0.1, 1.0, 23)
    p = inst.params()
    D64 = torch.from_numpy(inst.D).cuda()
    with P.Solver(p["beta"], p["gamma"], 1e-10, precision="fp64", beta_init=p["beta_init"], mu_trim=p["mu"]) as s:
        s.init(D64, r)
        s.iterate(6)
        _, zeta, _ = s.state()
        U, sig, V = s.lowrank()
    D32 = D64.float().contiguous()
    code, nnz, idx, val = _noalloc(D32, U, sig, V, zeta, m * n)
    assert code == P.OK and nnz == len(idx)
    Dh = D32.double().cpu().numpy()
    L = (U.cpu().numpy() * sig.cpu().numpy()) @ V.cpu().numpy().T
    diff, ok = support_mismatch(idx, Dh, L, zeta, band_abs_rel_D=1e-6)
    assert ok, diff[:10]
    R = (Dh - L).reshape(-1)[idx]
    assert np.allclose(val, R, rtol=0.0, atol=1e-6 * np.abs(Dh).max())


def test_noalloc_rejects_more_rows_than_its_scratch():
    big = 65536 + 1
    D = torch.zeros(2, 8, device="cuda")  # never read: the size check comes first
    U = torch.zeros(2, 1, dtype=torch.float64, device="cuda")
    s = torch.zeros(1, dtype=torch.float64, device="cuda")
    nnz = ctypes.c_int64(0)
    code = P.lib().rpca_get_sparse_noalloc(ctypes.c_void_p(D.data_ptr()), big, 8, 8, 1, ctypes.c_void_p(U.data_ptr()),
                                           ctypes.c_void_p(s.data_ptr()), ctypes.c_void_p(U.data_ptr()), 0.5, None,
                                           None, 0, ctypes.byref(nnz), None)
    assert code == P.INVALID_ARG
