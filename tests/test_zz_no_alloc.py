"""rpca_get_sparse_noalloc, the support extraction that allocates no device memory, against
rpca_get_sparse (GPU).  It is meant for callers that may not allocate device memory
themselves (memory owned by another framework's pool, a fixed device-memory budget, or a
loop that must not synchronise on an allocation).  This file is collected last so that a
run stopping at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1711_05519_gb300")


def _noalloc(D, U, s, V, zeta, cap):
    m, n = D.shape
    r = U.shape[1]
    idx = torch.empty(max(cap, 1), dtype=torch.int64, device="cuda")
    val = torch.empty(max(cap, 1), dtype=torch.float64, device="cuda")
    nnz = ctypes.c_int64(-1)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = P.lib().rpca_get_sparse_noalloc(ctypes.c_void_p(D.data_ptr()), m, n, D.stride(0), r,
                                           ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(s.data_ptr()),
                                           ctypes.c_void_p(V.data_ptr()), zeta, ctypes.c_void_p(idx.data_ptr()),
                                           ctypes.c_void_p(val.data_ptr()), cap, ctypes.byref(nnz), stream)
    return code, nnz.value, idx[: max(nnz.value, 0)].cpu().numpy(), val[: max(nnz.value, 0)].cpu().numpy()


def test_noalloc_extraction_matches_get_sparse():
    inst = synth.planted_instance(700, 520, 4, 0.1, 1.0, 21)
    p = inst.params()
    D = torch.from_numpy(inst.D).float().cuda()
    with P.Solver(p["beta"], p["gamma"], 1e-5, precision="fp32", beta_init=p["beta_init"], mu_trim=p["mu"]) as s:
        s.init(D, 4)
        code, stats = s.run()
        assert code == P.OK
        U, sig, V = s.lowrank()
        idx_ref, val_ref = (t.cpu().numpy() for t in s.sparse())
    zeta = stats[-1]["zeta"]
    assert len(idx_ref) > 0
    for _ in range(2):  # two calls in a row share the static scratch
        code, nnz, idx, val = _noalloc(D, U, sig, V, zeta, 700 * 520)
        assert code == P.OK and nnz == len(idx_ref)
        assert np.array_equal(idx, idx_ref)
        assert np.allclose(val, val_ref, rtol=0.0, atol=0.0)
    # too small an output buffer: capacity error with the required size
    code, nnz, _, _ = _noalloc(D, U, sig, V, zeta, 1)
    assert code == P.CAPACITY and nnz == len(idx_ref)


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
