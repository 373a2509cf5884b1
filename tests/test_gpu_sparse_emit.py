"""The sparse output S_k (Eq. (10)) from the support words of the last fused pass (GPU).

After a converged FP32 solve on the tensor-core pass, rpca_get_sparse builds supp(S_k) from
the bit masks that pass wrote and rebuilds the values only at the support.  It must agree with
an independent extraction of the same iterate (rpca_get_sparse_noalloc: every entry rebuilt
and thresholded again) outside the threshold's tie band, list the indices in ascending order,
and hold exactly the pass's own support count.  A state whose last pass did not write the
words (an iteration cap reached before convergence) takes the extraction over D."""
import ctypes

import numpy as np
import pytest
import torch

import synth
from parity_helpers import support_mismatch

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1711_05519_gb300")


def _noalloc(D, U, s, V, zeta):
    m, n = D.shape
    cap = m * n
    idx = torch.empty(cap, dtype=torch.int64, device="cuda")
    val = torch.empty(cap, dtype=torch.float64, device="cuda")
    nnz = ctypes.c_int64(-1)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = P.lib().rpca_get_sparse_noalloc(ctypes.c_void_p(D.data_ptr()), m, n, D.stride(0), U.shape[1],
                                           ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(s.data_ptr()),
                                           ctypes.c_void_p(V.data_ptr()), zeta, ctypes.c_void_p(idx.data_ptr()),
                                           ctypes.c_void_p(val.data_ptr()), cap, ctypes.byref(nnz), stream)
    assert code == P.OK
    return idx[: nnz.value].cpu().numpy(), val[: nnz.value].cpu().numpy()


def _check_against_noalloc(D, D64, s, idx, val):
    _, zeta, _ = s.state()
    U, sig, V = s.lowrank()
    idx_ref, val_ref = _noalloc(D, U, sig, V, zeta)
    assert np.all(np.diff(idx) > 0)
    L = (U.double() * sig.double()) @ V.double().T
    diff, ok = support_mismatch(idx, D64, L.cpu().numpy(), zeta, band_abs_rel_D=1e-6)
    assert ok, diff[:10]
    common, ia, ib = np.intersect1d(idx, idx_ref, return_indices=True)
    assert len(common) >= len(idx_ref) - len(diff)
    scale = np.abs(D64).max()
    assert np.abs(val[ia] - val_ref[ib]).max() < 1e-6 * scale
    assert np.allclose(val, D64.reshape(-1)[idx] - L.cpu().numpy().reshape(-1)[idx], rtol=0, atol=1e-6 * scale)


@pytest.mark.parametrize("m,n,r,alpha", [(1500, 1300, 5, 0.1), (900, 1100, 12, 0.05), (333, 516, 3, 0.2)])
def test_support_words_of_the_last_pass(m, n, r, alpha):
    inst = synth.planted_instance(m, n, r, alpha, 1.0, 61)
    p = inst.params()
    D = torch.from_numpy(inst.D.astype(np.float32)).cuda()
    D64 = D.double().cpu().numpy()
    with P.Solver(p["beta"], p["gamma"], 1e-5, precision="fp32", beta_init=p["beta_init"], mu_trim=p["mu"]) as s:
        s.init(D, r)
        assert s.pass_kind()[0] == "tensor"
        code, stats = s.run()
        assert code == P.OK
        idx, val = (t.cpu().numpy() for t in s.sparse())
        # the words hold exactly the support the last pass counted
        assert len(idx) == stats[-1]["nnz"]
        _check_against_noalloc(D, D64, s, idx, val)
        # a second call gives the same list
        idx2, val2 = (t.cpu().numpy() for t in s.sparse())
        assert np.array_equal(idx, idx2) and np.array_equal(val, val2)


def test_capped_solve_extracts_over_d():
    # stopped by the iteration cap before the predicted last pass: the iterate held has no
    # support words, so the extraction reads D
    m, n, r = 800, 760, 4
    inst = synth.planted_instance(m, n, r, 0.1, 1.0, 62)
    p = inst.params()
    D = torch.from_numpy(inst.D.astype(np.float32)).cuda()
    D64 = D.double().cpu().numpy()
    with P.Solver(p["beta"], p["gamma"], 1e-5, precision="fp32", beta_init=p["beta_init"], mu_trim=p["mu"]) as s:
        s.init(D, r)
        s.iterate(4)
        idx, val = (t.cpu().numpy() for t in s.sparse())
        _check_against_noalloc(D, D64, s, idx, val)
