"""The video-shaped workload on the GPU (FP32): 176 x 144 frames as columns, n = 2000
frames, a rank-2 background, three moving rectangles and Gaussian noise (sigma = 1e-3), run
with r = 2, gamma = 0.7, tol 1e-4 as in the paper's video experiment (Section 3).

The tolerance is below the noise floor, so exact recovery is not expected: the test checks
that the error decays to the tolerance, that the background is recovered to within a small
multiple of the noise level, and that the large entries of S mark the planted rectangles.
"""
import numpy as np
import pytest
import torch

import synth
from synth.planted import incoherence, paper_parameters

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1711_05519_gb300")


def test_video_shaped_separation():
    v = synth.video_instance(seed=0)
    mu = incoherence(np.stack([v.background, np.ones(v.m)], axis=1), np.stack([np.ones(v.n), v.ramp], axis=1))
    p = paper_parameters(mu, v.m, v.n, 2, float(v.fg_mask.mean()))
    D = torch.from_numpy(v.D.astype(np.float32)).cuda()
    with P.Solver(p["beta"], 0.7, 1e-4, precision="fp32", beta_init=p["beta_init"], mu_trim=p["mu"],
                  max_iter=100) as s:
        s.init(D, 2)
        code, stats = s.run()
        U, sig, V = (t.double().cpu().numpy() for t in s.lowrank())
        idx, val = (t.cpu().numpy() for t in s.sparse())
    assert code == P.OK
    errs = np.array([x["err"] for x in stats])
    assert errs[-1] < 1e-4
    # the error decays: every tenth iterate is below the one ten steps before
    assert np.all(errs[10::10] < errs[:-10:10])
    L = (U * sig) @ V.T
    Lt = v.L
    noise_rel = v.noise * np.sqrt(v.m * v.n) / np.linalg.norm(Lt)
    assert np.linalg.norm(L - Lt) / np.linalg.norm(Lt) < 10 * noise_rel
    # foreground: entries of S above 0.01 against the rectangles' pixels
    pred = np.zeros(v.m * v.n, dtype=bool)
    pred[idx[np.abs(val) > 0.01]] = True
    pm = pred.reshape(v.m, v.n)
    tp = np.sum(pm & v.fg_mask)
    fp = np.sum(pm & ~v.fg_mask)
    fn = np.sum(~pm & v.fg_mask)
    assert 2 * tp / (2 * tp + fp + fn) > 0.85
