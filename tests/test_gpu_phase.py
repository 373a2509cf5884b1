"""Phase transition of Table 2 on the GPU (FP64, n = 2500, r = 5, tol 1e-6, at most 100
iterations, success if ||L_k - L*||_F / ||L*||_F <= 1e-4), at cells where the paper's
AccAltProj with trim succeeds 10 out of 10 times or fails 10 out of 10 times.  The full
grid runs with `bench.py --phase-transition 10`."""
import pytest
import torch

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1711_05519_gb300")
bench = pytest.importorskip("bench")


@pytest.mark.parametrize("c,alpha,succeeds", [(1.0, 0.3, True), (1.0, 0.6, True), (1.0, 0.75, False),
                                              (5.0, 0.55, True), (0.2, 0.75, False)])
def test_table2_cells(c, alpha, succeeds):
    dev = torch.device("cuda", 0)
    ci = {0.2: 0, 1.0: 1, 5.0: 2}[c]
    ai = bench.TABLE2_ALPHAS.index(alpha)
    for t in range(2):
        err, _ = bench.recovery_trial(2500, 5, alpha, c, 10000 * ci + 100 * ai + t, dev)
        assert (err <= 1e-4) == succeeds, (c, alpha, t, err)
