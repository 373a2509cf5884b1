"""The context's launch profile (diagnostics): with events around every launch and with
events around every k-th fused pass only, the same solve counts the same launches, and the
sampled pass times are the timed share of the pass launches."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1711_05519_gb300")


def _profiled_solve(D, p, r, every):
    with P.Solver(p["beta"], p["gamma"], 1e-5, precision="fp32", beta_init=p["beta_init"], mu_trim=p["mu"]) as s:
        s.set_profiling(True, every=every)
        s.init(D, r)
        code, stats = s.run()
        assert code == P.OK
        prof = s.profile()
        s.set_profiling(False)
        return prof, stats


@pytest.mark.parametrize("every", [2, 3, 5])
def test_sampled_pass_timing_counts_every_launch(every):
    m, n, r = 1200, 1100, 4
    inst = synth.planted_instance(m, n, r, 0.1, 1.0, 91)
    p = inst.params()
    D = torch.from_numpy(inst.D.astype(np.float32)).cuda()
    full, stats_full = _profiled_solve(D, p, r, 1)
    samp, stats_samp = _profiled_solve(D, p, r, every)
    assert stats_full[-1]["k"] == stats_samp[-1]["k"]
    total = full["pass_launches"] + full["other_launches"]
    assert samp["pass_launches"] + samp["other_launches"] == total
    # every pass that did work was timed with every = 1; with every = k about one in k of them
    passes = full["pass_launches"]
    assert passes > 0 and full["pass_ms"] > 0
    assert passes // every - 2 <= samp["pass_launches"] <= -(-passes // every)
    assert samp["pass_launches"] > 0 and samp["pass_ms"] > 0
    # only passes are timed when sampling: the other time is that of the timed passes queued
    # behind convergence, which returned at once
    assert 0.0 <= samp["other_ms"] < 0.5 * samp["pass_ms"]
    # the sampled average is a pass time (within the spread of pass launches)
    avg_full = full["pass_ms"] / passes
    avg_samp = samp["pass_ms"] / samp["pass_launches"]
    assert 0.3 * avg_full < avg_samp < 3.0 * avg_full


def test_negative_profiling_argument_is_refused():
    with P.Solver(1.0, 0.5, 1e-5, precision="fp32") as s:
        with pytest.raises(ValueError):
            s.set_profiling(True, every=0)
        assert P.lib().rpca_set_profiling(s._ctx, -1) == P.INVALID_ARG
