"""Properties of the seeded instance generators (CPU only)."""
import numpy as np

import synth


def test_planted_instance_follows_section3_recipe():
    inst = synth.planted_instance(120, 90, 3, 0.2, 2.0, 7)
    assert inst.D.shape == (120, 90)
    k = round(0.2 * 120 * 90)
    assert len(inst.support) == k == len(np.unique(inst.support))
    assert np.all(np.diff(inst.support) > 0)
    bound = 2.0 * np.mean(np.abs(inst.L))
    assert np.all(np.abs(inst.values) <= bound)
    assert np.allclose(inst.D, inst.L + inst.S, atol=1e-12)
    # Deterministic for a seed, different across seeds.
    again = synth.planted_instance(120, 90, 3, 0.2, 2.0, 7)
    assert np.array_equal(again.D, inst.D)
    assert not np.array_equal(synth.planted_instance(120, 90, 3, 0.2, 2.0, 8).D, inst.D)


def test_incoherence_matches_svd_definition():
    inst = synth.planted_instance(80, 60, 4, 0.1, 1.0, 1)
    U, s, Vt = np.linalg.svd(inst.L, full_matrices=False)
    U, V = U[:, :4], Vt[:4].T
    mu = max(80 / 4 * np.max(np.sum(U * U, 1)), 60 / 4 * np.max(np.sum(V * V, 1)))
    assert abs(mu - inst.mu) < 1e-10
    p = inst.params()
    assert abs(p["beta"] - 1.1 * mu * 4 / (2 * np.sqrt(80 * 60))) < 1e-14
    assert p["gamma"] == 0.5


def test_video_instance_is_rank2_background_plus_rectangles():
    v = synth.video_instance(frames=40, seed=3)
    assert v.D.shape == (176 * 144, 40)
    s = np.linalg.svd(v.L, compute_uv=False)
    assert s[2] < 1e-10 * s[0]
    occ = v.fg_mask.mean(axis=0)
    assert occ.min() > 0.01 and occ.max() < 0.12
    resid = (v.D - v.L)[~v.fg_mask]
    assert abs(resid.std() - 1e-3) < 2e-4
    assert 0.1 - 1e-9 <= v.background.min() and v.background.max() <= 0.7 + 1e-9
