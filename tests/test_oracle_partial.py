"""Pins of the partially observed oracle (oracle/partial.py) on the CPU: the fully observed
limit is the oracle of Algorithms 1-3, unobserved values never enter, planted instances are
recovered exactly from a subset of the entries, and plausible mistakes fail a pin."""
import numpy as np
import pytest

import synth
from oracle import accaltproj as O
from oracle import partial as OP


@pytest.fixture(scope="module")
def planted():
    inst = synth.planted_instance(400, 400, 3, 0.05, 1.0, 0)
    return inst, inst.params()


def _run(inst, p, obs, D=None, tol=1e-10):
    return OP.accaltproj_partial(inst.D if D is None else D, obs, 3, p["beta"], p["gamma"], tol, p["mu"],
                                 beta_init=p["beta_init"])


def test_fully_observed_limit_is_the_oracle(planted):
    inst, p = planted
    obs = np.ones(inst.D.shape, dtype=bool)
    part = _run(inst, p, obs)
    full = O.accaltproj(inst.D, 3, p["beta"], p["gamma"], 1e-10, p["mu"], beta_init=p["beta_init"])
    assert part["iters"] == full["iters"]
    assert np.linalg.norm(part["L"] - full["L"]) < 1e-12 * np.linalg.norm(full["L"])
    assert np.array_equal(np.flatnonzero(part["S"]), np.flatnonzero(full["S"]))
    assert np.allclose(part["history"]["err"], full["history"]["err"], rtol=1e-9, atol=1e-15)


def test_unobserved_values_never_enter(planted):
    inst, p = planted
    obs = np.random.default_rng(3).random(inst.D.shape) < 0.6
    a = _run(inst, p, obs)
    D2 = inst.D.copy()
    D2[~obs] = np.nan
    b = _run(inst, p, obs, D=D2)
    D3 = inst.D.copy()
    D3[~obs] = 1e6 * np.random.default_rng(4).standard_normal(int((~obs).sum()))
    c = _run(inst, p, obs, D=D3)
    for other in (b, c):
        assert other["iters"] == a["iters"]
        assert np.array_equal(other["L"], a["L"]) and np.array_equal(other["S"], a["S"])


@pytest.mark.parametrize("p_obs", [0.9, 0.5])
def test_planted_recovery_from_a_subset_of_entries(planted, p_obs):
    inst, p = planted
    obs = np.random.default_rng(int(10 * p_obs)).random(inst.D.shape) < p_obs
    res = _run(inst, p, obs)
    assert res["err"] < 1e-10
    assert np.linalg.norm(res["L"] - inst.L) < 1e-9 * np.linalg.norm(inst.L)
    # the sparse part lives on observed entries of the planted support (Theorem 1's
    # supp(S_k) in Omega, restricted to what is observed)
    supp = np.flatnonzero(res["S"])
    assert obs.reshape(-1)[supp].all() and np.isin(supp, inst.support).all()
    # the initialisation is on the scale of L*: the 1/p of the sampled matrix is applied
    init = res["init"]
    s1 = np.linalg.norm(inst.L, 2)
    assert init["sigma"][0] == pytest.approx(s1, rel=0.05)
    assert init["p"] == pytest.approx(obs.mean())


def test_pins_catch_planted_mistakes(planted, monkeypatch):
    inst, p = planted
    obs = np.random.default_rng(5).random(inst.D.shape) < 0.5

    def step_without_rescaling(D, observed, U, sigma, V, zeta, k, r, beta, gamma, mu, do_trim=True):
        L = (U * sigma) @ V.T
        S = O.hard_threshold(OP.sample(D - L, observed), zeta)
        Ut, Vt = O.trimmed_bases(U, V, mu, r, do_trim)
        Z = L + OP.sample(D - L - S, observed)  # step of size 1 instead of 1/p
        U1, s1, V1, sM = O.tangent_truncated_svd(Z, Ut, Vt, r)
        return {"U": U1, "sigma": s1, "V": V1, "zeta": O.next_threshold(beta, gamma, k + 1, sM, r)}

    monkeypatch.setattr(OP, "step", step_without_rescaling)
    bad = _run(inst, p, obs)
    assert not np.linalg.norm(bad["L"] - inst.L) < 1e-9 * np.linalg.norm(inst.L)
    monkeypatch.undo()

    good_init = OP.initialize

    def init_without_rescaling(D, observed, r, beta_init, beta):
        out = good_init(D, observed, r, beta_init, beta)
        out["sigma"] = out["sigma"] * out["p"]  # H_r of P_Obs(D - S) without the 1/p
        return out

    monkeypatch.setattr(OP, "initialize", init_without_rescaling)
    bad = _run(inst, p, obs)
    assert bad["init"]["sigma"][0] != pytest.approx(np.linalg.norm(inst.L, 2), rel=0.05)
