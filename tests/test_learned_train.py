"""The learned schedule gains over the plain beta-gamma^k schedule (GPU): a short training
run on small planted instances lowers the error reached after the same number of unrolled
iterations on held-out instances."""
import numpy as np
import pytest
import torch

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

P = pytest.importorskip("paper_1711_05519_gb300")
from paper_1711_05519_gb300 import learned as PL  # noqa: E402
from paper_1711_05519_gb300.train_schedule import make_instance  # noqa: E402


def test_trained_schedule_beats_plain_on_held_out_instances():
    rng = np.random.default_rng(5)
    train = [make_instance(600, 3000 + i, rng, r=int(rng.choice([3, 5]))) for i in range(4)]
    test = [make_instance(600, 4000 + i, rng, r=int(rng.choice([3, 5]))) for i in range(3)]
    mlp = PL.train(train, K=12, steps=40, lr=1e-2, seed=0)
    plain, learned = [], []
    for x in test:
        run = PL.Unrolled(x["D"], x["r"], x["beta"], x["gamma"], x["mu"], K=12)
        _, _, f0 = run.run(mlp=None, hard=True)
        _, _, f1 = run.run(mlp=mlp, hard=True)
        plain.append(PL.final_error(f0, x["P"], x["Q"]))
        learned.append(PL.final_error(f1, x["P"], x["Q"]))
    # geometric-mean improvement of the recovery error of L after 12 iterations
    gain = float(np.exp(np.mean(np.log(np.array(plain) / np.array(learned)))))
    assert gain > 1.5, (plain, learned)


def test_untrained_network_reproduces_plain_schedule():
    rng = np.random.default_rng(6)
    x = make_instance(400, 5000, rng, r=3)
    run = PL.Unrolled(x["D"], x["r"], x["beta"], x["gamma"], x["mu"], K=8)
    _, e0, f0 = run.run(mlp=None, hard=True)
    _, e1, f1 = run.run(mlp=PL.ThresholdMLP().cuda(), hard=True)
    assert e1 == pytest.approx(e0, rel=1e-3)  # atomics: summation order varies between runs
