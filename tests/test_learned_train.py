"""The learned schedule gains over the plain beta-gamma^k schedule (GPU): a short training
run on small planted instances, through the library's kernels only, lowers the error of L
reached after the same number of iterations on held-out instances."""
import numpy as np
import pytest

from parity_helpers import factored_rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

P = pytest.importorskip("paper_1711_05519_gb300")
from paper_1711_05519_gb300 import learned as PL  # noqa: E402
from paper_1711_05519_gb300.train_schedule import make_instance  # noqa: E402


def _l_error(x, theta, iters):
    _, _, (U, s, V) = PL.solve(x, theta, tol=0.0, max_iter=iters)
    return factored_rel_err(*(t.cpu().numpy() for t in (U, s, V)), x["P"].cpu().numpy(), x["Q"].cpu().numpy())


def test_trained_schedule_beats_plain_on_held_out_instances():
    rng = np.random.default_rng(5)
    train = [make_instance(600, 3000 + i, rng, r=int(rng.choice([3, 5]))) for i in range(4)]
    test = [make_instance(600, 4000 + i, rng, r=int(rng.choice([3, 5]))) for i in range(3)]
    log = []
    theta = PL.train(train, K=12, steps=40, lr=1e-2, seed=0, log=log)
    assert np.mean(log[-8:]) < np.mean(log[:8])
    plain = [_l_error(x, None, 12) for x in test]
    learned = [_l_error(x, theta, 12) for x in test]
    # geometric-mean improvement of the recovery error of L after 12 iterations
    gain = float(np.exp(np.mean(np.log(np.array(plain) / np.array(learned)))))
    assert gain > 1.5, (plain, learned)
