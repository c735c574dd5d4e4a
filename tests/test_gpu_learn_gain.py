"""What the trained correction gains.  Training: jets of flow seeds 10-19 at
128^2 (16,384 seeds, 1/64 of a 1,048,576-seed dense FLA cloud of the same
flow), samples at t = 0.6, 0.8, 1.0, 1,700 training cells each (51,000 in
all); the targets are the dense cloud's sources.  Held out: flow seeds 20-24.
The network is trained on the GPU by the library's own kernels; the test
compares the learned and the plain method's error against the dense
reference on the held-out flows."""
import numpy as np
import pytest

from paper_2512_20829_gb300 import fla
from paper_2512_20829_gb300 import learn as LRN

pytestmark = pytest.mark.gpu

WINDOWS = (59, 79, 99)


@pytest.fixture(scope="module")
def ctx():
    c = fla.Context(0)
    yield c
    c.close()


def test_trained_correction_beats_the_plain_method_on_held_out_flows(ctx):
    train = LRN.make_samples(ctx, range(10, 20), WINDOWS)
    held = LRN.make_samples(ctx, range(20, 25), WINDOWS)
    assert len(train) == 30 and len(held) == 15
    log, stats = [], {}
    net = LRN.train(ctx, train, iters=150, lr=2e-3, seed=0, log=lambda it, L: log.append((it, L)), stats=stats)
    assert ctx.sync_status(reset=True).flags == 0
    e_plain_tr = LRN.evaluate(ctx, train)
    e_learn_tr = LRN.evaluate(ctx, train, net)
    e_plain = LRN.evaluate(ctx, held)
    e_learn = LRN.evaluate(ctx, held, net)
    print("\ntraining loss", [(i, round(v, 5)) for i, v in log])
    print(f"training: {stats['ms_per_iter']:.2f} ms per iteration ({len(train)} samples, 1,700 cells each)")
    print(f"error vs dense (mean over fields of ||S-T||^2/||T||^2): train plain {e_plain_tr:.4f} learned "
          f"{e_learn_tr:.4f}; held-out plain {e_plain:.4f} learned {e_learn:.4f} "
          f"(gain {100 * (1 - e_learn / e_plain):.1f} %)")
    assert log[-1][1] < log[0][1]
    assert e_learn < 0.95 * e_plain
