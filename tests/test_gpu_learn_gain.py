"""What the trained correction gains (the c5 configuration).

Flows: the 512^2 jet and the 128^3 ABC + round-jet cone, flow seeds 10-19 for
training and 20-24 held out.  Each sample pairs a sparse FLA cloud (262,144
seeds) with a dense one of the same flow (2^24 droplets, 64 times the seeds)
at the same deposit time, each deposited at its own kernel scale.  Samples at
t = 0.6, 0.8, 1.0 (jet) and 0.3, 0.4, 0.5 (cone), 850 training cells each
(51,000 in all), drawn from the covered cells away from fold caustics (cells
within 3 h_max of a droplet with |det J| < 1e-2: there n = n0/|det J| is
singular and no seeding converges; the errors over all covered cells are
printed beside).  The network is trained on the GPU by the library's own
kernels; the test compares the learned and the plain method's error against
the dense reference on the held-out flows, per flow family.

The cone is deposited with the J-scaled kernel, whose Lagrangian bandwidth h0
the correction scales.  Measured (GB300): the plain method's error away from
caustics is 0.52 (jet) and 0.96 (cone); the learned correction takes the
held-out jet to 0.44 (-16 %) and leaves the cone at 0.96 (+0.2 %).  Over all
covered cells it is worse than the plain method on the jet (1.2 -> 2.9):
droplets just outside the fold band (|det J| of 1e-2..1e-1, n tens of times
the cloud's) get narrower kernels.
The test asserts what holds: both targets are within the plain method's
reach, and the held-out jet gains.
"""
import time

import numpy as np
import pytest

from paper_2512_20829_gb300 import fla
from paper_2512_20829_gb300 import learn as LRN

pytestmark = pytest.mark.gpu

JET_WINDOWS = (59, 79, 99)
CONE_WINDOWS = (29, 39, 49)


@pytest.fixture(scope="module")
def ctx():
    c = fla.Context(0)
    yield c
    c.close()


def test_trained_correction_beats_the_plain_method_on_held_out_flows(ctx):
    t0 = time.perf_counter()
    train = (LRN.make_samples(ctx, "jet", range(10, 20), JET_WINDOWS) +
             LRN.make_samples(ctx, "cone", range(10, 20), CONE_WINDOWS))
    held = {"jet": LRN.make_samples(ctx, "jet", range(20, 25), JET_WINDOWS),
            "cone": LRN.make_samples(ctx, "cone", range(20, 25), CONE_WINDOWS)}
    t_samples = time.perf_counter() - t0
    assert len(train) == 60 and all(len(v) == 15 for v in held.values())
    log, stats = [], {}
    net = LRN.train(ctx, train, iters=200, lr=2e-3, seed=0, log=lambda it, L: log.append((it, L)), stats=stats)
    assert ctx.sync_status(reset=True).flags == 0
    print(f"\nsamples generated in {t_samples:.1f} s; training loss", [(i, round(v, 5)) for i, v in log])
    print(f"training: {stats['ms_per_iter']:.2f} ms per iteration ({len(train)} samples, 850 cells each)")
    assert log[-1][1] < log[0][1]
    for name, samples in held.items():
        tr = [s for s in train if s.wl.dim == samples[0].wl.dim]
        e_plain_tr, e_learn_tr = LRN.evaluate(ctx, tr), LRN.evaluate(ctx, tr, net)
        e_plain, e_learn = LRN.evaluate(ctx, samples), LRN.evaluate(ctx, samples, net)
        e_all_p, e_all_l = LRN.evaluate(ctx, samples, all_cells=True), LRN.evaluate(ctx, samples, net, all_cells=True)
        frac = np.mean([s.covered.sum() / max(s.all_covered.sum(), 1) for s in samples])
        print(f"{name}: error vs dense (mean over fields of ||S-T||^2/||T||^2): train plain {e_plain_tr:.4f} "
              f"learned {e_learn_tr:.4f}; held-out plain {e_plain:.4f} learned {e_learn:.4f} "
              f"(gain {100 * (1 - e_learn / e_plain):.1f} %); {100 * frac:.1f} % of the covered cells away "
              f"from caustics; all covered cells: plain {e_all_p:.4f} learned {e_all_l:.4f}")
        assert e_plain < 1.0          # the target is one the plain method can approach
        if name == "jet":
            assert e_learn < 0.95 * e_plain
            # the plain method at four times the seeds (release count and seeds
            # per release each doubled) against the same dense targets: the error
            # the learned form reaches with the base seeding costs the plain
            # method this much more seeding (the bench's jet leg times both runs)
            denser = LRN.make_samples(ctx, "jet", range(20, 25), JET_WINDOWS, sparse_seeding=2)
            e_plain4 = LRN.evaluate(ctx, denser)
            print(f"jet held-out, plain with 4x seeds: {e_plain4:.4f} (plain {e_plain:.4f}, learned {e_learn:.4f})")
