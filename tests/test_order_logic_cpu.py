"""Host logic of the cell-sorted advance, on the CPU with the library calls
recorded instead of run: a cloud's advance gets the workspace's order only once
a deposit of that same cloud has binned it into the workspace, never the order
of another cloud that shares the workspace, and never on the first window of a
run or after a restore."""
import sys
import types

import numpy as np

sys.path.insert(0, ".")
import bench  # noqa: E402
from paper_2512_20829_gb300 import fla  # noqa: E402
from paper_2512_20829_gb300 import inputs as I  # noqa: E402


class _Cloud:
    def __init__(self, name, n):
        self.name, self.n = name, n


def _fake_fla(log):
    f = types.SimpleNamespace()
    f.carrier_sample = lambda *a, **k: None
    f.workspace_order = lambda ws, m, n: ("order", n)

    def advance(ctx, cloud, m, nodes, s, k, dt, reset_acc=False, order=None, stream=None):
        log.append(("advance", cloud.name, s, order))

    def deposit(ctx, cloud, m, cfg, out, ws, stream=None):
        log.append(("deposit", cloud.name))

    def parcels(ctx, cloud, m, wdt, out, ws, stream=None):
        log.append(("psicell", cloud.name))

    f.advance, f.deposit_sources = advance, deposit
    return f, parcels


def _path(with_lpt, ordered=True):
    log = []
    p = bench.RunPath.__new__(bench.RunPath)
    f, parcels = _fake_fla(log)
    p.fla, p.ctx, p.m, p.ws, p.cfg, p.out, p.psi, p.desc = f, None, None, None, None, None, None, None
    p.wl = types.SimpleNamespace(nsteps=40, window=10, dt=1e-3, carrier=types.SimpleNamespace(steady=True))
    p.cloud = _Cloud("fla", 100)
    p.lpt = _Cloud("lpt", 300) if with_lpt else None
    p.nodes = p.lnodes = None
    p.dtype = 0
    p.ordered = ordered
    p.parcel_deposit = parcels
    return p, log


def test_runpath_orders_each_cloud_by_its_own_binning():
    p, log = _path(with_lpt=False)
    p.issue()
    adv = [e for e in log if e[0] == "advance"]
    assert adv[0][3] is None                                    # first window: seed order
    assert all(e[3] == ("order", 100) for e in adv[1:])        # then its own binning
    p, log = _path(with_lpt=False, ordered=False)
    p.issue()
    assert all(e[3] is None for e in log if e[0] == "advance")


def test_runpath_shared_workspace_never_hands_one_cloud_the_others_order():
    p, log = _path(with_lpt=True)
    p.issue()
    for e in log:
        if e[0] == "advance" and e[1] == "fla":
            assert e[3] is None            # the parcels' deposit binned the workspace last
        if e[0] == "advance" and e[1] == "lpt" and e[2] > 0:
            assert e[3] == ("order", 300)


def test_simulation_order_follows_the_last_binning():
    sim = fla.Simulation.__new__(fla.Simulation)
    sim.ws, sim.m = None, None
    a, b = _Cloud("fla", 7), _Cloud("lpt", 9)
    sim._binned = None
    orig = fla.workspace_order
    try:
        fla.workspace_order = lambda ws, m, n: ("order", n)
        assert sim._order(a) is None
        sim._binned = a
        assert sim._order(a) == ("order", 7) and sim._order(b) is None
        sim.fla, sim.lpt, sim.step, sim._sampled_t = a, None, 0, 0.0
        a.restore = lambda snap: None
        sim.restore({"step": 30, "fla": {}})
        assert sim.step == 30 and sim._order(a) is None   # a restored run starts in seed order
    finally:
        fla.workspace_order = orig


def test_batch_workload_seeds_are_in_random_order():
    """The premise of the ordered batched advance: a batch cloud's seeds are
    uniform in a box, so consecutive seeds are far apart (a warp of 32 spans
    most of the cloud's extent)."""
    wl = I.batch_clouds(seed=4, n_clouds=2, n_min=4096, n_max=4096)[1]
    x = wl.fla.x0[:32]
    span = x.max(axis=0) - x.min(axis=0)
    box = wl.fla.x0.max(axis=0) - wl.fla.x0.min(axis=0)
    assert np.all(span > 0.5 * box)
