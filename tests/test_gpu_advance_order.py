"""fla_advance_ordered: the advance run in the cell-sorted order that the last
binning left in the workspace gives, bit for bit, the states of fla_advance
(each droplet's arithmetic does not depend on the thread that runs it), in every
precision, for both cloud kinds and with the fold guard; a random permutation
does too, and order entries out of range are skipped without touching the
cloud."""
import numpy as np
import pytest
import torch

from paper_2512_20829_gb300 import fla
from paper_2512_20829_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = fla.Context(0)
    yield c
    c.close()


def _cases():
    jet = I.jet_vortex_2d(scale=8, nsteps=120, lpt_per_batch=64)
    cone = I.abc_jet_3d(scale=16, nsteps=60)
    tg = I.taylor_green_2d(scale=2)
    return {"jet": (jet, jet.fla), "jet_lpt": (jet, jet.lpt), "cone": (cone, cone.fla), "tg": (tg, tg.fla)}


CASES = [("jet", fla.F32X2, False), ("jet", fla.F32, False), ("jet", fla.F32, True), ("jet", fla.F64, False),
         ("jet_lpt", fla.F32, False), ("jet_lpt", fla.F32X2, False), ("cone", fla.F32X2, False),
         ("cone", fla.F32, False), ("cone", fla.F32, True), ("tg", fla.F64, False)]


@pytest.mark.parametrize("name,dtype,fold", CASES)
def test_sorted_order_is_bit_identical(ctx, name, dtype, fold):
    wl, cloud = _cases()[name]
    m = fla.mesh(wl.dim, wl.n_cells_axis)
    desc = fla.carrier_desc(wl.carrier)
    nodes = fla.nodes_buffer(m, dtype)
    plain = fla.DeviceCloud.from_seeds(cloud, wl.dim, wl.delta, wl.dt, dtype)
    ordered = fla.DeviceCloud.from_seeds(cloud, wl.dim, wl.delta, wl.dt, dtype)
    if fold:
        plain.enable_fold()
        ordered.enable_fold()
    ws = fla.aligned_ws(fla.workspace(m, dtype, wl.kernel, cloud.n))
    steps = {}
    for s in range(0, wl.nsteps, wl.window):
        fla.carrier_sample(ctx, desc, m, 0.0 if wl.carrier.steady else s * wl.dt, dtype, nodes)
        ctx.sync_status(reset=True)
        fla.advance(ctx, plain, m, nodes, s, wl.window, wl.dt, reset_acc=True)
        steps["plain"] = steps.get("plain", 0) + ctx.sync_status(reset=True).droplet_steps
        order = fla.workspace_order(ws, m, cloud.n) if s > 0 else None
        fla.advance(ctx, ordered, m, nodes, s, wl.window, wl.dt, reset_acc=True, order=order)
        steps["ordered"] = steps.get("ordered", 0) + ctx.sync_status(reset=True).droplet_steps
        _, perm, _ = fla.cell_bins(ctx, ordered, m, ws)
        # the workspace holds the permutation fla_cell_bins returned
        assert torch.equal(perm, fla.workspace_order(ws, m, cloud.n))
    torch.cuda.synchronize()
    assert torch.equal(plain.state, ordered.state)
    assert torch.equal(plain.meta, ordered.meta)
    assert steps["plain"] == steps["ordered"] > 0
    st = fla.status_of(ordered.meta.cpu().numpy())
    assert (st == 1).sum() > 0


def test_random_and_out_of_range_orders(ctx):
    """A random permutation gives the same states; entries >= n advance no
    droplet, so the droplets they replace keep their states."""
    wl = I.jet_vortex_2d(scale=8, nsteps=40, lpt_per_batch=0)
    cloud = wl.fla
    n = cloud.n
    m = fla.mesh(2, wl.n_cells_axis)
    nodes = fla.nodes_buffer(m, fla.F32)
    fla.carrier_sample(ctx, fla.carrier_desc(wl.carrier), m, 0.0, fla.F32, nodes)
    g = torch.Generator().manual_seed(5)
    perm = torch.randperm(n, generator=g).to(torch.int32).cuda()
    holes = torch.arange(n, dtype=torch.int32)
    skipped = torch.randperm(n, generator=g)[: n // 7]
    holes[skipped] = n + 7 + torch.arange(skipped.numel(), dtype=torch.int32)
    holes = holes.cuda()
    clouds = [fla.DeviceCloud.from_seeds(cloud, 2, wl.delta, wl.dt, fla.F32) for _ in range(3)]
    before = clouds[2].state.clone(), clouds[2].meta.clone()
    for c, order in zip(clouds, (None, perm, holes)):
        fla.advance(ctx, c, m, nodes, 0, wl.window, wl.dt, reset_acc=True, order=order)
    torch.cuda.synchronize()
    assert torch.equal(clouds[0].state, clouds[1].state) and torch.equal(clouds[0].meta, clouds[1].meta)
    L = fla.state_layout(fla.CLOUD_FLA, 2)
    planes = clouds[2].state.view(L["n_planes"], n, -1)
    ref = clouds[0].state.view(L["n_planes"], n, -1)
    old = before[0].view(L["n_planes"], n, -1)
    keep = torch.ones(n, dtype=torch.bool)
    keep[skipped] = False
    keep = keep.cuda()
    assert torch.equal(planes[:, keep], ref[:, keep])
    assert torch.equal(planes[:, ~keep], old[:, ~keep])
    assert torch.equal(clouds[2].meta[~keep], before[1][~keep])
    moved = fla.status_of(clouds[0].meta.cpu().numpy())[skipped.numpy()] == 1
    assert moved.sum() > 0    # some of the skipped droplets would have moved
