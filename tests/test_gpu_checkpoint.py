"""Checkpoint and resume: a run saved to a file at a window boundary and resumed
in fresh objects gives, bit for bit, the states and sources of the run that was
not interrupted.  Covered: the compensated 2D jet, the single-precision 3D cone
with the fold guard, the two-way coupled run (droplets and carrier) and the
batched clouds."""
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


def _sim(ctx, wl, dtype, fold):
    return fla.Simulation(ctx, wl, dtype=dtype, fold_guard=fold)


@pytest.mark.parametrize("name,dtype,fold", [("jet", fla.F32X2, False), ("cone", fla.F32, True),
                                             ("jet", fla.F64, False)])
def test_simulation_resume_is_bit_identical(ctx, tmp_path, name, dtype, fold):
    wl = (I.jet_vortex_2d(scale=8, nsteps=160, lpt_per_batch=0) if name == "jet"
          else I.abc_jet_3d(scale=16, nsteps=60))
    half = (wl.nsteps // wl.window // 2) * wl.window
    a = _sim(ctx, wl, dtype, fold)
    a.run(half)
    path = tmp_path / "ck.pt"
    fla.save_checkpoint(path, a.checkpoint())
    a.run()
    b = _sim(ctx, wl, dtype, fold)
    b.restore(fla.load_checkpoint(path))
    assert b.step == half
    b.run()
    torch.cuda.synchronize()
    assert torch.equal(a.fla.state, b.fla.state) and torch.equal(a.fla.meta, b.fla.meta)
    if fold:
        assert torch.equal(a.fla.fold, b.fla.fold)
    assert torch.equal(a.out.s_mass, b.out.s_mass) and torch.equal(a.out.s_mom, b.out.s_mom)
    assert fla.status_of(b.fla.meta.cpu().numpy()).tolist().count(1) > 0


def test_two_way_resume_is_bit_identical(ctx, tmp_path):
    case = I.two_way_taylor_green(scale=4, nsteps=120, n0=5.0)
    wl = case.wl
    N = wl.n_cells_axis

    def make():
        ns = fla.NavierStokes(ctx, N, case.nu, case.diff, wl.dt, case.omega0, mean_u=case.mean_u)
        return fla.TwoWay(ctx, wl, ns, dtype=fla.F32)

    a = make()
    a.run(5)
    path = tmp_path / "tw.pt"
    fla.save_checkpoint(path, a.checkpoint())
    a.run(7)
    b = make()
    b.restore(fla.load_checkpoint(path))
    b.run(7)
    ga, gb = a.ns.fields(), b.ns.fields()
    torch.cuda.synchronize()
    for k in ("omega", "psi", "rho", "U"):
        assert np.array_equal(ga[k], gb[k]), k
    assert torch.equal(a.fla.state, b.fla.state) and torch.equal(a.fla.meta, b.fla.meta)


def test_batch_resume_is_bit_identical(ctx, tmp_path):
    wls = I.batch_clouds(seed=7, n_clouds=6, nsteps=60, n_min=1e3, n_max=2e4, meshes2=(32, 64), meshes3=(32,))
    a = fla.Batch(ctx, wls)
    a.run(3)
    path = tmp_path / "batch.pt"
    fla.save_checkpoint(path, a.checkpoint())
    a.run(3)
    b = fla.Batch(ctx, wls)
    b.restore(fla.load_checkpoint(path))
    assert b.step == 30
    b.run(3)
    torch.cuda.synchronize()
    for ca, cb, oa, ob in zip(a.clouds, b.clouds, a.outs, b.outs):
        assert torch.equal(ca.state, cb.state) and torch.equal(ca.meta, cb.meta)
        assert torch.equal(oa.s_mass, ob.s_mass) and torch.equal(oa.s_mom, ob.s_mom)
    a.close()
    b.close()
