"""Learned bandwidth correction on the GPU (tensor-core forward) against the
FP64 oracle: the network alone, the zero-network fallback (P13) and the
records + deposit with the correction fused in."""
import numpy as np
import pytest
import torch

from helpers import rel_l2
from oracle import oracle as O
from paper_2512_20829_gb300 import fla
from paper_2512_20829_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = fla.Context(0)
    yield c
    c.close()


def _bf16_exact(a):
    """float32 values that are exactly representable in bfloat16 (low half cleared)."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32) & np.uint32(0xFFFF0000)
    return u.view(np.float32)


@pytest.mark.parametrize("n,scale,seed", [(1000, 1.0, 1), (128, 2.0, 2), (7, 1.0, 3), (5000, 0.5, 4)])
def test_mlp_forward_matches_oracle(ctx, n, scale, seed):
    """c = g(f): the oracle's FP64 forward with BF16 weights and activations, and
    its bound on a single-precision-accumulating forward (no feature rounding:
    the inputs are BF16 values)."""
    rng = np.random.default_rng(seed)
    P = fla.init_mlp_params(seed, scale)
    P[fla.MLP_PARAMS - 1] = 0.1                  # b4
    P[64 * 6:64 * 7] = rng.uniform(-0.3, 0.3, 64)   # b1
    net = fla.LearnedCorrection(ctx, P)
    F = _bf16_exact(rng.uniform(-2.0, 2.0, (n, 6)))
    c_gpu = net.forward(torch.from_numpy(F).cuda()).cpu().numpy().astype(np.float64)
    torch.cuda.synchronize()
    assert ctx.sync_status(reset=True).flags == 0
    c_ora, bound = O.mlp_forward(P, F.astype(np.float64), FE=np.zeros_like(F, dtype=np.float64))
    dev = np.abs(c_gpu - c_ora)
    assert np.all(dev <= bound + 1e-6 * (1 + np.abs(c_ora))), (dev - bound).max()
    assert np.median(dev) <= 1e-5
    print(f"\nn={n}: |c_gpu - c_oracle| median {np.median(dev):.2e} max {dev.max():.2e}; bound max {bound.max():.2e}")


@pytest.mark.parametrize("dim,N,kernel", [(2, 128, 0), (2, 96, 1), (3, 24, 1)])
def test_mlp_zero_network_is_bit_identical_to_plain(ctx, dim, N, kernel):
    """P13: W4 = 0, b4 = 0 gives c = 0 and sources identical to the plain path,
    for the spherical and the J-scaled kernel."""
    s = I.synthetic_state(dim, 20000 if dim == 2 else 8000, N, seed=41, band=(0.2, 0.8), h0_cells=2.0)
    from helpers import gpu_cloud_from_state
    cl = gpu_cloud_from_state(s, fla.F32)
    m = fla.mesh(dim, N)
    ws = fla.aligned_ws(fla.workspace(m, fla.F32, kernel, cl.n))
    P = fla.init_mlp_params(5, 1.0, zero_last=True)
    net = fla.LearnedCorrection(ctx, P)
    h_max = (4.0 if kernel == 0 else 2.0) / N
    outs = []
    for mlp in (None, net):
        out = fla.SourceFields(m, fla.F32)
        fla.deposit_sources(ctx, cl, m, fla.deposit_cfg(kernel, 0.5 / N, h_max, 0.01, mlp=mlp), out, ws)
        torch.cuda.synchronize()
        outs.append([t.cpu().numpy() for t in (out.s_mass, out.s_mom, out.dsum)])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("dim,N,n,kernel", [(2, 96, 12000, 0), (3, 24, 9000, 0), (2, 96, 12000, 1),
                                             (3, 24, 9000, 1)])
def test_learned_deposit_matches_oracle(ctx, dim, N, n, kernel):
    """Records with the network fused in (tensor cores) and the gather, against
    the oracle's deposit with the same network, for the spherical kernel (h
    scaled) and the J-scaled kernel (its Lagrangian bandwidth h0 scaled).  g(f)
    is compared with the oracle's bound; the sources element-wise, where a cell
    may differ only if the support of one of its droplets moved by the
    network's rounding."""
    s = I.synthetic_state(dim, n, N, seed=50 + dim, band=(0.2, 0.8), h0_cells=1.5, jac_spread=0.4)
    from helpers import gpu_cloud_from_state
    cl = gpu_cloud_from_state(s, fla.F32)
    m = fla.mesh(dim, N)
    ws = fla.aligned_ws(fla.workspace(m, fla.F32, kernel, n))
    P = fla.init_mlp_params(60 + dim, 1.0)
    P[fla.MLP_PARAMS - 1] = 0.3
    net = fla.LearnedCorrection(ctx, P)
    c_out = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
    h_min, h_max = 0.5 / N, (4.0 if kernel == 0 else 3.0) / N
    out = fla.SourceFields(m, fla.F32)
    fla.deposit_sources(ctx, cl, m, fla.deposit_cfg(kernel, h_min, h_max, 0.01, mlp=net, mlp_out=c_out),
                        out, ws)
    torch.cuda.synchronize()
    assert ctx.sync_status(reset=True).flags == 0
    D = O.dep_struct(dim=dim, N=N, kernel=kernel, h_min=h_min, h_max=h_max, p=1.0, window_dt=0.01, fp32_decision=True,
                     mlp=P)
    c_ora, _, _ = O.learn_records(D, s.x, s.J, s.acc, s.batch, s.n0, s.h0)
    # c: the oracle's bound for features computed in single precision
    Fo = O.mlp_features(dim, s.J.astype(np.float64), s.n0[s.batch], s.h0[s.batch], 1.0 / N)
    _, bound = O.mlp_forward(P, Fo, FE=1e-5 * (1 + np.abs(Fo)))
    act = np.isfinite(c_out.cpu().numpy())
    dep = (s.status == 1) & np.all((s.x >= 0) & (s.x <= 1), axis=1)
    assert np.array_equal(act, dep)
    cg = c_out.cpu().numpy().astype(np.float64)
    dev = np.abs(cg[act] - c_ora[act])
    assert np.all(dev <= bound[act] + 1e-5 * (1 + np.abs(c_ora[act])))
    assert np.median(dev) <= 1e-4
    # sources
    om, ov, od = O.nw_deposit_celllist(D, s.x, s.J, s.acc, s.status, s.batch, s.n0, s.h0)
    am, av, _ = O.nw_deposit_celllist(D, s.x, s.J, np.abs(s.acc), s.status, s.batch, s.n0, s.h0)
    gm = out.s_mass.double().cpu().numpy()
    gv = out.s_mom.double().cpu().numpy().T
    bad = (np.abs(gm - om) > 1e-4 * np.abs(am) + 1e-30) | np.any(np.abs(gv - ov) > 1e-4 * np.abs(av) + 1e-30, axis=1)
    print(f"\ndim {dim} kernel {kernel}: g(f) deviation median {np.median(dev):.2e} max {dev.max():.2e}; "
          f"cells outside the element bound {int(bad.sum())} of {bad.size}; "
          f"rel-L2 S_mass {rel_l2(gm, om):.2e} S_mom {rel_l2(gv, ov):.2e}")
    assert bad.mean() <= 2e-3
    assert rel_l2(gm, om) <= 3e-4 and rel_l2(gv, ov) <= 3e-4
