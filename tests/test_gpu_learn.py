"""Training of the learned correction on the GPU: the loss and its parameter
gradient (tensor-core forward, CUDA-core backward, dL/dc gather) against the
FP64 oracle's, the Adam step against its definition, and a short training run
that lowers the loss."""
import numpy as np
import pytest
import torch

from helpers import gpu_cloud_from_state, rel_l2
from oracle import oracle as O
from paper_2512_20829_gb300 import fla
from paper_2512_20829_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = fla.Context(0)
    yield c
    c.close()


def _hmax(kernel, N):
    return (4.0 if kernel == fla.KERNEL_ISO else 3.0) / N


def _problem(dim, N, n, seed, kernel=0, h0_cells=1.5):
    s = I.synthetic_state(dim, n, N, seed=seed, band=(0.15, 0.85), h0_cells=h0_cells, jac_spread=0.3)
    rng = np.random.default_rng(seed + 1)
    nc = N ** dim
    cells = np.sort(rng.choice(nc, min(nc, 600), replace=False))
    # targets: the plain method's sources at those cells, perturbed
    D0 = O.dep_struct(dim=dim, N=N, kernel=kernel, h_min=0.5 / N, h_max=_hmax(kernel, N), p=1.0, window_dt=0.01)
    sm, sv, _ = O.nw_deposit_celllist(D0, s.x, s.J, s.acc, s.status, s.batch, s.n0, s.h0, cells=cells)
    T = np.concatenate([sm[:, None], sv], axis=1) * (1 + 0.2 * rng.standard_normal((cells.size, 1 + dim)))
    return s, cells, T


@pytest.mark.parametrize("dim,N,n,seed,kernel,h0c", [(2, 32, 700, 3, 0, 1.5), (3, 12, 900, 4, 0, 1.5),
                                                     (2, 48, 3000, 5, 0, 1.5), (2, 32, 900, 6, 1, 1.2),
                                                     (3, 12, 1200, 7, 1, 0.8)])
def test_learn_grad_matches_oracle(ctx, dim, N, n, seed, kernel, h0c):
    """Spherical kernel (h scaled) and J-scaled kernel (its Lagrangian bandwidth
    h0 scaled; h_max = 3 cells, so that most supports stay below the trace cap)."""
    s, cells, T = _problem(dim, N, n, seed, kernel, h0c)
    P = fla.init_mlp_params(seed, 0.7)
    P[fla.MLP_PARAMS - 1] = 0.2
    net = fla.LearnedCorrection(ctx, P)
    cl = gpu_cloud_from_state(s, fla.F32)
    m = fla.mesh(dim, N)
    b = fla.LearnBuffers(ctx, cl, m, cells, T, kernel=kernel)
    cfg = fla.deposit_cfg(kernel, 0.5 / N, _hmax(kernel, N), 0.01, mlp=net)
    grad = torch.zeros(fla.MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    fla.learn_grad(ctx, b, cfg, grad, loss)
    torch.cuda.synchronize()
    assert ctx.sync_status(reset=True).flags == 0
    D = O.dep_struct(dim=dim, N=N, kernel=kernel, h_min=0.5 / N, h_max=_hmax(kernel, N), p=1.0, window_dt=0.01,
                     fp32_decision=True, mlp=P)
    L_o, g_o = O.learn_loss_grad(D, s.x, s.J, s.acc, s.status, s.batch, s.n0, s.h0, cells, T)
    if kernel == fla.KERNEL_ANISO:
        _, act, _ = O.learn_records(D, s.x, s.J, s.acc, s.batch, s.n0, s.h0)
        assert act.mean() > 0.3        # Sigma moves with c for a good share of the droplets
    g = grad.double().cpu().numpy()
    L = float(loss.item())
    cos = float(g @ g_o / (np.linalg.norm(g) * np.linalg.norm(g_o)))
    print(f"\ndim {dim} N {N} n {n}: loss {L:.6e} vs {L_o:.6e}; grad rel-L2 {rel_l2(g, g_o):.2e}, cos {cos:.8f}")
    assert L == pytest.approx(L_o, rel=1e-4)
    assert np.linalg.norm(g_o) > 0
    assert rel_l2(g, g_o) <= 2e-3
    # a second call adds the same amounts: the sums are deterministic
    fla.learn_grad(ctx, b, cfg, grad, loss)
    torch.cuda.synchronize()
    assert np.array_equal(grad.double().cpu().numpy(), 2 * g) or rel_l2(grad.double().cpu().numpy(), 2 * g) < 1e-7


def test_adam_step_matches_definition(ctx):
    rng = np.random.default_rng(7)
    n = 10_000
    p = rng.standard_normal(n).astype(np.float32)
    g = rng.standard_normal(n).astype(np.float32)
    m = (0.1 * rng.standard_normal(n)).astype(np.float32)
    v = np.abs(0.1 * rng.standard_normal(n)).astype(np.float32)
    t = [torch.from_numpy(a.copy()).cuda() for a in (p, g, m, v)]
    lr, b1, b2, eps, step = 1e-3, 0.9, 0.999, 1e-8, 5
    fla.adam_step(ctx, t[0], t[1], t[2], t[3], step, lr, b1, b2, eps)
    torch.cuda.synchronize()
    m1 = b1 * m.astype(np.float64) + (1 - b1) * g
    v1 = b2 * v.astype(np.float64) + (1 - b2) * g.astype(np.float64) ** 2
    p1 = p - lr * (m1 / (1 - b1**step)) / (np.sqrt(v1 / (1 - b2**step)) + eps)
    # single-precision update: a few roundings of the inputs' size
    assert np.allclose(t[2].cpu().numpy(), m1, rtol=0, atol=4 * 6e-8 * (np.abs(m) + np.abs(g)).max())
    assert np.allclose(t[3].cpu().numpy(), v1, rtol=1e-6, atol=4 * 6e-8 * (v + g.astype(np.float64)**2).max())
    assert np.allclose(t[0].cpu().numpy(), p1, rtol=0, atol=4 * 6e-8 * np.abs(p).max() + 1e-6 * lr)


def test_short_training_lowers_the_loss(ctx):
    """Targets made by the oracle with every h0 scaled by e^0.5: a network with
    c = 0.5 reaches zero loss wherever h is not clamped."""
    dim, N, n = 2, 48, 3000
    s, cells, _ = _problem(dim, N, n, 11)
    D0 = O.dep_struct(dim=dim, N=N, kernel=0, h_min=0.5 / N, h_max=4.0 / N, p=1.0, window_dt=0.01)
    sm, sv, _ = O.nw_deposit_celllist(D0, s.x, s.J, s.acc, s.status, s.batch, s.n0, s.h0 * np.exp(0.5), cells=cells)
    T = np.concatenate([sm[:, None], sv], axis=1)
    net = fla.LearnedCorrection(ctx, fla.init_mlp_params(12, 0.5, zero_last=True))
    cl = gpu_cloud_from_state(s, fla.F32)
    m = fla.mesh(dim, N)
    b = fla.LearnBuffers(ctx, cl, m, cells, T)
    cfg = fla.deposit_cfg(fla.KERNEL_ISO, 0.5 / N, 4.0 / N, 0.01, mlp=net)
    grad = torch.zeros(fla.MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    mom = torch.zeros_like(grad)
    var = torch.zeros_like(grad)
    losses = []
    for step in range(1, 61):
        grad.zero_()
        loss.zero_()
        fla.learn_grad(ctx, b, cfg, grad, loss)
        fla.adam_step(ctx, net.params, grad, mom, var, step, lr=2e-2)
        net.pack()
        losses.append(float(loss.item()))
    print("\nloss", losses[0], "->", losses[-1])
    assert losses[-1] < 0.5 * losses[0]
