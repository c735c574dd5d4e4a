"""Pins of the oracle's learned bandwidth correction (CPU): bfloat16 rounding,
a network that reduces to a closed form, the features' invariants, the
parameter gradient against central differences, the training loss gradient
against central differences, and the zero-network fallback (P13)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2512_20829_gb300 import inputs as I

H, F = O.MLP_HIDDEN, O.MLP_IN
OFF_W1, OFF_B1 = 0, H * F
OFF_W2 = OFF_B1 + H
OFF_B2 = OFF_W2 + H * H
OFF_W3 = OFF_B2 + H
OFF_B3 = OFF_W3 + H * H
OFF_W4 = OFF_B3 + H
OFF_B4 = OFF_W4 + H


def test_parameter_count():
    assert O.mlp_nparam() == H * F + H + 2 * (H * H + H) + H + 1 == 8833


def _single_path(w4, b3, b4=0.0):
    """W1 = W2 = W3 = 0: c = sum_k bf16(W4_k) silu(b3_k) + b4 with only unit 0 non-zero."""
    P = np.zeros(O.mlp_nparam(), np.float32)
    P[OFF_B3] = b3
    P[OFF_W4] = w4
    P[OFF_B4] = b4
    c, _ = O.mlp_forward(P, np.zeros((1, F)))
    return c[0]


def test_closed_form_last_layer():
    s = lambda z: z / (1 + math.exp(-z))
    # weights exactly representable in bfloat16 pass through unchanged
    assert _single_path(0.75, 1.5, 0.25) == pytest.approx(0.75 * s(1.5) + 0.25, rel=1e-15)
    assert _single_path(-2.0, -3.0) == pytest.approx(-2.0 * s(-3.0), rel=1e-15)


def test_bfloat16_round_to_nearest_even():
    s = lambda z: z / (1 + math.exp(-z))
    z = 2.0
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: ties to the even mantissa (1)
    assert _single_path(1.0 + 2.0**-8, z) == pytest.approx(s(z), rel=1e-15)
    # 1 + 3 * 2^-8 lies halfway between 1 + 2^-7 (odd) and 1 + 2^-6 (even)
    assert _single_path(1.0 + 3 * 2.0**-8, z) == pytest.approx((1.0 + 2.0**-6) * s(z), rel=1e-15)
    # just above a tie rounds up
    assert _single_path(np.float32(1.0 + 2.0**-8 + 2.0**-20), z) == pytest.approx((1.0 + 2.0**-7) * s(z), rel=1e-15)
    # the exact network does not round
    with O.exact_mlp():
        assert _single_path(1.0 + 2.0**-8, z) == pytest.approx((1.0 + 2.0**-8) * s(z), rel=1e-12)


def test_hidden_layers_propagate_through_bias_path():
    """W1 = 0, W2 = identity-like on unit 0: z2_0 = bf16(silu(b1_0)) + b2_0."""
    s = lambda z: z / (1 + math.exp(-z))
    P = np.zeros(O.mlp_nparam(), np.float32)
    P[OFF_B1] = 0.5          # a1_0 = bf16(silu(0.5))
    P[OFF_W2 + 0] = 1.0      # z2_0 = a1_0
    P[OFF_W3 + 0] = 1.0      # z3_0 = bf16(silu(z2_0))
    P[OFF_W4 + 0] = 1.0      # c = silu(z3_0)
    with O.exact_mlp():
        c, _ = O.mlp_forward(P, np.zeros((1, F)))
    assert c[0] == pytest.approx(s(s(s(0.5))), rel=1e-13)


def test_features_invariants():
    rng = np.random.default_rng(1)
    # diagonal J: ||J||^2 = a^2 + b^2, det = ab
    a, b = 3.0, 0.25
    f = O.mlp_features(2, np.diag([a, b]), 2.0, 0.01, 1 / 64)[0]
    assert f[0] == pytest.approx(math.log(a * a + b * b) / 8)
    assert f[1] == pytest.approx(math.log((a * b) ** 2) / 8)
    assert f[2] == pytest.approx(math.log(a * b) / 8)
    assert f[3] == pytest.approx(math.log(2.0 / (a * b)) / 8)
    assert f[4] == pytest.approx(math.log(0.01 * math.sqrt(a * b) * 64) / 4)
    assert f[5] == pytest.approx(a * b / 4)
    # invariance under rotations on either side (3D), and the invariants of J^T J
    J = rng.standard_normal((3, 3))
    Q1, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    Q2, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    f1 = O.mlp_features(3, J, 1.0, 0.02, 1 / 32)[0]
    f2 = O.mlp_features(3, Q1 @ J @ Q2, 1.0, 0.02, 1 / 32)[0]
    assert np.allclose(f1, f2, rtol=0, atol=1e-12)
    sv = np.linalg.svd(J, compute_uv=False)
    assert f1[0] == pytest.approx(math.log(np.sum(sv**2)) / 8)
    I2 = sv[0]**2 * sv[1]**2 + sv[0]**2 * sv[2]**2 + sv[1]**2 * sv[2]**2
    assert f1[1] == pytest.approx(math.log(I2) / 8)
    assert f1[2] == pytest.approx(math.log(np.prod(sv)) / 8)


def _random_params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    parts = []
    for fo, fi in ((H, F), (H, H), (H, H)):
        parts.append(rng.uniform(-1, 1, fo * fi) * scale / math.sqrt(fi))
        parts.append(rng.uniform(-0.2, 0.2, fo))
    parts.append(rng.uniform(-1, 1, H) * scale / math.sqrt(H))
    parts.append(rng.uniform(-0.2, 0.2, 1))
    return np.concatenate(parts).astype(np.float32)


def test_parameter_gradient_matches_central_differences():
    """Backward of the exact network against central differences of the forward."""
    P = _random_params(3)
    f = np.random.default_rng(4).uniform(-1, 1, F)
    with O.exact_mlp():
        g = O.mlp_backward(P, f, 1.0)
        rng = np.random.default_rng(5)
        idx = np.concatenate([rng.choice(np.arange(OFF_W1, OFF_B1), 6), rng.choice(np.arange(OFF_B1, OFF_W2), 4),
                              rng.choice(np.arange(OFF_W2, OFF_B2), 8), rng.choice(np.arange(OFF_W3, OFF_B3), 8),
                              rng.choice(np.arange(OFF_W4, OFF_B4), 4), [OFF_B4, OFF_B2, OFF_B3]])
        for j in idx:
            eps = 1e-3 * max(1.0, abs(float(P[j])))
            Pp, Pm = P.astype(np.float64).copy(), P.astype(np.float64).copy()
            Pp[j] += eps
            Pm[j] -= eps
            # float32 masters: perturb through exactly representable values
            Pp32, Pm32 = Pp.astype(np.float32), Pm.astype(np.float32)
            cp, _ = O.mlp_forward(Pp32, f[None])
            cm, _ = O.mlp_forward(Pm32, f[None])
            fd = (cp[0] - cm[0]) / (float(Pp32[j]) - float(Pm32[j]))
            assert fd == pytest.approx(g[j], rel=1e-4, abs=1e-7), j


def _tiny_cloud(seed, n=48, N=16, dim=2, h0_cells=1.5):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.15, 0.85, (n, dim))
    J = np.eye(dim)[None] + 0.3 * rng.standard_normal((n, dim, dim))
    acc = np.empty((n, 1 + dim))
    acc[:, 0] = -1e-3 * rng.uniform(0.5, 1.5, n)
    acc[:, 1:] = 1e-2 * rng.standard_normal((n, dim))
    status = np.ones(n, np.int32)
    batch = np.zeros(n, np.int32)
    return x, J, acc, status, batch, np.array([1.0]), np.array([h0_cells / N])


# (dim, kernel, mesh, droplets, h0 and h_max in cells): the J-scaled cases keep
# most supports below the trace cap, so that Sigma moves with c
GRAD_CASES = [(2, 0, 16, 48, 1.5, 4.0), (2, 1, 16, 48, 1.5, 4.0), (3, 1, 8, 40, 0.8, 3.0)]


@pytest.mark.parametrize("dim,kernel,N,n,h0c,hmaxc", GRAD_CASES)
def test_training_loss_gradient_matches_central_differences(dim, kernel, N, n, h0c, hmaxc):
    """dL/dtheta through the Nadaraya-Watson ratio (exact network) against
    central differences of the loss, for the spherical kernel (dh/dc = h) and
    the J-scaled kernel (Sigma = e^2c A + h_min^2 I)."""
    x, J, acc, status, batch, n0, h0 = _tiny_cloud(7, n=n, N=N, dim=dim, h0_cells=h0c)
    P = _random_params(8, scale=0.5)
    rng = np.random.default_rng(9)
    cells = np.sort(rng.choice(N ** dim, 120, replace=False))
    target = rng.standard_normal((cells.size, 1 + dim)) * np.array([0.05] + [0.5] * dim)
    kw = dict(dim=dim, N=N, kernel=kernel, h_min=0.5 / N, h_max=hmaxc / N, p=1.0, window_dt=0.01)
    with O.exact_mlp():
        D = O.dep_struct(**kw, mlp=P)
        L, g = O.learn_loss_grad(D, x, J, acc, status, batch, n0, h0, cells, target)
        _, act, _ = O.learn_records(D, x, J, acc, batch, n0, h0)
        assert act.sum() > 20          # most droplets move their bandwidth with c
        idx = np.concatenate([rng.choice(np.arange(OFF_W1, OFF_B1), 6), rng.choice(np.arange(OFF_W2, OFF_B2), 6),
                              rng.choice(np.arange(OFF_W3, OFF_B3), 6), rng.choice(np.arange(OFF_W4, OFF_B4), 6),
                              [OFF_B4]])
        checked = 0
        for j in idx:
            # small steps: a larger one moves some (cell, droplet) pairs across the
            # q = 9 truncation edge, whose jump the gradient (edge held fixed) omits
            eps = 2e-6 * max(1.0, abs(float(P[j])))
            Pp, Pm = P.copy(), P.copy()
            Pp[j] = np.float32(P[j] + eps)
            Pm[j] = np.float32(P[j] - eps)
            Lp, _ = O.learn_loss_grad(O.dep_struct(**kw, mlp=Pp), x, J, acc, status, batch, n0, h0, cells, target,
                                      with_grad=False)
            Lm, _ = O.learn_loss_grad(O.dep_struct(**kw, mlp=Pm), x, J, acc, status, batch, n0, h0, cells, target,
                                      with_grad=False)
            fd = (Lp - Lm) / (float(Pp[j]) - float(Pm[j]))
            assert fd == pytest.approx(g[j], rel=1e-4, abs=1e-8 * max(1.0, abs(L))), (j, fd, g[j])
            checked += 1
        assert checked == idx.size
    assert np.abs(g).max() > 0


@pytest.mark.parametrize("dim", [2, 3])
def test_constant_correction_scales_the_lagrangian_bandwidth(dim):
    """A network whose output is the constant c0 (W4 = 0, b4 = c0) gives the
    J-scaled sources of the plain method with h0 replaced by h0 e^c0 (no droplet
    near a fold, no support at the trace cap)."""
    N = 16 if dim == 2 else 8
    x, J, acc, status, batch, n0, h0 = _tiny_cloud(21, n=60, N=N, dim=dim, h0_cells=1.0)
    dets = np.abs(np.linalg.det(J))
    keep = dets > 0.05
    x, J, acc, status, batch = x[keep], J[keep], acc[keep], status[keep], batch[keep]
    c0 = 0.375
    P = _random_params(22)
    P[OFF_W4:OFF_B4] = 0.0
    P[OFF_B4] = c0
    kw = dict(dim=dim, N=N, kernel=1, h_min=0.5 / N, h_max=6.0 / N, p=1.0, window_dt=0.01)
    with O.exact_mlp():
        c, act, _ = O.learn_records(O.dep_struct(**kw, mlp=P), x, J, acc, batch, n0, h0)
        assert np.all(c == c0) and np.all(act)
        a = O.nw_deposit_celllist(O.dep_struct(**kw, mlp=P), x, J, acc, status, batch, n0, h0)
    b = O.nw_deposit_celllist(O.dep_struct(**kw), x, J, acc, status, batch, n0, h0 * np.exp(c0))
    for u, v in zip(a, b):
        assert np.allclose(u, v, rtol=1e-12, atol=1e-300)
    assert np.abs(a[2]).max() > 0


def test_zero_network_is_the_plain_method():
    """P13: zero last layer gives c = 0, h unchanged, and sources identical to
    the method without the network, bit for bit."""
    N = 32
    s = I.synthetic_state(2, 800, N, seed=12, band=(0.2, 0.8), h0_cells=2.0)
    P = _random_params(13)
    P[OFF_W4:OFF_B4 + 1] = 0.0
    kw = dict(dim=2, N=N, kernel=0, h_min=0.5 / N, h_max=4.0 / N, p=1.0, window_dt=0.01, fp32_decision=True)
    a = O.nw_deposit_celllist(O.dep_struct(**kw), s.x, s.J, s.acc, s.status, s.batch, s.n0, s.h0)
    b = O.nw_deposit_celllist(O.dep_struct(**kw, mlp=P), s.x, s.J, s.acc, s.status, s.batch, s.n0, s.h0)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
