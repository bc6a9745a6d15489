"""Pins of the warm-start network oracle against things other than itself:
scipy's n-d correlation, torch's bfloat16 cast, exact identities (adjoints,
stride-2 = subsampled stride-1, trilinear reproduction, Adam under a constant
gradient, zero-weight network) and central finite differences of the loss."""

from __future__ import annotations

import numpy as np
import pytest
import torch
from scipy.ndimage import correlate

from oracle import warmnet as W
from paper_2604_26441_b300 import inputs


def _rng(seed=0):
    return np.random.default_rng(seed)


@pytest.mark.parametrize("dims,ci,co", [((5, 6, 7), 3, 2), ((3, 4, 9), 2, 4)])
def test_conv_stride1_matches_scipy_correlate(dims, ci, co):
    r = _rng(1)
    x = r.normal(size=(*dims, ci))
    Wt = r.normal(size=(co, 27, ci))
    b = r.normal(size=co)
    got = W.conv3d(x, Wt, b, 1)
    for o in range(co):
        ref = np.full(dims, b[o])
        for c in range(ci):
            k = Wt[o, :, c].reshape(3, 3, 3)  # [dz][dy][dx] since t = dx + 3 dy + 9 dz
            ref += correlate(x[..., c], k, mode="constant", cval=0.0)
        np.testing.assert_allclose(got[..., o], ref, rtol=1e-12, atol=1e-12)


def test_stride2_is_subsampled_stride1():
    r = _rng(2)
    x = r.normal(size=(9, 5, 17, 3))
    Wt = r.normal(size=(4, 27, 3))
    b = r.normal(size=4)
    np.testing.assert_allclose(W.conv3d(x, Wt, b, 2), W.conv3d(x, Wt, b, 1)[::2, ::2, ::2], rtol=1e-13, atol=1e-13)
    assert W.out_dims((9, 5, 17), 2) == (5, 3, 9)


@pytest.mark.parametrize("stride", [1, 2])
def test_conv_backward_is_the_adjoint(stride):
    r = _rng(3)
    x = r.normal(size=(5, 7, 9, 3))
    Wt = r.normal(size=(2, 27, 3))
    b = np.zeros(2)
    y = W.conv3d(x, Wt, b, stride)
    gout = r.normal(size=y.shape)
    gx, gW, gb = W.conv3d_backward(x, Wt, gout, stride)
    # linear in x: <A x, g> = <x, A^T g>
    np.testing.assert_allclose((y * gout).sum(), (x * gx).sum(), rtol=1e-12)
    # linear in W: <A_W x, g> = <W, dW>
    np.testing.assert_allclose((y * gout).sum(), (Wt * gW).sum(), rtol=1e-12)
    np.testing.assert_allclose(gb, gout.reshape(-1, 2).sum(axis=0), rtol=1e-12)


def test_upsample_reproduces_trilinear_fields_and_has_its_adjoint():
    Zc, Yc, Xc = 3, 4, 5
    f = lambda x, y, z: 1.0 + 2.0 * x - 3.0 * y + 0.5 * z + 0.25 * x * y * z - 0.7 * x * z
    kc, jc, ic = np.meshgrid(np.arange(Zc), np.arange(Yc), np.arange(Xc), indexing="ij")
    coarse = f(2.0 * ic, 2.0 * jc, 2.0 * kc)[..., None]
    kf, jf, i_f = np.meshgrid(np.arange(2 * Zc - 1), np.arange(2 * Yc - 1), np.arange(2 * Xc - 1), indexing="ij")
    np.testing.assert_allclose(W.upsample(coarse)[..., 0], f(1.0 * i_f, 1.0 * jf, 1.0 * kf), rtol=1e-13, atol=1e-12)
    r = _rng(4)
    a = r.normal(size=(Zc, Yc, Xc, 2))
    g = r.normal(size=(2 * Zc - 1, 2 * Yc - 1, 2 * Xc - 1, 2))
    np.testing.assert_allclose((W.upsample(a) * g).sum(), (a * W.upsample_adjoint(g)).sum(), rtol=1e-12)


def test_bf16_round_matches_torch():
    r = _rng(5)
    x = np.concatenate([r.normal(size=4000) * 10.0 ** r.integers(-6, 6, size=4000),
                        # exact ties: mantissa low half = 0x8000
                        np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8), 0.0, -0.0])])
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(W.bf16_round(x), ref)
    assert W.bf16_round(np.array([1.0 + 2.0 ** -8]))[0] == 1.0  # tie to even goes down
    assert W.bf16_round(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6  # tie to even goes up


def test_zero_weights_give_the_output_bias():
    theta = np.zeros(W.n_params())
    P = W.unpack(theta)
    for name in P:
        P[name][1][:] = 0.3  # views into theta
    x = _rng(6).normal(size=(9, 9, 9, W.N_IN))
    g, _ = W.forward(theta, x)
    np.testing.assert_allclose(g, 0.3)
    assert W.n_params() == 27 * 28400 + 467


def _tiny_problem(seed=7, n=8):
    rho = inputs.filtered_random_density(n, n, n, seed)
    fixed = inputs.clamp_xmin_mask(n, n, n)
    f = inputs.rotated_tip_edge_load(n, n, n, 3)
    x = W.node_features(n, n, n, rho, f, fixed)
    tgt = _rng(seed).normal(size=(n + 1, n + 1, n + 1, 3))
    theta = inputs.he_normal_params(W.layer_shapes(), seed).astype(np.float64)
    theta += 0.05 * _rng(seed + 1).normal(size=theta.size) * (np.abs(theta) == 0)  # non-zero biases
    return x, tgt, theta


def _loss(theta, x, tgt):
    g, _ = W.forward(theta, x, round_weights=False)
    return W.mse_loss(g, tgt, W.loss_mask(x))[0]


def test_gradient_matches_central_differences_per_layer():
    x, tgt, theta = _tiny_problem()
    g, cache = W.forward(theta, x, round_weights=False)
    _, dg = W.mse_loss(g, tgt, W.loss_mask(x))
    grad, gx = W.backward(cache, dg)
    r = _rng(8)
    k = 0
    # A step may straddle a kink of the leaky ReLU, which spoils that one
    # difference; the best of three step sizes is taken (a wrong gradient term
    # is off at every step size).
    steps = (1e-6, 1e-7, 1e-8)
    for name, ci, co, _, _ in W.LAYERS:
        n = co * 27 * ci + co
        for part in ("W", "b"):
            v = np.zeros_like(theta)
            lo, hi = (k, k + co * 27 * ci) if part == "W" else (k + co * 27 * ci, k + n)
            v[lo:hi] = r.normal(size=hi - lo)
            an = float(grad @ v)
            err = min(abs((_loss(theta + e * v, x, tgt) - _loss(theta - e * v, x, tgt)) / (2 * e) - an)
                      for e in steps)
            assert err <= 1e-6 * max(abs(an), 1e-3), (name, part, err, an)
        k += n
    # input gradient
    v = r.normal(size=x.shape)
    m = W.loss_mask(x)
    an = float((gx * v).sum())

    def fd(e):
        gp, _ = W.forward(theta, x + e * v, round_weights=False)
        gm, _ = W.forward(theta, x - e * v, round_weights=False)
        return (W.mse_loss(gp, tgt, m)[0] - W.mse_loss(gm, tgt, m)[0]) / (2 * e)

    assert min(abs(fd(e) - an) for e in steps) <= 1e-6 * abs(an)


def test_mse_loss_closed_form():
    r = _rng(9)
    t = r.normal(size=(3, 4, 5, 3))
    mask = (r.uniform(size=(3, 4, 5, 1)) > 0.3).astype(float)
    loss, dg = W.mse_loss(t + 0.5, t, mask)
    assert loss == pytest.approx(0.25)
    np.testing.assert_allclose(dg, mask * 1.0 / (3 * mask.sum()) * np.ones_like(t))


def test_adam_under_a_constant_gradient():
    r = _rng(10)
    w0 = r.normal(size=50)
    g = r.normal(size=50)
    w, m, v = w0.copy(), np.zeros(50), np.zeros(50)
    for t in range(1, 8):
        w, m, v = W.adam_step(w, m, v, g, t, 1e-2)
        # bias correction makes m_hat = g and v_hat = g^2 exactly
        np.testing.assert_allclose(w, w0 - t * 1e-2 * g / (np.abs(g) + W.ADAM_EPS), rtol=1e-12, atol=1e-14)


def test_node_features():
    nx, ny, nz = 8, 4, 6
    ex = np.arange(nx)
    rho = np.broadcast_to(0.2 + 0.1 * (ex + 0.5), (nz, ny, nx)).astype(np.float64)
    fixed = inputs.clamp_xmin_mask(nx, ny, nz)
    f = inputs.rotated_tip_edge_load(nx, ny, nz, 5)
    x = W.node_features(nx, ny, nz, rho, f, fixed)
    # a field linear in x averages to its nodal value at interior nodes
    np.testing.assert_allclose(x[:, :, 1:-1, 0], np.broadcast_to(0.2 + 0.1 * np.arange(1, nx), (nz + 1, ny + 1, nx - 1)))
    np.testing.assert_allclose(x[:, :, 0, 0], 0.25)
    assert np.abs(x[..., 1:4]).max() == pytest.approx(1.0)
    np.testing.assert_array_equal(x[:, :, 0, 4], 1.0)
    assert x[:, :, 1:, 4].sum() == 0
    np.testing.assert_allclose(x[2, 3, 5, 5:8], [5 / nx, 3 / ny, 2 / nz])
    th = 2 * np.pi * 5 / 16  # rotated_tip_edge_load direction 5 of 16: (0, sin, -cos)
    np.testing.assert_allclose(x[..., 8:11], np.broadcast_to([0.0, np.sin(th), -np.cos(th)], x[..., 8:11].shape),
                               atol=1e-15)
    np.testing.assert_array_equal(x[..., 11], 1.0)
    assert np.all(W.node_features(nx, ny, nz, rho, 0 * f, fixed)[..., 8:11] == 0)
    np.testing.assert_allclose(W.node_features(nx, ny, nz, np.full((nz, ny, nx), 0.7), f, fixed)[..., 0], 0.7)


def test_warm_start_scaling():
    r = _rng(11)
    A = r.normal(size=(30, 30))
    K = A @ A.T + 30 * np.eye(30)
    f = r.normal(size=30)
    fixed = np.zeros(30, dtype=np.uint8)
    u = np.linalg.solve(K, f)
    for s_ in (3.0, -0.5):
        u0, alpha = W.warm_start(lambda v: K @ v, f, s_ * u, fixed)
        assert alpha == pytest.approx(1 / s_)
        np.testing.assert_allclose(u0, u, rtol=1e-12)
    g = r.normal(size=30)
    u0, alpha = W.warm_start(lambda v: K @ v, f, g, fixed)
    e0, e = u, u - u0
    assert e @ K @ e <= e0 @ K @ e0  # never worse than the cold start in the energy norm
    # the error left is the scale-free energy loss of g against u
    assert (e @ K @ e) / (u @ K @ u) == pytest.approx(W.energy_loss(g, u, fixed, lambda v: K @ v)[0], rel=1e-10)
    u0n, alphan = W.warm_start(lambda v: K @ v, f, -g, fixed)
    assert alphan == pytest.approx(-alpha) and np.allclose(u0n, u0)
    assert W.warm_start(lambda v: K @ v, f, np.zeros(30), fixed)[1] == 0.0


def _tiny_operator(n=8, seed=7):
    from oracle import fem
    rho = inputs.filtered_random_density(n, n, n, seed)
    fixed = inputs.clamp_xmin_mask(n, n, n)
    grid = fem.Grid(n, n, n)
    E, Ke = fem.moduli(rho, 3.0), fem.element_stiffness(0.3)
    return fixed, (lambda v: fem.matfree_apply(grid, E, Ke, v))


def test_energy_loss_closed_forms():
    fixed, K = _tiny_operator()
    free = fixed == 0
    r = _rng(13)
    t = r.normal(size=fixed.size) * free
    for g in (t, 2.5 * t, -0.3 * t, t + 5.0 * fixed):  # scale-free, sign-free, blind to fixed DOFs
        assert W.energy_loss(g, t, fixed, K)[0] == pytest.approx(0.0, abs=1e-12)
    assert W.energy_loss(np.zeros_like(t), t, fixed, K)[0] == 1.0
    # against the definition: the best rescaling by a scan in the K inner product
    g = r.normal(size=fixed.size) * free
    Kt, Kg = K(t) * free, K(g) * free
    alphas = np.linspace(-2, 2, 40001) * (t @ Kg) / (g @ Kg)
    brute = min(((t - a * g) @ (Kt - a * Kg)) for a in alphas) / (t @ Kt)
    L = W.energy_loss(g, t, fixed, K)[0]
    assert 0.0 <= L <= 1.0 and L == pytest.approx(brute, rel=1e-6)


def test_energy_loss_gradient_matches_central_differences():
    """The loss is a smooth function of the output g, so central differences in
    g are accurate; the network's own backward pass is pinned per layer
    above, and train_step is checked to chain the two."""
    fixed, K = _tiny_operator(seed=14)
    r = _rng(15)
    t = r.normal(size=fixed.size)
    g = r.normal(size=fixed.size)
    L, dg = W.energy_loss(g, t, fixed, K)
    for _ in range(3):
        v = r.normal(size=g.size)
        fd = (W.energy_loss(g + 1e-5 * v, t, fixed, K)[0] - W.energy_loss(g - 1e-5 * v, t, fixed, K)[0]) / 2e-5
        assert fd == pytest.approx(float(dg @ v), rel=1e-6)
    x, _, theta = _tiny_problem(14)
    tgt = t.reshape(9, 9, 9, 3)
    x2 = x.copy()
    x2[..., 0] = 0.5
    loss, grad, _, _, _ = W.train_step(theta, np.zeros_like(theta), np.zeros_like(theta), 1, 0.0,
                                       [(x, tgt), (x2, -tgt)], ops=[(fixed, K), (fixed, K)])
    parts = []
    for xx, tt in ((x, tgt), (x2, -tgt)):
        gr, cr = W.forward(theta, xx)
        Lr, dr = W.energy_loss(gr, tt, fixed, K)
        parts.append((Lr, W.backward(cr, (dr / 2).reshape(gr.shape))[0]))
    assert loss == pytest.approx(0.5 * (parts[0][0] + parts[1][0]), rel=1e-14)
    np.testing.assert_allclose(grad, parts[0][1] + parts[1][1], rtol=1e-12, atol=1e-15)


def test_gradient_clipping():
    g = np.array([3.0, 4.0])
    np.testing.assert_allclose(W.clip_gradient(g, 1.0), [0.6, 0.8])
    np.testing.assert_array_equal(W.clip_gradient(g, 10.0), g)
    np.testing.assert_array_equal(W.clip_gradient(g, 0.0), g)
    assert np.all(W.clip_gradient(np.array([np.inf, 1.0]), 1.0) == 0)


def test_training_lowers_the_loss():
    x, tgt, theta = _tiny_problem(12)
    tgt = np.broadcast_to(x[..., 5:6] ** 2, tgt.shape).copy()  # a smooth target
    m, v = np.zeros_like(theta), np.zeros_like(theta)
    losses = []
    for t in range(1, 16):
        loss, _, theta, m, v = W.train_step(theta, m, v, t, 3e-3, [(x, tgt)])
        losses.append(loss)
    assert losses[-1] < 0.5 * losses[0]
