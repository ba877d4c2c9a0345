"""Pins of the FP64 oracle against things other than itself (CPU only).

* closed-form input derivatives of one-hidden-layer tanh networks;
* complex-step input derivatives of deep networks (first order, exact to rounding)
  and Richardson central differences of those for the second order;
* complex-step directional derivatives of the loss for the reverse sweep, and the
  same per coordinate on a tiny network;
* analytic PDE solutions: the viscous Burgers travelling wave (exactly a
  one-neuron tanh network), Kovasznay flow (Navier-Stokes), a TE standing mode
  with PEC walls (Maxwell);
* closed-form losses of constant networks on symmetric point sets;
* torch float64 double-backward autograd (the paper's own method);
* torch.optim.Adam in float64.
Mutation tests plant a mistake in the oracle and check that a pin catches it.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import pinn_oracle as po
from synth import Batch, NetSpec, Problem, init_params, ff_matrix, make_batch, make_workload
from synth.workloads import PDE_BURGERS, PDE_NS, PDE_MAXWELL, PDE_ADVECTION, PDE_ALLEN_CAHN


def _model(spec):
    return oracle.Model.from_spec(spec)


# ------------------------------------------------------------------ tanh derivatives

def test_tanh_identities_against_differences():
    z = np.linspace(-4, 4, 41)
    t, t1, t2, t3 = oracle.tanh_derivs(z)
    # tanh'' = -2 tanh tanh' (the identity used by the GPU jet rule)
    np.testing.assert_allclose(t2, -2 * t * t1, rtol=1e-13, atol=1e-15)
    # each derivative is the derivative of the previous one (Richardson central differences)
    def rich(f, h=1e-3):
        d = lambda hh: (f(z + hh) - f(z - hh)) / (2 * hh)
        return (4 * d(h / 2) - d(h)) / 3
    np.testing.assert_allclose(rich(np.tanh), t1, atol=1e-11)
    np.testing.assert_allclose(rich(lambda x: oracle.tanh_derivs(x)[1]), t2, atol=1e-10)
    np.testing.assert_allclose(rich(lambda x: oracle.tanh_derivs(x)[2]), t3, atol=1e-9)
    # t''' = t' (6 t^2 - 2)
    np.testing.assert_allclose(t3, t1 * (6 * t * t - 2), atol=1e-13)


# ------------------------------------------------------------------ input jets

@pytest.mark.parametrize("rwf", [False, True])
def test_one_hidden_layer_closed_form(rwf):
    spec = NetSpec(PDE_BURGERS, 2, 1, [5], rwf=rwf)
    theta = init_params(spec, 11, random_bias=0.3).astype(np.float64)
    m = _model(spec)
    layers = po.unpack(theta, m.dims, rwf)
    W1 = po.effective_weight(layers[0][0], layers[0][1]); b1 = layers[0][2]
    c = po.effective_weight(layers[1][0], layers[1][1])[0]; d = layers[1][2][0]
    X = np.random.default_rng(1).uniform(-1, 1, (7, 2))
    u, u1, u2 = oracle.output_jets(m, theta, None, X, 2)
    z = X @ W1.T + b1
    sech2 = 1 / np.cosh(z) ** 2
    np.testing.assert_allclose(u[:, 0], np.tanh(z) @ c + d, rtol=1e-14)
    for k in range(2):
        np.testing.assert_allclose(u1[k, :, 0], (sech2 * W1[:, k]) @ c, rtol=1e-13, atol=1e-15)
        for l in range(2):
            closed = (-2 * np.tanh(z) * sech2 * W1[:, k] * W1[:, l]) @ c
            np.testing.assert_allclose(u2[k, l, :, 0], closed, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("ff", [0, 3])
@pytest.mark.parametrize("d_in", [2, 3])
def test_deep_jets_complex_step_and_differences(ff, d_in):
    spec = NetSpec(PDE_NS, d_in, 3, [4, 5, 4], ff_m=ff, ff_sigma=1.3, rwf=True)
    theta = init_params(spec, 21, random_bias=0.2).astype(np.float64)
    B = ff_matrix(spec, 22)
    m = _model(spec)
    X = np.random.default_rng(2).uniform(0, 1, (6, d_in))
    u, u1, u2 = oracle.output_jets(m, theta, B, X, 2)
    h = 1e-30
    for k in range(d_in):
        Xc = X.astype(complex); Xc[:, k] += 1j * h
        uc, _, _ = oracle.output_jets(m, theta, B, Xc, 0)
        np.testing.assert_allclose(u1[k], uc.imag / h, rtol=1e-12, atol=1e-14)
    # second order: Richardson central differences of the (complex-step-pinned) first order
    for l in range(d_in):
        def g(hh):
            Xp, Xm = X.copy(), X.copy(); Xp[:, l] += hh; Xm[:, l] -= hh
            return (oracle.output_jets(m, theta, B, Xp, 1)[1] - oracle.output_jets(m, theta, B, Xm, 1)[1]) / (2 * hh)
        hh = 2e-4
        fd = (4 * g(hh / 2) - g(hh)) / 3
        for k in range(d_in):
            np.testing.assert_allclose(u2[k, l], fd[k], rtol=1e-7, atol=1e-8)
    np.testing.assert_allclose(u2, np.swapaxes(u2, 0, 1), rtol=1e-13, atol=1e-14)


def test_fourier_feature_jets_complex_step():
    rng = np.random.default_rng(3)
    B = rng.normal(0, 2.0, (2, 5))
    X = rng.uniform(0, 1, (4, 2))
    a, a1, a2 = oracle.input_jets(X, B, 2)
    # cosine block first (Eq. 14)
    np.testing.assert_allclose(a[:, :5], np.cos(X @ B), rtol=1e-15)
    np.testing.assert_allclose(a[:, 5:], np.sin(X @ B), rtol=1e-15)
    h = 1e-30
    for k in range(2):
        Xc = X.astype(complex); Xc[:, k] += 1j * h
        ac, _, _ = oracle.input_jets(Xc, B, 0)
        np.testing.assert_allclose(a1[k], ac.imag / h, rtol=1e-13, atol=1e-15)
        for l in range(2):
            Xc2 = X.astype(complex); Xc2[:, l] += 1j * h
            def first(Xr):
                return oracle.input_jets(Xr, B, 1)[1][k]
            dd = 1e-4
            Xp, Xm = X.copy(), X.copy(); Xp[:, l] += dd; Xm[:, l] -= dd
            np.testing.assert_allclose(a2[k, l], (first(Xp) - first(Xm)) / (2 * dd), atol=2e-7)


# ------------------------------------------------------------------ analytic solutions

@pytest.mark.parametrize("rwf", [False, True])
def test_burgers_travelling_wave_is_a_one_neuron_network(rwf):
    # u = c - a tanh(a (x - c t) / (2 nu)) solves u_t + u u_x = nu u_xx exactly.
    a, c, nu = 0.5, 0.3, 0.05
    k = a / (2 * nu)
    spec = NetSpec(PDE_BURGERS, 2, 1, [1], rwf=rwf)
    if rwf:
        theta = np.array([1.0, -c, math.log(k), 0.0, -a, 0.0, c])
    else:
        theta = np.array([k, -k * c, 0.0, -a, c])
    X = np.random.default_rng(4).uniform([-1, 0], [1, 1], (50, 2))
    u, u1, u2 = oracle.output_jets(_model(spec), theta, None, X, 2)
    np.testing.assert_allclose(u[:, 0], c - a * np.tanh(k * (X[:, 0] - c * X[:, 1])), rtol=1e-14)
    r = oracle.residuals(PDE_BURGERS, u, u1, u2, nu)
    assert np.max(np.abs(r)) < 1e-13
    # the residual has teeth: a wrong viscosity leaves a clearly nonzero residual
    assert np.max(np.abs(oracle.residuals(PDE_BURGERS, u, u1, u2, 1.1 * nu))) > 1e-3


def _kovasznay(X, Re):
    lam = Re / 2 - math.sqrt(Re ** 2 / 4 + 4 * math.pi ** 2)
    kk = 2 * math.pi
    x, y = X[:, 0], X[:, 1]
    e, C, S = np.exp(lam * x), np.cos(kk * y), np.sin(kk * y)
    N = X.shape[0]
    u = np.stack([1 - e * C, lam / kk * e * S, 0.5 * (1 - e * e)], axis=1)
    u1 = np.zeros((2, N, 3)); u2 = np.zeros((2, 2, N, 3))
    u1[0, :, 0], u1[1, :, 0] = -lam * e * C, kk * e * S
    u1[0, :, 1], u1[1, :, 1] = lam ** 2 / kk * e * S, lam * e * C
    u1[0, :, 2], u1[1, :, 2] = -lam * e * e, 0.0
    u2[0, 0, :, 0], u2[1, 1, :, 0] = -lam ** 2 * e * C, kk ** 2 * e * C
    u2[0, 0, :, 1], u2[1, 1, :, 1] = lam ** 3 / kk * e * S, -lam * kk * e * S
    return u, u1, u2


def test_kovasznay_flow_zero_navier_stokes_residual():
    Re = 100.0
    X = np.random.default_rng(5).uniform(0, 1, (64, 2))
    u, u1, u2 = _kovasznay(X, Re)
    r = oracle.residuals(PDE_NS, u, u1, u2, 1 / Re)
    assert np.max(np.abs(r)) < 1e-12
    assert np.max(np.abs(oracle.residuals(PDE_NS, u, u1, u2, 1 / 50.0))) > 1e-3


def test_te_standing_mode_zero_maxwell_residual():
    mx, ny = 2, 3
    w = math.pi * math.sqrt(mx * mx + ny * ny)
    X = np.random.default_rng(6).uniform(0, 1, (64, 3))
    x, y, t = X[:, 0], X[:, 1], X[:, 2]
    sx, cx = np.sin(mx * math.pi * x), np.cos(mx * math.pi * x)
    sy, cy = np.sin(ny * math.pi * y), np.cos(ny * math.pi * y)
    st, ct = np.sin(w * t), np.cos(w * t)
    N = X.shape[0]
    u = np.stack([sx * sy * ct, -(ny * math.pi / w) * sx * cy * st, (mx * math.pi / w) * cx * sy * st], axis=1)
    u1 = np.zeros((3, N, 3))
    u1[:, :, 0] = [mx * math.pi * cx * sy * ct, ny * math.pi * sx * cy * ct, -w * sx * sy * st]
    u1[:, :, 1] = [-(ny * math.pi / w) * mx * math.pi * cx * cy * st,
                   (ny * math.pi / w) * ny * math.pi * sx * sy * st,
                   -(ny * math.pi) * sx * cy * ct]
    u1[:, :, 2] = [-(mx * math.pi / w) * mx * math.pi * sx * sy * st,
                   (mx * math.pi / w) * ny * math.pi * cx * cy * st,
                   (mx * math.pi) * cx * sy * ct]
    r = oracle.residuals(PDE_MAXWELL, u, u1, None, 0.0)
    assert np.max(np.abs(r)) < 1e-12
    # PEC: Ez vanishes on the walls
    assert abs(math.sin(mx * math.pi * 1.0)) < 1e-12 and abs(math.sin(ny * math.pi * 0.0)) < 1e-15
    # a sign slip (Hy_x + Hx_y) would be caught
    bad = u1.copy(); bad[1, :, 1] *= -1
    assert np.max(np.abs(oracle.residuals(PDE_MAXWELL, u, bad, None, 0.0))) > 1e-2


def test_advection_exact_solution_zero_residual():
    # u = sin(x - c t) solves u_t + c u_x = 0 (Sec. 4.1); jets written out by hand.
    c = 10.0
    X = np.random.default_rng(7).uniform([0, 0], [2 * math.pi, 1], (64, 2))
    ph = X[:, 0] - c * X[:, 1]
    N = X.shape[0]
    u = np.sin(ph)[:, None]
    u1 = np.zeros((2, N, 1)); u1[0, :, 0] = np.cos(ph); u1[1, :, 0] = -c * np.cos(ph)
    assert np.max(np.abs(oracle.residuals(PDE_ADVECTION, u, u1, None, c))) < 1e-12
    assert np.max(np.abs(oracle.residuals(PDE_ADVECTION, u, u1, None, 0.9 * c))) > 0.5


def test_allen_cahn_stationary_kink_is_a_one_neuron_network():
    # u = tanh(x / delta) with delta = sqrt(2 eps / 5) solves u_t - eps u_xx + 5u^3 - 5u = 0:
    # eps u_xx = -2 eps/delta^2 u (1 - u^2) = 5 (u^3 - u).  It is one tanh neuron.
    eps = 1e-2
    k = 1.0 / math.sqrt(2 * eps / 5)
    spec = NetSpec(PDE_ALLEN_CAHN, 2, 1, [1])
    theta = np.array([k, 0.0, 0.0, 1.0, 0.0])
    X = np.random.default_rng(8).uniform([-1, 0], [1, 1], (50, 2))
    u, u1, u2 = oracle.output_jets(_model(spec), theta, None, X, 2)
    np.testing.assert_allclose(u[:, 0], np.tanh(k * X[:, 0]), rtol=1e-14)
    assert np.max(np.abs(oracle.residuals(PDE_ALLEN_CAHN, u, u1, u2, eps))) < 1e-11
    assert np.max(np.abs(oracle.residuals(PDE_ALLEN_CAHN, u, u1, u2, 1.2 * eps))) > 1e-2


# ------------------------------------------------------------------ loss definitions

def _constant_net_theta(spec, const):
    m = _model(spec)
    theta = np.zeros(sum(fo * fi + fo + (fo if spec.rwf else 0) for fi, fo in m.dims))
    theta[-spec.d_out:] = const      # output bias is the last block
    return m, theta


def test_constant_network_burgers_loss_closed_form():
    spec = NetSpec(PDE_BURGERS, 2, 1, [3, 3])
    c = 0.7
    m, theta = _constant_net_theta(spec, [c])
    n = 64
    xi = -1 + (2 * np.arange(n) + 1) / n           # midpoint grid over one full period of sin(pi x)
    batch = Batch(np.random.default_rng(7).uniform(0, 1, (2, 16)),
                  np.stack([xi, np.zeros(n)]), -np.sin(np.pi * xi)[None], 1,
                  np.stack([np.r_[-np.ones(4), np.ones(4)], np.linspace(0, 1, 8)]), np.zeros((1, 8)), 1)
    terms = oracle.loss_terms(m, theta, None, batch, 0.01, (1.0, 2.0, 3.0))
    assert abs(terms["pde"]) < 1e-30
    assert terms["ic"] == pytest.approx(c * c + 0.5, rel=1e-13)
    assert terms["bc"] == pytest.approx(c * c, rel=1e-13)
    assert terms["total"] == pytest.approx(2.0 * (c * c + 0.5) + 3.0 * c * c, rel=1e-13)


def test_constant_network_cavity_wall_loss_closed_form():
    spec = NetSpec(PDE_NS, 2, 3, [4], ff_m=2, ff_sigma=1.0, rwf=True)
    u0, v0, p0 = 0.4, -0.2, 5.0
    m, theta = _constant_net_theta(spec, [u0, v0, p0])
    B = ff_matrix(spec, 8)
    batch = make_batch(PDE_NS, 32, 0, 400, 9, 10)
    terms = oracle.loss_terms(m, theta, B, batch, 0.01)
    assert abs(terms["pde"]) < 1e-30      # constant outputs have zero derivatives
    # 1/4 of the wall points are on the lid (u = 1); v = 0 everywhere; p unconstrained
    assert terms["bc"] == pytest.approx(0.75 * u0 ** 2 + 0.25 * (u0 - 1) ** 2 + v0 ** 2, rel=1e-6)


# ------------------------------------------------------------------ gradient

@pytest.mark.parametrize("name", ["burgers1d_4x64", "ns_cavity_6x256", "maxwell_te_5x512"])
def test_gradient_complex_step_directions(name):
    w, p, B, b = make_workload(name, n_res=48, n_ic=16, n_bc=16, random_bias=0.1)
    if w.spec.widths[0] > 64:
        w.spec.widths = [16] * 3
        from synth import init_params as ip
        p = ip(w.spec, 99, 0.1)
    m = _model(w.spec)
    terms, g = oracle.loss_and_grad(m, p, B, b, w.problem.nu, (1.0, 0.5, 2.0))
    rng = np.random.default_rng(8)
    h = 1e-30
    for _ in range(3):
        v = rng.standard_normal(p.shape)
        tc = oracle.loss_terms(m, p.astype(np.float64) + 1j * h * v, B, b, w.problem.nu, (1.0, 0.5, 2.0))
        assert tc["total"].real == pytest.approx(terms["total"], rel=1e-13)
        assert tc["total"].imag / h == pytest.approx(g @ v, rel=1e-11)


@pytest.mark.parametrize("pde,d_in,ff", [(PDE_BURGERS, 2, 0), (PDE_NS, 2, 2), (PDE_MAXWELL, 3, 0),
                                         (PDE_ADVECTION, 2, 2), (PDE_ALLEN_CAHN, 2, 0)])
def test_gradient_every_coordinate_complex_step(pde, d_in, ff):
    spec = NetSpec(pde, d_in, 3 if pde in (PDE_NS, PDE_MAXWELL) else 1, [3, 4], ff_m=ff, ff_sigma=1.0, rwf=True)
    p = init_params(spec, 31, 0.2).astype(np.float64)
    B = ff_matrix(spec, 32)
    b = make_batch(pde, 8, 4, 8, 33, 34)
    if pde == PDE_NS:
        b = Batch(b.x_res, b.x_ic, b.g_ic, 0, b.x_bc, b.g_bc, 0b111)
    m = _model(spec)
    _, g = oracle.loss_and_grad(m, p, B, b, 0.02)
    h = 1e-30
    cs = np.empty_like(p)
    for i in range(p.size):
        pc = p.astype(complex); pc[i] += 1j * h
        cs[i] = oracle.loss_terms(m, pc, B, b, 0.02)["total"].imag / h
    np.testing.assert_allclose(g, cs, rtol=1e-10, atol=1e-14 * np.max(np.abs(cs)))


@pytest.mark.parametrize("name", ["burgers1d_4x64", "ns_cavity_6x256", "maxwell_te_5x512", "advection1d_4x128",
                                  "allen_cahn1d_4x128"])
def test_agrees_with_torch_float64_double_backward(name):
    from baseline import torch_autograd
    w, p, B, b = make_workload(name, n_res=64, n_ic=32, n_bc=32, random_bias=0.1)
    if w.spec.widths[0] > 64:
        w.spec.widths = [32] * len(w.spec.widths)
        p = init_params(w.spec, 77, 0.1)
    m = _model(w.spec)
    terms, g = oracle.loss_and_grad(m, p, B, b, w.problem.nu, (1.0, 0.7, 1.3))
    tl, tg, _ = torch_autograd.loss_and_grad(w.spec, p, B, b, w.problem.nu, lambdas=(1.0, 0.7, 1.3))
    assert float(tl) == pytest.approx(terms["total"], rel=1e-12)
    np.testing.assert_allclose(tg.numpy(), g, rtol=1e-9, atol=1e-12 * np.max(np.abs(g)))


# ------------------------------------------------------------------ Adam

def test_adam_matches_torch_float64():
    rng = np.random.default_rng(9)
    theta = rng.standard_normal(50)
    t = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([t], lr=1e-3)
    m = np.zeros(50); v = np.zeros(50); th = theta.copy()
    for step in range(1, 6):
        g = rng.standard_normal(50)
        t.grad = torch.tensor(g)
        opt.step()
        th, m, v = oracle.adam_step(th, g, m, v, step, 1e-3)
    np.testing.assert_allclose(th, t.detach().numpy(), rtol=1e-14, atol=1e-16)


# ------------------------------------------------------------------ mutations

def test_mutation_dropped_second_order_term_is_caught(monkeypatch):
    """Plant a mistake (drop t'' from the jet rule's second-order term); the
    closed-form pin must see it."""
    orig = po.tanh_derivs

    def broken(z):
        t, t1, t2, t3 = orig(z)
        return t, t1, 0 * t2, t3
    spec = NetSpec(PDE_BURGERS, 2, 1, [5])
    theta = init_params(spec, 11, random_bias=0.3).astype(np.float64)
    m = _model(spec)
    X = np.random.default_rng(1).uniform(-1, 1, (7, 2))
    good = oracle.output_jets(m, theta, None, X, 2)[2]
    monkeypatch.setattr(po, "tanh_derivs", broken)
    bad = oracle.output_jets(m, theta, None, X, 2)[2]
    assert np.max(np.abs(good - bad)) > 1e-3


def test_mutation_wrong_adjoint_sign_is_caught(monkeypatch):
    """Plant a sign error in a residual seed; the complex-step pin must see it."""
    w, p, B, b = make_workload("burgers1d_4x64", n_res=16, n_ic=4, n_bc=4, random_bias=0.1)
    m = _model(w.spec)
    orig = po.residual_seeds

    def broken(*a, **k):
        ub, u1b, u2b = orig(*a, **k)
        return ub, u1b, -u2b
    monkeypatch.setattr(po, "residual_seeds", broken)
    _, g = oracle.loss_and_grad(m, p, B, b, w.problem.nu)
    v = np.random.default_rng(3).standard_normal(p.shape)
    cs = oracle.loss_terms(m, p.astype(np.float64) + 1e-30j * v, B, b, w.problem.nu)["total"].imag / 1e-30
    assert abs(cs - g @ v) > 1e-6 * abs(cs)


def test_loss_balance_closed_form():
    """Eqs. 18-19 on gradients with norms 5, 1 and 10: lambda_hat = 16/5, 16, 16/10,
    then one moving-average step with alpha = 0.9 from lambda = (1, 1, 1)."""
    g = np.array([[3.0, 4.0, 0.0], [0.0, 1.0, 0.0], [6.0, 0.0, 8.0]])
    lam, norms = oracle.loss_balance(g, [1.0, 1.0, 1.0], alpha=0.9, eps=0.0)
    assert np.allclose(norms, [5.0, 1.0, 10.0], rtol=0, atol=1e-15)
    assert np.allclose(lam, [0.9 + 0.1 * 3.2, 0.9 + 0.1 * 16.0, 0.9 + 0.1 * 1.6], rtol=1e-15)
    same, _ = oracle.loss_balance(g, [2.0, 3.0, 4.0], update=False)
    assert np.array_equal(same, [2.0, 3.0, 4.0])
    # a term without points (zero gradient) keeps its weight
    g[1] = 0.0
    lam, _ = oracle.loss_balance(g, [1.0, 7.0, 1.0], alpha=0.5, eps=0.0)
    assert lam[1] == 7.0 and np.isclose(lam[0], 0.5 + 0.5 * 15.0 / 5.0)


@pytest.mark.parametrize("name", ["burgers1d_4x64", "maxwell_te_5x512"])
def test_term_gradients_sum_to_the_weighted_gradient(name):
    """Linearity: sum_i lambda_i dL_i/dtheta equals the gradient of the weighted loss,
    and a term without points has a zero gradient."""
    w, p, B, b = make_workload(name, n_res=40, n_ic=12, n_bc=16, random_bias=0.1)
    m = oracle.Model.from_spec(w.spec)
    G = oracle.term_gradients(m, p, B, b, w.problem.nu)
    lam = (0.7, 1.9, 3.1)
    _, g = oracle.loss_and_grad(m, p, B, b, w.problem.nu, lam)
    assert np.allclose(lam[0] * G[0] + lam[1] * G[1] + lam[2] * G[2], g, rtol=1e-12, atol=1e-14 * np.abs(g).max())
    assert all(np.abs(G[i]).max() > 0 for i in range(3))
    b0 = b.subset(40, 0, 16)
    G0 = oracle.term_gradients(m, p, B, b0, w.problem.nu)
    assert np.abs(G0[1]).max() == 0.0


# ------------------------------------------------------------------ temporal causality

def test_causal_weights_closed_form():
    """Eq. 20: omega = (1, e^{-eps L1}, e^{-eps (L1 + L2)}, ...)."""
    w = oracle.causal_weights(np.array([2.0, 3.0, 5.0]), 0.5)
    assert np.allclose(w, [1.0, math.exp(-1.0), math.exp(-2.5)], rtol=1e-15)


def test_causal_loss_reduces_to_segment_mean():
    """eps = 0 gives omega = 1, so L_pde = (1/M) sum_i L^i; with one segment this is the
    plain mean, and the gradient equals the plain gradient."""
    w, p, B, b = make_workload("burgers1d_4x64", n_res=60, n_ic=10, n_bc=10, random_bias=0.1)
    m = oracle.Model.from_spec(w.spec)
    one = dict(segments=1, eps=3.0, t_index=1, t0=0.0, t1=1.0)
    t1, g1 = oracle.loss_and_grad(m, p, B, b, w.problem.nu, causal=one)
    t0, g0 = oracle.loss_and_grad(m, p, B, b, w.problem.nu)
    assert t1["pde"] == pytest.approx(t0["pde"], rel=1e-14) and np.allclose(g1, g0, rtol=1e-13, atol=0)
    four = dict(segments=4, eps=0.0, t_index=1, t0=0.0, t1=1.0)
    t4, _ = oracle.loss_and_grad(m, p, B, b, w.problem.nu, causal=four)
    seg = oracle.causal_segments(b, four)
    (u, u1, u2) = oracle.output_jets(m, p, B, b.x_res.T.astype(np.float64), 2)
    r = oracle.residuals(w.spec.pde, u, u1, u2, w.problem.nu)[0]
    assert t4["pde"] == pytest.approx(np.mean([np.mean(r[seg == i] ** 2) for i in range(4)]), rel=1e-13)


@pytest.mark.parametrize("t0,t1,M,cases", [
    # (t, segment) pairs written out by hand from the definition: segment i is
    # [t0 + i D, t0 + (i + 1) D) with D = (t1 - t0) / M, the last one closed at t1, and
    # times outside [t0, t1] join the first or last segment
    (0.0, 1.0, 4, [(0.0, 0), (0.125, 0), (0.2490234375, 0), (0.25, 1), (0.5, 2), (0.625, 2), (0.75, 3),
                   (0.9990234375, 3), (1.0, 3), (-0.5, 0), (-1e-7, 0), (1.5, 3), (1.0000001, 3)]),
    (-1.0, 1.0, 8, [(-1.0, 0), (-0.75, 1), (-0.5, 2), (-0.25, 3), (0.0, 4), (0.25, 5), (0.5, 6), (0.75, 7),
                    (1.0, 7), (-0.7509765625, 0), (0.7490234375, 6), (-3.0, 0), (2.0, 7)]),
    (0.0, 1.5, 3, [(0.0, 0), (0.4990234375, 0), (0.5, 1), (1.0, 2), (0.9990234375, 1), (1.5, 2), (1.75, 2)]),
    (0.5, 1.0, 1, [(0.5, 0), (0.75, 0), (1.0, 0), (0.0, 0), (2.0, 0)]),
])
def test_causal_segments_hand_placed_times(t0, t1, M, cases):
    """Sec. 2.6.8 cuts the time domain into M equal segments.  Times on t0, on t1, exactly
    on every segment edge (which belongs to the segment above it), just below an edge,
    and outside [t0, t1]: every index is written out by hand, none from the oracle."""
    from synth import Batch
    t = np.array([c[0] for c in cases], dtype=np.float32)
    x_res = np.stack([np.zeros_like(t), t])                  # (x, t): time is input 1
    empty = np.zeros((2, 0), np.float32)
    b = Batch(x_res, empty, np.zeros((1, 0), np.float32), 0, empty, np.zeros((1, 0), np.float32), 0)
    seg = oracle.causal_segments(b, dict(segments=M, eps=1.0, t_index=1, t0=t0, t1=t1))
    assert seg.tolist() == [c[1] for c in cases]


@pytest.mark.parametrize("name", ["burgers1d_4x64", "maxwell_te_5x512"])
def test_causal_gradient_complex_step_with_frozen_weights(name):
    """The gradient holds omega fixed: complex-step on the loss with omega frozen at
    its current value gives the same directional derivatives."""
    w, p, B, b = make_workload(name, n_res=48, n_ic=8, n_bc=8, random_bias=0.1)
    m = oracle.Model.from_spec(w.spec)
    ti = 2 if w.spec.pde == PDE_MAXWELL else 1
    cz = dict(segments=3, eps=0.7, t_index=ti, t0=0.0, t1=1.0)
    terms, g = oracle.loss_and_grad(m, p, B, b, w.problem.nu, (1.0, 0.5, 2.0), causal=cz)
    assert terms["causal_weights"][0] == 1.0 and np.all(np.diff(terms["causal_weights"]) < 0)
    rng = np.random.default_rng(12)
    h = 1e-30
    for _ in range(3):
        v = rng.standard_normal(p.size)
        tc = oracle.loss_terms(m, p.astype(np.float64) + 1j * h * v, B, b, w.problem.nu, (1.0, 0.5, 2.0), causal=cz,
                               omega=terms["causal_weights"])
        assert tc["total"].real == pytest.approx(terms["total"], rel=1e-13)
        assert tc["total"].imag / h == pytest.approx(g @ v, rel=1e-11)


# ------------------------------------------------------------------ L-BFGS

def test_lbfgs_secant_condition():
    """Eq. 24: with the newest pair, H y = s holds exactly for the two-loop matrix."""
    rng = np.random.default_rng(21)
    n = 12
    S = [rng.standard_normal(n) for _ in range(4)]
    A = rng.standard_normal((n, n)); A = A @ A.T + n * np.eye(n)
    Y = [A @ s for s in S]
    Hy = -oracle.lbfgs_direction(Y[-1], S, Y)
    np.testing.assert_allclose(Hy, S[-1], rtol=1e-10, atol=1e-12)
    # without history the direction is steepest descent
    g = rng.standard_normal(n)
    np.testing.assert_array_equal(oracle.lbfgs_direction(g, [], []), -g)


def test_lbfgs_minimises_a_quadratic():
    """On f = x.A x / 2 - b.x the iterates decrease monotonically and reach the
    minimiser A^-1 b."""
    rng = np.random.default_rng(22)
    n = 8
    A = rng.standard_normal((n, n)); A = A @ A.T + np.eye(n)
    b = rng.standard_normal(n)
    fg = lambda x: (0.5 * x @ A @ x - b @ x, A @ x - b)
    losses, x = oracle.lbfgs_minimize(fg, np.zeros(n), history=10, steps=60)
    assert all(l1 <= l0 + 1e-12 for l0, l1 in zip(losses, losses[1:]))
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-6, atol=1e-8)


# ------------------------------------------------------------------ sine activation

def _sine_spec(pde, d_in, d_out, widths, ff=0, rwf=True, omega0=2.0):
    return NetSpec(pde, d_in, d_out, widths, ff_m=ff, ff_sigma=1.0, rwf=rwf, activation="sine", omega0=omega0)


def test_sine_derivatives_against_differences():
    z = np.linspace(-3, 3, 37)
    w = 2.5
    t, t1, t2, t3 = po.sine_derivs(z, w)
    np.testing.assert_allclose(t, np.sin(w * z), rtol=1e-15)
    def rich(f, h=1e-3):
        d = lambda hh: (f(z + hh) - f(z - hh)) / (2 * hh)
        return (4 * d(h / 2) - d(h)) / 3
    np.testing.assert_allclose(rich(lambda x: po.sine_derivs(x, w)[0]), t1, atol=1e-9)
    np.testing.assert_allclose(rich(lambda x: po.sine_derivs(x, w)[1]), t2, atol=1e-8)
    np.testing.assert_allclose(rich(lambda x: po.sine_derivs(x, w)[2]), t3, atol=1e-7)
    # sin'' = -w^2 sin: the second derivative is the function itself, scaled
    np.testing.assert_allclose(t2, -w * w * t, atol=1e-13)


@pytest.mark.parametrize("rwf", [False, True])
def test_sine_one_hidden_layer_closed_form(rwf):
    w0 = 1.7
    spec = _sine_spec(PDE_BURGERS, 2, 1, [5], rwf=rwf, omega0=w0)
    theta = init_params(spec, 13, random_bias=0.3).astype(np.float64)
    m = _model(spec)
    assert m.act == ("sine", w0)
    layers = po.unpack(theta, m.dims, rwf)
    W1 = po.effective_weight(layers[0][0], layers[0][1]); b1 = layers[0][2]
    c = po.effective_weight(layers[1][0], layers[1][1])[0]; d = layers[1][2][0]
    X = np.random.default_rng(6).uniform(-1, 1, (7, 2))
    u, u1, u2 = oracle.output_jets(m, theta, None, X, 2)
    z = X @ W1.T + b1
    np.testing.assert_allclose(u[:, 0], np.sin(w0 * z) @ c + d, rtol=1e-14)
    for k in range(2):
        np.testing.assert_allclose(u1[k, :, 0], (w0 * np.cos(w0 * z) * W1[:, k]) @ c, rtol=1e-13, atol=1e-15)
        for l in range(2):
            closed = (-w0 ** 2 * np.sin(w0 * z) * W1[:, k] * W1[:, l]) @ c
            np.testing.assert_allclose(u2[k, l, :, 0], closed, rtol=1e-12, atol=1e-14)


def test_sine_neuron_is_an_exact_advection_solution():
    # u = sin(k (x - c t)) solves u_t + c u_x = 0: one sine neuron, omega0 folded into W
    k, c, w0 = 1.0, 10.0, 3.0
    spec = _sine_spec(PDE_ADVECTION, 2, 1, [1], rwf=False, omega0=w0)
    theta = np.array([k / w0, -k * c / w0, 0.0, 1.0, 0.0])
    X = np.random.default_rng(7).uniform([0, 0], [2 * np.pi, 1], (40, 2))
    u, u1, u2 = oracle.output_jets(_model(spec), theta, None, X, 2)
    np.testing.assert_allclose(u[:, 0], np.sin(k * (X[:, 0] - c * X[:, 1])), rtol=1e-12, atol=1e-14)
    r = oracle.residuals(PDE_ADVECTION, u, u1, u2, c)
    assert np.max(np.abs(r)) < 1e-12
    assert np.max(np.abs(oracle.residuals(PDE_ADVECTION, u, u1, u2, 1.1 * c))) > 1e-2


@pytest.mark.parametrize("pde,d_in,ff", [(PDE_BURGERS, 2, 0), (PDE_NS, 2, 2), (PDE_MAXWELL, 3, 0),
                                         (PDE_ALLEN_CAHN, 2, 2)])
def test_sine_gradient_every_coordinate_complex_step(pde, d_in, ff):
    spec = _sine_spec(pde, d_in, 3 if pde in (PDE_NS, PDE_MAXWELL) else 1, [3, 4], ff=ff)
    p = init_params(spec, 35, 0.2).astype(np.float64)
    B = ff_matrix(spec, 36)
    b = make_batch(pde, 8, 4, 8, 37, 38)
    if pde == PDE_NS:
        b = Batch(b.x_res, b.x_ic, b.g_ic, 0, b.x_bc, b.g_bc, 0b111)
    m = _model(spec)
    _, g = oracle.loss_and_grad(m, p, B, b, 0.02)
    h = 1e-30
    cs = np.empty_like(p)
    for i in range(p.size):
        pc = p.astype(complex); pc[i] += 1j * h
        cs[i] = oracle.loss_terms(m, pc, B, b, 0.02)["total"].imag / h
    np.testing.assert_allclose(g, cs, rtol=1e-10, atol=1e-14 * np.max(np.abs(cs)))


@pytest.mark.parametrize("name", ["burgers1d_4x64", "ns_cavity_6x256", "maxwell_te_5x512"])
def test_sine_agrees_with_torch_float64_double_backward(name):
    from baseline import torch_autograd
    w, p, B, b = make_workload(name, n_res=48, n_ic=16, n_bc=16, random_bias=0.1)
    w.spec.widths = [24] * 3
    w.spec.activation, w.spec.omega0 = "sine", 1.5
    p = init_params(w.spec, 79, 0.1)
    m = _model(w.spec)
    terms, g = oracle.loss_and_grad(m, p, B, b, w.problem.nu)
    tl, tg, _ = torch_autograd.loss_and_grad(w.spec, p, B, b, w.problem.nu)
    assert float(tl) == pytest.approx(terms["total"], rel=1e-12)
    np.testing.assert_allclose(tg.numpy(), g, rtol=1e-9, atol=1e-12 * np.max(np.abs(g)))


def test_mutation_sine_third_derivative_sign_is_caught(monkeypatch):
    """Plant a sign error in sin''' (used only by the reverse sweep); the complex-step
    gradient pin must see it."""
    good = po.sine_derivs
    monkeypatch.setattr(po, "sine_derivs", lambda z, w: (lambda t: (t[0], t[1], t[2], -t[3]))(good(z, w)))
    with pytest.raises(AssertionError):
        test_sine_gradient_every_coordinate_complex_step(PDE_BURGERS, 2, 0)


# ------------------------------------------------------------------ input-map gradients, periodic map

def _small_case(pde, d_in, d_out, ff, seed):
    spec = NetSpec(pde, d_in, d_out, [5, 4], ff_m=ff, ff_sigma=1.0, rwf=True)
    p = init_params(spec, seed, 0.2).astype(np.float64)
    b = make_batch(pde, 9, 4, 6, seed + 1, seed + 2)
    if pde == PDE_NS:
        b = Batch(b.x_res, b.x_ic, b.g_ic, 0, b.x_bc, b.g_bc, 0b111)
    return spec, p, b


@pytest.mark.parametrize("pde,d_in,d_out", [(PDE_BURGERS, 2, 1), (PDE_NS, 2, 3), (PDE_MAXWELL, 3, 3)])
def test_fourier_matrix_gradient_complex_step(pde, d_in, d_out):
    spec, p, b = _small_case(pde, d_in, d_out, 3, 41)
    B = ff_matrix(spec, 44).astype(np.float64)
    m = _model(spec)
    t, _ = oracle.loss_and_grad(m, p, B, b, 0.02, input_grad=True)
    cs = np.zeros_like(B)
    for e in range(B.shape[0]):
        for j in range(B.shape[1]):
            Bc = B.astype(complex); Bc[e, j] += 1e-30j
            cs[e, j] = oracle.loss_terms(m, p, Bc, b, 0.02)["total"].imag / 1e-30
    np.testing.assert_allclose(t["grad_B"], cs, rtol=1e-10, atol=1e-13 * np.max(np.abs(cs)))


def _periodic_model(pde, d_in, d_out, P):
    return oracle.Model(pde, d_in, d_out, [5, 4], 0, True, None, np.asarray(P, dtype=np.float64))


@pytest.mark.parametrize("pde,d_in,d_out", [(PDE_ADVECTION, 2, 1), (PDE_NS, 2, 3), (PDE_MAXWELL, 3, 3)])
def test_period_gradient_complex_step(pde, d_in, d_out):
    spec, p, b = _small_case(pde, d_in, d_out, d_in, 51)     # fan-in 2 d_in, like the map
    P = np.array([2 * np.pi, 1.3, 0.9])[:d_in]
    m = _periodic_model(pde, d_in, d_out, P)
    t, g = oracle.loss_and_grad(m, p, None, b, 0.02, input_grad=True)
    cs = np.zeros(d_in)
    for k in range(d_in):
        Pc = P.astype(complex); Pc[k] += 1e-30j
        m.periods = Pc
        cs[k] = oracle.loss_terms(m, p, None, b, 0.02)["total"].imag / 1e-30
    np.testing.assert_allclose(t["grad_periods"], cs, rtol=1e-10, atol=1e-14 * np.max(np.abs(cs)))


def test_periodic_map_is_periodic_with_its_derivatives():
    # the paper's point of Eq. 16: values and derivatives agree one period apart
    P = np.array([2.0, 1.5])
    spec, p, _ = _small_case(PDE_BURGERS, 2, 1, 2, 61)
    m = _periodic_model(PDE_BURGERS, 2, 1, P)
    X = np.random.default_rng(9).uniform(0, 1, (10, 2))
    for k in range(2):
        Xs = X.copy(); Xs[:, k] += P[k]
        a = oracle.output_jets(m, p, None, X, 2)
        c = oracle.output_jets(m, p, None, Xs, 2)
        for u, v in zip(a, c):
            np.testing.assert_allclose(u, v, rtol=1e-11, atol=1e-12)
    # a different period breaks it
    m.periods = P * 1.1
    a = oracle.output_jets(m, p, None, X, 0)[0]
    c = oracle.output_jets(m, p, None, X + np.array([P[0], 0.0]), 0)[0]
    assert np.max(np.abs(a - c)) > 1e-3


def ff_column_order(d):
    """Fourier-feature column q of the diagonal map holds periodic-map column perm[q]."""
    return [2 * q for q in range(d)] + [2 * q + 1 for q in range(d)]


def periodic_to_ff_params(theta, dims, d):
    """Permute the first layer's input columns from the paper's order
    [cos x1, sin x1, cos x2, ...] to the Fourier-feature order [cos x1, cos x2, ..., sin x1, ...]."""
    fin, fout = dims[0]
    V = theta[:fin * fout].reshape(fout, fin)
    out = theta.copy()
    out[:fin * fout] = V[:, ff_column_order(d)].ravel()
    return out


@pytest.mark.parametrize("pde,d_in,d_out", [(PDE_ALLEN_CAHN, 2, 1), (PDE_MAXWELL, 3, 3)])
def test_periodic_map_equals_diagonal_fourier_features(pde, d_in, d_out):
    """Eq. 16 is Eq. 14 with B = diag(2 pi / P) up to the first layer's column order,
    and dL/dP_k = -(2 pi / P_k^2) dL/dB_kk: the form the GPU path computes it in."""
    spec, p, b = _small_case(pde, d_in, d_out, d_in, 71)
    P = np.array([2.0, 1.0, 1.5])[:d_in]
    mp = _periodic_model(pde, d_in, d_out, P)
    tp, gp = oracle.loss_and_grad(mp, p, None, b, 0.02, input_grad=True)
    mf = _model(spec)
    pf = periodic_to_ff_params(p, mf.dims, d_in)
    B = np.diag(2 * np.pi / P)
    tf, gf = oracle.loss_and_grad(mf, pf, B, b, 0.02, input_grad=True)
    assert tf["total"] == pytest.approx(tp["total"], rel=1e-13)
    np.testing.assert_allclose(gf, periodic_to_ff_params(gp, mf.dims, d_in), rtol=1e-11, atol=1e-14)
    dP = -2 * np.pi / P ** 2 * np.diag(tf["grad_B"])
    np.testing.assert_allclose(dP, tp["grad_periods"], rtol=1e-11)


def test_mutation_dropped_direction_term_in_fourier_gradient_is_caught(monkeypatch):
    """Plant a mistake in dL/dB (drop the -sin [k=e] term of the derivative rows); the
    complex-step pin on B must see it."""
    good = po.ff_matrix_grad_terms

    def bad(X, B, abar, a1bar, a2bar):
        # the same contraction without the [k=e] terms of the first-derivative rows
        g = good(X, B, abar, a1bar, a2bar)
        if a1bar is None:
            return g
        m = B.shape[1]
        phi = X @ B
        c, s = np.cos(phi), np.sin(phi)
        for e in range(X.shape[1]):
            g[e] -= np.sum(a1bar[e][:, :m] * (-s) + a1bar[e][:, m:] * c, axis=0)
        return g
    monkeypatch.setattr(po, "ff_matrix_grad_terms", bad)
    with pytest.raises(AssertionError):
        test_fourier_matrix_gradient_complex_step(PDE_MAXWELL, 3, 3)


def test_mutation_period_chain_factor_is_caught(monkeypatch):
    """Plant a mistake in dL/dP (return dL/dtheta, forgetting dtheta/dP = -theta/P);
    the complex-step pin on P must see it."""
    good = po.period_grad_terms

    def bad(X, P, abar, a1bar, a2bar):
        th = 2.0 * np.pi / np.asarray(P)
        return good(X, P, abar, a1bar, a2bar) / (-th / np.asarray(P))
    monkeypatch.setattr(po, "period_grad_terms", bad)
    with pytest.raises(AssertionError):
        test_period_gradient_complex_step(PDE_ADVECTION, 2, 1)
