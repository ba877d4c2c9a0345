"""FP64 CPU oracle for the PINN loss and its parameter gradient.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's CPU
baseline may import this module; the library's compute path never does.  It
shares no code with the CUDA path (it imports only numpy).

What it computes, in the paper's order and notation:
  * Random Fourier features (Sec. 2.6.1, Eq. 14): gamma(x) = [cos(xB), sin(xB)],
    B of shape [d, m] drawn N(0, sigma^2) and frozen (not trained).
  * Random weight factorisation (Sec. 2.6.2, Eq. 15): W^(l) = diag(exp(s^(l))) V^(l)
    for every layer l = 1..L+1.
  * The MLP (Sec. 2.2, Eqs. 4-6): f^(l) = W^(l) g^(l-1) + b^(l), g^(l) = tanh(f^(l))
    for l = 1..L, and a final linear layer without activation.
  * Input derivatives by the explicit chain rule (forward-mode jets): for each
    point the value, the full gradient and (when the PDE needs it) the full
    Hessian with respect to the inputs are carried through every layer.  This is
    what the paper obtains with autograd (Sec. 2.3, "autoGrad" terms).
  * Residuals: viscous Burgers u_t + u u_x - nu u_xx (Sec. 4.3 with viscosity),
    steady incompressible Navier-Stokes (Sec. 4.4, continuity and two momentum
    equations, nu = 1/Re), TE Maxwell with eps = mu = 1 (Sec. 4.8, Eqs. for
    dEz/dt, dHx/dt, dHy/dt).
  * Loss (Sec. 2.3, Eqs. 10-13 and Sec. 2.6.4 Eq. 17): each term is a mean of
    squares over its own point set; several equations or output components are
    summed; L = lambda_pde L_pde + lambda_ic L_ic + lambda_bc L_bc.
  * Gradient: an explicit reverse sweep through the jets (adjoint of each step
    above), then the RWF chain rule dL/dV = exp(s) * dL/dW, dL/ds_i =
    sum_j dL/dW_ij W_ij.  B gets no gradient in training; ff_matrix_grad gives
    dL/dB from the adjoint of the input jets for callers that want it.
  * Strict periodic input map (Sec. 2.6.3, Eq. 16): w = [cos(2 pi x_k / P_k),
    sin(2 pi x_k / P_k)] per input k, in that order; the gradient with respect to
    the periods P_k (P_t is trainable in the paper) by the same input adjoint.
  * Periodic activation (Sec. 2.6, Table 1): sin(omega0 z) in place of tanh.
  * Adam (Sec. 2.6.5): biased moments, bias correction, theta -= alpha m_hat /
    (sqrt(v_hat) + eps).

All arithmetic is float64 (or complex128 when a caller passes complex parameters
for complex-step differentiation; every operation used here is analytic).

Readings where the paper is silent or garbled (also listed in the design notes):
  * Adam betas are garbled in the text; the paper trains with torch's Adam at its
    defaults, so beta1 = 0.9, beta2 = 0.999; eps = 1e-8 as printed.
  * Every layer (including RWF layers) has a bias b^(l) as in Eq. 4.
  * Multi-equation / multi-component terms are sums of per-equation means.
  * tanh'(z) is evaluated as 1/cosh(z)^2 here (the GPU path uses (1-t)(1+t)).
  * The periodic map keeps the paper's column order, cos then sin per input; a network
    whose first layer takes [cos x1, cos x2, ..., sin x1, ...] is the same function with
    its first-layer columns permuted.
  * The sine activation takes omega0 as given, with no special initialisation (the
    paper names the hyper-parameter only).
"""
from __future__ import annotations

import numpy as np

PDE_BURGERS, PDE_NS, PDE_MAXWELL, PDE_ADVECTION, PDE_ALLEN_CAHN = 0, 1, 2, 3, 4

# Which input-derivative order each residual needs (Burgers/NS: second, Maxwell: first).
PDE_ORDER = {PDE_BURGERS: 2, PDE_NS: 2, PDE_MAXWELL: 1, PDE_ADVECTION: 1, PDE_ALLEN_CAHN: 2}
PDE_N_EQ = {PDE_BURGERS: 1, PDE_NS: 3, PDE_MAXWELL: 3, PDE_ADVECTION: 1, PDE_ALLEN_CAHN: 1}


# --------------------------------------------------------------------------------------
# Parameters
# --------------------------------------------------------------------------------------

def layer_dims(d_in, d_out, widths, ff_m):
    """(fan_in, fan_out) for l = 1..L+1; the first fan_in is 2m with Fourier features."""
    dims, prev = [], (2 * ff_m if ff_m else d_in)
    for w in widths:
        dims.append((prev, w))
        prev = w
    dims.append((prev, d_out))
    return dims


def unpack(theta, dims, rwf):
    """Split the packed vector: per layer V[out,in] row-major | s[out] (RWF) | b[out]."""
    layers, off = [], 0
    for fi, fo in dims:
        V = theta[off:off + fo * fi].reshape(fo, fi); off += fo * fi
        s = None
        if rwf:
            s = theta[off:off + fo]; off += fo
        b = theta[off:off + fo]; off += fo
        layers.append((V, s, b))
    assert off == theta.shape[0], "parameter vector length does not match the layer layout"
    return layers


def effective_weight(V, s):
    """Eq. 15: W = diag(exp(s)) V (or V itself without RWF)."""
    if s is None:
        return V
    return np.exp(s)[:, None] * V


# --------------------------------------------------------------------------------------
# tanh and its derivatives (from sech^2, independently of the identity t'' = -2 t t')
# --------------------------------------------------------------------------------------

def sine_derivs(z, omega):
    """The periodic activation sin(omega z) (appendix, periodic activation function) and
    its first three derivatives."""
    s, c = np.sin(omega * z), np.cos(omega * z)
    return s, omega * c, -omega ** 2 * s, -omega ** 3 * c


def act_derivs(z, act):
    """(t, t', t'', t''') of the hidden activation: act None / "tanh" or ("sine", omega)."""
    if act is None or act == "tanh":
        return tanh_derivs(z)
    return sine_derivs(z, act[1])


def tanh_derivs(z):
    t = np.tanh(z)
    sech2 = 1.0 / np.cosh(z) ** 2
    t1 = sech2                                   # d/dz tanh
    t2 = -2.0 * sech2 * t                        # d/dz sech^2
    t3 = 4.0 * sech2 * t * t - 2.0 * sech2 * sech2   # d/dz (-2 sech^2 tanh)
    return t, t1, t2, t3


# --------------------------------------------------------------------------------------
# Input jets
# --------------------------------------------------------------------------------------

def periodic_input_jets(X, P, order):
    """Jets of the strict periodic input map of Eq. 16 at points X [N, d], in the
    paper's order [cos(2 pi x_1/P_1), sin(2 pi x_1/P_1), cos(2 pi x_2/P_2), ...].
    With theta_k = 2 pi / P_k: d cos/dx_k = -sin theta_k, d sin/dx_k = cos theta_k,
    d^2 cos/dx_k^2 = -cos theta_k^2, d^2 sin/dx_k^2 = -sin theta_k^2 (other
    directions 0).  Complex-safe in X and P."""
    N, d = X.shape
    th = 2.0 * np.pi / np.asarray(P)
    dt = np.result_type(X, th)
    a = np.zeros((N, 2 * d), dtype=dt)
    a1 = np.zeros((d, N, 2 * d), dtype=dt) if order >= 1 else None
    a2 = np.zeros((d, d, N, 2 * d), dtype=dt) if order >= 2 else None
    for k in range(d):
        c, s = np.cos(th[k] * X[:, k]), np.sin(th[k] * X[:, k])
        a[:, 2 * k], a[:, 2 * k + 1] = c, s
        if order >= 1:
            a1[k, :, 2 * k], a1[k, :, 2 * k + 1] = -s * th[k], c * th[k]
        if order >= 2:
            a2[k, k, :, 2 * k], a2[k, k, :, 2 * k + 1] = -c * th[k] ** 2, -s * th[k] ** 2
    return a, a1, a2


def input_jets(X, B, order):
    """Jets of the network input for points X [N, d].

    Returns (a, a1, a2): a [N, w0]; a1 [d, N, w0] with a1[k] = d a / d x_k;
    a2 [d, d, N, w0] with a2[k, l] = d^2 a / d x_k d x_l (None when order < 2).
    Without Fourier features the input is x itself (unit gradient, zero Hessian).
    With them (Eq. 14): phi = X B, gamma = [cos phi, sin phi] (cosine block first),
    d cos(phi_j)/dx_k = -sin(phi_j) B_kj, d sin(phi_j)/dx_k = cos(phi_j) B_kj,
    d^2 cos(phi_j)/dx_k dx_l = -cos(phi_j) B_kj B_lj, d^2 sin = -sin(phi_j) B_kj B_lj.
    """
    N, d = X.shape
    if B is None:
        a = X.copy()
        a1 = np.zeros((d, N, d), dtype=X.dtype) if order >= 1 else None
        if order >= 1:
            for k in range(d):
                a1[k, :, k] = 1.0
        a2 = np.zeros((d, d, N, d), dtype=X.dtype) if order >= 2 else None
        return a, a1, a2
    phi = X @ B
    c, s = np.cos(phi), np.sin(phi)
    a = np.concatenate([c, s], axis=1)
    a1 = a2 = None
    if order >= 1:
        a1 = np.stack([np.concatenate([-s * B[k][None, :], c * B[k][None, :]], axis=1) for k in range(d)])
    if order >= 2:
        a2 = np.empty((d, d) + a.shape, dtype=a.dtype)
        for k in range(d):
            for l in range(d):
                bb = (B[k] * B[l])[None, :]
                a2[k, l] = np.concatenate([-c * bb, -s * bb], axis=1)
    return a, a1, a2


# --------------------------------------------------------------------------------------
# Forward jets through the MLP
# --------------------------------------------------------------------------------------

def forward(Ws, bs, X, B, order, act=None, periods=None):
    """Propagate jets through hidden tanh layers and the final linear layer.

    Linear layer (Eq. 4): z = a W^T + b on the value; derivatives are linear:
    z1_k = a1_k W^T, z2_kl = a2_kl W^T.  Activation (Eq. 5) by the chain rule:
    a = t(z), a1_k = t'(z) z1_k, a2_kl = t''(z) z1_k z1_l + t'(z) z2_kl.
    Returns output jets (u, u1, u2) and the per-layer cache for the reverse sweep.
    With `periods` the input is the periodic map of Eq. 16 instead.
    """
    a, a1, a2 = input_jets(X, B, order) if periods is None else periodic_input_jets(X, periods, order)
    cache = []
    L = len(Ws) - 1
    for l in range(L):
        W, b = Ws[l], bs[l]
        z = a @ W.T + b
        z1 = a1 @ W.T if order >= 1 else None
        z2 = a2 @ W.T if order >= 2 else None
        cache.append((a, a1, a2, z, z1, z2))
        t, t1, t2, _ = act_derivs(z, act)
        na = t
        na1 = t1[None] * z1 if order >= 1 else None
        na2 = None
        if order >= 2:
            na2 = t2[None, None] * z1[:, None] * z1[None, :] + t1[None, None] * z2
        a, a1, a2 = na, na1, na2
    W, b = Ws[L], bs[L]
    cache.append((a, a1, a2, None, None, None))
    u = a @ W.T + b
    u1 = a1 @ W.T if order >= 1 else None
    u2 = a2 @ W.T if order >= 2 else None
    return (u, u1, u2), cache


def backward(Ws, cache, ubar, u1bar, u2bar, order, act=None, input_adjoint=False):
    """Reverse sweep through the jets of forward().  Returns (dW list, db list), and
    with `input_adjoint` also the adjoint of the input jets (abar, a1bar, a2bar) =
    (gbar W_1, g1bar W_1, g2bar W_1) of the first layer.

    Output layer: abar = ubar W, a1bar_k = u1bar_k W, a2bar_kl = u2bar_kl W;
    dW = ubar^T a + sum_k u1bar_k^T a1_k + sum_kl u2bar_kl^T a2_kl; db = sum ubar.
    Hidden layer (adjoint of the activation chain rule above):
      zbar    = abar t' + sum_k a1bar_k t'' z1_k + sum_kl a2bar_kl (t''' z1_k z1_l + t'' z2_kl)
      z1bar_k = a1bar_k t' + sum_l (a2bar_kl + a2bar_lk) t'' z1_l
      z2bar_kl = a2bar_kl t'
    """
    L = len(Ws) - 1
    dWs, dbs = [None] * (L + 1), [None] * (L + 1)
    gbar, g1bar, g2bar = ubar, u1bar, u2bar     # adjoint of this layer's output (pre-activation side)
    for l in range(L, -1, -1):
        a, a1, a2, _, _, _ = cache[l]
        dW = gbar.T @ a
        if order >= 1:
            dW = dW + np.einsum("kni,knj->ij", g1bar, a1)
        if order >= 2:
            dW = dW + np.einsum("klni,klnj->ij", g2bar, a2)
        dWs[l] = dW
        dbs[l] = gbar.sum(axis=0)
        if l == 0:
            if input_adjoint:
                W = Ws[0]
                return dWs, dbs, (gbar @ W, g1bar @ W if order >= 1 else None, g2bar @ W if order >= 2 else None)
            break
        W = Ws[l]
        abar = gbar @ W
        a1bar = g1bar @ W if order >= 1 else None
        a2bar = g2bar @ W if order >= 2 else None
        _, _, _, z, z1, z2 = cache[l - 1]
        t, t1, t2, t3 = act_derivs(z, act)
        zbar = abar * t1
        if order >= 1:
            zbar = zbar + np.sum(a1bar * t2[None] * z1, axis=0)
        if order >= 2:
            zbar = zbar + np.sum(a2bar * (t3[None, None] * z1[:, None] * z1[None, :] + t2[None, None] * z2),
                                 axis=(0, 1))
        z1bar = None
        if order >= 1:
            z1bar = a1bar * t1[None]
            if order >= 2:
                sym = a2bar + np.swapaxes(a2bar, 0, 1)
                z1bar = z1bar + np.sum(sym * t2[None, None] * z1[None, :], axis=1)
        z2bar = a2bar * t1[None, None] if order >= 2 else None
        gbar, g1bar, g2bar = zbar, z1bar, z2bar
    return dWs, dbs


# --------------------------------------------------------------------------------------
# Residuals and their partial derivatives with respect to the output jets
# --------------------------------------------------------------------------------------

def residuals(pde, u, u1, u2, nu):
    """Residuals r_eq [n_eq, N] from output jets (u [N,c], u1 [d,N,c], u2 [d,d,N,c]).

    Burgers (inputs x, t; output u):           r = u_t + u u_x - nu u_xx
    Navier-Stokes (inputs x, y; outputs u,v,p): r1 = u u_x + v u_y + p_x - nu (u_xx + u_yy)
                                                r2 = u v_x + v v_y + p_y - nu (v_xx + v_yy)
                                                r3 = u_x + v_y
    Maxwell TE (inputs x, y, t; Ez, Hx, Hy):     r1 = Ez_t - (Hy_x - Hx_y)
                                                r2 = Hx_t + Ez_y
                                                r3 = Hy_t - Ez_x
    Advection (Sec. 4.1; inputs x, t; u):        r = u_t + c u_x, with c = nu
    Allen-Cahn (Sec. 4.2; inputs x, t; u):       r = u_t - eps u_xx + 5 u^3 - 5 u, with eps = nu
    """
    if pde == PDE_BURGERS:
        U, Ux, Ut, Uxx = u[:, 0], u1[0, :, 0], u1[1, :, 0], u2[0, 0, :, 0]
        return np.stack([Ut + U * Ux - nu * Uxx])
    if pde == PDE_NS:
        U, V, P = u[:, 0], u[:, 1], u[:, 2]
        Ux, Uy, Vx, Vy, Px, Py = u1[0, :, 0], u1[1, :, 0], u1[0, :, 1], u1[1, :, 1], u1[0, :, 2], u1[1, :, 2]
        lapU = u2[0, 0, :, 0] + u2[1, 1, :, 0]
        lapV = u2[0, 0, :, 1] + u2[1, 1, :, 1]
        r1 = U * Ux + V * Uy + Px - nu * lapU
        r2 = U * Vx + V * Vy + Py - nu * lapV
        r3 = Ux + Vy
        return np.stack([r1, r2, r3])
    if pde == PDE_MAXWELL:
        Ez_x, Ez_y, Ez_t = u1[0, :, 0], u1[1, :, 0], u1[2, :, 0]
        Hx_y, Hx_t = u1[1, :, 1], u1[2, :, 1]
        Hy_x, Hy_t = u1[0, :, 2], u1[2, :, 2]
        return np.stack([Ez_t - (Hy_x - Hx_y), Hx_t + Ez_y, Hy_t - Ez_x])
    if pde == PDE_ADVECTION:
        return np.stack([u1[1, :, 0] + nu * u1[0, :, 0]])
    if pde == PDE_ALLEN_CAHN:
        U = u[:, 0]
        return np.stack([u1[1, :, 0] - nu * u2[0, 0, :, 0] + 5.0 * U ** 3 - 5.0 * U])
    raise ValueError(pde)


def residual_seeds(pde, u, u1, u2, nu, coef):
    """Adjoint of sum_eq coef * sum_i r_eq,i^2 with respect to the output jets.

    With rbar = 2 coef r, each jet entry q receives sum_eq rbar_eq dr_eq/dq,
    the partials of the residual polynomials above written out by hand.
    """
    r = residuals(pde, u, u1, u2, nu)
    rb = 2.0 * coef * r
    ub = np.zeros_like(u)
    u1b = np.zeros_like(u1)
    u2b = np.zeros_like(u2) if u2 is not None else None
    if pde == PDE_BURGERS:
        U, Ux = u[:, 0], u1[0, :, 0]
        g = rb[0]
        ub[:, 0] = g * Ux              # d r / d u = u_x
        u1b[0, :, 0] = g * U           # d r / d u_x = u
        u1b[1, :, 0] = g               # d r / d u_t = 1
        u2b[0, 0, :, 0] = -nu * g      # d r / d u_xx = -nu
    elif pde == PDE_NS:
        U, V = u[:, 0], u[:, 1]
        Ux, Uy, Vx, Vy = u1[0, :, 0], u1[1, :, 0], u1[0, :, 1], u1[1, :, 1]
        g1, g2, g3 = rb
        ub[:, 0] = g1 * Ux + g2 * Vx
        ub[:, 1] = g1 * Uy + g2 * Vy
        u1b[0, :, 0] = g1 * U + g3     # u_x
        u1b[1, :, 0] = g1 * V          # u_y
        u1b[0, :, 1] = g2 * U          # v_x
        u1b[1, :, 1] = g2 * V + g3     # v_y
        u1b[0, :, 2] = g1              # p_x
        u1b[1, :, 2] = g2              # p_y
        u2b[0, 0, :, 0] = -nu * g1
        u2b[1, 1, :, 0] = -nu * g1
        u2b[0, 0, :, 1] = -nu * g2
        u2b[1, 1, :, 1] = -nu * g2
    elif pde == PDE_MAXWELL:
        g1, g2, g3 = rb
        u1b[2, :, 0] = g1              # Ez_t in r1
        u1b[0, :, 2] = -g1             # Hy_x in r1
        u1b[1, :, 1] = g1              # Hx_y in r1
        u1b[2, :, 1] = g2              # Hx_t in r2
        u1b[1, :, 0] = g2              # Ez_y in r2
        u1b[2, :, 2] = g3              # Hy_t in r3
        u1b[0, :, 0] = -g3             # Ez_x in r3
    elif pde == PDE_ADVECTION:
        g = rb[0]
        u1b[0, :, 0] = nu * g          # d r / d u_x = c
        u1b[1, :, 0] = g               # d r / d u_t = 1
    elif pde == PDE_ALLEN_CAHN:
        U = u[:, 0]
        g = rb[0]
        ub[:, 0] = g * (15.0 * U ** 2 - 5.0)   # d r / d u = 15 u^2 - 5
        u1b[1, :, 0] = g               # d r / d u_t = 1
        u2b[0, 0, :, 0] = -nu * g      # d r / d u_xx = -eps
    return ub, u1b, u2b


# --------------------------------------------------------------------------------------
# Loss and gradient
# --------------------------------------------------------------------------------------

class Model:
    """Architecture description for the oracle (plain data)."""

    def __init__(self, pde, d_in, d_out, widths, ff_m=0, rwf=False, act=None, periods=None):
        self.pde, self.d_in, self.d_out = pde, d_in, d_out
        self.widths, self.ff_m, self.rwf = list(widths), ff_m, rwf
        self.act = act       # None (tanh) or ("sine", omega0)
        self.periods = periods   # None, or [P_1..P_d]: the periodic input map of Eq. 16
        self.dims = layer_dims(d_in, d_out, widths, d_in if periods is not None else ff_m)

    @classmethod
    def from_spec(cls, spec):
        act = ("sine", spec.omega0) if getattr(spec, "activation", "tanh") == "sine" else None
        return cls(spec.pde, spec.d_in, spec.d_out, spec.widths, spec.ff_m, spec.rwf, act)


def _weights(model, theta):
    layers = unpack(theta, model.dims, model.rwf)
    Ws = [effective_weight(V, s) for V, s, _ in layers]
    bs = [b for _, _, b in layers]
    return layers, Ws, bs


def _coords(x):
    return np.asarray(x, dtype=np.float64).T      # SoA [d][N] -> [N, d]


def loss_terms(model, theta, B, batch, nu, lambdas=(1.0, 1.0, 1.0), causal=None, omega=None):
    """Loss terms as a dict: total, pde, pde_eq (list), ic, bc.  Complex-safe.  With
    `causal` (see loss_and_grad) the PDE term is causally weighted, with the weights
    `omega` held fixed when given (for complex-step checks of the stop-gradient
    gradient), else evaluated from the segment losses."""
    theta = np.asarray(theta)
    if not np.iscomplexobj(theta):
        theta = theta.astype(np.float64)
    Bd = None if B is None else (np.asarray(B) if np.iscomplexobj(B) else np.asarray(B, dtype=np.float64))
    _, Ws, bs = _weights(model, theta)
    lam_pde, lam_ic, lam_bc = lambdas
    order = PDE_ORDER[model.pde]
    out = {"pde_eq": [0.0] * PDE_N_EQ[model.pde], "pde": 0.0, "ic": 0.0, "bc": 0.0}
    if batch.n_res:
        (u, u1, u2), _ = forward(Ws, bs, _coords(batch.x_res), Bd, order, model.act, model.periods)
        r = residuals(model.pde, u, u1, u2, nu)
        if causal is None:
            per_eq = [np.mean(r[e] * r[e]) for e in range(r.shape[0])]
        else:
            M = causal["segments"]
            seg = causal_segments(batch, causal)
            seg_eq = []
            for i in range(M):
                sel = seg == i
                seg_eq.append([np.mean(r[e][sel] ** 2) if np.any(sel) else 0.0 for e in range(r.shape[0])])
            seg_eq = np.array(seg_eq)
            w = causal_weights(seg_eq.real.sum(axis=1), causal["eps"]) if omega is None else np.asarray(omega)
            per_eq = [np.sum(w * seg_eq[:, e]) / M for e in range(r.shape[0])]
        out["pde_eq"] = per_eq
        out["pde"] = sum(per_eq)
    for key, x, g, mask in (("ic", batch.x_ic, batch.g_ic, batch.ic_mask),
                            ("bc", batch.x_bc, batch.g_bc, batch.bc_mask)):
        n = x.shape[1]
        if n == 0 or mask == 0:
            continue
        (u, _, _), _ = forward(Ws, bs, _coords(x), Bd, 0, model.act, model.periods)
        term = 0.0
        for c in range(model.d_out):
            if mask >> c & 1:
                e = u[:, c] - np.asarray(g[c], dtype=np.float64)
                term = term + np.mean(e * e)
        out[key] = term
    out["total"] = lam_pde * out["pde"] + lam_ic * out["ic"] + lam_bc * out["bc"]
    return out


def causal_segments(batch, causal):
    """Time segment of every interior point (Sec. 2.6.8): the time domain [t0, t1] is cut
    into M equal segments [t0 + i D, t0 + (i + 1) D), D = (t1 - t0) / M, the last one
    closed at t1; a point at time t falls in floor((t - t0) * M / (t1 - t0)), clamped to
    0..M-1 (points outside [t0, t1] join the end segments).

    The index is an integer decided by floating point, so it is decided in the
    precision the GPU path uses for it: the FP32 time, FP32 t0, the FP32-rounded factor
    M / (t1 - t0), and FP32 rounding after the subtraction and after the product."""
    t = np.asarray(batch.x_res[causal["t_index"]], dtype=np.float32)
    M = causal["segments"]
    t0 = np.float32(causal["t0"])
    tinv = np.float32(M / (float(causal["t1"]) - float(causal["t0"])))
    seg = np.floor((t - t0) * tinv).astype(np.int64)
    return np.clip(seg, 0, M - 1)


def causal_weights(seg_losses, eps):
    """Eq. 20: omega_1 = 1, omega_i = exp(-eps sum_{k<i} L^k)."""
    w = np.ones(len(seg_losses))
    for i in range(1, len(seg_losses)):
        w[i] = np.exp(-eps * np.sum(seg_losses[:i]))
    return w


def ff_matrix_grad_terms(X, B, abar, a1bar, a2bar):
    """dL/dB [d, m] of the Fourier embedding (Eq. 14) from the adjoint of its jets.
    With phi_j = sum_e x_e B_ej, c = cos phi_j, s = sin phi_j, the jets are
      value [c, s];  d/dx_k [-s B_kj, c B_kj];  d2/dx_k dx_l [-c B_kj B_lj, -s B_kj B_lj],
    and their derivatives with respect to B_ej (dphi/dB_ej = x_e):
      value        [-s x_e, c x_e]
      d/dx_k       [-c x_e B_kj - s [k=e],  -s x_e B_kj + c [k=e]]
      d2/dx_k dx_l [s x_e B_kj B_lj - c ([k=e] B_lj + [l=e] B_kj),
                    -c x_e B_kj B_lj - s ([k=e] B_lj + [l=e] B_kj)]."""
    N, d = X.shape
    m = B.shape[1]
    phi = X @ B
    c, s = np.cos(phi), np.sin(phi)
    g = np.zeros((d, m))
    for e in range(d):
        xe = X[:, e:e + 1]
        g[e] += np.sum(abar[:, :m] * (-s * xe) + abar[:, m:] * (c * xe), axis=0)
        if a1bar is not None:
            for k in range(d):
                Bk = B[k][None, :]
                dc = -c * xe * Bk - (s if k == e else 0.0)
                ds = -s * xe * Bk + (c if k == e else 0.0)
                g[e] += np.sum(a1bar[k][:, :m] * dc + a1bar[k][:, m:] * ds, axis=0)
        if a2bar is not None:
            for k in range(d):
                for l in range(d):
                    Bk, Bl = B[k][None, :], B[l][None, :]
                    cross = (Bl if k == e else 0.0) + (Bk if l == e else 0.0)
                    dc = s * xe * Bk * Bl - c * cross
                    ds = -c * xe * Bk * Bl - s * cross
                    g[e] += np.sum(a2bar[k, l][:, :m] * dc + a2bar[k, l][:, m:] * ds, axis=0)
    return g


def period_grad_terms(X, P, abar, a1bar, a2bar):
    """dL/dP [d] of the periodic map (Eq. 16) from the adjoint of its jets.  With
    theta_k = 2 pi / P_k (dtheta_k/dP_k = -theta_k / P_k), c = cos(theta_k x_k),
    s = sin(theta_k x_k), the derivatives with respect to theta_k are
      value [-s x_k, c x_k];  d/dx_k [-c x_k theta_k - s, -s x_k theta_k + c];
      d2/dx_k^2 [s x_k theta_k^2 - 2 c theta_k, -c x_k theta_k^2 - 2 s theta_k]."""
    N, d = X.shape
    g = np.zeros(d)
    for k in range(d):
        th = 2.0 * np.pi / P[k]
        x = X[:, k]
        c, s = np.cos(th * x), np.sin(th * x)
        gt = np.sum(abar[:, 2 * k] * (-s * x) + abar[:, 2 * k + 1] * (c * x))
        if a1bar is not None:
            gt += np.sum(a1bar[k][:, 2 * k] * (-c * x * th - s) + a1bar[k][:, 2 * k + 1] * (-s * x * th + c))
        if a2bar is not None:
            gt += np.sum(a2bar[k, k][:, 2 * k] * (s * x * th ** 2 - 2 * c * th)
                         + a2bar[k, k][:, 2 * k + 1] * (-c * x * th ** 2 - 2 * s * th))
        g[k] = gt * (-th / P[k])
    return g


def _input_grad(model, Bd, X, adj, terms):
    """Adds one point set's dL/dB (Fourier features) or dL/dP (periodic map) to terms."""
    if model.periods is not None:
        g = period_grad_terms(X, np.asarray(model.periods, dtype=np.float64), *adj)
        terms["grad_periods"] = terms.get("grad_periods", 0.0) + g
    elif Bd is not None:
        g = ff_matrix_grad_terms(X, Bd, *adj)
        terms["grad_B"] = terms.get("grad_B", 0.0) + g


def loss_and_grad(model, theta, B, batch, nu, lambdas=(1.0, 1.0, 1.0), causal=None, input_grad=False):
    """Loss terms and dL/dtheta (packed like theta), float64.

    With `causal` = dict(segments=M, eps=eps, t_index=j, t0=t0, t1=t1) the PDE term is
    the causally weighted one of Sec. 2.6.8 (Eq. 21): L_pde = (1/M) sum_i omega_i L^i,
    L^i the mean squared residual over segment i's points and omega_i from Eq. 20.  The
    weights are evaluated at the current parameters and held constant in the gradient
    (the paper does not say; this is the usual stop-gradient reading of causal
    weighting).  terms["causal_weights"] holds the omega_i.

    With `input_grad`, terms["grad_B"] ([d, m], Fourier features) or
    terms["grad_periods"] ([d], periodic map) holds the gradient with respect to the
    input map's matrix or periods."""
    theta = np.asarray(theta, dtype=np.float64)
    Bd = None if B is None else np.asarray(B, dtype=np.float64)
    layers, Ws, bs = _weights(model, theta)
    lam_pde, lam_ic, lam_bc = lambdas
    order = PDE_ORDER[model.pde]
    L1 = len(Ws)
    dW = [np.zeros_like(W) for W in Ws]
    db = [np.zeros_like(b) for b in bs]
    terms = {"pde_eq": [0.0] * PDE_N_EQ[model.pde], "pde": 0.0, "ic": 0.0, "bc": 0.0}

    if batch.n_res:
        N = batch.n_res
        (u, u1, u2), cache = forward(Ws, bs, _coords(batch.x_res), Bd, order, model.act, model.periods)
        r = residuals(model.pde, u, u1, u2, nu)
        if causal is None:
            per_eq = [float(np.mean(r[e] * r[e])) for e in range(r.shape[0])]
            coef = lam_pde / N
        else:
            M = causal["segments"]
            seg = causal_segments(batch, causal)
            cnt = np.array([np.sum(seg == i) for i in range(M)], dtype=np.float64)
            seg_eq = np.zeros((M, r.shape[0]))
            for i in range(M):
                if cnt[i]:
                    seg_eq[i] = [np.mean(r[e][seg == i] ** 2) for e in range(r.shape[0])]
            omega = causal_weights(seg_eq.sum(axis=1), causal["eps"])
            per_eq = [float(np.sum(omega * seg_eq[:, e]) / M) for e in range(r.shape[0])]
            terms["causal_weights"] = omega
            safe = np.where(cnt > 0, cnt, 1.0)
            coef = lam_pde * (omega / (M * safe))[seg]      # per-point seed scale
        terms["pde_eq"], terms["pde"] = per_eq, sum(per_eq)
        ub, u1b, u2b = residual_seeds(model.pde, u, u1, u2, nu, coef)
        if input_grad:
            gW, gb, adj = backward(Ws, cache, ub, u1b, u2b, order, model.act, input_adjoint=True)
            _input_grad(model, Bd, _coords(batch.x_res), adj, terms)
        else:
            gW, gb = backward(Ws, cache, ub, u1b, u2b, order, model.act)
        for l in range(L1):
            dW[l] += gW[l]
            db[l] += gb[l]

    for key, x, g, mask, lam in (("ic", batch.x_ic, batch.g_ic, batch.ic_mask, lam_ic),
                                 ("bc", batch.x_bc, batch.g_bc, batch.bc_mask, lam_bc)):
        n = x.shape[1]
        if n == 0 or mask == 0:
            continue
        (u, _, _), cache = forward(Ws, bs, _coords(x), Bd, 0, model.act, model.periods)
        ub = np.zeros_like(u)
        term = 0.0
        for c in range(model.d_out):
            if mask >> c & 1:
                e = u[:, c] - np.asarray(g[c], dtype=np.float64)
                term += float(np.mean(e * e))
                ub[:, c] = 2.0 * lam * e / n
        terms[key] = term
        if input_grad:
            gW, gb, adj = backward(Ws, cache, ub, None, None, 0, model.act, input_adjoint=True)
            _input_grad(model, Bd, _coords(x), adj, terms)
        else:
            gW, gb = backward(Ws, cache, ub, None, None, 0, model.act)
        for l in range(L1):
            dW[l] += gW[l]
            db[l] += gb[l]

    terms["total"] = lam_pde * terms["pde"] + lam_ic * terms["ic"] + lam_bc * terms["bc"]

    # RWF chain rule (Eq. 15): W = exp(s) V  =>  dV = exp(s) dW, ds_i = sum_j dW_ij W_ij.
    grad = []
    for l, (V, s, _) in enumerate(layers):
        if s is None:
            grad.append(dW[l].ravel())
        else:
            grad.append((np.exp(s)[:, None] * dW[l]).ravel())
            grad.append(np.sum(dW[l] * Ws[l], axis=1))
        grad.append(db[l])
    return terms, np.concatenate(grad)


def output_jets(model, theta, B, X, order):
    """Network outputs and their input derivatives at points X [N, d] (for pins)."""
    theta = np.asarray(theta)
    if not np.iscomplexobj(theta):
        theta = theta.astype(np.float64)
    Bd = None if B is None else np.asarray(B, dtype=np.float64)
    _, Ws, bs = _weights(model, theta)
    (u, u1, u2), _ = forward(Ws, bs, X, Bd, order, model.act, model.periods)
    return u, u1, u2


# --------------------------------------------------------------------------------------
# Adam (Sec. 2.6.5)
# --------------------------------------------------------------------------------------

def adam_step(theta, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step is 1-based).  Returns new (theta, m, v), float64."""
    theta = np.asarray(theta, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    theta = theta - lr * mhat / (np.sqrt(vhat) + eps)
    return theta, m, v


# --------------------------------------------------------------------------------------
# Loss balancing (Sec. 2.6.4, Eqs. 17-19)
# --------------------------------------------------------------------------------------

def term_gradients(model, theta, B, batch, nu):
    """Unweighted gradients of L_pde, L_ic and L_bc (Eq. 17's terms), stacked [3][P]:
    the plain loss gradient with unit weight on one term and zero on the others."""
    return np.stack([loss_and_grad(model, theta, B, batch, nu, lam)[1]
                     for lam in ((1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0))])


def loss_balance(grads, lambdas, alpha=0.9, eps=1e-9, update=True):
    """Eq. 18: lambda_hat_i = (|g_pde| + |g_ic| + |g_bc|) / |g_i| (the eps guards the
    division, as the paper's code does); Eq. 19: lambda = alpha lambda + (1 - alpha)
    lambda_hat.  A term whose gradient is zero (no points) keeps its weight.
    Returns (new lambdas, norms), float64, order (pde, ic, bc)."""
    g = np.asarray(grads, dtype=np.float64)
    norms = np.array([np.sqrt(np.sum(g[i] * g[i])) for i in range(3)])
    total = norms.sum()
    lam = np.array(lambdas, dtype=np.float64).copy()
    if update:
        for i in range(3):
            if norms[i] > 0.0:
                lam[i] = alpha * lam[i] + (1.0 - alpha) * total / (norms[i] + eps)
    return lam, norms


# --------------------------------------------------------------------------------------
# L-BFGS (Sec. 2.6.5, Eqs. 22-26)
# --------------------------------------------------------------------------------------

def lbfgs_direction(g, S, Y):
    """p = -H g with H the L-BFGS inverse-Hessian approximation built from the pairs
    (s_i, y_i), oldest first (Eqs. 22-24; the two-loop recursion of Nocedal and
    Wright, Algorithm 7.4).  The initial matrix is gamma I, gamma = s.y / y.y of the
    newest pair (I without pairs)."""
    q = np.array(g, dtype=np.float64)
    m = len(S)
    rho = [1.0 / float(np.dot(Y[i], S[i])) for i in range(m)]
    alpha = [0.0] * m
    for i in range(m - 1, -1, -1):
        alpha[i] = rho[i] * float(np.dot(S[i], q))
        q = q - alpha[i] * Y[i]
    gamma = float(np.dot(S[-1], Y[-1]) / np.dot(Y[-1], Y[-1])) if m else 1.0
    r = gamma * q
    for i in range(m):
        beta = rho[i] * float(np.dot(Y[i], r))
        r = r + (alpha[i] - beta) * S[i]
    return -r


def lbfgs_minimize(f_and_g, x0, history=10, steps=20, c1=1e-4, max_backtracks=30):
    """L-BFGS with a backtracking line search (Eq. 26) that accepts the first step
    length lambda in 1, 1/2, 1/4, ... meeting the sufficient-decrease condition
    f(x + lambda p) <= f(x) + c1 lambda g.p; pairs with s.y <= 0 are not stored.
    Returns the iterates' losses and the final x."""
    x = np.array(x0, dtype=np.float64)
    fx, g = f_and_g(x)
    S, Y, losses = [], [], [fx]
    for _ in range(steps):
        p = lbfgs_direction(g, S, Y)
        gp = float(np.dot(g, p))
        if gp >= 0.0:                       # not a descent direction: restart from -g
            S, Y = [], []
            p, gp = -g, -float(np.dot(g, g))
        lam = 1.0
        for _ in range(max_backtracks):
            fn, gn = f_and_g(x + lam * p)
            if fn <= fx + c1 * lam * gp:
                break
            lam *= 0.5
        s, y = lam * p, gn - g
        if float(np.dot(s, y)) > 0.0:
            S.append(s); Y.append(y)
            if len(S) > history:
                S.pop(0); Y.pop(0)
        x, fx, g = x + lam * p, fn, gn
        losses.append(fx)
    return losses, x
