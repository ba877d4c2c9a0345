"""The paper's own way of computing the PINN loss gradient: plain PyTorch autograd.

Derivatives of the network outputs with respect to the inputs come from
``torch.autograd.grad(..., create_graph=True)`` (Sec. 2.3, the "autoGrad" terms),
second derivatives from a second such call, then ``loss.backward()`` differentiates
through that derivative graph (double backward).  The model uses RFF (Eq. 14) and
RWF (Eq. 15) the same way as the paper's model blocks, with W = exp(s) * V.

Used twice: in float64 it is an independent check of the oracle (a different
differentiation method), and in float32 on the GPU it is the speed baseline the
CUDA path is compared with.  It never calls the CUDA library.
"""
from __future__ import annotations

import torch


class TorchPINN:
    def __init__(self, spec, params, B, device="cpu", dtype=torch.float64):
        self.spec = spec
        self.device, self.dtype = device, dtype
        first_in = 2 * spec.ff_m if spec.ff_m else spec.d_in
        dims, prev = [], first_in
        for w in spec.widths:
            dims.append((prev, w)); prev = w
        dims.append((prev, spec.d_out))
        self.dims = dims
        p = torch.as_tensor(params, dtype=dtype, device=device)
        self.tensors, off = [], 0
        for fi, fo in dims:
            V = p[off:off + fo * fi].reshape(fo, fi).clone().requires_grad_(True); off += fo * fi
            s = None
            if spec.rwf:
                s = p[off:off + fo].clone().requires_grad_(True); off += fo
            b = p[off:off + fo].clone().requires_grad_(True); off += fo
            self.tensors.append((V, s, b))
        self.B = None if B is None else torch.as_tensor(B, dtype=dtype, device=device)

    def parameters(self):
        out = []
        for V, s, b in self.tensors:
            out.append(V)
            if s is not None:
                out.append(s)
            out.append(b)
        return out

    def __call__(self, X):
        h = X
        if self.B is not None:
            xm = X @ self.B
            h = torch.cat([torch.cos(xm), torch.sin(xm)], dim=-1)
        n = len(self.tensors)
        for i, (V, s, b) in enumerate(self.tensors):
            W = V if s is None else torch.exp(s)[:, None] * V
            h = h @ W.T + b
            if i < n - 1:
                if getattr(self.spec, "activation", "tanh") == "sine":
                    h = torch.sin(self.spec.omega0 * h)
                else:
                    h = torch.tanh(h)
        return h

    def flat_grad(self):
        return torch.cat([t.grad.reshape(-1) for t in self.parameters()])

    def zero_grad(self):
        for t in self.parameters():
            t.grad = None


def _d(y, x):
    return torch.autograd.grad(y.sum(), x, create_graph=True)[0]


def loss(model, batch_t, nu, lambdas=(1.0, 1.0, 1.0)):
    """Composite MSE loss (Eqs. 10-13, 17) through autograd input derivatives.

    batch_t: dict of tensors x_res [d, N], x_ic, g_ic, x_bc, g_bc and int masks.
    Returns (total, dict of terms as tensors)."""
    spec = model.spec
    lam_pde, lam_ic, lam_bc = lambdas
    terms = {}
    total = 0.0
    if batch_t["x_res"].shape[1]:
        X = batch_t["x_res"].T.contiguous().requires_grad_(True)
        U = model(X)
        if spec.pde == 0:
            u = U[:, 0]
            gu = _d(u, X)
            u_x, u_t = gu[:, 0], gu[:, 1]
            u_xx = _d(u_x, X)[:, 0]
            rs = [u_t + u * u_x - nu * u_xx]
        elif spec.pde == 1:
            u, v = U[:, 0], U[:, 1]
            gu, gv, gp = _d(U[:, 0], X), _d(U[:, 1], X), _d(U[:, 2], X)
            u_x, u_y, v_x, v_y = gu[:, 0], gu[:, 1], gv[:, 0], gv[:, 1]
            u_xx, u_yy = _d(u_x, X)[:, 0], _d(u_y, X)[:, 1]
            v_xx, v_yy = _d(v_x, X)[:, 0], _d(v_y, X)[:, 1]
            rs = [u * u_x + v * u_y + gp[:, 0] - nu * (u_xx + u_yy),
                  u * v_x + v * v_y + gp[:, 1] - nu * (v_xx + v_yy),
                  u_x + v_y]
        elif spec.pde == 2:
            ge, gx, gy = _d(U[:, 0], X), _d(U[:, 1], X), _d(U[:, 2], X)
            rs = [ge[:, 2] - (gy[:, 0] - gx[:, 1]), gx[:, 2] + ge[:, 1], gy[:, 2] - ge[:, 0]]
        elif spec.pde == 3:      # advection u_t + c u_x, c = nu (Sec. 4.1)
            gu = _d(U[:, 0], X)
            rs = [gu[:, 1] + nu * gu[:, 0]]
        else:                    # Allen-Cahn u_t - eps u_xx + 5u^3 - 5u, eps = nu (Sec. 4.2)
            u = U[:, 0]
            gu = _d(u, X)
            u_xx = _d(gu[:, 0], X)[:, 0]
            rs = [gu[:, 1] - nu * u_xx + 5.0 * u ** 3 - 5.0 * u]
        per_eq = [torch.mean(r * r) for r in rs]
        terms["pde_eq"] = per_eq
        terms["pde"] = sum(per_eq)
        total = total + lam_pde * terms["pde"]
    for key, lam in (("ic", lam_ic), ("bc", lam_bc)):
        x, g, mask = batch_t["x_" + key], batch_t["g_" + key], batch_t[key + "_mask"]
        if x.shape[1] == 0 or mask == 0:
            continue
        U = model(x.T.contiguous())
        term = 0.0
        for c in range(spec.d_out):
            if mask >> c & 1:
                e = U[:, c] - g[c]
                term = term + torch.mean(e * e)
        terms[key] = term
        total = total + lam * term
    terms["total"] = total
    return total, terms


def batch_to_torch(batch, device, dtype):
    t = lambda a: torch.as_tensor(a, device=device, dtype=dtype)
    return {"x_res": t(batch.x_res), "x_ic": t(batch.x_ic), "g_ic": t(batch.g_ic), "ic_mask": batch.ic_mask,
            "x_bc": t(batch.x_bc), "g_bc": t(batch.g_bc), "bc_mask": batch.bc_mask}


def loss_and_grad(spec, params, B, batch, nu, device="cpu", dtype=torch.float64, lambdas=(1.0, 1.0, 1.0)):
    model = TorchPINN(spec, params, B, device, dtype)
    total, terms = loss(model, batch_to_torch(batch, device, dtype), nu, lambdas)
    total.backward()
    return total.detach(), model.flat_grad().detach(), terms
