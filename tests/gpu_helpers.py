"""Shared helpers of the GPU tests: run the CUDA path and the oracle on the same
seeded inputs and compare them."""
import numpy as np
import torch

import oracle
from paper_2604_15645_gb300 import api

from parity_blocks import check_blocks, report

TOL = {"fp32": 1e-5, "tf32": 1e-3, "bf16": 2e-2}


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def run_gpu(spec, params, B, batch, problem, precision, want_grad=True, value_split=False):
    net = api.PinnNet.from_spec(spec, precision, value_split=value_split)
    if B is not None:
        net.set_ff_matrix(B)
    db = api.DeviceBatch.from_host(batch)
    p = torch.as_tensor(params, dtype=torch.float32, device="cuda")
    prob = api.make_problem(problem.nu, problem.lambda_pde, problem.lambda_ic, problem.lambda_bc)
    if want_grad:
        terms, grad = net.loss_grad(p, db, prob)
        torch.cuda.synchronize()
        assert net.status_poll() == 0
        return terms.cpu().numpy().copy(), grad.cpu().numpy().astype(np.float64)
    terms = net.loss(p, db, prob)
    torch.cuda.synchronize()
    return terms.cpu().numpy().copy(), None


def run_oracle(spec, params, B, batch, problem, chunk=None):
    """Oracle loss terms (as the 8-vector layout of the library) and gradient.
    With `chunk`, interior points are split into chunks whose sums are combined
    (every loss term is a sum over points divided by its count)."""
    m = oracle.Model.from_spec(spec)
    lam = (problem.lambda_pde, problem.lambda_ic, problem.lambda_bc)
    n = batch.n_res
    if chunk is None or n <= chunk:
        t, g = oracle.loss_and_grad(m, params, B, batch, problem.nu, lam)
        return _pack(t), g
    from synth import Batch
    g_tot = 0.0
    pde_eq = np.zeros(3)
    first = True
    bd = None
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        sub = Batch(batch.x_res[:, s:e], batch.x_ic if first else batch.x_ic[:, :0],
                    batch.g_ic if first else batch.g_ic[:, :0], batch.ic_mask,
                    batch.x_bc if first else batch.x_bc[:, :0], batch.g_bc if first else batch.g_bc[:, :0],
                    batch.bc_mask)
        frac = (e - s) / n
        t, g = oracle.loss_and_grad(m, params, B, sub, problem.nu, (lam[0] * frac, lam[1], lam[2]))
        g_tot = g_tot + g
        pde_eq[:len(t["pde_eq"])] += frac * np.array(t["pde_eq"])
        if first:
            bd = (t["ic"], t["bc"])
        first = False
    out = np.zeros(8)
    out[2:5] = pde_eq
    out[1] = pde_eq.sum()
    out[5], out[6] = bd
    out[0] = lam[0] * out[1] + lam[1] * out[5] + lam[2] * out[6]
    return out, g_tot


def _pack(t):
    out = np.zeros(8)
    out[0], out[1] = t["total"], t["pde"]
    out[2:2 + len(t["pde_eq"])] = t["pde_eq"]
    out[5], out[6] = t["ic"], t["bc"]
    return out


def assert_parity(gpu_terms, gpu_grad, ref_terms, ref_grad, tol, what="", spec=None, block_tol=None):
    """Loss terms element by element; the gradient as a whole (relative L2) and, given
    the network's spec, block by block (every layer's V, s and b; see parity_blocks) at
    `block_tol` (default: tol).  The per-block errors and norms are printed (shown with
    pytest -s or -rP)."""
    for i in (0, 1, 2, 3, 4, 5, 6):
        if abs(ref_terms[i]) > 0:
            e = abs(gpu_terms[i] - ref_terms[i]) / abs(ref_terms[i])
            assert e <= tol, f"{what} loss term {i}: rel err {e:.3e} > {tol} ({gpu_terms[i]} vs {ref_terms[i]})"
        else:
            assert abs(gpu_terms[i]) <= 1e-30, f"{what} term {i} should be 0, got {gpu_terms[i]}"
    if gpu_grad is not None:
        e = rel(gpu_grad, ref_grad)
        assert e <= tol, f"{what} gradient rel L2 err {e:.3e} > {tol}"
        if spec is not None:
            rows = check_blocks(gpu_grad, ref_grad, spec, tol if block_tol is None else block_tol, what)
            print(f"{what}: gradient rel L2 {e:.3e}; per block:\n{report(rows)}")


def torch_loss_grad(spec, params, B, batch, problem, dtype, chunk=65536, want_grad=True):
    """The paper's own method at any size: torch double-backward autograd (Sec. 2.3),
    in `dtype`, over chunks of the interior points.  Every loss term is a sum over its
    points divided by its count, so chunk losses weighted by their share of the interior
    points (initial and boundary sets in the first chunk) add up to the whole loss, and
    so do their gradients.  Returns (loss total, gradient as float64 numpy or None)."""
    from baseline import torch_autograd as ta
    from synth import Batch
    model = ta.TorchPINN(spec, params, B, "cuda", dtype)
    lam = (problem.lambda_pde, problem.lambda_ic, problem.lambda_bc)
    n = batch.n_res
    total = 0.0
    for s in range(0, max(n, 1), chunk):
        e = min(n, s + chunk)
        first = s == 0
        sub = Batch(batch.x_res[:, s:e], batch.x_ic if first else batch.x_ic[:, :0],
                    batch.g_ic if first else batch.g_ic[:, :0], batch.ic_mask,
                    batch.x_bc if first else batch.x_bc[:, :0], batch.g_bc if first else batch.g_bc[:, :0],
                    batch.bc_mask)
        frac = (e - s) / n if n else 1.0
        t, _ = ta.loss(model, ta.batch_to_torch(sub, "cuda", dtype), problem.nu, (lam[0] * frac, lam[1], lam[2]))
        if want_grad:
            t.backward()
        total += float(t.detach())
        del t
    g = model.flat_grad().detach().double().cpu().numpy() if want_grad else None
    del model
    torch.cuda.empty_cache()
    return total, g


def layer_coordinates(spec, per_layer_v, seed, layers=None):
    """Seeded parameter indices: per weight layer `per_layer_v` entries of V, one of s
    (with RWF) and one of b (Eqs. 4 and 15 blocks), for the layers listed (default all)."""
    from parity_blocks import param_blocks
    rng = np.random.default_rng(seed)
    blocks = {n: (a, b) for n, a, b in param_blocks(spec)}
    n_layers = len(spec.widths) + 1
    out = []
    for l in (layers or range(1, n_layers + 1)):
        a, b = blocks[f"V{l}"]
        out.extend(rng.choice(np.arange(a, b), size=per_layer_v, replace=False).tolist())
        for name in (f"s{l}", f"b{l}"):
            if name in blocks:
                a, b = blocks[name]
                out.append(int(rng.integers(a, b)))
    return np.array(sorted(out))
