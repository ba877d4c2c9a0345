"""Input-map gradients on the GPU against the FP64 oracle: dL/dB of the Fourier
embedding (Eq. 14) and dL/dP of the strict periodic map (Sec. 2.6.3, Eq. 16), which
the library realises as the embedding with B = diag(2 pi / P)."""
import numpy as np
import pytest
import torch

import oracle
from synth import NetSpec, Problem, init_params, ff_matrix, make_batch, make_workload
from synth.workloads import PDE_ADVECTION, PDE_ALLEN_CAHN, PDE_MAXWELL, PDE_NS

from gpu_helpers import TOL, assert_parity, rel, _pack

pytestmark = pytest.mark.gpu


def _gpu(spec, params, batch, problem, precision, B=None, periods=None, chunk=0):
    from paper_2604_15645_gb300 import api
    net = api.PinnNet.from_spec(spec, precision, chunk_points=chunk)
    if periods is not None:
        net.set_periodic(periods)
    else:
        net.set_ff_matrix(B)
    db = api.DeviceBatch.from_host(batch)
    p = torch.as_tensor(params, dtype=torch.float32, device="cuda")
    prob = api.make_problem(problem.nu, problem.lambda_pde, problem.lambda_ic, problem.lambda_bc)
    t, g, gff = net.loss_grad_ff(p, db, prob)
    torch.cuda.synchronize()
    assert net.status_poll() == 0
    return t.cpu().numpy().copy(), g.cpu().numpy().astype(np.float64), gff.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16"])
@pytest.mark.parametrize("name", ["ns_cavity_6x256", "maxwell_te_5x512"])
def test_fourier_matrix_gradient(cuda_lib, name, precision):
    w, p, B, b = make_workload(name, n_res=700, n_ic=120, n_bc=150, random_bias=0.1)
    w.spec.widths = [64, 64, 64]
    w.spec.ff_m = 16
    p = init_params(w.spec, 21, 0.1)
    B = ff_matrix(w.spec, 22)
    gt, gg, gB = _gpu(w.spec, p, b, w.problem, precision, B=B)
    m = oracle.Model.from_spec(w.spec)
    lam = (w.problem.lambda_pde, w.problem.lambda_ic, w.problem.lambda_bc)
    rt, rg = oracle.loss_and_grad(m, p, B, b, w.problem.nu, lam, input_grad=True)
    assert_parity(gt, gg, _pack(rt), rg, TOL[precision], f"{name} {precision}", spec=w.spec)
    e = rel(gB.reshape(B.shape), rt["grad_B"])
    assert e <= TOL[precision], f"dL/dB rel err {e:.3e}"


def ff_column_order(d):
    return [2 * q for q in range(d)] + [2 * q + 1 for q in range(d)]


def _permute_first_layer(theta, fin, fout, order):
    out = np.array(theta, dtype=np.float64).copy()
    V = out[:fin * fout].reshape(fout, fin)
    out[:fin * fout] = V[:, order].ravel()
    return out


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("pde,widths,P,nu", [(PDE_ADVECTION, [64, 64, 64], [2 * np.pi, 1.0], 10.0),
                                             (PDE_ALLEN_CAHN, [48, 48], [2.0, 1.0], 1e-4),
                                             (PDE_MAXWELL, [64, 64], [2.0, 2.0, 1.5], 0.0)])
def test_periodic_map_and_period_gradient(cuda_lib, pde, widths, P, nu, precision):
    d_in = 3 if pde == PDE_MAXWELL else 2
    d_out = 3 if pde == PDE_MAXWELL else 1
    spec = NetSpec(pde, d_in, d_out, widths, ff_m=d_in, rwf=True)
    p_paper = init_params(spec, 31, 0.1)          # first layer in the paper's column order
    b = make_batch(pde, 1500, 200, 0 if pde != PDE_MAXWELL else 100, 32, 33)
    problem = Problem(nu)
    m = oracle.Model(pde, d_in, d_out, widths, 0, True, None, np.array(P, dtype=np.float64))
    rt, rg = oracle.loss_and_grad(m, p_paper, None, b, nu, input_grad=True)
    fin, fout = 2 * d_in, widths[0]
    order = ff_column_order(d_in)
    p_lib = _permute_first_layer(p_paper, fin, fout, order)
    gt, gg, gP = _gpu(spec, p_lib, b, problem, precision, periods=P)
    inv = np.argsort(order)
    assert_parity(gt, _permute_first_layer(gg, fin, fout, inv), _pack(rt), rg, TOL[precision],
                  f"periodic pde {pde} {precision}", spec=spec)
    e = rel(gP, rt["grad_periods"])
    assert e <= TOL[precision], f"dL/dP rel err {e:.3e}: {gP} vs {rt['grad_periods']}"


def test_input_map_gradient_chunked_matches_one_pass(cuda_lib):
    w, p, B, b = make_workload("ns_cavity_6x256", n_res=3000, n_bc=700, random_bias=0.1)
    w.spec.widths = [64, 64]
    w.spec.ff_m = 8
    p = init_params(w.spec, 41, 0.1)
    B = ff_matrix(w.spec, 42)
    t1, g1, f1 = _gpu(w.spec, p, b, w.problem, "fp32", B=B)
    t2, g2, f2 = _gpu(w.spec, p, b, w.problem, "fp32", B=B, chunk=1024)
    assert rel(f2, f1) < 1e-5 and rel(g2, g1) < 1e-5


def test_input_map_errors(cuda_lib):
    from paper_2604_15645_gb300 import _lib, api
    w, p, B, b = make_workload("burgers1d_4x64", n_res=64)
    net = api.PinnNet.from_spec(w.spec, "fp32")           # no Fourier features
    db = api.DeviceBatch.from_host(b)
    with pytest.raises(_lib.PinnError):
        net.loss_grad_ff(torch.tensor(p, device="cuda"), db, api.make_problem(w.problem.nu),
                         grad_ff=torch.zeros(4, device="cuda"))
    with pytest.raises(_lib.PinnError):
        net.set_periodic([1.0, 1.0])                      # ff_m != d_in
    spec = NetSpec(PDE_ADVECTION, 2, 1, [16], ff_m=2)
    net2 = api.PinnNet.from_spec(spec, "fp32")
    with pytest.raises(_lib.PinnError):
        net2.set_periodic([1.0, -2.0])
    net2.set_periodic([2 * np.pi, 1.0])
