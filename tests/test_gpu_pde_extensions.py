"""More residuals and temporal causality (the survey's next rows): advection
(Sec. 4.1) and Allen-Cahn (Sec. 4.2) against the FP64 oracle, and the causally
weighted PDE term (Sec. 2.6.8, Eqs. 20-21) with its segment weights."""
import numpy as np
import pytest
import torch

import oracle
from synth import make_workload

from gpu_helpers import TOL, assert_parity, rel, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["advection1d_4x128", "allen_cahn1d_4x128"])
@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16"])
def test_new_residuals_match_oracle(cuda_lib, name, precision):
    w, p, B, b = make_workload(name, n_res=1000, n_ic=120, n_bc=90, random_bias=0.1)
    gt, gg = run_gpu(w.spec, p, B, b, w.problem, precision)
    rt, rg = run_oracle(w.spec, p, B, b, w.problem)
    assert_parity(gt, gg, rt, rg, TOL[precision], f"{name} {precision}", spec=w.spec)


def _causal_case(name, precision, M, eps, **sizes):
    from paper_2604_15645_gb300 import api
    w, p, B, b = make_workload(name, random_bias=0.1, **sizes)
    ti = 2 if w.spec.pde == 2 else 1
    cz = dict(segments=M, eps=eps, t_index=ti, t0=0.0, t1=1.0)
    net = api.PinnNet.from_spec(w.spec, precision)
    if B is not None:
        net.set_ff_matrix(B)
    net.set_causal(M, eps, 0.0, 1.0)
    db = api.DeviceBatch.from_host(b)
    lam = (1.0, 0.5, 2.0)
    prob = api.make_problem(w.problem.nu, *lam)
    return api, w, p, B, b, cz, net, db, prob, lam


@pytest.mark.parametrize("name,precision", [("burgers1d_4x64", "fp32"), ("maxwell_te_5x512", "fp32"),
                                            ("maxwell_te_5x512", "bf16"), ("advection1d_4x128", "tf32"),
                                            ("advection1d_4x128", "bf16")])
def test_causal_loss_and_gradient_match_oracle(cuda_lib, name, precision):
    api, w, p, B, b, cz, net, db, prob, lam = _causal_case(name, precision, 4, 0.5, n_res=900, n_ic=100, n_bc=100)
    t, g = net.loss_grad(torch.tensor(p, device="cuda"), db, prob)
    torch.cuda.synchronize()
    assert net.status_poll() == 0
    terms, rg = oracle.loss_and_grad(oracle.Model.from_spec(w.spec), p, B, b, w.problem.nu, lam, causal=cz)
    t = t.cpu().numpy()
    tol = TOL[precision]
    assert abs(t[0] - terms["total"]) <= tol * abs(terms["total"])
    assert abs(t[1] - terms["pde"]) <= tol * abs(terms["pde"])
    assert rel(g.cpu().numpy().astype(np.float64), rg) <= tol
    om = net.causal_weights().cpu().numpy()
    assert om[0] == 1.0
    assert np.allclose(om, terms["causal_weights"], rtol=10 * tol)


def test_causal_loss_only_and_term_gradients(cuda_lib):
    api, w, p, B, b, cz, net, db, prob, lam = _causal_case("burgers1d_4x64", "fp32", 3, 2.0, n_res=900, n_ic=100,
                                                           n_bc=100)
    params = torch.tensor(p, device="cuda")
    tl = net.loss(params, db, prob).cpu().numpy().copy()
    m = oracle.Model.from_spec(w.spec)
    terms, _ = oracle.loss_and_grad(m, p, B, b, w.problem.nu, lam, causal=cz)
    assert abs(tl[0] - terms["total"]) <= 1e-5 * abs(terms["total"])
    _, G = net.loss_grad_terms(params, db, prob)
    G = G.cpu().numpy().astype(np.float64)
    for i, unit in enumerate(((1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0))):
        _, ref = oracle.loss_and_grad(m, p, B, b, w.problem.nu, unit, causal=cz)
        assert rel(G[i], ref) <= 1e-5, f"term {i}"


def test_causal_refusals(cuda_lib):
    from paper_2604_15645_gb300 import _lib, api
    w, p, B, b = make_workload("ns_cavity_6x256", n_res=256, n_bc=64)
    net = api.PinnNet.from_spec(w.spec, "fp32")
    with pytest.raises(_lib.PinnError):
        net.set_causal(4, 1.0)                    # steady problem: no time input
    w, p, B, b = make_workload("burgers1d_4x64", n_res=512, n_ic=64, n_bc=64)
    net = api.PinnNet.from_spec(w.spec, "fp32", chunk_points=256)
    net.set_causal(4, 1.0)
    with pytest.raises(_lib.PinnError):          # causality needs all points in one pass
        net.loss_grad(torch.tensor(p, device="cuda"), api.DeviceBatch.from_host(b), api.make_problem(w.problem.nu))
    with pytest.raises(_lib.PinnError):
        net.set_causal(33, 1.0)


def test_periodic_map_with_causality_maxwell(cuda_lib):
    """The paper's Maxwell configuration combines the strict periodic input map (Eq. 16)
    with temporal causality (Eqs. 20-21): both on the GPU against the oracle, which
    implements the map in the paper's column order."""
    from paper_2604_15645_gb300 import api
    from synth import NetSpec, Problem, init_params, make_batch
    from synth.workloads import PDE_MAXWELL
    P = np.array([2.0, 2.0, 1.5])
    widths = [64, 64]
    spec = NetSpec(PDE_MAXWELL, 3, 3, widths, ff_m=3, rwf=True)
    p_paper = init_params(spec, 91, 0.1)
    b = make_batch(PDE_MAXWELL, 1200, 150, 0, 92, 93)
    cz = dict(segments=4, eps=0.002, t_index=2, t0=0.0, t1=1.0)   # weights well inside (0, 1)
    lam = (1.0, 0.5, 1.0)
    m = oracle.Model(PDE_MAXWELL, 3, 3, widths, 0, True, None, P)
    rt, rg = oracle.loss_and_grad(m, p_paper, None, b, 0.0, lam, causal=cz)
    # the library's first layer takes the map's columns in Fourier-feature order
    order = [0, 2, 4, 1, 3, 5]
    fin, fout = 6, widths[0]
    p_lib = np.array(p_paper, dtype=np.float64).copy()
    p_lib[:fin * fout] = p_lib[:fin * fout].reshape(fout, fin)[:, order].ravel()
    net = api.PinnNet.from_spec(spec, "bf16")
    net.set_periodic(P)
    net.set_causal(4, 0.002, 0.0, 1.0)
    t, g = net.loss_grad(torch.tensor(p_lib, device="cuda", dtype=torch.float32), api.DeviceBatch.from_host(b),
                         api.make_problem(0.0, *lam))
    torch.cuda.synchronize()
    assert net.status_poll() == 0
    t = t.cpu().numpy()
    g = g.cpu().numpy().astype(np.float64)
    g_paper = g.copy()
    g_paper[:fin * fout] = g[:fin * fout].reshape(fout, fin)[:, np.argsort(order)].ravel()
    assert abs(t[0] - rt["total"]) <= TOL["bf16"] * abs(rt["total"])
    assert abs(t[1] - rt["pde"]) <= TOL["bf16"] * abs(rt["pde"])
    assert rel(g_paper, rg) <= TOL["bf16"]
    assert 0.01 < rt["causal_weights"][-1] < 0.99
    assert np.allclose(net.causal_weights().cpu().numpy(), rt["causal_weights"], rtol=TOL["bf16"])
