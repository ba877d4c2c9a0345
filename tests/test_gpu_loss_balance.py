"""Per-term gradients and the loss-balancing weights (Sec. 2.6.4): the library's
three reverse sweeps against the oracle's per-term gradients, their weighted sum
against the weighted loss gradient, and the device weight update against the
oracle's Eqs. 18-19."""
import numpy as np
import pytest
import torch

import oracle
from synth import make_workload

from gpu_helpers import TOL, rel

pytestmark = pytest.mark.gpu


def _setup(name, precision, chunk=0, **sizes):
    from paper_2604_15645_gb300 import api
    w, p, B, b = make_workload(name, random_bias=0.1, **sizes)
    net = api.PinnNet.from_spec(w.spec, precision, chunk_points=chunk)
    if B is not None:
        net.set_ff_matrix(B)
    db = api.DeviceBatch.from_host(b)
    prob = api.make_problem(w.problem.nu, 1.0, 1.0, 1.0)
    return api, w, p, B, b, net, db, prob


def _terms_gpu(net, p, db, prob):
    params = torch.tensor(p, device="cuda")
    terms, G = net.loss_grad_terms(params, db, prob)
    torch.cuda.synchronize()
    assert net.status_poll() == 0
    return terms.cpu().numpy().copy(), G.cpu().numpy().astype(np.float64), params


@pytest.mark.parametrize("name,precision,sizes", [
    ("ns_cavity_6x256", "fp32", dict(n_res=1000, n_bc=300)),
    ("maxwell_te_5x512", "fp32", dict(n_res=600, n_ic=100, n_bc=150)),
    ("ns_cavity_6x256", "bf16", dict(n_res=1000, n_bc=300)),
    ("maxwell_te_5x512", "tf32", dict(n_res=600, n_ic=100, n_bc=150)),
])
def test_term_gradients_match_oracle(cuda_lib, name, precision, sizes):
    api, w, p, B, b, net, db, prob = _setup(name, precision, **sizes)
    _, G, _ = _terms_gpu(net, p, db, prob)
    ref = oracle.term_gradients(oracle.Model.from_spec(w.spec), p, B, b, w.problem.nu)
    for i in range(3):
        if np.abs(ref[i]).max() == 0.0:          # a term without points (the cavity has no IC set)
            assert np.abs(G[i]).max() == 0.0
        else:
            assert rel(G[i], ref[i]) <= TOL[precision], f"term {i}: {rel(G[i], ref[i]):.3e}"


def test_weighted_sum_of_terms_is_the_loss_gradient(cuda_lib):
    api, w, p, B, b, net, db, prob = _setup("maxwell_te_5x512", "fp32", n_res=600, n_ic=100, n_bc=150)
    lam = (0.7, 1.9, 3.1)
    t3, G, params = _terms_gpu(net, p, db, api.make_problem(w.problem.nu, *lam))
    t1, g = net.loss_grad(params, db, api.make_problem(w.problem.nu, *lam))
    g = g.cpu().numpy().astype(np.float64)
    assert rel(lam[0] * G[0] + lam[1] * G[1] + lam[2] * G[2], g) < 1e-6
    assert rel(t3[:7], t1.cpu().numpy()[:7]) < 1e-12       # the same loss terms and weighted total


def test_chunked_term_gradients(cuda_lib):
    api, w, p, B, b, net, db, prob = _setup("maxwell_te_5x512", "fp32", n_res=600, n_ic=100, n_bc=150)
    _, G1, _ = _terms_gpu(net, p, db, prob)
    api2, w2, p2, B2, b2, net2, db2, prob2 = _setup("maxwell_te_5x512", "fp32", chunk=192, n_res=600, n_ic=100,
                                                    n_bc=150)
    _, G2, _ = _terms_gpu(net2, p2, db2, prob2)
    for i in range(3):
        assert rel(G2[i], G1[i]) < 1e-6


def test_loss_balance_update_matches_oracle(cuda_lib):
    api, w, p, B, b, net, db, prob = _setup("maxwell_te_5x512", "fp32", n_res=600, n_ic=100, n_bc=150)
    _, G, _ = _terms_gpu(net, p, db, prob)
    grads = torch.tensor(G, dtype=torch.float32, device="cuda")
    lam0 = [1.0, 2.0, 0.5]
    lam = torch.tensor(lam0, dtype=torch.float64, device="cuda")
    norms = torch.zeros(3, dtype=torch.float64, device="cuda")
    net.loss_balance(grads, lam, norms, alpha=0.9, eps=1e-9, update=True)
    ref_lam, ref_norms = oracle.loss_balance(grads.cpu().numpy().astype(np.float64), lam0, 0.9, 1e-9)
    assert np.allclose(norms.cpu().numpy(), ref_norms, rtol=1e-12)
    assert np.allclose(lam.cpu().numpy(), ref_lam, rtol=1e-12)
    # no update: the weights stay, the norms are still reported
    lam2 = torch.tensor(lam0, dtype=torch.float64, device="cuda")
    net.loss_balance(grads, lam2, norms, update=False)
    assert lam2.cpu().numpy().tolist() == lam0
    # the cavity has no initial set: its weight stays while the others move
    api, w, p, B, b, net, db, prob = _setup("ns_cavity_6x256", "fp32", n_res=500, n_bc=100)
    _, G, _ = _terms_gpu(net, p, db, prob)
    lam3 = torch.tensor([1.0, 5.0, 1.0], dtype=torch.float64, device="cuda")
    net.loss_balance(torch.tensor(G, dtype=torch.float32, device="cuda"), lam3)
    out = lam3.cpu().numpy()
    assert out[1] == 5.0 and out[0] != 1.0 and out[2] != 1.0
