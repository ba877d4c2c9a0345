"""CUDA-graph replay of whole calls (pinn_set_graph): results equal to the eager
calls bit for bit, re-capture on any argument change, and replays that read the
current contents of the caller's buffers."""
import numpy as np
import pytest
import torch

from synth import make_workload, init_params

pytestmark = pytest.mark.gpu


def _setup(name, precision, **kw):
    from paper_2604_15645_gb300 import api
    w, p, B, b = make_workload(name, random_bias=0.1, **kw)
    net = api.PinnNet.from_spec(w.spec, precision, value_split=w.value_split and precision == "bf16")
    if B is not None:
        net.set_ff_matrix(B)
    db = api.DeviceBatch.from_host(b)
    prob = api.make_problem(w.problem.nu, w.problem.lambda_pde, w.problem.lambda_ic, w.problem.lambda_bc)
    return api, w, net, torch.tensor(p, device="cuda"), db, prob


@pytest.mark.parametrize("precision", ["bf16", "tf32", "fp32"])
def test_graph_replay_is_bitwise_equal(cuda_lib, precision):
    api, w, net, p, db, prob = _setup("ns_cavity_6x256", precision, n_res=8192, n_bc=1024)
    g0 = torch.empty_like(p)
    t0, _ = net.loss_grad(p, db, prob, grad=g0)
    t0 = t0.clone()
    net.set_graph(True)
    g1 = torch.empty_like(p)
    for _ in range(3):                      # capture, then two replays
        t1, _ = net.loss_grad(p, db, prob, grad=g1)
        torch.cuda.synchronize()
        assert torch.equal(t1, t0) and torch.equal(g1, g0)
    assert net.status_poll() == 0


def test_graph_recaptures_and_reads_current_buffers(cuda_lib):
    api, w, net, p, db, prob = _setup("burgers1d_4x64", "fp32", n_res=4096, n_ic=256, n_bc=256)
    net.set_graph(True)
    g = torch.empty_like(p)
    ta = net.loss_grad(p, db, prob, grad=g)[0].clone()
    # new parameter values in the same buffer: the replay sees them
    p2 = torch.tensor(init_params(w.spec, 99, 0.1), device="cuda")
    p.copy_(p2)
    tb = net.loss_grad(p, db, prob, grad=g)[0].clone()
    net.set_graph(False)
    tref = net.loss_grad(p2, db, prob)[0].clone()
    assert torch.equal(tb, tref) and not torch.equal(ta, tb)
    # a changed problem value is a different graph
    net.set_graph(True)
    prob2 = api.make_problem(2 * w.problem.nu, 1.0, 0.5, 2.0)
    tc = net.loss_grad(p, db, prob2, grad=g)[0].clone()
    net.set_graph(False)
    td = net.loss_grad(p, db, prob2)[0].clone()
    assert torch.equal(tc, td)


def test_graph_with_chunking_and_loss_only(cuda_lib):
    api, w, net, p, db, prob = _setup("burgers1d_4x64", "bf16", n_res=5000, n_ic=300, n_bc=300)
    net.set_chunk_points(2048)
    t0 = net.loss(p, db, prob).clone()
    g0 = net.loss_grad(p, db, prob)[1].clone()
    net.set_graph(True)
    for _ in range(2):
        t1 = net.loss(p, db, prob).clone()
        g1 = net.loss_grad(p, db, prob)[1].clone()
        torch.cuda.synchronize()
        assert torch.equal(t1, t0) and torch.equal(g1, g0)


def test_graph_replay_at_full_bench_size(cuda_lib):
    """The bench's configuration: the full cavity workload (65,536 + 4,096 points, BF16
    with the value-row weight split) replayed from a graph equals the eager call bit for
    bit; the eager call is the one the full-size parity test checks against the oracle."""
    from paper_2604_15645_gb300 import api
    w, pp, B, b = make_workload("ns_cavity_6x256")      # the full-size parity test's inputs
    assert w.value_split
    net = api.PinnNet.from_spec(w.spec, "bf16", value_split=True)
    net.set_ff_matrix(B)
    db = api.DeviceBatch.from_host(b)
    prob = api.make_problem(w.problem.nu, w.problem.lambda_pde, w.problem.lambda_ic, w.problem.lambda_bc)
    p = torch.tensor(pp, device="cuda")
    g0 = torch.empty_like(p)
    t0 = net.loss_grad(p, db, prob, grad=g0)[0].clone()
    net.set_graph(True)
    g1 = torch.empty_like(p)
    for _ in range(3):
        t1 = net.loss_grad(p, db, prob, grad=g1)[0].clone()
    torch.cuda.synchronize()
    assert torch.equal(t1, t0) and torch.equal(g1, g0)
    assert net.status_poll() == 0


def test_training_loop_with_graph_replay_decreases_the_loss(cuda_lib):
    """A short Adam training loop through the public API, each step replayed from one
    captured graph (same buffers every step): the loss goes down and stays finite."""
    from paper_2604_15645_gb300 import api
    w, pp, B, b = make_workload("ns_cavity_6x256", n_res=4096, n_bc=1024)
    w.spec.widths = [128] * 3
    pp = init_params(w.spec, 17, 0.0)
    net = api.PinnNet.from_spec(w.spec, "bf16", value_split=True)
    net.set_ff_matrix(B)
    net.set_graph(True)
    db = api.DeviceBatch.from_host(b)
    prob = api.make_problem(w.problem.nu)
    theta = torch.tensor(pp, device="cuda")
    grad, m, v = (torch.zeros_like(theta) for _ in range(3))
    losses = []
    for step in range(1, 41):
        loss, _ = net.loss_grad(theta, db, prob, grad=grad)
        losses.append(float(loss[0]))
        api.adam_step(theta, grad, m, v, step, lr=1e-3)
    torch.cuda.synchronize()
    assert net.status_poll() == 0
    assert np.all(np.isfinite(losses)) and losses[-1] < 0.5 * losses[0]
