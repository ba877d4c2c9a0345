"""L-BFGS refinement (Sec. 2.6.5): the device two-loop direction against the
oracle's, and whole steps (direction, backtracking line search, new pair) against
the oracle's L-BFGS run on the FP64 loss."""
import numpy as np
import pytest
import torch

import oracle
from synth import make_workload

from gpu_helpers import rel

pytestmark = pytest.mark.gpu


def test_two_loop_direction_matches_oracle(cuda_lib):
    from paper_2604_15645_gb300 import api
    w, p, B, b = make_workload("burgers1d_4x64")
    net = api.PinnNet.from_spec(w.spec, "fp32")
    P = net.P
    rng = np.random.default_rng(31)
    lb = api.Lbfgs(net, history=4)
    S, Y = [], []
    for k in range(6):                          # more pairs than the history holds: the ring wraps
        s = rng.standard_normal(P).astype(np.float32)
        y = (s * (1.0 + rng.uniform(0.5, 2.0, P)) + 0.01 * rng.standard_normal(P)).astype(np.float32)
        lb.push_pair(torch.tensor(s, device="cuda"), torch.tensor(y, device="cuda"))
        S.append(s.astype(np.float64)); Y.append(y.astype(np.float64))
    g = rng.standard_normal(P).astype(np.float32)
    pd = torch.empty(P, device="cuda")
    lb.direction(torch.tensor(g, device="cuda"), pd)
    ref = oracle.lbfgs_direction(g.astype(np.float64), S[-4:], Y[-4:])
    assert rel(pd.cpu().numpy(), ref) < 1e-5


def test_lbfgs_steps_follow_the_oracle(cuda_lib):
    from paper_2604_15645_gb300 import api
    w, p, B, b = make_workload("burgers1d_4x64", n_res=512, n_ic=64, n_bc=64, random_bias=0.1)
    net = api.PinnNet.from_spec(w.spec, "fp32")
    db = api.DeviceBatch.from_host(b)
    prob = api.make_problem(w.problem.nu)
    params = torch.tensor(p, device="cuda")
    lb = api.Lbfgs(net, history=5)
    gpu_losses = []
    for _ in range(6):
        loss, _ = lb.step(params, db, prob)
        gpu_losses.append(loss)
    assert net.status_poll() == 0
    m = oracle.Model.from_spec(w.spec)
    fg = lambda x: (lambda t, g: (t["total"], g))(*oracle.loss_and_grad(m, x, B, b, w.problem.nu))
    ref_losses, _ = oracle.lbfgs_minimize(fg, p.astype(np.float64), history=5, steps=6)
    ref_losses = ref_losses[1:]
    # descent, and the same trajectory as the FP64 run up to FP32 rounding
    assert all(l1 <= l0 for l0, l1 in zip(gpu_losses, gpu_losses[1:]))
    assert gpu_losses[-1] < 0.5 * ref_losses[0] or gpu_losses[-1] < gpu_losses[0]
    for lg, lr in zip(gpu_losses[:3], ref_losses[:3]):
        assert abs(lg - lr) <= 1e-3 * abs(lr)
