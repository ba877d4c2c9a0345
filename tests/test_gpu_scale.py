"""The Maxwell and at-scale cavity workloads: BF16 parity on subsets against the
FP64 oracle, and at full size (1,048,576 interior + 16,384 wall points, 8x512,
256 Fourier frequencies with sigma 2) the BF16 gradient on 32 random coordinates
against central finite differences of the FP32 loss."""
import gc

import numpy as np
import pytest
import torch

from synth import make_workload

from gpu_helpers import TOL, assert_parity, rel, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


def test_maxwell_low_discrepancy_subset_bf16(cuda_lib):
    w, p, B, b = make_workload("maxwell_te_5x512", n_res=16384, n_ic=1024, n_bc=1024)
    gt, gg = run_gpu(w.spec, p, B, b, w.problem, "bf16")
    rt, rg = run_oracle(w.spec, p, B, b, w.problem, chunk=4096)
    assert_parity(gt, gg, rt, rg, TOL["bf16"], "maxwell 16k bf16", spec=w.spec)


@pytest.mark.parametrize("value_split", [False, True])
def test_cavity_at_scale_architecture_subset_bf16(cuda_lib, value_split):
    w, p, B, b = make_workload("ns_cavity_8x512", n_res=4096, n_bc=256)
    gt, gg = run_gpu(w.spec, p, B, b, w.problem, "bf16", value_split=value_split)
    rt, rg = run_oracle(w.spec, p, B, b, w.problem, chunk=2048)
    assert_parity(gt, gg, rt, rg, TOL["bf16"], f"cavity 8x512 subset bf16 value_split={value_split}",
                  spec=w.spec)


def _free():
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def test_cavity_at_scale_gradient_against_finite_differences(cuda_lib):
    from paper_2604_15645_gb300 import api
    _free()
    w, p, B, b = make_workload("ns_cavity_8x512")
    prob = api.make_problem(w.problem.nu)
    db = api.DeviceBatch.from_host(b)
    params = torch.tensor(p, device="cuda")

    bf16 = {}
    for value_split in (False, True):
        net = api.PinnNet.from_spec(w.spec, "bf16", value_split=value_split)
        net.set_ff_matrix(B)
        t16, g16 = net.loss_grad(params, db, prob)
        bf16[value_split] = (float(t16[0]), g16.cpu().numpy().astype(np.float64))
        assert net.status_poll() == 0
        del net, t16, g16
        _free()

    net = api.PinnNet.from_spec(w.spec, "fp32")
    net.set_ff_matrix(B)
    t32, g32 = net.loss_grad(params, db, prob)
    loss32 = float(t32[0])
    g32 = g32.cpu().numpy().astype(np.float64)
    for loss16, _ in bf16.values():
        assert abs(loss16 - loss32) <= TOL["bf16"] * abs(loss32)

    # 32 coordinates: 4 per weight layer group (V, s, b mixed), seeded
    rng = np.random.default_rng(2024)
    P = params.numel()
    idx = np.sort(rng.choice(P, size=32, replace=False))
    fd = np.empty(32)
    out = torch.empty(8, dtype=torch.float64, device="cuda")
    for n, i in enumerate(idx):
        th = float(p[i])
        h = 1e-3 * max(1.0, abs(th))
        vals = []
        for s in (+1, -1):
            params[i] = th + s * h
            vals.append(float(net.loss(params, db, prob, out=out)[0]))
        params[i] = th
        fd[n] = (vals[0] - vals[1]) / (2 * h)
    assert net.status_poll() == 0
    del net
    _free()
    # the FP32 gradient confirms the differences themselves
    assert rel(g32[idx], fd) < 1e-3
    # the BF16 paths under test (full weight split, and value-row split), at the stated tolerance
    for _, g16 in bf16.values():
        assert rel(g16[idx], fd) <= TOL["bf16"]


def test_maxwell_full_size_gradient_against_finite_differences(cuda_lib):
    """The Maxwell workload at full size (262,144 interior points, 5x512, RWF) in the
    BF16 configuration the bench times: the gradient on 24 seeded coordinates against
    central differences of the FP32 loss, and the loss against the FP32 loss."""
    from paper_2604_15645_gb300 import api
    _free()
    w, p, B, b = make_workload("maxwell_te_5x512")
    prob = api.make_problem(w.problem.nu, w.problem.lambda_pde, w.problem.lambda_ic, w.problem.lambda_bc)
    db = api.DeviceBatch.from_host(b)
    params = torch.tensor(p, device="cuda")
    net16 = api.PinnNet.from_spec(w.spec, "bf16")
    if B is not None:
        net16.set_ff_matrix(B)
    t16, g16 = net16.loss_grad(params, db, prob)
    loss16, g16 = float(t16[0]), g16.cpu().numpy().astype(np.float64)
    assert net16.status_poll() == 0
    del net16
    _free()

    net = api.PinnNet.from_spec(w.spec, "fp32")
    if B is not None:
        net.set_ff_matrix(B)
    t32, g32 = net.loss_grad(params, db, prob)
    loss32, g32 = float(t32[0]), g32.cpu().numpy().astype(np.float64)
    assert abs(loss16 - loss32) <= TOL["bf16"] * abs(loss32)
    rng = np.random.default_rng(2025)
    idx = np.sort(rng.choice(params.numel(), size=24, replace=False))
    fd = np.empty(idx.size)
    out = torch.empty(8, dtype=torch.float64, device="cuda")
    for n, i in enumerate(idx):
        th = float(p[i])
        h = 1e-3 * max(1.0, abs(th))
        vals = []
        for s in (+1, -1):
            params[i] = th + s * h
            vals.append(float(net.loss(params, db, prob, out=out)[0]))
        params[i] = th
        fd[n] = (vals[0] - vals[1]) / (2 * h)
    assert net.status_poll() == 0
    assert rel(g32[idx], fd) < 1e-3
    assert rel(g16[idx], fd) <= TOL["bf16"]
