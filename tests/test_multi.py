"""Many independent networks in one graph-captured training step (pinn_multi_*):
per-network loss and gradient against the FP64 oracle, the fused Adam update,
bitwise equality of graph replays with eager single-network steps and of the grouped
per-level launches with the per-network launch sequences (the default), and the
engine autotuner's JSON cache."""
import json

import numpy as np
import pytest
import torch

import oracle
from synth import make_family

from gpu_helpers import TOL, assert_parity, rel, run_oracle

pytestmark = pytest.mark.gpu


def _setup(n, max_res, precision):
    from paper_2604_15645_gb300 import api
    fam = make_family(n, max_res=max_res, random_bias=0.1)
    multi = api.PinnMulti([s for s, _, _, _ in fam], precision)
    multi.set_inputs([api.DeviceBatch.from_host(b) for _, _, b, _ in fam],
                     [api.make_problem(pr.nu) for _, _, _, pr in fam])
    p0 = np.concatenate([p for _, p, _, _ in fam]).astype(np.float32)
    assert p0.size == multi.P
    return api, fam, multi, p0


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_multi_step_matches_oracle_per_network(cuda_lib, precision):
    api, fam, multi, p0 = _setup(8, 1536, precision)
    params = torch.tensor(p0, device="cuda")
    grad = torch.zeros_like(params)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    loss = multi.train_step(params, grad, m, v, step=1, lr=1e-3)
    torch.cuda.synchronize()
    assert multi.status_poll() == 0
    g = grad.cpu().numpy().astype(np.float64)
    L = loss.cpu().numpy()
    off = multi.offsets
    for i, (spec, p, b, pr) in enumerate(fam):
        rt, rg = run_oracle(spec, p, None, b, pr)
        assert_parity(L[i], g[off[i]:off[i + 1]], rt, rg, TOL[precision], f"net {i} {spec.widths}", spec=spec)
    b1, b2, lr, eps = (float(np.float32(x)) for x in (0.9, 0.999, 1e-3, 1e-8))
    th, _, _ = oracle.adam_step(p0.astype(np.float64), g, np.zeros_like(g), np.zeros_like(g), 1, lr, b1, b2, eps)
    assert rel(params.cpu().numpy(), th) < 1e-6


def test_multi_graph_replays_equal_eager_steps(cuda_lib):
    api, fam, multi, p0 = _setup(5, 1024, "bf16")
    params = torch.tensor(p0, device="cuda")
    grad, m, v = (torch.zeros_like(params) for _ in range(3))
    for step in range(1, 4):
        multi.train_step(params, grad, m, v, step=step, lr=1e-3)
    torch.cuda.synchronize()
    # the same three steps, one network at a time, without a graph
    nets = []
    for spec, _, b, pr in fam:
        net = api.PinnNet.from_spec(spec, "bf16")
        nets.append((net, api.DeviceBatch.from_host(b), api.make_problem(pr.nu)))
    p2 = torch.tensor(p0, device="cuda")
    g2, m2, v2 = (torch.zeros_like(p2) for _ in range(3))
    off = multi.offsets
    for step in range(1, 4):
        for i, (net, db, prob) in enumerate(nets):
            net.loss_grad(p2[off[i]:off[i + 1]], db, prob, grad=g2[off[i]:off[i + 1]])
        api.adam_step(p2, g2, m2, v2, step, lr=1e-3)
    torch.cuda.synchronize()
    assert torch.equal(params, p2) and torch.equal(m, m2) and torch.equal(v, v2)


def test_multi_autotune_cache(cuda_lib, tmp_path):
    api, fam, multi, p0 = _setup(6, 2048, "bf16")
    params = torch.tensor(p0, device="cuda")
    grad = torch.zeros_like(params)
    path = str(tmp_path / "tune.json")
    multi.autotune(params, grad, path)
    with open(path) as f:
        cache = json.load(f)
    assert cache and all(v in api.PinnMulti.CONFIGS for v in cache.values())
    first = multi.configs()
    for i in range(multi.n):
        multi.set_engine(i, i % 2)
    multi.autotune(params, grad, path)          # reads the cache, no re-timing
    assert multi.configs() == first
    # a step after tuning still matches the oracle
    m, v = torch.zeros_like(params), torch.zeros_like(params)
    loss = multi.train_step(params, grad, m, v, step=1)
    torch.cuda.synchronize()
    spec, p, b, pr = fam[0]
    rt, rg = run_oracle(spec, p, None, b, pr)
    assert_parity(loss[0].cpu().numpy(), grad[:multi.offsets[1]].cpu().numpy(), rt, rg, TOL["bf16"], "tuned net 0",
                  spec=spec)


@pytest.mark.parametrize("config", ["tc", "cuda_cores", "tc_unfused", "tc_unfused_dw128"])
def test_every_kernel_configuration_matches_oracle(cuda_lib, config):
    """The configurations the autotuner chooses among (fused or separate adjoint and
    weight gradient, 256- or 128-row weight-gradient tiles, CUDA cores) all give the
    oracle's loss and gradient, on networks of the family with 256-wide layers."""
    api, fam, multi, p0 = _setup(12, 1536, "bf16")
    wide = [i for i, (s, _, _, _) in enumerate(fam) if s.widths[0] >= 128][:3]
    assert wide
    for i in range(multi.n):
        multi.set_config(i, config)
    assert multi.configs() == [config] * multi.n
    params = torch.tensor(p0, device="cuda")
    grad, m, v = (torch.zeros_like(params) for _ in range(3))
    loss = multi.train_step(params, grad, m, v, step=1)
    torch.cuda.synchronize()
    assert multi.status_poll() == 0
    g = grad.cpu().numpy().astype(np.float64)
    for i in wide:
        spec, p, b, pr = fam[i]
        rt, rg = run_oracle(spec, p, None, b, pr)
        assert_parity(loss[i].cpu().numpy(), g[multi.offsets[i]:multi.offsets[i + 1]], rt, rg, TOL["bf16"],
                      f"{config} net {i} {spec.widths}", spec=spec)


def test_full_family_every_network_against_torch_float64(cuda_lib):
    """The benchmark's 64-network family at its full sizes (widths 32-256, depths 3-6,
    1,024-65,536 interior points each) after autotuning: one training step's loss and
    gradient of every network against the paper's method run in float64 on the GPU
    (torch double-backward autograd), and against the oracle on each network's first
    256 interior points plus its initial and boundary sets (a separate call)."""
    from paper_2604_15645_gb300 import api
    from gpu_helpers import torch_loss_grad
    fam = make_family(64)
    multi = api.PinnMulti([s for s, _, _, _ in fam], "bf16")
    multi.set_inputs([api.DeviceBatch.from_host(b) for _, _, b, _ in fam],
                     [api.make_problem(pr.nu) for _, _, _, pr in fam])
    p0 = np.concatenate([p for _, p, _, _ in fam]).astype(np.float32)
    params = torch.tensor(p0, device="cuda")
    grad, m, v = (torch.zeros_like(params) for _ in range(3))
    multi.autotune(params, grad)
    loss = multi.train_step(params, grad, m, v, step=1)
    torch.cuda.synchronize()
    assert multi.status_poll() == 0
    L = loss.cpu().numpy()
    g = grad.cpu().numpy().astype(np.float64)
    off = multi.offsets
    worst = 0.0
    for i, (spec, p, b, pr) in enumerate(fam):
        l64, g64 = torch_loss_grad(spec, p, None, b, pr, torch.float64)
        assert abs(L[i][0] - l64) <= TOL["bf16"] * abs(l64), (i, L[i][0], l64)
        e = rel(g[off[i]:off[i + 1]], g64)
        worst = max(worst, e)
        assert e <= TOL["bf16"], (i, spec.widths, b.n_res, e)
    print(f"64 networks, full sizes: worst gradient error against torch float64 {worst:.2e}")
    # the oracle on subsets: one network call per member on its leading 256 interior points
    for i in range(0, 64, 8):
        spec, p, b, pr = fam[i]
        sub = b.subset(256)
        net = api.PinnNet.from_spec(spec, "bf16")
        t, gg = net.loss_grad(torch.tensor(p, device="cuda"), api.DeviceBatch.from_host(sub), api.make_problem(pr.nu))
        rt, rg = run_oracle(spec, p, None, sub, pr)
        assert_parity(t.cpu().numpy(), gg.cpu().numpy().astype(np.float64), rt, rg, TOL["bf16"], f"family net {i}",
                      spec=spec)


def _two_steps(api, fam, multi, p0, grouped):
    multi.grouped = grouped
    assert multi.grouped == grouped
    params = torch.tensor(p0, device="cuda")
    grad, m, v = (torch.zeros_like(params) for _ in range(3))
    losses = []
    for step in (1, 2):
        losses.append(multi.train_step(params, grad, m, v, step=step, lr=1e-3).clone())
    torch.cuda.synchronize()
    assert multi.status_poll() == 0
    return params, grad, m, v, losses


@pytest.mark.parametrize("precision,config", [("bf16", "tc"), ("bf16", "tc_unfused"), ("bf16", "tc_unfused_dw128"),
                                              ("bf16", "mixed"), ("tf32", "tc"), ("fp32", "cuda_cores")])
def test_grouped_step_equals_per_network_step(cuda_lib, precision, config):
    """One grouped tcgen05 launch per layer level over all networks gives bitwise the
    step of the per-network launch sequences (each GEMM keeps its CTAs and work split),
    for every kernel configuration and a mix of them; both graphs are replayed twice."""
    api, fam, multi, p0 = _setup(12, 1536, precision)
    cfgs = api.PinnMulti.CONFIGS
    for i in range(multi.n):
        multi.set_config(i, cfgs[i % len(cfgs)] if config == "mixed" else config)
    a = _two_steps(api, fam, multi, p0, True)
    b = _two_steps(api, fam, multi, p0, False)
    for x, y in zip(a[:4], b[:4]):
        assert torch.equal(x, y)
    for x, y in zip(a[4], b[4]):
        assert torch.equal(x, y)


def test_full_family_grouped_equals_per_network_step(cuda_lib):
    """The benchmark's 64-network family at full size after autotuning: the grouped
    step and the per-network step agree bitwise over two replays."""
    from paper_2604_15645_gb300 import api
    fam = make_family(64)
    multi = api.PinnMulti([s for s, _, _, _ in fam], "bf16")
    multi.set_inputs([api.DeviceBatch.from_host(b) for _, _, b, _ in fam],
                     [api.make_problem(pr.nu) for _, _, _, pr in fam])
    p0 = np.concatenate([p for _, p, _, _ in fam]).astype(np.float32)
    params = torch.tensor(p0, device="cuda")
    multi.autotune(params, torch.zeros_like(params))
    a = _two_steps(api, fam, multi, p0, True)
    b = _two_steps(api, fam, multi, p0, False)
    for x, y in zip(a[:4], b[:4]):
        assert torch.equal(x, y)
