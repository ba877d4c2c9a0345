"""CUDA path vs the FP64 oracle, element by element on the same seeded inputs.

Tolerances (relative; loss per term, gradient in L2 norm over all parameters):
FP32 1e-5, TF32 1e-3, BF16 2e-2.
"""
import numpy as np
import pytest
import torch

from synth import Batch, NetSpec, Problem, init_params, ff_matrix, make_batch, make_workload
from synth.workloads import PDE_BURGERS, PDE_NS, PDE_MAXWELL

from gpu_helpers import TOL, assert_parity, rel, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


def _check(spec, params, B, batch, problem, precision, what, chunk=None):
    gt, gg = run_gpu(spec, params, B, batch, problem, precision)
    rt, rg = run_oracle(spec, params, B, batch, problem, chunk=chunk)
    assert_parity(gt, gg, rt, rg, TOL[precision], what, spec=spec)
    return gt, gg, rt, rg


@pytest.mark.parametrize("random_bias", [0.0, 0.2])
def test_burgers_full_size_fp32(cuda_lib, random_bias):
    w, p, B, b = make_workload("burgers1d_4x64", random_bias=random_bias)
    _check(w.spec, p, B, b, w.problem, "fp32", "burgers fp32")


def test_cavity_value_split_ragged_subset(cuda_lib):
    w, p, B, b = make_workload("ns_cavity_6x256", n_res=1000, n_bc=300, random_bias=0.1)
    gt, gg = run_gpu(w.spec, p, B, b, w.problem, "bf16", value_split=True)
    rt, rg = run_oracle(w.spec, p, B, b, w.problem)
    assert_parity(gt, gg, rt, rg, TOL["bf16"], "cavity bf16 value split", spec=w.spec)


@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16"])
def test_cavity_architecture_ragged_subset(cuda_lib, precision):
    # 6x256 with 128 Fourier frequencies and RWF; 1000 interior + 300 wall points
    # (the column count is not a multiple of the tile, so the ragged tail is exercised)
    w, p, B, b = make_workload("ns_cavity_6x256", n_res=1000, n_bc=300, random_bias=0.1)
    _check(w.spec, p, B, b, w.problem, precision, f"cavity {precision}")


@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16"])
def test_maxwell_architecture_subset(cuda_lib, precision):
    w, p, B, b = make_workload("maxwell_te_5x512", n_res=600, n_ic=100, n_bc=150, random_bias=0.1)
    _check(w.spec, p, B, b, w.problem, precision, f"maxwell {precision}")


@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16"])
def test_ragged_widths_and_weights(cuda_lib, precision):
    spec = NetSpec(PDE_NS, 2, 3, [48, 80, 48], ff_m=20, ff_sigma=1.5, rwf=True)
    p = init_params(spec, 51, 0.2)
    B = ff_matrix(spec, 52)
    b = make_batch(PDE_NS, 333, 0, 77, 53, 54)
    _check(spec, p, B, b, Problem(0.02, 0.3, 2.0, 5.0), precision, "ragged")


@pytest.mark.parametrize("pde,d_in,d_out,widths,ff", [(PDE_BURGERS, 2, 1, [13, 7], 0), (PDE_NS, 2, 3, [5, 11, 3], 6),
                                                       (PDE_MAXWELL, 3, 3, [9, 1], 0)])
def test_widths_not_multiples_of_eight(cuda_lib, pde, d_in, d_out, widths, ff):
    # the output layer's feature slices run uneven passes; every lane still joins the shuffles
    spec = NetSpec(pde, d_in, d_out, widths, ff_m=ff, ff_sigma=1.0, rwf=True)
    p = init_params(spec, 57, 0.2)
    B = ff_matrix(spec, 58) if ff else None
    b = make_batch(pde, 300, 40 if pde != PDE_NS else 0, 50, 59, 60)
    for precision in ("fp32", "bf16"):
        _check(spec, p, B, b, Problem(0.02, 0.3, 2.0, 5.0), precision, f"odd widths {widths} {precision}")


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_maximum_width(cuda_lib, precision):
    # the widest layer the library takes (2048): the output kernel's shared-memory
    # accumulators (weights, dW and bias slots) are at their largest
    spec = NetSpec(PDE_NS, 2, 3, [64, 2048], ff_m=16, ff_sigma=1.0, rwf=True)
    p = init_params(spec, 63, 0.05)
    B = ff_matrix(spec, 64)
    b = make_batch(PDE_NS, 200, 0, 56, 65, 66)
    _check(spec, p, B, b, Problem(0.01, 1.0, 1.0, 1.0), precision, f"width 2048 {precision}")


@pytest.mark.parametrize("precision,expect_tc", [("fp32", False), ("tf32", True), ("bf16", True)])
def test_tensor_core_engine_selection(cuda_lib, precision, expect_tc):
    # FP32 runs the exact CUDA-core GEMMs; TF32 and BF16 run every hidden layer on tcgen05
    from paper_2604_15645_gb300 import api
    w, p, B, b = make_workload("ns_cavity_6x256", n_res=4096, n_bc=512)
    net = api.PinnNet.from_spec(w.spec, precision)
    n_tc = net.tensor_core_layers(b.n_res, 0, b.n_bc)
    n_layers = len(w.spec.widths)           # every layer into a hidden width (the Fourier one included)
    assert n_tc == (n_layers if expect_tc else 0)
    _check(w.spec, p, B, b, w.problem, precision, f"engine {precision}")


def test_only_boundary_points(cuda_lib):
    w, p, B, b = make_workload("burgers1d_4x64", n_res=0, random_bias=0.1)
    _check(w.spec, p, B, b, w.problem, "fp32", "boundary only")


def test_only_interior_points(cuda_lib):
    w, p, B, b = make_workload("maxwell_te_5x512", n_res=257, n_ic=0, n_bc=0)
    w.spec.widths = [64] * 3
    p = init_params(w.spec, 61, 0.1)
    _check(w.spec, p, B, b, w.problem, "fp32", "interior only")


def test_single_points(cuda_lib):
    spec = NetSpec(PDE_BURGERS, 2, 1, [32, 32])
    p = init_params(spec, 71, 0.3)
    b = make_batch(PDE_BURGERS, 1, 1, 1, 72, 73)
    _check(spec, p, None, b, Problem(0.05), "fp32", "single points")


def test_masks_select_outputs(cuda_lib):
    w, p, B, b = make_workload("ns_cavity_6x256", n_res=64, n_bc=64, random_bias=0.1)
    w.spec.widths = [64, 64]
    p = init_params(w.spec, 81, 0.1)
    b = Batch(b.x_res, b.x_ic, b.g_ic, 0, b.x_bc, b.g_bc, 0b101)
    _check(w.spec, p, B, b, w.problem, "fp32", "mask 0b101")


def test_deterministic_bitwise(cuda_lib):
    w, p, B, b = make_workload("ns_cavity_6x256", n_res=2000, n_bc=512, random_bias=0.1)
    t1, g1 = run_gpu(w.spec, p, B, b, w.problem, "bf16")
    t2, g2 = run_gpu(w.spec, p, B, b, w.problem, "bf16")
    assert np.array_equal(t1, t2) and np.array_equal(g1, g2)


def test_loss_only_matches_loss_grad(cuda_lib):
    w, p, B, b = make_workload("maxwell_te_5x512", n_res=300, n_ic=50, n_bc=60, random_bias=0.1)
    w.spec.widths = [128] * 3
    p = init_params(w.spec, 91, 0.1)
    t1, _ = run_gpu(w.spec, p, B, b, w.problem, "fp32", want_grad=False)
    t2, _ = run_gpu(w.spec, p, B, b, w.problem, "fp32")
    assert np.array_equal(t1, t2)


def test_adam_matches_oracle(cuda_lib):
    import oracle
    from paper_2604_15645_gb300 import api
    rng = np.random.default_rng(5)
    n = 10007
    theta = rng.standard_normal(n).astype(np.float32)
    m = np.zeros(n, np.float32); v = np.zeros(n, np.float32)
    tp, tm, tv = (torch.tensor(a, device="cuda") for a in (theta, m, v))
    th64, m64, v64 = theta.astype(np.float64), m.astype(np.float64), v.astype(np.float64)
    # the kernel receives float32 hyper-parameters; give the oracle the same values
    b1, b2, lr, eps = (float(np.float32(x)) for x in (0.9, 0.999, 1e-3, 1e-8))
    for step in range(1, 4):
        g = rng.standard_normal(n).astype(np.float32)
        api.adam_step(tp, torch.tensor(g, device="cuda"), tm, tv, step, lr=1e-3)
        th64, m64, v64 = oracle.adam_step(th64, g.astype(np.float64), m64, v64, step, lr, b1, b2, eps)
    torch.cuda.synchronize()
    assert rel(tp.cpu().numpy(), th64) < 1e-6
    assert rel(tm.cpu().numpy(), m64) < 1e-6 and rel(tv.cpu().numpy(), v64) < 1e-6


def test_autograd_function_backward_is_the_adjoint(cuda_lib):
    from paper_2604_15645_gb300 import api
    w, p, B, b = make_workload("burgers1d_4x64", n_res=512, random_bias=0.1)
    net = api.PinnNet.from_spec(w.spec, "fp32")
    params = torch.tensor(p, device="cuda", requires_grad=True)
    db = api.DeviceBatch.from_host(b)
    prob = api.make_problem(w.problem.nu)
    loss = api.PinnLoss.apply(params, net, db, prob)
    (3.0 * loss).backward()
    _, rg = run_oracle(w.spec, p, B, b, w.problem)
    assert rel(params.grad.cpu().numpy() / 3.0, rg) < 1e-5


def test_error_paths(cuda_lib):
    from paper_2604_15645_gb300 import _lib, api
    w, p, B, b = make_workload("ns_cavity_6x256", n_res=64, n_bc=64)
    net = api.PinnNet.from_spec(w.spec, "bf16")
    db = api.DeviceBatch.from_host(b)
    params = torch.tensor(p, device="cuda")
    prob = api.make_problem(w.problem.nu)
    with pytest.raises(_lib.PinnError) as e:       # Fourier matrix not registered
        net.loss_grad(params, db, prob)
    assert e.value.status == 1
    net.set_ff_matrix(B)
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    grad = torch.empty_like(params)
    with pytest.raises(_lib.PinnError) as e:       # workspace too small
        _lib.pinn_loss_grad(net.h, prob, db.c_struct(), params.data_ptr(), ws.data_ptr(), ws.numel(),
                            net.loss_buf.data_ptr(), grad.data_ptr(), 0)
    assert e.value.status == 4


def test_nonfinite_loss_is_latched(cuda_lib):
    from paper_2604_15645_gb300 import api
    w, p, B, b = make_workload("burgers1d_4x64", n_res=64)
    p = p.copy(); p[-1] = np.inf     # output bias
    net = api.PinnNet.from_spec(w.spec, "fp32")
    db = api.DeviceBatch.from_host(b)
    net.loss_grad(torch.tensor(p, device="cuda"), db, api.make_problem(w.problem.nu))
    assert net.status_poll() == 5
    assert net.status_poll() == 0     # cleared after reading


_FULL_ORACLE = {}


@pytest.mark.parametrize("precision,value_split", [("bf16", True), ("bf16", False), ("tf32", False)])
def test_cavity_full_size_against_chunked_oracle(cuda_lib, precision, value_split):
    """The bench workload at full size (65,536 interior + 4,096 wall points) in the
    launch configuration the bench times (BF16 with the value-row weight split is the
    workload's default); the oracle sums chunks of points (computed once)."""
    w, p, B, b = make_workload("ns_cavity_6x256")
    gt, gg = run_gpu(w.spec, p, B, b, w.problem, precision, value_split=value_split)
    if "ref" not in _FULL_ORACLE:
        _FULL_ORACLE["ref"] = run_oracle(w.spec, p, B, b, w.problem, chunk=8192)
    rt, rg = _FULL_ORACLE["ref"]
    assert_parity(gt, gg, rt, rg, TOL[precision], f"cavity full {precision}", spec=w.spec)
