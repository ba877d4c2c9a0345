"""The periodic activation sin(omega0 z) (Sec. 2.6, Table 1) on the CUDA-core path
against the FP64 oracle, element by element on the same seeded inputs.  A sine
network keeps its pre-activation jets for the adjoint and runs no tensor-core layer."""
import numpy as np
import pytest
import torch

from synth import Batch, NetSpec, Problem, init_params, ff_matrix, make_batch, make_workload
from synth.workloads import PDE_BURGERS, PDE_NS, PDE_MAXWELL, PDE_ADVECTION

from gpu_helpers import TOL, assert_parity, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


def _sine(spec, omega0):
    spec.activation, spec.omega0 = "sine", omega0
    return spec


@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16"])
def test_sine_burgers_raw_inputs(cuda_lib, precision):
    # no Fourier features: the first layer is the elementwise one (it writes Z_1 too)
    w, p, B, b = make_workload("burgers1d_4x64", n_res=3000, n_ic=200, n_bc=200, random_bias=0.1)
    _sine(w.spec, 2.0)
    p = init_params(w.spec, 5, 0.1)
    gt, gg = run_gpu(w.spec, p, B, b, w.problem, precision)
    rt, rg = run_oracle(w.spec, p, B, b, w.problem)
    # TF32 with sine computes in FP32 on CUDA cores
    assert_parity(gt, gg, rt, rg, TOL["fp32" if precision == "tf32" else precision], f"sine burgers {precision}",
                  spec=w.spec)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_sine_cavity_fourier_rwf_ragged(cuda_lib, precision):
    w, p, B, b = make_workload("ns_cavity_6x256", n_res=1000, n_bc=300, random_bias=0.1)
    w.spec.widths = [128] * 4
    _sine(w.spec, 1.0)
    p = init_params(w.spec, 6, 0.1)
    gt, gg = run_gpu(w.spec, p, B, b, w.problem, precision)
    rt, rg = run_oracle(w.spec, p, B, b, w.problem)
    assert_parity(gt, gg, rt, rg, TOL[precision], f"sine cavity {precision}", spec=w.spec)


@pytest.mark.parametrize("omega0", [1.5, 3.0])
def test_sine_maxwell_first_order_rows(cuda_lib, omega0):
    # Rounding of each pre-activation enters sin(omega0 z) multiplied by omega0, so the
    # FP32 bound grows with it: 1e-5 up to omega0 = 2, then in proportion.  Per block,
    # the layers nearest the input take that factor once more: their gradient is the
    # adjoint carried back through the sine layers, whose rounding is amplified alike.
    w, p, B, b = make_workload("maxwell_te_5x512", n_res=600, n_ic=100, n_bc=150, random_bias=0.1)
    w.spec.widths = [96, 80, 96]
    _sine(w.spec, omega0)
    p = init_params(w.spec, 7, 0.1)
    gt, gg = run_gpu(w.spec, p, B, b, w.problem, "fp32")
    rt, rg = run_oracle(w.spec, p, B, b, w.problem)
    amp = max(1.0, omega0 / 2.0)
    assert_parity(gt, gg, rt, rg, TOL["fp32"] * amp, f"sine maxwell omega0={omega0}", spec=w.spec,
                  block_tol=TOL["fp32"] * amp * amp)


def test_sine_advection_single_neuron_solution(cuda_lib):
    # u = sin(x - c t) is one sine neuron: the residual loss is zero up to FP32 rounding
    c, w0 = 10.0, 2.0
    spec = NetSpec(PDE_ADVECTION, 2, 1, [1], activation="sine", omega0=w0)
    theta = np.array([1.0 / w0, -c / w0, 0.0, 1.0, 0.0])
    b = make_batch(PDE_ADVECTION, 4096, 0, 0, 11, 12, wave_speed=c)
    gt, _ = run_gpu(spec, theta, None, b, Problem(c), "fp32")
    assert gt[1] < 1e-9


def test_sine_workspace_and_engine(cuda_lib):
    from paper_2604_15645_gb300 import api
    w, p, B, b = make_workload("ns_cavity_6x256", n_res=4096, n_bc=512)
    tanh_net = api.PinnNet.from_spec(w.spec, "bf16")
    sine_net = api.PinnNet.from_spec(_sine(w.spec, 1.0), "bf16")
    assert tanh_net.tensor_core_layers(b.n_res, 0, b.n_bc) == len(w.spec.widths)
    # BF16 sine networks run on tcgen05 too, with separate adjoint and weight-gradient
    # kernels (the fused one carries the tanh rule only)
    assert sine_net.tensor_core_layers(b.n_res, 0, b.n_bc) == len(w.spec.widths)
    assert 2 not in sine_net.layer_engines(b.n_res, 0, b.n_bc) and 2 in tanh_net.layer_engines(b.n_res, 0, b.n_bc)
    # on the same (CUDA-core, FP32) engine, one FP32 pre-activation jet array per hidden
    # layer on top of the tanh workspace
    w.spec.activation = "tanh"
    tanh32 = api.PinnNet.from_spec(w.spec, "fp32")
    sine32 = api.PinnNet.from_spec(_sine(w.spec, 1.0), "fp32")
    extra = sine32.workspace_bytes(b.n_res, 0, b.n_bc) - tanh32.workspace_bytes(b.n_res, 0, b.n_bc)
    n_cols = 4 * (b.n_res + b.n_bc)
    assert 4 * n_cols * sum(w.spec.widths) <= extra <= 4 * n_cols * sum(w.spec.widths) + 256 * len(w.spec.widths)
    from paper_2604_15645_gb300 import _lib
    with pytest.raises(_lib.PinnError):
        sine_net.set_activation("sine", 0.0)
    with pytest.raises(_lib.PinnError):
        _lib.pinn_set_activation(sine_net.h, 7, 1.0)


def test_sine_chunked_matches_one_pass(cuda_lib):
    w, p, B, b = make_workload("burgers1d_4x64", n_res=5000, n_ic=300, n_bc=300, random_bias=0.1)
    _sine(w.spec, 2.0)
    p = init_params(w.spec, 8, 0.1)
    from paper_2604_15645_gb300 import api
    prob = api.make_problem(w.problem.nu)
    db = api.DeviceBatch.from_host(b)
    pt = torch.tensor(p, device="cuda")
    one = api.PinnNet.from_spec(w.spec, "fp32")
    t1, g1 = (x.clone() for x in one.loss_grad(pt, db, prob))
    ch = api.PinnNet.from_spec(w.spec, "fp32", chunk_points=1024)
    t2, g2 = ch.loss_grad(pt, db, prob)
    torch.cuda.synchronize()
    assert abs(float(t1[0]) - float(t2[0])) <= 1e-5 * abs(float(t1[0]))
    assert float((g1 - g2).norm() / g1.norm()) < 1e-5


@pytest.mark.parametrize("name,widths", [("ns_cavity_6x256", [128] * 4), ("burgers1d_4x64", [64] * 4)])
def test_sine_bf16_runs_on_tensor_cores(cuda_lib, name, widths):
    """BF16 sine networks run their hidden jet GEMMs on tcgen05 (the forward epilogue
    applies the sine jet rule and stores the pre-activations, the adjoint evaluates the
    rule from them); FP32 sine networks stay on CUDA cores."""
    from paper_2604_15645_gb300 import api
    w, p, B, b = make_workload(name, n_res=1000, n_ic=120, n_bc=90, random_bias=0.1)
    w.spec.widths = widths
    _sine(w.spec, 2.0)
    first_gemm = 0 if w.spec.ff_m else 1
    for precision, expect in (("bf16", len(widths) - first_gemm), ("fp32", 0)):
        net = api.PinnNet.from_spec(w.spec, precision)
        assert net.tensor_core_layers(b.n_res, b.n_ic, b.n_bc) == expect, precision
    p = init_params(w.spec, 8, 0.1)
    gt, gg = run_gpu(w.spec, p, B, b, w.problem, "bf16")
    rt, rg = run_oracle(w.spec, p, B, b, w.problem)
    assert_parity(gt, gg, rt, rg, TOL["bf16"], f"sine {name} bf16 tensor cores", spec=w.spec)
