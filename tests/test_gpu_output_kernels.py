"""The three output/loss kernels against the FP64 oracle, BF16 (their only precision
for the first two):

* width <= 256, a multiple of 32: the output layer's contractions on warp-level
  tensor-core MMAs (k_out_loss_mma), for one output (Burgers jet rule) and three
  (Navier-Stokes and Maxwell jet rules), with initial and boundary sets and masks;
* width <= 512, a multiple of 32: the CUDA-core kernel fed by the same TMA ring
  (k_out_loss_tma);
* any other width: the register-tiled kernel (k_out_loss).
Each case runs a few hundred points over several tiles and a ragged tail, so every
consumer warp of the TMA kernels sees interior, initial, boundary and padding points."""
import dataclasses

import pytest

from synth import NetSpec, Problem, init_params, ff_matrix, make_batch
from synth.workloads import PDE_BURGERS, PDE_NS, PDE_MAXWELL, PDE_ALLEN_CAHN

from gpu_helpers import TOL, assert_parity, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


def _case(pde, d_in, d_out, widths, ff, n_res, n_ic, n_bc, seed, masks=None):
    spec = NetSpec(pde, d_in, d_out, widths, ff_m=ff, ff_sigma=1.0, rwf=True)
    p = init_params(spec, seed, 0.15)
    B = ff_matrix(spec, seed + 1) if ff else None
    b = make_batch(pde, n_res, n_ic, n_bc, seed + 2, seed + 3)
    if masks is not None:
        b = dataclasses.replace(b, ic_mask=masks[0], bc_mask=masks[1])
    return spec, p, B, b


@pytest.mark.parametrize("widths", [[64, 32], [96, 128], [64, 256]])
def test_mma_output_kernel_navier_stokes(cuda_lib, widths):
    spec, p, B, b = _case(PDE_NS, 2, 3, widths, 16, 700, 0, 190, 301)
    gt, gg = run_gpu(spec, p, B, b, Problem(0.02, 0.7, 1.0, 3.0), "bf16")
    rt, rg = run_oracle(spec, p, B, b, Problem(0.02, 0.7, 1.0, 3.0))
    assert_parity(gt, gg, rt, rg, TOL["bf16"], f"NS {widths}", spec=spec)


@pytest.mark.parametrize("widths,masks", [([128, 128, 128], None), ([64, 160], (0b110, 0b011))])
def test_mma_output_kernel_maxwell(cuda_lib, widths, masks):
    spec, p, B, b = _case(PDE_MAXWELL, 3, 3, widths, 0, 500, 120, 150, 311, masks)
    gt, gg = run_gpu(spec, p, B, b, Problem(0.0, 1.0, 2.0, 0.5), "bf16")
    rt, rg = run_oracle(spec, p, B, b, Problem(0.0, 1.0, 2.0, 0.5))
    assert_parity(gt, gg, rt, rg, TOL["bf16"], f"Maxwell {widths}", spec=spec)


@pytest.mark.parametrize("pde,widths", [(PDE_BURGERS, [64, 64, 64]), (PDE_ALLEN_CAHN, [32, 224])])
def test_mma_output_kernel_one_output(cuda_lib, pde, widths):
    spec, p, B, b = _case(pde, 2, 1, widths, 0, 650, 90, 110, 321)
    prob = Problem(0.01, 1.0, 4.0, 2.0)
    gt, gg = run_gpu(spec, p, B, b, prob, "bf16")
    rt, rg = run_oracle(spec, p, B, b, prob)
    assert_parity(gt, gg, rt, rg, TOL["bf16"], f"one output {widths}", spec=spec)


@pytest.mark.parametrize("widths", [[64, 288], [32, 512]])
def test_tma_output_kernel_wider_layers(cuda_lib, widths):
    spec, p, B, b = _case(PDE_NS, 2, 3, widths, 16, 600, 0, 140, 331)
    gt, gg = run_gpu(spec, p, B, b, Problem(0.02, 1.0, 1.0, 1.0), "bf16")
    rt, rg = run_oracle(spec, p, B, b, Problem(0.02, 1.0, 1.0, 1.0))
    assert_parity(gt, gg, rt, rg, TOL["bf16"], f"NS {widths}", spec=spec)


@pytest.mark.parametrize("widths", [[64, 40], [48, 200]])
def test_register_output_kernel_other_widths(cuda_lib, widths):
    spec, p, B, b = _case(PDE_MAXWELL, 3, 3, widths, 0, 400, 60, 90, 341)
    gt, gg = run_gpu(spec, p, B, b, Problem(0.0, 1.0, 1.0, 1.0), "bf16")
    rt, rg = run_oracle(spec, p, B, b, Problem(0.0, 1.0, 1.0, 1.0))
    assert_parity(gt, gg, rt, rg, TOL["bf16"], f"Maxwell {widths}", spec=spec)
