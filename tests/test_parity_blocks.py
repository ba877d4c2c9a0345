"""The per-block gradient check that the GPU parity tests run next to the global
relative L2 norm (parity_blocks.py), tested on the CPU against the oracle.

Mutations are planted in the oracle's gradient, on the CPU: the RWF scale gradient
dL/ds of one layer dropped (Eq. 15's chain rule ds_i = sum_j dW_ij W_ij left out) or
its sign flipped, and one layer's bias gradient dropped.  Each changes the whole
gradient by far less than the BF16 tolerance of 2e-2, so the global check alone lets
it through; the per-block check must name the block."""
import numpy as np
import pytest

import oracle
from synth import NetSpec, make_workload, param_count
from synth.workloads import PDE_MAXWELL, PDE_NS

from parity_blocks import FLOOR, block_errors, check_blocks, param_blocks

TOL_BF16 = 2e-2


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("spec", [NetSpec(PDE_NS, 2, 3, [48, 80, 48], ff_m=20, rwf=True),
                                  NetSpec(PDE_MAXWELL, 3, 3, [9, 1], rwf=True),
                                  NetSpec(0, 2, 1, [64] * 4)])
def test_blocks_tile_the_packed_layout(spec):
    blocks = param_blocks(spec)
    assert blocks[0][1] == 0 and blocks[-1][2] == param_count(spec)
    assert all(a[2] == b[1] for a, b in zip(blocks, blocks[1:]))
    n_layers = len(spec.widths) + 1
    assert len(blocks) == n_layers * (3 if spec.rwf else 2)


@pytest.fixture(scope="module")
def cavity_grad():
    w, p, B, b = make_workload("ns_cavity_6x256", n_res=256, n_bc=64, random_bias=0.1)
    m = oracle.Model.from_spec(w.spec)
    _, g = oracle.loss_and_grad(m, p, B, b, w.problem.nu)
    return w.spec, g


def _block(spec, name):
    return next((a, b) for n, a, b in param_blocks(spec) if n == name)


@pytest.mark.parametrize("name,mutate", [("s6", lambda x: 0.0 * x), ("s6", lambda x: -x), ("s4", lambda x: 0.0 * x),
                                         ("b7", lambda x: 0.0 * x)])
def test_block_check_catches_what_the_global_norm_misses(cavity_grad, name, mutate):
    spec, g = cavity_grad
    a, b = _block(spec, name)
    bad = g.copy()
    bad[a:b] = mutate(g[a:b])
    assert _rel(bad, g) < TOL_BF16                       # the global check passes it
    with pytest.raises(AssertionError) as e:
        check_blocks(bad, g, spec, TOL_BF16, "mutant")
    assert f" {name} err" in str(e.value).split("all blocks")[0]


def test_block_check_passes_rounding_noise(cavity_grad):
    # BF16-sized relative noise on every entry stays inside every block's tolerance
    spec, g = cavity_grad
    rng = np.random.default_rng(3)
    noisy = g * (1.0 + 4e-3 * rng.standard_normal(g.size))
    rows = check_blocks(noisy, g, spec, TOL_BF16, "noise")
    assert max(r[1] for r in rows) < 1e-2


def test_floor_applies_only_to_negligible_blocks():
    spec = NetSpec(0, 2, 1, [4, 4])
    g = np.zeros(param_count(spec))
    g[0] = 1.0
    a, b = _block(spec, "b3")
    noisy = g.copy()
    noisy[a:b] = 0.5 * FLOOR                 # a block with zero true gradient, error half the floor
    rows = {r[0]: r for r in block_errors(noisy, g, param_blocks(spec))}
    assert rows["b3"][1] == pytest.approx(0.5)
    assert rows["V1"][1] == 0.0
