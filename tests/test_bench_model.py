"""The bench's algorithmic work model against the jet-GEMM FLOP counts worked out
independently for the five configurations (GEMM units x 2 MAC per jet row, rows
4 N_res + N_ic + N_bc; 1.25e9, 5.93e11, 6.80e12 and 5.08e13 FLOP per step)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.mark.parametrize("name,expected", [("burgers1d_4x64", 1.25e9), ("ns_cavity_6x256", 5.93e11),
                                           ("maxwell_te_5x512", 6.80e12), ("ns_cavity_8x512", 5.08e13)])
def test_jet_gemm_flops_per_step(name, expected):
    import bench
    from synth import make_workload
    w, _, _, b = make_workload(name)
    rows = 4 * b.n_res + b.n_ic + b.n_bc
    fl, by = bench.algorithmic_work(w, rows, b.n_res + b.n_ic + b.n_bc, "bf16")
    assert sum(fl.values()) == pytest.approx(expected, rel=5e-3)
    # bytes: every phase moves at least its activations once
    assert all(v > 0 for v in by.values())
