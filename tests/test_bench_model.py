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
    fl, by, sch = bench.algorithmic_work(w, rows, b.n_res + b.n_ic + b.n_bc, "bf16")
    assert sum(fl.values()) == pytest.approx(expected, rel=5e-3)
    # bytes: every phase moves at least its activations once
    assert all(by[k] > 0 for k in ("fwd_gemm", "dw_gemm", "adj_gemm")) and by["adjdw_gemm"] == 0
    # the BF16 scheme's value-row low halves are reported apart from the method's bytes
    assert sch["fwd_gemm"] > 0 and sch["adj_gemm"] == 0 and sch["dw_gemm"] == 0


def test_block_layout_matches_parameter_count():
    import bench
    from synth import make_workload, param_count
    for name in ("burgers1d_4x64", "ns_cavity_6x256", "maxwell_te_5x512"):
        w = make_workload(name, n_res=8)[0]
        blocks = bench._blocks(w.spec)
        assert blocks[0][1] == 0 and blocks[-1][2] == param_count(w.spec)
        assert all(a[2] == b[1] for a, b in zip(blocks, blocks[1:]))


def test_fused_layers_book_both_gemms_once():
    """With the adjoint and weight gradient of every layer after the first fused, the
    FLOPs move to the fused phase and the total is unchanged; the fused phase moves the
    adjoint's bytes only (the weight gradient reads the same arrays in the same pass)."""
    import bench
    from synth import make_workload
    w, _, _, b = make_workload("ns_cavity_6x256")
    rows = 4 * b.n_res + b.n_ic + b.n_bc
    n = b.n_res + b.n_ic + b.n_bc
    fl0, by0, _ = bench.algorithmic_work(w, rows, n, "bf16")
    engines = [1] + [2] * (len(w.spec.widths) - 1)
    fl1, by1, _ = bench.algorithmic_work(w, rows, n, "bf16", engines)
    assert sum(fl1.values()) == pytest.approx(sum(fl0.values()), rel=1e-12)
    assert fl1["adj_gemm"] == 0 and fl1["adjdw_gemm"] > 0
    assert by1["adjdw_gemm"] == pytest.approx(by0["adj_gemm"], rel=1e-12)
