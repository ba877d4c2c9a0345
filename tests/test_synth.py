"""The seeded input generator (shared by the CUDA path's tests and the oracle)."""
import math
import os

import numpy as np

from synth import SplitMix64, make_workload, param_count, family_specs
from synth.workloads import _r_sequence

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_ints(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [int(l) for l in f if l.strip() and not l.startswith("#")]


def test_splitmix64_reference_vector():
    want = _golden_ints("splitmix64_seed1234567.txt")
    got = SplitMix64(1234567).next_u64(5)
    assert [int(x) for x in got] == want
    # drawing in pieces gives the same stream
    r = SplitMix64(1234567)
    assert [int(x) for x in np.concatenate([r.next_u64(2), r.next_u64(3)])] == want


def test_box_muller_moments():
    z = SplitMix64(7).normal(200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01
    u = SplitMix64(8).uniform(100000)
    assert u.min() >= 0 and u.max() < 1 and abs(u.mean() - 0.5) < 0.01


def test_low_discrepancy_sequence_is_in_unit_cube_and_even():
    p = _r_sequence(4096, 3, np.array([0.1, 0.2, 0.3]))
    assert p.shape == (3, 4096) and p.min() >= 0 and p.max() < 1
    # every octant holds close to 1/8 of the points
    octant = (p[0] > .5).astype(int) * 4 + (p[1] > .5) * 2 + (p[2] > .5)
    counts = np.bincount(octant, minlength=8)
    assert np.all(np.abs(counts - 512) < 20)


def test_workload_shapes_and_param_counts():
    w, p, B, b = make_workload("ns_cavity_6x256", n_res=100)
    assert B.shape == (2, 128) and b.x_res.shape == (2, 100) and b.x_bc.shape == (2, 4096)
    # FF 256 -> 6 x 256 -> 3 with RWF: six 256x256 layers plus the output layer
    assert param_count(w.spec) == 6 * (256 * 256 + 2 * 256) + (3 * 256 + 2 * 3) == p.size
    w, p, B, b = make_workload("burgers1d_4x64")
    assert b.n_res == 4096 and b.n_ic == 256 and b.n_bc == 256 and B is None
    assert np.allclose(b.g_ic[0], -np.sin(np.pi * b.x_ic[0]), atol=1e-6)
    assert np.all(np.abs(b.x_bc[0]) == 1)


def test_family_specs():
    fam = family_specs()
    assert len(fam) == 64
    for m in fam:
        assert m["spec"].widths[0] in (32, 64, 128, 256) and 3 <= len(m["spec"].widths) <= 6
        assert 1e-3 <= m["nu"] <= 1e-1 and 1024 <= m["n_res"] <= 65536 and m["n_res"] % 32 == 0
