"""The library from plain C: tests/c_abi_burgers.c uses only include/pinn.h and the
CUDA runtime.  Its loss and gradient on its own inputs match the FP64 oracle at the
FP32 tolerance, and its Adam steps lower the loss."""
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from synth import Batch, NetSpec
from synth.workloads import PDE_BURGERS

from gpu_helpers import TOL, rel

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_caller_matches_oracle(cuda_lib, tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    pkg = os.path.join(ROOT, "paper_2604_15645_gb300")
    exe = str(tmp_path / "c_abi_burgers")
    subprocess.run([nvcc, "-O2", os.path.join(ROOT, "tests", "c_abi_burgers.c"), "-I", os.path.join(ROOT, "include"),
                    "-L", pkg, "-lpinn", "-Xlinker", "-rpath", "-Xlinker", pkg, "-o", exe], check=True, timeout=300)
    out = str(tmp_path / "result.bin")
    r = subprocess.run([exe, out], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    summary = json.loads(r.stdout.strip().splitlines()[-1])
    assert np.isfinite(summary["loss_last"]) and summary["loss_last"] < summary["loss_first"]

    raw = open(out, "rb").read()
    P, n_res, n_ic, n_bc = np.frombuffer(raw[:32], dtype=np.int64)
    off = 32

    def take(n, dt):
        nonlocal off
        a = np.frombuffer(raw[off:off + n * np.dtype(dt).itemsize], dtype=dt)
        off += n * np.dtype(dt).itemsize
        return a

    params = take(P, np.float32)
    x_res = take(2 * n_res, np.float32).reshape(2, n_res)
    x_ic = take(2 * n_ic, np.float32).reshape(2, n_ic)
    g_ic = take(n_ic, np.float32).reshape(1, n_ic)
    x_bc = take(2 * n_bc, np.float32).reshape(2, n_bc)
    g_bc = take(n_bc, np.float32).reshape(1, n_bc)
    loss = take(8, np.float64)
    grad = take(P, np.float32).astype(np.float64)
    assert off == len(raw)

    spec = NetSpec(PDE_BURGERS, 2, 1, [32, 32, 32], rwf=True)
    b = Batch(x_res, x_ic, g_ic, 1, x_bc, g_bc, 1)
    t, g = oracle.loss_and_grad(oracle.Model.from_spec(spec), params.astype(np.float64), None, b,
                                0.01 / np.pi)
    assert P == g.size
    for i, key in ((0, "total"), (1, "pde"), (5, "ic"), (6, "bc")):
        assert abs(loss[i] - t[key]) <= TOL["fp32"] * abs(t[key]), (key, loss[i], t[key])
    assert rel(grad, g) <= TOL["fp32"]
