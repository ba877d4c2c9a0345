"""pinn_loss_grad_static, the entry point for callers that cannot allocate device
memory (code in host callbacks or real-time loops where allocating may block or
fail, plug-ins whose host runtime owns the memory pool).  Instead of a caller
workspace it uses a 64 MiB scratch array compiled into the library.  Its results
must match pinn_loss_grad (caller-provided workspace) within the parity tolerance,
on two calls in a row, and it must refuse batches that do not fit the array.

It always launches eagerly: on a handle with CUDA-graph replay switched on it
captures no graph (capturing and instantiating one would allocate).  And it must
find its array again after the device's context has been reset (tests/c_static_reset.c,
a plain-C caller, since a reset would also pull device memory out from under torch).

This file is collected last on purpose, so a stop-at-first-failure run has already
run every other test if it fails."""
import os
import shutil
import subprocess

import numpy as np
import pytest
import torch

from synth import init_params, make_workload

from gpu_helpers import TOL, rel

pytestmark = pytest.mark.gpu


def _static_call(net, prob, db, params, loss, grad):
    from paper_2604_15645_gb300 import _lib
    _lib.pinn_loss_grad_static(net.h, prob, db.c_struct(), params.data_ptr(), loss.data_ptr(), grad.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("name,precision,n_res,n_bc", [("burgers1d_4x64", "fp32", 4096, 256),
                                                       ("ns_cavity_6x256", "bf16", 256, 64)])
def test_static_entry_matches_workspace_entry_twice(cuda_lib, name, precision, n_res, n_bc):
    from paper_2604_15645_gb300 import _lib, api
    w, p, B, b = make_workload(name, n_res=n_res, n_bc=n_bc, random_bias=0.1)
    net = api.PinnNet.from_spec(w.spec, precision)
    if B is not None:
        net.set_ff_matrix(B)
    db = api.DeviceBatch.from_host(b)
    assert net.workspace_bytes(*db.sizes) <= _lib.PINN_STATIC_WS_BYTES
    prob = api.make_problem(w.problem.nu, 1.0, 0.5, 2.0)
    for call, seed in enumerate((11, 12)):      # two calls in a row, different parameters
        params = torch.tensor(init_params(w.spec, seed, 0.1) if call else p, device="cuda")
        loss_s = torch.full((8,), np.nan, dtype=torch.float64, device="cuda")
        grad_s = torch.full_like(params, np.nan)
        _static_call(net, prob, db, params, loss_s, grad_s)
        loss_w, grad_w = net.loss_grad(params, db, prob, out=torch.empty_like(loss_s))
        torch.cuda.synchronize()
        assert net.status_poll() == 0
        ls, lw = loss_s.cpu().numpy(), loss_w.cpu().numpy()
        assert np.all(np.isfinite(ls)) and np.all(np.isfinite(grad_s.cpu().numpy()))
        for i in range(7):
            if lw[i] != 0:
                assert abs(ls[i] - lw[i]) <= TOL[precision] * abs(lw[i]), (call, i, ls[i], lw[i])
        assert rel(grad_s.cpu().numpy(), grad_w.cpu().numpy()) <= TOL[precision]


def test_static_entry_rejects_batches_beyond_its_array(cuda_lib):
    from paper_2604_15645_gb300 import _lib, api
    w, p, B, b = make_workload("ns_cavity_6x256")          # about 3 GB of workspace
    net = api.PinnNet.from_spec(w.spec, "bf16")
    net.set_ff_matrix(B)
    db = api.DeviceBatch.from_host(b)
    assert net.workspace_bytes(*db.sizes) > _lib.PINN_STATIC_WS_BYTES
    params = torch.tensor(p, device="cuda")
    loss = torch.zeros(8, dtype=torch.float64, device="cuda")
    grad = torch.zeros_like(params)
    with pytest.raises(_lib.PinnError) as e:
        _static_call(net, api.make_problem(w.problem.nu), db, params, loss, grad)
    assert e.value.status == 4 and "static array" in str(e.value)
    torch.cuda.synchronize()
    assert float(grad.abs().sum()) == 0.0      # nothing was queued


def test_static_entry_captures_no_graph(cuda_lib):
    from paper_2604_15645_gb300 import _lib, api
    w, p, B, b = make_workload("ns_cavity_6x256", n_res=300, n_bc=64, random_bias=0.1)
    net = api.PinnNet.from_spec(w.spec, "bf16")
    net.set_ff_matrix(B)
    net.set_graph(True)
    db = api.DeviceBatch.from_host(b)
    prob = api.make_problem(w.problem.nu)
    params = torch.tensor(p, device="cuda")
    loss_s = torch.zeros(8, dtype=torch.float64, device="cuda")
    grad_s = torch.zeros_like(params)
    _static_call(net, prob, db, params, loss_s, grad_s)
    torch.cuda.synchronize()
    assert not _lib.pinn_graph_held(net.h)          # graph mode on, yet nothing captured
    loss_w, grad_w = net.loss_grad(params, db, prob, out=torch.empty_like(loss_s))
    torch.cuda.synchronize()
    assert _lib.pinn_graph_held(net.h)              # the workspace entry point did capture
    _static_call(net, prob, db, params, loss_s, grad_s)
    torch.cuda.synchronize()
    assert _lib.pinn_graph_held(net.h) and net.status_poll() == 0
    assert rel(grad_s.cpu().numpy(), grad_w.cpu().numpy()) <= 1e-6
    assert rel(loss_s.cpu().numpy()[:7], loss_w.cpu().numpy()[:7]) <= 1e-12


def test_static_entry_survives_a_device_reset(cuda_lib, tmp_path):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    pkg = os.path.join(root, "paper_2604_15645_gb300")
    exe = str(tmp_path / "c_static_reset")
    subprocess.run([nvcc, "-O2", os.path.join(root, "tests", "c_static_reset.c"), "-I", os.path.join(root, "include"),
                    "-L", pkg, "-lpinn", "-Xlinker", "-rpath", "-Xlinker", pkg, "-o", exe], check=True, timeout=300)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
