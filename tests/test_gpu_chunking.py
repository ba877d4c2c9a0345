"""Point chunking (bounded memory at the largest sizes): chunked calls against the
FP64 oracle and against the one-pass call on the same inputs."""
import numpy as np
import pytest
import torch

from synth import make_workload

from gpu_helpers import TOL, assert_parity, rel, run_oracle

pytestmark = pytest.mark.gpu


def _run(w, p, B, b, precision, chunk=0, want_grad=True):
    from paper_2604_15645_gb300 import api
    net = api.PinnNet.from_spec(w.spec, precision, chunk_points=chunk)
    if B is not None:
        net.set_ff_matrix(B)
    db = api.DeviceBatch.from_host(b)
    prob = api.make_problem(w.problem.nu, w.problem.lambda_pde, w.problem.lambda_ic, w.problem.lambda_bc)
    params = torch.tensor(p, device="cuda")
    nbytes = net.workspace_bytes(*db.sizes)
    if want_grad:
        t, g = net.loss_grad(params, db, prob)
        out = t.cpu().numpy().copy(), g.cpu().numpy().astype(np.float64)
    else:
        out = net.loss(params, db, prob).cpu().numpy().copy(), None
    torch.cuda.synchronize()
    assert net.status_poll() == 0
    return out, nbytes


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_chunked_cavity_matches_oracle_and_one_pass(cuda_lib, precision):
    # 1000 interior + 300 wall points in chunks of 256: one chunk straddles both sets
    w, p, B, b = make_workload("ns_cavity_6x256", n_res=1000, n_bc=300, random_bias=0.1)
    (t1, g1), _ = _run(w, p, B, b, precision)
    (tc, gc), _ = _run(w, p, B, b, precision, chunk=256)
    rt, rg = run_oracle(w.spec, p, B, b, w.problem)
    assert_parity(tc, gc, rt, rg, TOL[precision], f"chunked cavity {precision}", spec=w.spec)
    assert rel(tc[:7], t1[:7]) < 1e-6 and rel(gc, g1) < 1e-6


def test_chunked_maxwell_sets_straddle_chunks(cuda_lib):
    # chunks of 192 over 600 interior + 100 initial + 150 boundary points: chunks hold
    # interior+initial and initial+boundary mixes; all three terms and masks active
    w, p, B, b = make_workload("maxwell_te_5x512", n_res=600, n_ic=100, n_bc=150, random_bias=0.1)
    (tc, gc), _ = _run(w, p, B, b, "fp32", chunk=192)
    rt, rg = run_oracle(w.spec, p, B, b, w.problem)
    assert_parity(tc, gc, rt, rg, TOL["fp32"], "chunked maxwell", spec=w.spec)


def test_chunked_loss_only(cuda_lib):
    w, p, B, b = make_workload("burgers1d_4x64", random_bias=0.1)
    (tl, _), _ = _run(w, p, B, b, "fp32", chunk=1000, want_grad=False)
    rt, rg = run_oracle(w.spec, p, B, b, w.problem)
    for i in range(7):
        if rt[i]:
            assert abs(tl[i] - rt[i]) <= TOL["fp32"] * abs(rt[i])


def test_chunking_bounds_memory_at_scale(cuda_lib):
    # the 8x512 network on 65,536 + 1,024 points: chunks of 8,192 points need a
    # fraction of the one-pass workspace and give the same result (same per-point
    # arithmetic; only the order of the cross-chunk sums differs)
    w, p, B, b = make_workload("ns_cavity_8x512", n_res=65536, n_bc=1024)
    (t1, g1), n_full = _run(w, p, B, b, "bf16")
    (tb, gb), n_small = _run(w, p, B, b, "bf16", chunk=8192)
    assert n_small * 4 < n_full
    assert rel(tb[:7], t1[:7]) < 1e-5 and rel(gb, g1) < 1e-4
