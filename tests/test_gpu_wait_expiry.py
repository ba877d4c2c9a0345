"""Failure detection without a GPU fault: a bounded device-side wait that runs out.

Every mbarrier wait of the tensor-core kernels is bounded; when a bound expires the
kernel latches PINN_ERR_TIMEOUT in the handle's status word, stops its other warp
roles, waits (bounded) for its own copies in flight, frees its tensor memory and
returns.  pinn_debug_wait_expiry launches that same kernel with its MMA-issuing
thread first waiting on an mbarrier no thread arrives on, under a 1 ms bound.  The
host must then read PINN_ERR_TIMEOUT, and the context must stay usable: the same GEMM
without the stall and a whole loss + gradient evaluation still give correct results.
No trap, no device assert, no wait without a bound."""
import pytest
import torch

from synth import make_workload

from gpu_helpers import TOL, assert_parity, run_oracle

pytestmark = pytest.mark.gpu


def _tiles(X):
    R, C = X.shape
    return X.reshape(R, C // 256, 256).permute(1, 0, 2).contiguous()


def test_expired_wait_is_reported_and_the_context_stays_usable(cuda_lib):
    from paper_2604_15645_gb300 import _lib, api
    w, p, B, b = make_workload("ns_cavity_6x256", n_res=1000, n_bc=300, random_bias=0.1)
    net = api.PinnNet.from_spec(w.spec, "bf16")
    net.set_ff_matrix(B)
    stream = torch.cuda.current_stream().cuda_stream
    M, N, K = 128, 512, 64
    g = torch.Generator(device="cuda").manual_seed(7)
    A = torch.randn(M, K, device="cuda", generator=g).bfloat16()
    Bm = torch.randn(K, N, device="cuda", generator=g).bfloat16()
    Bt = _tiles(Bm)
    D = torch.zeros(N // 256, M, 256, device="cuda")
    assert net.status_poll() == 0
    for _ in range(2):                                 # twice: the status clears in between
        _lib.pinn_debug_wait_expiry(net.h, M, N, K, A.data_ptr(), Bt.data_ptr(), D.data_ptr(), 1000, stream)
        assert net.status_poll() == 6                  # PINN_ERR_TIMEOUT
        assert "bound" in _lib.load().pinn_last_error(net.h).decode()
        assert net.status_poll() == 0                  # read and cleared

    # the same kernel without the stall on the same context
    D2 = torch.full((N // 256, M, 256), float("nan"), device="cuda")
    _lib.pinn_tc_selftest(0, M, N, K, A.data_ptr(), None, Bt.data_ptr(), D2.data_ptr(), stream)
    ref = A.float() @ Bm.float()
    got = D2.permute(1, 0, 2).reshape(M, N)
    assert float((got - ref).norm() / ref.norm()) < 1e-5

    # and a whole loss + gradient evaluation on the tensor-core path against the oracle
    terms, grad = net.loss_grad(torch.tensor(p, device="cuda"), api.DeviceBatch.from_host(b),
                                api.make_problem(w.problem.nu, w.problem.lambda_pde, w.problem.lambda_ic,
                                                 w.problem.lambda_bc))
    torch.cuda.synchronize()
    assert net.status_poll() == 0
    rt, rg = run_oracle(w.spec, p, B, b, w.problem)
    assert_parity(terms.cpu().numpy(), grad.cpu().numpy().astype("float64"), rt, rg, TOL["bf16"],
                  "after an expired wait", spec=w.spec)


def test_wait_expiry_hook_refuses_bad_arguments(cuda_lib):
    from paper_2604_15645_gb300 import _lib, api
    w, p, B, b = make_workload("burgers1d_4x64", n_res=64)
    net = api.PinnNet.from_spec(w.spec, "bf16")
    x = torch.zeros(256 * 128, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for args in ((128, 256, 64, 0), (128, 256, 64, 3000000), (128, 100, 64, 1000), (12, 256, 64, 1000)):
        M, N, K, us = args
        with pytest.raises(_lib.PinnError) as e:
            _lib.pinn_debug_wait_expiry(net.h, M, N, K, x.data_ptr(), x.data_ptr(), x.data_ptr(), us, stream)
        assert e.value.status == 1
    assert net.status_poll() == 0
