"""A batch split into shards, each call normalised by the whole batch's point counts
(pinn_set_global_counts): the shard results sum to the whole-batch result."""
import numpy as np
import pytest
import torch

from synth import make_workload

from gpu_helpers import rel

pytestmark = pytest.mark.gpu


def _run(net, p, b, prob):
    from paper_2604_15645_gb300 import api
    t, g = net.loss_grad(p, api.DeviceBatch.from_host(b), prob)
    torch.cuda.synchronize()
    assert net.status_poll() == 0
    return t.cpu().numpy().copy(), g.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("name,precision", [("ns_cavity_6x256", "bf16"), ("burgers1d_4x64", "fp32"),
                                            ("maxwell_te_5x512", "bf16")])
def test_shards_sum_to_the_whole_batch(cuda_lib, name, precision):
    from paper_2604_15645_gb300 import api
    w, pp, B, b = make_workload(name, n_res=6000, n_ic=500, n_bc=700, random_bias=0.1)
    if w.spec.widths[0] > 256:
        w.spec.widths = [128] * 3
        from synth import init_params
        pp = init_params(w.spec, 5, 0.1)
    net = api.PinnNet.from_spec(w.spec, precision, value_split=w.value_split and precision == "bf16")
    if B is not None:
        net.set_ff_matrix(B)
    prob = api.make_problem(w.problem.nu, 1.0, 0.7, 1.3)
    p = torch.tensor(pp, device="cuda")
    t_full, g_full = _run(net, p, b, prob)

    net.set_global_counts(b.n_res, b.n_ic, b.n_bc)
    cuts = [(0, 2500, 0, 100, 0, 400), (2500, 6000, 100, 500, 400, 700)]   # uneven, ragged shards
    t_sum, g_sum = np.zeros_like(t_full), np.zeros_like(g_full)
    for r0, r1, i0, i1, c0, c1 in cuts:
        sb = type(b)(b.x_res[:, r0:r1].copy(), b.x_ic[:, i0:i1].copy(), b.g_ic[:, i0:i1].copy(), b.ic_mask,
                     b.x_bc[:, c0:c1].copy(), b.g_bc[:, c0:c1].copy(), b.bc_mask)
        t, g = _run(net, p, sb, prob)
        t_sum += t
        g_sum += g
    for i in range(7):
        if t_full[i] != 0:
            assert abs(t_sum[i] - t_full[i]) <= 1e-5 * abs(t_full[i]), (i, t_sum[i], t_full[i])
    assert rel(g_sum, g_full) <= 1e-5

    # a shard larger than the global counts is refused; switching off restores the batch's own means
    from paper_2604_15645_gb300 import _lib
    net.set_global_counts(100, 0, 0)
    with pytest.raises(_lib.PinnError):
        _run(net, p, b, prob)
    net.set_global_counts(0, 0, 0)
    t_again, _ = _run(net, p, b, prob)
    assert np.array_equal(t_again, t_full)
