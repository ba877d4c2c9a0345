"""PyTorch-facing wrapper of libpinn: device buffers and streams come from torch,
all computation from the library's kernels."""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib


def _ptr(t):
    return 0 if t is None else t.data_ptr()


def _stream():
    return torch.cuda.current_stream().cuda_stream


class DeviceBatch:
    """Collocation sets resident on the GPU (FP32, SoA [d][n])."""

    def __init__(self, x_res, x_ic, g_ic, ic_mask, x_bc, g_bc, bc_mask, device="cuda"):
        f = lambda a: torch.as_tensor(a, dtype=torch.float32, device=device).contiguous()
        self.x_res, self.x_ic, self.g_ic = f(x_res), f(x_ic), f(g_ic)
        self.x_bc, self.g_bc = f(x_bc), f(g_bc)
        self.ic_mask, self.bc_mask = int(ic_mask), int(bc_mask)

    @classmethod
    def from_host(cls, b, device="cuda"):
        return cls(b.x_res, b.x_ic, b.g_ic, b.ic_mask, b.x_bc, b.g_bc, b.bc_mask, device)

    @property
    def sizes(self):
        return self.x_res.shape[1], self.x_ic.shape[1], self.x_bc.shape[1]

    def c_struct(self) -> _lib.pinn_batch:
        s = _lib.pinn_batch()
        s.x_res, s.n_res = _ptr(self.x_res), self.x_res.shape[1]
        s.x_ic, s.g_ic, s.n_ic, s.ic_mask = _ptr(self.x_ic), _ptr(self.g_ic), self.x_ic.shape[1], self.ic_mask
        s.x_bc, s.g_bc, s.n_bc, s.bc_mask = _ptr(self.x_bc), _ptr(self.g_bc), self.x_bc.shape[1], self.bc_mask
        return s


def make_problem(nu, lambda_pde=1.0, lambda_ic=1.0, lambda_bc=1.0) -> _lib.pinn_problem:
    p = _lib.pinn_problem()
    p.nu, p.lambda_pde, p.lambda_ic, p.lambda_bc = float(nu), float(lambda_pde), float(lambda_ic), float(lambda_bc)
    return p


class PinnNet:
    """One network handle (pinn_create) plus a cached workspace."""

    def __init__(self, pde, widths, ff_m=0, rwf=False, precision="fp32", device="cuda", chunk_points=0,
                 value_split=False, activation="tanh", omega0=1.0):
        self.device = torch.device(device)
        self.precision = precision
        flags = _lib.PINN_FLAG_BF16_VALUE_SPLIT if value_split else 0
        with torch.cuda.device(self.device):
            self.spec = _lib.make_spec(pde, widths, ff_m, rwf, _lib.PRECISIONS[precision], flags)
            self.h = _lib.pinn_create(self.spec)
        self.P = _lib.pinn_param_count(self.h)
        if chunk_points:
            _lib.pinn_set_chunk_points(self.h, chunk_points)
        if activation != "tanh":
            self.set_activation(activation, omega0)
        self._B = None
        self._periodic = False
        self._ws = None
        self._ws_key = None
        self.loss_buf = torch.zeros(_lib.PINN_LOSS_TERMS, dtype=torch.float64, device=self.device)

    @classmethod
    def from_spec(cls, spec, precision="fp32", device="cuda", chunk_points=0, value_split=False):
        return cls(spec.pde, spec.widths, spec.ff_m, spec.rwf, precision, device, chunk_points, value_split,
                   getattr(spec, "activation", "tanh"), getattr(spec, "omega0", 1.0))

    def set_global_counts(self, n_res=0, n_ic=0, n_bc=0):
        """Normalise the means by the whole batch's counts (this net sees one shard of it)."""
        _lib.pinn_set_global_counts(self.h, n_res, n_ic, n_bc)

    def set_graph(self, on=True):
        """Replay each call from a captured CUDA graph while its arguments stay the same."""
        _lib.pinn_set_graph(self.h, on)

    def set_activation(self, activation, omega0=1.0):
        """Hidden activation: "tanh" or "sine" (sin(omega0 z), CUDA-core jet GEMMs)."""
        act = {"tanh": _lib.PINN_ACT_TANH, "sine": _lib.PINN_ACT_SINE}[activation]
        _lib.pinn_set_activation(self.h, act, omega0)
        self._ws_key = None

    def set_chunk_points(self, points):
        """Process batches in chunks of at most `points` points (0: one pass)."""
        _lib.pinn_set_chunk_points(self.h, points)
        self._ws_key = None

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            try:
                _lib.pinn_destroy(h)
            except Exception:
                pass
            self.h = None

    def set_ff_matrix(self, B):
        self._B = torch.as_tensor(B, dtype=torch.float32, device=self.device).contiguous()
        _lib.pinn_set_ff_matrix(self.h, self._B.data_ptr())
        self._periodic = False

    def workspace_bytes(self, n_res, n_ic, n_bc):
        return _lib.pinn_workspace_bytes(self.h, n_res, n_ic, n_bc)

    def workspace(self, batch: DeviceBatch):
        key = batch.sizes
        if self._ws_key != key:
            nbytes = self.workspace_bytes(*key)
            self._ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
            self._ws_key = key
        return self._ws

    def loss(self, params, batch: DeviceBatch, problem, out=None):
        ws = self.workspace(batch)
        out = self.loss_buf if out is None else out
        _lib.pinn_loss(self.h, problem, batch.c_struct(), params.data_ptr(), ws.data_ptr(), ws.numel(),
                       out.data_ptr(), _stream())
        return out

    def loss_grad(self, params, batch: DeviceBatch, problem, grad=None, out=None):
        assert params.dtype == torch.float32 and params.is_contiguous() and params.numel() == self.P
        ws = self.workspace(batch)
        out = self.loss_buf if out is None else out
        grad = torch.empty_like(params) if grad is None else grad
        _lib.pinn_loss_grad(self.h, problem, batch.c_struct(), params.data_ptr(), ws.data_ptr(), ws.numel(),
                            out.data_ptr(), grad.data_ptr(), _stream())
        return out, grad

    def set_periodic(self, periods):
        """Strict periodic input map (Eq. 16) with these periods [d_in]; needs ff_m = d_in."""
        _lib.pinn_set_periodic(self.h, list(periods))
        self._B = None
        self._periodic = True

    def loss_grad_ff(self, params, batch: DeviceBatch, problem, grad=None, grad_ff=None, out=None):
        """Loss, dL/dparams and the input-map gradient: dL/dB [d_in][m] with a Fourier
        matrix, dL/dP [d_in] with the periodic map."""
        assert params.dtype == torch.float32 and params.is_contiguous() and params.numel() == self.P
        ws = self.workspace(batch)
        out = self.loss_buf if out is None else out
        grad = torch.empty_like(params) if grad is None else grad
        if grad_ff is None:
            d_in = 3 if self.spec.pde == _lib.PINN_MAXWELL_TE_2D else 2
            n = d_in if self._periodic else d_in * self.spec.ff_m
            grad_ff = torch.empty(n, dtype=torch.float32, device=self.device)
        _lib.pinn_loss_grad_ff(self.h, problem, batch.c_struct(), params.data_ptr(), ws.data_ptr(), ws.numel(),
                               out.data_ptr(), grad.data_ptr(), grad_ff.data_ptr(), _stream())
        return out, grad, grad_ff

    def loss_grad_terms(self, params, batch: DeviceBatch, problem, grads=None, out=None):
        """Loss and the unweighted gradients of the PDE, initial and boundary terms,
        [3][P] (Sec. 2.6.4): one forward sweep, three reverse sweeps."""
        assert params.dtype == torch.float32 and params.is_contiguous() and params.numel() == self.P
        ws = self.workspace(batch)
        out = self.loss_buf if out is None else out
        grads = torch.empty(3, self.P, dtype=torch.float32, device=self.device) if grads is None else grads
        _lib.pinn_loss_grad_terms(self.h, problem, batch.c_struct(), params.data_ptr(), ws.data_ptr(), ws.numel(),
                                  out.data_ptr(), grads.data_ptr(), _stream())
        return out, grads

    def loss_balance(self, grads, lambdas, norms=None, alpha=0.9, eps=1e-9, update=True):
        """Loss-balancing weights (Sec. 2.6.4, Eqs. 18-19) from loss_grad_terms' gradients;
        `lambdas` is an FP64 device tensor [3] (pde, ic, bc), updated in place."""
        assert lambdas.dtype == torch.float64 and lambdas.numel() == 3
        _lib.pinn_loss_balance(self.h, grads.data_ptr(), lambdas.data_ptr(),
                               norms.data_ptr() if norms is not None else None, alpha, eps, update, _stream())
        return lambdas

    def set_causal(self, segments, eps, t0=0.0, t1=1.0):
        """Temporal causality (Sec. 2.6.8): `segments` time segments over [t0, t1]
        (0 switches it off), decay `eps`."""
        _lib.pinn_set_causal(self.h, segments, eps, t0, t1)
        self._ws_key = None
        self.causal_segments = segments

    def causal_weights(self):
        """The segment weights omega_i of the last call, FP64 device tensor."""
        w = torch.empty(self.causal_segments, dtype=torch.float64, device=self.device)
        _lib.pinn_causal_weights(self.h, w.data_ptr(), _stream())
        return w

    def layer_engines(self, n_res, n_ic, n_bc):
        """Per hidden layer: 0 CUDA cores, 1 tensor cores, 2 tensor cores with the fused
        adjoint + weight-gradient kernel."""
        return _lib.pinn_layer_engines(self.h, self.spec.n_hidden, n_res, n_ic, n_bc)

    def tensor_core_layers(self, n_res, n_ic, n_bc):
        return _lib.pinn_tensor_core_layers(self.h, n_res, n_ic, n_bc)

    def status_poll(self):
        return _lib.pinn_status_poll(self.h, _stream())


def adam_step(params, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    _lib.pinn_adam_step(params.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(), params.numel(), step,
                        lr, beta1, beta2, eps, _stream())


class PinnLoss(torch.autograd.Function):
    """torch.autograd.Function whose backward is the library's hand-written adjoint
    (computed together with the loss), replacing double-backward autograd."""

    @staticmethod
    def forward(ctx, params, net, batch, problem):
        terms, grad = net.loss_grad(params, batch, problem, out=torch.empty_like(net.loss_buf))
        ctx.save_for_backward(grad)
        return terms[0].clone()

    @staticmethod
    def backward(ctx, gout):
        (grad,) = ctx.saved_tensors
        return grad * gout.to(grad.dtype), None, None, None


class PinnMulti:
    """Many independent networks, one graph-captured training step (pinn_multi_*)."""

    def __init__(self, specs, precision="bf16", device="cuda"):
        self.device = torch.device(device)
        self.n = len(specs)
        arr = (_lib.pinn_spec * self.n)(*[_lib.make_spec(s.pde, s.widths, s.ff_m, s.rwf, _lib.PRECISIONS[precision])
                                          for s in specs])
        h = _lib.C.c_void_p()
        with torch.cuda.device(self.device):
            _lib.check(_lib.load().pinn_multi_create(arr, self.n, _lib.C.byref(h)))
        self.h = h.value
        off = (_lib.C.c_int64 * (self.n + 1))()
        _lib.check_multi(_lib.load().pinn_multi_param_offsets(self.h, off), self.h)
        self.offsets = list(off)
        self.P = self.offsets[-1]
        self._ws = None
        self._keep = None

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            try:
                _lib.load().pinn_multi_destroy(h)
            except Exception:
                pass
            self.h = None

    def set_inputs(self, batches, problems):
        """batches: DeviceBatch per network; problems: pinn_problem per network."""
        self._batches = list(batches)
        self._cb = (_lib.pinn_batch * self.n)(*[b.c_struct() for b in batches])
        self._cp = (_lib.pinn_problem * self.n)(*problems)
        nbytes = _lib.C.c_size_t()
        _lib.check_multi(_lib.load().pinn_multi_workspace_bytes(self.h, self._cb, _lib.C.byref(nbytes)), self.h)
        if self._ws is None or self._ws.numel() < nbytes.value:
            self._ws = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=self.device)
        self.loss = torch.zeros(self.n, _lib.PINN_LOSS_TERMS, dtype=torch.float64, device=self.device)

    def engines(self):
        out = []
        for i in range(self.n):
            v = _lib.C.c_int32()
            _lib.check_multi(_lib.load().pinn_multi_get_engine(self.h, i, _lib.C.byref(v)), self.h)
            out.append("cuda_cores" if v.value else "tc")
        return out

    CONFIGS = ("tc", "cuda_cores", "tc_unfused", "tc_unfused_dw128")

    def configs(self):
        """Kernel configuration of every network (one of CONFIGS)."""
        out = []
        for i in range(self.n):
            v = _lib.C.c_int32()
            _lib.check_multi(_lib.load().pinn_multi_get_config(self.h, i, _lib.C.byref(v)), self.h)
            out.append(self.CONFIGS[v.value])
        return out

    def set_config(self, i, config):
        _lib.check_multi(_lib.load().pinn_multi_set_config(self.h, i, self.CONFIGS.index(config)), self.h)

    @property
    def grouped(self):
        """True: one grouped tcgen05 launch per layer level over all networks; False
        (the default): each network's launches on its own worker stream."""
        v = _lib.C.c_int32()
        _lib.check_multi(_lib.load().pinn_multi_get_grouped(self.h, _lib.C.byref(v)), self.h)
        return bool(v.value)

    @grouped.setter
    def grouped(self, on):
        _lib.check_multi(_lib.load().pinn_multi_set_grouped(self.h, int(bool(on))), self.h)

    def set_engine(self, i, cuda_cores):
        _lib.check_multi(_lib.load().pinn_multi_set_engine(self.h, i, int(bool(cuda_cores))), self.h)

    def autotune(self, params, grad, cache_path=None):
        path = cache_path.encode() if cache_path else None
        _lib.check_multi(_lib.load().pinn_multi_autotune(
            self.h, self._cp, self._cb, params.data_ptr(), self._ws.data_ptr(), self._ws.numel(),
            self.loss.data_ptr(), grad.data_ptr(), path, _stream()), self.h)

    def train_step(self, params, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        _lib.check_multi(_lib.load().pinn_multi_train_step(
            self.h, self._cp, self._cb, params.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(), step,
            lr, beta1, beta2, eps, self._ws.data_ptr(), self._ws.numel(), self.loss.data_ptr(), _stream()), self.h)
        return self.loss

    def status_poll(self):
        return _lib.load().pinn_multi_status_poll(self.h, _stream())


class Lbfgs:
    """L-BFGS refinement (Sec. 2.6.5) over a PinnNet's loss and gradient: the history,
    the two-loop direction and the backtracking line search run in the library."""

    def __init__(self, net: PinnNet, history=10):
        self.net = net
        h = C.c_void_p()
        _lib.check(_lib.load().pinn_lbfgs_create(net.h, history, C.byref(h)), net.h)
        self.lb = h.value

    def __del__(self):
        lb = getattr(self, "lb", None)
        if lb:
            try:
                _lib.load().pinn_lbfgs_destroy(lb)
            except Exception:
                pass
            self.lb = None

    def reset(self):
        _lib.check(_lib.load().pinn_lbfgs_reset(self.lb))

    def step(self, params, batch: DeviceBatch, problem):
        """One L-BFGS step in place on params; returns (loss, line-search halvings)."""
        ws = self.net.workspace(batch)
        loss, bt = C.c_double(), C.c_int()
        _lib.check(_lib.load().pinn_lbfgs_step(self.lb, C.byref(problem), C.byref(batch.c_struct()), params.data_ptr(),
                                               ws.data_ptr(), ws.numel(), C.byref(loss), C.byref(bt), _stream()),
                   self.net.h)
        return loss.value, bt.value

    def direction(self, g, p):
        _lib.check(_lib.load().pinn_lbfgs_direction(self.lb, g.data_ptr(), p.data_ptr(), _stream()))

    def push_pair(self, s, y):
        _lib.check(_lib.load().pinn_lbfgs_push_pair(self.lb, s.data_ptr(), y.data_ptr(), _stream()))
