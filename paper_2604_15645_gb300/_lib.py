"""ctypes binding of libpinn.so (include/pinn.h).  Argument marshalling only:
every step of the computation runs in the library's CUDA kernels.  The library
must have been built (``python -m paper_2604_15645_gb300._build`` or
``__graft_entry__.build()``); there is no fallback when it is missing."""
from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libpinn.so")

PINN_MAX_HIDDEN = 16
PINN_LOSS_TERMS = 8
PINN_FP32, PINN_TF32, PINN_BF16 = 0, 1, 2
PINN_BURGERS_1D, PINN_NS_STEADY_2D, PINN_MAXWELL_TE_2D, PINN_ADVECTION_1D, PINN_ALLEN_CAHN_1D = 0, 1, 2, 3, 4
PINN_FLAG_CUDA_CORES, PINN_FLAG_BF16_VALUE_SPLIT = 1, 4
PINN_FLAG_UNFUSED_ADJOINT, PINN_FLAG_DW_ROWS_128 = 8, 16
PRECISIONS = {"fp32": PINN_FP32, "tf32": PINN_TF32, "bf16": PINN_BF16}
STATUS = {0: "PINN_OK", 1: "PINN_ERR_INVALID_ARG", 2: "PINN_ERR_UNSUPPORTED", 3: "PINN_ERR_CUDA",
          4: "PINN_ERR_WORKSPACE", 5: "PINN_ERR_NONFINITE", 6: "PINN_ERR_TIMEOUT", 7: "PINN_ERR_OOM"}

# Every symbol declared in include/pinn.h (checked by the CPU tests).
EXPORTS = ["pinn_create", "pinn_destroy", "pinn_param_count", "pinn_workspace_bytes", "pinn_set_ff_matrix",
           "pinn_loss", "pinn_loss_grad", "pinn_adam_step", "pinn_status_poll", "pinn_last_error",
           "pinn_status_string", "pinn_version", "pinn_set_profiling", "pinn_profile_read", "pinn_tensor_core_layers", "pinn_tc_selftest",
           "pinn_loss_grad_static", "pinn_tanh_selftest", "pinn_multi_create", "pinn_multi_destroy",
           "pinn_multi_param_offsets", "pinn_multi_workspace_bytes", "pinn_multi_set_ff_matrix",
           "pinn_multi_set_engine", "pinn_multi_get_engine", "pinn_multi_train_step", "pinn_multi_autotune",
           "pinn_multi_status_poll", "pinn_multi_last_error", "pinn_set_chunk_points",
           "pinn_loss_grad_terms", "pinn_loss_balance", "pinn_set_causal", "pinn_causal_weights",
           "pinn_lbfgs_create", "pinn_lbfgs_destroy", "pinn_lbfgs_reset", "pinn_lbfgs_step", "pinn_lbfgs_direction",
           "pinn_lbfgs_push_pair", "pinn_set_activation", "pinn_set_periodic", "pinn_loss_grad_ff",
           "pinn_set_graph", "pinn_set_global_counts", "pinn_graph_held", "pinn_debug_wait_expiry",
           "pinn_layer_engines", "pinn_multi_set_config", "pinn_multi_get_config", "pinn_multi_set_grouped",
           "pinn_multi_get_grouped"]
PINN_ACT_TANH, PINN_ACT_SINE = 0, 1
PINN_STATIC_WS_BYTES = 64 << 20
PINN_PROF_PHASES = 9
PHASE_NAMES = ["rwf", "embed", "fwd_gemm", "out_loss", "dw_gemm", "adj_gemm", "reduce", "other", "adjdw_gemm"]


class pinn_spec(C.Structure):
    _fields_ = [("pde", C.c_int32), ("n_hidden", C.c_int32), ("widths", C.c_int32 * PINN_MAX_HIDDEN),
                ("ff_m", C.c_int32), ("rwf", C.c_int32), ("precision", C.c_int32), ("flags", C.c_int32)]


class pinn_problem(C.Structure):
    _fields_ = [("nu", C.c_double), ("lambda_pde", C.c_double), ("lambda_ic", C.c_double),
                ("lambda_bc", C.c_double)]


class pinn_batch(C.Structure):
    _fields_ = [("x_res", C.c_void_p), ("n_res", C.c_int64),
                ("x_ic", C.c_void_p), ("g_ic", C.c_void_p), ("n_ic", C.c_int64), ("ic_mask", C.c_uint32),
                ("x_bc", C.c_void_p), ("g_bc", C.c_void_p), ("n_bc", C.c_int64), ("bc_mask", C.c_uint32)]


class PinnError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load libpinn.so and declare the C signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libpinn.so not built at {path}; run __graft_entry__.build() first")
    lib = C.CDLL(path)
    H = C.c_void_p
    lib.pinn_create.argtypes = [C.POINTER(pinn_spec), C.POINTER(H)]
    lib.pinn_destroy.argtypes = [H]
    lib.pinn_param_count.argtypes = [H, C.POINTER(C.c_int64)]
    lib.pinn_workspace_bytes.argtypes = [H, C.c_int64, C.c_int64, C.c_int64, C.POINTER(C.c_size_t)]
    lib.pinn_set_ff_matrix.argtypes = [H, C.c_void_p]
    lib.pinn_loss.argtypes = [H, C.POINTER(pinn_problem), C.POINTER(pinn_batch), C.c_void_p, C.c_void_p,
                              C.c_size_t, C.c_void_p, C.c_void_p]
    lib.pinn_loss_grad.argtypes = [H, C.POINTER(pinn_problem), C.POINTER(pinn_batch), C.c_void_p, C.c_void_p,
                                   C.c_size_t, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.pinn_adam_step.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64,
                                   C.c_float, C.c_float, C.c_float, C.c_float, C.c_void_p]
    lib.pinn_status_poll.argtypes = [H, C.c_void_p]
    lib.pinn_last_error.argtypes = [H]
    lib.pinn_last_error.restype = C.c_char_p
    lib.pinn_status_string.argtypes = [C.c_int]
    lib.pinn_status_string.restype = C.c_char_p
    lib.pinn_version.restype = C.c_char_p
    lib.pinn_set_profiling.argtypes = [H, C.c_int]
    lib.pinn_multi_create.argtypes = [C.POINTER(pinn_spec), C.c_int32, C.POINTER(H)]
    lib.pinn_multi_destroy.argtypes = [H]
    lib.pinn_multi_param_offsets.argtypes = [H, C.POINTER(C.c_int64)]
    lib.pinn_multi_workspace_bytes.argtypes = [H, C.POINTER(pinn_batch), C.POINTER(C.c_size_t)]
    lib.pinn_multi_set_ff_matrix.argtypes = [H, C.c_int32, C.c_void_p]
    lib.pinn_multi_set_engine.argtypes = [H, C.c_int32, C.c_int32]
    lib.pinn_multi_get_engine.argtypes = [H, C.c_int32, C.POINTER(C.c_int32)]
    lib.pinn_multi_set_config.argtypes = [H, C.c_int32, C.c_int32]
    lib.pinn_multi_get_config.argtypes = [H, C.c_int32, C.POINTER(C.c_int32)]
    lib.pinn_multi_set_grouped.argtypes = [H, C.c_int32]
    lib.pinn_multi_get_grouped.argtypes = [H, C.POINTER(C.c_int32)]
    lib.pinn_multi_train_step.argtypes = [H, C.POINTER(pinn_problem), C.POINTER(pinn_batch), C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.c_int64, C.c_float, C.c_float, C.c_float,
                                          C.c_float, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p]
    lib.pinn_multi_autotune.argtypes = [H, C.POINTER(pinn_problem), C.POINTER(pinn_batch), C.c_void_p, C.c_void_p,
                                        C.c_size_t, C.c_void_p, C.c_void_p, C.c_char_p, C.c_void_p]
    lib.pinn_multi_status_poll.argtypes = [H, C.c_void_p]
    lib.pinn_multi_last_error.argtypes = [H]
    lib.pinn_multi_last_error.restype = C.c_char_p
    lib.pinn_tanh_selftest.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.pinn_loss_grad_static.argtypes = [H, C.POINTER(pinn_problem), C.POINTER(pinn_batch), C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.c_void_p]
    lib.pinn_tc_selftest.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_void_p]
    lib.pinn_tensor_core_layers.argtypes = [H, C.c_int64, C.c_int64, C.c_int64, C.POINTER(C.c_int32)]
    lib.pinn_layer_engines.argtypes = [H, C.c_int64, C.c_int64, C.c_int64, C.POINTER(C.c_int32)]
    lib.pinn_profile_read.argtypes = [H, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
    lib.pinn_set_chunk_points.argtypes = [H, C.c_int64]
    lib.pinn_set_activation.argtypes = [H, C.c_int, C.c_double]
    lib.pinn_set_graph.argtypes = [H, C.c_int]
    lib.pinn_graph_held.argtypes = [H, C.POINTER(C.c_int32)]
    lib.pinn_debug_wait_expiry.argtypes = [H, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.c_int64, C.c_void_p]
    lib.pinn_set_global_counts.argtypes = [H, C.c_int64, C.c_int64, C.c_int64]
    lib.pinn_set_periodic.argtypes = [H, C.POINTER(C.c_double)]
    lib.pinn_loss_grad_ff.argtypes = [H, C.POINTER(pinn_problem), C.POINTER(pinn_batch), C.c_void_p, C.c_void_p,
                                      C.c_size_t, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.pinn_set_causal.argtypes = [H, C.c_int, C.c_double, C.c_double, C.c_double]
    lib.pinn_causal_weights.argtypes = [H, C.c_void_p, C.c_void_p]
    lib.pinn_lbfgs_create.argtypes = [H, C.c_int, C.POINTER(C.c_void_p)]
    lib.pinn_lbfgs_destroy.argtypes = [C.c_void_p]
    lib.pinn_lbfgs_reset.argtypes = [C.c_void_p]
    lib.pinn_lbfgs_step.argtypes = [C.c_void_p, C.POINTER(pinn_problem), C.POINTER(pinn_batch), C.c_void_p,
                                    C.c_void_p, C.c_size_t, C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_void_p]
    lib.pinn_lbfgs_direction.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.pinn_lbfgs_push_pair.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.pinn_loss_grad_terms.argtypes = [H, C.POINTER(pinn_problem), C.POINTER(pinn_batch), C.c_void_p, C.c_void_p,
                                         C.c_size_t, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.pinn_loss_balance.argtypes = [H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_int,
                                      C.c_void_p]
    for name in EXPORTS:
        if name not in ("pinn_last_error", "pinn_status_string", "pinn_version", "pinn_multi_last_error"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def check(status: int, handle=None):
    if status != 0:
        msg = load().pinn_last_error(handle).decode() if handle else ""
        raise PinnError(status, msg)


def make_spec(pde: int, widths, ff_m: int = 0, rwf: bool = False, precision: int = PINN_FP32,
              flags: int = 0) -> pinn_spec:
    s = pinn_spec()
    s.pde = pde
    s.n_hidden = len(widths)
    for i, w in enumerate(widths):
        s.widths[i] = int(w)
    s.ff_m = ff_m
    s.rwf = int(bool(rwf))
    s.precision = precision
    s.flags = flags
    return s


# ---- thin wrappers with the C names ---------------------------------------------------

def pinn_create(spec: pinn_spec) -> int:
    h = C.c_void_p()
    check(load().pinn_create(C.byref(spec), C.byref(h)))
    return h.value


def pinn_destroy(h: int):
    check(load().pinn_destroy(h))


def pinn_param_count(h: int) -> int:
    P = C.c_int64()
    check(load().pinn_param_count(h, C.byref(P)), h)
    return P.value


def pinn_workspace_bytes(h: int, n_res: int, n_ic: int, n_bc: int) -> int:
    b = C.c_size_t()
    check(load().pinn_workspace_bytes(h, n_res, n_ic, n_bc, C.byref(b)), h)
    return b.value


def pinn_loss_grad_terms(h, prob, batch, d_params, d_ws, ws_bytes, d_loss, d_grad_terms, stream):
    check(load().pinn_loss_grad_terms(h, C.byref(prob), C.byref(batch), d_params, d_ws, ws_bytes, d_loss,
                                      d_grad_terms, stream), h)


def pinn_loss_balance(h, d_grad_terms, d_lambda, d_norms, alpha, eps, update, stream):
    check(load().pinn_loss_balance(h, d_grad_terms, d_lambda, d_norms, alpha, eps, int(update), stream), h)


def pinn_set_causal(h, segments, eps, t0, t1):
    check(load().pinn_set_causal(h, segments, eps, t0, t1), h)


def pinn_causal_weights(h, d_weights, stream):
    check(load().pinn_causal_weights(h, d_weights, stream), h)


def pinn_set_chunk_points(h: int, points: int):
    check(load().pinn_set_chunk_points(h, points), h)


def pinn_set_global_counts(h: int, n_res: int, n_ic: int, n_bc: int):
    check(load().pinn_set_global_counts(h, n_res, n_ic, n_bc), h)


def pinn_set_graph(h: int, on: bool):
    check(load().pinn_set_graph(h, 1 if on else 0), h)


def pinn_graph_held(h: int) -> bool:
    held = C.c_int32()
    check(load().pinn_graph_held(h, C.byref(held)), h)
    return bool(held.value)


def pinn_debug_wait_expiry(h, M, N, K, d_A, d_B, d_D, wait_us, stream):
    check(load().pinn_debug_wait_expiry(h, M, N, K, d_A, d_B, d_D, wait_us, stream), h)


def pinn_set_activation(h: int, act: int, omega0: float):
    check(load().pinn_set_activation(h, act, omega0), h)


def pinn_set_ff_matrix(h: int, d_B: int):
    check(load().pinn_set_ff_matrix(h, d_B), h)


def pinn_loss(h, prob, batch, d_params, d_ws, ws_bytes, d_loss, stream):
    check(load().pinn_loss(h, C.byref(prob), C.byref(batch), d_params, d_ws, ws_bytes, d_loss, stream), h)


def pinn_loss_grad(h, prob, batch, d_params, d_ws, ws_bytes, d_loss, d_grad, stream):
    check(load().pinn_loss_grad(h, C.byref(prob), C.byref(batch), d_params, d_ws, ws_bytes, d_loss, d_grad,
                                stream), h)


def pinn_loss_grad_ff(h, prob, batch, d_params, d_ws, ws_bytes, d_loss, d_grad, d_grad_ff, stream):
    check(load().pinn_loss_grad_ff(h, C.byref(prob), C.byref(batch), d_params, d_ws, ws_bytes, d_loss, d_grad,
                                   d_grad_ff, stream), h)


def pinn_set_periodic(h, periods):
    arr = (C.c_double * len(periods))(*[float(x) for x in periods])
    check(load().pinn_set_periodic(h, arr), h)


def pinn_adam_step(d_params, d_grad, d_m, d_v, n, step, lr, beta1, beta2, eps, stream):
    check(load().pinn_adam_step(d_params, d_grad, d_m, d_v, n, step, lr, beta1, beta2, eps, stream))


def pinn_status_poll(h, stream) -> int:
    return load().pinn_status_poll(h, stream)


def pinn_version() -> str:
    return load().pinn_version().decode()


def pinn_set_profiling(h, enable: bool):
    check(load().pinn_set_profiling(h, int(enable)), h)


def pinn_profile_read(h):
    """{phase name: (ms, launches)} since the last read."""
    ms = (C.c_double * PINN_PROF_PHASES)()
    n = (C.c_int64 * PINN_PROF_PHASES)()
    check(load().pinn_profile_read(h, ms, n), h)
    return {PHASE_NAMES[i]: (ms[i], n[i]) for i in range(PINN_PROF_PHASES)}


def pinn_tensor_core_layers(h, n_res, n_ic, n_bc) -> int:
    n = C.c_int32()
    check(load().pinn_tensor_core_layers(h, n_res, n_ic, n_bc, C.byref(n)), h)
    return n.value


def pinn_layer_engines(h, n_hidden, n_res, n_ic, n_bc):
    """Per hidden layer: 0 CUDA cores, 1 tensor cores, 2 tensor cores with the fused
    adjoint + weight-gradient kernel."""
    out = (C.c_int32 * n_hidden)()
    check(load().pinn_layer_engines(h, n_res, n_ic, n_bc, out), h)
    return list(out)


def pinn_tc_selftest(kind, M, N, K, d_A, d_A2, d_B, d_D, stream):
    check(load().pinn_tc_selftest(kind, M, N, K, d_A, d_A2, d_B, d_D, stream))


def pinn_loss_grad_static(h, prob, batch, d_params, d_loss, d_grad, stream):
    check(load().pinn_loss_grad_static(h, C.byref(prob), C.byref(batch), d_params, d_loss, d_grad, stream), h)


def pinn_tanh_selftest(n, d_z, d_t, d_tp, stream):
    check(load().pinn_tanh_selftest(n, d_z, d_t, d_tp, stream))


def check_multi(status: int, m):
    if status != 0:
        raise PinnError(status, load().pinn_multi_last_error(m).decode() if m else "")
