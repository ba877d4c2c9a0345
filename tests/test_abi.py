"""The C-ABI library builds, loads and exports every symbol include/pinn.h declares,
and rejects bad specs on the host (CPU only: no compute calls)."""
import ctypes as C
import os
import re

import pytest

from paper_2604_15645_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pinn.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2604_15645_gb300 import _build
        _build.build()
    return _lib.load()


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"PINN_API[^;]*?\b(pinn_[a-z0-9_]+)\s*\(", text, flags=re.S)))


def test_header_declares_the_abi():
    syms = declared_symbols()
    for name in ["pinn_create", "pinn_destroy", "pinn_loss", "pinn_loss_grad", "pinn_adam_step",
                 "pinn_workspace_bytes", "pinn_param_count", "pinn_set_ff_matrix", "pinn_status_poll"]:
        assert name in syms
    assert sorted(_lib.EXPORTS) == syms


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_strings(lib):
    assert lib.pinn_version().decode().startswith("pinn-gb300")
    assert lib.pinn_status_string(0).decode() == "PINN_OK"
    assert lib.pinn_status_string(4).decode() == "PINN_ERR_WORKSPACE"


def test_struct_layout_matches_header():
    # pinn_spec: 6 int32 + 16 widths; pinn_batch has natural alignment padding.
    assert C.sizeof(_lib.pinn_spec) == 4 * (6 + _lib.PINN_MAX_HIDDEN)
    assert C.sizeof(_lib.pinn_problem) == 32
    assert C.sizeof(_lib.pinn_batch) == 8 * 2 + 8 * 3 + 8 + 8 * 3 + 8


@pytest.mark.parametrize("field,value", [("pde", 7), ("n_hidden", 0), ("n_hidden", 17), ("ff_m", -1),
                                         ("rwf", 2), ("precision", 5), ("flags", 2), ("flags", 32)])
def test_invalid_spec_rejected_on_host(lib, field, value):
    spec = _lib.make_spec(1, [64, 64], 8, True, _lib.PINN_BF16)
    setattr(spec, field, value)
    h = C.c_void_p()
    assert lib.pinn_create(C.byref(spec), C.byref(h)) == 1
    assert not h.value


def test_invalid_width_and_null_args(lib):
    spec = _lib.make_spec(0, [64, 0], 0, False)
    h = C.c_void_p()
    assert lib.pinn_create(C.byref(spec), C.byref(h)) == 1
    spec = _lib.make_spec(0, [64, 2049], 0, False)
    assert lib.pinn_create(C.byref(spec), C.byref(h)) == 1
    assert lib.pinn_create(None, C.byref(h)) == 1
    assert lib.pinn_param_count(None, None) == 1
    assert lib.pinn_destroy(None) == 0
    assert lib.pinn_set_chunk_points(None, 64) == 1
    assert lib.pinn_set_activation(None, 1, 2.0) == 1
    assert lib.pinn_set_graph(None, 1) == 1
    assert lib.pinn_set_periodic(None, None) == 1
    # Adam argument checks happen before any device work
    assert lib.pinn_adam_step(None, None, None, None, 10, 1, 1e-3, 0.9, 0.999, 1e-8, None) == 1


def test_no_gpu_fails_loudly(lib):
    """Without a usable GPU the library refuses (PINN_ERR_CUDA, no handle) and the
    Python layer raises: there is no CPU fallback."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    spec = _lib.make_spec(0, [64, 64], 0, False)
    h = C.c_void_p()
    assert lib.pinn_create(C.byref(spec), C.byref(h)) == 3
    assert not h.value
    from paper_2604_15645_gb300 import api
    with pytest.raises(Exception):
        api.PinnNet(0, [64, 64], device="cpu")
