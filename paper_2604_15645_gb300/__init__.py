"""GB300 (sm_103a) PINN loss + gradient library: Fourier-feature / RWF tanh MLP
jets, Burgers / Navier-Stokes / Maxwell residuals, hand-written adjoint and fused
Adam behind a C ABI (include/pinn.h).  This package holds the build script and
the thin Python binding."""
from ._lib import load, PinnError, PRECISIONS  # noqa: F401


def __getattr__(name):
    if name in ("PinnNet", "DeviceBatch", "make_problem", "adam_step", "PinnLoss", "PinnMulti"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
