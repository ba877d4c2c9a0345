"""FP64 CPU oracle for the PINN loss and gradient (test infrastructure only).

Only the tests, the smoke check and the bench's CPU baseline may import this
package.  It shares no code with the CUDA path.  Every function is pinned by the
non-GPU tests against closed forms, analytic PDE solutions, complex-step and
finite differences, and torch float64 autograd (see tests/test_oracle_pins.py).
"""
from .pinn_oracle import (  # noqa: F401
    Model, loss_terms, loss_and_grad, output_jets, adam_step, residuals,
    residual_seeds, input_jets, tanh_derivs, layer_dims, unpack, term_gradients, loss_balance,
    causal_segments, causal_weights, lbfgs_direction, lbfgs_minimize,
    PDE_BURGERS, PDE_NS, PDE_MAXWELL, PDE_ADVECTION, PDE_ALLEN_CAHN,
)
