"""Per-block comparison of a packed parameter gradient with a reference.

A gradient over all P parameters compared through one relative L2 norm can hide a
wrong block whose norm is small next to the rest (one layer's RWF scale gradient
dL/ds, a bias block, the first layer after the embedding).  So every block of the
packed layout is also checked on its own:

    per layer l = 1..L+1:  V_l [fout x fin] | s_l [fout] (RWF only) | b_l [fout]

(Eq. 4 for W, b; Eq. 15 for the factorisation W = diag(exp(s)) V), with the error

    err_k = |g_k - g*_k| / max(|g*_k|, FLOOR * |g*|)      (L2 norms)

held to the same tolerance as the whole gradient.  The floor keeps a block whose
true gradient is negligible next to the whole (a bias of a layer whose biases are
all near zero, say) from being judged on the rounding of its few entries alone;
any block above FLOOR of the whole is judged on its own relative error.

Pure numpy: the CPU tests use it too (the mutation test in test_parity_blocks.py).
"""
from __future__ import annotations

import numpy as np

# Absolute floor of a block's error denominator, as a fraction of the whole
# gradient's L2 norm.
FLOOR = 1e-3


def param_blocks(spec):
    """(name, start, stop) of every block of the packed parameter vector."""
    first_in = 2 * spec.ff_m if spec.ff_m else spec.d_in
    dims, prev = [], first_in
    for w in spec.widths:
        dims.append((prev, w))
        prev = w
    dims.append((prev, spec.d_out))
    out, off = [], 0
    for l, (fi, fo) in enumerate(dims, start=1):
        out.append((f"V{l}", off, off + fo * fi))
        off += fo * fi
        if spec.rwf:
            out.append((f"s{l}", off, off + fo))
            off += fo
        out.append((f"b{l}", off, off + fo))
        off += fo
    return out


def block_errors(g, g_ref, blocks, floor=FLOOR):
    """[(name, err, |g*_k|, |g*_k| / |g*|)] for every block."""
    g = np.asarray(g, dtype=np.float64)
    g_ref = np.asarray(g_ref, dtype=np.float64)
    assert g.shape == g_ref.shape, (g.shape, g_ref.shape)
    assert blocks[-1][2] == g_ref.shape[0], "block layout does not cover the gradient"
    whole = float(np.linalg.norm(g_ref))
    rows = []
    for name, a, b in blocks:
        nk = float(np.linalg.norm(g_ref[a:b]))
        den = max(nk, floor * whole)
        err = float(np.linalg.norm(g[a:b] - g_ref[a:b]) / den) if den > 0 else float(np.linalg.norm(g[a:b]))
        rows.append((name, err, nk, nk / whole if whole > 0 else 0.0))
    return rows


def report(rows):
    """One line per block: name, error, reference norm and share of the whole."""
    return "\n".join(f"  {n:>5s} err {e:.3e}  |g*_k| {nk:.3e}  share {s:.2e}" for n, e, nk, s in rows)


def check_blocks(g, g_ref, spec, tol, what="", floor=FLOOR):
    """Raise AssertionError naming every block whose error exceeds tol."""
    rows = block_errors(g, g_ref, param_blocks(spec), floor)
    bad = [r for r in rows if not (r[1] <= tol)]
    if bad:
        raise AssertionError(f"{what}: {len(bad)} gradient block(s) above {tol}:\n" + report(bad)
                             + "\nall blocks:\n" + report(rows))
    return rows
