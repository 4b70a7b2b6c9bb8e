"""The largest networks the boundary accepts (46000 genes, or 46000 TFs), one
iteration (needs a GB300).  Padded to 46080, a C (or P) of 46080^2 entries is
just under 2^31, so any 32-bit element index on the path would overflow here
first.  The oracle cannot afford whole rows of P' or C' at this size (each
needs all of W'), so: rows of W' against the oracle (Eqs. 2-4), and
properties that hold at any size for P' and C' (exact symmetry, finite
entries, the diagonal above the damped old one: Eq. 6 adds a non-negative
term), and h against the mean |W' - W| (Eq. 7)."""
from __future__ import annotations

import os

import numpy as np
import pytest

import gpu_helpers as gh
from oracle.oracle import Oracle
from paper_1507_07039_gb300 import synth

pytestmark = pytest.mark.gpu


def _blocks_symmetric(X, rng, n_blocks=64, b=64):
    """Random b x b blocks and the last block against their mirrors."""
    n = X.shape[0]
    starts = [(n - b, n - b), (0, n - b), (n - b, 0)]
    starts += [tuple(rng.integers(0, n - b, 2)) for _ in range(n_blocks)]
    for i, j in starts:
        if not np.array_equal(X[i:i + b, j:j + b], X[j:j + b, i:i + b].T):
            return False
    return True


@pytest.mark.parametrize("T,G,prec", [(300, 46000, 1), (300, 46000, 0), (46000, 300, 1)])
def test_largest_network_one_iteration(T, G, prec):
    from paper_1507_07039_gb300 import panda
    wl = synth.custom(T, G, 46000, n_samples=30, n_factors=4)
    W0, P0, C0 = synth.make_inputs(wl)
    orc = Oracle()
    orc.set_threads(os.cpu_count() or 1)
    W, P, C = orc.normalize(W0, P0, C0)  # both sides Z-score the same raw networks
    alpha = gh.f32_alpha(0.1)
    rng = np.random.default_rng(T + G + prec)
    rows = np.sort(rng.choice(T, 2 if G > T else 8, replace=False))
    rows[-1] = T - 1  # the last row of the last, ragged tile
    Wn = orc.w_rows(W, P, C, alpha, rows)

    with panda.PandaContext(W0, P0, C0, prec=prec) as ctx:
        h = ctx.step(0.1)
        gW, gP, gC = ctx.get()
    del W0, P0, C0
    tol = gh.TOL[prec]
    err = float(np.max(np.abs(gW[rows].astype(np.float64) - Wn)))
    assert err <= tol["W"], f"W' rows {rows}: err {err:.3e}"
    # Eq. 7: h against the mean |W' - W| of the GPU's W' and the oracle's Z-scored W
    # (the two Z-scores agree to an FP32 ulp, far below this bound)
    assert abs(h - float(np.mean(np.abs(gW.astype(np.float64) - W)))) <= 2e-6
    for name, X, old in (("P", gP, P), ("C", gC, C)):
        assert np.isfinite(X).all(), name
        assert _blocks_symmetric(X, rng), name
        # Eq. 6: new diagonal = (1 - alpha) old + alpha N sigma e^{2 alpha} with sigma >= 0
        d_new, d_old = np.diag(X).astype(np.float64), np.diag(old)
        assert np.all(d_new >= (1.0 - alpha) * d_old - 1e-5 * np.maximum(1.0, np.abs(d_old))), name
