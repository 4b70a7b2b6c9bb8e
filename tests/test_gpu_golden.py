"""The CUDA path against the worked iteration of tests/golden/ (a 2 x 3
network with identity priors, values derived by hand from Eqs. 1-7): one
step in every precision mode, within the mode's tolerance (needs a GB300).

The diagonals of Eq. 6 take each row's sigma from one-pass sums of x and
x^2 over its off-diagonal entries, accumulated from FP32 values: x^2 is
rounded (relative error u = 2^-24) before it is added, so where sigma is far
below the row's mean the computed variance E[x^2] - E[x]^2 keeps an error of
about 2 u mean^2, and sigma one of up to sqrt(4 u) |mean|.  The worked
case has such a row (row 2 of C' holds {s, s}, sigma = 0): its diagonal is
allowed alpha N e^(2 alpha t) sqrt(4 u) max|x| on top of the mode's
tolerance (4.1e-3 here; measured 9.1e-4)."""
from __future__ import annotations

import numpy as np
import pytest

import golden
import gpu_helpers as gh

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_one_iteration_worked_by_hand(prec):
    from paper_1507_07039_gb300 import panda
    if not panda.panda_precision_supported(prec):
        pytest.skip("precision mode not supported on this device")
    g = golden.step_2x3()
    W0, P0, C0 = (np.asarray(g[k], np.float32) for k in ("W", "P", "C"))
    tol = gh.TOL[prec]
    for case in g["cases"]:
        with panda.PandaContext(W0, P0, C0, prec=prec, normalize=False) as ctx:
            conv, n, h = ctx.run(case["alpha"], 0.0, 1)
            W, P, C = ctx.get()
        assert n == 1
        np.testing.assert_allclose(W, case["W"], rtol=0, atol=tol["W"])
        assert h == pytest.approx(case["h"], abs=tol["W"])
        if "P" in case:
            np.testing.assert_allclose(P, case["P"], rtol=0, atol=tol["off"])
            off = ~np.eye(3, dtype=bool)
            np.testing.assert_allclose(C[off], case["C"][off], rtol=0, atol=tol["off"])
            # one-pass variance bound per row (see the module docstring): N = T for C (Eq. 6, rule D1)
            u = 2.0 ** -24
            want = np.diag(case["C"])
            rowmax = np.max(np.abs(np.where(off, case["C"], 0.0)), axis=1)
            onepass = case["alpha"] * W0.shape[0] * np.exp(2 * case["alpha"]) * np.sqrt(4 * u) * rowmax
            err = np.abs(np.diag(C).astype(np.float64) - want)
            assert np.all(err <= tol["diag"] * np.maximum(np.abs(want), 1.0) + onepass), (np.diag(C), want)
