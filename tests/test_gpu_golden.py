"""The CUDA path against the worked iteration of tests/golden/ (a 2 x 3
network with identity priors, values derived by hand from Eqs. 1-7): one
step in every precision mode, within the mode's tolerance (needs a GB300)."""
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
            np.testing.assert_allclose(np.diag(C), np.diag(case["C"]), rtol=tol["diag"], atol=tol["diag"])
