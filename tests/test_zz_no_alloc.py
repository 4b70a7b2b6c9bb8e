"""panda_step_static, the iteration for callers that may not allocate device
memory, checked through the C ABI against the allocating path (a context's
panda_step) on the same networks, over two iterations in a row.

It is collected last on purpose: if it fails, a run that stops at the first
failure has already run every other test.  It needs a GB300.
"""
from __future__ import annotations

import numpy as np
import pytest

import gpu_helpers as gh
from paper_1507_07039_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("diag", [0, 1, 2])
def test_static_step_matches_context_step(diag):
    """Every diagonal rule (D1, D0, D2)."""
    import torch
    from paper_1507_07039_gb300 import panda
    T, G = 100, 300
    W0, P0, C0 = synth.make_inputs(synth.custom(T, G, 4242, n_samples=30, n_factors=3))

    # the allocating path: a context (no normalisation, so both see the same networks)
    with panda.PandaContext(W0, P0, C0, normalize=False, diag=diag) as ctx:
        ref_h = [ctx.step(0.1), ctx.step(0.1)]
        rW, rP, rC = ctx.get()

    torch.cuda.set_device(0)
    dW, dP, dC = (torch.from_numpy(x).cuda() for x in (W0, P0, C0))
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    h = [panda.panda_step_static(T, G, dW, dP, dC, 0.1, t, diag=diag, stream=stream) for t in (1, 2)]
    sW, sP, sC = (x.cpu().numpy() for x in (dW, dP, dC))

    tol = gh.TOL[0]
    assert np.max(np.abs(sW - rW)) <= tol["W"]
    e = gh.errors({"W": sW, "P": sP, "C": sC}, {"W": rW.astype(np.float64), "P": rP.astype(np.float64),
                                                "C": rC.astype(np.float64)})
    assert e["Poff"] <= tol["off"] and e["Coff"] <= tol["off"], e
    assert e["Pdiag"] <= tol["diag"] and e["Cdiag"] <= tol["diag"], e
    np.testing.assert_allclose(h, ref_h, rtol=1e-6)


def test_static_step_rejects_sizes_beyond_its_scratch():
    from paper_1507_07039_gb300 import panda
    n = panda.PANDA_STATIC_MAX_NODES + 1
    with pytest.raises(panda.PandaError) as e:
        # rejected on the shape before any device pointer is touched
        panda.panda_step_static(n, 8, 16, 16, 16, 0.1, 1)
    assert e.value.code == -1
    assert "static scratch" in panda.panda_last_error(None)
