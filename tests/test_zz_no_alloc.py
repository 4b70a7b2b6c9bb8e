"""panda_step_static, the iteration for callers that may not allocate device
memory (a framework that hands out all device memory from its own pool, a
plug-in that must not call cudaMalloc once running, a loop that cannot take
cudaMalloc's implicit synchronisation), checked through the C ABI:

* two successive calls against the FP64 oracle at the FP32 path's tolerances,
  under every diagonal rule, on shapes that fill the fixed working array to
  its ends (512 x 512 = PANDA_STATIC_MAX_NODES), lopsided and ragged ones;
* two calls against the allocating path (a context's panda_step), which runs
  the same kernels, on the same networks;
* the device's free memory is the same before and after the second and third
  calls (the first may load the library's device code);
* shapes past the working array are refused before any device work.

It is collected last on purpose: if it fails, a run that stops at the first
failure has already run every other test.  It needs a GB300.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

import gpu_helpers as gh
from oracle.oracle import Oracle
from paper_1507_07039_gb300 import synth

pytestmark = pytest.mark.gpu

ALPHA = 0.1


def _networks(T, G, seed):
    """Z-scored synthetic networks rounded to FP32 (what panda_get returns),
    the same values for the GPU and the oracle."""
    orc = Oracle()
    W0, P0, C0 = synth.make_inputs(synth.custom(T, G, seed, n_samples=30, n_factors=3))
    if T > 1 and G > 1:
        W, P, C = orc.normalize(W0, P0, C0)
    else:  # a single node has no spread to Z-score: random values instead
        rng = np.random.default_rng(seed)
        W = rng.standard_normal((T, G))
        P, C = gh.random_symmetric(rng, T), gh.random_symmetric(rng, G)
    return tuple(np.ascontiguousarray(x, np.float32) for x in (W, P, C))


def _static_steps(panda, torch, W, P, C, diag, ts=(1, 2)):
    T, G = W.shape
    torch.cuda.set_device(0)
    dW, dP, dC = (torch.from_numpy(x).cuda() for x in (W, P, C))
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    h = [panda.panda_step_static(T, G, dW, dP, dC, ALPHA, t, diag=diag, stream=stream) for t in ts]
    return (x.cpu().numpy() for x in (dW, dP, dC)), h


@pytest.mark.parametrize("diag", [0, 1, 2])
@pytest.mark.parametrize("T,G", [(512, 512), (512, 7), (129, 511), (1, 1)])
def test_static_steps_match_the_oracle(T, G, diag):
    import torch
    from paper_1507_07039_gb300 import panda
    W, P, C = _networks(T, G, 4000 + T + G)
    (sW, sP, sC), h = _static_steps(panda, torch, W, P, C, diag)
    orc = Oracle()
    orc.set_threads(os.cpu_count() or 1)
    o = gh.oracle_run(orc, W, P, C, ALPHA, 0.0, 2, normalize=False, diag=diag)
    gh.assert_parity({"W": sW, "P": sP, "C": sC}, o, 0, f"static {T}x{G} D{diag}")
    np.testing.assert_allclose(h, o["hist"], rtol=1e-4, atol=1e-7)


@pytest.mark.parametrize("diag", [0, 1, 2])
def test_static_step_matches_context_step(diag):
    import torch
    from paper_1507_07039_gb300 import panda
    T, G = 100, 300
    W0, P0, C0 = synth.make_inputs(synth.custom(T, G, 4242, n_samples=30, n_factors=3))

    # the allocating path: a context (no normalisation, so both see the same networks)
    with panda.PandaContext(W0, P0, C0, normalize=False, diag=diag) as ctx:
        ref_h = [ctx.step(ALPHA), ctx.step(ALPHA)]
        rW, rP, rC = ctx.get()
    (sW, sP, sC), h = _static_steps(panda, torch, W0, P0, C0, diag)

    tol = gh.TOL[0]
    assert np.max(np.abs(sW - rW)) <= tol["W"]
    e = gh.errors({"W": sW, "P": sP, "C": sC}, {"W": rW.astype(np.float64), "P": rP.astype(np.float64),
                                                "C": rC.astype(np.float64)})
    assert e["Poff"] <= tol["off"] and e["Coff"] <= tol["off"], e
    assert e["Pdiag"] <= tol["diag"] and e["Cdiag"] <= tol["diag"], e
    np.testing.assert_allclose(h, ref_h, rtol=1e-6)


def test_static_calls_allocate_no_device_memory():
    import torch
    from paper_1507_07039_gb300 import panda
    T = G = panda.PANDA_STATIC_MAX_NODES
    W, P, C = _networks(T, G, 99)
    torch.cuda.set_device(0)
    dW, dP, dC = (torch.from_numpy(x).cuda() for x in (W, P, C))
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    panda.panda_step_static(T, G, dW, dP, dC, ALPHA, 1, stream=stream)  # may load device code
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for t in (2, 3):
        panda.panda_step_static(T, G, dW, dP, dC, ALPHA, t, stream=stream)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, f"free device memory changed during call t={t}"
    assert np.isfinite(dW.cpu().numpy()).all()


def test_static_step_rejects_sizes_beyond_its_scratch():
    from paper_1507_07039_gb300 import panda
    n = panda.PANDA_STATIC_MAX_NODES + 1
    for T, G in ((n, 8), (8, n)):
        with pytest.raises(panda.PandaError) as e:
            # rejected on the shape before any device pointer is touched
            panda.panda_step_static(T, G, 16, 16, 16, 0.1, 1)
        assert e.value.code == -1
        assert "static scratch" in panda.panda_last_error(None)
