"""The human-sized network (1000 TFs x 17000 genes, the benchmark's workload
and launch configuration) against the oracle after one and after three
iterations: all of W, P and C, diagonals included, and h (needs a GB300; the
oracle's three full iterations take about two minutes on 16 host cores)."""
from __future__ import annotations

import os

import numpy as np
import pytest

import gpu_helpers as gh
from oracle.oracle import Oracle

pytestmark = pytest.mark.gpu

PRECS = [0, 1, 2, 3]  # PANDA_FP32, PANDA_BF16X3, PANDA_BF16X2, PANDA_FP8MIX


@pytest.fixture(scope="module")
def case():
    orc = Oracle()
    orc.set_threads(os.cpu_count() or 1)
    W0, P0, C0 = gh.inputs("human1000x17000")
    W, P, C = orc.normalize(W0, P0, C0)
    alpha = gh.f32_alpha(0.1)
    W1, P1, C1, n1, h1, _ = orc.run(W, P, C, alpha, 0.0, 1)
    W3, P3, C3, n3, h23, _ = orc.run(W1, P1, C1, alpha, 0.0, 2, t0=1)
    assert n1 == 1 and n3 == 2
    return dict(inputs=(W0, P0, C0), W0n=W, s1=dict(W=W1, P=P1, C=C1, hist=h1),
                s3=dict(W=W3, P=P3, C=C3, hist=np.concatenate([h1, h23])))


def _gpu(case, prec, iters):
    from paper_1507_07039_gb300 import panda
    W0, P0, C0 = case["inputs"]
    with panda.PandaContext(W0, P0, C0, prec=prec) as ctx:
        conv, n, _ = ctx.run(0.1, 0.0, iters)
        gW, gP, gC = ctx.get()
        hist = ctx.history()
    assert n == iters and not conv
    return dict(W=gW, P=gP, C=gC, hist=hist)


@pytest.mark.parametrize("prec", PRECS)
def test_human_sized_one_iteration(case, prec):
    g, o = _gpu(case, prec, 1), case["s1"]
    e = gh.assert_parity(g, o, prec, "1000 x 17000, one iteration")
    # |h_gpu - h| <= mean |W'_gpu - W'| (triangle inequality), plus the FP32 sum's rounding
    Wn = o["W"]
    bound = float(np.mean(np.abs(g["W"].astype(np.float64) - Wn))) + 1e-6 * g["hist"][0]
    assert abs(g["hist"][0] - o["hist"][0]) <= bound, (g["hist"][0], o["hist"][0])
    # properties at full size
    assert np.array_equal(g["P"], g["P"].T) and np.array_equal(g["C"], g["C"].T)
    print(f"\n1000 x 17000 prec {prec}, iteration 1: " + ", ".join(f"{k} {v:.3e}" for k, v in e.items()))


@pytest.mark.parametrize("prec", PRECS)
def test_human_sized_three_iterations(case, prec):
    g, o = _gpu(case, prec, 3), case["s3"]
    e = gh.assert_parity(g, o, prec, "1000 x 17000, three iterations")
    rtol, atol = {0: (1e-4, 1e-7), 1: (1e-3, 1e-6), 2: (0.0, 1e-3), 3: (0.0, 1e-2)}[prec]
    np.testing.assert_allclose(g["hist"], o["hist"], rtol=rtol, atol=atol)
    print(f"\n1000 x 17000 prec {prec}, iteration 3: " + ", ".join(f"{k} {v:.3e}" for k, v in e.items()))


@pytest.fixture(scope="module")
def large_subnetwork():
    """The large network (1600 TFs x 30000 genes, 300 samples from 30 factors)
    restricted to the first 2000 genes of a seeded permutation: their W
    columns and C block, all of P."""
    from paper_1507_07039_gb300 import synth
    wl = synth.get("large1600x30000")
    W0, P0, C0 = synth.make_inputs(wl)
    genes = synth.gene_subsample(wl.G, 2000, wl.seed + 99)
    return (np.ascontiguousarray(W0[:, genes]), P0, np.ascontiguousarray(C0[np.ix_(genes, genes)]))


@pytest.mark.parametrize("prec", PRECS)
def test_large_network_gene_subsample(large_subnetwork, prec):
    W0, P0, C0 = large_subnetwork
    orc = Oracle()
    orc.set_threads(os.cpu_count() or 1)
    o = gh.oracle_run(orc, W0, P0, C0, 0.1, 0.0, 4)
    g = gh.gpu_run(W0, P0, C0, prec, 0.1, 0.0, 4)
    e = gh.assert_parity(g, o, prec, "1600 x 2000 subsample")
    print(f"\n1600 x 2000 subsample prec {prec}, 4 iterations: " + ", ".join(f"{k} {v:.3e}" for k, v in e.items()))
