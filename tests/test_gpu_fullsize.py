"""One iteration of the human-sized network (1000 TFs x 17000 genes, the
benchmark's workload and launch configuration) against the oracle: the whole
of W', whole sampled rows of P' and C', and their diagonals (needs a GB300)."""
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
    Wn = orc.w_rows(W, P, C, alpha, np.arange(W.shape[0]))  # all of W' (Eqs. 2-4)
    return dict(orc=orc, inputs=(W0, P0, C0), state=(W, P, C), Wn=Wn, alpha=alpha)


@pytest.mark.parametrize("prec", PRECS)
def test_human_sized_one_iteration(case, prec):
    from paper_1507_07039_gb300 import panda
    W0, P0, C0 = case["inputs"]
    T, G = W0.shape
    with panda.PandaContext(W0, P0, C0, prec=prec) as ctx:
        h = ctx.step(0.1)
        gW, gP, gC = ctx.get()
    orc, Wn, alpha = case["orc"], case["Wn"], case["alpha"]
    W, P, C = case["state"]
    tol = gh.TOL[prec]
    # W' everywhere, and h
    errW = float(np.max(np.abs(gW.astype(np.float64) - Wn)))
    assert errW <= tol["W"], f"W' err {errW:.3e}"
    # |h_gpu - h| <= mean |W'_gpu - W'| (triangle inequality), plus the FP32 sum's rounding
    bound = float(np.mean(np.abs(gW.astype(np.float64) - Wn))) + 1e-6 * h
    assert abs(h - np.mean(np.abs(Wn - W))) <= bound, f"h {h} vs {np.mean(np.abs(Wn - W))}" 
    # whole rows of P' and C' (Eq. 5) and their diagonals (Eq. 6)
    rng = np.random.default_rng(7)
    prow = np.sort(rng.choice(T, 4, replace=False))
    crow = np.sort(rng.choice(G, 4, replace=False))
    oP = orc.p_rows(Wn, P, alpha, prow)
    oC = orc.c_rows(Wn, C, alpha, crow)
    for q, i in enumerate(prow):
        off = np.arange(T) != i
        scale = max(1.0, float(np.max(np.abs(oP[q][off]))))
        e = float(np.max(np.abs(gP[i][off] - oP[q][off]))) / scale
        assert e <= tol["off"], f"P' row {i} err {e:.3e}"
        d = orc.diag_value(oP[q], i, G, P[i, i], alpha, 1)
        assert abs(gP[i, i] - d) <= tol["diag"] * max(1.0, abs(d)), f"P'_{i}{i} {gP[i, i]} vs {d}"
    for q, k in enumerate(crow):
        off = np.arange(G) != k
        scale = max(1.0, float(np.max(np.abs(oC[q][off]))))
        e = float(np.max(np.abs(gC[k][off] - oC[q][off]))) / scale
        assert e <= tol["off"], f"C' row {k} err {e:.3e}"
        d = orc.diag_value(oC[q], k, T, C[k, k], alpha, 1)
        assert abs(gC[k, k] - d) <= tol["diag"] * max(1.0, abs(d)), f"C'_{k}{k} {gC[k, k]} vs {d}"
    # properties at full size
    assert np.array_equal(gP, gP.T) and np.array_equal(gC, gC.T)


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
    gh.assert_parity(g, o, prec, "1600 x 2000 subsample")
