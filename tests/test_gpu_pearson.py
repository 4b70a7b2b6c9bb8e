"""panda_create_from_expression: the co-regulation prior as the Pearson
correlation of the expression data (Sec. II-A), computed on the GPU, against
the FP64 oracle (needs a GB300).

Tolerance on C0: each gene's centred samples are scaled to unit norm (FP64)
and rounded to FP32 (2^-24 relative), then split into BF16 hi + lo.  BF16
keeps 8 significant bits (unit roundoff 2^-8), so |z - hi| <= 2^-8 |z| and
|z - hi - lo| <= 2^-8 |z - hi| <= 2^-16 |z|.  A correlation is the dot
product of two such unit vectors; the three products kept (hi.hi + hi.lo +
lo.hi) miss lo.lo and the two representation errors, each at most
2^-16 |z_g z_h| per sample, so the error is at most about
3 * 2^-16 * sum_k |z_gk z_hk| <= 4.6e-5 (Cauchy-Schwarz), plus FP32
accumulation (a few 1e-7 at these sample counts).  With many samples the
terms' signs cancel (about 1e-6 at N = 200); with few samples the error
approaches the typical size of one term (9.6e-6 at N = 7).  Bound: 5e-5
absolute.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

import gpu_helpers as gh
from oracle.oracle import Oracle
from paper_1507_07039_gb300 import synth

pytestmark = pytest.mark.gpu

C_TOL = 5e-5


@pytest.fixture(scope="module")
def orc():
    o = Oracle()
    o.set_threads(os.cpu_count() or 1)
    return o


def _gpu_c0(W0, P0, X, prec=1):
    from paper_1507_07039_gb300 import panda
    with panda.PandaContext.from_expression(W0, P0, X, prec=prec, normalize=False) as ctx:
        return ctx.get()


@pytest.mark.parametrize("G,N", [(300, 7), (700, 50), (257, 200), (1000, 333)])
def test_correlations_match_oracle(orc, G, N):
    rng = np.random.default_rng(G + N)
    X = (rng.standard_normal((G, 4)) @ rng.standard_normal((4, N)) + 0.5 * rng.standard_normal((G, N))
         + rng.uniform(-3, 3, (G, 1))).astype(np.float32)
    W0 = (rng.random((20, G)) < 0.05).astype(np.float32)
    W, P, C = _gpu_c0(W0, None, X)
    ref = orc.pearson(X)
    assert np.max(np.abs(C.astype(np.float64) - ref)) <= C_TOL
    assert np.array_equal(C, C.T) and np.all(np.diag(C) == 1.0)
    assert np.array_equal(P, np.eye(20, dtype=np.float32))  # P0 = NULL: the identity
    assert np.array_equal(W, W0)                            # normalize off: W0 as given


def test_same_result_in_every_precision_mode():
    """The prior is computed the same way whatever the context's precision
    (BF16X3 and BF16X2 then hold it as its split pair: hi + lo of each entry)."""
    W0, P0, X = synth.make_expression(synth.get("small64x256"))
    Cs = [_gpu_c0(W0, P0, X, prec)[2] for prec in (0, 1, 2, 3)]
    assert np.array_equal(Cs[3], Cs[0])
    for C in Cs[1:3]:
        assert np.array_equal(C, gh.split_held(Cs[0]))


@pytest.mark.parametrize("prec", [0, 1])
def test_pipeline_from_expression(orc, prec):
    """Expression -> Pearson prior -> Z-score -> 6 iterations, against the oracle
    doing the same from the same expression."""
    from paper_1507_07039_gb300 import panda
    W0, P0, X = synth.make_expression(synth.get("mid250x2100"))
    C = orc.pearson(X)
    W, P, C = orc.normalize(W0, P0, C)
    oW, oP, oC, n, hist, _ = orc.run(W, P, C, gh.f32_alpha(0.1), 0.0, 6)
    with panda.PandaContext.from_expression(W0, P0, X, prec=prec) as ctx:
        conv, k, h = ctx.run(0.1, 0.0, 6)
        gW, gP, gC = ctx.get()
    assert k == 6
    gh.assert_parity({"W": gW, "P": gP, "C": gC}, {"W": oW, "P": oP, "C": oC}, prec, "from expression")


def test_human_sized_prior(orc):
    """17000 genes x 200 samples: sampled rows of C0 against the oracle (the
    oracle's full matrix would take minutes), plus symmetry and the diagonal."""
    W0, P0, X = synth.make_expression(synth.get("human1000x17000"))
    W, P, C = _gpu_c0(W0, P0, X)
    G = X.shape[0]
    for r in np.random.default_rng(5).choice(G, 4, replace=False):
        # row r of the oracle's matrix, a block of genes at a time (r prepended to each block)
        ref = np.concatenate([orc.pearson(np.vstack([X[r:r + 1], X[b:b + 1000]]))[0, 1:]
                              for b in range(0, G, 1000)])
        assert np.max(np.abs(C[r].astype(np.float64) - ref)) <= C_TOL, r
    assert np.array_equal(C, C.T) and np.all(np.diag(C) == 1.0)


def test_errors():
    from paper_1507_07039_gb300 import panda
    rng = np.random.default_rng(3)
    X = rng.standard_normal((40, 12)).astype(np.float32)
    W0 = np.ones((5, 40), np.float32)
    bad = X.copy()
    bad[7] = 1.5  # a gene that never changes
    with pytest.raises(panda.PandaError) as e:
        panda.PandaContext.from_expression(W0, None, bad)
    assert e.value.code == -6 and "zero variance" in str(e.value)
    bad = X.copy()
    bad[3, 4] = np.nan
    with pytest.raises(panda.PandaError) as e:
        panda.PandaContext.from_expression(W0, None, bad)
    assert e.value.code == -4
