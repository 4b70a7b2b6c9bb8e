"""CUDA library against the FP64 oracle, through the C ABI (needs a GB300)."""
from __future__ import annotations

import os

import numpy as np
import pytest

import gpu_helpers as gh
from oracle.oracle import Oracle
from paper_1507_07039_gb300 import synth

pytestmark = pytest.mark.gpu

PRECS = [0, 1, 2, 3]  # PANDA_FP32, PANDA_BF16X3, PANDA_BF16X2, PANDA_FP8MIX


@pytest.fixture(scope="module")
def orc():
    o = Oracle()
    o.set_threads(os.cpu_count() or 1)
    return o


@pytest.fixture(scope="module")
def panda():
    from paper_1507_07039_gb300 import panda as p
    return p


def _fixed_or_same_count(o, tol):
    """True when the oracle's stop decision sits within 1e-6 of tol."""
    return bool(np.any(np.abs(o["hist"] - tol) < 1e-6))


@pytest.mark.parametrize("prec", PRECS)
def test_small_network_full_trajectory(orc, prec):
    """64 TFs x 256 genes, alpha 0.1, tol 1e-3, up to 200 iterations."""
    W0, P0, C0 = gh.inputs("small64x256")
    o = gh.oracle_run(orc, W0, P0, C0, 0.1, 1e-3, 200)
    g = gh.gpu_run(W0, P0, C0, prec, 0.1, 1e-3, 200)
    if _fixed_or_same_count(o, 1e-3) or prec >= 2:  # BF16X2, FP8MIX: at the oracle's count
        o = gh.oracle_run(orc, W0, P0, C0, 0.1, 0.0, o["iters"])
        g = gh.gpu_run(W0, P0, C0, prec, 0.1, 0.0, o["iters"])
    assert g["iters"] == o["iters"] and g["converged"] == o["converged"]
    # h is a mean of |dW|; its error is bounded by the mean error of W and W'
    rtol, atol = {0: (1e-4, 1e-7), 1: (1e-3, 1e-6), 2: (0.0, 1e-3), 3: (0.0, 1e-2)}[prec]
    np.testing.assert_allclose(g["hist"], o["hist"], rtol=rtol, atol=atol)
    gh.assert_parity(g, o, prec, "small")


@pytest.mark.parametrize("prec", PRECS)
def test_mid_network_fixed_iterations(orc, prec):
    """250 TFs x 2100 genes (two ragged tile edges), 12 fixed iterations."""
    W0, P0, C0 = gh.inputs("mid250x2100")
    o = gh.oracle_run(orc, W0, P0, C0, 0.1, 0.0, 12)
    g = gh.gpu_run(W0, P0, C0, prec, 0.1, 0.0, 12)
    assert g["iters"] == 12 and not g["converged"]
    gh.assert_parity(g, o, prec, "mid")


EDGE_SHAPES = [(1, 1), (1, 5), (3, 1), (2, 3), (5, 130), (130, 7), (129, 257), (128, 128), (200, 385), (256, 512),
               (257, 256)]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("T,G", EDGE_SHAPES)
def test_edge_shapes(orc, prec, T, G):
    """Tiny, single-node and ragged networks, without normalisation, 3 iterations."""
    rng = np.random.default_rng(1000 * T + G)
    W0 = rng.standard_normal((T, G)).astype(np.float32)
    P0, C0 = gh.random_symmetric(rng, T), gh.random_symmetric(rng, G)
    o = gh.oracle_run(orc, W0, P0, C0, 0.2, 0.0, 3, normalize=False)
    g = gh.gpu_run(W0, P0, C0, prec, 0.2, 0.0, 3, normalize=False)
    gh.assert_parity(g, o, prec, f"{T}x{G}")


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("diag", [1, 2])
@pytest.mark.parametrize("T,G", [(40, 150), (300, 700)])
def test_other_diagonal_rules(orc, prec, diag, T, G):
    """Rules D0 (Eq. 6 as printed, no alpha) and D2 (sigma of the new
    similarities instead of the new entries) in every precision mode; 300 x 700
    spans diagonal and off-diagonal 256-tiles of both P and C."""
    W0, P0, C0 = gh.inputs(synth.custom(T, G, 77, n_samples=30, n_factors=3))
    o = gh.oracle_run(orc, W0, P0, C0, 0.1, 0.0, 6, diag=diag)
    g = gh.gpu_run(W0, P0, C0, prec, 0.1, 0.0, 6, diag=diag)
    gh.assert_parity(g, o, prec, f"diag rule {diag}", gh.FP8MIX_D0 if (prec, diag) == (3, 1) else None)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n", [125, 500])
def test_identity_priors(orc, prec, n):
    """The paper's Table I shape: P = C = I, random W (two of its sizes)."""
    W0, P0, C0 = gh.inputs(synth.table1(n))
    o = gh.oracle_run(orc, W0, P0, C0, 0.1, 0.0, 10)
    g = gh.gpu_run(W0, P0, C0, prec, 0.1, 0.0, 10)
    gh.assert_parity(g, o, prec, "identity priors")


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name,offset", [("small64x256", 0.0), ("mid250x2100", 0.0), ("mid250x2100", 7.0)])
def test_normalized_state_matches_oracle(orc, panda, name, offset, prec):
    """The Z-scored networks a context starts from (Sec. II-A) against the
    oracle's FP64 Z-score rounded to FP32.  The GPU sums in another order and
    divides through FP32 pairs accurate to about 2^-44, so an entry may round
    the other way when the exact quotient sits that close to a rounding
    midpoint: at most one unit in the last place apart, and rarely (about
    1e-6 of the entries expected).  An offset of 7 makes the mean large
    against the spread of W0 and P0, the hardest case for the pair arithmetic."""
    W0, P0, C0 = (x + np.float32(offset) for x in gh.inputs(name))
    oW, oP, oC = orc.normalize(W0, P0, C0)
    with panda.PandaContext(W0, P0, C0, prec=prec) as ctx:
        gW, gP, gC = ctx.get()
    nets = (("W", gW, oW), ("P", gP, oP), ("C", gC, oC))
    if prec == 1:  # BF16X3 holds C as hi + lo of the FP32 Z-score: within 2^-16 |x| of it
        o32 = oC.astype(np.float32).astype(np.float64)
        off = ~np.eye(oC.shape[0], dtype=bool)
        assert np.all(np.abs(gC.astype(np.float64) - o32)[off] <= 2.0 ** -16 * np.abs(o32)[off])
        dg, do = np.diag(gC), np.diag(oC).astype(np.float32)  # the diagonal: from its FP64 vector
        assert np.all(np.abs(dg.astype(np.float64) - do) <= np.spacing(np.maximum(np.abs(dg), np.abs(do))))
        nets = nets[:2]
    for label, g, o in nets:
        o32 = o.astype(np.float32)
        diff = np.abs(g.astype(np.float64) - o32.astype(np.float64))
        ulp = np.spacing(np.maximum(np.abs(g), np.abs(o32))).astype(np.float64)
        assert np.all(diff <= ulp), f"{label}: {np.max(diff / ulp):.1f} ulp"
        assert np.count_nonzero(diff) <= 1e-4 * g.size + 2, f"{label}: {np.count_nonzero(diff)} of {g.size} differ"


def test_alpha_zero_leaves_networks_unchanged(panda):
    W0, P0, C0 = gh.inputs("small64x256")
    with panda.PandaContext(W0, P0, C0) as ctx:
        W1, P1, C1 = ctx.get()
        for _ in range(3):
            assert ctx.step(0.0) == 0.0
        W2, P2, C2 = ctx.get()
    assert np.array_equal(W1, W2) and np.array_equal(P1, P2) and np.array_equal(C1, C2)


@pytest.mark.parametrize("prec", PRECS)
def test_symmetry_and_determinism(prec):
    W0, P0, C0 = gh.inputs("mid250x2100")
    a = gh.gpu_run(W0, P0, C0, prec, 0.1, 0.0, 5)
    b = gh.gpu_run(W0, P0, C0, prec, 0.1, 0.0, 5, graph_iters=0)
    for k in ("W", "P", "C"):
        assert np.array_equal(a[k], b[k]), f"{k} differs between two runs"
    assert np.array_equal(a["P"], a["P"].T) and np.array_equal(a["C"], a["C"].T)
    assert np.all(a["hist"] >= 0)


@pytest.mark.parametrize("prec", PRECS)
def test_checkpoint_resume_is_bitwise(panda, prec):
    W0, P0, C0 = gh.inputs("small64x256")
    with panda.PandaContext(W0, P0, C0, prec=prec) as a:
        a.run(0.1, 0.0, 4)
        blob = panda.panda_save(a.h)
        a.run(0.1, 0.0, 5)
        ref = a.get()
        ref_hist = a.history()
    with panda.PandaContext(W0, P0, C0, prec=prec) as b:
        panda.panda_load(b.h, blob)
        assert b.info()[3] == 4
        b.run(0.1, 0.0, 5)
        got = b.get()
        hist = b.history()
    for x, y in zip(ref, got):
        assert np.array_equal(x, y)
    assert np.array_equal(ref_hist, hist)


def test_checkpoint_from_another_context_is_rejected(panda):
    """A checkpoint loads only into a context of the same shape, precision
    and diagonal rule; a truncated or corrupted one is refused too, and the
    context keeps working afterwards."""
    W0, P0, C0 = gh.inputs("small64x256")
    with panda.PandaContext(W0, P0, C0, prec=1) as a:
        a.run(0.1, 0.0, 2)
        blob = panda.panda_save(a.h)
    others = [dict(prec=0), dict(prec=3), dict(prec=1, diag=2)]
    for kw in others:
        with panda.PandaContext(W0, P0, C0, **kw) as b:
            with pytest.raises(panda.PandaError) as e:
                panda.panda_load(b.h, blob)
            assert e.value.code == -1
            b.run(0.1, 0.0, 1)
    W1, P1, C1 = W0[:, :200].copy(), P0, np.ascontiguousarray(C0[:200, :200])
    with panda.PandaContext(W1, P1, C1, prec=1) as b:
        with pytest.raises(panda.PandaError) as e:
            panda.panda_load(b.h, blob)
        assert e.value.code == -1
    with panda.PandaContext(W0, P0, C0, prec=1) as b:
        for bad in (blob[:-1], b"X" + blob[1:]):
            with pytest.raises(panda.PandaError) as e:
                panda.panda_load(b.h, bad)
            assert e.value.code == -1
        panda.panda_load(b.h, blob)  # the genuine one still loads
        assert b.info()[3] == 2


@pytest.mark.parametrize("prec", [0, 1])
def test_set_state_continues_close(panda, prec):
    """A state read out and set into another context continues where the
    first one does (the derived vectors are recomputed, so in a summation
    order of their own: close, not bitwise)."""
    W0, P0, C0 = gh.inputs("small64x256")
    with panda.PandaContext(W0, P0, C0, prec=prec) as a:
        a.run(0.1, 0.0, 3)
        W, P, C, t = panda.panda_get_state(a.h, 64, 256)
        a.run(0.1, 0.0, 3)
        ref = a.get()
    with panda.PandaContext(W0, P0, C0, prec=prec) as b:
        panda.panda_set_state(b.h, W, P, C, t)
        b.run(0.1, 0.0, 3)
        got = b.get()
    assert np.max(np.abs(ref[0] - got[0])) < (1e-5 if prec == 0 else 1e-4)


def test_rejected_state_blocks_the_context_until_a_valid_one(panda):
    """panda_set_state with an asymmetric C is refused (EASYM); the context
    then refuses to step, run, get or save (EINVAL) instead of iterating on
    networks it has not validated, until a valid state is set."""
    W0, P0, C0 = gh.inputs("small64x256")
    with panda.PandaContext(W0, P0, C0, prec=1) as ctx:
        ctx.run(0.1, 0.0, 2)
        W, P, C, t = panda.panda_get_state(ctx.h, 64, 256)
        bad = C.copy()
        bad[3, 9] += 1.0
        with pytest.raises(panda.PandaError) as e:
            panda.panda_set_state(ctx.h, W, P, bad, t)
        assert e.value.code == -5
        for call in (lambda: ctx.step(0.1), lambda: ctx.run(0.1, 0.0, 2), lambda: ctx.get(),
                     lambda: panda.panda_save(ctx.h)):
            with pytest.raises(panda.PandaError) as e:
                call()
            assert e.value.code == -1 and "no valid state" in str(e.value)
        panda.panda_set_state(ctx.h, W, P, C, t)
        ctx.step(0.1)
        assert ctx.info()[3] == t + 1


@pytest.mark.parametrize("prec", [0, 1, 3])
def test_device_pointer_create_matches_host(panda, prec):
    """panda_create_device on torch-owned buffers and panda_get_device into
    them give the host path's results bit for bit (W, P and C)."""
    import torch
    W0, P0, C0 = gh.inputs("small64x256")
    dW, dP, dC = (torch.from_numpy(x).cuda() for x in (W0, P0, C0))
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    with panda.PandaContext(dW, dP, dC, prec=prec, device=True, stream=stream) as a:
        a.run(0.1, 0.0, 4)
        outs = [torch.empty_like(x) for x in (dW, dP, dC)]
        panda.panda_get_device(a.h, *outs)
        torch.cuda.synchronize()
        got = [x.cpu().numpy() for x in outs]
    ref = gh.gpu_run(W0, P0, C0, prec, 0.1, 0.0, 4)
    for g, k in zip(got, ("W", "P", "C")):
        assert np.array_equal(g, ref[k]), k


@pytest.mark.parametrize("prec", [0, 1])
def test_start_index_t0(orc, panda, prec):
    """opts.t0 = 7: the first iteration uses t = 8 in the e^{2 alpha t} factor
    of the diagonals (Eq. 6), against the oracle started at the same t."""
    W0, P0, C0 = gh.inputs("small64x256")
    W, P, C = orc.normalize(W0, P0, C0)
    oW, oP, oC, n, hist, _ = orc.run(W, P, C, gh.f32_alpha(0.1), 0.0, 4, 7)
    with panda.PandaContext(W0, P0, C0, prec=prec, t0=7) as ctx:
        conv, k, h = ctx.run(0.1, 0.0, 4)
        gW, gP, gC = ctx.get()
        t = ctx.info()[3]
    assert k == 4 and t == 11
    gh.assert_parity({"W": gW, "P": gP, "C": gC}, {"W": oW, "P": oP, "C": oC}, prec, "t0 = 7")


def test_error_codes(panda):
    W0, P0, C0 = gh.inputs("small64x256")
    bad = C0.copy()
    bad[3, 7] += 1.0
    with pytest.raises(panda.PandaError) as e:
        panda.PandaContext(W0, P0, bad)
    assert e.value.code == -5
    nan = W0.copy()
    nan[1, 2] = np.nan
    with pytest.raises(panda.PandaError) as e:
        panda.PandaContext(nan, P0, C0)
    assert e.value.code == -4
    with pytest.raises(panda.PandaError) as e:
        panda.PandaContext(np.ones_like(W0), P0, C0)
    assert e.value.code == -6
    with panda.PandaContext(W0, P0, C0) as ctx:
        with pytest.raises(panda.PandaError) as e:
            ctx.step(1.5)
        assert e.value.code == -1
        with pytest.raises(panda.PandaError) as e:
            ctx.run(0.1, -1.0, 3)
        assert e.value.code == -1
        conv, n, h = ctx.run(0.1, 0.0, 2)
        assert not conv and n == 2


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("T,G", [(3, 31), (33, 97), (40, 300)])
def test_validation_finds_every_position(panda, prec, T, G):
    """The create-time checks read P and C as mirror pairs of 32 x 32 blocks:
    one asymmetric entry or one non-finite entry is found wherever it sits
    (first and last block, diagonal blocks, across a block edge, the ragged
    last block), and exactly symmetric finite inputs pass."""
    rng = np.random.default_rng(T * 1000 + G)
    W0 = rng.standard_normal((T, G)).astype(np.float32)
    P0 = gh.random_symmetric(rng, T)
    C0 = gh.random_symmetric(rng, G)
    with panda.PandaContext(W0, P0, C0, prec=prec, normalize=False) as ctx:
        gW, gP, gC = ctx.get()
    # BF16X3 holds C as its split pair: hi + lo of each entry, the diagonal exact
    assert np.array_equal(gW, W0) and np.array_equal(gP, P0)
    assert np.array_equal(gC, gh.split_held(C0) if prec == 1 else C0)

    def expect(code, W=W0, P=P0, C=C0):
        with pytest.raises(panda.PandaError) as e:
            panda.PandaContext(W, P, C, prec=prec, normalize=False)
        assert e.value.code == code

    for X, n, which in ((C0, G, "C"), (P0, T, "P")):
        pos = {(0, 1), (1, 0), (n - 1, n - 2), (n - 2, n - 1), (0, n - 1), (n - 1, 0)}
        if n > 32:
            pos |= {(31, 32), (32, 31), (n - 1, 32), (5, n - 1)}
        pos = {(i, j) for i, j in pos if i != j}  # a diagonal entry has no mirror to differ from
        for i, j in sorted(pos):
            bad = X.copy()
            bad[i, j] += 0.5
            expect(-5, **{which: bad})
        for i, j in sorted(pos | {(0, 0), (n - 1, n - 1)}):
            bad = X.copy()
            bad[i, j] = np.nan if (i + j) % 2 else np.inf
            expect(-4, **{which: bad})
    bad = W0.copy()
    bad[T - 1, G - 1] = -np.inf
    expect(-4, W=bad)


def test_device_bytes_follow_the_memory_plan(panda, monkeypatch):
    """panda_device_bytes counts what a context holds between calls: at least
    the padded FP32 state (W and W^T twice, P, C) on the FP32 path; under
    BF16X3 and BF16X2 C is held only as its split pair (2 + 2 bytes per
    entry), so both modes hold the same, and their peak adds the FP32 C staged
    while the state is derived.  (Both also hold the running-sum slots of the
    chunked long products.)  A create capped at the peak succeeds while one
    byte less fails."""
    W0, P0, C0 = gh.inputs("mid250x2100")
    T, G = W0.shape
    got, peak = {}, {}
    for prec in (0, 1, 2):
        with panda.PandaContext(W0, P0, C0, prec=prec) as ctx:
            got[prec], peak[prec] = ctx.device_bytes, ctx.device_bytes_peak
    Tp, Gp = -(-T // 128) * 128, -(-G // 128) * 128
    assert got[0] >= 4 * (4 * Tp * Gp + Tp * Tp + Gp * Gp) and peak[0] == got[0]
    Tp, Gp = -(-T // 256) * 256, -(-G // 256) * 256
    assert got[1] >= 4 * (4 * Tp * Gp + Tp * Tp) + 2 * 2 * Gp * Gp
    # no FP32 C held: less than an FP32 C's 4 Gp^2 on top of the plan, whose largest other item is
    # the running-sum slots of the long products (128 x 256 floats per SM)
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    slots = nsm * 128 * 256 * 4
    assert got[1] < 4 * (4 * Tp * Gp + Tp * Tp) + 2 * 2 * Gp * Gp + slots + 4 * Gp * Gp
    assert got[2] == got[1]
    assert peak[1] == got[1] + 4 * Gp * Gp
    monkeypatch.setenv("PANDA_ALLOC_LIMIT_BYTES", str(peak[1]))
    with panda.PandaContext(W0, P0, C0, prec=1) as ctx:
        assert ctx.device_bytes == got[1]
    monkeypatch.setenv("PANDA_ALLOC_LIMIT_BYTES", str(peak[1] - 1))
    with pytest.raises(panda.PandaError) as e:
        panda.PandaContext(W0, P0, C0, prec=1)
    assert e.value.code == -2


def test_allocation_cap_gives_enomem(panda, monkeypatch):
    W0, P0, C0 = gh.inputs("small64x256")
    monkeypatch.setenv("PANDA_ALLOC_LIMIT_BYTES", "100000")
    with pytest.raises(panda.PandaError) as e:
        panda.PandaContext(W0, P0, C0)
    assert e.value.code == -2
    monkeypatch.delenv("PANDA_ALLOC_LIMIT_BYTES")
    with panda.PandaContext(W0, P0, C0) as ctx:
        ctx.step(0.1)
