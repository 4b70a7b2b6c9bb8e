"""Sets of networks (panda_batch_*): each network of an uneven set must match
the same network run alone (bit for bit) and the FP64 oracle (needs a GB300).
In the tensor-core modes the set runs as one launch per phase over every
network's tiles (persistent CTA pairs over LPT lists), with the schedules of
both phases picked by timing real iterations; any schedule gives the same
bits."""
from __future__ import annotations

import os

import numpy as np
import pytest

import gpu_helpers as gh
from oracle.oracle import Oracle
from paper_1507_07039_gb300 import synth

pytestmark = pytest.mark.gpu


def uneven_set(count=5, seed=77):
    wls = synth.set_of_networks(count, seed=seed, t_range=(10, 150), g_range=(40, 400), n_samples=20,
                                n_factors=3)
    return [synth.make_inputs(w) for w in wls]


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_batch_matches_single_runs_and_oracle(prec):
    from paper_1507_07039_gb300 import panda
    nets = uneven_set()
    with panda.PandaBatch(nets, prec=prec) as b:
        conv, iters, hl = b.run(0.1, 1e-3, 60)
        got = [b.get(k) for k in range(len(b))]
        hist0 = panda.panda_get_history(b.context(0))
    orc = Oracle()
    orc.set_threads(os.cpu_count() or 1)
    for k, (W0, P0, C0) in enumerate(nets):
        single = gh.gpu_run(W0, P0, C0, prec, 0.1, 1e-3, 60)
        assert single["iters"] == iters[k]
        for a, g in zip((single["W"], single["P"], single["C"]), got[k]):
            assert np.array_equal(a, g), f"network {k} differs from its single run"
        o = gh.oracle_run(orc, W0, P0, C0, 0.1, 0.0, iters[k])
        gh.assert_parity({"W": got[k][0], "P": got[k][1], "C": got[k][2]}, o, prec, f"network {k}")
    assert hist0.size == iters[0]


@pytest.mark.parametrize("prec", [1, 3])
def test_batch_runs_in_pieces(prec):
    """Forty fixed iterations split over several calls (the schedule trials
    spread over them, then the captured graph) end where one call of forty
    ends, bit for bit.  (Networks that stop early are covered above.)"""
    from paper_1507_07039_gb300 import panda
    nets = uneven_set(6, seed=91)
    with panda.PandaBatch(nets, prec=prec) as one:
        _, iters1, _ = one.run(0.1, 0.0, 40)
        ref = [one.get(k) for k in range(len(one))]
    with panda.PandaBatch(nets, prec=prec) as b:
        done = np.zeros(len(nets), int)
        for chunk in (1, 2, 1, 3, 33):
            _, it, _ = b.run(0.1, 0.0, chunk)
            done += np.asarray(it)
        got = [b.get(k) for k in range(len(b))]
        sch = b.schedule()
    assert list(done) == list(iters1) == [40] * len(nets)
    for k in range(len(nets)):
        for a, g in zip(ref[k], got[k]):
            assert np.array_equal(a, g), f"network {k} differs"
    # every candidate of both phases was timed (median of three) and the fastest is in use
    assert sch["done"] and len(sch["p1_names"]) == 2 and len(sch["p2_names"]) == 6
    assert all(t > 0 for t in sch["p1_ms"]) and all(t > 0 for t in sch["p2_ms"])
    assert sch["p1"] == int(np.argmin(sch["p1_ms"])) and sch["p2"] == int(np.argmin(sch["p2_ms"]))


def test_batch_with_a_set_sized_network():
    """A network of the set workload's size (250 TFs x 15000 genes, 100
    samples from 10 factors) among small ones, two iterations on the set
    engine: the big network against the FP64 oracle, every network against
    its single run bit for bit."""
    from paper_1507_07039_gb300 import panda
    wl = synth.custom(250, 15000, synth.BASE_SEED + 1999, n_samples=100, n_factors=10, p_density=0.01)
    nets = [synth.make_inputs(wl)] + uneven_set(3, seed=31)
    with panda.PandaBatch(nets, prec=1) as b:
        conv, iters, _ = b.run(0.1, 0.0, 2)
        got = [b.get(k) for k in range(len(b))]
    assert list(iters) == [2] * len(nets)
    for k, (W0, P0, C0) in enumerate(nets):
        single = gh.gpu_run(W0, P0, C0, 1, 0.1, 0.0, 2)
        for a, g in zip((single["W"], single["P"], single["C"]), got[k]):
            assert np.array_equal(a, g), f"network {k} differs from its single run"
    orc = Oracle()
    orc.set_threads(os.cpu_count() or 1)
    W0, P0, C0 = nets[0]
    o = gh.oracle_run(orc, W0, P0, C0, 0.1, 0.0, 2)
    e = gh.assert_parity({"W": got[0][0], "P": got[0][1], "C": got[0][2]}, o, 1, "250 x 15000 in a set")
    print("\n250 x 15000 in a set, 2 iterations: " + ", ".join(f"{k} {v:.3e}" for k, v in e.items()))


def test_batch_mixing_phase2_configurations():
    """A network whose C' tiles are long enough for phase 2's eight-warp,
    three-stage kernel (T = 1400 under BF16X3: 24 k-blocks, 288 MMA slots per
    tile) in a set with small networks (twelve warps, two stages): the set
    runs one phase-2 launch per configuration, each network in the one its
    single run uses, so every network equals its single run bit for bit."""
    from paper_1507_07039_gb300 import panda
    wl = synth.custom(1400, 300, synth.BASE_SEED + 1401, n_samples=40, n_factors=4, p_density=0.01)
    nets = [synth.make_inputs(wl)] + uneven_set(2, seed=13)
    with panda.PandaBatch(nets, prec=1) as b:
        _, iters, _ = b.run(0.1, 0.0, 3)
        got = [b.get(k) for k in range(len(b))]
    assert list(iters) == [3] * len(nets)
    for k, (W0, P0, C0) in enumerate(nets):
        single = gh.gpu_run(W0, P0, C0, 1, 0.1, 0.0, 3)
        for a, g in zip((single["W"], single["P"], single["C"]), got[k]):
            assert np.array_equal(a, g), f"network {k} differs from its single run"
    orc = Oracle()
    orc.set_threads(os.cpu_count() or 1)
    W0, P0, C0 = nets[0]
    o = gh.oracle_run(orc, W0, P0, C0, 0.1, 0.0, 3)
    gh.assert_parity({"W": got[0][0], "P": got[0][1], "C": got[0][2]}, o, 1, "1400 x 300 in a mixed set")


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_cut_tiles_give_the_bits_of_whole_tiles(prec):
    """1000 TFs x 5200 genes: 84 phase-1 tiles on 76 CTA pairs, so a context
    of its own cuts the tiles of its last rounds between two pairs at chunk
    boundaries (panda_phase1_plan), while the set engine runs whole tiles.
    The chunks of every entry are added in the same order either way: the
    network alone and in a set of one agree bit for bit."""
    from paper_1507_07039_gb300 import panda
    W0, P0, C0 = gh.inputs("human1000x5200")
    cuts, _ = panda.panda_phase1_plan(1000, 5200, prec, 76)
    assert cuts > 0
    with panda.PandaBatch([(W0, P0, C0)], prec=prec) as b:
        _, iters, _ = b.run(0.1, 0.0, 3)
        got = b.get(0)
    assert list(iters) == [3]
    single = gh.gpu_run(W0, P0, C0, prec, 0.1, 0.0, 3)
    for a, g in zip((single["W"], single["P"], single["C"]), got):
        assert np.array_equal(a, g), "a context's cut tiles differ from the set engine's whole tiles"


@pytest.mark.parametrize("prec", [1, 3])
def test_batch_diagonal_rule_d2(prec):
    """The set engine under rule D2 (its phase 2 also sums the new
    similarities per row): every network as in its single run, bit for bit,
    and close to the oracle."""
    from paper_1507_07039_gb300 import panda
    nets = uneven_set(4, seed=55)
    with panda.PandaBatch(nets, prec=prec, diag=2) as b:
        conv, iters, hl = b.run(0.1, 0.0, 5)
        got = [b.get(k) for k in range(len(b))]
    orc = Oracle()
    orc.set_threads(os.cpu_count() or 1)
    for k, (W0, P0, C0) in enumerate(nets):
        single = gh.gpu_run(W0, P0, C0, prec, 0.1, 0.0, 5, diag=2)
        for a, g in zip((single["W"], single["P"], single["C"]), got[k]):
            assert np.array_equal(a, g), f"network {k} differs from its single run"
        o = gh.oracle_run(orc, W0, P0, C0, 0.1, 0.0, 5, diag=2)
        gh.assert_parity({"W": got[k][0], "P": got[k][1], "C": got[k][2]}, o, prec, f"network {k}")


@pytest.mark.parametrize("prec", [0, 1, 3])
def test_batch_of_degenerate_shapes(prec):
    """Single nodes, a single TF, single genes and ragged tiles in one set
    (without normalisation: a 1 x 1 network has no spread to Z-score), each
    network as in its single run, bit for bit, and close to the oracle."""
    from paper_1507_07039_gb300 import panda
    rng = np.random.default_rng(9)
    nets = []
    for T, G in ((1, 1), (1, 5), (3, 1), (2, 3), (129, 257), (300, 40)):
        W0 = rng.standard_normal((T, G)).astype(np.float32)
        nets.append((W0, gh.random_symmetric(rng, T), gh.random_symmetric(rng, G)))
    with panda.PandaBatch(nets, prec=prec, normalize=False) as b:
        conv, iters, hl = b.run(0.2, 0.0, 3)
        got = [b.get(k) for k in range(len(b))]
    assert list(iters) == [3] * len(nets)
    orc = Oracle()
    orc.set_threads(os.cpu_count() or 1)
    for k, (W0, P0, C0) in enumerate(nets):
        single = gh.gpu_run(W0, P0, C0, prec, 0.2, 0.0, 3, normalize=False)
        for a, g in zip((single["W"], single["P"], single["C"]), got[k]):
            assert np.array_equal(a, g), f"network {k} differs from its single run"
        o = gh.oracle_run(orc, W0, P0, C0, 0.2, 0.0, 3, normalize=False)
        gh.assert_parity({"W": got[k][0], "P": got[k][1], "C": got[k][2]}, o, prec, f"network {k}")
    with pytest.raises(panda.PandaError) as e:
        panda.PandaBatch([], prec=prec)
    assert e.value.code == -1


def test_batch_errors_name_the_network():
    from paper_1507_07039_gb300 import panda
    nets = uneven_set(3)
    W0, P0, C0 = nets[1]
    bad = C0.copy()
    bad[0, 1] += 1.0
    nets[1] = (W0, P0, bad)
    with pytest.raises(panda.PandaError) as e:
        panda.PandaBatch(nets)
    assert e.value.code == -5 and "network 1" in str(e.value)
