"""How phase 1 spreads a network's W' tiles (Eqs. 2-3 and 7) over the
persistent CTA pairs: panda_phase1_plan is host code, so these run on the CPU.

Every 256 x 256 tile's availability sum is cut into chunks of 32 k-blocks;
whole tiles run in rounds, and when that leaves the busiest pair more than 5%
above the average the last two rounds are cut at chunk boundaries into equal
shares.
Checked: every chunk of every tile is computed exactly once, a cut tile has
exactly two pieces on two different pairs that share one cut index, a head
piece (which others wait for) runs on its pair before anything that waits and
after the whole-tile rounds (which every pair runs in step), a tail piece
(which waits) runs last, the MMA work per pair is balanced, and nothing is cut
when the pairs are not known to be resident together."""
from __future__ import annotations

import numpy as np
import pytest


@pytest.fixture(scope="module", autouse=True)
def library():
    from paper_1507_07039_gb300 import build
    build.build()


def chunk_costs(T, G, prec):
    """MMA issue slots per chunk of one tile, the last chunk carrying the
    responsibility numerator and the epilogue (64 slots)."""
    Tp, Gp = -(-T // 256) * 256, -(-G // 256) * 256
    fp8, terms = prec == 3, (2 if prec == 2 else 3)
    nA, nR = Gp // (128 if fp8 else 64), Tp // 64
    nc = -(-nA // 32)
    cost = [(4 if fp8 else 4 * terms) * min(32, nA - 32 * c) for c in range(nc)]
    cost[-1] += 4 * terms * nR + 64
    return Tp // 256, Gp // 256, nc, cost


def check_plan(T, G, prec, pairs, resident=True):
    from paper_1507_07039_gb300 import panda
    cuts, pc = panda.panda_phase1_plan(T, G, prec, pairs, resident)
    nmt, nnt, nc, cost = chunk_costs(T, G, prec)
    used = min(pairs, nmt * nnt)
    assert set(pc[:, 0]) == set(range(used))
    pieces = {}
    for p, mt, nt, c0, c1, cut in pc:
        pieces.setdefault((int(mt), int(nt)), []).append((int(c0), int(c1), int(cut), int(p)))
    assert sorted(pieces) == [(m, n) for m in range(nmt) for n in range(nnt)]
    for tile, v in pieces.items():
        v.sort()
        assert v[0][0] == 0 and v[-1][1] == nc, (tile, v)
        assert all(a[1] == b[0] and a[0] < a[1] for a, b in zip(v, v[1:])), (tile, v)
        if len(v) == 1:
            assert v[0][2] == -1
        else:
            assert len(v) == 2 and v[0][2] == v[1][2] >= 0 and v[0][3] != v[1][3], (tile, v)
    assert sorted({int(c) for c in pc[:, 5] if c >= 0}) == list(range(cuts))
    load = np.zeros(used)
    # the whole-tile rounds: pair p's first tiles are p, p + pairs, ... of the gene-block-major order
    ndp = (nmt * nnt // used - 1) * used if cuts else nmt * nnt
    for p in range(used):
        rows = pc[pc[:, 0] == p]
        dp = [(q % nmt, q // nmt) for q in range(p, ndp, used)]
        assert [(int(r[1]), int(r[2])) for r in rows[:len(dp)]] == dp, f"pair {p}: rounds out of step"
        assert all(r[5] == -1 for r in rows[:len(dp)])
        for i, (_, _, _, c0, c1, cut) in enumerate(rows):
            if cut >= 0 and c0 == 0:
                assert i == len(dp), f"pair {p}: a head piece not right after the rounds"
            if cut >= 0 and c0 > 0:
                assert i == len(rows) - 1, f"pair {p}: a tail piece that is not last"
            load[p] += sum(cost[c0:c1])
    whole = np.zeros(used)
    for q in range(nmt * nnt):
        whole[q % used] += sum(cost)
    return cuts, load.max() / load.mean(), whole.max() / whole.mean()


@pytest.mark.parametrize("prec", [1, 2, 3])
@pytest.mark.parametrize("T,G", [(1000, 17000), (1600, 30000), (1000, 5200), (700, 23000), (1024, 46080),
                                 (250, 15000), (2000, 2000), (300, 40), (1, 1)])
def test_every_chunk_once_heads_first_tails_last(T, G, prec):
    cuts, bal, whole = check_plan(T, G, prec, 76)
    assert bal <= whole + 1e-12
    if cuts == 0:
        assert bal == pytest.approx(whole)


def test_human_sized_network_is_balanced():
    """1000 x 17000: 4 x 67 = 268 tiles on 76 pairs leave 36 pairs idle for
    the last 12% of a whole-tile schedule; the cut one is within 1%."""
    cuts, bal, whole = check_plan(1000, 17000, 1, 76)
    assert whole == pytest.approx(4 / (268 / 76))
    assert cuts > 0 and bal < 1.01


def test_no_cuts_where_whole_tiles_are_nearly_even():
    """1600 x 30000: 7 x 118 = 826 tiles on 76 pairs, the busiest pair 1.2%
    above the average: whole tiles only."""
    cuts, bal, whole = check_plan(1600, 30000, 1, 76)
    assert cuts == 0 and whole == pytest.approx(11 / (826 / 76))


def test_no_cuts_without_co_resident_pairs():
    cuts, bal, whole = check_plan(1000, 17000, 1, 76, resident=False)
    assert cuts == 0 and bal == pytest.approx(whole)


@pytest.mark.parametrize("pairs", [1, 2, 3, 7, 74, 76, 300])
def test_any_pair_count(pairs):
    check_plan(1000, 17000, 1, pairs)


def test_bad_arguments_are_refused():
    from paper_1507_07039_gb300 import panda
    for args in ((0, 10, 1, 76), (10, 0, 1, 76), (10, 10, 0, 76), (10, 10, 1, 0)):
        with pytest.raises(panda.PandaError):
            panda.panda_phase1_plan(*args)


@pytest.mark.parametrize("T,G,pairs", [(1000, 17000, 76), (1000, 5200, 76), (700, 23000, 76), (1600, 30000, 76),
                                       (1000, 17000, 3), (1000, 17000, 7)])
def test_pieces_run_to_the_end_and_balance(T, G, pairs):
    """Every pair runs its list in order; a tail piece may not start before
    the head of its tile has finished (a stricter rule than the kernel's,
    which waits only before touching the running sum).  Played out in MMA
    slots, every list ends (no pair waits on a piece that waits itself) and
    the last pair ends within 2% of an even split of the work whenever tiles
    were cut (within one chunk's worth of it for coarse chunks)."""
    from paper_1507_07039_gb300 import panda
    cuts, pc = panda.panda_phase1_plan(T, G, 1, pairs)
    nmt, nnt, nc, cost = chunk_costs(T, G, 1)
    lists = {}
    for row in pc:
        lists.setdefault(int(row[0]), []).append(tuple(int(x) for x in row[1:]))
    head_end, pos, t = {}, {p: 0 for p in lists}, {p: 0.0 for p in lists}
    for _ in range(sum(len(v) for v in lists.values()) + 1):
        moved = False
        for p, items in lists.items():
            while pos[p] < len(items):
                mt, nt, c0, c1, cut = items[pos[p]]
                start = t[p]
                if cut >= 0 and c0 > 0:
                    if cut not in head_end:
                        break
                    start = max(start, head_end[cut])
                t[p] = start + sum(cost[c0:c1])
                if cut >= 0 and c0 == 0:
                    head_end[cut] = t[p]
                pos[p] += 1
                moved = True
        if not moved:
            break
    assert all(pos[p] == len(items) for p, items in lists.items()), "a pair never finished its list"
    total = sum(sum(cost) for _ in range(nmt * nnt))
    ideal = total / len(lists)
    if cuts:
        assert max(t.values()) <= ideal * 1.02 + max(cost)
    if T == 1000 and G == 17000 and pairs == 76:
        assert max(t.values()) <= ideal * 1.02
