"""The FP64 oracle against the facts that pin it (CPU only)."""
import pytest

from oracle.oracle import Oracle
import pins


@pytest.fixture(scope="module")
def orc():
    return Oracle()


@pytest.mark.parametrize("pin", pins.PINS, ids=lambda f: f.__name__)
def test_pin(orc, pin):
    pin(orc)


def test_thread_count_does_not_change_results(orc):
    import numpy as np
    W, P, C = orc.normalize(*pins._small_inputs(9, 40, 41))
    orc.set_threads(1)
    a = orc.step(W, P, C, 0.1, 1)
    orc.set_threads(4)
    b = orc.step(W, P, C, 0.1, 1)
    orc.set_threads(1)
    for x, y in zip(a, b):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def test_rows_match_full_step(orc):
    import numpy as np
    W, P, C = orc.normalize(*pins._small_inputs(6, 11, 43))
    Wn, Pn, Cn, _ = orc.step(W, P, C, 0.1, 1)
    rows = [0, 3, 5]
    assert np.array_equal(orc.w_rows(W, P, C, 0.1, rows), Wn[rows])
    for j in (0, 4, 10):
        assert np.array_equal(orc.w_col(W, P, C, 0.1, j), Wn[:, j])
    pr = orc.p_rows(Wn, P, 0.1, rows)
    cr = orc.c_rows(Wn, C, 0.1, [1, 7])
    for q, i in enumerate(rows):
        off = np.arange(6) != i
        assert np.array_equal(pr[q][off], Pn[i][off])
    for q, k in enumerate([1, 7]):
        off = np.arange(11) != k
        assert np.array_equal(cr[q][off], Cn[k][off])


def test_rejects_asymmetric(orc):
    import numpy as np
    W, P, C = pins._tiny_state(np.random.default_rng(1), 3, 4)
    C[0, 1] += 1.0
    with pytest.raises(ValueError):
        orc.step(W, P, C, 0.1, 1)
