"""The oracle against the worked examples of tests/golden/ (values derived
by hand from the paper's equations, each file citing the passage it
follows): Eq. 1 on worked vectors, one whole iteration (Eqs. 1-7, rule D1)
of a 2 x 3 network with identity priors at alpha = 1 and 0.1, and the
Pearson prior of Sec. II-A on a 3 x 3 case."""
from __future__ import annotations

import numpy as np
import pytest

import golden


@pytest.fixture(scope="module")
def orc():
    from oracle.oracle import Oracle
    return Oracle()


def test_tanimoto_worked_values(orc):
    for x, y, want in golden.tanimoto_cases():
        assert orc.tanimoto(x, y) == pytest.approx(want, rel=1e-15, abs=1e-15), (x, y)


def test_one_iteration_worked_by_hand(orc):
    g = golden.step_2x3()
    for case in g["cases"]:
        Wn, Pn, Cn, h = orc.step(g["W"], g["P"], g["C"], case["alpha"], 1)
        np.testing.assert_allclose(Wn, case["W"], rtol=0, atol=1e-15)
        assert h == pytest.approx(case["h"], rel=1e-14)
        if "P" in case:
            np.testing.assert_allclose(Pn, case["P"], rtol=0, atol=1e-15)
            np.testing.assert_allclose(Cn, case["C"], rtol=1e-14, atol=1e-15)


def test_pearson_worked_case(orc):
    X, R = golden.pearson_3x3()
    np.testing.assert_allclose(orc.pearson(X), R, rtol=0, atol=1e-15)


def test_fixtures_are_what_they_say():
    g = golden.step_2x3()
    assert g["W"].shape == (2, 3) and np.array_equal(g["P"], np.eye(2)) and np.array_equal(g["C"], np.eye(3))
    assert [c["alpha"] for c in g["cases"]] == [1.0, 0.1]
    assert len(golden.tanimoto_cases()) == 5
