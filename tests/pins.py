"""Pins for the FP64 oracle: facts the paper and the mathematics fix.

Each ``pin_*`` function takes an :class:`oracle.oracle.Oracle` and raises
``AssertionError`` when the oracle disagrees with the fact it checks.  They are
run against the real oracle (``test_oracle_pins.py``) and against builds of the
oracle with a planted mistake (``test_oracle_planted.py``), every one of which
must trip at least one pin.

None of these re-types the oracle's own code: the expected values are closed
forms, hand-worked numbers, library routines standing in for a special case,
or a different statement of the same operation (the matrix form of Eq. 9).
"""
from __future__ import annotations

import math

import numpy as np

from oracle.oracle import DIAG_D0, DIAG_D1, DIAG_D2

SQ2 = math.sqrt(2.0)


def _close(got, want, tol, what=""):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    assert got.shape == want.shape, (what, got.shape, want.shape)
    assert np.all(np.isfinite(got)), (what, "non-finite")
    err = float(np.max(np.abs(got - want))) if got.size else 0.0
    assert err <= tol, f"{what}: max abs err {err:.3e} > {tol:.1e}"


# ---------------------------------------------------------------------------
# Eq. 1: closed forms of the similarity
# ---------------------------------------------------------------------------

def pin_tanimoto_closed_forms(orc):
    # Tan(x, x) = x.x / sqrt(2|x|^2 - |x|^2) = |x|; (3, 4) has norm 5.
    _close(orc.tanimoto([3.0, 4.0], [3.0, 4.0]), 5.0, 1e-15, "Tan(x,x)")
    # Tan(x, -x) = -|x|
    _close(orc.tanimoto([3.0, 4.0], [-3.0, -4.0]), -5.0, 1e-15, "Tan(x,-x)")
    # (1,0) vs (1,1): 1 / sqrt(1 + 2 - 1) = 1/sqrt(2)
    _close(orc.tanimoto([1.0, 0.0], [1.0, 1.0]), 1.0 / SQ2, 1e-15, "Tan(e1, 1)")
    # orthogonal vectors give 0
    _close(orc.tanimoto([1.0, 2.0, 0.0], [-2.0, 1.0, 5.0]), 0.0, 1e-15, "orthogonal")
    # two zero vectors: defined as 0
    _close(orc.tanimoto([0.0, 0.0], [0.0, 0.0]), 0.0, 0.0, "zero vectors")
    # (1,2,2) vs (2,0,1): dot 4, norms 9 and 5: 4 / sqrt(9 + 5 - 4) = 4/sqrt(10)
    _close(orc.tanimoto([1.0, 2.0, 2.0], [2.0, 0.0, 1.0]), 4.0 / math.sqrt(10.0), 1e-15, "worked")
    # (1,2,2) vs (-2,0,-1): dot -4: -4/sqrt(10) (the |x.y| keeps the denominator)
    _close(orc.tanimoto([1.0, 2.0, 2.0], [-2.0, 0.0, -1.0]), -4.0 / math.sqrt(10.0), 1e-15,
           "worked, negative")


def pin_tanimoto_properties(orc):
    rng = np.random.default_rng(11)
    for n in (1, 2, 7, 33):
        for _ in range(10):
            x, y = rng.standard_normal(n), rng.standard_normal(n)
            c = float(rng.uniform(0.1, 10.0))
            t = orc.tanimoto(x, y)
            _close(orc.tanimoto(y, x), t, 0.0, "symmetry")
            _close(orc.tanimoto(c * x, c * y), c * t, 1e-12 * max(1.0, abs(c * t)), "scaling")
            bound = math.sqrt(np.linalg.norm(x) * np.linalg.norm(y))
            assert abs(t) <= bound * (1 + 1e-12), "bound |Tan| <= sqrt(|x||y|)"
            # parallel vectors: c|x|^2 / sqrt(|x|^2 (1 + c^2 - c)) = c|x| / sqrt(1 - c + c^2)
            nx = float(np.linalg.norm(x))
            _close(orc.tanimoto(x, c * x), c * nx / math.sqrt(1.0 - c + c * c),
                   1e-12 * max(1.0, c * nx), "parallel")


# ---------------------------------------------------------------------------
# Normalisation
# ---------------------------------------------------------------------------

def pin_zscore(orc):
    # [1,2,3,4]: mean 2.5, population std sqrt(1.25)
    z = orc.zscore([1.0, 2.0, 3.0, 4.0])
    s = math.sqrt(1.25)
    _close(z, [-1.5 / s, -0.5 / s, 0.5 / s, 1.5 / s], 1e-15, "zscore [1,2,3,4]")
    a = np.random.default_rng(3).standard_normal(1000) * 7.0 + 3.0
    z = orc.zscore(a)
    _close(np.mean(z), 0.0, 1e-13, "zscore mean")
    _close(np.std(z), 1.0, 1e-13, "zscore population std")
    try:
        orc.zscore([2.0, 2.0, 2.0])
    except ValueError:
        pass
    else:
        raise AssertionError("zscore of a constant must fail")


# ---------------------------------------------------------------------------
# Eq. 9: the matrix form, written as the paper's Tfunction over numpy
# ---------------------------------------------------------------------------

def tfunction(X, Y):
    """Eq. 9: X*Y, then the column sums of Y.^2 and row sums of X.^2 repeated to
    the output's shape, then the elementwise divide."""
    Amat = X @ Y
    Bmat = np.tile(np.sum(Y ** 2, axis=0), (X.shape[0], 1))
    Cmat = np.tile(np.sum(X ** 2, axis=1)[:, None], (1, Y.shape[1]))
    return Amat / np.sqrt(Bmat + Cmat - np.abs(Amat))


def matrix_form_step(W, P, C, alpha, t, diag):
    """One iteration in the matrix form: R = Tfunction(P, W), A = Tfunction(W, C),
    then W, then P and C from the new W and their diagonals."""
    T, G = W.shape
    R = tfunction(P, W)
    A = tfunction(W, C)
    Wn = (1 - alpha) * W + alpha / 2 * (A + R)
    h = np.mean(np.abs(Wn - W))
    SP = tfunction(Wn, Wn.T)
    SC = tfunction(Wn.T, Wn)
    Pn = (1 - alpha) * P + alpha * SP
    Cn = (1 - alpha) * C + alpha * SC
    gain = 1.0 if diag == DIAG_D0 else alpha
    for X, Xold, S, n, mult in ((Pn, P, SP, T, G), (Cn, C, SC, G, T)):
        src = S if diag == DIAG_D2 else X
        off = ~np.eye(n, dtype=bool)
        for i in range(n):
            sig = np.std(src[i][off[i]]) if n > 1 else 0.0
            X[i, i] = (1 - alpha) * Xold[i, i] + gain * mult * sig * math.exp(2 * alpha * t)
    return Wn, Pn, Cn, h


def _tiny_state(rng, T, G):
    W = rng.standard_normal((T, G))
    P = rng.standard_normal((T, T))
    P = (P + P.T) / 2
    C = rng.standard_normal((G, G))
    C = (C + C.T) / 2
    return W, P, C


def pin_matrix_form(orc):
    rng = np.random.default_rng(5)
    for (T, G) in ((1, 1), (1, 4), (3, 1), (2, 3), (4, 7), (8, 8), (5, 8)):
        W, P, C = _tiny_state(rng, T, G)
        for alpha, t, diag in ((0.1, 1, DIAG_D1), (0.3, 4, DIAG_D0), (0.7, 2, DIAG_D2), (1.0, 3, DIAG_D1)):
            got = orc.step(W, P, C, alpha, t, diag)
            want = matrix_form_step(W, P, C, alpha, t, diag)
            for name, g, w in zip(("W", "P", "C", "h"), got, want):
                scale = max(1.0, float(np.max(np.abs(w))))
                _close(g, w, 1e-12 * scale, f"matrix form {name} T={T} G={G} a={alpha} d={diag}")


# ---------------------------------------------------------------------------
# Identity priors: closed forms of R and A (Section II-A default priors)
# ---------------------------------------------------------------------------

def pin_identity_priors(orc):
    rng = np.random.default_rng(9)
    T, G = 5, 7
    W = rng.standard_normal((T, G))
    P, C = np.eye(T), np.eye(G)
    colsq = np.sum(W * W, axis=0)  # |W_.j|^2
    rowsq = np.sum(W * W, axis=1)  # |W_i.|^2
    for i in range(T):
        for j in range(G):
            w = W[i, j]
            r = w / math.sqrt(1.0 + colsq[j] - abs(w))       # Tan(e_i, W_.j)
            a = w / math.sqrt(rowsq[i] + 1.0 - abs(w))       # Tan(W_i., e_j)
            _close(orc.responsibility(W, P, i, j), r, 1e-14, "R with P = I")
            _close(orc.availability(W, C, i, j), a, 1e-14, "A with C = I")
            _close(orc.w_entry(W, P, C, 0.25, i, j), 0.75 * w + 0.125 * (r + a), 1e-14, "W' with I priors")


# ---------------------------------------------------------------------------
# alpha = 0 and alpha = 1
# ---------------------------------------------------------------------------

def pin_alpha_zero(orc):
    rng = np.random.default_rng(13)
    W, P, C = _tiny_state(rng, 4, 6)
    for diag in (DIAG_D1, DIAG_D2):
        Wn, Pn, Cn, h = orc.step(W, P, C, 0.0, 3, diag)
        _close(Wn, W, 0.0, "alpha=0 W")
        _close(Pn, P, 0.0, "alpha=0 P")
        _close(Cn, C, 0.0, "alpha=0 C")
        assert h == 0.0, "alpha=0 h"
    # the literal rule D0 still moves the diagonals by N * sigma * e^0 = N * sigma
    Wn, Pn, Cn, h = orc.step(W, P, C, 0.0, 3, DIAG_D0)
    for X, X0, n, mult in ((Pn, P, 4, 6), (Cn, C, 6, 4)):
        off = ~np.eye(n, dtype=bool)
        want = np.diag(X0) + mult * np.array([np.std(X0[i][off[i]]) for i in range(n)])
        _close(np.diag(X), want, 1e-12, "alpha=0, D0 diagonal")


def pin_alpha_one(orc):
    rng = np.random.default_rng(17)
    T, G = 3, 5
    W = rng.standard_normal((T, G))
    P, C = np.eye(T), np.eye(G)
    Wn, Pn, Cn, _ = orc.step(W, P, C, 1.0, 2, DIAG_D1)
    colsq, rowsq = np.sum(W * W, axis=0), np.sum(W * W, axis=1)
    R = W / np.sqrt(1.0 + colsq[None, :] - np.abs(W))
    A = W / np.sqrt(rowsq[:, None] + 1.0 - np.abs(W))
    _close(Wn, (R + A) / 2, 1e-14, "alpha=1 W' = (R + A)/2")
    for i in range(T):
        for m in range(T):
            if i != m:
                _close(Pn[i, m], orc.tanimoto(Wn[i], Wn[m]), 1e-15, "alpha=1 P'_off")
    for k in range(G):
        for j in range(G):
            if k != j:
                _close(Cn[k, j], orc.tanimoto(Wn[:, k], Wn[:, j]), 1e-15, "alpha=1 C'_off")
    # D1 with alpha = 1: X'_ii = N * sigma_i * e^{2 t}
    e = math.exp(2.0 * 2)
    for X, n, mult in ((Pn, T, G), (Cn, G, T)):
        off = ~np.eye(n, dtype=bool)
        want = np.array([mult * np.std(X[i][off[i]]) * e for i in range(n)])
        _close(np.diag(X), want, 1e-12 * max(1.0, float(np.max(want))), "alpha=1 diagonal")


# ---------------------------------------------------------------------------
# Hand-worked 2 x 3 example (no normalisation)
# ---------------------------------------------------------------------------
#
# W = [[1, 0, 1], [0, 1, 1]], P = I_2, C = I_3, t = 1, rule D1.
# Column norms |W_.j|^2 = (1, 1, 2); row norms |W_i.|^2 = (2, 2).
# With P = I, R_ij = W_ij / sqrt(1 + |W_.j|^2 - |W_ij|):
#     R = [[1, 0, 1/sqrt2], [0, 1, 1/sqrt2]]
# With C = I, A_ij = W_ij / sqrt(|W_i.|^2 + 1 - |W_ij|):
#     A = [[1/sqrt2, 0, 1/sqrt2], [0, 1/sqrt2, 1/sqrt2]]
#
# alpha = 1: W' = (R + A)/2 = [[a, 0, b], [0, a, b]] with
#     a = (1 + 1/sqrt2)/2 = 0.85355339..., b = 1/sqrt2 = 0.70710678...
#   h = (2(1 - a) + 2(1 - b)) / 6 = (1 - 1/sqrt2)/2 = 0.14644661...
#   P'_01 = Tan((a,0,b), (0,a,b)) = b^2 / sqrt(2a^2 + 2b^2 - b^2)
#         = 0.5 / sqrt(2a^2 + 0.5) = 1/sqrt(5 + 2 sqrt2) = 0.35740674...
#   columns of W': (a,0), (0,a), (b,b)
#   C'_01 = 0 (orthogonal);  C'_02 = C'_12 = ab / sqrt(a^2 + 2b^2 - ab);
#         ab = (sqrt2 + 1)/4, a^2 - ab = a(a - b) = 1/8, so the root is
#         sqrt(9/8) and C'_02 = (2 + sqrt2)/6 = 0.56903559...
#   diagonals (alpha = 1, t = 1, factor e^2):
#     P: each row has one off-diagonal entry, sigma = 0, so P'_ii = 0.
#     C: rows 0 and 1 hold {0, s} (s = C'_02), sigma = s/2, and N_e = 2:
#        C'_00 = C'_11 = 2 * (s/2) * e^2 = s e^2 = 4.20463592...
#        row 2 holds {s, s}, sigma = 0, so C'_22 = 0.
#
# alpha = 0.1: W' = 0.9 W + 0.05 (R + A):
#   W'_00 = W'_11 = 0.9 + 0.05 (1 + 1/sqrt2) = 0.98535534...
#   W'_02 = W'_12 = 0.9 + 0.05 sqrt2 = 0.97071068...; zeros stay 0.

HAND_W = np.array([[1.0, 0.0, 1.0], [0.0, 1.0, 1.0]])


def pin_hand_2x3(orc):
    W, P, C = HAND_W, np.eye(2), np.eye(3)
    a, b = (1 + 1 / SQ2) / 2, 1 / SQ2
    s = (2 + SQ2) / 6
    Wn, Pn, Cn, h = orc.step(W, P, C, 1.0, 1, DIAG_D1)
    _close(Wn, [[a, 0, b], [0, a, b]], 1e-15, "hand alpha=1 W'")
    _close(h, (1 - 1 / SQ2) / 2, 1e-15, "hand alpha=1 h")
    p01 = 1 / math.sqrt(5 + 2 * SQ2)
    _close(Pn, [[0.0, p01], [p01, 0.0]], 1e-15, "hand alpha=1 P'")
    e2 = math.exp(2.0)
    _close(Cn, [[s * e2, 0.0, s], [0.0, s * e2, s], [s, s, 0.0]], 1e-14, "hand alpha=1 C'")

    Wn, Pn, Cn, h = orc.step(W, P, C, 0.1, 1, DIAG_D1)
    w0, w2 = 0.9 + 0.05 * (1 + 1 / SQ2), 0.9 + 0.05 * SQ2
    _close(Wn, [[w0, 0, w2], [0, w0, w2]], 1e-15, "hand alpha=0.1 W'")
    _close(h, (2 * (1 - w0) + 2 * (1 - w2)) / 6, 1e-15, "hand alpha=0.1 h")


# ---------------------------------------------------------------------------
# Structure: symmetry, equivariance, stop rule
# ---------------------------------------------------------------------------

def _small_inputs(T=6, G=9, seed=21):
    from paper_1507_07039_gb300 import synth
    wl = synth.custom(T, G, seed, n_samples=12, n_factors=3, w_density=0.3, p_density=0.3)
    W0, P0, C0 = synth.make_inputs(wl)
    return [np.asarray(x, dtype=np.float64) for x in (W0, P0, C0)]


def pin_symmetry(orc):
    W, P, C = orc.normalize(*_small_inputs())
    for t in range(1, 4):
        W, P, C, _ = orc.step(W, P, C, 0.1, t, DIAG_D1)
        assert np.array_equal(P, P.T), "P' symmetric"
        assert np.array_equal(C, C.T), "C' symmetric"


def pin_permutation_equivariance(orc):
    W, P, C = orc.normalize(*_small_inputs(7, 10, 23))
    rng = np.random.default_rng(29)
    pg, pt = rng.permutation(W.shape[1]), rng.permutation(W.shape[0])
    base = orc.step(W, P, C, 0.2, 2, DIAG_D1)
    got = orc.step(W[pt][:, pg], P[pt][:, pt], C[pg][:, pg], 0.2, 2, DIAG_D1)
    _close(got[0], base[0][pt][:, pg], 1e-12, "equivariance W")
    _close(got[1], base[1][pt][:, pt], 1e-10, "equivariance P")
    _close(got[2], base[2][pg][:, pg], 1e-10, "equivariance C")
    _close(got[3], base[3], 1e-14, "equivariance h")


def pin_h_and_stop_rule(orc):
    W, P, C = orc.normalize(*_small_inputs(5, 8, 31))
    Wn, _, _, h = orc.step(W, P, C, 0.1, 1, DIAG_D1)
    _close(h, np.mean(np.abs(Wn - W)), 1e-15, "h = mean |W' - W| (Eq. 7)")
    # the stop test is strict and taken after the whole iteration
    _, _, _, n, hist, conv = orc.run(W, P, C, 0.1, 1e-3, 500)
    assert conv and n >= 2 and hist[-1] < 1e-3 and np.all(hist[:-1] >= 1e-3), "stop rule"
    _, _, _, n2, hist2, conv2 = orc.run(W, P, C, 0.1, 1e-3, n - 1)
    assert (not conv2) and n2 == n - 1, "max_iter reached"
    _close(hist2, hist[:n - 1], 0.0, "history prefix")
    # tol = h exactly: h < tol is false, so the loop continues
    _, _, _, n3, _, _ = orc.run(W, P, C, 0.1, hist[0], 2)
    assert n3 == 2, "h == tol continues"


def pin_pearson(orc):
    """Sec. II-A: the initial co-regulation network is the Pearson correlation
    of the genes' expression across samples."""
    rng = np.random.default_rng(61)
    # a library routine of the same definition
    for G, N in ((7, 13), (40, 25)):
        X = rng.standard_normal((G, N)) * rng.uniform(0.5, 3.0, (G, 1)) + rng.uniform(-2, 2, (G, 1))
        _close(orc.pearson(X), np.corrcoef(X), 1e-12, "numpy corrcoef")
    # a worked case: rows 1 and 2 are affine images (r = 1), row 3 reversed (r = -1)
    X = np.array([[1.0, 2.0, 3.0], [2.0, 4.0, 6.0], [3.0, 2.0, 1.0]])
    _close(orc.pearson(X), np.array([[1, 1, -1], [1, 1, -1], [-1, -1, 1]], float), 1e-15, "hand 3 x 3")
    # invariance under a positive scale and shift of a row; a negated row flips its sign
    X = rng.standard_normal((9, 30))
    C = orc.pearson(X)
    Y = X.copy()
    Y[4] = 7.5 * Y[4] - 3.0
    _close(orc.pearson(Y), C, 1e-13, "affine invariance")
    Y = X.copy()
    Y[2] = -Y[2]
    D = C.copy()
    D[2, :] *= -1
    D[:, 2] *= -1
    _close(orc.pearson(Y), D, 1e-13, "negated row")
    # symmetric, unit diagonal, |r| <= 1 (Cauchy-Schwarz)
    assert np.array_equal(C, C.T) and np.all(np.diag(C) == 1.0) and np.all(np.abs(C) <= 1.0 + 1e-15)
    # a constant gene has no correlation
    X[5] = 2.0
    try:
        orc.pearson(X)
    except ValueError:
        pass
    else:
        raise AssertionError("zero-variance row accepted")


PINS = [
    pin_pearson,
    pin_tanimoto_closed_forms,
    pin_tanimoto_properties,
    pin_zscore,
    pin_matrix_form,
    pin_identity_priors,
    pin_alpha_zero,
    pin_alpha_one,
    pin_hand_2x3,
    pin_symmetry,
    pin_permutation_equivariance,
    pin_h_and_stop_rule,
]
