"""Seeded synthetic inputs shaped like the paper's networks.

This module draws prior networks only; it holds none of the message-passing
arithmetic (no similarity, no normalisation, no update rule) and serves the
oracle and the CUDA path alike.

Recipe (numpy PCG64, FP64 on the host, rounded once to FP32, the library's
input type; the oracle receives the same FP32 values widened to FP64):

* ``W0`` (T x G): iid Bernoulli(``w_density``) 0/1 entries, the motif prior of
  Section II-A (a TF-gene edge where a binding motif is found).
* ``P0`` (T x T): iid Bernoulli(``p_density``) on the strict upper triangle,
  mirrored, unit diagonal: a protein-interaction prior.
* ``C0`` (G x G): Pearson correlation of genes across samples of a synthetic
  expression matrix ``X = L F + E`` (``L`` G x k, ``F`` k x n, iid N(0,1);
  ``E`` iid N(0, 0.5^2)), the co-expression prior of Section II-A.  Exactly
  symmetric with unit diagonal.
* Identity priors (``P0 = I``, ``C0 = I``) are the paper's default when PPI or
  expression data are missing, and the workload of its Table I.

The draw order is fixed: W, then P, then L, F, E.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

BASE_SEED = 150707039


@dataclass(frozen=True)
class Workload:
    name: str
    T: int                 # transcription factors (effector nodes, N_e)
    G: int                 # genes (affected nodes, N_a)
    n_samples: int = 0     # expression samples; 0 = identity P and C
    n_factors: int = 0
    w_density: float = 0.05
    p_density: float = 0.01
    seed: int = BASE_SEED

    @property
    def identity_priors(self) -> bool:
        return self.n_samples == 0


WORKLOADS = {
    # 64 TFs x 256 genes, 50 samples from 5 factors: the small case.
    "small64x256": Workload("small64x256", 64, 256, 50, 5, 0.05, 0.02, BASE_SEED + 0),
    # ~human-sized: 1000 TFs x 17000 genes, 200 samples from 20 factors.
    "human1000x17000": Workload("human1000x17000", 1000, 17000, 200, 20, 0.05, 0.01, BASE_SEED + 1),
    # large network: 1600 TFs x 30000 genes, 300 samples from 30 factors.
    "large1600x30000": Workload("large1600x30000", 1600, 30000, 300, 30, 0.05, 0.01, BASE_SEED + 4),
    # profiling case: same TF count, C (268 MB) still larger than L2, a few GB on the device.
    "prof1000x8192": Workload("prof1000x8192", 1000, 8192, 100, 10, 0.05, 0.01, BASE_SEED + 8),
    # the human-sized generators at fewer genes: 1000 TFs (ragged in 256-tiles) x 5200 genes,
    # two waves of phase-1 tiles and a ragged last gene tile; cheap enough for the oracle to
    # follow a whole converging trajectory.
    "human1000x5200": Workload("human1000x5200", 1000, 5200, 200, 20, 0.05, 0.01, BASE_SEED + 9),
    # mid-size parity case spanning many tiles with ragged edges.
    "mid250x2100": Workload("mid250x2100", 250, 2100, 100, 10, 0.05, 0.02, BASE_SEED + 7),
}


def get(name: str) -> Workload:
    return WORKLOADS[name]


def custom(T: int, G: int, seed: int, n_samples: int = 40, n_factors: int = 4,
           w_density: float = 0.05, p_density: float = 0.02) -> Workload:
    return Workload(f"custom{T}x{G}s{seed}", T, G, n_samples, n_factors, w_density, p_density, seed)


def table1(n: int, rep: int = 0) -> Workload:
    """The paper's Table I shape: N_e = N_a = n, identity P and C, random W."""
    return Workload(f"table1_{n}_{rep}", n, n, 0, 0, 0.05, 0.0, BASE_SEED + 5000 + 10 * n + rep)


def set_of_networks(count: int = 64, seed: int = BASE_SEED + 1000, t_range=(200, 1000),
                    g_range=(2000, 17000), n_samples: int = 100, n_factors: int = 10):
    """Uneven networks: T ~ U[t_range], G ~ U[g_range] (integers, seeded); network
    k draws its priors from seed + k."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Ts = rng.integers(t_range[0], t_range[1] + 1, size=count)
    Gs = rng.integers(g_range[0], g_range[1] + 1, size=count)
    return [Workload(f"set{k}", int(Ts[k]), int(Gs[k]), n_samples, n_factors, 0.05, 0.01, seed + k)
            for k in range(count)]


def _expression(rng: np.random.Generator, G: int, n: int, k: int) -> np.ndarray:
    """G genes x n samples: k latent N(0, 1) factors plus N(0, 0.5^2) noise."""
    L = rng.standard_normal((G, k))
    F = rng.standard_normal((k, n))
    E = rng.normal(0.0, 0.5, size=(G, n))
    return L @ F + E


def _expression_correlation(rng: np.random.Generator, G: int, n: int, k: int,
                            block: int = 2048) -> np.ndarray:
    X = _expression(rng, G, n, k)
    X -= X.mean(axis=1, keepdims=True)
    X /= np.sqrt((X * X).sum(axis=1, keepdims=True))
    C = np.empty((G, G), dtype=np.float32)
    # upper block-rows, mirrored, so C is exactly symmetric
    for r0 in range(0, G, block):
        r1 = min(G, r0 + block)
        blk = (X[r0:r1] @ X[r0:].T).astype(np.float32)
        C[r0:r1, r0:] = blk
        C[r0:, r0:r1] = blk.T
    np.fill_diagonal(C, 1.0)
    return C


def make_inputs(wl: Workload):
    """Return (W0, P0, C0) as C-contiguous float32 arrays."""
    rng = np.random.Generator(np.random.PCG64(wl.seed))
    T, G = wl.T, wl.G
    W0 = (rng.random((T, G)) < wl.w_density).astype(np.float32)
    if wl.identity_priors:
        return W0, np.eye(T, dtype=np.float32), np.eye(G, dtype=np.float32)
    up = np.triu(rng.random((T, T)) < wl.p_density, 1)
    P0 = (up | up.T).astype(np.float32)
    np.fill_diagonal(P0, 1.0)
    C0 = _expression_correlation(rng, G, wl.n_samples, wl.n_factors)
    return W0, P0, C0


def make_expression(wl: Workload):
    """Return (W0, P0, X): the same W0 and P0 as make_inputs and the expression
    matrix (G x n_samples, float32) whose gene correlations make_inputs' C0 is."""
    assert not wl.identity_priors, "identity-prior workloads have no expression data"
    rng = np.random.Generator(np.random.PCG64(wl.seed))
    T, G = wl.T, wl.G
    W0 = (rng.random((T, G)) < wl.w_density).astype(np.float32)
    up = np.triu(rng.random((T, T)) < wl.p_density, 1)
    P0 = (up | up.T).astype(np.float32)
    np.fill_diagonal(P0, 1.0)
    X = _expression(rng, G, wl.n_samples, wl.n_factors).astype(np.float32)
    return W0, P0, X


def gene_subsample(G: int, n: int, seed: int) -> np.ndarray:
    """The first n genes of a seeded permutation of range(G)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.sort(rng.permutation(G)[:n])
