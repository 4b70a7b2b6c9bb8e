"""The tcgen05 pipeline on its own: D = A . B^T through TMA, the BF16 MMA and
TMEM, against FP64 products on the host (needs a GB300)."""
from __future__ import annotations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def bf16_split(x: np.ndarray):
    """hi = bf16(x) (round to nearest even), lo = bf16(x - hi), as float64."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
    hi = t.to(torch.bfloat16).to(torch.float32)
    lo = (t - hi).to(torch.bfloat16).to(torch.float32)
    return hi.double().numpy(), lo.double().numpy()


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (300, 260, 200), (129, 385, 1000), (64, 700, 37)])
def test_hi_only_product(M, N, K):
    from paper_1507_07039_gb300 import panda
    rng = np.random.default_rng(M * N + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((N, K)).astype(np.float32)
    D = panda.panda_selftest_tc_gemm(A, B, terms=1)
    Ah, _ = bf16_split(A)
    Bh, _ = bf16_split(B)
    ref = Ah @ Bh.T  # products of BF16 values are exact in FP32; only the FP32 sums round
    err = np.max(np.abs(D - ref)) / max(1.0, np.max(np.abs(ref)))
    assert err < 2e-6, err


@pytest.mark.parametrize("M,N,K", [(256, 256, 512), (130, 300, 1000)])
def test_three_term_split_product(M, N, K):
    from paper_1507_07039_gb300 import panda
    rng = np.random.default_rng(7 * M + N + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((N, K)).astype(np.float32)
    D = panda.panda_selftest_tc_gemm(A, B, terms=3)
    Ah, Al = bf16_split(A)
    Bh, Bl = bf16_split(B)
    ref3 = Ah @ Bh.T + Ah @ Bl.T + Al @ Bh.T
    exact = A.astype(np.float64) @ B.astype(np.float64).T
    scale = max(1.0, np.max(np.abs(exact)))
    # the tensor core's FP32 accumulation rounds each MMA's K=16 partial into the
    # accumulator; three MMAs per slice triple the number of such additions
    assert np.max(np.abs(D - ref3)) / scale < 1e-5
    # plus the dropped lo*lo term and the split residuals (below 2^-16 relative per product)
    assert np.max(np.abs(D - exact)) / scale < 3e-5


@pytest.mark.parametrize("M,N,K", [(256, 256, 64), (300, 600, 1000), (512, 256, 130)])
def test_cta_pair_product(M, N, K):
    """The same product on CTA pairs (cta_group::2 MMAs over 256 x 256 tiles)."""
    from paper_1507_07039_gb300 import panda
    rng = np.random.default_rng(3 * M + N + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((N, K)).astype(np.float32)
    D1 = panda.panda_selftest_tc_gemm(A, B, terms=11)
    Ah, Al = bf16_split(A)
    Bh, Bl = bf16_split(B)
    ref1 = Ah @ Bh.T
    scale = max(1.0, np.max(np.abs(ref1)))
    assert np.max(np.abs(D1 - ref1)) / scale < 2e-6
    D3 = panda.panda_selftest_tc_gemm(A, B, terms=13)
    ref3 = Ah @ Bh.T + Ah @ Bl.T + Al @ Bh.T
    assert np.max(np.abs(D3 - ref3)) / scale < 1e-5


@pytest.mark.parametrize("M,N,K", [(256, 256, 64), (300, 600, 1000), (512, 256, 130)])
def test_cta_pair_product_mn_major_b(M, N, K):
    """CTA pairs with B held transposed ([K][N], N contiguous) and fed to the
    MMAs MN-major: the same products as the K-major form."""
    from paper_1507_07039_gb300 import panda
    rng = np.random.default_rng(5 * M + N + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((N, K)).astype(np.float32)
    Ah, Al = bf16_split(A)
    Bh, Bl = bf16_split(B)
    D1 = panda.panda_selftest_tc_gemm(A, B, terms=21)
    ref1 = Ah @ Bh.T
    scale = max(1.0, np.max(np.abs(ref1)))
    assert np.max(np.abs(D1 - ref1)) / scale < 2e-6
    D3 = panda.panda_selftest_tc_gemm(A, B, terms=23)
    ref3 = Ah @ Bh.T + Ah @ Bl.T + Al @ Bh.T
    assert np.max(np.abs(D3 - ref3)) / scale < 1e-5
    # the K-major form of the same pair kernel gives the same sums up to accumulation order
    assert np.max(np.abs(D3 - panda.panda_selftest_tc_gemm(A, B, terms=13))) / scale < 1e-5


@pytest.mark.parametrize("mode", [40, 50])
@pytest.mark.parametrize("M,N,K", [(256, 256, 64), (300, 600, 1000), (512, 256, 130)])
def test_cta_pair_product_mn_major_a(mode, M, N, K):
    """CTA pairs with A held transposed ([K][M], M contiguous) and fed to the
    MMAs MN-major, with B so too (mode 40) or K-major (mode 50): the same
    products as the K-major form."""
    from paper_1507_07039_gb300 import panda
    rng = np.random.default_rng(7 * M + N + K + mode)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((N, K)).astype(np.float32)
    Ah, Al = bf16_split(A)
    Bh, Bl = bf16_split(B)
    D1 = panda.panda_selftest_tc_gemm(A, B, terms=mode + 1)
    ref1 = Ah @ Bh.T
    scale = max(1.0, np.max(np.abs(ref1)))
    assert np.max(np.abs(D1 - ref1)) / scale < 2e-6
    D3 = panda.panda_selftest_tc_gemm(A, B, terms=mode + 3)
    ref3 = Ah @ Bh.T + Ah @ Bl.T + Al @ Bh.T
    assert np.max(np.abs(D3 - ref3)) / scale < 1e-5
    assert np.max(np.abs(D3 - panda.panda_selftest_tc_gemm(A, B, terms=13))) / scale < 1e-5


def e4m3(x: np.ndarray) -> np.ndarray:
    """x rounded to E4M3 (nearest even), as float64 (|x| stays below 448 here)."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
    return t.to(torch.float8_e4m3fn).to(torch.float32).double().numpy()


@pytest.mark.parametrize("M,N,K", [(256, 256, 128), (300, 600, 1000), (512, 256, 130)])
def test_cta_pair_e4m3_product(M, N, K):
    """kind::f8f6f4 MMAs on CTA pairs: products of E4M3 values are exact in
    FP32, so only the FP32 accumulation separates D from the FP64 product of
    the rounded operands."""
    from paper_1507_07039_gb300 import panda
    rng = np.random.default_rng(11 * M + N + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((N, K)).astype(np.float32)
    D = panda.panda_selftest_tc_gemm(A, B, terms=8)
    ref = e4m3(A) @ e4m3(B).T
    scale = max(1.0, np.max(np.abs(ref)))
    assert np.max(np.abs(D - ref)) / scale < 1e-5
    # and E4M3 keeps about 2^-4 of each operand: far from the exact product, as it should be
    exact = A.astype(np.float64) @ B.astype(np.float64).T
    assert np.max(np.abs(D - exact)) / scale > 1e-4


def test_bounded_wait_reports_timeout_and_device_stays_usable():
    """A pipeline stage armed but never loaded: the kernel's bounded waits
    must end it with PANDA_ETIMEOUT (about a second), not hang; the next
    product on the same device is still right."""
    import time
    from paper_1507_07039_gb300 import panda
    t0 = time.time()
    rc = panda.panda_selftest_timeout()
    assert rc == -7, (rc, panda.panda_last_error(None))
    assert time.time() - t0 < 30
    A = np.ones((128, 64), np.float32)
    B = np.full((128, 64), 2.0, np.float32)
    D = panda.panda_selftest_tc_gemm(A, B, terms=1)
    assert np.all(D == 128.0)


@pytest.mark.parametrize("K", [1024, 4096, 17152])
def test_accumulation_drift_of_a_long_mma_chain(K):
    """Sums of positive products on the pair pipeline (three-term split, one
    accumulator over all of K) drift toward zero as K grows, while signed
    sums do not: the MMA's FP32 accumulation drops low bits on every step.
    Bound: each of the 3 K / 16 accumulating MMAs loses at most one unit of
    the running sum's last place, |error| <= (3 K / 16) 2^-23 sum |a||b|.
    (This is why the library sums its products over all genes in chunks.)"""
    from paper_1507_07039_gb300 import panda
    rng = np.random.default_rng(K)
    out = {}
    for kind in ("positive", "signed"):
        A = rng.random((256, K)).astype(np.float32)
        B = rng.random((256, K)).astype(np.float32)
        if kind == "signed":
            A -= 0.5
            B -= 0.5
        D = panda.panda_selftest_tc_gemm(A, B, terms=13)
        A64, B64 = A.astype(np.float64), B.astype(np.float64)
        rel = (D - A64 @ B64.T) / (np.abs(A64) @ np.abs(B64).T)
        out[kind] = (float(np.abs(rel).max()), float(rel.mean()))
        assert np.abs(rel).max() <= 3 * K / 16 * 2.0 ** -23, (kind, out[kind])
    print(f"\nK={K}: positive max {out['positive'][0]:.2e} mean {out['positive'][1]:+.2e}; "
          f"signed max {out['signed'][0]:.2e} mean {out['signed'][1]:+.2e}")
    assert out["positive"][1] < 0  # toward zero
