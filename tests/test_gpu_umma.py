"""The tcgen05 BF16 contraction engine alone, through the C ABI (gfcc_selftest_gemm_bf16).

Reference: the same BF16-rounded operands multiplied in float64; the kernel accumulates
in FP32, so the bound is a few FP32 roundings per output relative to sum_k |a_k b_k|.
"""
import numpy as np
import pytest

from paper_2010_04768_gb300 import gfcc
from paper_2010_04768_gb300.synthetic import normal

pytestmark = pytest.mark.gpu


def bf16_round(x):
    x32 = np.asarray(x, dtype=np.float32)
    u = x32.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (128, 256, 256), (300, 520, 200), (1, 1, 8), (257, 100, 1000),
                                   (512, 768, 4096)])
def test_umma_bf16_gemm(M, N, K):
    A = normal(1, 1, M * K).reshape(M, K).astype(np.float32)
    B = normal(2, 1, N * K).reshape(N, K).astype(np.float32)
    D = gfcc.selftest_gemm_bf16(A, B)
    Ab, Bb = bf16_round(A), bf16_round(B)
    ref = Ab @ Bb.T
    scale = np.abs(Ab) @ np.abs(Bb).T
    err = np.abs(D.astype(np.float64) - ref) / scale
    assert err.max() <= 4 * K * 2.0**-24 + 1e-7


def test_umma_integer_products_are_exact():
    """Digit products |a b| <= 2^10 summed over K = 2^14 stay exact in the FP32 accumulator
    (the property the FP64 emulation rests on)."""
    M, N, K = 256, 256, 16384
    rng = np.random.default_rng(5)
    A = rng.integers(-32, 33, size=(M, K)).astype(np.float32)
    B = rng.integers(-32, 33, size=(N, K)).astype(np.float32)
    A[0, :] = 32
    B[0, :] = 32                                   # one entry reaches exactly 2^24
    D = gfcc.selftest_gemm_bf16(A, B)
    ref = A.astype(np.int64) @ B.astype(np.int64).T
    assert np.array_equal(D.astype(np.int64), ref)


# N <= 512: all digit pairs of a tile in one kernel (with a K split for K > 2048); wider: one GEMM
# per digit pair
@pytest.mark.parametrize("M,N,K", [(200, 300, 700), (128, 256, 20000), (1, 5, 8), (300, 80, 40), (100, 700, 300),
                                   (130, 600, 5000)])
def test_f64_emulation_accuracy(M, N, K):
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-3, 3, size=(M, 1)))
    B = rng.standard_normal((N, K)) * np.exp(rng.uniform(-3, 3, size=(N, 1)))
    ref = A @ B.T
    scale = np.abs(A) @ np.abs(B).T
    C = gfcc.selftest_gemm_f64emu(A, B, S=8, P=9)
    assert (np.abs(C - ref) / scale).max() <= 1e-13
    C6 = gfcc.selftest_gemm_f64emu(A, B, S=6, P=7)
    assert (np.abs(C6 - ref) / scale).max() <= 3e-10


def test_tile_autotuner_gives_the_same_products():
    # the first call of a shape times the 64 / 128 / 256-column tiles; the tile width does not change
    # the order of the K accumulation, so every choice gives the same FP32 result
    from paper_2010_04768_gb300.synthetic import workload
    g = gfcc.GFCC(workload("tiny").problem(), sectors="IP")
    rng = np.random.default_rng(8)
    out = {}
    for tune in (0, 1):
        g.set_option(gfcc.OPT_AUTOTUNE, tune)
        for (M, N, K) in ((384, 80, 200), (256, 300, 640), (128, 40, 1000)):
            A = rng.normal(size=(M, K)).astype(np.float32) if tune == 0 else out[(M, N, K)][1]
            B = rng.normal(size=(N, K)).astype(np.float32) if tune == 0 else out[(M, N, K)][2]
            D = gfcc.selftest_gemm_bf16(A, B)
            if tune == 0:
                out[(M, N, K)] = (D, A, B)
            else:
                assert np.max(np.abs(D - out[(M, N, K)][0])) <= 1e-5 * np.max(np.abs(D))
    g.set_option(gfcc.OPT_AUTOTUNE, 1)
    g.close()


@pytest.fixture
def pair_mode():
    # force the CTA-pair (cta_group::2) kernel where it applies; restore autotuning afterwards
    gfcc.set_process_option(gfcc.OPT_GEMM_PAIR, 1.0)
    yield
    gfcc.set_process_option(gfcc.OPT_GEMM_PAIR, 0.0)


@pytest.mark.parametrize("M,N,K", [(256, 256, 512), (300, 520, 700), (640, 300, 4096), (129, 257, 520),
                                   (1024, 1024, 8192)])
def test_pair_gemm_matches_reference(pair_mode, M, N, K):
    # 256 x 256 tiles over CTA pairs: row tails inside a pair and past it, column tails inside a half
    A = normal(3, 1, M * K).reshape(M, K).astype(np.float32)
    B = normal(4, 1, N * K).reshape(N, K).astype(np.float32)
    D = gfcc.selftest_gemm_bf16(A, B)
    Ab, Bb = bf16_round(A), bf16_round(B)
    ref = Ab @ Bb.T
    scale = np.abs(Ab) @ np.abs(Bb).T
    err = np.abs(D.astype(np.float64) - ref) / scale
    assert err.max() <= 4 * K * 2.0**-24 + 1e-7


def test_pair_gemm_integer_products_are_exact(pair_mode):
    M, N, K = 512, 384, 16384
    rng = np.random.default_rng(6)
    A = rng.integers(-32, 33, size=(M, K)).astype(np.float32)
    B = rng.integers(-32, 33, size=(N, K)).astype(np.float32)
    A[0, :] = 32
    B[0, :] = 32
    D = gfcc.selftest_gemm_bf16(A, B)
    ref = A.astype(np.int64) @ B.astype(np.int64).T
    assert np.array_equal(D.astype(np.int64), ref)


def test_pair_emulated_product_is_fp64_accurate(pair_mode):
    # the wide digit-pair products of the FP64 emulation on the pair kernel
    rng = np.random.default_rng(9)
    M, N, K = 600, 700, 3000
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-3, 3, size=(M, 1)))
    B = rng.standard_normal((N, K)) * np.exp(rng.uniform(-3, 3, size=(N, 1)))
    C = gfcc.selftest_gemm_f64emu(A, B, S=8, P=9)
    assert (np.abs(C - A @ B.T) / (np.abs(A) @ np.abs(B).T)).max() <= 1e-13


@pytest.fixture
def persist_mode():
    # force the persistent kernel (two TMEM accumulators, one CTA per SM); restore autotuning afterwards
    gfcc.set_process_option(gfcc.OPT_GEMM_PERSIST, 1.0)
    yield
    gfcc.set_process_option(gfcc.OPT_GEMM_PERSIST, 0.0)


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (300, 520, 700), (5000, 60, 540), (2000, 300, 64),
                                   (1024, 1024, 4096), (77, 1000, 130), (40000, 100, 64), (20000, 300, 200)])
def test_persistent_gemm_matches_reference(persist_mode, M, N, K):
    # up to three tiles per CTA (both accumulators reused, their barriers in their second phase), one
    # K block per tile, ragged edges
    A = normal(5, 1, M * K).reshape(M, K).astype(np.float32)
    B = normal(6, 1, N * K).reshape(N, K).astype(np.float32)
    D = gfcc.selftest_gemm_bf16(A, B)
    Ab, Bb = bf16_round(A), bf16_round(B)
    ref = Ab @ Bb.T
    scale = np.abs(Ab) @ np.abs(Bb).T
    err = np.abs(D.astype(np.float64) - ref) / scale
    assert err.max() <= 4 * K * 2.0**-24 + 1e-7


def test_persistent_emulated_product_is_fp64_accurate(persist_mode):
    # the digit-pair products (accumulating calls, split K) on the persistent kernel
    rng = np.random.default_rng(10)
    for M, N, K in ((600, 700, 3000), (130, 600, 20000)):
        A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-3, 3, size=(M, 1)))
        B = rng.standard_normal((N, K)) * np.exp(rng.uniform(-3, 3, size=(N, 1)))
        C = gfcc.selftest_gemm_f64emu(A, B, S=8, P=9)
        assert (np.abs(C - A @ B.T) / (np.abs(A) @ np.abs(B).T)).max() <= 1e-13
