"""Failure paths on the GPU, made to happen without a fault.

* Bounded device waits: the tensor-core kernels wait on mbarriers with a limit (process option
  GFCC_OPT_WAIT_NS).  With the test-only switch GFCC_OPT_TEST_NO_LOADS their producers issue no
  loads, so the consumer's first wait runs out with nothing in flight; the kernel sets the error
  flag, frees its TMEM and returns, and the call reports GFCC_ERR_TIMEOUT.  The context stays usable:
  with the defaults restored the same product is correct.
* Device allocation failure: a batch whose GMRES workspace exceeds the device memory makes the solve
  return GFCC_ERR_OOM (the allocation is refused; nothing is half-allocated), and the same context
  solves normally afterwards.
"""
import numpy as np
import pytest

from paper_2010_04768_gb300 import gfcc
from paper_2010_04768_gb300.synthetic import make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session", autouse=True)
def _built():
    from paper_2010_04768_gb300 import build
    build.build()
    gfcc.load()


def test_bounded_wait_runs_out_and_the_context_recovers():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((256, 192), dtype=np.float32)
    B = rng.standard_normal((128, 192), dtype=np.float32)
    ref = gfcc.selftest_gemm_bf16(A, B)
    gfcc.set_process_option(gfcc.OPT_WAIT_NS, 2000.0)   # 2 microseconds
    gfcc.set_process_option(gfcc.OPT_TEST_NO_LOADS, 1.0)
    try:
        with pytest.raises(gfcc.GFCCError) as e:
            gfcc.selftest_gemm_bf16(A, B)
        assert e.value.code == gfcc.ERR_TIMEOUT
        with pytest.raises(gfcc.GFCCError) as e:
            gfcc.selftest_gemm_f64emu(A.astype(np.float64), B.astype(np.float64), S=3, P=4)
        assert e.value.code == gfcc.ERR_TIMEOUT
    finally:
        gfcc.set_process_option(gfcc.OPT_TEST_NO_LOADS, 0.0)
        gfcc.set_process_option(gfcc.OPT_WAIT_NS, 1e9)
    D = gfcc.selftest_gemm_bf16(A, B)
    assert np.array_equal(D, ref)
    # the CTA-pair kernel: its waits run out the same way, and it recovers
    A2 = rng.standard_normal((512, 1024), dtype=np.float32)
    B2 = rng.standard_normal((384, 1024), dtype=np.float32)
    gfcc.set_process_option(gfcc.OPT_GEMM_PAIR, 1.0)
    try:
        ref2 = gfcc.selftest_gemm_bf16(A2, B2)
        gfcc.set_process_option(gfcc.OPT_WAIT_NS, 2000.0)
        gfcc.set_process_option(gfcc.OPT_TEST_NO_LOADS, 1.0)
        try:
            with pytest.raises(gfcc.GFCCError) as e:
                gfcc.selftest_gemm_bf16(A2, B2)
            assert e.value.code == gfcc.ERR_TIMEOUT
        finally:
            gfcc.set_process_option(gfcc.OPT_TEST_NO_LOADS, 0.0)
            gfcc.set_process_option(gfcc.OPT_WAIT_NS, 1e9)
        assert np.array_equal(gfcc.selftest_gemm_bf16(A2, B2), ref2)
    finally:
        gfcc.set_process_option(gfcc.OPT_GEMM_PAIR, 0.0)
    # the persistent kernel likewise
    gfcc.set_process_option(gfcc.OPT_GEMM_PERSIST, 1.0)
    try:
        ref3 = gfcc.selftest_gemm_bf16(A2, B2)
        gfcc.set_process_option(gfcc.OPT_WAIT_NS, 2000.0)
        gfcc.set_process_option(gfcc.OPT_TEST_NO_LOADS, 1.0)
        try:
            with pytest.raises(gfcc.GFCCError) as e:
                gfcc.selftest_gemm_bf16(A2, B2)
            assert e.value.code == gfcc.ERR_TIMEOUT
        finally:
            gfcc.set_process_option(gfcc.OPT_TEST_NO_LOADS, 0.0)
            gfcc.set_process_option(gfcc.OPT_WAIT_NS, 1e9)
        assert np.array_equal(gfcc.selftest_gemm_bf16(A2, B2), ref3)
    finally:
        gfcc.set_process_option(gfcc.OPT_GEMM_PERSIST, 0.0)
    # a solver context on the same device works after the time-out
    pr = make_problem(3, 5, 7, seed=1)
    g = gfcc.GFCC(pr, sectors="IP", precision="mixed")
    G, code = g.solve([-0.5], 0.01, [0, 1, 2], 1e-10)
    g.close()
    assert code == gfcc.OK and np.isfinite(G).all()


def test_allocation_failure_is_reported_and_the_context_recovers():
    # EA at o=12 v=120: 85800 packed coordinates; 4096 systems with 65 Krylov vectors of complex FP64
    # need about 365 GB of GMRES workspace, more than the device holds
    o, v = 12, 120
    pr = make_problem(o, v, 40, seed=2)
    g = gfcc.GFCC(pr, sectors="EA")
    g.set_option(gfcc.OPT_RESTART, 64)
    g.set_option(gfcc.OPT_BATCH, 4096)
    om = np.linspace(-0.5, -0.1, 32)
    orbs = np.arange(o + v, dtype=np.int32)            # 32 x 132 = 4224 systems, batch 4096
    with pytest.raises(gfcc.GFCCError) as e:
        g.solve(om, 0.01, orbs, 1e-8)
    assert e.value.code == gfcc.ERR_OOM
    g.set_option(gfcc.OPT_BATCH, 0)
    g.set_option(gfcc.OPT_RESTART, 30)
    G, code = g.solve(om[:1], 0.01, orbs[o:o + 2], 1e-8)
    g.close()
    assert code == gfcc.OK and np.isfinite(G).all()
