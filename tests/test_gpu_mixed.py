"""Mixed precision (BF16 tensor-core couplings + FP64 refinement) against the FP64 oracle.

The bar of the mixed path: G(omega) within 1e-6 relative of the FP64 result.  The sigma
product itself is only BF16-accurate in its couplings; its Fock-like diagonal is exact.
"""
import numpy as np
import pytest

from paper_2010_04768_gb300 import gfcc
from paper_2010_04768_gb300.synthetic import make_problem, random_vector, workload
from oracle.gfcc_ref import GFCCOracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session", autouse=True)
def _built():
    from paper_2010_04768_gb300 import build
    build.build()
    gfcc.load()


def rel_err(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("o,v,L", [(3, 5, 7), (4, 12, 48), (7, 70, 90), (10, 50, 100)])
def test_mixed_sigma_is_bf16_close(o, v, L):
    pr = make_problem(o, v, L, seed=o + v, t1_std=0.05, t2_std=0.05, chol_sigma=0.3)
    g = gfcc.GFCC(pr, sectors="IP", precision="mixed")
    orc = GFCCOracle(pr.fock, pr.chol, pr.t1, pr.t2, o=o, sectors=("IP",))
    di, _ = g.dims()
    X = np.stack([random_vector(k, di) + 1j * random_vector(50 + k, di) for k in range(3)])
    Y = g.sigma("IP", X, precision="mixed")
    ref = np.stack([orc.ip_sigma(x) for x in X])
    off = ref - orc.ip_diag()[None, :] * X                     # the part computed in BF16
    err = np.abs(Y - ref).max() / np.abs(off).max()
    assert err <= 2e-2
    # the FP64 entry point of the same context is unaffected
    assert rel_err(g.sigma("IP", X), ref) <= 1e-12
    g.close()


@pytest.mark.parametrize("precond", [gfcc.PRECOND_NONE, gfcc.PRECOND_DIAG])
def test_mixed_green_tiny_workload(precond):
    wl = workload("tiny")
    pr = wl.problem()
    g = gfcc.GFCC(pr, sectors="IP", precision="mixed")
    g.set_option(gfcc.OPT_PRECOND, precond)
    G, code = g.solve(wl.omegas, wl.eta, wl.orbitals, 1e-10)
    assert code == gfcc.OK
    ref = GFCCOracle(pr.fock, pr.chol, pr.t1, pr.t2, o=wl.o, sectors=("IP",)).green_dense(
        wl.omegas, wl.eta, list(wl.orbitals), sectors=("IP",))
    assert rel_err(G, ref) <= 1e-6
    it, rr, st = g.stats()
    assert np.all(st == 0) and np.all(rr <= 1e-10)
    g.close()


def test_mixed_matches_fp64_path_medium():
    o, v, L = 10, 50, 100
    pr = make_problem(o, v, L, seed=3)
    om = np.array([-1.1, -0.6, -0.35])
    orbs = np.array([0, o - 2, o - 1, o], dtype=np.int32)
    g64 = gfcc.GFCC(pr, sectors="IP")
    G64, c64 = g64.solve(om, 0.005, orbs, 1e-10)
    g64.close()
    gm = gfcc.GFCC(pr, sectors="IP", precision="mixed")
    Gm, cm = gm.solve(om, 0.005, orbs, 1e-10)
    it, rr, st = gm.stats()
    gm.close()
    assert c64 == gfcc.OK and cm == gfcc.OK
    for w in range(om.size):
        for a in range(orbs.size):
            row, ref = Gm[w, a], G64[w, a]
            assert np.linalg.norm(row - ref) <= 1e-6 * np.linalg.norm(ref)
