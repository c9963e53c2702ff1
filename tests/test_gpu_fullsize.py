"""Parity at the sizes the bench runs, and of the paths that only large problems take.

* The FP64 path of a mixed-precision context whose setup contractions all went through the
  FP64-accurate digit-plane branch (forced at o=10 v=50) against the CPU oracle: sigma products to
  1e-12, G to 1e-10.  Large contexts (the C60-shaped one) take that branch for their big setup
  contractions, so this pins the FP64 reference the full-size checks below compare with.
* The C60-shaped workload (o=90 v=450 L=1800, IP) in the bench's launch configuration: one frequency
  x the 30 valence orbitals in one mixed-precision batch; the HOMO's G row against the plain FP64
  GPU path (gfcc_solve_block: the sampled row over all 30 columns) at 1e-6.
* The medium workload's EA sector (o=40 v=200 L=800) in the bench's batch configuration: one
  frequency below the 1p band x the 40 orbitals nearest the gap, mixed precision; a sampled G
  column (the EA systems are solved per column orbital, eq. yq) against the plain FP64 path at
  1e-6, and one FP64 EA sigma product of that context against the oracle at 1e-12.
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


def test_emulated_setup_fp64_path_matches_oracle():
    o, v, L = 10, 50, 100
    pr = make_problem(o, v, L, seed=3)
    gfcc.set_process_option(gfcc.OPT_SETUP_EMULATE_FLOPS, 0.0)   # every setup contraction from digit planes
    try:
        g = gfcc.GFCC(pr, sectors="IP+EA", precision="mixed")
    finally:
        gfcc.set_process_option(gfcc.OPT_SETUP_EMULATE_FLOPS, 4e12)
    g.set_option(gfcc.OPT_PRECISION, gfcc.PREC_FP64)
    orc = GFCCOracle(pr.fock, pr.chol, pr.t1, pr.t2, o=o)
    di, de = g.dims()
    X = np.stack([random_vector(11 + k, di) + 1j * random_vector(31 + k, di) for k in range(2)])
    assert rel_err(g.sigma("IP", X), np.stack([orc.ip_sigma(x) for x in X])) <= 1e-12
    X = np.stack([random_vector(12 + k, de) + 1j * random_vector(32 + k, de) for k in range(2)])
    assert rel_err(g.sigma("EA", X), np.stack([orc.ea_sigma(x) for x in X])) <= 1e-12
    om = np.array([-0.9, 0.2])
    orbs = np.array([o - 1, o], dtype=np.int32)
    G, code = g.solve(om, 0.01, orbs, 1e-13)
    it, rr, st = g.stats()
    g.close()
    assert code == gfcc.OK and np.all(st == 0)
    ref = orc.green(om, 0.01, list(orbs), tol=1e-14, restart=60, max_restarts=60, precond=True)
    assert rel_err(G, ref) <= 1e-10


def test_c60_rows_mixed_match_fp64_path():
    """C60-shaped, bench configuration: the frequency of timed step 1 (grid index 17), the 30 valence
    orbitals in one mixed-precision batch.  The HOMO's mixed G row against the plain FP64 GPU path
    (FP64 GMRES on the FP64 sigma, same tol; about 40 iterations of 0.9 s) at 1e-6; every mixed
    system converged."""
    wl = workload("c60")
    pr = wl.problem()
    g = gfcc.GFCC(pr, sectors="IP", precision="mixed")
    del pr
    om = wl.omegas[17:18]
    G, code = g.solve(om, wl.eta, wl.orbitals, wl.tol)
    it, rr, st = g.stats()
    assert code == gfcc.OK and np.all(st == 0) and np.all(rr <= wl.tol)
    rows = [wl.orbitals.size - 1]
    g.set_option(gfcc.OPT_PRECISION, gfcc.PREC_FP64)
    G64, code64 = g.solve_block(om, wl.eta, wl.orbitals[rows], wl.orbitals, wl.tol)
    it64, rr64, st64 = g.stats()
    g.close()
    assert code64 == gfcc.OK and np.all(st64 == 0)
    for a, r in enumerate(rows):
        assert np.linalg.norm(G[0, r] - G64[0, a]) <= 1e-6 * np.linalg.norm(G64[0, a])


def test_medium_ea_column_mixed_matches_fp64_path():
    """Medium workload, EA sector, bench batch configuration (one frequency x the 40 orbitals nearest
    the gap in one batch), at omega = -0.2 Ha (below the 1p band, outside the 2p1h continuum)."""
    wl = workload("medium")
    pr = wl.problem()
    g = gfcc.GFCC(pr, sectors="EA", precision="mixed")
    om = np.array([-0.2])
    G, code = g.solve(om, wl.eta, wl.orbitals, wl.tol)
    it, rr, st = g.stats()
    assert code == gfcc.OK and np.all(st == 0) and np.all(rr <= wl.tol)
    # the EA systems Y_q are solved per column orbital q: column of the lowest virtual of the list
    col = int(np.argmax(wl.orbitals >= wl.o))
    g.set_option(gfcc.OPT_PRECISION, gfcc.PREC_FP64)
    G64, code64 = g.solve_block(om, wl.eta, wl.orbitals, wl.orbitals[col:col + 1], wl.tol)
    it64, rr64, st64 = g.stats()
    assert code64 == gfcc.OK and np.all(st64 == 0)
    ref = G64[0, :, 0]
    assert np.linalg.norm(G[0, :, col] - ref) <= 1e-6 * np.linalg.norm(ref)
    # the FP64 EA sigma of this context (setup through the digit-plane branch for its largest
    # contractions) against the oracle, one vector
    orc = GFCCOracle(pr.fock, pr.chol, pr.t1, pr.t2, o=wl.o, sectors=("EA",))
    _, de = g.dims()
    x = random_vector(5, de) + 1j * random_vector(6, de)
    y = g.sigma("EA", x[None, :])[0]
    g.close()
    assert rel_err(y, orc.ea_sigma(x)) <= 1e-12
