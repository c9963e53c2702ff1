"""The ground-state CCSD / Lambda-CCSD step on the device (gfcc_ccsd) against the CPU oracle
(oracle/ccsd_ref.py, pinned to the Fock-space definition):

* one Jacobi step from random amplitudes: with max_iter = 1 the call returns x + Omega(x) / D
  (antisymmetrised), so every T residual element is compared, at T1 and T2 switched on together;
  the same for the Lambda residual at converged T and random Lambda;
* converged T, Lambda and E_corr against the oracle's solver, at shapes that span several contraction
  tiles with ragged edges, FP64 and with every large contraction through the digit-plane products;
* two electrons, where CCSD is exact: the device amplitudes fed to gfcc_create give the exact Lehmann
  G of the two-electron system (eq. gfxn0; IP, and IP + EA where the EA space is complete) -- the
  ground-state step and the Green's-function path end to end.
"""
import numpy as np
import pytest

from paper_2010_04768_gb300 import gfcc
from paper_2010_04768_gb300.synthetic import Problem, make_problem
from oracle import ccsd_ref as C
from oracle import fock_space as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session", autouse=True)
def _built():
    from paper_2010_04768_gb300 import build
    build.build()
    gfcc.load()


def amplitudes(o, v, seed, s1, s2):
    rng = np.random.default_rng(seed)
    t1 = s1 * rng.standard_normal((o, v))
    g = s2 * rng.standard_normal((o, o, v, v))
    return t1, 0.25 * (g - g.transpose(1, 0, 2, 3) - g.transpose(0, 1, 3, 2) + g.transpose(1, 0, 3, 2))


def jacobi(fock, o, x1, x2, r1, r2):
    D1, D2 = C.denominators(fock, o)
    u2 = x2 + r2 / D2
    return x1 + r1 / D1, 0.25 * (u2 - u2.transpose(1, 0, 2, 3) - u2.transpose(0, 1, 3, 2) + u2.transpose(1, 0, 3, 2))


@pytest.mark.parametrize("o,v,L", [(3, 9, 11), (6, 21, 30)])
def test_t_residual_one_jacobi_step(o, v, L):
    pr = make_problem(o, v, L, seed=o + v, chol_sigma=0.15)
    t1, t2 = amplitudes(o, v, 5, 0.05, 0.05)
    g1, g2, _, _, info, code = gfcc.ccsd(pr.fock, pr.chol, o, tol=1e-14, max_iter=1, want_lambda=False,
                                         guess=(t1, t2))
    assert code == gfcc.WARN_NOT_CONVERGED and info["t_iters"] == 1
    r1, r2 = C.t_residuals(pr.fock, pr.chol, t1, t2, o)
    e1, e2 = jacobi(pr.fock, o, t1, t2, r1, r2)
    scale = max(np.abs(r1).max(), np.abs(r2).max())
    assert info["t_residual"] == pytest.approx(scale, rel=1e-12)
    D1, D2 = C.denominators(pr.fock, o)
    dmin = min(np.abs(D1).min(), np.abs(D2).min())
    assert np.abs(g1 - e1).max() <= 1e-12 * scale / dmin
    assert np.abs(g2 - e2).max() <= 1e-12 * scale / dmin


@pytest.mark.parametrize("o,v,L", [(3, 9, 11), (6, 21, 30)])
def test_lambda_residual_one_jacobi_step(o, v, L):
    pr = make_problem(o, v, L, seed=2 * o + v, chol_sigma=0.1)
    t1, t2, _, _ = C.solve_t(pr.fock, pr.chol, o, tol=1e-13)
    l1, l2 = amplitudes(o, v, 6, 0.1, 0.1)
    # T is already converged (its residual below tol), Lambda takes one Jacobi step
    g1, g2, m1, m2, info, code = gfcc.ccsd(pr.fock, pr.chol, o, tol=1e-11, max_iter=1, guess=(t1, t2, l1, l2))
    assert code == gfcc.WARN_NOT_CONVERGED and info["t_iters"] == 1 and info["lambda_iters"] == 1
    assert np.array_equal(g1, t1) and np.array_equal(g2, t2)
    E = C.lambda_elements(pr.fock, pr.chol, t1, t2, o)
    r1, r2 = C.lambda_residuals(E, t2, l1, l2)
    e1, e2 = jacobi(pr.fock, o, l1, l2, r1, r2)
    scale = max(np.abs(r1).max(), np.abs(r2).max())
    assert info["lambda_residual"] == pytest.approx(scale, rel=1e-12)
    D1, D2 = C.denominators(pr.fock, o)
    dmin = min(np.abs(D1).min(), np.abs(D2).min())
    assert np.abs(m1 - e1).max() <= 1e-12 * scale / dmin
    assert np.abs(m2 - e2).max() <= 1e-12 * scale / dmin


@pytest.mark.parametrize("o,v,L,emulate", [(4, 12, 20, False), (8, 40, 60, False), (8, 40, 60, True)])
def test_converged_amplitudes_match_oracle(o, v, L, emulate):
    pr = make_problem(o, v, L, seed=o * v, chol_sigma=0.6 / np.sqrt(o * v))
    t1, t2, ec, _ = C.solve_t(pr.fock, pr.chol, o, tol=1e-12)
    l1, l2, _ = C.solve_lambda(pr.fock, pr.chol, t1, t2, o, tol=1e-12)
    if emulate:
        gfcc.set_process_option(gfcc.OPT_SETUP_EMULATE_FLOPS, 0.0)   # every large contraction from digit planes
    try:
        g1, g2, m1, m2, info, code = gfcc.ccsd(pr.fock, pr.chol, o, tol=1e-12, max_iter=200, emulate=emulate)
    finally:
        gfcc.set_process_option(gfcc.OPT_SETUP_EMULATE_FLOPS, 4e12)
    assert code == gfcc.OK and info["t_residual"] <= 1e-12 and info["lambda_residual"] <= 1e-12
    # both sides stop at max |residual| <= 1e-12; the amplitudes then agree to about that over the gap
    assert np.abs(g1 - t1).max() <= 1e-10 and np.abs(g2 - t2).max() <= 1e-10
    assert np.abs(m1 - l1).max() <= 1e-10 and np.abs(m2 - l2).max() <= 1e-10
    assert info["e_corr"] == pytest.approx(ec, abs=1e-11)
    assert info["e_corr"] == pytest.approx(C.correlation_energy(pr.fock, pr.chol, g1, g2, o), abs=1e-12)


@pytest.mark.parametrize("v,sectors", [(6, "IP"), (2, "IP+EA")])
def test_two_electrons_ground_state_to_exact_green_function(v, sectors):
    # two electrons: CCSD is exact and the IP space (1h + 2h1p) is the whole N-1 sector; the EA space
    # (1p + 2p1h) is the whole N+1 sector only without 3p2h determinants, i.e. for v = 2
    o, L = 2, 8
    pr = make_problem(o, v, L, seed=21 + v, chol_sigma=0.3)
    t1, t2, l1, l2, info, code = gfcc.ccsd(pr.fock, pr.chol, o, tol=1e-13, max_iter=300)
    assert code == gfcc.OK
    fs = F.FockSpace(o + v)
    H = F.hamiltonian(fs, pr.fock, pr.chol, o, o).toarray()
    masks, index = fs.sector(o)
    phi = np.zeros(fs.dim(o))
    phi[index[(1 << o) - 1]] = 1.0
    assert info["e_corr"] == pytest.approx(np.linalg.eigvalsh(H)[0] - phi @ H @ phi, abs=1e-11)
    g = gfcc.GFCC(Problem(o=o, v=v, L=L, fock=pr.fock, chol=pr.chol, t1=t1, t2=t2, lam1=l1, lam2=l2), sectors=sectors)
    g.set_option(gfcc.OPT_RESTART, 64)   # the packed spaces in one Krylov cycle
    orbs = np.arange(o + v, dtype=np.int32)
    om = np.array([-1.3, -0.4, 0.35, 1.2])
    G, code = g.solve(om, 0.05, orbs, 1e-13)
    g.close()
    assert code == gfcc.OK
    Gx = F.exact_green(pr.fock, pr.chol, o, om, 0.05, list(orbs), parts=tuple(sectors.split("+")))
    assert np.abs(G - Gx).max() <= 1e-9 * np.abs(Gx).max()


def test_bad_arguments_are_rejected():
    pr = make_problem(2, 4, 3, seed=1)
    with pytest.raises(gfcc.GFCCError):
        gfcc.ccsd(pr.fock, pr.chol, 2, tol=0.0)
    with pytest.raises(gfcc.GFCCError):
        gfcc.ccsd(pr.fock, pr.chol, 2, max_iter=0)
    bad = pr.chol.copy()
    bad[0, 0, 1] += 1.0   # not symmetric in the orbital pair
    with pytest.raises(gfcc.GFCCError):
        gfcc.ccsd(pr.fock, bad, 2)
