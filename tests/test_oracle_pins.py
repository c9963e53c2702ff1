"""Pins of the CPU oracle to facts outside itself (CPU only).

Chain of pins:
  1. the brute-force Fock-space definition (oracle/fock_space.py) reproduces the
     exact Lehmann Green's function of eq. gfxn0 whenever CCSD is the exact CC
     (one or two electrons) and the IP/EA space of eqs. xp/yq is complete;
  2. the closed-form oracle (oracle/gfcc_ref.py) reproduces every matrix element,
     right-hand side and left vector of the brute force with random T1, T2,
     Lambda and Cholesky vectors, term by term;
  3. closed forms: the Hartree-Fock limit G_pp = 1/(omega - eps_p -/+ i eta) and the
     diagonal-operator limit (no two-electron integrals) of eq. xplin;
  4. mathematics: Hermiticity and the sum-over-states form at T = 0, linearity of
     the sigma product, GMRES against dense LU, monotone GMRES residuals and
     convergence within dim steps (GFCC Workflow and Bottlenecks section), and the
     large-omega moment expansion of the resolvent.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from paper_2010_04768_gb300.synthetic import make_problem, random_vector
from oracle.fock_space import BruteForceGFCC, exact_green, solve_cc_exact
from oracle.gfcc_ref import GFCCOracle, gmres, ip_dim, ea_dim

OMEGAS = np.array([-0.9, -0.35, 0.45, 1.3])
ETA = 0.05


# ---------------------------------------------------------------- 1. definition vs eq. gfxn0
@pytest.mark.parametrize("v", [2, 3, 4])
def test_definition_is_exact_ip_two_electrons(v):
    pr = make_problem(2, v, 6, seed=11 + v, chol_sigma=0.3)
    t1, t2, l1, l2, _ = solve_cc_exact(pr.fock, pr.chol, 2)
    assert np.abs(t2).max() > 1e-3 and np.abs(l2).max() > 1e-3
    bf = BruteForceGFCC(pr.fock, pr.chol, t1, t2, l1, l2, 2)
    orbs = list(range(2 + v))
    g = bf.green_ip(OMEGAS, ETA, orbs)
    ref = exact_green(pr.fock, pr.chol, 2, OMEGAS, ETA, orbs, parts=("IP",))
    assert np.abs(g - ref).max() <= 1e-11 * np.abs(ref).max()


def test_definition_is_exact_ip_and_ea_minimal():
    pr = make_problem(2, 2, 5, seed=5, chol_sigma=0.4)
    t1, t2, l1, l2, _ = solve_cc_exact(pr.fock, pr.chol, 2)
    bf = BruteForceGFCC(pr.fock, pr.chol, t1, t2, l1, l2, 2)
    orbs = [0, 1, 2, 3]
    g = bf.green_ip(OMEGAS, ETA, orbs) + bf.green_ea(OMEGAS, ETA, orbs)
    ref = exact_green(pr.fock, pr.chol, 2, OMEGAS, ETA, orbs)
    assert np.abs(g - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("v", [3, 5])
def test_definition_is_exact_ea_one_electron(v):
    pr = make_problem(1, v, 6, seed=21 + v, chol_sigma=0.3)
    # a non-canonical reference (f_ov != 0) so that T1 and Lambda1 are non-zero for one electron
    off = 0.05 * np.outer(np.arange(1, v + 2), np.ones(v + 1)) / (v + 1)
    pr.fock = pr.fock + off + off.T
    t1, t2, l1, l2, _ = solve_cc_exact(pr.fock, pr.chol, 1)
    assert np.abs(t1).max() > 1e-4
    bf = BruteForceGFCC(pr.fock, pr.chol, t1, t2, l1, l2, 1)
    orbs = list(range(1 + v))
    g = bf.green_ip(OMEGAS, ETA, orbs) + bf.green_ea(OMEGAS, ETA, orbs)
    ref = exact_green(pr.fock, pr.chol, 1, OMEGAS, ETA, orbs)
    assert np.abs(g - ref).max() <= 1e-11 * np.abs(ref).max()


# ---------------------------------------------------------------- 2. closed form vs definition
def _pair(o, v, seed, *, t1=True, t2=True, chol=True, L=5):
    pr = make_problem(o, v, L, seed=seed, chol_sigma=0.3, t1_std=0.1, t2_std=0.1, separate_lambda=True)
    a1 = pr.t1 if t1 else 0 * pr.t1
    a2 = pr.t2 if t2 else 0 * pr.t2
    if not chol:
        pr.chol[:] = 0.0
    bf = BruteForceGFCC(pr.fock, pr.chol, a1, a2, pr.lam1, pr.lam2, o)
    orc = GFCCOracle(pr.fock, pr.chol, a1, a2, pr.lam1, pr.lam2, o)
    return pr, bf, orc


@pytest.mark.parametrize("o,v", [(2, 3), (3, 4), (4, 5)])
@pytest.mark.parametrize("terms", ["chol", "chol+t1", "chol+t2", "all"])
def test_closed_form_matches_definition(o, v, terms):
    pr, bf, orc = _pair(o, v, seed=100 * o + v, t1="t1" in terms or terms == "all",
                        t2="t2" in terms or terms == "all")
    for name, Mb, Mo in [("IP", bf.ip_matrix(), orc.ip_matrix()), ("EA", bf.ea_matrix(), orc.ea_matrix())]:
        assert Mb.shape == Mo.shape
        assert np.abs(Mb - Mo).max() <= 1e-12 * max(1.0, np.abs(Mb).max()), name
    for p in range(o + v):
        np.testing.assert_allclose(orc.ip_rhs(p), bf.ip_rhs(p), atol=1e-13)
        np.testing.assert_allclose(orc.ip_left(p), bf.ip_left(p), atol=1e-13)
        np.testing.assert_allclose(orc.ea_rhs(p), bf.ea_rhs(p), atol=1e-13)
        np.testing.assert_allclose(orc.ea_left(p), bf.ea_left(p), atol=1e-13)


@pytest.fixture(scope="module")
def tiny_pair():
    """The 'tiny' workload (o=4, v=12, L=48, seed 0): brute force and closed form."""
    pr = make_problem(4, 12, 48, seed=0)
    bf = BruteForceGFCC(pr.fock, pr.chol, pr.t1, pr.t2, pr.t1, pr.t2, 4)
    orc = GFCCOracle(pr.fock, pr.chol, pr.t1, pr.t2, o=4)
    return pr, bf, orc


@pytest.mark.slow
def test_closed_form_matches_definition_tiny_workload(tiny_pair):
    pr, bf, orc = tiny_pair
    Mb, Mo = bf.ip_matrix(), orc.ip_matrix()
    assert np.abs(Mb - Mo).max() <= 1e-12 * np.abs(Mb).max()
    Mb, Mo = bf.ea_matrix(), orc.ea_matrix()
    assert np.abs(Mb - Mo).max() <= 1e-12 * np.abs(Mb).max()
    for p in (0, 3, 4, 15):
        np.testing.assert_allclose(orc.ip_rhs(p), bf.ip_rhs(p), atol=1e-14)
        np.testing.assert_allclose(orc.ip_left(p), bf.ip_left(p), atol=1e-14)
        np.testing.assert_allclose(orc.ea_rhs(p), bf.ea_rhs(p), atol=1e-14)
        np.testing.assert_allclose(orc.ea_left(p), bf.ea_left(p), atol=1e-14)


# ---------------------------------------------------------------- 3. closed forms
def test_hartree_fock_limit():
    """chol = 0 and T = Lambda = 0: G_ii = 1/(omega - eps_i - i eta), G_aa = 1/(omega - eps_a + i eta)."""
    o, v = 3, 5
    pr = make_problem(o, v, 4, seed=7, with_t=False)
    pr.chol[:] = 0.0
    eps = pr.eps()
    orbs = list(range(o + v))
    orc = GFCCOracle(pr.fock, pr.chol, pr.t1, pr.t2, o=o)
    G = orc.green(OMEGAS, ETA, orbs, tol=1e-13)
    ref = np.zeros_like(G)
    for w, om in enumerate(OMEGAS):
        for p in orbs:
            ref[w, p, p] = 1.0 / (om - eps[p] - 1j * ETA) if p < o else 1.0 / (om - eps[p] + 1j * ETA)
    np.testing.assert_allclose(G, ref, atol=1e-12)
    bf = BruteForceGFCC(pr.fock, pr.chol, pr.t1, pr.t2, pr.t1, pr.t2, o)
    np.testing.assert_allclose(bf.green_ip(OMEGAS, ETA, orbs) + bf.green_ea(OMEGAS, ETA, orbs), ref, atol=1e-12)


def test_no_two_electron_integrals_closed_form():
    """chol = 0, any T and Lambda: the operator is diagonal, M_i = -eps_i, M_ija = eps_a - eps_i - eps_j,
    M_a = eps_a, M_iab = eps_a + eps_b - eps_i, so G is a sum over the basis of c(mu) b(mu) / denominator."""
    o, v = 3, 4
    pr = make_problem(o, v, 4, seed=9, t1_std=0.1, t2_std=0.1, separate_lambda=True)
    pr.chol[:] = 0.0
    eps = pr.eps()
    eo, ev = eps[:o], eps[o:]
    orc = GFCCOracle(pr.fock, pr.chol, pr.t1, pr.t2, pr.lam1, pr.lam2, o)
    ii, jj = np.triu_indices(o, 1)
    d_ip = np.concatenate([-eo, (ev[None, :] - eo[ii][:, None] - eo[jj][:, None]).reshape(-1)])
    aa, bb = np.triu_indices(v, 1)
    d_ea = np.concatenate([ev, (ev[aa][None, :] + ev[bb][None, :] - eo[:, None]).reshape(-1)])
    orbs = list(range(o + v))
    G = orc.green(OMEGAS, ETA, orbs, tol=1e-13)
    ref = np.zeros_like(G)
    for w, om in enumerate(OMEGAS):
        for a, p in enumerate(orbs):
            for b, q in enumerate(orbs):
                ref[w, a, b] = (np.sum(orc.ip_left(q) * orc.ip_rhs(p) / (om - 1j * ETA + d_ip))
                                + np.sum(orc.ea_left(p) * orc.ea_rhs(q) / (om + 1j * ETA - d_ea)))
    np.testing.assert_allclose(G, ref, atol=1e-11)


# ---------------------------------------------------------------- 4. mathematics
def test_T0_operator_is_symmetric_and_sum_over_states():
    o, v = 3, 6
    pr = make_problem(o, v, 12, seed=4, with_t=False)
    orc = GFCCOracle(pr.fock, pr.chol, pr.t1, pr.t2, o=o)
    orbs = list(range(o + v))
    for M in (orc.ip_matrix(), orc.ea_matrix()):
        assert np.abs(M - M.T).max() <= 1e-13 * np.abs(M).max()
    Mi, Me = orc.ip_matrix(), orc.ea_matrix()
    li, Ui = sla.eigh(Mi)
    le, Ue = sla.eigh(Me)
    G = orc.green(OMEGAS, ETA, orbs, tol=1e-13)
    Bi = np.stack([orc.ip_rhs(p) for p in orbs]); Ci = np.stack([orc.ip_left(q) for q in orbs])
    Be = np.stack([orc.ea_rhs(q) for q in orbs]); Ce = np.stack([orc.ea_left(p) for p in orbs])
    for w, om in enumerate(OMEGAS):
        ref = ((Bi @ Ui) / (om - 1j * ETA + li)) @ (Ci @ Ui).T      # [p][q]
        ref = ref + ((Ce @ Ue) / (om + 1j * ETA - le)) @ (Be @ Ue).T
        np.testing.assert_allclose(G[w], ref, atol=1e-11)


def test_sigma_is_linear():
    o, v = 4, 7
    pr = make_problem(o, v, 10, seed=12, t1_std=0.05, t2_std=0.05)
    orc = GFCCOracle(pr.fock, pr.chol, pr.t1, pr.t2, o=o)
    for dim, sig in ((ip_dim(o, v), orc.ip_sigma), (ea_dim(o, v), orc.ea_sigma)):
        x = random_vector(1, dim) + 1j * random_vector(2, dim)
        y = random_vector(3, dim) + 1j * random_vector(4, dim)
        al, be = 0.3 - 1.7j, -2.1 + 0.4j
        np.testing.assert_allclose(sig(al * x + be * y), al * sig(x) + be * sig(y), atol=1e-12)
        # planar form: sigma of a complex vector is sigma(Re) + i sigma(Im) (real Hbar)
        np.testing.assert_allclose(sig(x), sig(x.real) + 1j * sig(x.imag), atol=1e-12)


def test_gmres_matches_dense_lu_and_is_monotone(tiny_pair):
    pr, bf, orc = tiny_pair
    orbs = list(range(16))
    om = np.linspace(-1.0, -0.2, 4)
    G_lu = orc.green_dense(om, 0.01, orbs, sectors=("IP",))
    n = ip_dim(4, 12)
    stats = []
    G_gm = orc.green(om, 0.01, orbs, tol=1e-12, restart=n, max_restarts=3, sectors=("IP",), stats=stats)
    assert np.abs(G_gm - G_lu).max() <= 1e-10 * np.abs(G_lu).max()
    assert all(s[5] for s in stats)
    assert max(s[3] for s in stats) <= n            # full GMRES converges within dim steps
    A = orc.ip_apply(-0.5, 0.01)
    hist = []
    gmres(A, orc.ip_rhs(2), 1e-12, restart=10, max_restarts=20, history=hist)
    # monotone up to the rounding between the Givens estimate and the recomputed true residual
    assert all(b <= a * (1 + 1e-8) + 1e-15 for a, b in zip(hist, hist[1:]))
    # against the brute-force definition as well
    G_bf = bf.green_ip(om, 0.01, orbs)
    assert np.abs(G_gm - G_bf).max() <= 1e-10 * np.abs(G_bf).max()


def test_large_omega_moments():
    """G(omega) = c.b/(omega - i eta) - c.(M b)/(omega - i eta)^2 + O(omega^-3) for the IP part."""
    o, v = 3, 5
    pr = make_problem(o, v, 8, seed=2, t1_std=0.05, t2_std=0.05)
    orc = GFCCOracle(pr.fock, pr.chol, pr.t1, pr.t2, o=o)
    p, q = 1, 4
    b, c = orc.ip_rhs(p), orc.ip_left(q)
    m0, m1 = c @ b, c @ orc.ip_sigma(b)
    for om in (200.0, 400.0):
        z = om - 1j * ETA
        g = orc.green(np.array([om]), ETA, [p, q], tol=1e-14, sectors=("IP",))[0, 0, 1]
        err = abs(g - (m0 / z - m1 / z ** 2))
        assert err <= 50.0 / om ** 3


def test_preconditioned_gmres_same_solution(tiny_pair):
    """A diagonal right preconditioner changes the Krylov space, not the solution of eq. xplin."""
    pr, bf, orc = tiny_pair
    orbs = [0, 3, 4, 9]
    om = np.array([-0.9, -0.3])
    G_lu = orc.green_dense(om, 0.01, orbs)
    G_pc = orc.green(om, 0.01, orbs, tol=1e-12, restart=30, max_restarts=40, precond=True)
    assert np.abs(G_pc - G_lu).max() <= 1e-10 * np.abs(G_lu).max()
