"""Pins of the closed-shell spin-adapted GFCCSD-IP oracle (oracle/rhf_ref.py) on the CPU.

* The spin-adapted coordinates are exact: the spin-orbital sigma of the embedding maps the doublet
  subspace into itself, and the right-hand sides lie in it (so the spatial solve is the spin-orbital
  solve).
* The closed-form spatial sigma, right-hand sides, left vectors and Fock-like diagonal equal the
  definition (spin-orbital quantities of the embedding, gfcc_ref) element by element, with T1, T2,
  Lambda and the Cholesky vectors switched on one at a time and together.
* The spatial G equals the spin-orbital G_{p alpha, q alpha} of the embedding (dense solves), and the
  closed-form GMRES G equals the dense one.
* Two electrons (one doubly occupied spatial orbital): with the converged CCSD / Lambda-CCSD
  amplitudes of the embedding (oracle/ccsd_ref.py) the spatial G is the exact Lehmann G of eq. gfxn0
  (oracle/fock_space.py), a pin of the whole chain to the formula-free definition.
"""
import numpy as np
import pytest

from oracle import ccsd_ref as CC
from oracle import fock_space as F
from oracle import gfcc_ref as S
from oracle import rhf_ref as R
from paper_2010_04768_gb300.synthetic import make_problem


def closed_shell_amplitudes(o, v, seed, s1=0.05, s2=0.05):
    rng = np.random.default_rng(seed)
    t1 = s1 * rng.standard_normal((o, v))
    g = s2 * rng.standard_normal((o, o, v, v))
    return t1, g + g.transpose(1, 0, 3, 2)          # t_ij^ab = t_ji^ba


def test_embedding_of_amplitudes_is_antisymmetric_and_spin_conserving():
    o, v = 3, 4
    t1, t2 = closed_shell_amplitudes(o, v, 1)
    T1, T2 = R.embed_amplitudes(t1, t2, o, v)
    assert np.allclose(T2, -T2.transpose(1, 0, 2, 3)) and np.allclose(T2, -T2.transpose(0, 1, 3, 2))
    assert np.array_equal(T1[:o, :v], t1) and np.all(T1[:o, v:] == 0) and np.array_equal(T1[o:, v:], t1)
    assert np.array_equal(T2[:o, o:, :v, v:], t2)                       # alpha beta alpha beta
    assert np.allclose(T2[:o, :o, :v, :v], t2 - t2.transpose(0, 1, 3, 2))   # all alpha
    assert np.all(T2[:o, :o, v:, v:] == 0) and np.all(T2[:o, o:, :v, :v] == 0)


@pytest.mark.parametrize("mode", ["bare", "t1", "t2", "lambda", "all"])
@pytest.mark.parametrize("o,v", [(2, 3), (3, 3)])
def test_closed_form_equals_definition(o, v, mode):
    pr = make_problem(o, v, 4, seed=10 * o + v, chol_sigma=0.3)
    t1, t2 = closed_shell_amplitudes(o, v, 2)
    l1, l2 = closed_shell_amplitudes(o, v, 3, 0.08, 0.08)
    a1 = t1 if mode in ("t1", "all") else np.zeros_like(t1)
    a2 = t2 if mode in ("t2", "all") else np.zeros_like(t2)
    b1, b2 = (l1, l2) if mode in ("lambda", "all") else (None, None)
    D = R.RHFIP(pr.fock, pr.chol, a1, a2, b1, b2, o=o)
    C = R.RHFClosed(pr.fock, pr.chol, a1, a2, b1, b2, o=o)
    rng = np.random.default_rng(4)
    for _ in range(3):
        x = rng.standard_normal(D.dim())
        X = D.so.ip_sigma(D.embed(x))
        assert np.abs(D.embed(D.project(X)) - X).max() <= 1e-13 * np.abs(X).max()   # the subspace is invariant
        sd = D.sigma(x)
        assert np.abs(C.sigma(x) - sd).max() <= 1e-13 * np.abs(sd).max()
    for p in range(o + v):
        b = D.so.ip_rhs(int(D.alpha[p]))
        assert np.abs(D.embed(D.project(b)) - b).max() <= 1e-15                  # b_p in the subspace
        assert np.abs(C.rhs(p) - D.rhs(p)).max() <= 1e-15
        assert np.abs(C.left(p) - D.left(p)).max() <= 1e-14
    assert np.abs(C.diag() - D.diag()).max() <= 1e-13


def test_spatial_green_function_equals_spin_orbital_alpha_block():
    o, v = 2, 4
    pr = make_problem(o, v, 5, seed=7, chol_sigma=0.3)
    t1, t2 = closed_shell_amplitudes(o, v, 5)
    l1, l2 = closed_shell_amplitudes(o, v, 6, 0.08, 0.08)
    D = R.RHFIP(pr.fock, pr.chol, t1, t2, l1, l2, o=o)
    om, eta = np.array([-1.1, -0.5, 0.2]), 0.05
    orbs = list(range(o + v))
    Gs = D.green_dense(om, eta, orbs)
    M = D.so.ip_matrix()
    al = D.alpha
    B = np.stack([D.so.ip_rhs(int(al[p])) for p in orbs], axis=1).astype(complex)
    Cl = np.stack([D.so.ip_left(int(al[q])) for q in orbs], axis=1)
    for w, z in enumerate(om):
        X = np.linalg.solve((z - 1j * eta) * np.eye(M.shape[0]) + M, B)
        assert np.abs(Gs[w] - (Cl.T @ X).T).max() <= 1e-12 * np.abs(Gs[w]).max()
    C = R.RHFClosed(pr.fock, pr.chol, t1, t2, l1, l2, o=o)
    Gg = C.green(om, eta, orbs, tol=1e-13, restart=D.dim(), max_restarts=5)
    assert np.abs(Gg - Gs).max() <= 1e-10 * np.abs(Gs).max()


def test_two_electrons_spatial_green_function_is_exact():
    o, v = 1, 4
    pr = make_problem(o, v, 5, seed=9, chol_sigma=0.3)
    Fs, Ls = R.embed_problem(pr.fock, pr.chol, o)
    T1, T2, _, _ = CC.solve_t(Fs, Ls, 2 * o, tol=1e-13)
    L1, L2, _ = CC.solve_lambda(Fs, Ls, T1, T2, 2 * o, tol=1e-13)
    # the converged amplitudes are spin adapted; their alpha / alpha-beta components are the spatial ones
    t1, t2 = T1[:o, :v], T2[:o, o:, :v, v:]
    l1, l2 = L1[:o, :v], L2[:o, o:, :v, v:]
    E1, E2 = R.embed_amplitudes(t1, t2, o, v)
    assert np.abs(E1 - T1).max() <= 1e-12 and np.abs(E2 - T2).max() <= 1e-12
    C = R.RHFClosed(pr.fock, pr.chol, t1, t2, l1, l2, o=o)
    om, eta = np.array([-1.3, -0.6, 0.3]), 0.05
    orbs = list(range(o + v))
    Gc = C.green(om, eta, orbs, tol=1e-13, restart=C.dim(), max_restarts=5)
    al, _ = R.so_index(o, v)
    Gx = F.exact_green(Fs, Ls, 2 * o, om, eta, [int(a) for a in al], parts=("IP",))
    assert np.abs(Gc - Gx).max() <= 1e-10 * np.abs(Gx).max()


def test_spatial_space_is_smaller_than_spin_orbital():
    # o + o^2 v spatial coordinates against 2o + o(2o - 1) 2v spin-orbital ones
    assert R.ip_dim(90, 450) == 90 + 90 * 90 * 450
    assert S.ip_dim(180, 900) > 3.9 * R.ip_dim(90, 450)
