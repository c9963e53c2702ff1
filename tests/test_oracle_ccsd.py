"""Pins of the CCSD / Lambda-CCSD oracle (oracle/ccsd_ref.py) on the CPU, against the Fock-space
definition (oracle/fock_space.py):

* the T residuals are the projections <mu| e^-T H e^T |Phi> on every single and double, at random T1,
  T2 with the Cholesky vectors, T1 and T2 switched on one at a time and together;
* the correlation energy is <Phi| e^-T H e^T |Phi> - <Phi|H|Phi>;
* the Lambda residuals are <Phi|(1 + Lambda)(Hbar - E0)|mu> at random Lambda and converged T;
* for two electrons CCSD is exact: the converged energy equals the full-CI ground state of the
  two-electron sector, and T and Lambda equal the full-space CC solution of the definition.
"""
import itertools

import numpy as np
import pytest

from oracle import ccsd_ref as C
from oracle import fock_space as F
from paper_2010_04768_gb300.synthetic import make_problem


def brute(pr, o, t1, t2):
    n = pr.n
    fs = F.FockSpace(n)
    H = F.hamiltonian(fs, pr.fock, pr.chol, o, o)
    masks, index = fs.sector(o)
    phi = np.zeros(fs.dim(o))
    phi[index[(1 << o) - 1]] = 1.0
    T = F.excitation_operator(fs, o, t1, t2, o)

    def hbar(x):
        return F.apply_exp(T, H @ F.apply_exp(T, x, 1.0), -1.0)

    v = n - o
    singles = {(i, a): fs.excitation(o + a, i, o) @ phi for i in range(o) for a in range(v)}
    doubles = {(i, j, a, b): fs.excitation(o + a, i, o) @ (fs.excitation(o + b, j, o) @ phi)
               for i, j in itertools.combinations(range(o), 2) for a, b in itertools.combinations(range(v), 2)}
    return fs, H, phi, hbar, singles, doubles


def amplitudes(o, v, seed, s1=0.05, s2=0.05):
    rng = np.random.default_rng(seed)
    t1 = s1 * rng.standard_normal((o, v))
    g = s2 * rng.standard_normal((o, o, v, v))
    t2 = 0.25 * (g - g.transpose(1, 0, 2, 3) - g.transpose(0, 1, 3, 2) + g.transpose(1, 0, 3, 2))
    return t1, t2


@pytest.mark.parametrize("o,v,mode", [(2, 4, "t1"), (2, 4, "t2"), (3, 4, "t2"), (3, 4, "both"), (2, 5, "both")])
def test_t_residuals_and_energy_match_definition(o, v, mode):
    pr = make_problem(o, v, 5, seed=o * 10 + v, chol_sigma=0.3)
    t1, t2 = amplitudes(o, v, 7)
    if mode == "t1":
        t2 = np.zeros_like(t2)
    if mode == "t2":
        t1 = np.zeros_like(t1)
    fs, H, phi, hbar, singles, doubles = brute(pr, o, t1, t2)
    r = hbar(phi)
    r1, r2 = C.t_residuals(pr.fock, pr.chol, t1, t2, o)
    scale = np.abs(r).max()
    for (i, a), s in singles.items():
        assert abs(s @ r - r1[i, a]) <= 1e-12 * scale
    for (i, j, a, b), d in doubles.items():
        assert abs(d @ r - r2[i, j, a, b]) <= 1e-12 * scale
    assert np.allclose(r2, -r2.transpose(1, 0, 2, 3), atol=1e-14) and np.allclose(r2, -r2.transpose(0, 1, 3, 2),
                                                                                     atol=1e-14)
    e_ref = phi @ (H @ phi)
    assert C.correlation_energy(pr.fock, pr.chol, t1, t2, o) == pytest.approx(phi @ r - e_ref, abs=1e-12)


@pytest.mark.parametrize("o,v", [(2, 4), (3, 4)])
def test_lambda_residuals_match_definition(o, v):
    pr = make_problem(o, v, 5, seed=o * 11 + v, chol_sigma=0.2)
    # the Lambda equations hold where T solves the T equations (the disconnected terms of
    # <nu|Hbar|mu> that carry a T residual are dropped from them); Lambda is random
    t1, t2, _, _ = C.solve_t(pr.fock, pr.chol, o, tol=1e-14)
    l1, l2 = amplitudes(o, v, 9, 0.1, 0.1)
    fs, H, phi, hbar, singles, doubles = brute(pr, o, t1, t2)
    E0 = phi @ hbar(phi)
    # <Phi|(1 + Lambda) as a vector: the de-excitation Lambda is the transpose of the excitation
    # operator with the same amplitudes
    Lexc = F.excitation_operator(fs, o, l1, l2, o)
    ell = phi + Lexc @ phi
    E = C.lambda_elements(pr.fock, pr.chol, t1, t2, o)
    r1, r2 = C.lambda_residuals(E, t2, l1, l2)
    vals = {}
    for key, mu in list(singles.items()) + list(doubles.items()):
        vals[key] = ell @ (hbar(mu) - E0 * mu)
    scale = max(abs(x) for x in vals.values())
    for (i, a), s in singles.items():
        assert abs(vals[(i, a)] - r1[i, a]) <= 1e-11 * scale
    for (i, j, a, b), d in doubles.items():
        assert abs(vals[(i, j, a, b)] - r2[i, j, a, b]) <= 1e-11 * scale


def test_two_electron_ccsd_is_exact():
    o, v = 2, 5
    pr = make_problem(o, v, 6, seed=3, chol_sigma=0.3)
    t1, t2, ec, its = C.solve_t(pr.fock, pr.chol, o, tol=1e-12)
    l1, l2, lits = C.solve_lambda(pr.fock, pr.chol, t1, t2, o, tol=1e-12)
    fs = F.FockSpace(o + v)
    H = F.hamiltonian(fs, pr.fock, pr.chol, o, o).toarray()
    masks, index = fs.sector(o)
    phi = np.zeros(fs.dim(o))
    phi[index[(1 << o) - 1]] = 1.0
    e_fci = np.linalg.eigvalsh(H)[0]
    assert ec == pytest.approx(e_fci - phi @ H @ phi, abs=1e-10)
    et1, et2, el1, el2, E0 = F.solve_cc_exact(pr.fock, pr.chol, o)
    assert np.abs(t1 - et1).max() <= 1e-9 and np.abs(t2 - et2).max() <= 1e-9
    assert np.abs(l1 - el1).max() <= 1e-8 and np.abs(l2 - el2).max() <= 1e-8
