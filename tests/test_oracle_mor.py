"""Pins of the model-order-reduction oracle (oracle/mor_ref.py) on the CPU.

* a subspace spanning the whole space reproduces the exact G (dense LU of the full operator);
* the Galerkin model interpolates: at the sampled frequencies it reproduces the full solutions' G;
* Hhat = S^T Hbar S against the explicit dense operator matrix; S orthonormal; dependent vectors
  dropped;
* the model residual from W = Hbar S equals the dense residual of the lifted model solution;
* spectral function: the Hartree-Fock closed form (T = Lambda = 0, no Cholesky vectors);
* levels: the paper's worked example of the level bound (tests/golden/lmax_worked_example.txt),
  N_max(L), and a driver whose indicator never falls below the tolerance bisects down to the
  resolution in exactly that many levels.
"""
import math
import os

import numpy as np
import pytest

from oracle import mor_ref as R
from oracle.gfcc_ref import GFCCOracle, ip_dim, ea_dim
from paper_2010_04768_gb300.synthetic import make_problem

HERE = os.path.dirname(os.path.abspath(__file__))


def small(o=3, v=5, L=6, seed=4, **kw):
    pr = make_problem(o, v, L, seed=seed, t1_std=0.05, t2_std=0.05, chol_sigma=0.3, **kw)
    return pr, GFCCOracle(pr.fock, pr.chol, pr.t1, pr.t2, o=o)


@pytest.mark.parametrize("sector", ["IP", "EA"])
def test_whole_space_subspace_reproduces_exact_green(sector):
    pr, orc = small()
    n = ip_dim(3, 5) if sector == "IP" else ea_dim(3, 5)
    rng = np.random.default_rng(1)
    S = R.orthonormal_extend(None, list(rng.normal(size=(n, n))))
    assert S.shape == (n, n)
    sig = orc.ip_sigma if sector == "IP" else orc.ea_sigma
    Hh, W = R.project(sig, S)
    orbs = list(range(8))
    B = np.stack([(orc.ip_rhs(p) if sector == "IP" else orc.ea_rhs(p)) for p in orbs], axis=1)
    C = np.stack([(orc.ip_left(p) if sector == "IP" else orc.ea_left(p)) for p in orbs], axis=1)
    om = np.array([-0.7, 0.1, 0.9])
    G = R.model_green(Hh, S, B, C, om, 0.02, sector)
    ref = orc.green_dense(om, 0.02, orbs, sectors=(sector,))
    assert np.abs(G - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("sector", ["IP", "EA"])
def test_model_interpolates_at_sampled_frequencies(sector):
    pr, orc = small(o=3, v=6, L=8, seed=5)
    M = orc.ip_matrix() if sector == "IP" else orc.ea_matrix()
    n = M.shape[0]
    orbs = [1, 2, 3, 4]
    B = np.stack([(orc.ip_rhs(p) if sector == "IP" else orc.ea_rhs(p)) for p in orbs], axis=1).astype(complex)
    C = np.stack([(orc.ip_left(p) if sector == "IP" else orc.ea_left(p)) for p in orbs], axis=1)
    eta = 0.02
    samp = [-0.6, 0.2]
    X = []
    for om in samp:
        A = ((om - 1j * eta) * np.eye(n) + M) if sector == "IP" else ((om + 1j * eta) * np.eye(n) - M)
        X += list(np.linalg.solve(A, B).T)
    S = R.orthonormal_extend(None, R.real_parts(X))
    assert S.shape[1] <= 2 * len(X) and S.shape[1] < n
    assert np.abs(S.T @ S - np.eye(S.shape[1])).max() <= 1e-13
    Hh, W = R.project(orc.ip_sigma if sector == "IP" else orc.ea_sigma, S)
    # the projection against the explicit operator matrix
    assert np.abs(Hh - S.T @ M @ S).max() <= 1e-12 * np.abs(Hh).max()
    G = R.model_green(Hh, S, B.real, C, np.array(samp), eta, sector)
    ref = orc.green_dense(np.array(samp), eta, orbs, sectors=(sector,))
    assert np.abs(G - ref).max() <= 1e-10 * np.abs(ref).max()
    # between the samples the model is an approximation, not the exact G
    Gm = R.model_green(Hh, S, B.real, C, np.array([-0.2]), eta, sector)
    refm = orc.green_dense(np.array([-0.2]), eta, orbs, sectors=(sector,))
    assert np.abs(Gm - refm).max() > 1e-8 * np.abs(refm).max()
    # the model residual from W equals the dense residual of the lifted solution
    for om in (-0.6, -0.2):
        b = B[:, 0]
        r = R.model_relres(Hh, S, W, b, om, eta, sector)
        xh = R.model_solution(Hh, S, b, om, eta, sector)
        A = ((om - 1j * eta) * np.eye(n) + M) if sector == "IP" else ((om + 1j * eta) * np.eye(n) - M)
        ref_r = np.linalg.norm(b - A @ (S @ xh)) / np.linalg.norm(b)
        assert r == pytest.approx(ref_r, rel=1e-9, abs=1e-14)
    assert R.model_relres(Hh, S, W, B[:, 0], -0.6, eta, sector) <= 1e-10


def test_dependent_vectors_are_dropped():
    rng = np.random.default_rng(3)
    a, b = rng.normal(size=40), rng.normal(size=40)
    S = R.orthonormal_extend(None, [a, b, 2.0 * a - 3.0 * b, np.zeros(40)])
    assert S.shape == (40, 2)
    S2 = R.orthonormal_extend(S, [a + 1e-3 * rng.normal(size=40)])
    assert S2.shape == (40, 3) and np.abs(S2.T @ S2 - np.eye(3)).max() <= 1e-13


def test_spectral_function_hartree_fock_limit():
    o, v = 3, 4
    pr = make_problem(o, v, 2, seed=6, with_t=False)
    pr.chol[:] = 0.0
    eps = pr.eps()
    orc = GFCCOracle(pr.fock, pr.chol, pr.t1, pr.t2, o=o)
    om = np.linspace(-2.0, 2.5, 19)
    eta = 0.05
    orbs = list(range(o + v))
    Gip = orc.green_dense(om, eta, orbs, sectors=("IP",))
    Gea = orc.green_dense(om, eta, orbs, sectors=("EA",))
    A = R.spectral_function(np.einsum("wpp->wp", Gip), np.einsum("wpp->wp", Gea))
    ref = np.array([sum(eta / ((w - e) ** 2 + eta ** 2) for e in eps) / math.pi for w in om])
    assert np.allclose(A, ref, rtol=1e-12, atol=0)
    assert np.all(A > 0)


def read_golden():
    vals = {}
    for line in open(os.path.join(HERE, "golden", "lmax_worked_example.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, x = line.split()
        vals[k] = float(x)
    return vals


def test_level_bound_worked_example():
    g = read_golden()
    assert R.l_max_bound(g["omega_min"], g["omega_max"], g["d_omega"]) == int(g["l_max"])
    assert [R.n_max(L) for L in range(1, 6)] == [3, 2, 4, 8, 16]
    # an indicator that never falls below the tolerance: full bisection down to the resolution
    levels = R.adaptive_levels(lambda w, s: 1.0, g["omega_min"], g["omega_max"], g["d_omega"], 1e-3)
    assert len(levels) == int(g["l_max"])
    assert [len(x) for x in levels] == [3, 2, 4, 8, 16]
    allw = np.sort(np.concatenate([np.array(x) for x in levels]))
    assert np.allclose(np.diff(allw), (g["omega_max"] - g["omega_min"]) / 32)
    n_tot = round((g["omega_max"] - g["omega_min"]) / g["d_omega"]) + 1
    assert sum(len(x) for x in levels) <= n_tot
    # an indicator that is satisfied after the first level stops there
    assert len(R.adaptive_levels(lambda w, s: 0.0, -0.8, -0.4, 0.01, 1e-3)) == 1
