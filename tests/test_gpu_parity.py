"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Tolerances: the sigma product is a fixed sequence of FP64 contractions, so it
must agree with the oracle to rounding (1e-12 relative to the largest element);
G(omega) from GMRES at tol 1e-12 must agree with the oracle's dense solution to
1e-10 relative (the FP64 parity bar of the hot path).
"""
import numpy as np
import pytest

from paper_2010_04768_gb300 import gfcc
from paper_2010_04768_gb300.synthetic import make_problem, random_vector, workload
from oracle.gfcc_ref import GFCCOracle, ip_dim, ea_dim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session", autouse=True)
def _built():
    from paper_2010_04768_gb300 import build
    build.build()
    gfcc.load()


def rel_err(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def rand_vectors(dim, count, seed):
    return np.stack([random_vector(seed + k, dim) + 1j * random_vector(seed + 100 + k, dim) for k in range(count)])


# (o, v, L): degenerate spaces (o=1 has no 2h1p pairs, v=1 no 2p1h pairs), the tiny workload,
# sizes that are not multiples of the 64-wide tiles, and several tiles in every GEMM dimension
SIGMA_CASES = [(1, 3, 4), (2, 1, 3), (3, 5, 7), (4, 12, 48), (5, 17, 20), (7, 70, 90)]


@pytest.mark.parametrize("o,v,L", SIGMA_CASES)
def test_sigma_matches_oracle(o, v, L):
    pr = make_problem(o, v, L, seed=o * 31 + v, t1_std=0.05, t2_std=0.05, chol_sigma=0.3)
    g = gfcc.GFCC(pr)
    orc = GFCCOracle(pr.fock, pr.chol, pr.t1, pr.t2, o=o)
    di, de = g.dims()
    assert (di, de) == (ip_dim(o, v), ea_dim(o, v))
    X = rand_vectors(di, 3, 1)
    Y = g.sigma("IP", X)
    ref = np.stack([orc.ip_sigma(x) for x in X])
    assert rel_err(Y, ref) <= 1e-12
    X = rand_vectors(de, 3, 2)
    Y = g.sigma("EA", X)
    ref = np.stack([orc.ea_sigma(x) for x in X])
    assert rel_err(Y, ref) <= 1e-12
    g.close()


@pytest.mark.parametrize("precond", [gfcc.PRECOND_NONE, gfcc.PRECOND_DIAG])
def test_green_tiny_workload_matches_oracle(precond):
    wl = workload("tiny")
    pr = wl.problem()
    g = gfcc.GFCC(pr, sectors="IP")
    g.set_option(gfcc.OPT_PRECOND, precond)
    g.set_option(gfcc.OPT_RESTART, 40)
    G, code = g.solve(wl.omegas, wl.eta, wl.orbitals, 1e-12)
    assert code == gfcc.OK
    orc = GFCCOracle(pr.fock, pr.chol, pr.t1, pr.t2, o=wl.o, sectors=("IP",))
    ref = orc.green_dense(wl.omegas, wl.eta, list(wl.orbitals), sectors=("IP",))
    assert rel_err(G, ref) <= 1e-10
    it, rr, st = g.stats()
    assert it.size == wl.omegas.size * wl.orbitals.size
    assert np.all(st == 0) and np.all(rr <= 1e-12) and np.all(it > 0)
    g.close()


@pytest.mark.parametrize("precond", [gfcc.PRECOND_NONE, gfcc.PRECOND_DIAG])
@pytest.mark.parametrize("batch", [0, 5])
def test_green_ip_ea_separate_lambda(precond, batch):
    o, v = 3, 6
    pr = make_problem(o, v, 9, seed=5, t1_std=0.05, t2_std=0.05, separate_lambda=True, chol_sigma=0.3)
    om = np.array([-0.8, -0.1, 0.6])
    orbs = np.array([0, 2, 3, 8], dtype=np.int32)
    g = gfcc.GFCC(pr)
    g.set_option(gfcc.OPT_PRECOND, precond)
    g.set_option(gfcc.OPT_BATCH, batch)
    G, code = g.solve(om, 0.05, orbs, 1e-12)
    assert code == gfcc.OK
    orc = GFCCOracle(pr.fock, pr.chol, pr.t1, pr.t2, pr.lam1, pr.lam2, o)
    ref = orc.green_dense(om, 0.05, list(orbs))
    assert rel_err(G, ref) <= 1e-10
    g.close()


def test_green_hartree_fock_limit():
    o, v = 3, 5
    pr = make_problem(o, v, 4, seed=7, with_t=False)
    pr.chol[:] = 0.0
    eps = pr.eps()
    om = np.array([-0.7, 0.3])
    orbs = np.arange(o + v, dtype=np.int32)
    g = gfcc.GFCC(pr)
    G, code = g.solve(om, 0.02, orbs, 1e-13)
    assert code == gfcc.OK
    ref = np.zeros_like(G)
    for w, x in enumerate(om):
        for p in orbs:
            ref[w, p, p] = 1.0 / (x - eps[p] - 0.02j) if p < o else 1.0 / (x - eps[p] + 0.02j)
    np.testing.assert_allclose(G, ref, atol=1e-12)
    g.close()


def test_medium_columns_match_oracle():
    """Several 64-wide tiles in every contraction; a few (omega, p) columns of G against the oracle's GMRES."""
    o, v, L = 10, 50, 100
    pr = make_problem(o, v, L, seed=3)
    orc = GFCCOracle(pr.fock, pr.chol, pr.t1, pr.t2, o=o)
    g = gfcc.GFCC(pr)
    di, de = g.dims()
    X = rand_vectors(di, 2, 7)
    assert rel_err(g.sigma("IP", X), np.stack([orc.ip_sigma(x) for x in X])) <= 1e-12
    X = rand_vectors(de, 2, 8)
    assert rel_err(g.sigma("EA", X), np.stack([orc.ea_sigma(x) for x in X])) <= 1e-12
    om = np.array([-0.9, 0.2])
    orbs = np.array([o - 1, o], dtype=np.int32)
    # both solvers well below the 1e-10 bar: the G error of a solve is at most ||c_q|| ||A^-1|| times
    # its residual (||A^-1|| <= 1 / eta on the dominant diagonal), so residuals of 1e-13 (GPU) and
    # 1e-14 (oracle) leave G agreeing to about 1e-11
    G, code = g.solve(om, 0.01, orbs, 1e-13)
    it, rr, st = g.stats()
    assert code == gfcc.OK and np.all(st == 0) and np.all(rr <= 1e-13)
    ref = orc.green(om, 0.01, list(orbs), tol=1e-14, restart=60, max_restarts=60, precond=True)
    assert rel_err(G, ref) <= 1e-10
    g.close()


def test_block_solve_matches_full_solve():
    # gfcc_solve_block: rows over P, columns over Q, IP solved per row orbital and EA per column orbital;
    # the block equals the same entries of the full solve over the union of the lists
    o, v, L = 4, 12, 48
    pr = make_problem(o, v, L, seed=8)
    om = np.array([-0.7, 0.35])
    allo = np.arange(o + v, dtype=np.int32)
    P = np.array([1, 3, 9], dtype=np.int32)
    Q = np.array([0, 3, 5, 12, 15], dtype=np.int32)
    g = gfcc.GFCC(pr)
    Gf, code = g.solve(om, 0.01, allo, 1e-12)
    assert code == gfcc.OK
    Gb, code = g.solve_block(om, 0.01, P, Q, 1e-12)
    assert code == gfcc.OK and Gb.shape == (2, 3, 5)
    it, rr, st = g.stats()
    assert it.size == om.size * (P.size + Q.size)       # IP systems over P, EA systems over Q
    assert rel_err(Gb, Gf[:, P][:, :, Q]) <= 1e-10
    ref = GFCCOracle(pr.fock, pr.chol, pr.t1, pr.t2, o=o).green_dense(om, 0.01, list(allo))
    assert rel_err(Gb, ref[:, P][:, :, Q]) <= 1e-10
    g.close()


def test_ea_inside_the_2p1h_continuum_has_a_defined_outcome():
    # frequencies inside the EA 2p1h continuum (eps_a + eps_b - eps_i), mixed precision with the
    # preconditioner: every column either converges (true residual <= tol, G within 1e-6 of the
    # oracle's dense solution) or is reported not converged with a finite G
    o, v, L = 4, 12, 48
    pr = make_problem(o, v, L, seed=9)
    om = np.array([0.9, 1.6, 2.4])
    orbs = np.array([o - 1, o, o + 1, o + 5], dtype=np.int32)
    g = gfcc.GFCC(pr, sectors="EA", precision="mixed")
    g.set_option(gfcc.OPT_MAX_ITERS, 3000)
    G, code = g.solve(om, 0.01, orbs, 1e-10)
    it, rr, st = g.stats()
    g.close()
    assert code in (gfcc.OK, gfcc.WARN_NOT_CONVERGED) and np.isfinite(G).all()
    assert (code == gfcc.OK) == bool(np.all(st == 0))
    ref = GFCCOracle(pr.fock, pr.chol, pr.t1, pr.t2, o=o, sectors=("EA",)).green_dense(om, 0.01, list(orbs),
                                                                                       sectors=("EA",))
    for w in range(om.size):
        for b in range(orbs.size):
            k = w * orbs.size + b          # EA statistics: omega-major over the column orbitals
            if st[k] == 0:
                assert rr[k] <= 1e-10
                assert np.linalg.norm(G[w, :, b] - ref[w, :, b]) <= 1e-6 * np.linalg.norm(ref[w, :, b])
            else:
                assert st[k] == 1 and rr[k] > 1e-10


def test_bad_inputs_are_rejected():
    pr = make_problem(3, 4, 5, seed=1)
    bad = make_problem(3, 4, 5, seed=1)
    bad.t2[0, 1, 0, 1] += 1e-3                      # breaks antisymmetry
    with pytest.raises(gfcc.GFCCError) as e:
        gfcc.GFCC(bad)
    assert e.value.code == gfcc.ERR_ARG
    bad = make_problem(3, 4, 5, seed=1)
    bad.chol[2, 1, 1] = np.nan
    with pytest.raises(gfcc.GFCCError):
        gfcc.GFCC(bad)
    g = gfcc.GFCC(pr)
    with pytest.raises(gfcc.GFCCError):
        g.solve([0.1], 0.01, [7], 1e-8)             # orbital out of range
    with pytest.raises(gfcc.GFCCError):
        g.solve([0.1], -0.01, [0], 1e-8)            # eta <= 0
    with pytest.raises(gfcc.GFCCError):
        g.set_option(gfcc.OPT_RESTART, 0)
    G, code = g.solve([0.1], 0.01, [0], 1e-8)      # the context is still usable
    assert code == gfcc.OK and np.isfinite(G).all()
    g.close()


def test_not_converged_is_reported():
    wl = workload("tiny")
    pr = wl.problem()
    g = gfcc.GFCC(pr, sectors="IP")
    g.set_option(gfcc.OPT_PRECOND, gfcc.PRECOND_NONE)
    g.set_option(gfcc.OPT_RESTART, 2)
    g.set_option(gfcc.OPT_MAX_ITERS, 3)
    G, code = g.solve(wl.omegas[:1], wl.eta, wl.orbitals[:4], 1e-12)
    assert code == gfcc.WARN_NOT_CONVERGED
    it, rr, st = g.stats()
    assert np.all(st == 1) and np.all(it <= 4) and np.isfinite(G).all()
    g.close()


def test_solve_batch_matches_individual_solves():
    # molecules of uneven sizes solved concurrently (one stream and host thread per context)
    shapes = [(3, 9, 20), (5, 15, 30), (4, 12, 48), (6, 20, 40)]
    ctxs, reqs, refs = [], [], []
    for k, (o, v, L) in enumerate(shapes):
        pr = make_problem(o, v, L, seed=20 + k)
        om = np.linspace(-1.0, 0.4, 3 + k)
        orbs = np.arange(max(0, o - 2), min(o + v, o + 2), dtype=np.int32)
        g = gfcc.GFCC(pr, sectors="IP+EA", precision="fp64" if k % 2 == 0 else "mixed")
        ref, code = g.solve(om, 0.01, orbs, 1e-10)
        ctxs.append(g)
        reqs.append((om, 0.01, orbs, 1e-10))
        refs.append(ref)
    Gs, codes = gfcc.solve_batch(ctxs, reqs)
    assert np.all(codes >= 0)
    for G, ref in zip(Gs, refs):
        assert rel_err(G, ref) <= 1e-8
    # every molecule against the oracle's dense solution: FP64 contexts at 1e-8 (solver tol 1e-10
    # times ||A^-1|| <= 1 / eta = 100), mixed ones at the mixed-precision bar of 1e-6
    for k, ((o, v, L), G, (om, eta, orbs, tol)) in enumerate(zip(shapes, Gs, reqs)):
        pr = make_problem(o, v, L, seed=20 + k)
        ref = GFCCOracle(pr.fock, pr.chol, pr.t1, pr.t2, o=o).green_dense(om, eta, list(orbs))
        assert rel_err(G, ref) <= (1e-8 if k % 2 == 0 else 1e-6)
    for g in ctxs:
        g.close()
