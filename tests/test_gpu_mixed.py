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


@pytest.mark.parametrize("o,v,L", [(2, 1, 3), (3, 5, 7), (4, 12, 48), (7, 30, 40)])
def test_mixed_ea_sigma_is_bf16_close(o, v, L):
    pr = make_problem(o, v, L, seed=o + 2 * v, t1_std=0.05, t2_std=0.05, chol_sigma=0.3)
    g = gfcc.GFCC(pr, sectors="EA", precision="mixed")
    orc = GFCCOracle(pr.fock, pr.chol, pr.t1, pr.t2, o=o, sectors=("EA",))
    _, de = g.dims()
    X = np.stack([random_vector(k, de) + 1j * random_vector(60 + k, de) for k in range(3)])
    Y = g.sigma("EA", X, precision="mixed")
    ref = np.stack([orc.ea_sigma(x) for x in X])
    off = ref - orc.ea_diag()[None, :] * X
    if np.abs(off).max() > 0:
        assert np.abs(Y - ref).max() / np.abs(off).max() <= 2e-2
    else:   # v = 1: a single 1p state, the operator is its FP64 diagonal
        assert rel_err(Y, ref) <= 1e-12
    assert rel_err(g.sigma("EA", X), ref) <= 1e-12
    g.close()


@pytest.mark.parametrize("sector", ["IP", "EA"])
@pytest.mark.parametrize("o,v,L", [(3, 5, 7), (4, 12, 48), (7, 30, 40)])
def test_emulated_sigma_is_fp64_accurate(sector, o, v, L):
    # the FP64-accurate operator of the refinement residual: digit planes on the tensor cores
    pr = make_problem(o, v, L, seed=o * 7 + v, t1_std=0.05, t2_std=0.05, chol_sigma=0.3)
    g = gfcc.GFCC(pr, sectors=sector, precision="mixed")
    orc = GFCCOracle(pr.fock, pr.chol, pr.t1, pr.t2, o=o, sectors=(sector,))
    di, de = g.dims()
    dim = di if sector == "IP" else de
    X = np.stack([random_vector(k + 3, dim) + 1j * random_vector(70 + k, dim) for k in range(3)])
    Y = g.sigma(sector, X, precision="fp64emu")
    ref = np.stack([orc.ip_sigma(x) if sector == "IP" else orc.ea_sigma(x) for x in X])
    assert rel_err(Y, ref) <= 1e-12
    g.close()


@pytest.mark.parametrize("precond", [gfcc.PRECOND_NONE, gfcc.PRECOND_DIAG])
def test_mixed_ea_green_matches_oracle(precond):
    # frequencies below and at the bottom of the EA spectrum (deep in the dense 2p1h continuum even
    # plain FP64 GMRES(30) stalls at eta = 0.01 on this size)
    o, v, L = 4, 12, 48
    pr = make_problem(o, v, L, seed=9)
    om = np.array([-0.2, 0.05, 0.3])
    orbs = np.array([o - 1, o, o + 1, o + 5], dtype=np.int32)
    g = gfcc.GFCC(pr, sectors="EA", precision="mixed")
    g.set_option(gfcc.OPT_PRECOND, precond)
    G, code = g.solve(om, 0.01, orbs, 1e-10)
    assert code == gfcc.OK
    ref = GFCCOracle(pr.fock, pr.chol, pr.t1, pr.t2, o=o, sectors=("EA",)).green_dense(om, 0.01, list(orbs),
                                                                                       sectors=("EA",))
    assert rel_err(G, ref) <= 1e-6
    it, rr, st = g.stats()
    assert np.all(st == 0) and np.all(rr <= 1e-10)
    g.close()


def test_mixed_ip_ea_matches_fp64_path():
    o, v, L = 8, 40, 80
    pr = make_problem(o, v, L, seed=5)
    om = np.array([-0.8, 0.3])
    orbs = np.array([o - 2, o - 1, o, o + 1], dtype=np.int32)
    g64 = gfcc.GFCC(pr, sectors="IP+EA")
    G64, c64 = g64.solve(om, 0.005, orbs, 1e-10)
    g64.close()
    gm = gfcc.GFCC(pr, sectors="IP+EA", precision="mixed")
    Gm, cm = gm.solve(om, 0.005, orbs, 1e-10)
    gm.close()
    assert c64 == gfcc.OK and cm == gfcc.OK
    for w in range(om.size):
        for a in range(orbs.size):
            assert np.linalg.norm(Gm[w, a] - G64[w, a]) <= 1e-6 * np.linalg.norm(G64[w, a])


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


@pytest.mark.parametrize("sector", ["IP", "EA"])
def test_incremental_residual_matches_full_residuals(sector):
    # r -= A d at the digit level the correction needs gives the G of the FP64 path, like b - A x at
    # the full level every step, and its products drop digit levels once the corrections shrink
    o, v, L = 8, 40, 80
    pr = make_problem(o, v, L, seed=7)
    om = np.array([-0.9, -0.4, 0.3])
    orbs = np.array([o - 2, o - 1, o, o + 1], dtype=np.int32)
    g64 = gfcc.GFCC(pr, sectors=sector)
    G64, c64 = g64.solve(om, 0.005, orbs, 1e-10)
    g64.close()
    g = gfcc.GFCC(pr, sectors=sector, precision="mixed")
    g.set_option(gfcc.OPT_INCREMENTAL, 0)
    Gf, cf = g.solve(om, 0.005, orbs, 1e-10)
    full0, inc0, _ = g.residual_stats()
    g.set_option(gfcc.OPT_INCREMENTAL, 1)
    Gi, ci = g.solve(om, 0.005, orbs, 1e-10)
    full1, inc1, level = g.residual_stats()
    it, rr, st = g.stats()
    g.close()
    assert c64 == gfcc.OK and cf == gfcc.OK and ci == gfcc.OK
    assert full0 > 0 and inc0 == 0
    assert full1 == 0 and inc1 > 0 and 2 <= level < 9
    assert np.all(st == 0) and np.all(rr <= 1e-10)
    for w in range(om.size):
        for a in range(orbs.size):
            ref = np.linalg.norm(G64[w, a])
            assert np.linalg.norm(Gi[w, a] - G64[w, a]) <= 1e-6 * ref
            assert np.linalg.norm(Gf[w, a] - G64[w, a]) <= 1e-6 * ref


def test_full_size_sampled_row_matches_oracle():
    """Full size in the bench's launch configuration: the medium workload (o=40 v=200 L=800), IP,
    mixed precision, one frequency x the 40 orbitals of the list in one batch.  The G row of one
    sampled orbital (the bench's CPU sample: grid frequency 17, first orbital) against the oracle's
    preconditioned GMRES for that (omega, p) and the oracle's left vectors (about two minutes of CPU)."""
    from oracle.gfcc_ref import gmres
    wl = workload("medium")
    pr = wl.problem()
    om = wl.omegas[17]
    g = gfcc.GFCC(pr, sectors="IP", precision="mixed")
    G, code = g.solve(np.array([om]), wl.eta, wl.orbitals, 1e-10)
    it, rr, st = g.stats()
    g.close()
    assert code == gfcc.OK and np.all(st == 0) and np.all(rr <= 1e-10)
    orc = GFCCOracle(pr.fock, pr.chol, pr.t1, pr.t2, o=wl.o, sectors=("IP",))
    p = int(wl.orbitals[0])
    D = (om - 1j * wl.eta) + orc.ip_diag()
    x, its, rel, ok = gmres(orc.ip_apply(om, wl.eta), orc.ip_rhs(p), 1e-10, 30, 50, diag=D)
    assert ok
    row = np.stack([orc.ip_left(int(q)) for q in wl.orbitals]) @ x
    assert np.linalg.norm(G[0, 0] - row) <= 1e-6 * np.linalg.norm(row)


@pytest.mark.parametrize("krylov", [32, 64])
def test_inner_krylov_precision_does_not_change_the_result(krylov):
    # the inner GMRES of the refinement runs on FP32 (default) or FP64 Krylov vectors; the FP64
    # residual decides convergence either way, so G agrees with the FP64 path to the tolerance
    o, v, L = 10, 50, 100
    pr = make_problem(o, v, L, seed=4)
    om = np.array([-0.9, -0.45])
    orbs = np.array([o - 2, o - 1, o, o + 1], dtype=np.int32)
    g64 = gfcc.GFCC(pr, sectors="IP")
    G64, _ = g64.solve(om, 0.005, orbs, 1e-10)
    g64.close()
    gm = gfcc.GFCC(pr, sectors="IP", precision="mixed")
    gm.set_option(gfcc.OPT_INNER_KRYLOV, krylov)
    Gm, code = gm.solve(om, 0.005, orbs, 1e-10)
    it, rr, st = gm.stats()
    gm.close()
    assert code == gfcc.OK and np.all(st == 0) and np.all(rr <= 1e-10)
    assert rel_err(Gm, G64) <= 1e-7


@pytest.mark.parametrize("batch", [3, 5, 7])
def test_continuous_batching_refills_slots(batch):
    # mixed precision refills a slot as soon as its system converges; task counts that are not a
    # multiple of the batch leave empty slots at the end
    wl = workload("tiny")
    pr = wl.problem()
    orbs = wl.orbitals[:5]
    g = gfcc.GFCC(pr, sectors="IP", precision="mixed")
    g.set_option(gfcc.OPT_BATCH, batch)
    G, code = g.solve(wl.omegas, wl.eta, orbs, 1e-10)
    it, rr, st = g.stats()
    outer = g.refine_stats()
    g.close()
    assert code == gfcc.OK and np.all(st == 0) and np.all(rr <= 1e-10) and np.all(outer >= 2)
    ref = GFCCOracle(pr.fock, pr.chol, pr.t1, pr.t2, o=wl.o, sectors=("IP",)).green_dense(
        wl.omegas, wl.eta, list(orbs), sectors=("IP",))
    assert rel_err(G, ref) <= 1e-6


def test_fp64_batches_with_a_short_last_batch():
    # n_IP = 9114 > 8192, so the G overlaps are summed over two K-split partials; 2 frequencies x 5
    # orbitals = 10 tasks in batches of 4 leave a last batch of 2 systems.  The same G must come out
    # of a single batch of 10.
    o, v, L = 14, 100, 120
    pr = make_problem(o, v, L, seed=12)
    om = np.array([-0.9, -0.5])
    orbs = np.array([o - 3, o - 2, o - 1, o, o + 1], dtype=np.int32)
    out = []
    for batch in (4, 10):
        g = gfcc.GFCC(pr, sectors="IP")
        g.set_option(gfcc.OPT_BATCH, batch)
        G, code = g.solve(om, 0.01, orbs, 1e-10)
        g.close()
        assert code == gfcc.OK
        out.append(G)
    assert rel_err(out[0], out[1]) <= 1e-9


def test_cuda_graph_replay_gives_the_same_result():
    # the Arnoldi steps of the inner solves replayed from CUDA graphs run the same kernels
    o, v, L = 10, 50, 100
    pr = make_problem(o, v, L, seed=6)
    om = np.array([-0.9, -0.45, -0.3])
    orbs = np.array([o - 2, o - 1, o, o + 1], dtype=np.int32)
    out = []
    for graphs in (0, 1):
        g = gfcc.GFCC(pr, sectors="IP", precision="mixed")
        g.set_option(gfcc.OPT_GRAPHS, graphs)
        g.set_option(gfcc.OPT_BATCH, 4)
        l0 = gfcc.launch_count()
        G, code = g.solve(om, 0.005, orbs, 1e-10)
        out.append((G, gfcc.launch_count() - l0))
        g.close()
        assert code == gfcc.OK
    assert rel_err(out[1][0], out[0][0]) <= 1e-12
    # every replayed kernel is counted
    assert abs(out[1][1] - out[0][1]) <= 0.02 * out[0][1]
