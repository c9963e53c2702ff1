"""The closed-shell spin-adapted IP path (gfcc_create_rhf, rhf.cu) against the CPU oracle
(oracle/rhf_ref.py, pinned to the spin-orbital definition and the exact two-electron G):

* the spin-adapted sigma product element by element (closed form and definition), at shapes that
  span several contraction tiles with ragged edges, T1, T2 and Lambda on;
* G(omega) of the FP64 GMRES path against the oracle at 1e-10, with separate Lambda, preconditioned
  and plain GMRES;
* the same G from the spin-orbital GPU path on the spin-orbital embedding (G_{p alpha, q alpha}): two
  device code paths of different shape that must agree;
* two electrons (one doubly occupied orbital) with the converged CCSD / Lambda amplitudes of the
  device's own ground-state step: the exact Lehmann G;
* the operator with its large contractions on the digit-plane path against the FP64 units and the
  oracle at the medium closed-shell shape, and a sampled G row of that workload (o=30 v=150 L=600,
  digit-plane operator) against the oracle's GMRES.
"""
import numpy as np
import pytest

from paper_2010_04768_gb300 import gfcc
from paper_2010_04768_gb300.synthetic import Problem, make_closed_shell_problem, random_vector, workload
from oracle import fock_space as F
from oracle import gfcc_ref as S
from oracle import rhf_ref as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session", autouse=True)
def _built():
    from paper_2010_04768_gb300 import build
    build.build()
    gfcc.load()


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("o,v,L", [(3, 7, 9), (7, 23, 30)])
def test_sigma_matches_oracle(o, v, L):
    pr = make_closed_shell_problem(o, v, L, seed=o + v, t1_std=0.05, t2_std=0.05, separate_lambda=True)
    g = gfcc.GFCC(pr, sectors="IP", closed_shell=True)
    di, _ = g.dims()
    assert di == R.ip_dim(o, v)
    C = R.RHFClosed(pr.fock, pr.chol, pr.t1, pr.t2, pr.lam1, pr.lam2, o=o)
    X = np.stack([random_vector(3 + k, di) + 1j * random_vector(13 + k, di) for k in range(3)])
    Y = g.sigma("IP", X)
    g.close()
    ref = np.stack([C.sigma(x.real) + 1j * C.sigma(x.imag) for x in X])
    assert rel(Y, ref) <= 1e-12
    if o == 3:
        D = R.RHFIP(pr.fock, pr.chol, pr.t1, pr.t2, pr.lam1, pr.lam2, o=o)
        assert rel(Y[0], D.sigma(X[0].real) + 1j * D.sigma(X[0].imag)) <= 1e-12


@pytest.mark.parametrize("precond", [True, False])
def test_green_function_matches_oracle(precond):
    o, v, L = 4, 11, 14
    pr = make_closed_shell_problem(o, v, L, seed=5, t1_std=0.05, t2_std=0.05, separate_lambda=True)
    g = gfcc.GFCC(pr, sectors="IP", closed_shell=True)
    g.set_option(gfcc.OPT_RESTART, 64)
    g.set_option(gfcc.OPT_PRECOND, gfcc.PRECOND_DIAG if precond else gfcc.PRECOND_NONE)
    om = np.array([-1.3, -0.8, -0.45])
    orbs = np.array([0, o - 2, o - 1, o, o + 3], dtype=np.int32)
    G, code = g.solve(om, 0.02, orbs, 1e-13)
    it, rr, st = g.stats()
    g.close()
    assert code == gfcc.OK and np.all(st == 0)
    D = R.RHFIP(pr.fock, pr.chol, pr.t1, pr.t2, pr.lam1, pr.lam2, o=o)
    assert rel(G, D.green_dense(om, 0.02, list(orbs))) <= 1e-10


def test_matches_spin_orbital_path_on_the_embedding():
    o, v, L = 3, 8, 10
    pr = make_closed_shell_problem(o, v, L, seed=8, t1_std=0.05, t2_std=0.05, separate_lambda=True)
    om = np.array([-1.1, -0.6])
    orbs = np.arange(o + v, dtype=np.int32)
    g = gfcc.GFCC(pr, sectors="IP", closed_shell=True)
    g.set_option(gfcc.OPT_RESTART, 64)
    G, code = g.solve(om, 0.02, orbs, 1e-13)
    g.close()
    assert code == gfcc.OK
    Fs, Ls = R.embed_problem(pr.fock, pr.chol, o)
    T1, T2 = R.embed_amplitudes(pr.t1, pr.t2, o, v)
    L1, L2 = R.embed_amplitudes(pr.lam1, pr.lam2, o, v)
    so = gfcc.GFCC(Problem(o=2 * o, v=2 * v, L=L, fock=Fs, chol=Ls, t1=T1, t2=T2, lam1=L1, lam2=L2), sectors="IP")
    so.set_option(gfcc.OPT_RESTART, 64)
    al, _ = R.so_index(o, v)
    Gso, code2 = so.solve(om, 0.02, al.astype(np.int32), 1e-13)
    so.close()
    assert code2 == gfcc.OK
    assert rel(G, Gso) <= 1e-10


def test_two_electrons_from_the_device_ground_state_is_exact():
    o, v, L = 1, 5, 6
    pr = make_closed_shell_problem(o, v, L, seed=9, chol_sigma=0.3)
    Fs, Ls = R.embed_problem(pr.fock, pr.chol, o)
    T1, T2, L1, L2, info, code = gfcc.ccsd(Fs, Ls, 2 * o, tol=1e-13, max_iter=300)
    assert code == gfcc.OK
    cs = Problem(o=o, v=v, L=L, fock=pr.fock, chol=pr.chol, t1=T1[:o, :v].copy(), t2=T2[:o, o:, :v, v:].copy(),
                 lam1=L1[:o, :v].copy(), lam2=L2[:o, o:, :v, v:].copy())
    g = gfcc.GFCC(cs, sectors="IP", closed_shell=True)
    g.set_option(gfcc.OPT_RESTART, 64)
    om = np.array([-1.3, -0.6, 0.3])
    orbs = np.arange(o + v, dtype=np.int32)
    G, code = g.solve(om, 0.05, orbs, 1e-13)
    g.close()
    assert code == gfcc.OK
    al, _ = R.so_index(o, v)
    Gx = F.exact_green(Fs, Ls, 2 * o, om, 0.05, [int(a) for a in al], parts=("IP",))
    assert rel(G, Gx) <= 1e-9


def test_digit_plane_operator_matches_fp64_operator_and_oracle():
    # medium closed-shell shape: the ring sums and the oooo term (above 1e9 flops) from digit planes
    wl = workload("medium-closed-shell")
    pr = wl.problem()
    g = gfcc.GFCC(pr, sectors="IP", closed_shell=True)
    di, _ = g.dims()
    X = np.stack([random_vector(21 + k, di) + 1j * random_vector(41 + k, di) for k in range(4)])
    Ye = g.sigma("IP", X)
    g.set_option(gfcc.OPT_CLOSED_SHELL_EMULATE, 0)
    Yf = g.sigma("IP", X)
    g.close()
    # a level-9 product of 8 base-64 digits carries an error below 2^-50 of the row scale per term,
    # so at most K 2^-50 over a contraction of length K (the ring sums: K = o v)
    bound = wl.o * wl.v * 2.0 ** -50
    assert rel(Ye, Yf) <= bound
    C = R.RHFClosed(pr.fock, pr.chol, pr.t1, pr.t2, o=wl.o)
    assert rel(Ye[0], C.sigma(X[0])) <= bound
    assert rel(Yf[0], C.sigma(X[0])) <= 1e-12


def test_medium_closed_shell_row_matches_oracle():
    """The FP64 path (every contraction on the FP64 units) at 1e-10 against the oracle; the digit-plane
    operator (the default) at tol 1e-10 against it at 1e-8 (its products carry up to ~4e-12 relative
    error, which sets the floor of its GMRES residual)."""
    wl = workload("medium-closed-shell")
    pr = wl.problem()
    g = gfcc.GFCC(pr, sectors="IP", closed_shell=True)
    om = wl.omegas[40:41]
    Ge, code_e = g.solve(om, wl.eta, wl.orbitals, 1e-10)
    st_e = g.stats()[2]
    g.set_option(gfcc.OPT_CLOSED_SHELL_EMULATE, 0)
    G, code = g.solve(om, wl.eta, wl.orbitals, 1e-12)
    it, rr, st = g.stats()
    g.close()
    assert code == gfcc.OK and np.all(st == 0)
    assert code_e == gfcc.OK and np.all(st_e == 0)
    C = R.RHFClosed(pr.fock, pr.chol, pr.t1, pr.t2, o=wl.o)
    row = wl.orbitals.size - 1          # the highest occupied orbital: its system by the oracle's GMRES,
    z = om[0] - 1j * wl.eta             # overlapped with every column's left vector
    x, _, _, ok = S.gmres(lambda y: z * y + C.sigma(y), C.rhs(int(wl.orbitals[row])), 1e-13, 30, 60,
                          diag=z + C.diag())
    assert ok
    ref_row = np.stack([C.left(int(q)) for q in wl.orbitals]) @ x
    assert np.linalg.norm(G[0, row] - ref_row) <= 1e-10 * np.linalg.norm(ref_row)
    for a in range(wl.orbitals.size):
        assert np.linalg.norm(Ge[0, a] - G[0, a]) <= 1e-8 * np.linalg.norm(G[0, a])


def test_closed_shell_arguments_are_rejected():
    o, v = 2, 4
    pr = make_closed_shell_problem(o, v, 3, seed=1)
    bad = Problem(o=o, v=v, L=3, fock=pr.fock, chol=pr.chol, t1=pr.t1,
                  t2=pr.t2 + 0.1 * np.arange(pr.t2.size).reshape(pr.t2.shape) / pr.t2.size)
    with pytest.raises(gfcc.GFCCError):
        gfcc.GFCC(bad, sectors="IP", closed_shell=True)      # t2 without t_ij^ab = t_ji^ba
    g = gfcc.GFCC(pr, sectors="IP", closed_shell=True)
    with pytest.raises(gfcc.GFCCError):
        g.set_option(gfcc.OPT_GUESS, gfcc.GUESS_MINRES)
    g.close()
