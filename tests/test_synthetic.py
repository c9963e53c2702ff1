"""The synthetic input recipe (the stand-in for the paper's molecules): symmetries, widths and
determinism of the seeded generators (CPU only).  These generators hold none of the method's
arithmetic; both the oracle and the GPU path read their inputs from them."""
import math

import numpy as np
import pytest

from paper_2010_04768_gb300.synthetic import make_problem, normal, uniform, workload


def test_tensors_have_the_symmetries_of_the_method():
    pr = make_problem(5, 9, 20, seed=3)
    assert np.array_equal(pr.chol, pr.chol.transpose(0, 2, 1))              # L^K_pq = L^K_qp
    t2 = pr.t2
    assert np.array_equal(t2, -t2.transpose(1, 0, 2, 3))                     # antisymmetric in (i, j)
    assert np.array_equal(t2, -t2.transpose(0, 1, 3, 2))                     # and in (a, b)
    assert np.all(t2[np.arange(5), np.arange(5)] == 0)
    f = pr.fock
    assert np.array_equal(f, np.diag(np.diag(f)))
    eo, ev = np.diag(f)[:5], np.diag(f)[5:]
    assert np.all(np.diff(eo) >= 0) and np.all(np.diff(ev) >= 0)             # sorted within each space
    assert eo.min() >= -1.5 and eo.max() < -0.3 and ev.min() >= 0.1 and ev.max() < 2.0


def test_widths_follow_the_recipe():
    o, v, L = 10, 30, 24
    pr = make_problem(o, v, L, seed=1)
    assert abs(pr.t1.std() / 0.01 - 1) < 0.1
    iu = np.triu_indices(o, 1)
    au = np.triu_indices(v, 1)
    indep = pr.t2[iu[0], iu[1]][:, au[0], au[1]]                             # the independent elements
    assert abs(indep.std() / 0.02 - 1) < 0.03
    # Cholesky vector K: N(0, sigma^2) exp(-K / 12), sigma = (o v)^(-1/2)
    n = o + v
    ut = np.triu_indices(n)
    sig = 1.0 / math.sqrt(o * v)
    for K in (0, 6, 12):
        s = pr.chol[K][ut].std() / (sig * math.exp(-K / 12.0))
        assert abs(s - 1) < 0.05


def test_generators_are_deterministic_and_streams_independent():
    a, b = make_problem(4, 6, 8, seed=9), make_problem(4, 6, 8, seed=9)
    for x, y in ((a.chol, b.chol), (a.t1, b.t1), (a.t2, b.t2), (a.fock, b.fock)):
        assert np.array_equal(x, y)
    c = make_problem(4, 6, 8, seed=10)
    assert not np.array_equal(a.t2, c.t2)
    assert not np.array_equal(normal(0, 1, 64), normal(0, 2, 64))
    # chunked fills give the same numbers as one long draw (counter-based streams)
    long = uniform(5, 3, 1000)
    assert np.array_equal(long[:10], uniform(5, 3, 10))
    z = normal(5, 4, 20001)
    assert abs(z.mean()) < 0.03 and abs(z.std() - 1) < 0.02


def test_workload_shapes():
    tiny, med, c60 = workload("tiny"), workload("medium"), workload("c60")
    assert (tiny.o, tiny.v, tiny.L, tiny.omegas.size, tiny.orbitals.size) == (4, 12, 48, 4, 16)
    assert (med.o, med.v, med.L, med.omegas.size, med.orbitals.size) == (40, 200, 800, 64, 40)
    assert (c60.o, c60.v, c60.L, c60.omegas.size) == (90, 450, 1800, 128)
    assert np.array_equal(c60.orbitals, np.arange(60, 90))                   # the 30 highest occupied
    assert med.omegas[0] == -1.2 and med.omegas[-1] == 0.5 and med.eta == 0.005
    # medium: the 40 orbitals nearest the mid-gap, from both spaces
    assert med.orbitals.min() < med.o <= med.orbitals.max()


def test_closed_shell_recipe():
    from paper_2010_04768_gb300.synthetic import make_closed_shell_problem
    o, v, L = 6, 20, 30
    a = make_closed_shell_problem(o, v, L, seed=3)
    b = make_closed_shell_problem(o, v, L, seed=3)
    assert np.array_equal(a.t2, b.t2) and np.array_equal(a.chol, b.chol)         # deterministic
    assert np.array_equal(a.t2, a.t2.transpose(1, 0, 3, 2))                       # t_ij^ab = t_ji^ba
    assert np.allclose(a.chol, a.chol.transpose(0, 2, 1))
    # the width of the spin-orbital problem of the same system: (2o 2v)^-1/2 on the leading vector
    assert np.std(a.chol[0]) == pytest.approx((4 * o * v) ** -0.5, rel=0.15)
    # off-diagonal t2 entries have std t2_std / sqrt(2), the (i=j, a=b) ones t2_std
    off = a.t2[0, 1]
    assert np.std(off) == pytest.approx(0.02 / np.sqrt(2), rel=0.15)
    assert np.std(a.t1) == pytest.approx(0.01, rel=0.2)
    c = make_closed_shell_problem(o, v, L, seed=3, separate_lambda=True)
    assert np.array_equal(c.lam2, c.lam2.transpose(1, 0, 3, 2)) and not np.array_equal(c.lam2, c.t2)
