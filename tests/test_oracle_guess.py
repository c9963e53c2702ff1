"""Pins of the initial-guess oracle (oracle/mlp_ref.py) against what the mathematics fixes (CPU).

* the Gram-matrix residual equals the residual of the combined guess computed with the dense
  operator of eq. xplin (IP and EA), i.e. the identity A(omega) X_k = b + delta_k X_k;
* the minimal-residual coefficients equal an independent least-squares solve on the explicit
  vectors;
* the analytic gradients (of the loss in the outputs, and of the model in its parameters) equal
  central finite differences;
* the first Adam step has the closed form -lr g / (|g| + eps);
* the frequency order of a guessed sweep on a uniform grid is bisection order.
"""
import numpy as np
import pytest

from oracle import mlp_ref as M
from oracle.gfcc_ref import GFCCOracle
from paper_2010_04768_gb300.synthetic import make_problem, mlp_init_params


@pytest.fixture(scope="module")
def small():
    o, v = 3, 7
    P = make_problem(o, v, 10, seed=11)
    orc = GFCCOracle(P.fock, P.chol, P.t1, P.t2, o=o)
    return P, orc, orc.ip_matrix(), orc.ea_matrix()


def _solutions(A_of, b, omegas):
    return np.stack([np.linalg.solve(A_of(w), b) for w in omegas])


@pytest.mark.parametrize("sector", ["IP", "EA"])
def test_gram_residual_equals_dense_residual(small, sector):
    P, orc, Mip, Mea = small
    eta = 0.01
    rng = np.random.default_rng(5)
    if sector == "IP":
        n = Mip.shape[0]
        A_of = lambda w: (w - 1j * eta) * np.eye(n) + Mip
        b = orc.ip_rhs(P.o + 1)
    else:
        n = Mea.shape[0]
        A_of = lambda w: (w + 1j * eta) * np.eye(n) - Mea
        b = orc.ea_rhs(P.o - 1)
    om_k = np.linspace(-0.9, 0.6, 8)
    X = _solutions(A_of, b, om_k)
    omega = 0.137
    d = omega - om_k
    Gm = M.gram(b, X, d)
    for _ in range(4):
        c = rng.normal(size=8) + 1j * rng.normal(size=8)
        c *= 0.3
        x0 = c @ X
        direct = np.linalg.norm(b - A_of(omega) @ x0) ** 2 / np.linalg.norm(b) ** 2
        assert M.loss_of_coefficients(c, Gm) == pytest.approx(direct, rel=1e-9)
    # zero coefficients give the zero guess (loss 1); Gm is Hermitian positive semidefinite
    assert M.loss_of_coefficients(np.zeros(8), Gm) == pytest.approx(1.0, rel=1e-14)
    assert np.allclose(Gm, Gm.conj().T)
    assert np.min(np.linalg.eigvalsh(Gm)) > -1e-12 * np.max(np.abs(Gm))


def test_minres_equals_least_squares_on_explicit_vectors(small):
    P, orc, Mip, _ = small
    eta = 0.01
    n = Mip.shape[0]
    A_of = lambda w: (w - 1j * eta) * np.eye(n) + Mip
    b = orc.ip_rhs(1)
    om_k = np.array([-0.7, -0.55, -0.4, -0.2, 0.1, 0.3, 0.45, 0.6])
    X = _solutions(A_of, b, om_k)
    omega = -0.31
    d = omega - om_k
    Gm = M.gram(b, X, d)
    for k in (1, 3, 8):
        c = M.minres_coefficients(Gm, k, reg=0.0)
        # r(c) = b - sum_k c_k (b + delta_k X_k): least squares over the columns w_k = b + delta_k X_k
        W = (b[:, None] + d[None, :k] * X[:k].T)
        c_ls, *_ = np.linalg.lstsq(W, b, rcond=None)
        r_ls = np.linalg.norm(b - W @ c_ls) ** 2 / np.linalg.norm(b) ** 2
        assert M.loss_of_coefficients(c, Gm) == pytest.approx(r_ls, rel=1e-6, abs=1e-14)
        # and the true residual of the guess agrees
        x0 = c[:k] @ X[:k]
        true = np.linalg.norm(b - A_of(omega) @ x0) ** 2 / np.linalg.norm(b) ** 2
        assert true == pytest.approx(r_ls, rel=1e-6, abs=1e-14)
    # more neighbours never increase the minimal residual
    losses = [M.loss_of_coefficients(M.minres_coefficients(Gm, k, reg=0.0), Gm) for k in range(1, 9)]
    assert all(losses[i + 1] <= losses[i] * (1 + 1e-9) + 1e-15 for i in range(7))


def test_choose_falls_back_to_zero():
    Gm = np.eye(9, dtype=complex)
    # with orthonormal u_k any nonzero c raises the residual above ||b||: the zero guess is kept
    c, loss, kind = M.choose(Gm, 8, 1, y=np.full(16, 0.3))
    assert kind == 0 and loss == 1.0 and not np.any(c)
    c, loss, kind = M.choose(Gm, 3, 1, y=np.zeros(16))
    assert kind == 0
    c, loss, kind = M.choose(Gm, 0, 2)
    assert kind == 0


def test_loss_gradient_in_outputs_matches_finite_differences():
    rng = np.random.default_rng(1)
    U = rng.normal(size=(9, 40)) + 1j * rng.normal(size=(9, 40))
    Gm = U.conj() @ U.T
    y = 0.2 * rng.normal(size=16)
    g = M.loss_grad_y(y, Gm)
    h = 1e-6
    fd = np.array([(M.loss_from_gram(y + h * e, Gm) - M.loss_from_gram(y - h * e, Gm)) / (2 * h) for e in np.eye(16)])
    assert np.max(np.abs(g - fd)) <= 1e-7 * np.max(np.abs(g))


def test_model_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    hidden = 12
    flat = mlp_init_params(hidden, seed=3)
    nparam = M.MLPRef.num_params(hidden)
    assert flat.size == nparam
    flat[nparam - 54:nparam - 27] = rng.normal(size=27) * 0.1      # mu
    flat[nparam - 27:] = 0.5 + rng.uniform(size=27)                 # sd
    net = M.MLPRef(flat, hidden)
    B = 5
    F = rng.normal(size=(B, 27))
    Gms = []
    for _ in range(B):
        U = rng.normal(size=(9, 30)) + 1j * rng.normal(size=(9, 30))
        Gms.append(U.conj() @ U.T)
    loss, g = net.loss_and_grad(F, Gms)
    assert loss == pytest.approx(net.loss(F, Gms), rel=1e-14)
    assert np.all(g[nparam - 54:] == 0.0)
    h = 1e-6
    idx = rng.choice(nparam - 54, size=40, replace=False)
    for i in idx:
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        fd = (M.MLPRef(fp, hidden).loss(F, Gms) - M.MLPRef(fm, hidden).loss(F, Gms)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-8 * np.max(np.abs(g)))


def test_first_adam_step_closed_form():
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    flat = np.array([1.0, 2.0, 3.0, 4.0, 9.0])          # last entry untrained
    opt = M.AdamRef(4)
    out = opt.step(flat, np.concatenate([g, [7.0]]), lr=0.01)
    expect = flat[:4] - 0.01 * g / (np.abs(g) + M.ADAM_EPS)
    assert np.allclose(out[:4], expect, rtol=0, atol=1e-15)
    assert out[4] == 9.0


def test_frequency_order_is_bisection_on_a_uniform_grid():
    assert M.frequency_order(np.linspace(0.0, 1.0, 9)) == [0, 8, 4, 2, 6, 1, 3, 5, 7]
    assert M.frequency_order([0.3]) == [0]
    assert M.frequency_order([]) == []
    om = np.array([-0.5, -0.25, 0.0, 0.25, 0.5])          # exact binary distances: real ties
    assert M.neighbours(om, [1, 1, 1, 1, 1], 2, k=3) == [1, 3, 0]
    assert M.neighbours(om, [1, 0, 1, 1, 1], 2, k=3) == [3, 0, 4]
    assert M.neighbours(om, [0, 0, 1, 0, 0], 2, k=3) == []
