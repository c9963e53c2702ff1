"""CPU FP64 reference of the initial guesses and the learned-guess model (test infrastructure:
only tests/, the smoke check and the bench's CPU baseline use this package).

Algorithm 1 of the paper starts every (omega, p) solve from a "computed initial guess".  Here the
guess for a system combines the converged solutions X_k = X_p(omega_k) of the same orbital at K = 8
nearby frequencies,  x0 = sum_k c_k X_k.  Because A(omega) = A(omega_k) + delta_k with
delta_k = omega - omega_k (eq. xplin: the shift enters as omega times the identity, for IP and EA),
and A(omega_k) X_k = b,

    b - A(omega) x0 = (1 - sum_k c_k) b - sum_k c_k delta_k X_k,

so ||b - A x0||^2 = a^H Gm a with a = (sum_k c_k - 1, c_1, ..., c_K) and Gm the Gram matrix of
u_0 = b, u_k = delta_k X_k.  A guess is scored without a sigma product.

The model maps 27 features (omega, eta, p/n, delta_k, Re/Im <b|X_k> eta / ||b||^2) through
x^ = (x - mu)/sd and three weight layers with ReLU to the 16 real parts of c.  Its loss is the
relative residual a^H Gm a / Gm_00; training uses Adam.  Everything here is plain numpy in FP64.
"""
from __future__ import annotations

import numpy as np

K_NEIGHBOURS = 8
N_FEATURES = 3 + 3 * K_NEIGHBOURS
N_OUT = 2 * K_NEIGHBOURS
MINRES_REG = 1e-12          # relative Tikhonov shift of the normal equations of the minimal-residual guess
ADAM_BETA1, ADAM_BETA2, ADAM_EPS = 0.9, 0.999, 1e-8


def features(omega, eta, p_frac, deltas, overlaps, bnorm2):
    """Feature vector of one system; neighbours nearest first."""
    ov = np.asarray(overlaps, dtype=complex) * (eta / bnorm2)
    return np.concatenate([[omega, eta, p_frac], np.asarray(deltas, float), ov.real, ov.imag])


def gram(b, X, deltas):
    """Gm[j][l] = <u_j, u_l> (conjugate-linear in u_j) for u_0 = b, u_k = delta_k X_k."""
    U = np.vstack([np.asarray(b, complex)[None, :], np.asarray(deltas)[:, None] * np.asarray(X, complex)])
    return U.conj() @ U.T


def coefficients(y):
    """c_k = y[2k] + i y[2k+1]."""
    y = np.asarray(y)
    return y[..., 0::2] + 1j * y[..., 1::2]


def residual_vector_coeffs(c):
    """a = (sum c - 1, c_1, ..., c_K)."""
    c = np.asarray(c, complex)
    return np.concatenate([[c.sum() - 1.0], c])


def loss_of_coefficients(c, Gm):
    """||b - A x0||^2 / ||b||^2 for x0 = sum c_k X_k, from the Gram matrix."""
    a = residual_vector_coeffs(c)
    return float(np.real(a.conj() @ Gm @ a) / np.real(Gm[0, 0]))


def loss_from_gram(y, Gm):
    return loss_of_coefficients(coefficients(y), Gm)


def loss_grad_y(y, Gm):
    """d loss / d y (2K reals): 2 Re / Im of (Gm a)_0 + (Gm a)_k, over ||b||^2."""
    a = residual_vector_coeffs(coefficients(y))
    g = Gm @ a / np.real(Gm[0, 0])
    t = g[0] + g[1:]
    out = np.empty(2 * t.size)
    out[0::2] = 2.0 * t.real
    out[1::2] = 2.0 * t.imag
    return out


def minres_coefficients(Gm, navail=None, reg=MINRES_REG):
    """Minimiser of the predicted residual over the first `navail` neighbours: with P = [1^T; I] the
    minimiser of (P c - e0)^H Gm (P c - e0) solves (P^T Gm P + lambda I) c = P^T Gm e0, lambda = reg x
    the largest diagonal entry of P^T Gm P.  Absent neighbours get c = 0."""
    K = Gm.shape[0] - 1
    k = K if navail is None else navail
    c = np.zeros(K, dtype=complex)
    if k == 0:
        return c
    P = np.vstack([np.ones((1, k)), np.eye(k)])
    G = Gm[: k + 1, : k + 1]
    A = P.T @ G @ P
    r = P.T @ G[:, 0]
    lam = reg * np.max(np.real(np.diag(A)))
    c[:k] = np.linalg.solve(A + lam * np.eye(k), r)
    return c


def choose(Gm, navail, mode, y=None):
    """(coefficients, predicted loss, kind) of one system: mode 1 learned (needs all neighbours),
    mode 2 minimal residual; the zero guess (kind 0, loss 1) replaces a guess that is not better."""
    K = Gm.shape[0] - 1
    zero = (np.zeros(K, dtype=complex), 1.0, 0)
    if not np.real(Gm[0, 0]) > 0:
        return zero
    if mode == 1:
        if navail < K:
            return zero
        c = coefficients(y)
    else:
        if navail < 1:
            return zero
        c = minres_coefficients(Gm, navail)
    loss = loss_of_coefficients(c, Gm)
    if not loss < 1.0:
        return zero
    return c, max(loss, 0.0), mode


class MLPRef:
    """x^ = (x - mu)/sd; h1 = relu(W1 x^ + b1); h2 = relu(W2 h1 + b2); y = W3 h2 + b3.
    Flat parameter layout: W1 [h][27], b1, W2 [h][h], b2, W3 [16][h], b3, mu [27], sd [27]."""

    def __init__(self, flat, hidden, nin=N_FEATURES, nout=N_OUT):
        self.h, self.nin, self.nout = hidden, nin, nout
        self.flat = np.array(flat, dtype=np.float64)
        assert self.flat.size == self.num_params(hidden, nin, nout)

    @staticmethod
    def num_params(h, nin=N_FEATURES, nout=N_OUT):
        return h * nin + h + h * h + h + nout * h + nout + 2 * nin

    def unpack(self, flat=None):
        f = self.flat if flat is None else flat
        h, nin, nout = self.h, self.nin, self.nout
        out, o = [], 0
        for shape in ((h, nin), (h,), (h, h), (h,), (nout, h), (nout,), (nin,), (nin,)):
            cnt = int(np.prod(shape))
            out.append(f[o:o + cnt].reshape(shape))
            o += cnt
        return out

    def forward(self, F):
        W1, b1, W2, b2, W3, b3, mu, sd = self.unpack()
        X = (np.atleast_2d(F) - mu) / sd
        z1 = X @ W1.T + b1
        h1 = np.maximum(z1, 0.0)
        z2 = h1 @ W2.T + b2
        h2 = np.maximum(z2, 0.0)
        y = h2 @ W3.T + b3
        return X, z1, h1, z2, h2, y

    def loss(self, F, Gms):
        y = self.forward(F)[-1]
        return float(np.mean([loss_from_gram(y[s], Gms[s]) for s in range(y.shape[0])]))

    def loss_and_grad(self, F, Gms):
        """Mean loss over the batch and its gradient in the flat layout (zero for mu, sd)."""
        X, z1, h1, z2, h2, y = self.forward(F)
        W1, b1, W2, b2, W3, b3, mu, sd = self.unpack()
        B = X.shape[0]
        losses = [loss_from_gram(y[s], Gms[s]) for s in range(B)]
        dy = np.stack([loss_grad_y(y[s], Gms[s]) for s in range(B)]) / B
        dW3 = dy.T @ h2
        db3 = dy.sum(0)
        dz2 = (dy @ W3) * (z2 > 0)
        dW2 = dz2.T @ h1
        db2 = dz2.sum(0)
        dz1 = (dz2 @ W2) * (z1 > 0)
        dW1 = dz1.T @ X
        db1 = dz1.sum(0)
        g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3, np.zeros(2 * self.nin)])
        return float(np.mean(losses)), g


class AdamRef:
    """Adam (Kingma & Ba 2015) on the trained prefix of a flat parameter vector."""

    def __init__(self, ntrain):
        self.m = np.zeros(ntrain)
        self.v = np.zeros(ntrain)
        self.t = 0

    def step(self, flat, grad, lr):
        n = self.m.size
        self.t += 1
        g = grad[:n]
        self.m = ADAM_BETA1 * self.m + (1 - ADAM_BETA1) * g
        self.v = ADAM_BETA2 * self.v + (1 - ADAM_BETA2) * g * g
        mh = self.m / (1 - ADAM_BETA1 ** self.t)
        vh = self.v / (1 - ADAM_BETA2 ** self.t)
        flat = flat.copy()
        flat[:n] -= lr * mh / (np.sqrt(vh) + ADAM_EPS)
        return flat


def frequency_order(omegas):
    """Solve order of a guessed sweep: the two ends, then always the frequency farthest from those
    already taken (ties to the lower index)."""
    om = np.asarray(omegas, float)
    nw = om.size
    if nw == 0:
        return []
    order = [int(np.argmin(om))]
    hi = int(np.argmax(om))
    if hi != order[0]:
        order.append(hi)
    while len(order) < nw:
        d = np.min(np.abs(om[:, None] - om[order][None, :]), axis=1)
        d[order] = -1.0
        order.append(int(np.argmax(d)))
    return order


def neighbours(omegas, done, w, k=K_NEIGHBOURS):
    """The k nearest frequencies to omegas[w] with done[j] set (j != w), nearest first, ties to the
    lower index."""
    om = np.asarray(omegas, float)
    cand = [j for j in range(om.size) if j != w and done[j]]
    cand.sort(key=lambda j: (abs(om[j] - om[w]), j))
    return cand[:k]
