"""CPU FP64 reference of the model-order reduction (MOR) of the GFCCSD linear systems, the adaptive
frequency levels and the spectral function (test infrastructure: only tests/, the smoke check and the
bench's CPU legs use this module; the product never imports it).

Model-order reduction (Theory section, eq. model; Algorithm 1, the Gram-Schmidt, projection and
spectral-function steps after the frequency loop of a level).  From solutions X_p(omega_k) of the
full systems of eq. xplin an orthonormal subspace S = {v_1 .. v_m} is built by Gram-Schmidt, the
operator is projected, Hhat = S^T Hbar_N S, and the model systems
    IP: (omega - i eta + Hhat) Xhat = bhat,   Ghat^IP_pq = chat_q^T Xhat_p,
    EA: (omega + i eta - Hhat) Yhat = bhat,   Ghat^EA_pq = chat_p^T Yhat_q,
with bhat = S^T b and chat = S^T c are solved densely over any frequency grid.

Reading of S^T: Hbar, b and c are real, so S is taken real, spanned by the real and imaginary parts
of the complex solutions; its complex span contains every X_p(omega_k), so the model reproduces the
full solution at every sampled frequency (Galerkin interpolation), and Hhat is a real m x m matrix.

Gram-Schmidt: each new real vector is orthogonalised twice against the basis (classical passes;
"twice is enough"), and kept when the norm that remains is above drop_tol times its norm before
(otherwise it is linearly dependent on the basis to that tolerance and is dropped).

Model residual: with W = Hbar_N S (the sigma products of the basis vectors, needed for Hhat anyway),
the full-space residual of the model solution is b - A(omega) S Xhat = b - (omega -/+ i eta) S Xhat
(+/-) W Xhat (IP: -, EA: +), evaluated without a sigma product.

Adaptive levels (Implementation Details, eq. Lmax and its worked example): level 1 samples
omega_min, the midpoint and omega_max (N_max(1) = 3); level L > 1 samples midpoints of adjacent
sampled frequencies, at most 2^(L-1) of them (N_max(L) = 2^(L-1)); midpoints closer than the
resolution d_omega to a neighbour are not sampled, which bounds the number of levels by
log2((omega_max - omega_min) / d_omega).  Reading of the selection (the cited adaptive midpoint
refinement is not spelled out): a midpoint is sampled when the largest relative model residual over
the orbitals there exceeds the level tolerance; the driver stops when no midpoint does.

Spectral function (eq. specfxn): A = -(1/pi) Tr Im G^R.  Reading of the sign: with the paper's
-i eta in the IP resolvent and +i eta in the EA resolvent, Im G^IP_pp > 0 and Im G^EA_pp < 0 near
their poles; the function computed here is A(omega) = (1/pi) sum_p (Im G^IP_pp - Im G^EA_pp), a sum
of positive Lorentzians, i.e. -(1/pi) Tr Im of the retarded function in the usual +i eta convention.
"""
from __future__ import annotations

import math

import numpy as np


# ------------------------------------------------------------------------------------- subspace
def orthonormal_extend(S: np.ndarray | None, vectors, drop_tol: float = 1e-10) -> np.ndarray:
    """S (n x m, orthonormal columns, or None) extended by the real vectors given (each a length-n
    array), one at a time: two classical Gram-Schmidt passes against the current basis, kept when
    ||v'|| > drop_tol ||v||, then normalised."""
    cols = [] if S is None else [S[:, k] for k in range(S.shape[1])]
    for v in vectors:
        v = np.asarray(v, dtype=np.float64).copy()
        nv = np.linalg.norm(v)
        if nv == 0.0:
            continue
        for _ in range(2):
            if cols:
                B = np.stack(cols, axis=1)
                v -= B @ (B.T @ v)
        nr = np.linalg.norm(v)
        if nr > drop_tol * nv:
            cols.append(v / nr)
    n = len(vectors[0]) if S is None else S.shape[0]
    return np.stack(cols, axis=1) if cols else np.zeros((n, 0))


def real_parts(X) -> list:
    """The real vectors of a list of complex solutions: Re x_k, Im x_k for each (in that order)."""
    out = []
    for x in X:
        out.append(np.real(x).copy())
        out.append(np.imag(x).copy())
    return out


# ------------------------------------------------------------------------------------- projection
def project(sigma, S: np.ndarray):
    """(Hhat, W): W = sigma(S) column by column (sigma = the oracle's Hbar_N product, eq. xplin
    without the shift), Hhat = S^T W."""
    W = np.stack([np.real(sigma(S[:, k].astype(complex))) for k in range(S.shape[1])], axis=1)
    return S.T @ W, W


# ------------------------------------------------------------------------------------- model solves
def model_green(Hhat, S, B, C, omegas, eta, sector: str):
    """G[w][a][b] of eq. model over the frequencies: IP rows a over the right-hand sides B[:, a]
    (b_p), columns b over the left vectors C[:, b] (c_q); EA: columns b over the right-hand sides
    (b_q), rows a over the left vectors (c_p)."""
    m = Hhat.shape[0]
    bh = S.T @ B
    ch = S.T @ C
    G = np.zeros((len(omegas), C.shape[1] if sector == "EA" else B.shape[1],
                  B.shape[1] if sector == "EA" else C.shape[1]), dtype=complex)
    for w, om in enumerate(omegas):
        if sector == "IP":
            Xh = np.linalg.solve((om - 1j * eta) * np.eye(m) + Hhat, bh.astype(complex))
            G[w] = (ch.T @ Xh).T
        else:
            Yh = np.linalg.solve((om + 1j * eta) * np.eye(m) - Hhat, bh.astype(complex))
            G[w] = ch.T @ Yh
    return G


def model_solution(Hhat, S, b, omega, eta, sector: str):
    """Xhat (IP) or Yhat (EA) of one model system."""
    m = Hhat.shape[0]
    z = (omega - 1j * eta) if sector == "IP" else (omega + 1j * eta)
    Mz = z * np.eye(m) + (Hhat if sector == "IP" else -Hhat)
    return np.linalg.solve(Mz, (S.T @ b).astype(complex))


def model_relres(Hhat, S, W, b, omega, eta, sector: str) -> float:
    """||b - A(omega) S Xhat|| / ||b|| of the model solution, from W = Hbar_N S (no sigma product)."""
    xh = model_solution(Hhat, S, b, omega, eta, sector)
    z = (omega - 1j * eta) if sector == "IP" else (omega + 1j * eta)
    Ax = z * (S @ xh) + (W @ xh if sector == "IP" else -(W @ xh))
    return float(np.linalg.norm(b - Ax) / np.linalg.norm(b))


# ------------------------------------------------------------------------------------- spectral function
def spectral_function(G_ip_diag, G_ea_diag=None):
    """A(omega) = (1/pi) sum_p (Im G^IP_pp - Im G^EA_pp); arguments [n_omega][n_orb] diagonals."""
    A = np.sum(np.imag(G_ip_diag), axis=1) / math.pi
    if G_ea_diag is not None:
        A -= np.sum(np.imag(G_ea_diag), axis=1) / math.pi
    return A


# ------------------------------------------------------------------------------------- levels
def n_max(level: int) -> int:
    """Largest number of frequencies sampled at a level: 3 at level 1, 2^(L-1) after."""
    return 3 if level == 1 else 2 ** (level - 1)


def l_max_bound(omega_min: float, omega_max: float, d_omega: float) -> int:
    """Upper bound of the number of levels, floor(log2((omega_max - omega_min) / d_omega))."""
    return int(math.floor(math.log2((omega_max - omega_min) / d_omega) + 1e-12))


def midpoints(sampled, d_omega: float):
    """Midpoints of adjacent sampled frequencies (sorted) whose half-interval is at least d_omega."""
    s = np.sort(np.asarray(sampled, dtype=np.float64))
    out = []
    for a, b in zip(s[:-1], s[1:]):
        if (b - a) / 2 >= d_omega * (1 - 1e-12):
            out.append(0.5 * (a + b))
    return out


def adaptive_levels(indicator, omega_min, omega_max, d_omega, tol, max_levels=64):
    """The frequencies of each level of the adaptive driver.  indicator(omega, sampled) is the error
    estimate at a candidate midpoint given the frequencies sampled so far (the model of those).
    Returns the list of levels (each a sorted list of frequencies)."""
    levels = [[omega_min, 0.5 * (omega_min + omega_max), omega_max]]
    sampled = list(levels[0])
    for L in range(2, max_levels + 1):
        cand = midpoints(sampled, d_omega)
        err = [(indicator(w, sampled), w) for w in cand]
        pick = sorted(w for e, w in err if e > tol)
        if len(pick) > n_max(L):
            pick = sorted(w for e, w in sorted(err, key=lambda t: -t[0])[:n_max(L)])
        if not pick:
            break
        levels.append(pick)
        sampled += pick
    return levels
