"""Brute-force Fock-space definition of the GFCCSD Green's function (test infrastructure).

This is the formula-free statement of the method at tiny sizes: every operator
is a sparse matrix on determinant sectors of a spinless Fock space with n
spin-orbitals, and every GFCCSD quantity is evaluated straight from its
definition.  It is test infrastructure only; nothing in the product imports it.

  * Hamiltonian (Theory section, eq. gfxn0):
        H = sum_pq h_pq p^+ q + 1/4 sum_pqrs <pq||rs> p^+ q^+ s r,
    <pq||rs> = (pr|qs) - (ps|qr), (pr|qs) = sum_K L^K_pr L^K_qs, and
    h_pq = f_pq - sum_j <pj||qj> so that the reference Fock matrix is f.
  * T = sum t_i^a a^+ i + 1/4 sum t_ij^ab a^+ b^+ j i,
    Lambda = sum lambda_a^i i^+ a + 1/4 sum lambda_ab^ij i^+ j^+ b a (eqs. gfxn1, gfxn3).
  * IP space (eq. xp): |i> = a_i|Phi>, |ij^a> = a_a^+ a_j a_i|Phi> (i<j);
    EA space (eq. yq): |a> = a_a^+|Phi>, |i^ab> = a_a^+ a_b^+ a_i|Phi> (a<b).
    Coordinates are the packed amplitudes x_mu = <mu|X|Phi>.
  * The operator of the linear systems (eq. xplin) is taken in commutator form,
    M[mu,nu] = <mu|[Hbar, R_nu]|Phi>, Hbar = e^-T H e^T, which equals
    <mu|(Hbar - E0) R_nu|Phi> whenever T solves the CC equations.
  * b_p(mu) = <mu|e^-T a_p e^T|Phi>, left vector c_q(mu) = <Phi|(1+Lambda) e^-T a_q^+ e^T|mu>,
    G^IP_pq = c_q . X_p with (omega - i eta) X_p + M X_p = b_p (eqs. xplin, gfxn2);
    EA: (omega + i eta) Y_q - M_EA Y_q = e^-T a_q^+ e^T|Phi>, G^EA_pq = <Phi|(1+Lambda) e^-T a_p e^T Y_q|Phi>.
  * Exact Green's function (eq. gfxn0) from the full diagonalisation of H.
"""
from __future__ import annotations

import itertools
import numpy as np
import scipy.sparse as sp
import scipy.linalg as sla


class FockSpace:
    """Sparse second-quantisation operators on fixed-particle-number sectors of n spin-orbitals."""

    def __init__(self, n: int):
        self.n = n
        self._sectors = {}
        self._ops = {}

    def sector(self, N: int):
        """(list of occupation bitmasks, dict mask -> index) for N particles, masks in increasing order."""
        if N not in self._sectors:
            masks = []
            for occ in itertools.combinations(range(self.n), N):
                m = 0
                for p in occ:
                    m |= 1 << p
                masks.append(m)
            masks.sort()
            self._sectors[N] = (masks, {m: k for k, m in enumerate(masks)})
        return self._sectors[N]

    def dim(self, N: int) -> int:
        if N < 0 or N > self.n:
            return 0
        return len(self.sector(N)[0])

    def create(self, p: int, N: int) -> sp.csr_matrix:
        """a_p^+ : sector N -> sector N+1 (Jordan-Wigner sign (-1)^{#occupied q < p})."""
        key = ("c", p, N)
        if key not in self._ops:
            src, _ = self.sector(N)
            _, dst_index = self.sector(N + 1)
            rows, cols, vals = [], [], []
            below = (1 << p) - 1
            for k, m in enumerate(src):
                if m >> p & 1:
                    continue
                sign = -1.0 if bin(m & below).count("1") % 2 else 1.0
                rows.append(dst_index[m | (1 << p)])
                cols.append(k)
                vals.append(sign)
            self._ops[key] = sp.csr_matrix((vals, (rows, cols)), shape=(self.dim(N + 1), self.dim(N)))
        return self._ops[key]

    def annihilate(self, p: int, N: int) -> sp.csr_matrix:
        """a_p : sector N -> sector N-1 (the adjoint of a_p^+ from N-1)."""
        return self.create(p, N - 1).T.tocsr()

    def excitation(self, p: int, q: int, N: int) -> sp.csr_matrix:
        """E_pq = a_p^+ a_q on sector N."""
        key = ("E", p, q, N)
        if key not in self._ops:
            if N == 0:
                self._ops[key] = sp.csr_matrix((1, 1))
            else:
                self._ops[key] = (self.create(p, N - 1) @ self.annihilate(q, N)).tocsr()
        return self._ops[key]

    def excitation_table(self, N: int):
        """Entries of every E_pq on sector N: (rows, cols, signs, p, q) arrays."""
        key = ("table", N)
        if key not in self._ops:
            R, C, S, P, Q = [], [], [], [], []
            for p in range(self.n):
                for q in range(self.n):
                    e = self.excitation(p, q, N).tocoo()
                    R.append(e.row); C.append(e.col); S.append(e.data)
                    P.append(np.full(e.nnz, p)); Q.append(np.full(e.nnz, q))
            self._ops[key] = tuple(np.concatenate(x) for x in (R, C, S, P, Q))
        return self._ops[key]


def core_hamiltonian(fock: np.ndarray, chol: np.ndarray, o: int) -> np.ndarray:
    """h_pq = f_pq - sum_j [(pq|jj) - (pj|jq)], so that the Fock matrix of the reference is f."""
    J = np.einsum("kpq,kjj->pq", chol, chol[:, :o, :o])
    Kx = np.einsum("kpj,kjq->pq", chol[:, :, :o], chol[:, :o, :])
    return fock - J + Kx


def _operator_from(fs: FockSpace, coef: np.ndarray, N: int) -> sp.csr_matrix:
    """sum_pq coef[p][q] E_pq on sector N, assembled from the table of all E_pq entries."""
    rows, cols, signs, pi, qi = fs.excitation_table(N)
    d = fs.dim(N)
    return sp.csr_matrix((signs * coef[pi, qi], (rows, cols)), shape=(d, d))


def hamiltonian(fs: FockSpace, fock, chol, o, N) -> sp.csr_matrix:
    """H on sector N: sum h_pq E_pq + 1/2 sum_K (J_K J_K - sum_ps (L^K L^K)_ps E_ps), J_K = sum L^K_pq E_pq.

    (p^+ q^+ s r = E_pr E_qs - delta_qr E_ps, and 1/4 <pq||rs> p^+ q^+ s r sums to 1/2 (pr|qs) p^+ q^+ s r.)
    """
    h = core_hamiltonian(fock, chol, o)
    one = h - 0.5 * np.einsum("kpr,krs->ps", chol, chol)
    H = _operator_from(fs, one, N)
    for K in range(chol.shape[0]):
        J = _operator_from(fs, chol[K], N)
        H = H + 0.5 * (J @ J)
    return H.tocsr()


def excitation_operator(fs: FockSpace, o, amp1, amp2, N) -> sp.csr_matrix:
    """sum a1[i][a] a^+ i + 1/4 sum a2[i][j][a][b] a^+ b^+ j i on sector N (a^+ b^+ j i = E_ai E_bj)."""
    n = fs.n
    v = n - o
    c1 = np.zeros((n, n))
    c1[o:, :o] = amp1.T
    T = _operator_from(fs, c1, N)
    for i in range(o):
        for a in range(v):
            c2 = np.zeros((n, n))
            c2[o:, :o] = amp2[i, :, a, :].T          # [b][j] = t_ij^ab
            if not np.any(c2):
                continue
            T = T + 0.25 * (fs.excitation(o + a, i, N) @ _operator_from(fs, c2, N))
    return T.tocsr()


def apply_exp(T: sp.csr_matrix, x: np.ndarray, sign: float = 1.0) -> np.ndarray:
    """exp(sign*T) x for nilpotent T (series summed until the term vanishes)."""
    out = x.astype(np.result_type(x, np.float64)).copy()
    term = out.copy()
    k = 1
    while True:
        term = (sign / k) * (T @ term)
        if not np.any(term):
            break
        out = out + term
        k += 1
        if k > 64:
            raise RuntimeError("excitation operator is not nilpotent")
    return out


class BruteForceGFCC:
    """All GFCCSD quantities of one problem from their Fock-space definitions."""

    def __init__(self, fock, chol, t1, t2, lam1, lam2, o):
        self.o = o
        self.n = fock.shape[0]
        self.v = self.n - o
        self.fs = FockSpace(self.n)
        fs = self.fs
        self.N = o
        self.H = {N: hamiltonian(fs, fock, chol, o, N) for N in (o - 1, o, o + 1) if 0 <= N <= self.n}
        self.T = {N: excitation_operator(fs, o, t1, t2, N) for N in self.H}
        self.Ldag = excitation_operator(fs, o, lam1, lam2, o)   # Lambda^+ on the N sector
        masks, index = fs.sector(o)
        self.phi = np.zeros(fs.dim(o))
        self.phi[index[(1 << o) - 1]] = 1.0
        # <Phi|(1+Lambda) as a column vector: (1 + Lambda^+)|Phi>
        self.left_ref = self.phi + self.Ldag @ self.phi
        self.ip_ops = self._ip_operators()
        self.ea_ops = self._ea_operators() if o + 1 <= self.n else []

    # -- operator bases -------------------------------------------------------------------------
    def _ip_operators(self):
        fs, o, v, N = self.fs, self.o, self.v, self.N
        ops = [fs.annihilate(i, N) for i in range(o)]
        for i, j in itertools.combinations(range(o), 2):
            for a in range(v):
                ops.append((fs.create(o + a, N - 2) @ fs.annihilate(j, N - 1) @ fs.annihilate(i, N)).tocsr())
        return ops

    def _ea_operators(self):
        fs, o, v, N = self.fs, self.o, self.v, self.N
        ops = [fs.create(o + a, N) for a in range(v)]
        for i in range(o):
            for a, b in itertools.combinations(range(v), 2):
                ops.append((fs.create(o + a, N) @ fs.create(o + b, N - 1) @ fs.annihilate(i, N)).tocsr())
        return ops

    # -- similarity transform helpers ----------------------------------------------------------
    def hbar_apply(self, Nsec, x):
        """e^-T H e^T x on sector Nsec."""
        T = self.T[Nsec]
        return apply_exp(T, self.H[Nsec] @ apply_exp(T, x, +1.0), -1.0)

    # -- linear-system operators (commutator form) ---------------------------------------------
    def _matrix(self, ops, Ndst):
        N = self.N
        hphi = self.hbar_apply(N, self.phi)
        states = [op @ self.phi for op in ops]
        M = np.zeros((len(ops), len(ops)))
        for nu, op in enumerate(ops):
            col = self.hbar_apply(Ndst, op @ self.phi) - op @ hphi
            M[:, nu] = [s @ col for s in states]
        return M

    def ip_matrix(self):
        """M[mu,nu] = <mu|[Hbar, R_nu]|Phi> over the 1h + 2h1p space."""
        return self._matrix(self.ip_ops, self.N - 1)

    def ea_matrix(self):
        """M_EA[mu,nu] = <mu|[Hbar, Q_nu]|Phi> over the 1p + 2p1h space."""
        return self._matrix(self.ea_ops, self.N + 1)

    # -- right-hand sides and left vectors -----------------------------------------------------
    def _sim_single(self, op, Nsrc, Ndst, x):
        return apply_exp(self.T[Ndst], op @ apply_exp(self.T[Nsrc], x, +1.0), -1.0)

    def ip_rhs(self, p):
        """b_p(mu) = <mu| e^-T a_p e^T |Phi>."""
        N = self.N
        y = self._sim_single(self.fs.annihilate(p, N), N, N - 1, self.phi)
        return np.array([(op @ self.phi) @ y for op in self.ip_ops])

    def ip_left(self, q):
        """c_q(mu) = <Phi|(1+Lambda) e^-T a_q^+ e^T |mu>."""
        N = self.N
        out = []
        for op in self.ip_ops:
            y = self._sim_single(self.fs.create(q, N - 1), N - 1, N, op @ self.phi)
            out.append(self.left_ref @ y)
        return np.array(out)

    def ea_rhs(self, q):
        """b^EA_q(mu) = <mu| e^-T a_q^+ e^T |Phi>."""
        N = self.N
        y = self._sim_single(self.fs.create(q, N), N, N + 1, self.phi)
        return np.array([(op @ self.phi) @ y for op in self.ea_ops])

    def ea_left(self, p):
        """c^EA_p(mu) = <Phi|(1+Lambda) e^-T a_p e^T |mu>."""
        N = self.N
        out = []
        for op in self.ea_ops:
            y = self._sim_single(self.fs.annihilate(p, N + 1), N + 1, N, op @ self.phi)
            out.append(self.left_ref @ y)
        return np.array(out)

    # -- Green's function ----------------------------------------------------------------------
    def green_ip(self, omegas, eta, orbitals):
        """G^IP[w][p][q] = c_q . ((omega - i eta) + M)^-1 b_p  (eqs. xplin, gfxn2)."""
        M = self.ip_matrix()
        B = np.stack([self.ip_rhs(p) for p in orbitals], axis=1)
        C = np.stack([self.ip_left(q) for q in orbitals], axis=1)
        G = np.zeros((len(omegas), len(orbitals), len(orbitals)), dtype=complex)
        I = np.eye(M.shape[0])
        for w, om in enumerate(omegas):
            X = np.linalg.solve((om - 1j * eta) * I + M, B.astype(complex))
            G[w] = (C.T @ X).T
        return G

    def green_ea(self, omegas, eta, orbitals):
        """G^EA[w][p][q] = c^EA_p . ((omega + i eta) - M_EA)^-1 b^EA_q  (eqs. xplin, gfxn2)."""
        M = self.ea_matrix()
        B = np.stack([self.ea_rhs(q) for q in orbitals], axis=1)
        C = np.stack([self.ea_left(p) for p in orbitals], axis=1)
        G = np.zeros((len(omegas), len(orbitals), len(orbitals)), dtype=complex)
        I = np.eye(M.shape[0])
        for w, om in enumerate(omegas):
            Y = np.linalg.solve((om + 1j * eta) * I - M, B.astype(complex))
            G[w] = C.T @ Y
        return G


def exact_green(fock, chol, o, omegas, eta, orbitals, parts=("IP", "EA")):
    """Exact G_pq(omega) of eq. gfxn0 (Lehmann sum) from full diagonalisation of the N-1, N, N+1 sectors.

    parts selects the removal (IP, first term) and addition (EA, second term) contributions."""
    n = fock.shape[0]
    fs = FockSpace(n)
    H = {N: hamiltonian(fs, fock, chol, o, N).toarray() for N in (o - 1, o, o + 1) if 0 <= N <= n}
    e0s, v0s = np.linalg.eigh(H[o])
    E0, psi = e0s[0], v0s[:, 0]
    G = np.zeros((len(omegas), len(orbitals), len(orbitals)), dtype=complex)
    if "IP" in parts and o - 1 >= 0:
        em, vm = np.linalg.eigh(H[o - 1])
        A = np.stack([vm.T @ (fs.annihilate(p, o) @ psi) for p in orbitals])   # <n|a_p|Psi>
        for w, om in enumerate(omegas):
            den = om + (em - E0) - 1j * eta
            G[w] += (A / den) @ A.T.conj()       # sum_n <Psi|a_q^+|n><n|a_p|Psi> / den, index [p][q]
    if "EA" in parts and o + 1 <= n:
        ep, vp = np.linalg.eigh(H[o + 1])
        Bc = np.stack([vp.T @ (fs.create(q, o) @ psi) for q in orbitals])      # <n|a_q^+|Psi>
        for w, om in enumerate(omegas):
            den = om - (ep - E0) + 1j * eta
            G[w] += (Bc.conj() / den) @ Bc.T     # sum_n <Psi|a_p|n><n|a_q^+|Psi> / den, index [p][q]
    return G


def solve_cc_exact(fock, chol, o, tol=1e-13):
    """Full-space CC for N=2 (CCSD is exact there): T from the projected equations, Lambda from the
    left eigenvector of Hbar.  Returns t1, t2, lam1, lam2 (used to pin the definition to eq. gfxn0)."""
    n = fock.shape[0]
    v = n - o
    assert o in (1, 2), "CCSD is the full CC only for one or two electrons"
    fs = FockSpace(n)
    H = hamiltonian(fs, fock, chol, o, o)
    masks, index = fs.sector(o)
    phi = np.zeros(fs.dim(o))
    phi[index[(1 << o) - 1]] = 1.0
    singles = [fs.excitation(o + a, i, o) @ phi for i in range(o) for a in range(v)]
    vpairs = list(itertools.combinations(range(v), 2)) if o == 2 else []
    doubles = [(fs.excitation(o + a, 0, o) @ fs.excitation(o + b, 1, o)) @ phi for a, b in vpairs]
    basis = singles + doubles

    def unpack(x):
        t1 = x[:o * v].reshape(o, v)
        t2 = np.zeros((o, o, v, v))
        for k, (a, b) in enumerate(vpairs):
            val = x[o * v + k]
            t2[0, 1, a, b] = val
            t2[1, 0, a, b] = -val
            t2[0, 1, b, a] = -val
            t2[1, 0, b, a] = val
        return t1, t2

    def residual(x):
        t1, t2 = unpack(x)
        T = excitation_operator(fs, o, t1, t2, o)
        r = apply_exp(T, H @ apply_exp(T, phi, 1.0), -1.0)
        return np.array([s @ r for s in basis])

    x = np.zeros(len(basis))
    for _ in range(100):
        r = residual(x)
        if np.max(np.abs(r)) < tol:
            break
        J = np.zeros((len(basis), len(basis)))
        h = 1e-7
        for k in range(len(basis)):
            dx = np.zeros_like(x)
            dx[k] = h
            J[:, k] = (residual(x + dx) - residual(x - dx)) / (2 * h)
        x = x - np.linalg.solve(J, r)
    else:
        raise RuntimeError("CC did not converge")
    t1, t2 = unpack(x)
    T = excitation_operator(fs, o, t1, t2, o)
    d = fs.dim(o)
    Hbar = np.zeros((d, d))
    for k in range(d):
        e = np.zeros(d)
        e[k] = 1.0
        Hbar[:, k] = apply_exp(T, H @ apply_exp(T, e, 1.0), -1.0)
    E0 = phi @ Hbar @ phi
    w, vl = sla.eig(Hbar, left=True, right=False)
    k = np.argmin(np.abs(w - E0))
    ell = np.real(vl[:, k] / (phi @ vl[:, k]))
    lam1 = np.array([[ell @ singles[i * v + a] for a in range(v)] for i in range(o)])
    lam2 = np.zeros((o, o, v, v))
    for kk, (a, b) in enumerate(vpairs):
        val = ell @ doubles[kk]
        lam2[0, 1, a, b] = val
        lam2[1, 0, a, b] = -val
        lam2[0, 1, b, a] = -val
        lam2[1, 0, b, a] = val
    return t1, t2, lam1, lam2, E0
