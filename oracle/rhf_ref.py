"""CPU FP64 reference of the closed-shell spin-adapted GFCCSD-IP (test infrastructure: only tests/, the
smoke check and the bench's CPU legs use this module; the product never imports it).

The paper's production IP code for closed shells keeps only the alpha amplitudes (Table 2: the
closed-shell GFCCSD-IP deals with the alpha electrons only).  For a closed-shell reference the
spin-orbital system is two copies of the spatial orbitals, the Hamiltonian is spin free and T,
Lambda are spin adapted; removing an alpha electron from spatial orbital p keeps every Krylov vector
in the doublet subspace spanned by
    r_i     = R_{i alpha}                       (1h)
    r_ij^a  = R_{i alpha, j beta}^{a beta}      (2h1p, all i, j, a; no antisymmetry),
with R_{i alpha, j alpha}^{a alpha} = r_ij^a - r_ji^a and R_{i beta, j alpha}^{a beta} = -r_ji^a.

Definition (this module's RHFIP): the spin-orbital GFCCSD-IP of gfcc_ref (itself pinned to the
Fock-space definition) applied to the spin-orbital embedding of the closed-shell problem, read in
those coordinates: sigma(x) = P sigma_so(E x), b_p = P b_so(p alpha), and the left vector of q is
E^T c_so(q alpha), so that G_pq = left_q . X_p equals the spin-orbital G_{p alpha, q alpha} (E the
embedding, P the projection on the coordinates above).

Closed form (RHFClosed): the same quantities from spatial integrals, derived by summing the
spin-orbital IP-EOM-CCSD equations over the spins of a closed-shell reference (u_mnef = (me|nf)',
(pq|rs)' = sum_K L'^K_pq L'^K_rs with the T1-rotated Cholesky vectors):
  Fbar_mi = f'_mi + (2 u_mnef - u_mnfe) t_in^ef,   Fbar_ae = f'_ae - (2 u_mnef - u_mnfe) t_mn^af,
  Fbar_me = f'_me,  W_mnij = (mi|nj)' + u_mnef t_ij^ef,  W_mnie = (mi|ne)',
  W_maij = (mi|aj)' + Fbar_me t_ij^ea + (me|af)' t_ij^ef + (2 (mi|ne)' - (me|ni)') t_jn^ae
           - (mi|ne)' t_jn^ea - (me|nj)' t_in^ea,
  X_maei = (me|ai)' + (2 u_mnef - u_mnfe) t_in^af - u_mnef t_in^fa      (ovvo, alpha-beta-alpha-beta)
  Y_maie = (mi|ae)' - u_mnfe t_in^fa                                     (ovov, alpha-beta-alpha-beta)
  sigma_i   = -Fbar_mi r_m + Fbar_me (2 r_im^e - r_mi^e) + (W_nmie - 2 W_mnie) r_mn^e
  sigma_ija = -W_maij r_m + Fbar_ae r_ij^e - Fbar_mi r_mj^a - Fbar_mj r_im^a + W_mnij r_mn^a
              - Y_maie r_mj^e + (2 X_maej - Y_maje) r_im^e - X_maej r_mi^e - z_e t_ij^ea,
  z_e = (2 u_mnef - u_mnfe) r_mn^f;
  b_p: p = m occupied: r_i = delta_im;  p = b virtual: r_i = t_i^b, r_ij^a = t_ij^ba;
  left_q: q = b virtual: l_i = lambda_i^b, l_ij^a = 2 lambda_ij^ba - lambda_ij^ab;
          q = m occupied: l_i = delta_mi - t_m^c lambda_i^c - (2 t_ml^cd - t_ml^dc) lambda_il^cd,
          l_ij^a = 2 delta_im lambda_j^a - delta_jm lambda_i^a - 2 t_m^c lambda_ij^ca + t_m^c lambda_ij^ac.
Spatial amplitudes: t_i^a = T_{i alpha}^{a alpha}, t_ij^ab = T_{i alpha, j beta}^{a alpha, b beta}
(t_ij^ab = t_ji^ba), Lambda likewise.  Every closed-form quantity is pinned to the definition
(tests/test_oracle_rhf.py).
"""
from __future__ import annotations

import numpy as np

from oracle import gfcc_ref as S


# ---------------------------------------------------------------------------------------------- embedding
def so_index(o: int, v: int):
    """Spin-orbital indices of the spatial orbitals: (alpha, beta) arrays over p = 0..o+v-1 in the
    spin-orbital order [occ alpha | occ beta | vir alpha | vir beta]."""
    p = np.arange(o + v)
    alpha = np.where(p < o, p, 2 * o + (p - o))
    beta = np.where(p < o, o + p, 2 * o + v + (p - o))
    return alpha, beta


def embed_amplitudes(a1, a2, o, v):
    """Spin-orbital T1 [2o][2v], T2 [2o][2o][2v][2v] of spatial t1 [o][v], t2 [o][o][v][v]:
    T_{IJ}^{AB} = d(sI, sA) d(sJ, sB) t_ij^ab - d(sI, sB) d(sJ, sA) t_ij^ba."""
    O, V = 2 * o, 2 * v
    so = np.repeat([0, 1], o)          # spin of occupied spin-orbital I
    sv = np.repeat([0, 1], v)
    io, iv = np.tile(np.arange(o), 2), np.tile(np.arange(v), 2)
    T1 = (so[:, None] == sv[None, :]) * a1[io][:, iv]
    t = a2[io][:, io][:, :, iv][:, :, :, iv]                       # t[I,J,A,B] = t_ij^ab
    tx = np.swapaxes(t, 2, 3)                                       # t_ij^ba
    d1 = (so[:, None, None, None] == sv[None, None, :, None]) & (so[None, :, None, None] == sv[None, None, None, :])
    d2 = (so[:, None, None, None] == sv[None, None, None, :]) & (so[None, :, None, None] == sv[None, None, :, None])
    T2 = d1 * t - d2 * tx
    assert T1.shape == (O, V) and T2.shape == (O, O, V, V)
    return T1, T2


def embed_problem(fock, chol, o):
    """Spin-orbital (fock, chol) of a closed-shell spatial problem (spin-free, block diagonal in spin)."""
    n = fock.shape[0]
    v = n - o
    al, be = so_index(o, v)
    N = 2 * n
    F = np.zeros((N, N))
    F[np.ix_(al, al)] = fock
    F[np.ix_(be, be)] = fock
    Lso = np.zeros((chol.shape[0], N, N))
    Lso[:, al[:, None], al[None, :]] = chol
    Lso[:, be[:, None], be[None, :]] = chol
    return F, Lso


def ip_dim(o, v):
    return o + o * o * v


def split(x, o, v):
    return x[:o], x[o:].reshape(o, o, v)


class RHFIP:
    """Definition: spin-orbital GFCCSD-IP of the embedding, in the spin-adapted coordinates."""

    def __init__(self, fock, chol, t1, t2, lam1=None, lam2=None, o=None):
        o = t1.shape[0] if o is None else o
        self.o, self.v = o, fock.shape[0] - o
        lam1 = t1 if lam1 is None else lam1
        lam2 = t2 if lam2 is None else lam2
        F, L = embed_problem(fock, chol, o)
        T1, T2 = embed_amplitudes(t1, t2, o, self.v)
        L1, L2 = embed_amplitudes(lam1, lam2, o, self.v)
        self.so = S.GFCCOracle(F, L, T1, T2, L1, L2, o=2 * o, sectors=("IP",))
        self.alpha, _ = so_index(o, self.v)

    def dim(self):
        return ip_dim(self.o, self.v)

    def embed(self, x):
        """spin-adapted coordinates -> packed spin-orbital IP vector"""
        o, v = self.o, self.v
        r1, r2 = split(x, o, v)
        R1 = np.zeros(2 * o, dtype=x.dtype)
        R1[:o] = r1
        R2 = np.zeros((2 * o, 2 * o, 2 * v), dtype=x.dtype)
        R2[:o, o:, v:] = r2                                   # R_{i alpha, j beta}^{a beta}
        R2[o:, :o, v:] = -np.swapaxes(r2, 0, 1)               # R_{j beta, i alpha}^{a beta}
        R2[:o, :o, :v] = r2 - np.swapaxes(r2, 0, 1)           # R_{i alpha, j alpha}^{a alpha}
        return S.ip_pack(R1, R2)

    def project(self, X):
        o, v = self.o, self.v
        R1, R2 = S.ip_unpack(X, 2 * o, 2 * v)
        return np.concatenate([R1[:o], R2[:o, o:, v:].reshape(-1)])

    def sigma(self, x):
        return self.project(self.so.ip_sigma(self.embed(x)))

    def rhs(self, p):
        return self.project(self.so.ip_rhs(int(self.alpha[p])))

    def left(self, q):
        o, v = self.o, self.v
        c1, c2 = S.ip_unpack(self.so.ip_left(int(self.alpha[q])), 2 * o, 2 * v)
        return np.concatenate([c1[:o], (c2[:o, o:, v:] + c2[:o, :o, :v]).reshape(-1)])

    def matrix(self):
        return np.stack([self.sigma(e) for e in np.eye(self.dim())], axis=1)

    def diag(self):
        fo, fv = np.diag(self.so.ip.Foo)[:self.o], np.diag(self.so.ip.Fvv)[:self.v]
        return np.concatenate([-fo, (fv[None, None, :] - fo[:, None, None] - fo[None, :, None]).reshape(-1)])

    def green_dense(self, omegas, eta, orbitals):
        M = self.matrix()
        B = np.stack([self.rhs(p) for p in orbitals], axis=1).astype(complex)
        C = np.stack([self.left(q) for q in orbitals], axis=1)
        G = np.zeros((len(omegas), len(orbitals), len(orbitals)), dtype=complex)
        for w, om in enumerate(omegas):
            X = np.linalg.solve((om - 1j * eta) * np.eye(M.shape[0]) + M, B)
            G[w] = (C.T @ X).T
        return G


# ---------------------------------------------------------------------------------------------- closed form
class SpatialIntegrals:
    """T1-rotated spatial Cholesky vectors and Fock matrix of a closed-shell reference:
    L'^K = (1 - t) L^K (1 + t), h = f - sum_j [2 (pq|jj) - (pj|jq)], f' = h' + sum_j [2 (pq|jj)' - (pj|jq)']."""

    def __init__(self, fock, chol, t1, o):
        n = fock.shape[0]
        self.o, self.n, self.v = o, n, n - o
        t = np.zeros((n, n))
        t[o:, :o] = t1.T
        X, Y = np.eye(n) - t, np.eye(n) + t
        J = np.einsum("kpq,kjj->pq", chol, chol[:, :o, :o], optimize=True)
        K = np.einsum("kpj,kjq->pq", chol[:, :, :o], chol[:, :o, :], optimize=True)
        h = fock - 2.0 * J + K
        self.Lt = np.einsum("xp,kpq,qy->kxy", X, chol, Y, optimize=True)
        Lt = self.Lt
        Jp = np.einsum("kpq,kjj->pq", Lt, Lt[:, :o, :o], optimize=True)
        Kp = np.einsum("kpj,kjq->pq", Lt[:, :, :o], Lt[:, :o, :], optimize=True)
        self.f = X @ h @ Y + 2.0 * Jp - Kp

    def sl(self, c):
        return slice(0, self.o) if c == "o" else slice(self.o, self.n)

    def chem(self, blk: str) -> np.ndarray:
        """(pq|rs)' over the block named by four of 'o'/'v' (p, q, r, s order)."""
        P, Q, R, T = (self.sl(c) for c in blk)
        return np.einsum("kpq,krs->pqrs", self.Lt[:, P, Q], self.Lt[:, R, T], optimize=True)

    def fblk(self, blk: str) -> np.ndarray:
        return self.f[self.sl(blk[0]), self.sl(blk[1])]


class RHFClosed:
    """The closed-form spin-adapted elements, sigma, right-hand sides and left vectors (module docstring)."""

    def __init__(self, fock, chol, t1, t2, lam1=None, lam2=None, o=None):
        o = t1.shape[0] if o is None else o
        self.o, self.v = o, fock.shape[0] - o
        self.t1, self.t2 = t1, t2
        self.lam1 = t1 if lam1 is None else lam1
        self.lam2 = t2 if lam2 is None else lam2
        I = SpatialIntegrals(fock, chol, t1, o)
        f, c = I.fblk, I.chem
        u = np.einsum("menf->mnef", c("ovov"), optimize=True)          # u_mnef = (me|nf)'
        self.u = u
        u2 = 2.0 * u - np.swapaxes(u, 2, 3)                              # 2 u_mnef - u_mnfe
        self.Fov = f("ov").copy()
        self.Foo = f("oo") + np.einsum("mnef,inef->mi", u2, t2, optimize=True)
        self.Fvv = f("vv") - np.einsum("mnef,mnaf->ae", u2, t2, optimize=True)
        self.Woooo = np.einsum("minj->mnij", c("oooo"), optimize=True) + np.einsum("mnef,ijef->mnij", u, t2,
                                                                                   optimize=True)
        ooov = c("ooov")                                                 # (mi|ne)' as [m][i][n][e]
        self.Wooov = np.einsum("mine->mnie", ooov, optimize=True)
        mine = ooov                                                      # (mi|ne)'
        meni = c("ovoo")                                                 # (me|ni)' as [m][e][n][i]
        self.Wovoo = (np.einsum("miaj->maij", c("oovo"), optimize=True)
                      + np.einsum("me,ijea->maij", self.Fov, t2, optimize=True)
                      + np.einsum("meaf,ijef->maij", c("ovvv"), t2, optimize=True)
                      + np.einsum("mine,jnae->maij", 2.0 * mine - np.einsum("meni->mine", meni), t2, optimize=True)
                      - np.einsum("mine,jnea->maij", mine, t2, optimize=True)
                      - np.einsum("menj,inea->maij", meni, t2, optimize=True))
        self.X = (np.einsum("meai->maei", c("ovvo"), optimize=True)
                  + np.einsum("mnef,inaf->maei", u2, t2, optimize=True)
                  - np.einsum("mnef,infa->maei", u, t2, optimize=True))
        self.Y = (np.einsum("miae->maie", c("oovv"), optimize=True)
                  - np.einsum("mnfe,infa->maie", u, t2, optimize=True))

    def dim(self):
        return ip_dim(self.o, self.v)

    def sigma(self, x):
        o, v = self.o, self.v
        r1, r2 = split(x, o, v)
        u2 = 2.0 * self.u - np.swapaxes(self.u, 2, 3)
        s1 = (-np.einsum("mi,m->i", self.Foo, r1, optimize=True)
              + np.einsum("me,ime->i", self.Fov, 2.0 * r2, optimize=True)
              - np.einsum("me,mie->i", self.Fov, r2, optimize=True)
              + np.einsum("nmie,mne->i", self.Wooov, r2, optimize=True)
              - 2.0 * np.einsum("mnie,mne->i", self.Wooov, r2, optimize=True))
        s2 = (-np.einsum("maij,m->ija", self.Wovoo, r1, optimize=True)
              + np.einsum("ae,ije->ija", self.Fvv, r2, optimize=True)
              - np.einsum("mi,mja->ija", self.Foo, r2, optimize=True)
              - np.einsum("mj,ima->ija", self.Foo, r2, optimize=True)
              + np.einsum("mnij,mna->ija", self.Woooo, r2, optimize=True)
              - np.einsum("maie,mje->ija", self.Y, r2, optimize=True)
              + np.einsum("maej,ime->ija", 2.0 * self.X, r2, optimize=True)
              - np.einsum("maje,ime->ija", self.Y, r2, optimize=True)
              - np.einsum("maej,mie->ija", self.X, r2, optimize=True))
        z = np.einsum("mnef,mnf->e", u2, r2, optimize=True)
        s2 = s2 - np.einsum("e,ijea->ija", z, self.t2, optimize=True)
        return np.concatenate([s1, s2.reshape(-1)])

    def rhs(self, p):
        o, v = self.o, self.v
        r1 = np.zeros(o)
        r2 = np.zeros((o, o, v))
        if p < o:
            r1[p] = 1.0
        else:
            b = p - o
            r1[:] = self.t1[:, b]
            r2[:] = self.t2[:, :, b, :]          # r_ij^a = t_ij^ba
        return np.concatenate([r1, r2.reshape(-1)])

    def left(self, q):
        o, v = self.o, self.v
        t1, t2, l1, l2 = self.t1, self.t2, self.lam1, self.lam2
        c1 = np.zeros(o)
        c2 = np.zeros((o, o, v))
        if q >= o:
            b = q - o
            c1[:] = l1[:, b]
            c2[:] = 2.0 * l2[:, :, b, :] - l2[:, :, :, b]
        else:
            m = q
            c1[:] = (-np.einsum("c,ic->i", t1[m], l1, optimize=True)
                     - np.einsum("lcd,ilcd->i", 2.0 * t2[m] - np.swapaxes(t2[m], 1, 2), l2, optimize=True))
            c1[m] += 1.0
            c2[m, :, :] += 2.0 * l1
            c2[:, m, :] -= l1
            c2 -= 2.0 * np.einsum("c,ijca->ija", t1[m], l2, optimize=True)
            c2 += np.einsum("c,ijac->ija", t1[m], l2, optimize=True)
        return np.concatenate([c1, c2.reshape(-1)])

    def diag(self):
        fo, fv = np.diag(self.Foo), np.diag(self.Fvv)
        return np.concatenate([-fo, (fv[None, None, :] - fo[:, None, None] - fo[None, :, None]).reshape(-1)])

    def green(self, omegas, eta, orbitals, tol=1e-12, restart=30, max_restarts=50, precond=False, stats=None):
        """G[w][p][q] by GMRES per (omega, p) on the closed-form sigma (right-preconditioned by the
        Fock-like diagonal when precond)."""
        no = len(orbitals)
        G = np.zeros((len(omegas), no, no), dtype=complex)
        C = np.stack([self.left(q) for q in orbitals])
        dg = self.diag() if precond else None
        for w, om in enumerate(omegas):
            A = (lambda om_: (lambda x: (om_ - 1j * eta) * x + self.sigma(x)))(om)
            D = None if dg is None else (om - 1j * eta) + dg
            for a, p in enumerate(orbitals):
                x, its, rel, ok = S.gmres(A, self.rhs(p), tol, restart, max_restarts, diag=D)
                if stats is not None:
                    stats.append((its, rel, ok))
                G[w, a] = C @ x
        return G
