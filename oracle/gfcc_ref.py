"""Closed-form FP64 CPU oracle of the GFCCSD hot path (test infrastructure).

Plain numpy, fp64, no blocking or fusion: every quantity is written out as the
contraction that defines it, so that it can be checked against the paper and
against the brute-force Fock-space definition (oracle/fock_space.py) by eye.
Only tests/, the smoke check and the bench's CPU baseline use this module; the
product never imports it.

What it computes (paper, Theory section):
  * eq. xplin: (omega - i eta + Hbar_N) X_p|Phi> = a_p-bar|Phi> in the 1h + 2h1p
    space of eq. xp, and (omega + i eta - Hbar_N) Y_q|Phi> = a_q^+-bar|Phi> in the
    1p + 2p1h space of eq. yq; the operator is the commutator form
    <mu|[Hbar, R]|Phi> (identical to Hbar_N = Hbar - E0 when T solves CC).
  * eqs. gfxn2/gfxn3: G_pq = <Phi|(1+Lambda) a_q^+-bar X_p|Phi> + <Phi|(1+Lambda) a_p-bar Y_q|Phi>.
  * The linear systems are solved by non-preconditioned GMRES (GFCC Workflow and
    Bottlenecks section; Saad & Schultz 1986) with modified Gram-Schmidt Arnoldi
    and Givens rotations.

How Hbar is evaluated.  T = T1 + T2 with [T1, T2] = 0, so
Hbar = e^-T2 (e^-T1 H e^T1) e^T2.  The inner transform is an orbital rotation:
e^-T1 a_p^+ e^T1 = sum_x a_x^+ (1 - t)_xp and e^-T1 a_q e^T1 = sum_y (1 + t)_qy a_y
with t[a][i] = t_i^a (t^2 = 0), so e^-T1 H e^T1 is a two-body Hamiltonian with
integrals h' = (1-t) h (1+t) and Cholesky vectors L'^K = (1-t) L^K (1+t) (the
Cholesky representation of the integrals is the one of the Implementation
Details section).  The outer transform by T2 alone gives the Hbar elements below
(standard spin-orbital EOM-CCSD elements, restricted to T1 = 0; Stanton & Gauss
1994 for IP, Nooijen & Bartlett 1995 for EA), and the sigma products are the
standard IP/EA-EOM-CCSD equations in those elements.  Every element and every
sigma term is pinned to the brute-force definition in tests/test_oracle_pins.py.

Index conventions.  n = o + v orbitals, occupied first.  IP vector
X = sum_i r1[i] a_i + 1/2 sum_ija r2[i,j,a] a_a^+ a_j a_i (r2 antisymmetric in ij);
packed coordinates are r1 and r2[i<j, a] (pairs in lexicographic order, a fastest).
EA vector Y = sum_a y1[a] a_a^+ + 1/2 sum_iab y2[i,a,b] a_a^+ a_b^+ a_i (antisymmetric
in ab); packed coordinates y1 and y2[i, a<b].
"""
from __future__ import annotations

import numpy as np

# --------------------------------------------------------------------------------------------
# packing
# --------------------------------------------------------------------------------------------


def pair_index(m: int):
    """(i, j) arrays of the pairs i < j of range(m), lexicographic."""
    return np.triu_indices(m, 1)


def ip_dim(o, v):
    return o + (o * (o - 1) // 2) * v


def ea_dim(o, v):
    return v + o * (v * (v - 1) // 2)


def ip_unpack(x, o, v):
    """packed IP vector -> (r1[o], r2[o,o,v]) with r2 antisymmetric in (i,j)."""
    r1 = x[:o]
    ii, jj = pair_index(o)
    p = x[o:].reshape(len(ii), v)
    r2 = np.zeros((o, o, v), dtype=x.dtype)
    r2[ii, jj] = p
    r2[jj, ii] = -p
    return r1.copy(), r2


def ip_pack(r1, r2):
    o = r1.shape[0]
    ii, jj = pair_index(o)
    return np.concatenate([r1, r2[ii, jj].reshape(-1)])


def ea_unpack(y, o, v):
    y1 = y[:v]
    aa, bb = pair_index(v)
    p = y[v:].reshape(o, len(aa))
    y2 = np.zeros((o, v, v), dtype=y.dtype)
    y2[:, aa, bb] = p
    y2[:, bb, aa] = -p
    return y1.copy(), y2


def ea_pack(y1, y2):
    v = y1.shape[0]
    aa, bb = pair_index(v)
    return np.concatenate([y1, y2[:, aa, bb].reshape(-1)])


# --------------------------------------------------------------------------------------------
# integrals and the T1 transformation
# --------------------------------------------------------------------------------------------


class Integrals:
    """T1-transformed one-body and Cholesky integrals (see module docstring)."""

    def __init__(self, fock, chol, t1, o):
        n = fock.shape[0]
        self.o, self.n, self.v = o, n, n - o
        t = np.zeros((n, n))
        t[o:, :o] = t1.T                      # t[a][i] = t_i^a
        X = np.eye(n) - t                     # e^-T1 a_p^+ e^T1 = sum_x a_x^+ X[x,p]
        Y = np.eye(n) + t                     # e^-T1 a_q e^T1 = sum_y Y[q,y] a_y
        self.X, self.Y = X, Y
        # core Hamiltonian: reference Fock matrix of h with <pq||rs> is f
        J = np.einsum("kpq,kjj->pq", chol, chol[:, :o, :o], optimize=True)
        K = np.einsum("kpj,kjq->pq", chol[:, :, :o], chol[:, :o, :], optimize=True)
        h = fock - J + K
        self.Lt = np.einsum("xp,kpq,qy->kxy", X, chol, Y, optimize=True)    # L'^K = X L^K Y
        hp = X @ h @ Y
        Lt = self.Lt
        Jp = np.einsum("kpq,kjj->pq", Lt, Lt[:, :o, :o], optimize=True)
        Kp = np.einsum("kpj,kjq->pq", Lt[:, :, :o], Lt[:, :o, :], optimize=True)
        self.f = hp + Jp - Kp                 # f'_pq = h'_pq + sum_j <pj||qj>'

    def sl(self, c):
        return slice(0, self.o) if c == "o" else slice(self.o, self.n)

    def eri(self, blk: str) -> np.ndarray:
        """<pq||rs>' over the block named by four of 'o'/'v' (p, q, r, s order)."""
        P, Q, R, S = (self.sl(c) for c in blk)
        Lt = self.Lt
        return (np.einsum("kpr,kqs->pqrs", Lt[:, P, R], Lt[:, Q, S], optimize=True)
                - np.einsum("kps,kqr->pqrs", Lt[:, P, S], Lt[:, Q, R], optimize=True))

    def fblk(self, blk: str) -> np.ndarray:
        return self.f[self.sl(blk[0]), self.sl(blk[1])]


# --------------------------------------------------------------------------------------------
# Hbar elements (T2 part, T1 inside the integrals)
# --------------------------------------------------------------------------------------------


class HbarIP:
    """Hbar elements used by the IP sigma (Stanton & Gauss 1994, T1 = 0 forms)."""

    def __init__(self, ints: Integrals, t2):
        self.t2 = t2
        f = ints.fblk
        voovv = ints.eri("oovv")
        self.v_oovv = voovv
        self.Fov = f("ov").copy()
        self.Foo = f("oo") + 0.5 * np.einsum("mnef,inef->mi", voovv, t2, optimize=True)
        self.Fvv = f("vv") - 0.5 * np.einsum("mnef,mnaf->ae", voovv, t2, optimize=True)
        self.Woooo = ints.eri("oooo") + 0.5 * np.einsum("mnef,ijef->mnij", voovv, t2, optimize=True)
        self.Wooov = ints.eri("ooov")
        self.Wovvo = ints.eri("ovvo") - np.einsum("mnef,jnfb->mbej", voovv, t2, optimize=True)
        v_ooov = self.Wooov
        tmp = np.einsum("mnie,jnbe->mbij", v_ooov, t2, optimize=True)
        self.Wovoo = (ints.eri("ovoo")
                      - np.einsum("me,ijbe->mbij", self.Fov, t2, optimize=True)
                      + 0.5 * np.einsum("mbef,ijef->mbij", ints.eri("ovvv"), t2, optimize=True)
                      + tmp - tmp.transpose(0, 1, 3, 2))


class HbarEA:
    """Hbar elements used by the EA sigma (Nooijen & Bartlett 1995, T1 = 0 forms)."""

    def __init__(self, ints: Integrals, t2, ip: HbarIP | None = None):
        self.t2 = t2
        f = ints.fblk
        voovv = ints.eri("oovv")
        self.v_oovv = voovv
        self.Fov = f("ov").copy()
        self.Foo = f("oo") + 0.5 * np.einsum("mnef,inef->mi", voovv, t2, optimize=True)
        self.Fvv = f("vv") - 0.5 * np.einsum("mnef,mnaf->ae", voovv, t2, optimize=True)
        self.Wovvo = ints.eri("ovvo") - np.einsum("mnef,jnfb->mbej", voovv, t2, optimize=True)
        self.Wvovv = ints.eri("vovv")
        self.Wvvvv = ints.eri("vvvv") + 0.5 * np.einsum("mnef,mnab->abef", voovv, t2, optimize=True)
        v_ovvv = ints.eri("ovvv")
        tmp = np.einsum("mbef,miaf->abei", v_ovvv, t2, optimize=True)
        self.Wvvvo = (ints.eri("vvvo")
                      - np.einsum("me,miab->abei", self.Fov, t2, optimize=True)
                      + 0.5 * np.einsum("mnei,mnab->abei", ints.eri("oovo"), t2, optimize=True)
                      - tmp + tmp.transpose(1, 0, 2, 3))


# --------------------------------------------------------------------------------------------
# sigma products: <mu|[Hbar, R]|Phi>
# --------------------------------------------------------------------------------------------


def ip_sigma_unpacked(hb: HbarIP, r1, r2):
    """IP-EOM-CCSD sigma in Hbar elements (1h and 2h1p projections of [Hbar, R]|Phi>)."""
    t2 = hb.t2
    s1 = (-np.einsum("mi,m->i", hb.Foo, r1, optimize=True)
          - np.einsum("me,mie->i", hb.Fov, r2, optimize=True)
          + 0.5 * np.einsum("nmie,mne->i", hb.Wooov, r2, optimize=True))
    s2 = np.einsum("maji,m->ija", hb.Wovoo, r1, optimize=True)
    s2 = s2 + np.einsum("ae,ije->ija", hb.Fvv, r2, optimize=True)
    tmp = np.einsum("mi,mja->ija", hb.Foo, r2, optimize=True)
    s2 = s2 - tmp + tmp.transpose(1, 0, 2)
    s2 = s2 + 0.5 * np.einsum("mnij,mna->ija", hb.Woooo, r2, optimize=True)
    tmp = np.einsum("maei,mje->ija", hb.Wovvo, r2, optimize=True)
    s2 = s2 + tmp - tmp.transpose(1, 0, 2)
    z = 0.5 * np.einsum("mnef,mnf->e", hb.v_oovv, r2, optimize=True)          # three-body term
    s2 = s2 + np.einsum("e,ijae->ija", z, t2, optimize=True)
    return s1, s2


def ea_sigma_unpacked(hb: HbarEA, y1, y2):
    """EA-EOM-CCSD sigma in Hbar elements (1p and 2p1h projections of [Hbar, Q]|Phi>)."""
    t2 = hb.t2
    s1 = (np.einsum("ae,e->a", hb.Fvv, y1, optimize=True)
          + np.einsum("me,mae->a", hb.Fov, y2, optimize=True)
          + 0.5 * np.einsum("amef,mef->a", hb.Wvovv, y2, optimize=True))
    s2 = np.einsum("abei,e->iab", hb.Wvvvo, y1, optimize=True)
    s2 = s2 - np.einsum("mi,mab->iab", hb.Foo, y2, optimize=True)
    tmp = np.einsum("be,iae->iab", hb.Fvv, y2, optimize=True)
    s2 = s2 + tmp - tmp.transpose(0, 2, 1)
    s2 = s2 + 0.5 * np.einsum("abef,ief->iab", hb.Wvvvv, y2, optimize=True)
    tmp = np.einsum("mbei,mae->iab", hb.Wovvo, y2, optimize=True)
    s2 = s2 + tmp - tmp.transpose(0, 2, 1)
    z = 0.5 * np.einsum("mnef,nef->m", hb.v_oovv, y2, optimize=True)          # three-body term
    s2 = s2 - np.einsum("m,miab->iab", z, t2, optimize=True)
    return s1, s2


# --------------------------------------------------------------------------------------------
# right-hand sides and left vectors
# --------------------------------------------------------------------------------------------


def ip_rhs_unpacked(o, v, t1, t2, p):
    """b_p = a_p-bar|Phi> projected on 1h + 2h1p.

    a_m-bar = a_m; a_b-bar = a_b + sum_k t_k^b a_k + 1/2 sum_kld t_kl^bd a_d^+ a_l a_k."""
    r1 = np.zeros(o)
    r2 = np.zeros((o, o, v))
    if p < o:
        r1[p] = 1.0
    else:
        b = p - o
        r1[:] = t1[:, b]
        r2[:] = t2[:, :, b, :]
    return r1, r2


def ip_left(o, v, t1, t2, lam1, lam2, q):
    """c_q(mu) = <Phi|(1+Lambda) a_q^+-bar|mu> (packed-coordinate values, antisymmetric in ij).

    a_b^+-bar = a_b^+; a_m^+-bar = a_m^+ - sum_c t_m^c a_c^+ - 1/2 sum_lcd t_ml^cd a_c^+ a_d^+ a_l."""
    c1 = np.zeros(o)
    c2 = np.zeros((o, o, v))
    if q >= o:
        b = q - o
        c1[:] = lam1[:, b]
        c2[:] = lam2[:, :, b, :]
    else:
        m = q
        c1[:] = (-np.einsum("c,kc->k", t1[m], lam1, optimize=True)
                 - 0.5 * np.einsum("lcd,klcd->k", t2[m], lam2, optimize=True))
        c1[m] += 1.0
        c2[m, :, :] += lam1
        c2[:, m, :] -= lam1
        c2 -= np.einsum("c,ijca->ija", t1[m], lam2, optimize=True)
    return c1, c2


def ea_rhs_unpacked(o, v, t1, t2, q):
    """b^EA_q = a_q^+-bar|Phi> projected on 1p + 2p1h."""
    y1 = np.zeros(v)
    y2 = np.zeros((o, v, v))
    if q >= o:
        y1[q - o] = 1.0
    else:
        y1[:] = -t1[q]
        y2[:] = -t2[q]
    return y1, y2


def ea_left(o, v, t1, t2, lam1, lam2, p):
    """c^EA_p(mu) = <Phi|(1+Lambda) a_p-bar|mu> (packed-coordinate values, antisymmetric in ab)."""
    c1 = np.zeros(v)
    c2 = np.zeros((o, v, v))
    if p < o:
        m = p
        c1[:] = -lam1[m]
        c2[:] = lam2[:, m, :, :]
    else:
        e = p - o
        c1[:] = (-np.einsum("k,kc->c", t1[:, e], lam1, optimize=True)
                 + 0.5 * np.einsum("kld,kldc->c", t2[:, :, e, :], lam2, optimize=True))
        c1[e] += 1.0
        c2[:, e, :] += lam1
        c2[:, :, e] -= lam1
        c2 += np.einsum("k,ikcd->icd", t1[:, e], lam2, optimize=True)
    return c1, c2


# --------------------------------------------------------------------------------------------
# GMRES (Saad & Schultz 1986), complex, restarted, modified Gram-Schmidt + Givens
# --------------------------------------------------------------------------------------------


def gmres(apply_A, b, tol, restart=30, max_restarts=50, x0=None, history=None, diag=None):
    """Solve A x = b to ||b - A x|| <= tol ||b||.  Returns (x, iterations, true relative residual, converged).

    diag (optional) is a right preconditioner D (vector): GMRES runs on A D^-1 u = b, x = D^-1 u, so the
    residual it minimises is still the residual of A x = b."""
    if diag is not None:
        x1, its, rel, ok = gmres(lambda u: apply_A(u / diag), b, tol, restart, max_restarts,
                                 None if x0 is None else x0 * diag, history)
        return x1 / diag, its, rel, ok
    b = b.astype(complex)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return np.zeros_like(b), 0, 0.0, True
    x = np.zeros_like(b) if x0 is None else x0.astype(complex).copy()
    its = 0
    for _ in range(max_restarts):
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
        if history is not None:
            history.append(beta / nb)
        if beta <= tol * nb:
            return x, its, beta / nb, True
        m = restart
        V = np.zeros((m + 1, b.size), dtype=complex)
        Hh = np.zeros((m + 1, m), dtype=complex)
        cs = np.zeros(m, dtype=complex)
        sn = np.zeros(m, dtype=complex)
        g = np.zeros(m + 1, dtype=complex)
        g[0] = beta
        V[0] = r / beta
        k_used = 0
        for k in range(m):
            w = apply_A(V[k])
            its += 1
            for i in range(k + 1):                       # modified Gram-Schmidt
                Hh[i, k] = np.vdot(V[i], w)
                w = w - Hh[i, k] * V[i]
            Hh[k + 1, k] = np.linalg.norm(w)
            if Hh[k + 1, k] != 0.0:
                V[k + 1] = w / Hh[k + 1, k]
            for i in range(k):                           # previous rotations
                t = cs[i] * Hh[i, k] + sn[i] * Hh[i + 1, k]
                Hh[i + 1, k] = -np.conj(sn[i]) * Hh[i, k] + np.conj(cs[i]) * Hh[i + 1, k]
                Hh[i, k] = t
            a, bb = Hh[k, k], Hh[k + 1, k]
            den = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
            cs[k] = a / den if den != 0 else 1.0
            sn[k] = bb / den if den != 0 else 0.0
            cs[k], sn[k] = np.conj(cs[k]), np.conj(sn[k])
            Hh[k, k] = cs[k] * a + sn[k] * bb
            Hh[k + 1, k] = 0.0
            g[k + 1] = -np.conj(sn[k]) * g[k]
            g[k] = cs[k] * g[k]
            k_used = k + 1
            if history is not None:
                history.append(abs(g[k + 1]) / nb)
            if abs(g[k + 1]) <= tol * nb or Hh[k, k] == 0.0:
                break
        y = np.linalg.solve(np.triu(Hh[:k_used, :k_used]), g[:k_used])
        x = x + V[:k_used].T @ y
    r = b - apply_A(x)
    rel = np.linalg.norm(r) / nb
    return x, its, rel, rel <= tol


# --------------------------------------------------------------------------------------------
# the full problem
# --------------------------------------------------------------------------------------------


class GFCCOracle:
    """All oracle quantities for one problem (fock, chol, t1, t2, lambda)."""

    def __init__(self, fock, chol, t1, t2, lam1=None, lam2=None, o=None, sectors=("IP", "EA")):
        o = t1.shape[0] if o is None else o
        self.o, self.v = o, fock.shape[0] - o
        self.t1, self.t2 = t1, t2
        self.lam1 = t1 if lam1 is None else lam1       # Lambda = T^dagger by default
        self.lam2 = t2 if lam2 is None else lam2
        self.ints = Integrals(fock, chol, t1, o)
        self.ip = HbarIP(self.ints, t2) if "IP" in sectors else None
        self.ea = HbarEA(self.ints, t2) if "EA" in sectors else None

    # vectors (packed) ---------------------------------------------------------------------
    def ip_sigma(self, x):
        r1, r2 = ip_unpack(x, self.o, self.v)
        return ip_pack(*ip_sigma_unpacked(self.ip, r1, r2))

    def ea_sigma(self, y):
        y1, y2 = ea_unpack(y, self.o, self.v)
        return ea_pack(*ea_sigma_unpacked(self.ea, y1, y2))

    def ip_rhs(self, p):
        # a_p-bar with the T1 part through Y = 1 + t: a_p-bar = sum_q Y[p,q] e^-T2 a_q e^T2
        return ip_pack(*ip_rhs_unpacked(self.o, self.v, self.t1, self.t2, p))

    def ip_left(self, q):
        return ip_pack(*ip_left(self.o, self.v, self.t1, self.t2, self.lam1, self.lam2, q))

    def ea_rhs(self, q):
        return ea_pack(*ea_rhs_unpacked(self.o, self.v, self.t1, self.t2, q))

    def ea_left(self, p):
        return ea_pack(*ea_left(self.o, self.v, self.t1, self.t2, self.lam1, self.lam2, p))

    # diagonal preconditioners: the Fock-like diagonal of Hbar (Fbar_oo, Fbar_vv) ------------
    def ip_diag(self):
        fo, fv = np.diag(self.ip.Foo), np.diag(self.ip.Fvv)
        ii, jj = np.triu_indices(self.o, 1)
        return np.concatenate([-fo, (fv[None, :] - fo[ii][:, None] - fo[jj][:, None]).reshape(-1)])

    def ea_diag(self):
        fo, fv = np.diag(self.ea.Foo), np.diag(self.ea.Fvv)
        aa, bb = np.triu_indices(self.v, 1)
        return np.concatenate([fv, (fv[aa][None, :] + fv[bb][None, :] - fo[:, None]).reshape(-1)])

    # systems ------------------------------------------------------------------------------
    def ip_apply(self, omega, eta):
        return lambda x: (omega - 1j * eta) * x + self.ip_sigma(x)

    def ea_apply(self, omega, eta):
        return lambda y: (omega + 1j * eta) * y - self.ea_sigma(y)

    def ip_matrix(self):
        n = ip_dim(self.o, self.v)
        return np.stack([self.ip_sigma(e) for e in np.eye(n)], axis=1)

    def ea_matrix(self):
        n = ea_dim(self.o, self.v)
        return np.stack([self.ea_sigma(e) for e in np.eye(n)], axis=1)

    def green(self, omegas, eta, orbitals, tol=1e-12, restart=30, max_restarts=50, sectors=("IP", "EA"),
              stats=None, precond=False):
        """G[w][p][q] = G^IP + G^EA over the orbital list (eq. gfxn3), by GMRES per (omega, p).

        precond=True right-preconditions each system with its Fock-like diagonal."""
        no = len(orbitals)
        G = np.zeros((len(omegas), no, no), dtype=complex)
        if "IP" in sectors:
            C = np.stack([self.ip_left(q) for q in orbitals])
            dg = self.ip_diag() if precond else None
            for w, om in enumerate(omegas):
                A = self.ip_apply(om, eta)
                D = None if dg is None else (om - 1j * eta) + dg
                for a, p in enumerate(orbitals):
                    x, its, rel, ok = gmres(A, self.ip_rhs(p), tol, restart, max_restarts, diag=D)
                    if stats is not None:
                        stats.append(("IP", w, p, its, rel, ok))
                    G[w, a, :] += C @ x
        if "EA" in sectors:
            C = np.stack([self.ea_left(p) for p in orbitals])
            dg = self.ea_diag() if precond else None
            for w, om in enumerate(omegas):
                A = self.ea_apply(om, eta)
                D = None if dg is None else (om + 1j * eta) - dg
                for b, q in enumerate(orbitals):
                    y, its, rel, ok = gmres(A, self.ea_rhs(q), tol, restart, max_restarts, diag=D)
                    if stats is not None:
                        stats.append(("EA", w, q, its, rel, ok))
                    G[w, :, b] += C @ y
        return G

    def green_dense(self, omegas, eta, orbitals, sectors=("IP", "EA")):
        """Same G from dense LU solves (small sizes only)."""
        no = len(orbitals)
        G = np.zeros((len(omegas), no, no), dtype=complex)
        if "IP" in sectors:
            M = self.ip_matrix()
            B = np.stack([self.ip_rhs(p) for p in orbitals], axis=1)
            C = np.stack([self.ip_left(q) for q in orbitals], axis=1)
            for w, om in enumerate(omegas):
                X = np.linalg.solve((om - 1j * eta) * np.eye(M.shape[0]) + M, B.astype(complex))
                G[w] += (C.T @ X).T
        if "EA" in sectors:
            M = self.ea_matrix()
            B = np.stack([self.ea_rhs(q) for q in orbitals], axis=1)
            C = np.stack([self.ea_left(p) for p in orbitals], axis=1)
            for w, om in enumerate(omegas):
                Y = np.linalg.solve((om + 1j * eta) * np.eye(M.shape[0]) - M, B.astype(complex))
                G[w] += C.T @ Y
        return G
