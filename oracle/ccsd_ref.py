"""CPU FP64 reference of the ground-state coupled-cluster step before the Green's function: CCSD for
T and the Lambda-CCSD equations for the de-excitation operator (test infrastructure: only tests/, the
smoke check and the bench's CPU legs use this module; the product never imports it).

The paper obtains T and Lambda "from solving the conventional CC equations" (Theory section) with
Cholesky-decomposed two-electron integrals (Implementation Details; Workflow section: CCSD costs
O(O^2 V^4)).  Here, on the same synthetic Hamiltonian as the Green's-function path:

T equations.  T = T1 + T2 with [T1, T2] = 0, so e^-T H e^T = e^-T2 H' e^T2 with H' the T1-rotated
Hamiltonian of gfcc_ref.Integrals (h' = (1-t) h (1+t), L'^K = (1-t) L^K (1+t)).  The CCSD residuals
are the projections of that operator on the singles and doubles,
    Omega1[i][a] = <Phi_i^a| e^-T2 H' e^T2 |Phi>,   Omega2[i][j][a][b] = <Phi_ij^ab| e^-T2 H' e^T2 |Phi>,
i.e. the T1 = 0 forms of the spin-orbital CCSD equations in the rotated basis (f' has non-zero ov and vo
blocks; no f'_ov term reaches the doubles):
    Omega1_ia = f'_ai + f'_me t_im^ae + 1/2 <am||ef>' t_im^ef + 1/2 <mn||ei>' t_mn^ae
    Omega2_ijab = <ab||ij>' + P(ab) F_be t_ij^ae - P(ij) F_mj t_im^ab + 1/2 W_mnij t_mn^ab
                  + 1/2 W_abef t_ij^ef + P(ij) P(ab) W_mbej t_im^ae
with  F_be = f'_be - 1/2 <mn||ef>' t_mn^bf,  F_mj = f'_mj + 1/2 <mn||ef>' t_jn^ef,
      W_mnij = <mn||ij>' + 1/4 <mn||ef>' t_ij^ef,  W_abef = <ab||ef>' + 1/4 <mn||ef>' t_mn^ab,
      W_mbej = <mb||ej>' - 1/2 <mn||ef>' t_jn^fb      (summation over repeated indices).
Correlation energy: E_c = f_ia t_i^a + 1/4 <ij||ab> t_ij^ab + 1/2 <ij||ab> t_i^a t_j^b (original basis).

Lambda equations.  Lambda is the left ground state of Hbar: <Phi|(1 + Lambda)(Hbar - E) |mu> = 0 for
the singles and doubles mu.  With Hbar = e^-T2 H' e^T2 the equations take their T1 = 0 form in the
elements of that operator (the Hbar elements of gfcc_ref, built from the rotated integrals and T2).
The disconnected parts of <nu|Hbar|mu> that carry a T residual are left out, so the residuals below
equal the definition where T solves the T equations:
    0 = Fb_ia + lam_ie Fb_ea - lam_ma Fb_im + lam_me Wb_ieam + 1/2 lam_imef Wb_efam
        - 1/2 lam_mnae Wb_iemn - G_ef Wb_eifa - G_mn Wb_mina
    0 = <ij||ab>' + P(ab) lam_ijae Fb_eb - P(ij) lam_imab Fb_jm + 1/2 lam_mnab Wb_ijmn
        + 1/2 lam_ijef Wb_efab + P(ij) lam_ie Wb_ejab - P(ab) lam_ma Wb_ijmb
        + P(ij) P(ab) lam_imae Wb_jebm + P(ij) P(ab) lam_ia Fb_jb
        + P(ab) <ij||ae>' G_be - P(ij) <im||ab>' G_mj
with  G_ae = -1/2 t_mn^ef lam_mnaf,  G_mi = 1/2 t_mn^ef lam_inef,  lam_ia = lambda_a^i, lam_ijab = lambda_ab^ij.
The Hbar elements are those of the operator itself, <p|Hbar|q> blocks with T1 = 0 in the rotated basis
(listed in lambda_elements).  Every residual is pinned to the Fock-space definition
(tests/test_oracle_ccsd.py).

Solver: Jacobi updates with the Fock-like diagonal (t += Omega / D) accelerated by DIIS over the last
8 iterates (Pulay 1980), for T and then for Lambda.
"""
from __future__ import annotations

import numpy as np

from oracle.gfcc_ref import Integrals


def _P(x, axes):
    """x - x with the two given axes swapped (antisymmetriser P(pq) of the text)."""
    return x - np.swapaxes(x, *axes)


# --------------------------------------------------------------------------------------------- T
def t_residuals(fock, chol, t1, t2, o):
    """(Omega1 [o][v], Omega2 [o][o][v][v]) of the CCSD equations at (t1, t2)."""
    ints = Integrals(fock, chol, t1, o)
    f = ints.fblk
    e = ints.eri
    oovv = e("oovv")
    Fvv = f("vv") - 0.5 * np.einsum("mnef,mnbf->be", oovv, t2, optimize=True)
    Foo = f("oo") + 0.5 * np.einsum("mnef,jnef->mj", oovv, t2, optimize=True)
    Woooo = e("oooo") + 0.25 * np.einsum("mnef,ijef->mnij", oovv, t2, optimize=True)
    Wvvvv = e("vvvv") + 0.25 * np.einsum("mnef,mnab->abef", oovv, t2, optimize=True)
    Wovvo = e("ovvo") - 0.5 * np.einsum("mnef,jnfb->mbej", oovv, t2, optimize=True)
    r1 = (f("vo").T + np.einsum("me,imae->ia", f("ov"), t2, optimize=True)
          + 0.5 * np.einsum("amef,imef->ia", e("vovv"), t2, optimize=True)
          + 0.5 * np.einsum("mnei,mnae->ia", e("oovo"), t2, optimize=True))
    r2 = e("vvoo").transpose(2, 3, 0, 1).copy()    # <ab||ij>' (the rotated integrals are not symmetric)
    r2 += _P(np.einsum("be,ijae->ijab", Fvv, t2, optimize=True), (2, 3))
    r2 -= _P(np.einsum("mj,imab->ijab", Foo, t2, optimize=True), (0, 1))
    r2 += 0.5 * np.einsum("mnij,mnab->ijab", Woooo, t2, optimize=True)
    r2 += 0.5 * np.einsum("abef,ijef->ijab", Wvvvv, t2, optimize=True)
    ring = np.einsum("mbej,imae->ijab", Wovvo, t2, optimize=True)
    r2 += ring - ring.transpose(1, 0, 2, 3) - ring.transpose(0, 1, 3, 2) + ring.transpose(1, 0, 3, 2)
    return r1, r2


def correlation_energy(fock, chol, t1, t2, o):
    """E_c = f_ia t_i^a + 1/4 <ij||ab> t_ij^ab + 1/2 <ij||ab> t_i^a t_j^b in the original basis."""
    ints = Integrals(fock, chol, np.zeros_like(t1), o)
    oovv = ints.eri("oovv")
    fov = ints.fblk("ov")
    return float(np.einsum("ia,ia->", fov, t1) + 0.25 * np.einsum("ijab,ijab->", oovv, t2)
                 + 0.5 * np.einsum("ijab,ia,jb->", oovv, t1, t1, optimize=True))


def denominators(fock, o):
    """D1[i][a] = f_ii - f_aa, D2[i][j][a][b] = f_ii + f_jj - f_aa - f_bb (the Jacobi preconditioner)."""
    e = np.diag(fock)
    eo, ev = e[:o], e[o:]
    return eo[:, None] - ev[None, :], eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - \
        ev[None, None, None, :]


class _DIIS:
    def __init__(self, size=8):
        self.size, self.x, self.r = size, [], []

    def push(self, x, r):
        self.x.append(x.copy())
        self.r.append(r.copy())
        if len(self.x) > self.size:
            self.x.pop(0)
            self.r.pop(0)
        k = len(self.x)
        if k < 2:
            return x
        B = -np.ones((k + 1, k + 1))
        B[k, k] = 0.0
        for a in range(k):
            for b in range(k):
                B[a, b] = self.r[a] @ self.r[b]
        rhs = np.zeros(k + 1)
        rhs[k] = -1.0
        try:
            c = np.linalg.solve(B, rhs)[:k]
        except np.linalg.LinAlgError:
            return x
        return sum(ci * xi for ci, xi in zip(c, self.x))


def _antisym(t2):
    return 0.25 * (t2 - t2.transpose(1, 0, 2, 3) - t2.transpose(0, 1, 3, 2) + t2.transpose(1, 0, 3, 2))


def solve_t(fock, chol, o, tol=1e-10, max_iter=200, t1=None, t2=None):
    """Converged (t1, t2, E_c, iterations): max |Omega| <= tol."""
    n = fock.shape[0]
    v = n - o
    D1, D2 = denominators(fock, o)
    t1 = np.zeros((o, v)) if t1 is None else t1.copy()
    t2 = np.zeros((o, o, v, v)) if t2 is None else t2.copy()
    diis = _DIIS()
    for it in range(1, max_iter + 1):
        r1, r2 = t_residuals(fock, chol, t1, t2, o)
        if max(np.abs(r1).max(), np.abs(r2).max()) <= tol:
            return t1, t2, correlation_energy(fock, chol, t1, t2, o), it
        x = np.concatenate([(t1 + r1 / D1).ravel(), _antisym(t2 + r2 / D2).ravel()])
        r = np.concatenate([(r1 / D1).ravel(), (r2 / D2).ravel()])
        x = diis.push(x, r)
        t1 = x[:o * v].reshape(o, v)
        t2 = x[o * v:].reshape(o, o, v, v)
    raise RuntimeError("CCSD did not converge")


# --------------------------------------------------------------------------------------------- Lambda
def lambda_elements(fock, chol, t1, t2, o):
    """Hbar elements of e^-T2 H' e^T2 (T1 = 0 forms in the rotated basis) used by the Lambda equations,
    as a dict of arrays with the index order of their names."""
    ints = Integrals(fock, chol, t1, o)
    f = ints.fblk
    e = ints.eri
    oovv = e("oovv")
    E = {"oovv": oovv}
    E["Fov"] = f("ov").copy()
    E["Foo"] = f("oo") + 0.5 * np.einsum("mnef,inef->mi", oovv, t2, optimize=True)                  # Fb_mi
    E["Fvv"] = f("vv") - 0.5 * np.einsum("mnef,mnaf->ae", oovv, t2, optimize=True)                  # Fb_ae
    E["Woooo"] = e("oooo") + 0.5 * np.einsum("mnef,ijef->mnij", oovv, t2, optimize=True)            # Wb_mnij
    E["Wvvvv"] = e("vvvv") + 0.5 * np.einsum("mnef,mnab->abef", oovv, t2, optimize=True)            # Wb_abef
    E["Wovvo"] = e("ovvo") - np.einsum("mnef,jnfb->mbej", oovv, t2, optimize=True)                  # Wb_mbej
    E["Wooov"] = e("ooov")                                                                          # Wb_mnie
    E["Wvovv"] = e("vovv")                                                                          # Wb_amef
    tmp = np.einsum("mnie,jnbe->mbij", e("ooov"), t2, optimize=True)
    E["Wovoo"] = (e("ovoo") - np.einsum("me,ijbe->mbij", E["Fov"], t2, optimize=True)               # Wb_mbij
                  + 0.5 * np.einsum("mbef,ijef->mbij", e("ovvv"), t2, optimize=True) + tmp - tmp.transpose(0, 1, 3, 2))
    tmp = np.einsum("mbef,miaf->abei", e("ovvv"), t2, optimize=True)
    E["Wvvvo"] = (e("vvvo") - np.einsum("me,miab->abei", E["Fov"], t2, optimize=True)               # Wb_abei
                  + 0.5 * np.einsum("mnei,mnab->abei", e("oovo"), t2, optimize=True) - tmp + tmp.transpose(1, 0, 2, 3))
    return E


def lambda_residuals(E, t2, l1, l2):
    """(R1 [o][v], R2 [o][o][v][v]) of the Lambda-CCSD equations at (l1, l2) = (lam_ia, lam_ijab)."""
    oovv = E["oovv"]
    Fov, Foo, Fvv = E["Fov"], E["Foo"], E["Fvv"]
    Gvv = -0.5 * np.einsum("mnef,mnaf->ae", t2, l2, optimize=True)     # G_ae
    Goo = 0.5 * np.einsum("mnef,inef->mi", t2, l2, optimize=True)      # G_mi
    # Hbar elements in the index orders the equations name (all from the operator's blocks)
    W_ieam = E["Wovvo"].transpose(0, 1, 2, 3)     # Wb_ieam = Wb_mbej with (m, b, e, j) -> (i, e, a, m)
    W_efam = E["Wvvvo"]                            # Wb_efam = Wb_abei with (a, b, e, i) -> (e, f, a, m)
    W_iemn = E["Wovoo"]                            # Wb_iemn = Wb_mbij with (m, b, i, j) -> (i, e, m, n)
    W_eifa = E["Wvovv"]                            # Wb_eifa = Wb_amef with (a, m, e, f) -> (e, i, f, a)
    W_mina = E["Wooov"]                            # Wb_mina = Wb_mnie with (m, n, i, e) -> (m, i, n, a)
    r1 = (Fov.copy()
          + np.einsum("ie,ea->ia", l1, Fvv, optimize=True)
          - np.einsum("ma,im->ia", l1, Foo, optimize=True)
          + np.einsum("me,ieam->ia", l1, W_ieam, optimize=True)
          + 0.5 * np.einsum("imef,efam->ia", l2, W_efam, optimize=True)
          - 0.5 * np.einsum("mnae,iemn->ia", l2, W_iemn, optimize=True)
          - np.einsum("ef,eifa->ia", Gvv, W_eifa, optimize=True)
          - np.einsum("mn,mina->ia", Goo, W_mina, optimize=True))
    r2 = oovv.copy()
    r2 += _P(np.einsum("ijae,eb->ijab", l2, Fvv, optimize=True), (2, 3))
    r2 -= _P(np.einsum("imab,jm->ijab", l2, Foo, optimize=True), (0, 1))
    r2 += 0.5 * np.einsum("mnab,ijmn->ijab", l2, E["Woooo"], optimize=True)
    r2 += 0.5 * np.einsum("ijef,efab->ijab", l2, E["Wvvvv"], optimize=True)
    r2 += _P(np.einsum("ie,ejab->ijab", l1, E["Wvovv"], optimize=True), (0, 1))     # Wb_ejab = Wb_amef
    r2 -= _P(np.einsum("ma,ijmb->ijab", l1, E["Wooov"], optimize=True), (2, 3))     # Wb_ijmb = Wb_mnie
    ring = np.einsum("imae,jebm->ijab", l2, E["Wovvo"], optimize=True)              # Wb_jebm = Wb_mbej
    r2 += ring - ring.transpose(1, 0, 2, 3) - ring.transpose(0, 1, 3, 2) + ring.transpose(1, 0, 3, 2)
    fr = np.einsum("ia,jb->ijab", l1, Fov, optimize=True)
    r2 += fr - fr.transpose(1, 0, 2, 3) - fr.transpose(0, 1, 3, 2) + fr.transpose(1, 0, 3, 2)
    r2 += _P(np.einsum("ijae,be->ijab", oovv, Gvv, optimize=True), (2, 3))
    r2 -= _P(np.einsum("imab,mj->ijab", oovv, Goo, optimize=True), (0, 1))
    return r1, r2


def solve_lambda(fock, chol, t1, t2, o, tol=1e-10, max_iter=200):
    """Converged (lam1 [o][v] = lambda_a^i, lam2 [o][o][v][v] = lambda_ab^ij, iterations)."""
    E = lambda_elements(fock, chol, t1, t2, o)
    D1, D2 = denominators(fock, o)
    l1, l2 = t1.copy(), t2.copy()
    diis = _DIIS()
    o_, v = t1.shape
    for it in range(1, max_iter + 1):
        r1, r2 = lambda_residuals(E, t2, l1, l2)
        if max(np.abs(r1).max(), np.abs(r2).max()) <= tol:
            return l1, l2, it
        x = np.concatenate([(l1 + r1 / D1).ravel(), _antisym(l2 + r2 / D2).ravel()])
        r = np.concatenate([(r1 / D1).ravel(), (r2 / D2).ravel()])
        x = diis.push(x, r)
        l1 = x[:o_ * v].reshape(o_, v)
        l2 = x[o_ * v:].reshape(o_, o_, v, v)
    raise RuntimeError("Lambda-CCSD did not converge")
