"""Seeded synthetic GFCCSD inputs shared by the CUDA path, the oracle and the bench.

This module holds random-number generation and the workload recipes only; it
contains none of the method's arithmetic (no integrals transformation, no
similarity transformation, no linear algebra).

Generator: counter-based splitmix64 (Steele, Lea & Flood, OOPSLA 2014), one
independent stream per tensor.  Draw k of stream s with seed S is
``mix64(key(S, s) + (k + 1) * 0x9E3779B97F4A7C15)``; uniforms take the top 53
bits, normals come from the Box-Muller transform of consecutive uniform pairs.
Because every element is a pure function of (seed, stream, index), the tensors
can be generated in any order and in parallel chunks.

Workload recipes (the five workloads of the hot path):
  * occupied energies eps ~ U(-1.5, -0.3), virtual eps ~ U(0.1, 2.0) Hartree,
    each block sorted ascending; the Fock matrix is diag(eps), occupied first.
  * Cholesky vectors L[K][p][q] = L[K][q][p] ~ N(0, sigma_L^2) * exp(-K/12),
    K = 0..L-1; sigma_L = (o*v)^(-1/2) unless given (the Gaussian width is not
    fixed by the workload description; this width puts the leading eigenvalue
    of the (ov|ov) block near 1 Hartree).
  * t1[i][a] ~ N(0, 0.01^2); t2[i][j][a][b] antisymmetric in (i,j) and in
    (a,b), each independent element (i<j, a<b) ~ N(0, 0.02^2).
  * Lambda = T^dagger (lambda_a^i = t_i^a, lambda_ab^ij = t_ij^ab).
"""
from __future__ import annotations

import dataclasses
import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STREAM_EPS_OCC = 1
STREAM_EPS_VIR = 2
STREAM_CHOL = 3
STREAM_T1 = 4
STREAM_T2 = 5
STREAM_LAMBDA1 = 6
STREAM_LAMBDA2 = 7
STREAM_VECTOR = 8
STREAM_MLP_W1 = 101
STREAM_MLP_W2 = 102
STREAM_MLP_W3 = 103

_CHUNK = 1 << 22


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        z = np.array([(int(seed) * 0x2545F4914F6CDD1D + int(stream) * 0x9E3779B97F4A7C15)
                      & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        return _mix64(z)[0]


def _uniform_chunk(key: np.uint64, start: int, count: int) -> np.ndarray:
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _mix64(key + k * _GAMMA)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _parallel_fill(out: np.ndarray, fn) -> None:
    total = out.size
    flat = out.reshape(-1)
    starts = list(range(0, total, _CHUNK))
    if len(starts) <= 1:
        if total:
            flat[:] = fn(0, total)
        return

    def work(s):
        c = min(_CHUNK, total - s)
        flat[s:s + c] = fn(s, c)

    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        list(ex.map(work, starts))


def uniform(seed: int, stream: int, count: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """count uniforms in [lo, hi) from stream `stream` of `seed`."""
    key = _stream_key(seed, stream)
    out = np.empty(count, dtype=np.float64)
    _parallel_fill(out, lambda s, c: lo + (hi - lo) * _uniform_chunk(key, s, c))
    return out


def normal(seed: int, stream: int, count: int, std: float = 1.0) -> np.ndarray:
    """count N(0, std^2) draws: Box-Muller on uniform pairs (2k, 2k+1)."""
    key = _stream_key(seed, stream)
    out = np.empty(count, dtype=np.float64)

    def fn(s, c):
        # element e uses the uniform pair of index e // 2 (cos for even e, sin for odd e)
        first_pair = s // 2
        last_pair = (s + c - 1) // 2
        npair = last_pair - first_pair + 1
        u = _uniform_chunk(key, 2 * first_pair, 2 * npair).reshape(npair, 2)
        rad = np.sqrt(-2.0 * np.log1p(-u[:, 0]))  # 1 - u in (0, 1]
        ang = (2.0 * math.pi) * u[:, 1]
        z = np.empty((npair, 2))
        z[:, 0] = rad * np.cos(ang)
        z[:, 1] = rad * np.sin(ang)
        off = s - 2 * first_pair
        return std * z.reshape(-1)[off:off + c]

    _parallel_fill(out, fn)
    return out


@dataclasses.dataclass
class Problem:
    """Host-side inputs of gfcc_create (all float64, C-contiguous)."""
    o: int
    v: int
    L: int
    fock: np.ndarray      # (n, n), diagonal
    chol: np.ndarray      # (L, n, n), symmetric in the last two indices
    t1: np.ndarray        # (o, v)
    t2: np.ndarray        # (o, o, v, v)
    lam1: np.ndarray | None = None   # (o, v) [i][a]; None means Lambda = T^dagger
    lam2: np.ndarray | None = None   # (o, o, v, v) [i][j][a][b]

    @property
    def n(self) -> int:
        return self.o + self.v

    def lambdas(self):
        if self.lam1 is None:
            return self.t1, self.t2
        return self.lam1, self.lam2

    def eps(self) -> np.ndarray:
        return np.diag(self.fock).copy()


def _antisym_pairs(n: int) -> tuple[np.ndarray, np.ndarray]:
    i, j = np.triu_indices(n, 1)
    return i, j


def antisym_tensor(packed: np.ndarray, o: int, v: int) -> np.ndarray:
    """Expand packed (i<j, a<b) values into t[i][j][a][b], antisymmetric in both pairs."""
    t = np.zeros((o, o, v, v))
    if o < 2 or v < 2:
        return t
    ii, jj = _antisym_pairs(o)
    aa, bb = _antisym_pairs(v)
    p = packed.reshape(len(ii), len(aa))
    t[ii[:, None], jj[:, None], aa[None, :], bb[None, :]] = p
    t[jj[:, None], ii[:, None], aa[None, :], bb[None, :]] = -p
    t[ii[:, None], jj[:, None], bb[None, :], aa[None, :]] = -p
    t[jj[:, None], ii[:, None], bb[None, :], aa[None, :]] = p
    return t


def make_problem(o: int, v: int, L: int, seed: int = 0, *, chol_sigma: float | None = None,
                 t1_std: float = 0.01, t2_std: float = 0.02, chol_decay: float = 12.0,
                 eps_occ=(-1.5, -0.3), eps_vir=(0.1, 2.0), with_t: bool = True,
                 separate_lambda: bool = False, lambda_std: tuple[float, float] | None = None) -> Problem:
    """Synthetic GFCCSD inputs with the workload recipe of the module docstring.

    with_t=False gives T = Lambda = 0.  separate_lambda=True draws Lambda from its
    own streams (same widths as T unless lambda_std is given) instead of T^dagger.
    """
    n = o + v
    eo = np.sort(uniform(seed, STREAM_EPS_OCC, o, *eps_occ))
    ev = np.sort(uniform(seed, STREAM_EPS_VIR, v, *eps_vir))
    fock = np.diag(np.concatenate([eo, ev]))
    sig = (1.0 / math.sqrt(o * v)) if chol_sigma is None else float(chol_sigma)
    npq = n * (n + 1) // 2
    raw = normal(seed, STREAM_CHOL, L * npq, sig).reshape(L, npq)
    raw *= np.exp(-np.arange(L, dtype=np.float64) / chol_decay)[:, None]
    chol = np.empty((L, n, n))
    iu, ju = np.triu_indices(n)
    chol[:, iu, ju] = raw
    chol[:, ju, iu] = raw
    del raw
    if with_t:
        t1 = normal(seed, STREAM_T1, o * v, t1_std).reshape(o, v)
        npk = (o * (o - 1) // 2) * (v * (v - 1) // 2)
        t2 = antisym_tensor(normal(seed, STREAM_T2, npk, t2_std), o, v)
    else:
        t1 = np.zeros((o, v))
        t2 = np.zeros((o, o, v, v))
    lam1 = lam2 = None
    if separate_lambda:
        s1, s2 = lambda_std if lambda_std is not None else (t1_std, t2_std)
        lam1 = normal(seed, STREAM_LAMBDA1, o * v, s1).reshape(o, v)
        npk = (o * (o - 1) // 2) * (v * (v - 1) // 2)
        lam2 = antisym_tensor(normal(seed, STREAM_LAMBDA2, npk, s2), o, v)
    return Problem(o=o, v=v, L=L, fock=fock, chol=chol, t1=t1, t2=t2, lam1=lam1, lam2=lam2)


def make_closed_shell_problem(o: int, v: int, L: int, seed: int = 0, *, chol_sigma: float | None = None,
                              t1_std: float = 0.01, t2_std: float = 0.02, separate_lambda: bool = False) -> Problem:
    """Closed-shell synthetic inputs over spatial orbitals (o doubly occupied, v virtual): Fock matrix
    and Cholesky vectors by the recipe of make_problem (sigma_L = (2o * 2v)^(-1/2) unless given, the
    width of the spin-orbital problem of the same system); t1[i][a] ~ N(0, t1_std^2) (alpha block);
    t2[i][j][a][b] = (g[i][j][a][b] + g[j][i][b][a]) / 2 with g ~ N(0, t2_std^2), so that
    t_ij^ab = t_ji^ba (the alpha-beta block of a spin-adapted T2).  Lambda = T^dagger unless
    separate_lambda (its own streams, same widths and symmetry)."""
    sig = (1.0 / math.sqrt(4 * o * v)) if chol_sigma is None else float(chol_sigma)
    base = make_problem(o, v, L, seed=seed, chol_sigma=sig, with_t=False)
    t1 = normal(seed, STREAM_T1, o * v, t1_std).reshape(o, v)
    g = normal(seed, STREAM_T2, o * o * v * v, t2_std).reshape(o, o, v, v)
    t2 = 0.5 * (g + g.transpose(1, 0, 3, 2))
    lam1 = lam2 = None
    if separate_lambda:
        lam1 = normal(seed, STREAM_LAMBDA1, o * v, t1_std).reshape(o, v)
        h = normal(seed, STREAM_LAMBDA2, o * o * v * v, t2_std).reshape(o, o, v, v)
        lam2 = 0.5 * (h + h.transpose(1, 0, 3, 2))
    return Problem(o=o, v=v, L=L, fock=base.fock, chol=base.chol, t1=t1, t2=np.ascontiguousarray(t2), lam1=lam1,
                   lam2=None if lam2 is None else np.ascontiguousarray(lam2))


def random_vector(seed: int, count: int, stream_offset: int = 0) -> np.ndarray:
    """count N(0,1) draws for test vectors (a stream separate from the problem tensors)."""
    return normal(seed, STREAM_VECTOR + 16 * stream_offset, count)


# --------------------------------------------------------------------------------------------
# Workload recipes
# --------------------------------------------------------------------------------------------


def mlp_init_params(hidden: int, seed: int, nin: int = 27, nout: int = 16) -> np.ndarray:
    """Initial parameters of the guess model in its flat layout W1 b1 W2 b2 W3 b3 mu sd: He-scaled
    normal weights (std sqrt(2 / fan_in); the output layer 0.1 sqrt(1 / hidden)), zero biases,
    mu = 0, sd = 1."""
    W1 = normal(seed, STREAM_MLP_W1, hidden * nin, math.sqrt(2.0 / nin))
    W2 = normal(seed, STREAM_MLP_W2, hidden * hidden, math.sqrt(2.0 / hidden))
    W3 = normal(seed, STREAM_MLP_W3, nout * hidden, 0.1 * math.sqrt(1.0 / hidden))
    return np.concatenate([W1, np.zeros(hidden), W2, np.zeros(hidden), W3, np.zeros(nout), np.zeros(nin),
                           np.ones(nin)])


@dataclasses.dataclass
class Workload:
    name: str
    o: int
    v: int
    L: int
    omegas: np.ndarray
    eta: float
    orbitals: np.ndarray
    tol: float
    restart: int
    sectors: str            # "IP", "EA" or "IP+EA"
    seed: int = 0
    precision: str = "fp64"
    closed_shell: bool = False   # spatial orbitals (make_closed_shell_problem)

    def problem(self, **kw) -> Problem:
        if self.closed_shell:
            return make_closed_shell_problem(self.o, self.v, self.L, self.seed, **kw)
        return make_problem(self.o, self.v, self.L, self.seed, **kw)


def orbitals_nearest_gap(eps_o: np.ndarray, eps_v: np.ndarray, count: int) -> np.ndarray:
    """Indices of the `count` orbitals with the smallest |eps_p - mid-gap| (ties: lower index)."""
    eps = np.concatenate([eps_o, eps_v])
    mid = 0.5 * (eps_o.max() + eps_v.min())
    order = sorted(range(len(eps)), key=lambda p: (abs(eps[p] - mid), p))
    return np.array(sorted(order[:count]), dtype=np.int32)


def workload(name: str) -> Workload:
    """The named workload.  'tiny' (o=4 v=12 L=48), 'medium' (o=40 v=200 L=800),
    'c60' (o=90 v=450 L=1800, 128 frequencies), 'c60x256' (the same problem, 256 frequencies),
    closed-shell (spatial orbitals): 'medium-closed-shell' (o=30 v=150 L=600),
    'c60-closed-shell' (o=45 v=225 L=1800)."""
    if name == "tiny":
        return Workload("tiny", 4, 12, 48, np.linspace(-1.0, -0.2, 4), 0.01,
                        np.arange(16, dtype=np.int32), 1e-8, 30, "IP")
    if name == "medium":
        o, v = 40, 200
        eo = np.sort(uniform(0, STREAM_EPS_OCC, o, -1.5, -0.3))
        ev = np.sort(uniform(0, STREAM_EPS_VIR, v, 0.1, 2.0))
        return Workload("medium", o, v, 800, np.linspace(-1.2, 0.5, 64), 0.005,
                        orbitals_nearest_gap(eo, ev, 40), 1e-8, 30, "IP+EA")
    if name == "c60":
        o, v = 90, 450
        return Workload("c60", o, v, 1800, np.linspace(-1.0, -0.3, 128), 0.005,
                        np.arange(o - 30, o, dtype=np.int32), 1e-8, 30, "IP", precision="mixed")
    if name == "c60x256":
        # the C60-shaped problem on the denser grid of the learned-guess workload: 256 frequencies
        o, v = 90, 450
        return Workload("c60x256", o, v, 1800, np.linspace(-1.0, -0.3, 256), 0.005,
                        np.arange(o - 30, o, dtype=np.int32), 1e-8, 30, "IP", precision="mixed")
    if name == "c60x1024":
        # the C60-shaped problem on a grid 4x denser than c60x256 (spacing 0.14 eta): how dense a grid
        # the neighbour guesses need
        o, v = 90, 450
        return Workload("c60x1024", o, v, 1800, np.linspace(-1.0, -0.3, 1024), 0.005,
                        np.arange(o - 30, o, dtype=np.int32), 1e-8, 30, "IP", precision="mixed")
    if name == "c60-closed-shell":
        # the C60-shaped system as a closed shell: 45 doubly occupied and 225 virtual spatial orbitals
        # (the 90 / 450 spin-orbitals of 'c60'), the 30 highest occupied orbitals, spin-adapted IP
        o, v = 45, 225
        return Workload("c60-closed-shell", o, v, 1800, np.linspace(-1.0, -0.3, 128), 0.005,
                        np.arange(o - 30, o, dtype=np.int32), 1e-8, 30, "IP", closed_shell=True)
    if name == "medium-closed-shell":
        # 30 doubly occupied and 150 virtual spatial orbitals (the 60 / 300 spin-orbitals of a
        # medium-sized system), the 10 highest occupied orbitals, spin-adapted IP
        o, v = 30, 150
        return Workload("medium-closed-shell", o, v, 600, np.linspace(-1.2, -0.2, 64), 0.005,
                        np.arange(o - 10, o, dtype=np.int32), 1e-8, 30, "IP", closed_shell=True)
    raise KeyError(name)
