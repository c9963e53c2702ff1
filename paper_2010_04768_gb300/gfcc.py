"""ctypes binding of libgfcc.so (argument marshalling only; all arithmetic runs in the CUDA library).

The names follow the C ABI of include/gfcc.h.  The library is loaded from the
package's lib/ directory; if it is missing, every entry point raises instead of
falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libgfcc.so")

OK = 0
WARN_NOT_CONVERGED = 1
ERR_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_STATE = -1, -2, -3, -4, -5

SECTOR_IP, SECTOR_EA, SECTOR_BOTH = 1, 2, 3
PREC_FP64, PREC_MIXED_BF16, PREC_FP64_EMULATED = 0, 1, 2
PRECOND_NONE, PRECOND_DIAG = 0, 1
OPT_SECTOR, OPT_PRECISION, OPT_RESTART, OPT_MAX_ITERS, OPT_PRECOND, OPT_BATCH, OPT_INNER_TOL = 1, 2, 3, 4, 5, 6, 7
OPT_RESIDUAL, OPT_INNER_CYCLES, OPT_EMU_LEVEL = 8, 9, 10
OPT_GUESS, OPT_KEEP_SOLUTIONS, OPT_INNER_KRYLOV, OPT_AUTOTUNE, OPT_GRAPHS, OPT_EMU_FUSED_N = 11, 12, 13, 14, 15, 16
OPT_INCREMENTAL, OPT_INNER_RESTART = 17, 18
OPT_SETUP_EMULATE_FLOPS, OPT_WAIT_NS, OPT_TEST_NO_LOADS, OPT_GEMM_PAIR, OPT_GEMM_PERSIST = 19, 20, 21, 22, 23
OPT_CLOSED_SHELL_EMULATE = 24
GUESS_ZERO, GUESS_LEARNED, GUESS_MINRES = 0, 1, 2
MLP_FP32, MLP_FP64 = 0, 1
MLP_FEATURES, MLP_OUTPUTS = 27, 16

_SECTORS = {"IP": SECTOR_IP, "EA": SECTOR_EA, "IP+EA": SECTOR_BOTH, "BOTH": SECTOR_BOTH}
_PRECS = {"fp64": PREC_FP64, "mixed": PREC_MIXED_BF16, "bf16": PREC_MIXED_BF16, "fp64emu": PREC_FP64_EMULATED}

_lib = None


class _Request(ctypes.Structure):
    _fields_ = [("n_omega", ctypes.c_int), ("omegas", ctypes.POINTER(ctypes.c_double)), ("eta", ctypes.c_double),
                ("n_orb", ctypes.c_int), ("orbitals", ctypes.POINTER(ctypes.c_int)), ("tol", ctypes.c_double),
                ("G", ctypes.POINTER(ctypes.c_double))]


class GFCCError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libgfcc error {code}: {msg}")
        self.code = code


def load():
    """Load libgfcc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2010_04768_gb300/build.py "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.gfcc_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp, ctypes.POINTER(P)]
    lib.gfcc_create_ex.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp, ctypes.c_int,
                                   ctypes.c_int, ctypes.POINTER(P)]
    lib.gfcc_set_option.argtypes = [P, ctypes.c_int, ctypes.c_double]
    lib.gfcc_set_stream.argtypes = [P, P]
    lib.gfcc_solve.argtypes = [P, ctypes.c_int, dp, ctypes.c_double, ctypes.c_int, ip, ctypes.c_double, dp]
    lib.gfcc_solve_device.argtypes = [P, ctypes.c_int, P, ctypes.c_double, ctypes.c_int, P, ctypes.c_double, P]
    lib.gfcc_solve_block.argtypes = [P, ctypes.c_int, dp, ctypes.c_double, ctypes.c_int, ip, ctypes.c_int, ip,
                                     ctypes.c_double, dp]
    lib.gfcc_set_process_option.argtypes = [ctypes.c_int, ctypes.c_double]
    lib.gfcc_last_stats.argtypes = [P, ip, ip, dp, ip]
    lib.gfcc_sigma.argtypes = [P, ctypes.c_int, ctypes.c_int, dp, dp]
    lib.gfcc_sigma_ex.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]
    lib.gfcc_sigma_ex.restype = ctypes.c_int
    lib.gfcc_dims.argtypes = [P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
    lib.gfcc_profile.argtypes = [P, ctypes.c_int]
    lib.gfcc_profile_read.argtypes = [P, ctypes.c_int, dp, ctypes.POINTER(ctypes.c_longlong), dp]
    lib.gfcc_launch_count.restype = ctypes.c_longlong
    lib.gfcc_launch_count.argtypes = []
    lib.gfcc_sigma_noalloc.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P]
    lib.gfcc_sigma_noalloc.restype = ctypes.c_int
    fp = ctypes.POINTER(ctypes.c_float)
    lib.gfcc_selftest_gemm_bf16.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, fp, fp, fp]
    lib.gfcc_selftest_gemm_bf16.restype = ctypes.c_int
    lib.gfcc_selftest_gemm_f64emu.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int,
                                              ctypes.c_int, dp]
    lib.gfcc_selftest_gemm_f64emu.restype = ctypes.c_int
    lib.gfcc_destroy.argtypes = [P]
    lib.gfcc_destroy.restype = None
    lib.gfcc_guess_stats.argtypes = [P, ip, ip, dp, dp]
    lib.gfcc_set_guess_model.argtypes = [P, P]
    lib.gfcc_refine_stats.argtypes = [P, ip, ip]
    lib.gfcc_residual_stats.argtypes = [P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong), dp]
    lib.gfcc_solve_batch.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(_Request), ip]
    ull = ctypes.c_ulonglong
    lib.gfcc_mlp_create.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.POINTER(P)]
    lib.gfcc_mlp_destroy.argtypes = [P]
    lib.gfcc_mlp_destroy.restype = None
    lib.gfcc_mlp_num_params.argtypes = [P]
    lib.gfcc_mlp_num_params.restype = ctypes.c_longlong
    lib.gfcc_mlp_num_samples.argtypes = [P]
    lib.gfcc_mlp_num_samples.restype = ctypes.c_longlong
    lib.gfcc_mlp_get_params.argtypes = [P, dp]
    lib.gfcc_mlp_set_params.argtypes = [P, dp]
    lib.gfcc_mlp_forward.argtypes = [P, ctypes.c_int, dp, dp]
    lib.gfcc_mlp_loss_grad.argtypes = [P, ctypes.c_int, dp, dp, dp, dp]
    lib.gfcc_mlp_train_batch.argtypes = [P, ctypes.c_int, dp, dp, ctypes.c_double, dp]
    lib.gfcc_mlp_collect.argtypes = [P, P, ctypes.c_int, ull, ctypes.POINTER(ctypes.c_longlong)]
    lib.gfcc_mlp_train.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_double, ull, dp]
    lib.gfcc_mlp_eval.argtypes = [P, dp]
    lib.gfcc_mlp_get_samples.argtypes = [P, ctypes.c_longlong, ctypes.c_int, dp, dp]
    lib.gfcc_mor_create.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.POINTER(P)]
    lib.gfcc_mor_destroy.argtypes = [P]
    lib.gfcc_mor_destroy.restype = None
    lib.gfcc_mor_dim.argtypes = [P]
    lib.gfcc_mor_expand.argtypes = [P, ctypes.c_int, dp, ctypes.c_double, ctypes.c_int, ip, ctypes.c_double, dp]
    lib.gfcc_mor_green.argtypes = [P, ctypes.c_int, dp, ctypes.c_double, ctypes.c_int, ip, ctypes.c_int, ip, dp, dp]
    lib.gfcc_mor_projected.argtypes = [P, dp, dp, ctypes.c_int]
    lib.gfcc_spectral_adaptive.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int, ip, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_int, ctypes.c_int, dp, dp, ip, ip, dp, ctypes.c_int, ip]
    lib.gfcc_spectral_adaptive.restype = ctypes.c_int
    lib.gfcc_solve_checkpoint.argtypes = [P, ctypes.c_int, dp, ctypes.c_double, ctypes.c_int, ip, ctypes.c_double,
                                          ctypes.c_char_p, ip, dp]
    lib.gfcc_solve_checkpoint.restype = ctypes.c_int
    lib.gfcc_create_rhf.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp, ctypes.POINTER(P)]
    lib.gfcc_create_rhf.restype = ctypes.c_int
    lib.gfcc_ccsd.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_int,
                              ctypes.c_int, dp, dp, dp, dp]
    lib.gfcc_ccsd.restype = ctypes.c_int
    lib.gfcc_last_error.restype = ctypes.c_char_p
    for name in ("gfcc_create", "gfcc_create_ex", "gfcc_set_option", "gfcc_set_stream", "gfcc_solve",
                 "gfcc_solve_block", "gfcc_set_process_option",
                 "gfcc_solve_device", "gfcc_last_stats", "gfcc_sigma", "gfcc_dims", "gfcc_profile",
                 "gfcc_profile_read", "gfcc_guess_stats", "gfcc_set_guess_model", "gfcc_refine_stats",
                 "gfcc_residual_stats", "gfcc_solve_batch", "gfcc_mlp_create",
                 "gfcc_mlp_get_params", "gfcc_mlp_set_params", "gfcc_mlp_forward", "gfcc_mlp_loss_grad",
                 "gfcc_mlp_train_batch", "gfcc_mlp_collect", "gfcc_mlp_train", "gfcc_mlp_eval",
                 "gfcc_mlp_get_samples", "gfcc_mor_create", "gfcc_mor_dim", "gfcc_mor_expand", "gfcc_mor_green",
                 "gfcc_mor_projected"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def set_process_option(key: int, value: float):
    """gfcc_set_process_option: a process-wide option (applies to every context)."""
    _check(load().gfcc_set_process_option(int(key), float(value)))


def launch_count() -> int:
    """Kernels launched by libgfcc in this process."""
    return int(load().gfcc_launch_count())


def selftest_gemm_bf16(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """D = bf16(A) @ bf16(B).T with FP32 accumulation on the tensor cores (A: M x K, B: N x K)."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    M, K = A.shape
    N = B.shape[0]
    D = np.zeros((M, N), dtype=np.float32)
    fp = ctypes.POINTER(ctypes.c_float)
    _check(load().gfcc_selftest_gemm_bf16(M, N, K, A.ctypes.data_as(fp), B.ctypes.data_as(fp), D.ctypes.data_as(fp)))
    return D


def selftest_gemm_f64emu(A: np.ndarray, B: np.ndarray, S: int = 8, P: int = 9) -> np.ndarray:
    """C = A @ B.T (FP64 inputs) from BF16 digit planes on the tensor cores."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    M, K = A.shape
    N = B.shape[0]
    C = np.zeros((M, N), dtype=np.float64)
    _check(load().gfcc_selftest_gemm_f64emu(M, N, K, _dp(A), _dp(B), S, P, _dp(C)))
    return C


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(code):
    if code < 0:
        raise GFCCError(code, load().gfcc_last_error().decode())
    return code


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class GFCC:
    """One gfcc_ctx: the problem on the device with its Hbar elements."""

    def __init__(self, problem, sectors: str = "IP+EA", precision: str = "fp64", closed_shell: bool = False):
        """closed_shell=True: gfcc_create_rhf (spatial orbitals, spin-adapted IP; sectors "IP", FP64)."""
        lib = load()
        self.o, self.v, self.L = problem.o, problem.v, problem.L
        fock, chol, t1, t2 = (_f64(x) for x in (problem.fock, problem.chol, problem.t1, problem.t2))
        lam = None
        if problem.lam1 is not None:
            lam = np.concatenate([_f64(problem.lam1).reshape(-1), _f64(problem.lam2).reshape(-1)])
        h = ctypes.c_void_p()
        if closed_shell:
            if sectors != "IP" or precision != "fp64":
                raise ValueError("closed-shell contexts are IP-only and FP64")
            _check(lib.gfcc_create_rhf(self.o, self.v, self.L, _dp(fock), _dp(chol), _dp(t1), _dp(t2),
                                       None if lam is None else _dp(lam), ctypes.byref(h)))
        else:
            _check(lib.gfcc_create_ex(self.o, self.v, self.L, _dp(fock), _dp(chol), _dp(t1), _dp(t2),
                                      None if lam is None else _dp(lam), _SECTORS[sectors], _PRECS[precision],
                                      ctypes.byref(h)))
        self._h = h
        self.sectors = sectors

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().gfcc_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, key: int, value: float):
        _check(load().gfcc_set_option(self._h, key, float(value)))

    def set_stream(self, stream_handle: int | None):
        _check(load().gfcc_set_stream(self._h, ctypes.c_void_p(stream_handle or 0)))

    def dims(self):
        a, b = ctypes.c_longlong(), ctypes.c_longlong()
        _check(load().gfcc_dims(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def solve(self, omegas, eta: float, orbitals, tol: float):
        """G[w][p][q] (complex128) and the return code (0 or WARN_NOT_CONVERGED)."""
        om = _f64(omegas).reshape(-1)
        orb = np.ascontiguousarray(orbitals, dtype=np.int32).reshape(-1)
        G = np.zeros((om.size, orb.size, orb.size), dtype=np.complex128)
        code = _check(load().gfcc_solve(self._h, om.size, _dp(om), float(eta), orb.size,
                                        orb.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), float(tol),
                                        G.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return G, code

    def solve_checkpoint(self, omegas, eta: float, orbitals, tol: float, path: str):
        """gfcc_solve_checkpoint: (G, return code, frequencies restored from the file)."""
        om = _f64(omegas).reshape(-1)
        orb = np.ascontiguousarray(orbitals, dtype=np.int32).reshape(-1)
        G = np.zeros((om.size, orb.size, orb.size), dtype=np.complex128)
        nres = ctypes.c_int(0)
        ip = ctypes.POINTER(ctypes.c_int)
        code = _check(load().gfcc_solve_checkpoint(self._h, om.size, _dp(om), float(eta), orb.size,
                                                   orb.ctypes.data_as(ip), float(tol), str(path).encode(),
                                                   ctypes.byref(nres), G.view(np.float64).ctypes.data_as(
                                                       ctypes.POINTER(ctypes.c_double))))
        return G, code, nres.value

    def solve_block(self, omegas, eta: float, p_orbitals, q_orbitals, tol: float):
        """G[w][a][b] = G_{p_a q_b} (complex128) for rows p over p_orbitals and columns q over q_orbitals,
        and the return code."""
        om = _f64(omegas).reshape(-1)
        P = np.ascontiguousarray(p_orbitals, dtype=np.int32).reshape(-1)
        Q = np.ascontiguousarray(q_orbitals, dtype=np.int32).reshape(-1)
        G = np.zeros((om.size, P.size, Q.size), dtype=np.complex128)
        ip = ctypes.POINTER(ctypes.c_int)
        code = _check(load().gfcc_solve_block(self._h, om.size, _dp(om), float(eta), P.size, P.ctypes.data_as(ip),
                                              Q.size, Q.ctypes.data_as(ip), float(tol),
                                              G.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return G, code

    def solve_device(self, omegas_ptr: int, n_omega: int, eta: float, orbitals_ptr: int, n_orb: int, tol: float,
                     G_ptr: int):
        """gfcc_solve_device on caller-owned device buffers (e.g. torch tensors' data_ptr())."""
        return _check(load().gfcc_solve_device(self._h, n_omega, ctypes.c_void_p(omegas_ptr), float(eta), n_orb,
                                               ctypes.c_void_p(orbitals_ptr), float(tol), ctypes.c_void_p(G_ptr)))

    def stats(self):
        lib = load()
        cnt = ctypes.c_int(0)
        _check(lib.gfcc_last_stats(self._h, ctypes.byref(cnt), None, None, None))
        n = cnt.value
        it = np.zeros(n, dtype=np.int32)
        rr = np.zeros(n, dtype=np.float64)
        stt = np.zeros(n, dtype=np.int32)
        cnt = ctypes.c_int(n)
        _check(lib.gfcc_last_stats(self._h, ctypes.byref(cnt), it.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                   _dp(rr), stt.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
        return it, rr, stt

    def sigma_noalloc(self, sector: str, n_vec: int, x_ptr: int, y_ptr: int):
        """gfcc_sigma_noalloc on caller-owned device buffers (device pointers, packed complex128 vectors);
        the library allocates nothing during the call."""
        _check(load().gfcc_sigma_noalloc(self._h, _SECTORS[sector], n_vec, ctypes.c_void_p(x_ptr),
                                         ctypes.c_void_p(y_ptr)))

    def guess_stats(self):
        """(kind, predicted ||r0||^2/||b||^2, measured ||r0||/||b||) per statistics entry of the last solve."""
        lib = load()
        cnt = ctypes.c_int(0)
        _check(lib.gfcc_guess_stats(self._h, ctypes.byref(cnt), None, None, None))
        n = cnt.value
        kind = np.zeros(n, dtype=np.int32)
        pred = np.zeros(n, dtype=np.float64)
        rel0 = np.zeros(n, dtype=np.float64)
        cnt = ctypes.c_int(n)
        _check(lib.gfcc_guess_stats(self._h, ctypes.byref(cnt), kind.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                    _dp(pred), _dp(rel0)))
        return kind, pred, rel0

    def refine_stats(self) -> np.ndarray:
        """FP64-accurate residuals evaluated per statistics entry of the last solve (mixed precision)."""
        lib = load()
        cnt = ctypes.c_int(0)
        _check(lib.gfcc_refine_stats(self._h, ctypes.byref(cnt), None))
        out = np.zeros(cnt.value, dtype=np.int32)
        cnt = ctypes.c_int(out.size)
        _check(lib.gfcc_refine_stats(self._h, ctypes.byref(cnt), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
        return out

    def residual_stats(self) -> tuple[int, int, float]:
        """(full, incremental, mean digit level of the incremental) FP64-accurate residual products of
        the last solve."""
        full, inc, lvl = ctypes.c_longlong(0), ctypes.c_longlong(0), ctypes.c_double(0.0)
        _check(load().gfcc_residual_stats(self._h, ctypes.byref(full), ctypes.byref(inc), ctypes.byref(lvl)))
        return full.value, inc.value, lvl.value

    def set_guess_model(self, model: "MLP | None"):
        self._model = model   # keeps the model alive while attached
        _check(load().gfcc_set_guess_model(self._h, None if model is None else model.handle))

    PHASES = ("setup", "ring", "vvvv", "sigma", "arnoldi", "lsq", "overlap", "solve", "ring_bf16", "ring_emu",
              "unpack", "guess", "emu_other", "bf16_other", "epilogue", "ring_emu_work")

    def profile(self, enable: bool = True):
        _check(load().gfcc_profile(self._h, 1 if enable else 0))

    def profile_read(self) -> dict:
        """{phase: (ms, count, flops)} for every profiling phase."""
        out = {}
        for k, name in enumerate(self.PHASES):
            ms, n, fl = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double()
            _check(load().gfcc_profile_read(self._h, k, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(fl)))
            out[name] = (ms.value, n.value, fl.value)
        return out

    def sigma(self, sector: str, X: np.ndarray, precision: str = "fp64") -> np.ndarray:
        """sigma(x) for packed complex vectors X[n_vec][dim]."""
        X = np.ascontiguousarray(np.atleast_2d(X), dtype=np.complex128)
        Y = np.zeros_like(X)
        _check(load().gfcc_sigma_ex(self._h, _SECTORS[sector], _PRECS[precision], X.shape[0],
                                    X.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    Y.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return Y


def solve_batch(ctxs, requests):
    """gfcc_solve_batch: requests[i] = (omegas, eta, orbitals, tol) for context ctxs[i]; returns the G
    arrays and the per-context return codes."""
    n = len(ctxs)
    keep = []
    reqs = (_Request * n)()
    Gs = []
    for i, (om, eta, orb, tol) in enumerate(requests):
        om = _f64(om).reshape(-1)
        orb = np.ascontiguousarray(orb, dtype=np.int32).reshape(-1)
        G = np.zeros((om.size, orb.size, orb.size), dtype=np.complex128)
        keep += [om, orb]
        Gs.append(G)
        reqs[i] = _Request(om.size, _dp(om), float(eta), orb.size, orb.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                           float(tol), G.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    hs = (ctypes.c_void_p * n)(*[c.handle.value for c in ctxs])
    codes = np.zeros(n, dtype=np.int32)
    _check(load().gfcc_solve_batch(hs, n, reqs, codes.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
    return Gs, codes


class MLP:
    """One gfcc_mlp: the learned initial-guess model (3-layer perceptron, trained with Adam on the
    Gram-matrix loss of the kept solutions)."""

    def __init__(self, init_params: np.ndarray, hidden: int = 256, precision: int = MLP_FP32):
        lib = load()
        p = _f64(init_params).reshape(-1)
        h = ctypes.c_void_p()
        _check(lib.gfcc_mlp_create(int(hidden), int(precision), _dp(p), ctypes.byref(h)))
        self._h = h
        self.hidden = hidden
        self.precision = precision

    @staticmethod
    def num_params_for(hidden: int) -> int:
        return hidden * MLP_FEATURES + hidden + hidden * hidden + hidden + MLP_OUTPUTS * hidden + MLP_OUTPUTS + \
            2 * MLP_FEATURES

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().gfcc_mlp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def num_params(self) -> int:
        return int(load().gfcc_mlp_num_params(self._h))

    def num_samples(self) -> int:
        return int(load().gfcc_mlp_num_samples(self._h))

    def get_params(self) -> np.ndarray:
        p = np.zeros(self.num_params())
        _check(load().gfcc_mlp_get_params(self._h, _dp(p)))
        return p

    def set_params(self, p: np.ndarray):
        p = _f64(p).reshape(-1)
        assert p.size == self.num_params()
        _check(load().gfcc_mlp_set_params(self._h, _dp(p)))

    def forward(self, features: np.ndarray) -> np.ndarray:
        F = _f64(np.atleast_2d(features))
        y = np.zeros((F.shape[0], MLP_OUTPUTS))
        _check(load().gfcc_mlp_forward(self._h, F.shape[0], _dp(F), _dp(y)))
        return y

    def loss_grad(self, features: np.ndarray, gram: np.ndarray):
        F = _f64(np.atleast_2d(features))
        Gm = np.ascontiguousarray(gram, dtype=np.complex128).reshape(F.shape[0], 9, 9)
        loss = ctypes.c_double()
        g = np.zeros(self.num_params())
        _check(load().gfcc_mlp_loss_grad(self._h, F.shape[0], _dp(F), Gm.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         ctypes.byref(loss), _dp(g)))
        return loss.value, g

    def train_batch(self, features: np.ndarray, gram: np.ndarray, lr: float) -> float:
        F = _f64(np.atleast_2d(features))
        Gm = np.ascontiguousarray(gram, dtype=np.complex128).reshape(F.shape[0], 9, 9)
        loss = ctypes.c_double()
        _check(load().gfcc_mlp_train_batch(self._h, F.shape[0], _dp(F),
                                           Gm.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(lr),
                                           ctypes.byref(loss)))
        return loss.value

    def collect(self, ctx: GFCC, samples_per_system: int = 2, seed: int = 0) -> int:
        added = ctypes.c_longlong()
        _check(load().gfcc_mlp_collect(self._h, ctx.handle, int(samples_per_system), int(seed), ctypes.byref(added)))
        return added.value

    def samples(self, start: int = 0, count: int | None = None):
        """(features [count][27], Gram matrices [count][9][9] complex) of collected samples."""
        count = self.num_samples() - start if count is None else count
        F = np.zeros((count, MLP_FEATURES))
        Gm = np.zeros((count, 9, 9), dtype=np.complex128)
        _check(load().gfcc_mlp_get_samples(self._h, int(start), int(count), _dp(F),
                                           Gm.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return F, Gm

    def train(self, steps: int, minibatch: int = 256, lr: float = 1e-3, seed: int = 0) -> float:
        loss = ctypes.c_double()
        _check(load().gfcc_mlp_train(self._h, int(steps), int(minibatch), float(lr), int(seed), ctypes.byref(loss)))
        return loss.value

    def eval(self) -> dict:
        out = np.zeros(4)
        _check(load().gfcc_mlp_eval(self._h, _dp(out)))
        return {"loss": out[0], "loss_fallback": out[1], "loss_minres": out[2], "frac_better_than_zero": out[3]}


class MOR:
    """One gfcc_mor: the model-order reduction of one sector of a context (eq. model)."""

    def __init__(self, ctx: GFCC, sector: str = "IP", drop_tol: float = 1e-10):
        h = ctypes.c_void_p()
        _check(load().gfcc_mor_create(ctx.handle, _SECTORS[sector], float(drop_tol), ctypes.byref(h)))
        self._h = h
        self._ctx = ctx   # the context outlives the object
        self.sector = sector

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().gfcc_mor_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def dim(self) -> int:
        return int(load().gfcc_mor_dim(self._h))

    def expand(self, omegas, eta: float, orbitals, tol: float):
        """Solve the full systems and add their solutions to the subspace; (G of those systems, code)."""
        om = _f64(omegas).reshape(-1)
        orb = np.ascontiguousarray(orbitals, dtype=np.int32).reshape(-1)
        G = np.zeros((om.size, orb.size, orb.size), dtype=np.complex128)
        code = _check(load().gfcc_mor_expand(self._h, om.size, _dp(om), float(eta), orb.size,
                                             orb.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), float(tol),
                                             G.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return G, code

    def green(self, omegas, eta: float, p_orbitals, q_orbitals=None, residuals: bool = False):
        """Model G[w][a][b] (rows p, columns q) and, with residuals=True, the model solutions' relative
        full-space residuals."""
        om = _f64(omegas).reshape(-1)
        P = np.ascontiguousarray(p_orbitals, dtype=np.int32).reshape(-1)
        Q = P if q_orbitals is None else np.ascontiguousarray(q_orbitals, dtype=np.int32).reshape(-1)
        G = np.zeros((om.size, P.size, Q.size), dtype=np.complex128)
        rr = np.zeros((om.size, P.size if self.sector == "IP" else Q.size)) if residuals else None
        ip = ctypes.POINTER(ctypes.c_int)
        _check(load().gfcc_mor_green(self._h, om.size, _dp(om), float(eta), P.size, P.ctypes.data_as(ip), Q.size,
                                     Q.ctypes.data_as(ip), G.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     _dp(rr) if rr is not None else None))
        return (G, rr) if residuals else G

    def projected(self, rows: int = 0):
        """(Hhat m x m, the first `rows` basis vectors)."""
        m = self.dim()
        H = np.zeros((m, m))
        _, de = self._ctx.dims()
        di, _ = self._ctx.dims()
        n = di if self.sector == "IP" else de
        S = np.zeros((min(rows, m), n)) if rows > 0 else None
        _check(load().gfcc_mor_projected(self._h, _dp(H), _dp(S) if S is not None else None, int(min(rows, m))))
        return H, S


def spectral_adaptive(ctx: GFCC, sectors: str, omega_min: float, omega_max: float, d_omega: float, eta: float,
                      orbitals, tol: float, level_tol: float, fine_omegas, max_levels: int = 30):
    """gfcc_spectral_adaptive: (A on fine_omegas, levels [list of frequency lists], (m_IP, m_EA), code)."""
    orb = np.ascontiguousarray(orbitals, dtype=np.int32).reshape(-1)
    fine = _f64(fine_omegas).reshape(-1)
    A = np.zeros(fine.size)
    nlev = ctypes.c_int(0)
    sizes = np.zeros(max_levels, dtype=np.int32)
    cap = 4096
    samp = np.zeros(cap)
    mdim = np.zeros(2, dtype=np.int32)
    ip = ctypes.POINTER(ctypes.c_int)
    code = _check(load().gfcc_spectral_adaptive(ctx.handle, _SECTORS[sectors], float(omega_min), float(omega_max),
                                                float(d_omega), float(eta), orb.size, orb.ctypes.data_as(ip),
                                                float(tol), float(level_tol), int(max_levels), fine.size, _dp(fine),
                                                _dp(A), ctypes.byref(nlev), sizes.ctypes.data_as(ip), _dp(samp), cap,
                                                mdim.ctypes.data_as(ip)))
    levels, k = [], 0
    for L in range(nlev.value):
        levels.append(list(samp[k:k + sizes[L]]))
        k += sizes[L]
    return A, levels, (int(mdim[0]), int(mdim[1])), code


CCSD_EMULATE, CCSD_GUESS = 1, 2


def ccsd(fock, chol, o: int, tol: float = 1e-10, max_iter: int = 100, want_lambda: bool = True,
         emulate: bool = False, guess=None):
    """gfcc_ccsd: (t1, t2, lam1, lam2, info, code) for the Hamiltonian (fock, chol) with o occupied
    orbitals.  guess = (t1, t2[, lam1, lam2]) starts from those iterates; lam1 / lam2 are None when
    want_lambda is False.  info: dict of the call's info array."""
    fock = _f64(fock)
    chol = _f64(chol)
    n = fock.shape[0]
    L = chol.shape[0]
    v = n - o
    flags = (CCSD_EMULATE if emulate else 0) | (CCSD_GUESS if guess is not None else 0)
    t1 = np.zeros((o, v))
    t2 = np.zeros((o, o, v, v))
    lam = np.zeros(o * v + (o * v) ** 2) if want_lambda else None
    if guess is not None:
        t1[...] = guess[0]
        t2[...] = guess[1]
        if want_lambda and len(guess) > 2:
            lam[:o * v] = np.ravel(guess[2])
            lam[o * v:] = np.ravel(guess[3])
        elif want_lambda:
            lam[:o * v] = np.ravel(guess[0])
            lam[o * v:] = np.ravel(guess[1])
    info = np.zeros(8)
    code = _check(load().gfcc_ccsd(o, v, L, _dp(fock), _dp(chol), float(tol), int(max_iter), flags, _dp(t1), _dp(t2),
                                   _dp(lam) if lam is not None else None, _dp(info)))
    keys = ("e_corr", "t_iters", "t_residual", "lambda_iters", "lambda_residual", "t_seconds", "lambda_seconds",
            "t_flops_per_iter")
    d = {k: float(x) for k, x in zip(keys, info)}
    lam1 = lam[:o * v].reshape(o, v) if lam is not None else None
    lam2 = lam[o * v:].reshape(o, o, v, v) if lam is not None else None
    return t1, t2, lam1, lam2, d, code
