"""The digit-level rule of the incremental FP64-accurate residual, on a plain numpy model of the
digit splitting (no GPU; independent of the CUDA code).

An FP64-accurate product C = A B^T is formed from digit planes: each row of A (and each row of B,
one per planar column) is scaled by 2^-e, e the frexp exponent of its largest magnitude, and cut
into S digits of 6 bits, v 2^-e = sum_i a_i 64^-i + tail.  The product keeps the digit pairs with
i + j <= L, so its error in entry (r, c) is at most

    bound(L) = 2^(eA_r + eB_c) sum_k sum_{i + j > L} |a_i(A_rk)| |b_j(B_ck)| 64^-(i+j)
            <= 2^(eA_r + eB_c) K sum_{l > L} (l - 1) 64^2 64^-l.

After the first refinement step the residual is updated with the product A d of the step's
correction d at level P - k, k = floor(gap / 6), gap = e_x - e_d - 1 (frexp exponents of max|x| and
max|d|).  Because 2^e_d <= 2^(e_x - 6k), the bound of that product is no larger than the bound of
the level-P product A x that a full residual would take: the incremental residual is exactly as
accurate.  These tests check the bound and the rule on random operands.
"""
import numpy as np
import pytest


def split(M, S):
    """(digits [S][rows][K] as integers, row exponents): M[r] = 2^e_r sum_i digits[i][r] 64^-(i+1) + tail."""
    amax = np.max(np.abs(M), axis=1)
    e = np.frexp(np.where(amax > 0, amax, 1.0))[1]
    r = M / np.ldexp(1.0, e)[:, None]
    digits = []
    for i in range(1, S + 1):
        a = np.rint(r * 64.0 ** i)
        r = r - a / 64.0 ** i
        digits.append(a)
    return np.array(digits), e


def product(dA, eA, dB, eB, L):
    """sum over digit pairs i + j <= L of the scaled integer products."""
    S = dA.shape[0]
    C = np.zeros((dA.shape[1], dB.shape[1]))
    for i in range(1, S + 1):
        for j in range(1, S + 1):
            if i + j <= L:
                C += (dA[i - 1] @ dB[j - 1].T) * 64.0 ** -(i + j)
    return C * np.ldexp(1.0, eA[:, None] + eB[None, :])


def bound(dA, eA, dB, eB, L):
    """entrywise bound of the pairs left out at level L"""
    S = dA.shape[0]
    B = np.zeros((dA.shape[1], dB.shape[1]))
    for i in range(1, S + 1):
        for j in range(1, S + 1):
            if i + j > L:
                B += (np.abs(dA[i - 1]) @ np.abs(dB[j - 1]).T) * 64.0 ** -(i + j)
    return B * np.ldexp(1.0, eA[:, None] + eB[None, :])


S, P = 5, 6          # small enough that float64 rounding stays far below the truncation error


@pytest.fixture(scope="module")
def operands():
    rng = np.random.default_rng(7)
    A = rng.standard_normal((24, 300)) * np.exp(rng.uniform(-3, 3, (24, 1)))
    x = rng.standard_normal((6, 300)) * np.exp(rng.uniform(-2, 2, (6, 1)))
    return A, x


def test_digits_reconstruct_and_are_small(operands):
    A, _ = operands
    dA, eA = split(A, S)
    back = np.tensordot(64.0 ** -np.arange(1, S + 1), dA, axes=1) * np.ldexp(1.0, eA)[:, None]
    assert np.max(np.abs(back - A) / np.max(np.abs(A), axis=1, keepdims=True)) <= 64.0 ** -S
    assert np.max(np.abs(dA[0])) <= 64 and np.max(np.abs(dA[1:])) <= 32


def test_level_product_within_its_bound(operands):
    A, x = operands
    dA, eA = split(A, S)
    dx, ex = split(x, S)
    full = product(dA, eA, dx, ex, 2 * S)
    for L in range(2, 2 * S):
        err = np.abs(product(dA, eA, dx, ex, L) - full)
        assert np.all(err <= bound(dA, eA, dx, ex, L) * (1 + 1e-9) + 1e-300)


@pytest.mark.parametrize("shift", [3, 7, 13, 20, 27])
def test_correction_at_dropped_levels_keeps_the_full_level_bound(operands, shift):
    # d: a correction 2^-shift times the size of x (different values, same columns)
    A, x = operands
    rng = np.random.default_rng(shift)
    d = rng.standard_normal(x.shape) * np.max(np.abs(x), axis=1, keepdims=True) * 2.0 ** -shift
    dA, eA = split(A, S)
    dx, ex = split(x, S)
    dd, ed = split(d, S)
    # the rule of the implementation: the worst column decides, gap from frexp exponents minus one
    gap = int(np.min(ex - ed)) - 1
    k = max(gap, 0) // 6
    level = max(2, P - k)
    err_d = np.abs(product(dA, eA, dd, ed, level) - product(dA, eA, dd, ed, 2 * S))
    # the analytic bound of the full-level product of x (what a full residual would carry)
    K = A.shape[1]
    tail = sum((l - 1) * 64.0 ** 2 * 64.0 ** -l for l in range(P + 1, 2 * S + 1))
    bound_x = K * tail * np.ldexp(1.0, eA[:, None] + ex[None, :])
    assert np.all(err_d <= bound_x)
    assert level <= P and (shift < 13 or level < P)   # a correction 2^-13 of x or smaller drops levels
