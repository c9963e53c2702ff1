// Initial guesses of the GMRES solves from converged solutions at nearby frequencies
// (Algorithm 1: "compute initial guess").
//
// For a system (omega, p) and converged solutions X_k = X_p(omega_k) of the same orbital
// (A(omega_k) X_k = b), the residual of the combination x0 = sum_k c_k X_k at omega is
//     b - A(omega) x0 = (1 - sum_k c_k) b - sum_k c_k delta_k X_k,   delta_k = omega - omega_k
// (eq. xplin: A(omega) = A(omega_k) + delta_k for IP; the EA operator has the same form with
// the sign of Hbar flipped), up to the residuals of the X_k.  So its norm is the quadratic form
// a^H Gm a of the Gram matrix Gm of (b, delta_1 X_1, ..., delta_K X_K), a = (sum c - 1, c), and a
// guess is scored without a sigma product.
#pragma once
#include "ctx.cuh"

namespace gfcc {

constexpr int GUESS_K = 8;                             // neighbours per system
constexpr int GUESS_NF = 3 + 3 * GUESS_K;              // features: omega, eta, p/n, delta_k, Re/Im <b|X_k>
constexpr int GUESS_NO = 2 * GUESS_K;                  // model outputs: Re/Im c_k
constexpr int GUESS_G = (GUESS_K + 1) * (GUESS_K + 1); // complex Gram entries

long long guess_gram_work_doubles(int nsys, long long n);

// Gm[s] = Gram of (b_s, delta_s1 X_1, ...) (complex [9][9]) and the features of system s:
// omega_s, eta, pfrac_s, delta_sk, Re/Im <b_s|X_k> * eta / ||b_s||^2.  nbr[s][k]: kept-solution
// slot of neighbour k or -1 (absent: zero vector, delta 0).  B: right-hand sides, complex, row
// stride ldb (complex elements).  work: guess_gram_work_doubles(nsys, n) doubles.
int guess_gram(cudaStream_t st, int nsys, long long n, const double *B, long long ldb, const float2 *store,
               const int *nbr, const double *delta, const double *omega, double eta, const double *pfrac, double *Gm,
               double *feat, double *work);

// Coefficients of the guess of each system.  mode GFCC_GUESS_LEARNED: c from the model outputs y
// ([s][16], needs all 8 neighbours); GFCC_GUESS_MINRES: the minimiser of the residual over the
// available neighbours.  A guess whose predicted ||r||^2/||b||^2 is not below 1 is replaced by
// zero.  Writes coef [s][8] complex, pred [s] (predicted ||r||^2/||b||^2, 1 for zero) and kind [s]
// (the GFCC_GUESS_* used).
int guess_choose(cudaStream_t st, int nsys, int mode, const double *Gm, const double *y, const int *navail,
                 double *coef, double *pred, int *kind);

// Scores for model evaluation: loss of the model's coefficients (no fallback) and of the minimiser.
int guess_losses(cudaStream_t st, int nsys, const double *Gm, const double *y, double *loss_model,
                 double *loss_minres);

// X0[s] = sum_k coef[s][k] X_k (zero where kind[s] == 0), complex FP64 rows of stride ldx.
int guess_combine(cudaStream_t st, int nsys, long long n, const float2 *store, const int *nbr, const double *coef,
                  const int *kind, double *X0, long long ldx);

// store[slot[s]] = U[s] rounded to FP32, for s < nsys with slot[s] >= 0.
int guess_store_put(cudaStream_t st, int nsys, long long n, const double *U, long long ldu, const int *slot,
                    float2 *store);

// Frequency order of a guessed sweep: the two ends first, then repeatedly the frequency farthest
// from those already taken (ties to the lower index), so that later frequencies have close
// neighbours on both sides.
std::vector<int> guess_frequency_order(const std::vector<double> &omega);

// The k nearest frequencies (by |omega_w - omega_j|, ties to the lower index) among those with
// done[j] set, j != w; returns how many were found (<= k).
int guess_neighbours(const std::vector<double> &omega, const char *done, long long done_stride, int w, int k,
                     int *out);

}  // namespace gfcc
