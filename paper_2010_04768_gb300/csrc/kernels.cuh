// Declarations of the device-side building blocks of libgfcc.
#pragma once
#include "common.cuh"

namespace gfcc {

// ---------------------------------------------------------------- generic FP64 contraction
struct Contract {
  const double *A = nullptr;
  const double *B = nullptr;
  double *C = nullptr;
  long long M = 0, N = 0, K = 0;
  IMap am{0, 0, 0}, ak{0, 0, 0}, bk{0, 0, 0}, bn{0, 0, 0}, cm{0, 0, 0}, cn{0, 0, 0};
  long long batch = 1, sab = 0, sbb = 0, scb = 0;
  double alpha = 1.0, beta = 0.0;
  // split-K: nsplit partial products over K ranges of kchunk, partial z written at C + z * scz
  long long nsplit = 1, kchunk = 0, scz = 0;
};
int contract_f64(const Contract &c, cudaStream_t st);
// gemm_f64 sends contractions of at least g_emulate_min_flops to the FP64-accurate digit-plane
// path when g_emulate_big is set (mixed-precision contexts set it during their setup)
extern thread_local bool g_emulate_big;
extern double g_emulate_min_flops;
// the calling thread's threshold instead of g_emulate_min_flops while >= 0 (closed-shell operator)
extern thread_local double g_emulate_min_flops_local;
int gemm_f64(cudaStream_t st, long long M, long long N, long long K, double alpha,
             const double *A, IMap am, IMap ak, const double *B, IMap bk, IMap bn, double beta,
             double *C, IMap cm, IMap cn, long long batch = 1, long long sab = 0, long long sbb = 0,
             long long scb = 0);

// ---------------------------------------------------------------- Cholesky-vector building blocks
// C((p,r),(q,s)) (+)= alpha * sum_K Lt[K][P0+p][R0+r] Lt[K][Q0+q][S0+s] for Cholesky vectors Lt [L][n][n]
// (GEMM row index p * nr + r, column index q * ns + s, placed through cm / cn)
int chol_eri(cudaStream_t st, const double *Lt, int n, int L, long long P0, long long np, long long R0, long long nr,
             long long Q0, long long nq, long long S0, long long ns, double alpha, double beta, double *C, IMap cm,
             IMap cn);
// M <- (1 - t) M (1 + t) in place for `batch` n x n matrices spaced `stride` apart, t[o+a][i] = t1[i][a]
// (the T1 similarity transformation of a one-body operator, n = o + v)
int t1_dress(cudaStream_t st, const double *t1, int o, int v, double *M, long long batch, long long stride);
// F[p][q] += aj * sum_K M[K][p][q] tr_o(M[K]) + ak * sum_K sum_{j<o} M[K][p][j] M[K][j][q]
int chol_coulomb_exchange(cudaStream_t st, const double *M, int n, int o, int L, double *F, double aj, double ak);

// ---------------------------------------------------------------- elementwise helpers
// For every index (i0, i1, i2, i3) < d:
//   out[sum i_k * os[k]] = alpha * in[sum i_k * is[k]] + beta * out[sum i_k * os[k]]
int permute4(cudaStream_t st, const long long d[4], const double *in, const long long is[4], double *out,
             const long long os[4], double alpha, double beta);
int fill_f64(cudaStream_t st, double *p, long long n, double value);

}  // namespace gfcc
