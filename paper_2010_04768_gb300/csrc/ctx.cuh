// The gfcc_ctx structure: problem sizes, options, device-resident inputs and Hbar elements.
#pragma once
#include <vector>

#include "common.cuh"

struct gfcc_ctx {
  // sizes: n = o + v orbitals; packed pair counts Po = o(o-1)/2, Pv = v(v-1)/2
  int o = 0, v = 0, L = 0, n = 0;
  long long Po = 0, Pv = 0, dim_ip = 0, dim_ea = 0;
  int sectors = GFCC_SECTOR_BOTH;
  int precision = GFCC_PREC_FP64;

  // options
  int restart = 30;
  int max_iters = 1500;
  int precond = GFCC_PRECOND_DIAG;
  int batch = 0;
  double inner_tol = 1e-3;

  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;

  // device inputs (float64)
  double *t1 = nullptr, *t2 = nullptr;    // [o][v], [o][o][v][v]
  double *l1 = nullptr, *l2 = nullptr;    // Lambda (alias t1/t2 when Lambda = T^dagger)

  // Hbar elements shared by both sectors
  double *Foo = nullptr, *Fvv = nullptr, *Fov = nullptr;   // [o][o] (m,i), [v][v] (a,e), [o][v] (m,e)

  // IP sigma operands (layouts named by their GEMM role)
  double *Wr_ip = nullptr;   // [(i,a)][(m,e)]  Wovvo[m,a,e,i] + 1/2 d_im Fvv[a,e] - d_ae Foo[m,i]
  double *Woooo = nullptr;   // [m][n][i][j]
  double *W1 = nullptr;      // [(i,a,j)][m]    Wovoo[m,a,j,i]
  double *V3 = nullptr;      // [e][(m,f,n)]    1/2 <mn||ef>'
  double *T3 = nullptr;      // [(i,a,j)][e]    t2[i,j,a,e]
  double *U1 = nullptr;      // [i][(m,e,n)]    -d_in Fov[m,e] + 1/2 Wooov[n,m,i,e]
  double *diag_ip = nullptr; // packed Fock-like diagonal

  // EA sigma operands
  double *Wr_ea = nullptr;   // [(i,b)][(m,e)]  Wovvo[m,b,e,i] + d_mi Fvv[b,e] - 1/2 d_be Foo[m,i]
  double *Wp = nullptr;      // [(a<b)][(e<f)]  Wvvvv[a,b,e,f]
  double *W3 = nullptr;      // [(i,b,a)][e]    Wvvvo[a,b,e,i]
  double *V3e = nullptr;     // [m][(n,f,e)]    1/2 <mn||ef>'
  double *T3e = nullptr;     // [(i,b,a)][m]    -t2[m,i,a,b]
  double *U1e = nullptr;     // [a][(m,x,y)]    Fov / Wvovv couplings of the 1p row
  double *diag_ea = nullptr;

  std::vector<void *> allocs;

  // statistics of the last solve
  std::vector<int> st_iters, st_status;
  std::vector<double> st_relres;

  // scratch reused across solves (grown on demand)
  void *scratch = nullptr;
  size_t scratch_bytes = 0;
};

namespace gfcc {
int dev_alloc(gfcc_ctx *c, double **p, long long count);      // owned by the context
int dev_alloc_tmp(double **p, long long count);                  // caller frees with cudaFree
int build_hbar(gfcc_ctx *c, const double *d_fock, const double *d_chol);
}  // namespace gfcc
