// Batched restarted GMRES over the shifted operator of eq. xplin.
#pragma once
#include "ctx.cuh"

namespace gfcc {

long long gmres_work_doubles(const gfcc_ctx *c, int sector, long long n, int nsys, int m);

// One batch of nsys systems of packed dimension n in one sector.  The caller fills B
// (right-hand sides, complex interleaved, [s][n]) and omega, then calls solve(); the
// solution is left in U ([s][n], complex).  Per-system results: iters, relres, state
// (3 = converged, 4 = not converged).
struct Gmres {
  gfcc_ctx *c = nullptr;
  int sector = GFCC_SECTOR_IP;
  long long n = 0;
  int nsys = 0, m = 30, NV = 32, nch = 1;
  double eta = 0.0;
  bool use_precond = false;
  double *V = nullptr, *U = nullptr, *B = nullptr, *W = nullptr;
  double *partial = nullptr, *h = nullptr, *h2 = nullptr, *y = nullptr, *nrm = nullptr;
  double *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr;
  double *bnorm = nullptr, *relres = nullptr, *est = nullptr, *omega = nullptr;
  int *state = nullptr, *kcyc = nullptr, *iters = nullptr;
  double *sigma_work = nullptr;

  int init(gfcc_ctx *ctx, int sector, long long n, int nsys, int m, double *work);
  int op(const double *x, long long ldx, double *y, long long ldy);
  int mdot(const double *Vb, long long vs, long long vi, int nv, const double *w, long long ws, double *out, int want,
           int accumulate);
  int solve(double tol, int max_iters, int *h_state);
};

}  // namespace gfcc
