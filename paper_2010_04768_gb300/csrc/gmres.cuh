// Batched restarted GMRES over the shifted operator of eq. xplin.
#pragma once
#include <vector>

#include "ctx.cuh"

namespace gfcc {

long long gmres_work_doubles(const gfcc_ctx *c, int sector, long long n, int nsys, int m, bool mixed = false);

// One batch of nsys systems of packed dimension n in one sector.  The caller fills B
// (right-hand sides, complex interleaved, [s][n]; rhs()) and omega, then calls solve() or
// solve_refined(); the solution is left in solution() ([s][n], complex FP64).  Per-system results: iters, relres, state
// (3 = converged, 4 = not converged).
struct Gmres {
  Gmres() = default;
  Gmres(const Gmres &) = delete;
  Gmres &operator=(const Gmres &) = delete;
  ~Gmres();
  gfcc_ctx *c = nullptr;
  int sector = GFCC_SECTOR_IP;
  long long n = 0;
  int nsys = 0, m = 30, NV = 32, nch = 1;
  double eta = 0.0;
  double tol_outer = 0.0;  // continuous refinement: the outer (FP64) tolerance
  bool graphs_ok = true;   // the caller expects the batch size to stay (captured graphs pay off)
  bool use_precond = false;
  bool mixed = false;      // inner operator on the BF16 tensor cores (IP), FP64 residuals outside
  bool f32 = false;        // Krylov vectors V, U, B, W in FP32 (inner solves of the refinement)
  double *X = nullptr, *R = nullptr, *B0 = nullptr;   // refinement: solution, residual, original rhs
  double *D = nullptr, *Yd = nullptr;   // refinement: the last correction (FP64) and A D
  bool have_d = false;                  // D holds the correction of the last refine_correct
  double *b0norm = nullptr;
  double *V = nullptr, *U = nullptr, *B = nullptr, *W = nullptr;
  double *partial = nullptr, *h = nullptr, *h2 = nullptr, *y = nullptr, *nrm = nullptr;
  double *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr;
  double *bnorm = nullptr, *relres = nullptr, *est = nullptr, *omega = nullptr;
  int *state = nullptr, *kcyc = nullptr, *iters = nullptr, *rflag = nullptr;
  int *act = nullptr;   // the systems the operator runs on in an Arnoldi step (see solve_t)
  double *relres0 = nullptr;   // relative residual of the initial iterate (first true residual)
  double *sigma_work = nullptr;

  int init(gfcc_ctx *ctx, int sector, long long n, int nsys, int m, double *work, bool mixed = false);
  // where the caller puts the FP64 right-hand sides ([s][n] complex) and finds the solutions
  double *rhs() const { return mixed ? B0 : B; }
  double *solution() const { return mixed ? X : U; }
  // FP64 or FP64-accurate (digit planes; level > 0 caps the digit level), no preconditioner
  int op_fp64(const double *x, long long ldx, double *y, long long ldy, int level = 0);
  int mdot(const double *Vb, long long vs, long long vi, int nv, const double *w, long long ws, double *out, int want,
           int accumulate);
  // max_cycles > 0 bounds the number of restart cycles (systems left pending end in state 4).
  // use_x0: U holds an initial iterate (unpreconditioned coordinates) instead of zero.
  int solve(double tol, int max_iters, int *h_state, int max_cycles = 0, bool use_x0 = false);
  // iterative refinement: FP64 residual r = b - A x, inner GMRES on the mixed operator to
  // inner_tol, x += d, until ||r|| <= tol ||b||.  Leaves x in U, the FP64 relative residual in
  // relres, the summed inner iterations in h_iters and the final state (3 / 4) in h_state.
  // use_x0: X holds an initial iterate instead of zero.
  // h_outer (optional): per system, the FP64-accurate residuals evaluated (refinement steps + 1)
  int solve_refined(double tol, double inner_tol, int max_iters, int *h_state, int *h_iters, bool use_x0 = false,
                    int *h_outer = nullptr);

  // Pieces of solve_refined for continuous batching (slots refilled with new systems as others
  // finish).  refine_norms: ||b0|| of every slot.  refine_residual: R = B0 - A X (FP64-accurate),
  // or, after a correction with the incremental option, R -= A D with the digit level that
  // max|D| / max|X| allows; relres = ||R|| / ||b0||, per-slot done flags (device kcyc: 1 =
  // converged) copied to h_done.  refine_correct: for the slots with h_done[s] == 0, one inner
  // solve A d = R (BF16 operator), D = d and X += d; the inner iterations of each slot are added
  // to h_iters.
  int refine_norms();
  int refine_residual(int *h_done, double *h_relres);
  int refine_residual_free(int *h_done, double *h_relres);   // the checks on R as it is (no operator)
  // R = B0 - A X (FP64-accurate), or R -= A D at the digit level max|D| / max|X| allows when the
  // last step left its correction in D (incremental option, digit-plane residuals)
  int residual_update();
  int refine_correct(const int *h_done, int *h_state, int *h_iters);
  // X[s] = 0 and R[s] = B0[s] for the slots with mask[s] != 0 (device mask)
  int reset_slots(const int *d_mask);
  // keep slots perm[0..na) (device, increasing) as slots 0..na-1 (X, B0, R and D move) and continue
  // with nsys = na
  int compact_slots(const int *d_perm, int na);

 private:
  // CUDA graphs of the Arnoldi steps of the inner (FP32) solves: one per step k, captured for the
  // current number of systems once its contraction shapes have been seen (tuned) in an earlier call
  std::vector<cudaGraphExec_t> gexec;
  std::vector<long long> glaunch;
  int gnsys = -1, gseen = 0;
  bool gbroken = false;
  void drop_graphs();
  // y = A x for the batch (nact < 0) or for the nact systems listed in the device array idx (SysBatch::idx)
  template <typename T>
  int op_t(const T *x, long long ldx, T *y, long long ldy, int nact = -1, const int *idx = nullptr);
  template <typename T>
  int mdot_t(const T *Vb, long long vs, long long vi, int nv, const T *w, long long ws, double *out, int want,
             int accumulate);
  template <typename T>
  int cgs2_t(const T *Vb, long long vs, int nv, T *w, cudaStream_t st);
  template <typename T>
  int solve_t(double tol, int max_iters, int *h_state, int max_cycles, bool use_x0);
};

}  // namespace gfcc
