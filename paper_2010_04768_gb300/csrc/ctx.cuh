// The gfcc_ctx structure: problem sizes, options, device-resident inputs and Hbar elements.
#pragma once
#include <cuda_bf16.h>

#include <vector>

#include "common.cuh"
#include "ozaki.cuh"

// Profiling phases (gfcc_profile_read): CUDA-event timings on the context's stream.
enum GfccPhase {
  PH_SETUP = 0,       // gfcc_create: Hbar elements
  PH_RING = 1,        // the (ov) x (ov) ring contraction of the FP64 sigma product
  PH_VVVV = 2,        // EA vvvv contraction
  PH_SIGMA = 3,       // a whole sigma product (contains phases 1 and 2)
  PH_ARNOLDI = 4,     // Gram-Schmidt dots, updates, normalisation
  PH_LSQ = 5,         // Givens rotations, back substitution, cycle bookkeeping
  PH_OVERLAP = 6,     // right-hand sides, left vectors, G overlaps
  PH_SOLVE = 7,       // a whole gfcc_solve
  PH_RING_BF16 = 8,   // the ring contraction on the BF16 tensor cores (mixed precision)
  PH_RING_EMU = 9,    // the FP64-accurate ring contraction of the refinement residual (digit planes)
  PH_UNPACK = 10,     // expansion of packed vectors into the contraction layouts (BF16 / digits)
  PH_GUESS = 11,      // initial guesses: neighbour Gram matrices, model, coefficients, combination
  PH_EMU_OTHER = 12,  // the other FP64-accurate products of the refinement residual (oooo / vvvv,
                      // three-body, 1h / 1p row), digit slicing of their inputs included
  PH_BF16_OTHER = 13, // the other BF16 products of the inner sigma (oooo, three-body, 1h / 1p row)
  PH_EPILOGUE = 14,   // sigma epilogues (shift, diagonal, packing of y); "flops" = algorithmic bytes
  PH_RING_EMU_WORK = 15,  // same region as PH_RING_EMU; "flops" = the BF16 tensor-core work of all
                          // its digit pairs (PH_RING_EMU counts the one FP64 product it evaluates)
  PH_COUNT = 16
};

struct gfcc_mlp;

// Converged solutions kept after a solve (FP32 complex, [omega][orbital][dim]): the neighbours
// of the initial guesses, and training data for the guess model.
struct KeptSolutions {
  float2 *X = nullptr;
  size_t bytes = 0;
  int sector = 0;
  long long n = 0;
  int nw = 0, norb = 0;
  double eta = 0.0;
  std::vector<double> omega;
  std::vector<int> orb;
  std::vector<char> done;   // [omega][orbital]: slot holds a converged solution
};

struct gfcc_ctx {
  // sizes: n = o + v orbitals; packed pair counts Po = o(o-1)/2, Pv = v(v-1)/2
  int o = 0, v = 0, L = 0, n = 0;
  long long Po = 0, Pv = 0, dim_ip = 0, dim_ea = 0;
  int sectors = GFCC_SECTOR_BOTH;
  int precision = GFCC_PREC_FP64;

  // options
  int restart = 30;          // FP64 GMRES
  int inner_restart = 60;    // inner GMRES of the mixed-precision refinement
  int max_iters = 1500;
  int precond = GFCC_PRECOND_DIAG;
  int batch = 0;
  double mem_share = 1.0;    // fraction of the free device memory a solve may plan its batch for
  double inner_tol = 3e-4;
  int inner_cycles = 1;      // GMRES restart cycles per refinement step (each ends with an FP64-accurate residual)
  int inner_fp64 = 0;        // 1: FP64 Krylov vectors in the inner solves (default FP32)
  int use_graphs = 1;        // replay the Arnoldi steps of the inner solves from CUDA graphs

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
  // closed-shell spin-adapted IP context (gfcc_create_rhf; rhf.cu): spatial orbitals, vectors
  // [r_i (o) | r_ij^a ([i][j][a], o^2 v)], every element alpha-beta spin-summed
  int rhf = 0;
  int rhf_emulate = 1;      // GFCC_OPT_CLOSED_SHELL_EMULATE: its large contractions from digit planes
  double *rM1 = nullptr, *rM2 = nullptr, *rM3 = nullptr;   // ring matrices [(i,a)][(m,e)] (ov x ov)
  double *rWT = nullptr;    // [(i,j,a)][e | m]: -t_ij^ea | -W_maij  (o^2 v x (v + o))
  double *rVz = nullptr;    // [e][(m,n,f)]: 2 u_mnef - u_mnfe  (v x o^2 v)
  double *rU1 = nullptr;    // [i][m | (m,n,e)]: the 1h row (o x (o + o^2 v))
  gfcc::EmuOperand rM1e, rM2e, rM3e;   // digit planes of the ring matrices (when they fit)

  // mixed-precision IP operands: BF16, K-major, row strides padded to multiples of 8.  The exact
  // Fock-like diagonal d (diag_ip) is left out of them and applied in FP64 by the epilogue.
  __nv_bfloat16 *Wr_bf = nullptr;  // [(i,a)][(m,e)]   ring core + off-diagonal Fbar folding, ld_ov
  __nv_bfloat16 *Wq_bf = nullptr;  // [(i,j)][(m,n)]   1/2 Woooo[m,n,i,j], ld_o2
  __nv_bfloat16 *WT_bf = nullptr;  // [(i,a,j)][m | e] [Wovoo[m,a,j,i] | t2[i,j,a,e]] (ovoo and three-body), ld_ot
  __nv_bfloat16 *V3_bf = nullptr;  // [e][(m,f,n)]     1/2 <mn||ef>', ld_o2v
  __nv_bfloat16 *U1_bf = nullptr;  // [i][(m,e,n) | m] U1 and the off-diagonal -Fbar_oo of the 1h row, ld_k1
  long long ld_ov = 0, ld_o2 = 0, ld_o = 0, ld_o2v = 0, ld_v = 0, ld_k1 = 0, ld_ot = 0;

  // digit planes of the FP64 IP operands for the FP64-accurate residual on the tensor cores
  // (full Fock folding, same GEMM roles as the BF16 operands; V3 padded to the K of U1x)
  gfcc::EmuOperand eWr, eWq, eWT, eV3, eU1;   // eWT: [W1 | T3] over K = o + v
  int emu_S = 8, emu_P = 9;
  int residual_emulated = 1;   // 0: refinement residuals with the FP64 (DFMA) sigma
  int incremental = 1;         // 1: r -= A d at the digit level the correction needs (after the first step)
  long long res_full = 0, res_inc = 0, res_inc_levels = 0;   // residual products of the last solve

  // EA sigma operands
  double *Wr_ea = nullptr;   // [(i,b)][(m,e)]  Wovvo[m,b,e,i] + d_mi Fvv[b,e] - 1/2 d_be Foo[m,i]
  double *Wp = nullptr;      // [(a<b)][(e<f)]  Wvvvv[a,b,e,f]
  double *W3 = nullptr;      // [(i,b,a)][e]    Wvvvo[a,b,e,i]
  double *V3e = nullptr;     // [m][(n,f,e)]    1/2 <mn||ef>'
  double *T3e = nullptr;     // [(i,b,a)][m]    -t2[m,i,a,b]
  double *U1e = nullptr;     // [a][(m,x,y)]    Fov / Wvovv couplings of the 1p row
  double *diag_ea = nullptr;

  // mixed-precision EA operands (BF16, K-major, strides padded to multiples of 8; the Fock-like
  // diagonal diag_ea is left out and applied in FP64)
  __nv_bfloat16 *Wre_bf = nullptr;  // [(i,b)][(m,e)]   ring core + off-diagonal Fbar folding, ld_ov
  __nv_bfloat16 *Wp_bf = nullptr;   // [(a<b)][(e<f)]   Wvvvv, ld_pv
  __nv_bfloat16 *WTe_bf = nullptr;  // [(i,b,a)][e | m] [Wvvvo[a,b,e,i] | -t2[m,i,a,b]], ld_ot
  __nv_bfloat16 *V3e_bf = nullptr;  // [m][(n,f,e)]     1/2 <mn||ef>', ld_ov2
  __nv_bfloat16 *U1e_bf = nullptr;  // [a][(m,x,y) | e] U1e and the off-diagonal Fbar_vv of the 1p row, ld_k1e
  long long ld_pv = 0, ld_ov2 = 0, ld_k1e = 0;
  // digit planes of the FP64 EA operands (full Fock folding) for the FP64-accurate residual
  gfcc::EmuOperand eWre, eWp, eWTe, eV3e, eU1e;   // eWTe: [W3 | T3e] over K = v + o

  std::vector<void *> allocs;

  // initial guesses (Algorithm 1: "compute initial guess")
  int guess = 0;                 // GFCC_GUESS_*
  int keep_solutions = 0;        // keep the converged solutions of the last sector solved
  gfcc_mlp *mlp = nullptr;       // model of GFCC_GUESS_LEARNED (not owned)
  KeptSolutions kept;

  // statistics of the last solve
  std::vector<int> st_iters, st_status, st_guess, st_outer;
  std::vector<double> st_relres, st_guess_pred, st_relres0;

  // profiling (CUDA events on the context's stream)
  bool prof = false;
  struct PendingEv {
    cudaEvent_t a, b;
    int phase;
    double flops;
  };
  std::vector<PendingEv> pend;
  std::vector<cudaEvent_t> ev_pool;
  double prof_ms[PH_COUNT] = {0};
  long long prof_n[PH_COUNT] = {0};
  double prof_flops[PH_COUNT] = {0};

  // scratch reused across solves (grown on demand)
  void *scratch = nullptr;
  size_t scratch_bytes = 0;

  // when set, every solve copies each finished system's solution (FP64 complex) to sink[task][dim]
  // (task = omega index x number of orbitals + orbital index; the subspace builder of mor.cu)
  double *sink = nullptr;

  // left vectors c_q (eq. gfxn2) of the last orbital list of each sector ([0] IP, [1] EA): they depend
  // on the list and the amplitudes only, so repeated solves over the same list reuse them
  struct LeftCache {
    std::vector<int> orb;
    double *C = nullptr;   // [n_orb][dim]
    size_t bytes = 0;
  } left_cache[2];
};

namespace gfcc {
// Times the enclosed region on the context's stream when profiling is on.
struct PhaseTimer {
  gfcc_ctx *c;
  int phase;
  double flops;
  cudaEvent_t a = nullptr;
  PhaseTimer(gfcc_ctx *ctx, int ph, double fl = 0.0);
  ~PhaseTimer();
};
void prof_resolve(gfcc_ctx *c);   // after a stream synchronisation: fold pending events into the totals

int dev_alloc(gfcc_ctx *c, double **p, long long count);      // owned by the context
int dev_alloc_tmp(double **p, long long count);                  // caller frees with cudaFree
int build_hbar(gfcc_ctx *c, const double *d_fock, const double *d_chol);
// closed-shell spin-adapted elements (rhf.cu); c->t1, c->t2, c->l1, c->l2 are spatial
int build_hbar_rhf(gfcc_ctx *c, const double *d_fock, const double *d_chol);
int build_rhs_rhf(gfcc_ctx *c, int nsys, const int *d_porb, const int *d_mask, double *B, cudaStream_t st);
int build_left_rhf(gfcc_ctx *c, int nq, const int *d_orb, double *C, cudaStream_t st);
// Device-side input check of a [d0][d1][d2][d3] tensor: finite entries and, where s01 / s23 is set,
// x[i][j][.][.] == sign * x[j][i][.][.] / x[.][.][a][b] == sign * x[.][.][b][a] to rel * max(1, max|x|)
int check_input_tensor(cudaStream_t st, const double *x, long long d0, long long d1, long long d2, long long d3,
                       int s01, int s23, double sign, double rel, const char *name);
// gfcc_solve's argument checks and solve on host arrays (rows and columns over one orbital list)
int solve_rows_host(gfcc_ctx *c, int n_omega, const double *omegas, double eta, int n_orb, const int *orbitals,
                    double tol, double *G);
}  // namespace gfcc
