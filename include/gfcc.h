/*
 * gfcc.h - C ABI of the GB300 GFCCSD library (libgfcc.so).
 *
 * The library solves, for every frequency omega and orbital p, the shifted
 * complex linear systems of the GFCCSD method (Peng et al., "GFCCLib",
 * arXiv 2010.04768, Theory section, eq. xplin)
 *
 *     IP: (omega - i eta + Hbar_N) X_p |Phi> = a_p-bar |Phi>      (1h + 2h1p space, eq. xp)
 *     EA: (omega + i eta - Hbar_N) Y_q |Phi> = a_q^+-bar |Phi>    (1p + 2p1h space, eq. yq)
 *
 * by GMRES (GFCC Workflow and Bottlenecks section), and forms the Green's
 * function of eqs. gfxn2/gfxn3
 *
 *     G_pq(omega) = <Phi|(1+Lambda) a_q^+-bar X_p|Phi> + <Phi|(1+Lambda) a_p-bar Y_q|Phi>.
 *
 * Conventions (spin-orbital formalism, n = o + v orbitals, occupied first):
 *   Hbar = e^-T H e^T with H = sum h_pq p^+q + 1/4 sum <pq||rs> p^+q^+sr,
 *   <pq||rs> = (pr|qs) - (ps|qr), (pr|qs) = sum_K L[K][p][r] L[K][q][s]
 *   (the Cholesky representation of the Implementation Details section), and
 *   h = fock - sum_j <pj||qj> so that the reference Fock matrix is `fock`.
 *   The operator of eq. xplin is taken in commutator form <mu|[Hbar, R]|Phi>.
 *
 * All arrays are row-major float64 (IEEE binary64).  Unless stated otherwise,
 * pointers are HOST pointers; the library copies what it needs and never keeps
 * a caller pointer after a call returns.  A context owns all the device memory
 * it allocates and one CUDA stream (settable); it is not thread-safe.
 *
 * Return codes: 0 = success, > 0 = warning (results written), < 0 = error
 * (nothing written).  No error aborts the process; gfcc_last_error() gives a
 * message for the last failing call on the calling thread.
 */
#ifndef GFCC_H
#define GFCC_H

#ifdef __cplusplus
extern "C" {
#endif

#define GFCC_OK                    0
#define GFCC_WARN_NOT_CONVERGED    1   /* G written; gfcc_last_stats says which columns missed tol     */
#define GFCC_ERR_ARG             (-1)  /* bad size, ordering, symmetry, orbital index, eta/tol <= 0     */
#define GFCC_ERR_OOM             (-2)  /* device allocation failed                                      */
#define GFCC_ERR_CUDA            (-3)  /* a CUDA call or kernel launch failed                           */
#define GFCC_ERR_TIMEOUT         (-4)  /* a bounded device wait gave up                                 */
#define GFCC_ERR_STATE           (-5)  /* call not valid in the context's current state                 */

/* Sectors (gfcc_set_option key GFCC_OPT_SECTOR). */
#define GFCC_SECTOR_IP   1
#define GFCC_SECTOR_EA   2
#define GFCC_SECTOR_BOTH 3

/* Precisions (key GFCC_OPT_PRECISION). */
#define GFCC_PREC_FP64        0   /* every step in float64                                              */
#define GFCC_PREC_MIXED_BF16  1   /* sigma product on bf16 tensor cores + fp64 iterative refinement    */
#define GFCC_PREC_FP64_EMULATED 2 /* gfcc_sigma_ex only: FP64-accurate sigma from BF16 digit planes     */

/* Preconditioners (key GFCC_OPT_PRECOND). */
#define GFCC_PRECOND_NONE  0      /* plain GMRES, as in the paper's runs                                */
#define GFCC_PRECOND_DIAG  1      /* right preconditioning by the Fock-like diagonal of the operator    */

/* Option keys for gfcc_set_option. */
#define GFCC_OPT_SECTOR      1    /* GFCC_SECTOR_*; default BOTH (eq. gfxn3)                            */
#define GFCC_OPT_PRECISION   2    /* GFCC_PREC_*; default FP64                                           */
#define GFCC_OPT_RESTART     3    /* GMRES restart length m (1..64); default 30                          */
#define GFCC_OPT_MAX_ITERS   4    /* max sigma products per system; default 1500                         */
#define GFCC_OPT_PRECOND     5    /* GFCC_PRECOND_*; default DIAG                                        */
#define GFCC_OPT_BATCH       6    /* systems solved together (0 = chosen from free memory); default 0   */
#define GFCC_OPT_INNER_TOL   7    /* mixed precision: inner GMRES relative tolerance; default 3e-4       */
#define GFCC_OPT_RESIDUAL    8    /* mixed precision refinement residual: 1 (default) FP64-accurate from
                                     digit planes on the tensor cores, 0 the FP64 (DFMA) sigma          */
#define GFCC_OPT_INNER_CYCLES 9   /* mixed precision: GMRES restart cycles per refinement step; default 1 */
#define GFCC_OPT_EMU_LEVEL  10    /* digit pairs i + j <= level in the FP64-accurate products (8 digits of
                                     6 bits per operand, 2 <= level <= 16); default 9.  The products
                                     evaluate the operator's couplings; its Fock-like diagonal is exact
                                     in FP64                                                            */
#define GFCC_OPT_GUESS      11    /* GFCC_GUESS_*: initial iterate of each GMRES solve; default ZERO     */
#define GFCC_OPT_KEEP_SOLUTIONS 12 /* 1: keep the converged solutions of the last sector solved after
                                     gfcc_solve (for gfcc_mlp_collect); default 0                        */
#define GFCC_OPT_EMU_FUSED_N 16   /* FP64-accurate products with at most this many columns run all digit
                                     pairs of a tile in one kernel (levels in TMEM); wider ones one GEMM
                                     per digit pair.  Process-wide; default 512                          */
#define GFCC_OPT_GRAPHS     15    /* 1 (default): the Arnoldi steps of the inner solves of the mixed
                                     refinement are captured once per batch size into CUDA graphs and
                                     replayed (not while profiling, not on the legacy default stream)    */
#define GFCC_OPT_AUTOTUNE   14    /* 1 (default): the first tensor-core contraction of each shape times
                                     the 64 / 128 / 256-column tiles and later ones use the fastest;
                                     0: the narrowest tile covering N.  Process-wide.                    */
#define GFCC_OPT_INNER_KRYLOV 13  /* mixed precision: precision of the Krylov vectors of the inner GMRES
                                     solves, 32 (default) or 64 bits; the refinement residual and the
                                     solution stay FP64                                                  */
#define GFCC_OPT_INNER_RESTART 18 /* mixed precision: restart length of the inner GMRES solves (1..64);
                                     default 60 (GFCC_OPT_RESTART is that of the FP64 GMRES)             */
#define GFCC_OPT_INCREMENTAL 17   /* mixed precision, FP64-accurate residuals: 1 (default) after the first
                                     refinement step the residual is updated as r -= A d with the step's
                                     correction d, its product taking only the digit levels that the
                                     ratio max|d| / max|x| leaves significant (at most the error of the
                                     full product A x); 0: every residual is b - A x at the full level */

/* Process-wide option keys (gfcc_set_process_option; AUTOTUNE and EMU_FUSED_N above are also
 * accepted there). */
#define GFCC_OPT_SETUP_EMULATE_FLOPS 19 /* contexts created GFCC_PREC_MIXED_BF16 evaluate the setup
                                     contractions of at least this many flops from digit planes on
                                     the tensor cores (FP64-accurate); default 4e12, 0 = all of them   */
#define GFCC_OPT_WAIT_NS    20    /* limit of the bounded waits of the tensor-core kernels in
                                     nanoseconds (1 .. 1e11); default 1e9.  A wait that runs out makes
                                     the call return GFCC_ERR_TIMEOUT                                   */
#define GFCC_OPT_TEST_NO_LOADS 21 /* test only: 1 makes the tensor-core kernels issue no loads, so that
                                     their first wait runs out (with nothing in flight) and the call
                                     returns GFCC_ERR_TIMEOUT; default 0                               */
#define GFCC_OPT_GEMM_PAIR  22    /* BF16 tensor-core products on CTA pairs (256 x 256 tiles over two
                                     SMs, tcgen05 cta_group::2): 0 (default) the autotuner times them
                                     beside the one-CTA tiles, 1 whenever they apply, 2 never          */
#define GFCC_OPT_GEMM_PERSIST 23  /* BF16 tensor-core products with a persistent tile loop (one CTA per
                                     SM, two TMEM accumulators): 0 (default) timed by the autotuner on
                                     launches of several waves, 1 always (unless GFCC_OPT_GEMM_PAIR is
                                     1), 2 never                                                        */
#define GFCC_OPT_CLOSED_SHELL_EMULATE 24 /* closed-shell contexts (gfcc_create_rhf) only: 1 (default) the
                                     contractions of the operator of at least 1e9 flops (the ring sums,
                                     oooo) are FP64-accurate products of BF16 digit planes on the tensor
                                     cores; 0 every contraction on the FP64 units                       */

/* Initial guesses (Algorithm 1, "compute initial guess").  With a guess other than ZERO, gfcc_solve
 * keeps every converged solution X_p(omega) (FP32 complex, n_omega * n_orb * dim * 8 bytes of device
 * memory per sector), solves the frequencies in a spread-out order (the two ends first, then always
 * the frequency farthest from those already taken) and starts each system (omega, p) from a
 * combination x0 = sum_k c_k X_p(omega_k) of the converged solutions of the same orbital at the 8
 * nearest frequencies solved in earlier batches.  Because A(omega) X_k = b + (omega - omega_k) X_k,
 * the residual of x0 is known from the 9 x 9 Gram matrix of (b, (omega - omega_k) X_k) without a
 * sigma product; a guess whose predicted residual is not below ||b|| is replaced by zero.  The
 * converged G does not depend on the guess (to the solver tolerance). */
#define GFCC_GUESS_ZERO     0     /* x0 = 0                                                              */
#define GFCC_GUESS_LEARNED  1     /* c from the model attached with gfcc_set_guess_model (needs all 8
                                     neighbours, otherwise zero)                                         */
#define GFCC_GUESS_MINRES   2     /* c minimising the predicted residual over the available neighbours
                                     (normal equations with a relative shift of 1e-12)                   */

/* Per-column status values reported by gfcc_last_stats. */
#define GFCC_STATUS_CONVERGED      0
#define GFCC_STATUS_NOT_CONVERGED  1

typedef struct gfcc_ctx gfcc_ctx;

/*
 * gfcc_create - copy the problem to the device and build the Hbar elements.
 *   o, v      : occupied / virtual orbital counts (o >= 1, v >= 1); L >= 1 Cholesky vectors.
 *   fock      : n x n, symmetric (checked to 1e-12 relative).
 *   chol      : L x n x n, chol[K][p][q] == chol[K][q][p] (checked).
 *   t1        : o x v, t1[i][a] = t_i^a.
 *   t2        : o x o x v x v, t2[i][j][a][b] = t_ij^ab, antisymmetric in (i,j) and (a,b) (checked).
 *   lambda    : NULL for Lambda = T^dagger (lambda_a^i = t_i^a, lambda_ab^ij = t_ij^ab);
 *               otherwise o*v values lambda1[i][a] followed by o*o*v*v values lambda2[i][j][a][b].
 *   out       : receives the new context (NULL on error).
 * The T1 part of T is applied to the integrals (L' = (1-t) L (1+t), an orbital
 * rotation) and the T2 part gives the Hbar elements kept for the sigma product
 * (Implementation Details section: constant intermediates of size <= O(O^2 V^2),
 * plus the vvvv block when the EA sector is enabled).  Sector and precision
 * are fixed at creation: call gfcc_create_ex to choose them, gfcc_create builds both
 * sectors in FP64.
 */
int gfcc_create(int o, int v, int L, const double *fock, const double *chol,
                const double *t1, const double *t2, const double *lambda, gfcc_ctx **out);

/* gfcc_create_ex - gfcc_create with the sectors (GFCC_SECTOR_*) and precision (GFCC_PREC_*)
 * to build intermediates for. */
int gfcc_create_ex(int o, int v, int L, const double *fock, const double *chol,
                   const double *t1, const double *t2, const double *lambda,
                   int sectors, int precision, gfcc_ctx **out);

/* gfcc_create_rhf - closed-shell spin-adapted IP context (the paper's closed-shell GFCCSD-IP, Table 2:
 * alpha amplitudes only).  Spatial orbitals: o doubly occupied, v virtual; the Hamiltonian is the
 * spin-free one of a closed-shell reference (fock, chol spatial, as for gfcc_create).
 *   t1 [o][v] = t_i^a (alpha), t2 [o][o][v][v] = t_ij^ab = T_{i alpha, j beta}^{a alpha, b beta}, with
 *   t2[i][j][a][b] == t2[j][i][b][a] (checked); lambda: NULL (Lambda = T^dagger) or [lambda1 | lambda2]
 *   in the same spatial layout.
 * Sector IP, FP64.  G_pq(omega) over spatial orbitals equals the spin-orbital G of orbitals
 * p alpha, q alpha.  The systems are solved in the doublet coordinates r_i = R_{i alpha},
 * r_ij^a = R_{i alpha, j beta}^{a beta} (dimension o + o^2 v; gfcc_dims reports it, gfcc_sigma and
 * the solves take vectors in it: [r_i | r_ij^a at [i][j][a]]), with the spin-summed Hbar elements.
 * The operator's large contractions run as FP64-accurate digit-plane products on the tensor cores
 * unless GFCC_OPT_CLOSED_SHELL_EMULATE is 0.  Zero initial guesses only; model-order reduction is not
 * offered for these contexts.  Errors as gfcc_create.
 */
int gfcc_create_rhf(int o, int v, int L, const double *fock, const double *chol, const double *t1, const double *t2,
                    const double *lambda, gfcc_ctx **out);

/* gfcc_set_option - set one GFCC_OPT_* option (value cast from double).  Returns GFCC_ERR_ARG
 * for an unknown key or a value out of range. */
int gfcc_set_option(gfcc_ctx *ctx, int key, double value);

/* gfcc_set_process_option - set a process-wide option (GFCC_OPT_AUTOTUNE, GFCC_OPT_EMU_FUSED_N,
 * GFCC_OPT_SETUP_EMULATE_FLOPS, GFCC_OPT_WAIT_NS, GFCC_OPT_TEST_NO_LOADS, GFCC_OPT_GEMM_PAIR,
 * GFCC_OPT_GEMM_PERSIST).  It applies to every
 * later call of every context; do not change it while another thread is inside the library.
 * Returns GFCC_ERR_ARG for an unknown key or a value out of range. */
int gfcc_set_process_option(int key, double value);

/* gfcc_set_stream - run all of the context's work on `stream` (a cudaStream_t; NULL = the
 * context's own stream). */
int gfcc_set_stream(gfcc_ctx *ctx, void *stream);

/*
 * gfcc_solve - G(omega) for every omega in `omegas` and every (p, q) pair of `orbitals`.
 *   omegas   : n_omega frequencies (Hartree).  eta > 0 broadening.  tol > 0: a column is
 *              converged when ||b - A x||_2 <= tol ||b||_2 (true residual, packed coordinates).
 *   orbitals : n_orb indices in [0, o+v); p and q both run over this list.
 *   G        : out, complex128 interleaved (re, im), [n_omega][n_orb (p)][n_orb (q)], caller-allocated
 *              host memory of 2*n_omega*n_orb*n_orb doubles; G = G^IP + G^EA for the enabled sectors.
 * Returns GFCC_OK, GFCC_WARN_NOT_CONVERGED (G written, some columns missed tol), or an error.
 */
int gfcc_solve(gfcc_ctx *ctx, int n_omega, const double *omegas, double eta,
               int n_orb, const int *orbitals, double tol, double *G);

/*
 * gfcc_solve_block - the block of G(omega) with rows p over p_orbitals and columns q over q_orbitals
 * (eqs. gfxn2/gfxn3): G[w][a][b] = G^IP_{p_a q_b}(omega_w) + G^EA_{p_a q_b}(omega_w).  The IP systems
 * X_p (eq. xp) are solved for the row orbitals and overlapped with the left vectors of the column
 * orbitals; the EA systems Y_q (eq. yq) are solved for the column orbitals and overlapped with the
 * left vectors of the row orbitals.  gfcc_solve(orbitals) is gfcc_solve_block(orbitals, orbitals).
 *   G : out, host complex128 interleaved, [n_omega][n_p][n_q], caller-allocated.
 * Statistics (gfcc_last_stats): the IP systems (omega-major over p_orbitals), then the EA systems
 * (omega-major over q_orbitals).  Return codes and errors as gfcc_solve.
 */
int gfcc_solve_block(gfcc_ctx *ctx, int n_omega, const double *omegas, double eta, int n_p, const int *p_orbitals,
                     int n_q, const int *q_orbitals, double tol, double *G);

/* gfcc_solve_device - gfcc_solve with omegas, orbitals and G in DEVICE memory (same layouts);
 * the call is asynchronous on the context's stream except for the per-iteration
 * convergence checks, which synchronise it. */
int gfcc_solve_device(gfcc_ctx *ctx, int n_omega, const double *omegas_dev, double eta,
                      int n_orb, const int *orbitals_dev, double tol, double *G_dev);

/* One request of gfcc_solve_batch: the arguments of gfcc_solve (host arrays). */
typedef struct gfcc_request {
  int n_omega;
  const double *omegas;
  double eta;
  int n_orb;
  const int *orbitals;
  double tol;
  double *G;        /* out: as gfcc_solve */
} gfcc_request;

/*
 * gfcc_solve_batch - gfcc_solve on several contexts (molecules of different sizes) at once: each
 * context solves its request on its own stream from one of up to 8 host threads, so small problems
 * share the GPU (Algorithm 1's task list over molecules; the paper runs them on separate process
 * groups).  Contexts must be distinct and on the device current at the call; while they run, each
 * plans its batch for its share of the free device memory.  codes (optional, n_ctx entries) gets
 * every context's return code; the call returns GFCC_OK, GFCC_WARN_NOT_CONVERGED, or the first
 * error (gfcc_last_error names the context).
 */
int gfcc_solve_batch(gfcc_ctx *const *ctxs, int n_ctx, const gfcc_request *reqs, int *codes);

/*
 * gfcc_last_stats - statistics of the last gfcc_solve, one entry per (sector, omega, orbital)
 * in the order IP then EA, omega-major: `iters` sigma products, `relres` final true relative
 * residual, `status` GFCC_STATUS_*.  Any pointer may be NULL; `count` (in/out) is the capacity
 * on input and the number of entries on output.
 */
int gfcc_last_stats(gfcc_ctx *ctx, int *count, int *iters, double *relres, int *status);

/*
 * gfcc_sigma - apply the sigma product sigma(x) = <mu|[Hbar, X]|Phi> (the Hbar part of eq. xplin)
 * to n_vec packed complex vectors.  sector GFCC_SECTOR_IP or GFCC_SECTOR_EA.
 *   x, y : host, complex128 interleaved, [n_vec][dim]; dim = o + o(o-1)/2 * v (IP, packed
 *          order: 1h i, then pairs i<j lexicographic with a fastest) or v + o * v(v-1)/2
 *          (EA: 1p a, then i-major with pairs a<b lexicographic).
 * Uses the FP64 sigma regardless of the precision option.
 */
int gfcc_sigma(gfcc_ctx *ctx, int sector, int n_vec, const double *x, double *y);

/* gfcc_sigma_ex - gfcc_sigma in a chosen precision: GFCC_PREC_FP64; GFCC_PREC_MIXED_BF16 (IP only,
 * context created mixed): the couplings on the BF16 tensor cores with FP32 accumulation, the
 * Fock-like diagonal in FP64; GFCC_PREC_FP64_EMULATED (IP only, context created mixed): the
 * FP64-accurate sigma of the refinement residual (digit planes on the tensor cores). */
int gfcc_sigma_ex(gfcc_ctx *ctx, int sector, int precision, int n_vec, const double *x, double *y);

/*
 * gfcc_sigma_noalloc - the FP64 sigma product of gfcc_sigma on DEVICE buffers, without allocating
 * any memory.  The paper has no counterpart: this entry point exists for callers that cannot
 * allocate device memory on their call path, such as an application whose device memory is all
 * reserved up front by its own pool allocator (a cudaMalloc there fails or fragments the pool), or
 * a latency-critical path where cudaMalloc / cudaFree would synchronise the device and stall the
 * application's other streams.
 *   x_dev, y_dev : device, complex128 interleaved, [n_vec][dim] in the packed order of gfcc_sigma.
 * The workspace is a fixed array of 2^22 doubles (32 MiB) inside the library, present on every GPU
 * that loads it until the process exits; sizes that need more (or a contraction longer than 8191
 * elements, o*o*v for IP, o*v*v for EA) return GFCC_ERR_ARG.  The first call on a device looks the
 * array's device address up; make that first call before any stream capture.  All calls share the
 * array, so calls whose executions overlap on the GPU race: serialise them.  Runs on the context's
 * stream and returns after it has finished.
 */
int gfcc_sigma_noalloc(gfcc_ctx *ctx, int sector, int n_vec, const double *x_dev, double *y_dev);

/* gfcc_dims - packed dimensions of the IP and EA spaces of the context. */
int gfcc_dims(gfcc_ctx *ctx, long long *dim_ip, long long *dim_ea);

/*
 * Profiling.  gfcc_profile(ctx, 1) resets the counters and times every later solve phase with CUDA
 * events on the context's stream (gfcc_profile(ctx, 0) stops).  gfcc_profile_read returns, for one
 * phase, the summed device time in milliseconds, the number of timed regions and the algorithmic
 * floating-point operations they performed (counted from the problem sizes, not measured; for
 * phase 4 the count is algorithmic bytes of one classical Gram-Schmidt pass instead).
 * Phases: 0 setup (gfcc_create), 1 ring contraction of the sigma product, 2 EA vvvv contraction,
 * 3 whole sigma products (contains 1 and 2), 4 Arnoldi orthogonalisation, 5 Givens / least squares,
 * 6 right-hand sides, left vectors and overlaps, 7 whole gfcc_solve calls, 8 ring contraction on the
 * BF16 tensor cores (mixed precision; phase 1 is the FP64 ring contraction), 9 FP64-accurate ring
 * contraction of the refinement residual (digit planes; flops of the one FP64 product it evaluates), 10
 * expansion of packed vectors into contraction layouts, 11 initial guesses (Gram matrices, model,
 * combination), 12 the other FP64-accurate products of the refinement residual (oooo / vvvv,
 * three-body, 1h / 1p row; FP64 product flops), 13 the other BF16 products of the inner sigma (oooo,
 * three-body, 1h / 1p row), 14 sigma epilogues (shift, diagonal, packing; count = algorithmic bytes),
 * 15 the same region as phase 9 with the BF16 tensor-core work of all its digit pairs as the count.
 */
int gfcc_profile(gfcc_ctx *ctx, int enable);
int gfcc_profile_read(gfcc_ctx *ctx, int phase, double *ms, long long *count, double *flops);

/* gfcc_launch_count - number of CUDA kernels this library has launched in this process. */
long long gfcc_launch_count(void);

/*
 * gfcc_selftest_gemm_bf16 - run the tensor-core contraction engine of the mixed-precision sigma
 * product alone: D[M][N] = sum_k bf16(A[m][k]) bf16(B[n][k]) with FP32 accumulation.
 * A (M x K), B (N x K) and D (M x N) are row-major FP32 HOST arrays; the inputs are rounded to
 * BF16 (nearest even) on the host.  GFCC_ERR_TIMEOUT if a bounded device wait gave up.
 */
int gfcc_selftest_gemm_bf16(int M, int N, int K, const float *A, const float *B, float *D);

/*
 * gfcc_selftest_gemm_f64emu - the FP64-accurate product C[M][N] = sum_k A[m][k] B[n][k] computed from
 * S base-64 digit planes per operand on the BF16 tensor cores, keeping digit pairs i + j <= P
 * (Ozaki-Ogita-Oishi-Rump splitting; the error per term is about 2^-(6P-4) of the row scales).
 * A (M x K), B (N x K), C (M x N): row-major FP64 HOST arrays.
 */
int gfcc_selftest_gemm_f64emu(int M, int N, int K, const double *A, const double *B, int S, int P, double *C);

/*
 * gfcc_guess_stats - initial-guess statistics of the last gfcc_solve, in the entry order of
 * gfcc_last_stats: `kind` the GFCC_GUESS_* actually used, `pred` the predicted
 * ||b - A x0||^2 / ||b||^2 from the Gram matrix (1 for a zero guess), `relres0` the measured
 * ||b - A x0|| / ||b|| of the first true residual (FP64).  Pointers may be NULL; `count` as in
 * gfcc_last_stats.
 */
int gfcc_guess_stats(gfcc_ctx *ctx, int *count, int *kind, double *pred, double *relres0);

/* gfcc_refine_stats - mixed precision: per statistics entry of the last gfcc_solve, the number of
 * FP64-accurate residuals evaluated for the system (refinement steps + 1; 0 for FP64 sectors).
 * `count` as in gfcc_last_stats. */
int gfcc_refine_stats(gfcc_ctx *ctx, int *count, int *outer);

/* gfcc_residual_stats - mixed precision: FP64-accurate residual products of the last gfcc_solve (one
 * per batch evaluation): `full` of b - A x at the context's digit level, `incremental` of r -= A d,
 * and the mean digit level of the incremental ones (0 when there were none).  Any pointer may be
 * NULL.  Errors: GFCC_ERR_ARG for a NULL ctx. */
int gfcc_residual_stats(gfcc_ctx *ctx, long long *full, long long *incremental, double *mean_level);

/*
 * The learned-guess model: a 3-layer perceptron with ReLU activations,
 *     x^ = (x - mu) / sd,  h1 = relu(W1 x^ + b1),  h2 = relu(W2 h1 + b2),  y = W3 h2 + b3,
 * from the 27 features of a system (omega, eta, p / n, delta_k = omega - omega_k for the 8
 * neighbours nearest first, then Re and Im of <b|X_k> * eta / ||b||^2) to its 8 complex mixing
 * coefficients c_k = y_2k + i y_2k+1.  It is trained on the method's own converged solutions:
 * the loss of a sample is the predicted relative residual a^H Gm a / Gm_00 of its combination,
 * with a = (sum_k c_k - 1, c_1, ..., c_8) and Gm the 9 x 9 Gram matrix of
 * (b, delta_1 X_1, ..., delta_8 X_8) (complex, Gm[j][l] = <u_j, u_l>, conjugate-linear in the
 * first argument).  Optimiser: Adam (beta1 0.9, beta2 0.999, eps 1e-8).
 * Parameter layout (doubles, row-major): W1 [hidden][27], b1 [hidden], W2 [hidden][hidden],
 * b2 [hidden], W3 [16][hidden], b3 [16], mu [27], sd [27] (mu, sd are not trained).
 * A model lives on the device current at creation; calls on one model must not overlap, and a
 * model attached to a context must not be trained while that context solves.
 */
#define GFCC_MLP_FP32  0          /* FP32 master weights and training; FP16 weights for inference         */
#define GFCC_MLP_FP64  1          /* FP64 throughout (gradient checks)                                     */
#define GFCC_MLP_FEATURES 27
#define GFCC_MLP_OUTPUTS  16

typedef struct gfcc_mlp gfcc_mlp;

/* gfcc_mlp_create - new model with `hidden` (1..256) units per hidden layer.  init_params: host,
 * gfcc_mlp_num_params doubles in the layout above (the caller draws the initial weights; the mu /
 * sd entries are ignored and set from the samples at the first gfcc_mlp_train). */
int gfcc_mlp_create(int hidden, int precision, const double *init_params, gfcc_mlp **out);
void gfcc_mlp_destroy(gfcc_mlp *m);
long long gfcc_mlp_num_params(const gfcc_mlp *m);
/* gfcc_mlp_get_params / gfcc_mlp_set_params - host copies of all parameters (set also fixes mu, sd;
 * every sd must be non-zero). */
int gfcc_mlp_get_params(gfcc_mlp *m, double *params);
int gfcc_mlp_set_params(gfcc_mlp *m, const double *params);
/* gfcc_mlp_forward - y [nb][16] of features [nb][27] (host arrays) with the inference weights. */
int gfcc_mlp_forward(gfcc_mlp *m, int nb, const double *features, double *y);
/* gfcc_mlp_loss_grad - mean loss over a batch (features [nb][27], gram [nb][9][9] complex
 * interleaved; host) and its gradient with respect to every parameter (grad: host,
 * gfcc_mlp_num_params doubles; zero for mu, sd), in the training precision. */
int gfcc_mlp_loss_grad(gfcc_mlp *m, int nb, const double *features, const double *gram, double *loss, double *grad);
/* gfcc_mlp_train_batch - one Adam step with learning rate lr on the given batch; *loss = the
 * batch's mean loss before the step. */
int gfcc_mlp_train_batch(gfcc_mlp *m, int nb, const double *features, const double *gram, double lr, double *loss);
/* gfcc_mlp_collect - add training samples from the kept solutions of a context (after a gfcc_solve
 * with GFCC_OPT_KEEP_SOLUTIONS or a guess): for every converged (omega, p), samples_per_system
 * samples whose neighbours are the 8 nearest among a random subset of the other converged
 * frequencies (keep probability drawn in [0.15, 1) per sample; `seed` drives the draws).
 * *added = samples added (systems with fewer than 8 neighbours in the subset give none). */
int gfcc_mlp_collect(gfcc_mlp *m, gfcc_ctx *ctx, int samples_per_system, unsigned long long seed, long long *added);
long long gfcc_mlp_num_samples(const gfcc_mlp *m);
/* gfcc_mlp_get_samples - host copies of collected samples [start, start + count): features
 * [count][27] and Gram matrices [count][9][9] complex interleaved (either pointer may be NULL).
 * A sample's neighbours are identified by its features: omega_k = omega - delta_k, p = (p/n) n. */
int gfcc_mlp_get_samples(gfcc_mlp *m, long long start, int count, double *features, double *gram);
/* gfcc_mlp_train - `steps` Adam steps on minibatches of the collected samples (drawn with
 * replacement from `seed`).  *loss = mean minibatch loss over the last (up to) 50 steps. */
int gfcc_mlp_train(gfcc_mlp *m, int steps, int minibatch, double lr, unsigned long long seed, double *loss);
/* gfcc_mlp_eval - over the collected samples, with the inference weights: out[0] mean model loss,
 * out[1] mean loss after the zero-guess fallback (min(loss, 1)), out[2] mean loss of the
 * minimal-residual coefficients (clamped to [0, 1]), out[3] fraction of samples where the model
 * beats the zero guess. */
int gfcc_mlp_eval(gfcc_mlp *m, double *out);
/* gfcc_set_guess_model - model used by GFCC_GUESS_LEARNED (not owned; NULL detaches). */
int gfcc_set_guess_model(gfcc_ctx *ctx, gfcc_mlp *m);

/*
 * Model-order reduction (Theory section, eq. model; Algorithm 1: Gram-Schmidt, projection and the
 * spectral function after the frequency loop of a level).  A gfcc_mor object holds, for one sector
 * of a context, a real orthonormal subspace S = {v_1 .. v_m} of the packed space (spanned by the real
 * and imaginary parts of converged solutions X_p(omega_k) or Y_q(omega_k); Hbar, b and c are real,
 * so S^T of eq. model is the plain transpose), W = Hbar_N S and Hhat = S^T Hbar_N S (m x m).  The
 * model systems
 *     IP: (omega - i eta + Hhat) Xhat = S^T b_p,  G_pq = (S^T c_q)^T Xhat
 *     EA: (omega + i eta - Hhat) Yhat = S^T b_q,  G_pq = (S^T c_p)^T Yhat
 * are solved densely on the GPU for any frequency grid; at every frequency whose solutions entered S
 * they reproduce the full G (to the solver tolerance).  The object uses its context's stream and
 * must not be used concurrently with it; destroy it before the context.
 */
typedef struct gfcc_mor gfcc_mor;

/* gfcc_mor_create - empty subspace for sector GFCC_SECTOR_IP or GFCC_SECTOR_EA of ctx (the sector must
 * be built).  drop_tol (0 < drop_tol < 1): a new vector is kept when the norm left after two
 * Gram-Schmidt passes exceeds drop_tol times its norm (1e-10 is a good default). */
int gfcc_mor_create(gfcc_ctx *ctx, int sector, double drop_tol, gfcc_mor **out);
/* gfcc_mor_destroy - free the object and its device memory.  NULL is a no-op. */
void gfcc_mor_destroy(gfcc_mor *mor);
/* gfcc_mor_dim - the subspace dimension m (-1 for NULL). */
int gfcc_mor_dim(gfcc_mor *mor);
/*
 * gfcc_mor_expand - solve the full systems of the object's sector for every omega x orbital (the
 * context's solver and options, as gfcc_solve with that sector only), then orthonormalise the real
 * and imaginary parts of every converged solution into S (O(m^2 O^2 V)) and project the operator on
 * the new basis vectors (their sigma products, O(m O^3 V^2)).  G (optional, host, as gfcc_solve for
 * that sector alone) receives the full G at these frequencies.  Returns GFCC_OK or
 * GFCC_WARN_NOT_CONVERGED (unconverged systems do not enter S; gfcc_last_stats says which), or an error.
 */
int gfcc_mor_expand(gfcc_mor *mor, int n_omega, const double *omegas, double eta, int n_orb, const int *orbitals,
                    double tol, double *G);
/*
 * gfcc_mor_green - the model G block on a frequency grid: G[w][a][b] for rows p_orbitals[a] and columns
 * q_orbitals[b] (host, complex128 interleaved, [n_omega][n_p][n_q]; the object's sector only), by one
 * dense LU solve per frequency (O(N_omega m^3)).  relres (optional, host): the relative full-space
 * residual ||b - A(omega) S Xhat|| / ||b|| of every model solution ([n_omega][n_p] for IP, [n_omega][n_q]
 * for EA; from W, without a sigma product; needs m <= 1024).
 */
int gfcc_mor_green(gfcc_mor *mor, int n_omega, const double *omegas, double eta, int n_p, const int *p_orbitals,
                   int n_q, const int *q_orbitals, double *G, double *relres);
/* gfcc_mor_projected - host copies of Hhat (m x m row-major; may be NULL) and of the first row_count
 * basis vectors (row_count x dim row-major; may be NULL). */
int gfcc_mor_projected(gfcc_mor *mor, double *Hhat, double *S_rows, int row_count);

/*
 * gfcc_spectral_adaptive - the spectral function (eq. specfxn) over [omega_min, omega_max] from the
 * model-order reduction built level by level (Algorithm 1's outer loop; Implementation Details,
 * eq. Lmax).  Level 1 solves omega_min, the midpoint and omega_max; each later level L solves, for all
 * orbitals, the midpoints of adjacent sampled frequencies (at most 2^(L-1); a midpoint is a candidate
 * when its half-interval is at least d_omega, which bounds the levels by log2((omega_max -
 * omega_min) / d_omega)) whose largest relative model residual over the orbitals and sectors exceeds
 * level_tol, the largest first; it stops when no candidate exceeds level_tol or after max_levels
 * (1..30).  Each level's solutions expand one subspace per sector in `sectors` (GFCC_SECTOR_*).
 *   A            : out [n_fine], A(omega) = (1/pi) sum_p (Im G^IP_pp - Im G^EA_pp) over `orbitals`
 *                  from the final models (the paper's -(1/pi) Tr Im G^R, with the IP resolvent's
 *                  -i eta and the EA resolvent's +i eta of eq. gfxn1, so A > 0 near every pole).
 *   n_levels     : out, levels run; level_sizes: out [max_levels], frequencies per level;
 *   sampled      : out, the sampled frequencies in sampling order (up to sampled_cap);
 *   mdim         : out [2], subspace dimensions (IP, EA; 0 for a sector not requested).
 * Any output pointer but A may be NULL.  Returns GFCC_OK, GFCC_WARN_NOT_CONVERGED (a full system missed
 * tol; its solution was left out of the subspace) or an error.
 */
int gfcc_spectral_adaptive(gfcc_ctx *ctx, int sectors, double omega_min, double omega_max, double d_omega,
                           double eta, int n_orb, const int *orbitals, double tol, double level_tol, int max_levels,
                           int n_fine, const double *fine_omegas, double *A, int *n_levels, int *level_sizes,
                           double *sampled, int sampled_cap, int *mdim);

/* ---------------------------------------------------------------- ground state (the step before G)
 * gfcc_ccsd - solve the ground-state CCSD equations for T and, when lambda is given, the Lambda-CCSD
 * equations for the de-excitation amplitudes, on the device (FP64; Theory section: T and Lambda come
 * from the conventional CC equations, which the Green's function then takes as fixed inputs;
 * Workflow section and Table 1: Cholesky-decomposed CCSD, O(O^2 V^4) per iteration).  The integrals
 * enter only through the Cholesky vectors; the vvvv ladder term is formed block by block.
 *   o, v, L, fock, chol : the Hamiltonian, as for gfcc_create (host, row-major; fock symmetric, chol
 *                 symmetric in its orbital pair; checked on the device).
 *   tol         : convergence when max |residual| <= tol (every singles and doubles equation).
 *   max_iter    : iterations per equation set (>= 1); Jacobi steps with the Fock-diagonal denominators
 *                 f_ii (+ f_jj) - f_aa (- f_bb), extrapolated by DIIS over the last 8 iterates.
 *   flags       : GFCC_CCSD_EMULATE - contractions of at least 1e10 flops (or the setup threshold
 *                 GFCC_OPT_SETUP_EMULATE_FLOPS when that is lower) through the FP64-accurate digit-plane
 *                 products on the BF16 tensor cores; GFCC_CCSD_GUESS - t1, t2 (and lambda) hold initial iterates on entry
 *                 (else both start from zero, Lambda from T).
 *   t1 [o][v], t2 [o][o][v][v] : out (in with GFCC_CCSD_GUESS), host; t2 antisymmetric.
 *   lambda      : NULL (T only) or out [lambda1 (o x v) | lambda2 (o x o x v x v)], the layout
 *                 gfcc_create takes (lambda_a^i at [i][a], lambda_ab^ij at [i][j][a][b]).
 *   info        : out [8], may be NULL: E_corr (Hartree; f_ia t_i^a + 1/4 <ij||ab> t_ij^ab +
 *                 1/2 <ij||ab> t_i^a t_j^b), T iterations, final max |T residual|, Lambda iterations,
 *                 final max |Lambda residual|, seconds in the T iterations, seconds in the Lambda
 *                 iterations (both host-timed, stream-synchronised), FP64 multiply-adds x 2 of one T
 *                 iteration (the counted contraction flops).
 * Both equation sets are taken in their T1 = 0 forms for the T1-rotated Hamiltonian (whose T2
 * transform is e^-T H e^T exactly); the Lambda residuals leave out the terms that vanish when T
 * solves its equations.
 * Returns GFCC_OK, GFCC_WARN_NOT_CONVERGED (outputs hold the last iterate), GFCC_ERR_ARG (sizes, NULL
 * inputs, tol <= 0, bad symmetry), GFCC_ERR_OOM or GFCC_ERR_CUDA.  Device memory: about
 * (2 * 8 + 6) o^2 v^2 + o v^3 + 2 L (o + v)^2 doubles plus a 4 GB vvvv block; freed before returning.
 */
#define GFCC_CCSD_EMULATE 1
#define GFCC_CCSD_GUESS 2
int gfcc_ccsd(int o, int v, int L, const double *fock, const double *chol, double tol, int max_iter, int flags,
              double *t1, double *t2, double *lambda, double *info);

/* gfcc_solve_checkpoint - gfcc_solve with each frequency's G block written to the file `path` as
 * soon as it is solved, and resumed from it (Algorithm 1 writes each task's output; the Evaluation
 * section restarts long jobs).  A call whose file holds the checkpoint of the same request (same
 * frequencies, orbitals, eta, tol, and a context with the same sectors, precision and kind) restores
 * the finished frequencies into G without solving them and solves the others, one frequency per
 * internal solve; a record cut short by a killed job is dropped.  The file is created when absent.
 *   path      : file name (host string); path + ".tmp" is used while the file is rewritten.
 *   n_resumed : out (may be NULL), frequencies restored from the file.
 *   G         : out, as gfcc_solve.
 * Returns as gfcc_solve (WARN_NOT_CONVERGED also when a restored frequency had it); GFCC_ERR_ARG
 * when the file holds something else (it is left untouched) or cannot be written.  gfcc_last_stats
 * describes the last frequency solved in this call.
 */
int gfcc_solve_checkpoint(gfcc_ctx *ctx, int n_omega, const double *omegas, double eta, int n_orb, const int *orbitals,
                          double tol, const char *path, int *n_resumed, double *G);

/* gfcc_destroy - free the context and all its device memory.  NULL is a no-op. */
void gfcc_destroy(gfcc_ctx *ctx);

/* gfcc_last_error - message of the last failing call on this thread ("" if none). */
const char *gfcc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GFCC_H */
