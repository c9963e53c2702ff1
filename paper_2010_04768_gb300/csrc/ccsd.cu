// Ground-state CCSD and Lambda-CCSD on the device (FP64, Cholesky-vector integrals).
//
// The Green's function takes T and Lambda from the conventional ground-state CC equations (Theory
// section); the paper solves them with Cholesky-decomposed integrals at O(O^2 V^4) per iteration
// (Workflow section, Table 1).  Route, shared with the setup of the Hbar elements: T1 enters as the
// orbital rotation L'^K = (1-t) L^K (1+t), h' = (1-t) h (1+t), f' = h' + J' - K' (t[o+a][i] = t_i^a),
// and e^-T2 H' e^T2 gives the T1 = 0 forms of the spin-orbital equations in the rotated basis.
//
// T equations (<pq||rs>' = (pr|qs)' - (ps|qr)', (pr|qs)' = sum_K L'^K_pr L'^K_qs):
//   Omega1_ia   = f'_ai + f'_me t_im^ae + sum_mef (ae|mf)' t_im^ef + sum_mne (me|ni)' t_mn^ae
//   Omega2_ijab = <ab||ij>' + P(ab) F_be t_ij^ae - P(ij) F_mj t_im^ab + 1/2 (<mn||ij>' + 1/2 Z_mnij) t_mn^ab
//                 + sum_ef (ae|bf)' t_ij^ef + P(ij) P(ab) W_mbej t_im^ae
//   F_be = f'_be - 1/2 <mn||ef>' t_mn^bf,  F_mj = f'_mj + 1/2 <mn||ef>' t_jn^ef,  Z_mnij = <mn||ef>' t_ij^ef,
//   W_mbej = <mb||ej>' - 1/2 <mn||ef>' t_jn^fb.
// The antisymmetry of t2 folds 1/2 <am||ef>' t_im^ef, 1/2 <mn||ei>' t_mn^ae and 1/2 <ab||ef>' t_ij^ef
// into single Coulomb-like sums, and the two quarter-weighted quadratic terms of the oooo and vvvv
// intermediates into one; the singles sums run through the Cholesky index (O(L O^2 V^2)), and the vvvv
// ladder through blocks of (ae|bf)' for a range of a (never the whole v^4 block).
//
// Lambda equations (T fixed; the terms proportional to the T residuals dropped), with the Hbar
// elements of e^-T2 H' e^T2 (the setup's forms):
//   0 = Fb_ia + l_ie Fb_ea - l_ma Fb_im + l_me Wb_ieam + 1/2 l_imef Wb_efam - 1/2 l_mnae Wb_iemn
//       - G_ef Wb_eifa - G_mn Wb_mina
//   0 = <ij||ab>' + P(ab) l_ijae Fb_eb - P(ij) l_imab Fb_jm + 1/2 l_mnab Wb_ijmn + 1/2 l_ijef Wb_efab
//       + P(ij) l_ie Wb_ejab - P(ab) l_ma Wb_ijmb + P(ij) P(ab) (l_imae Wb_jebm + l_ia Fb_jb)
//       + P(ab) <ij||ae>' G_be - P(ij) <im||ab>' G_mj
//   G_ae = -1/2 t_mn^ef l_mnaf,  G_mi = 1/2 t_mn^ef l_inef.
// Wb_eifa = <ei||fa>' and Wb_ejab = <ej||ab>' enter through the Cholesky index; Wb_efab through the
// same (ea|fb)' blocks as the T ladder plus 1/4 (l_ijef t_mn^ef) <mn||ab>'.
//
// Solver: Jacobi steps x + Omega / D (D from the Fock diagonal), then DIIS (Pulay) over the last 8
// iterates: the coefficients minimise |sum_k c_k e_k| with sum_k c_k = 1, e_k = Omega_k / D.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "ctx.cuh"
#include "kernels.cuh"

namespace gfcc {

namespace {

constexpr int RED_BLOCKS = 304;   // reduction grids: two blocks per SM
constexpr int RED_THREADS = 256;
constexpr int DIIS_CAP = 8;
constexpr double CCSD_EMULATE_MIN_FLOPS = 1e10;   // GFCC_CCSD_EMULATE: digit planes from this size up

__global__ void diag_copy_kernel(const double *F, int n, double *eps) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) eps[p] = F[(long long)p * n + p];
}

// R[i][j][a][b] += alpha * (X[ijab] - X[jiab] - X[ijba] + X[jiba])
__global__ void antisym4_add_kernel(double *R, const double *X, int o, int v, double alpha) {
  const long long vv = (long long)v * v, ov2 = (long long)o * vv, tot = (long long)o * ov2;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < tot; x += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(x % v);
    const int a = (int)((x / v) % v);
    const long long ij = x / vv;
    const int j = (int)(ij % o), i = (int)(ij / o);
    const long long ji = (long long)j * o + i;
    const double s = X[x] - X[ji * vv + (long long)a * v + b] - X[ij * vv + (long long)b * v + a] +
                     X[ji * vv + (long long)b * v + a];
    R[x] += alpha * s;
  }
}

// Jacobi step of x = [x1 (o x v) | x2 (o x o x v x v)] with residual r: e = r / D into E, and
// X = [x1 + e1 | antisymmetrised x2 + e2] (the quarter sum over the four index swaps)
__global__ void jacobi_kernel(const double *x, const double *r, const double *eps, int o, int v, double *E,
                              double *X) {
  const long long ov = (long long)o * v, vv = (long long)v * v, tot = ov + ov * ov;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < tot; k += (long long)gridDim.x * blockDim.x) {
    if (k < ov) {
      const int i = (int)(k / v), a = (int)(k % v);
      const double e = r[k] / (eps[i] - eps[o + a]);
      E[k] = e;
      X[k] = x[k] + e;
      continue;
    }
    const long long q = k - ov;
    const int b = (int)(q % v);
    const int a = (int)((q / v) % v);
    const long long ij = q / vv;
    const int j = (int)(ij % o), i = (int)(ij / o);
    const double d = eps[i] + eps[j] - eps[o + a] - eps[o + b];
    const double *x2 = x + ov, *r2 = r + ov;
    const long long ji = (long long)j * o + i;
    const long long p1 = q, p2 = ji * vv + (long long)a * v + b, p3 = ij * vv + (long long)b * v + a,
                    p4 = ji * vv + (long long)b * v + a;
    E[k] = r2[p1] / d;
    X[k] = 0.25 * ((x2[p1] + r2[p1] / d) - (x2[p2] + r2[p2] / d) - (x2[p3] + r2[p3] / d) + (x2[p4] + r2[p4] / d));
  }
}

template <int OP>   // 0: dot products of enew with the rows 0..cnt-1 of H; 1: max |enew|
__global__ void reduce_kernel(const double *H, long long N, int cnt, const double *enew, double *partial) {
  double acc[DIIS_CAP];
#pragma unroll
  for (int j = 0; j < DIIS_CAP; j++) acc[j] = 0.0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < N; k += (long long)gridDim.x * blockDim.x) {
    const double e = enew[k];
    if (OP == 1) {
      acc[0] = fmax(acc[0], fabs(e));
    } else {
#pragma unroll
      for (int j = 0; j < DIIS_CAP; j++)
        if (j < cnt) acc[j] += e * H[(long long)j * N + k];
    }
  }
  __shared__ double sh[RED_THREADS];
  const int nred = OP == 1 ? 1 : cnt;
  for (int j = 0; j < nred; j++) {
    sh[threadIdx.x] = acc[j];
    __syncthreads();
    for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w)
        sh[threadIdx.x] = OP == 1 ? fmax(sh[threadIdx.x], sh[threadIdx.x + w]) : sh[threadIdx.x] + sh[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) partial[(long long)j * gridDim.x + blockIdx.x] = sh[0];
    __syncthreads();
  }
}

struct Coef {
  double c[DIIS_CAP];
};

// out = sum_j c_j H[j]
__global__ void combine_kernel(const double *H, long long N, int cnt, Coef c, double *out) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < N; k += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < cnt; j++) s += c.c[j] * H[(long long)j * N + k];
    out[k] = s;
  }
}

// partial sums of f_ia t_i^a + sum_ijab V[ijab] (1/4 t2[ijab] + 1/2 t1[ia] t1[jb])
__global__ void energy_kernel(const double *F, const double *V, const double *t1, const double *t2, int o, int v,
                              double *partial) {
  const int n = o + v;
  const long long ov = (long long)o * v, vv = (long long)v * v, tot = ov * ov;
  double acc = 0.0;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < tot; x += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(x % v);
    const int a = (int)((x / v) % v);
    const long long ij = x / vv;
    const int j = (int)(ij % o), i = (int)(ij / o);
    acc += V[x] * (0.25 * t2[x] + 0.5 * t1[(long long)i * v + a] * t1[(long long)j * v + b]);
    if (x < ov) acc += F[(x / v) * n + o + (x % v)] * t1[x];
  }
  __shared__ double sh[RED_THREADS];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// Solve the (k+1) x (k+1) DIIS system [[B, -1], [-1, 0]] [c; lambda] = [0; -1] by Gaussian elimination
// with partial pivoting.  False when singular.
bool diis_solve(const double B[DIIS_CAP][DIIS_CAP], int k, double *c) {
  const int m = k + 1;
  double A[DIIS_CAP + 1][DIIS_CAP + 2];
  for (int r = 0; r < m; r++) {
    for (int q = 0; q < m; q++) A[r][q] = (r < k && q < k) ? B[r][q] : (r == k && q == k ? 0.0 : -1.0);
    A[r][m] = r == k ? -1.0 : 0.0;
  }
  for (int col = 0; col < m; col++) {
    int piv = col;
    for (int r = col + 1; r < m; r++)
      if (std::fabs(A[r][col]) > std::fabs(A[piv][col])) piv = r;
    if (!(std::fabs(A[piv][col]) > 0.0)) return false;
    if (piv != col)
      for (int q = 0; q <= m; q++) std::swap(A[piv][q], A[col][q]);
    for (int r = col + 1; r < m; r++) {
      const double f = A[r][col] / A[col][col];
      for (int q = col; q <= m; q++) A[r][q] -= f * A[col][q];
    }
  }
  double sol[DIIS_CAP + 1];
  for (int r = m - 1; r >= 0; r--) {
    double s = A[r][m];
    for (int q = r + 1; q < m; q++) s -= A[r][q] * sol[q];
    sol[r] = s / A[r][r];
    if (!std::isfinite(sol[r])) return false;
  }
  for (int j = 0; j < k; j++) c[j] = sol[j];
  return true;
}

struct Ccsd {
  cudaStream_t st = nullptr;
  int o = 0, v = 0, n = 0, L = 0;
  long long ov = 0, oo = 0, vv = 0, ov2 = 0, o2v = 0, v3 = 0, nn = 0, N = 0;
  std::vector<double *> owned;
  double flops = 0.0;   // counted contraction flops of the current residual evaluation

  // device arrays
  double *chol = nullptr, *fock = nullptr, *eps = nullptr, *h0 = nullptr, *V0 = nullptr;
  double *Lt = nullptr, *fp = nullptr;
  double *x = nullptr, *r = nullptr;          // [x1 | x2], [r1 | r2]
  double *tfix = nullptr;                      // [t1 | t2] held fixed during the Lambda iterations
  double *voovv = nullptr, *Foo = nullptr, *Fvv = nullptr, *Fov = nullptr, *Wmnij = nullptr, *Wr = nullptr;
  double *tmp4 = nullptr, *Yk = nullptr, *Xc = nullptr, *Zm = nullptr;
  double *Wooov = nullptr, *Q = nullptr, *R3 = nullptr, *vc = nullptr, *Gvv = nullptr, *Goo = nullptr;
  double *gK = nullptr;
  double *hx = nullptr, *he = nullptr, *part = nullptr;
  long long ac = 1, mc = 1;   // block sizes of the vvvv and ovvv blocks

  ~Ccsd() {
    for (double *p : owned) dfree(p);
  }
  int get(double **p, long long count) {
    GFCC_TRY(dev_alloc_tmp(p, count));
    owned.push_back(*p);
    return GFCC_OK;
  }
  int gemm(long long M, long long Nn, long long K, double alpha, const double *A, IMap am, IMap ak, const double *B,
           IMap bk, IMap bn, double beta, double *C, IMap cm, IMap cn, long long batch = 1, long long sab = 0,
           long long sbb = 0, long long scb = 0) {
    flops += 2.0 * (double)M * (double)Nn * (double)K * (double)batch;
    return gemm_f64(st, M, Nn, K, alpha, A, am, ak, B, bk, bn, beta, C, cm, cn, batch, sab, sbb, scb);
  }
  int eri(long long P0, long long np, long long R0, long long nr, long long Q0, long long nq, long long S0,
          long long ns, double alpha, double beta, double *C, IMap cm, IMap cn) {
    flops += 2.0 * (double)(np * nr) * (double)(nq * ns) * (double)L;
    return chol_eri(st, Lt, n, L, P0, np, R0, nr, Q0, nq, S0, ns, alpha, beta, C, cm, cn);
  }
  int copy(const double *src, long long count, double *dst) {
    GFCC_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * count, cudaMemcpyDeviceToDevice, st));
    return GFCC_OK;
  }
  int antisym_add(double *R, const double *X, double alpha) {
    antisym4_add_kernel<<<grid1d(oo * vv), 256, 0, st>>>(R, X, o, v, alpha);
    GFCC_LAUNCH_CHECK();
    return GFCC_OK;
  }

  int init(int o_, int v_, int L_, const double *h_fock, const double *h_chol) {
    o = o_; v = v_; L = L_; n = o + v;
    ov = (long long)o * v; oo = (long long)o * o; vv = (long long)v * v;
    ov2 = (long long)o * vv; o2v = oo * v; v3 = vv * v; nn = (long long)n * n;
    N = ov + ov * ov;
    GFCC_TRY(get(&chol, (long long)L * nn));
    GFCC_TRY(get(&fock, nn));
    GFCC_CUDA(cudaMemcpyAsync(chol, h_chol, sizeof(double) * L * nn, cudaMemcpyHostToDevice, st));
    GFCC_CUDA(cudaMemcpyAsync(fock, h_fock, sizeof(double) * nn, cudaMemcpyHostToDevice, st));
    GFCC_TRY(check_input_tensor(st, fock, 1, 1, n, n, 0, 1, 1.0, 1e-12, "fock"));
    GFCC_TRY(check_input_tensor(st, chol, 1, L, n, n, 0, 1, 1.0, 1e-12, "chol"));
    GFCC_TRY(get(&eps, n));
    diag_copy_kernel<<<cdiv(n, 128), 128, 0, st>>>(fock, n, eps);
    GFCC_LAUNCH_CHECK();
    GFCC_TRY(get(&h0, nn));
    GFCC_TRY(copy(fock, nn, h0));
    GFCC_TRY(chol_coulomb_exchange(st, chol, n, o, L, h0, -1.0, 1.0));   // h = f - J + K
    GFCC_TRY(get(&Lt, (long long)L * nn));
    GFCC_TRY(get(&fp, nn));
    GFCC_TRY(get(&x, N));
    GFCC_TRY(get(&r, N));
    GFCC_TRY(get(&tfix, N));
    GFCC_TRY(get(&voovv, oo * vv));
    GFCC_TRY(get(&Foo, oo));
    GFCC_TRY(get(&Fvv, vv));
    GFCC_TRY(get(&Fov, ov));
    GFCC_TRY(get(&Wmnij, oo * oo));
    GFCC_TRY(get(&Wr, ov * ov));
    GFCC_TRY(get(&tmp4, ov * ov));
    GFCC_TRY(get(&Yk, std::max<long long>((long long)L * ov, oo * oo)));
    GFCC_TRY(get(&Zm, oo * oo));
    ac = std::max<long long>(1, std::min<long long>(v, (1LL << 29) / std::max<long long>(1, v3)));
    GFCC_TRY(get(&Xc, ac * v3));
    GFCC_TRY(get(&hx, (long long)DIIS_CAP * N));
    GFCC_TRY(get(&he, (long long)DIIS_CAP * N));
    GFCC_TRY(get(&part, (long long)DIIS_CAP * RED_BLOCKS));
    // <ij||ab> of the unrotated integrals for the correlation energy
    GFCC_TRY(get(&V0, oo * vv));
    GFCC_TRY(chol_eri(st, chol, n, L, 0, o, o, v, 0, o, o, v, 1.0, 0.0, V0, imap2(v, v, ov2), imap2(v, 1, vv)));
    GFCC_TRY(chol_eri(st, chol, n, L, 0, o, o, v, 0, o, o, v, -1.0, 1.0, V0, imap2(v, 1, ov2), imap2(v, v, vv)));
    return GFCC_OK;
  }

  // Lt, fp and the blocks shared by the T and Lambda equations at amplitudes t = [t1 | t2]
  int rotate(const double *t) {
    const double *t1 = t, *t2 = t + ov;
    GFCC_TRY(copy(chol, (long long)L * nn, Lt));
    GFCC_TRY(t1_dress(st, t1, o, v, Lt, L, nn));
    GFCC_TRY(copy(h0, nn, fp));
    GFCC_TRY(t1_dress(st, t1, o, v, fp, 1, nn));
    GFCC_TRY(chol_coulomb_exchange(st, Lt, n, o, L, fp, 1.0, -1.0));   // f' = h' + J' - K'
    flops += 4.0 * (double)L * nn * n;
    // <mn||ef>' [m][n][e][f]
    GFCC_TRY(eri(0, o, o, v, 0, o, o, v, 1.0, 0.0, voovv, imap2(v, v, ov2), imap2(v, 1, vv)));
    GFCC_TRY(eri(0, o, o, v, 0, o, o, v, -1.0, 1.0, voovv, imap2(v, 1, ov2), imap2(v, v, vv)));
    // Fbar_oo[m][j] = f'_mj + 1/2 <mn||ef>' t_jn^ef;  Fbar_vv[b][e] = f'_be - 1/2 t_mn^bf <mn||ef>';  f'_ov
    {
      const long long d[4] = {1, 1, o, o}, is[4] = {0, 0, n, 1}, os[4] = {0, 0, o, 1};
      GFCC_TRY(permute4(st, d, fp, is, Foo, os, 1.0, 0.0));
      const long long d2[4] = {1, 1, v, v}, is2[4] = {0, 0, n, 1}, os2[4] = {0, 0, v, 1};
      GFCC_TRY(permute4(st, d2, fp + (long long)o * n + o, is2, Fvv, os2, 1.0, 0.0));
      const long long d3[4] = {1, 1, o, v}, is3[4] = {0, 0, n, 1}, os3[4] = {0, 0, v, 1};
      GFCC_TRY(permute4(st, d3, fp + o, is3, Fov, os3, 1.0, 0.0));
    }
    GFCC_TRY(gemm(o, o, ov2, 0.5, voovv, imap1(ov2), imap1(1), t2, imap1(1), imap1(ov2), 1.0, Foo, imap1(o),
                  imap1(1)));
    GFCC_TRY(gemm(v, v, oo * v, -0.5, t2, imap1(v), imap2(v, 1, vv), voovv, imap2(v, 1, vv), imap1(v), 1.0, Fvv,
                  imap1(v), imap1(1)));
    // Wmnij[m][n][i][j] = <mn||ij>' + 1/2 <mn||ef>' t_ij^ef  (the Hbar oooo element)
    const long long o3 = oo * o;
    GFCC_TRY(eri(0, o, 0, o, 0, o, 0, o, 1.0, 0.0, Wmnij, imap2(o, o, o3), imap2(o, 1, oo)));
    GFCC_TRY(eri(0, o, 0, o, 0, o, 0, o, -1.0, 1.0, Wmnij, imap2(o, 1, o3), imap2(o, o, oo)));
    GFCC_TRY(gemm(oo, oo, vv, 0.5, voovv, imap1(vv), imap1(1), t2, imap1(1), imap1(vv), 1.0, Wmnij, imap1(oo),
                  imap1(1)));
    return GFCC_OK;
  }

  // Wr[(j,b)][(m,e)] = <mb||ej>' - w <mn||ef>' t_jn^fb
  int ring_matrix(const double *t2, double w) {
    GFCC_TRY(eri(0, o, o, v, o, v, 0, o, 1.0, 0.0, Wr, imap1(1), imap2(o, ov2, ov)));          // (me|bj)
    GFCC_TRY(eri(0, o, 0, o, o, v, o, v, -1.0, 1.0, Wr, imap2(o, ov2, v), imap2(v, 1, ov)));   // -(mj|be)
    return gemm(ov, ov, ov, -w, t2, imap2(v, 1, ov2), imap2(v, v, vv), voovv, imap2(v, 1, vv), imap2(v, v, ov2), 1.0,
                Wr, imap1(ov), imap1(1));
  }

  // R2[ij][ab] += sum_ef B(a, e, b, f) A2[ij][ef] with B = (ae|bf)' (lam = false) or (ea|fb)' (lam = true)
  int ladder(const double *A2, double *R2, bool lam) {
    for (long long a0 = 0; a0 < v; a0 += ac) {
      const long long na = std::min<long long>(ac, v - a0);
      if (!lam) {
        GFCC_TRY(eri(o + a0, na, o, v, o, v, o, v, 1.0, 0.0, Xc, imap1(vv), imap1(1)));        // Xc[a][e][b][f]
      } else {
        GFCC_TRY(eri(o, v, o + a0, na, o, v, o, v, 1.0, 0.0, Xc, imap2(na, v3, vv), imap2(v, v, 1)));
      }
      GFCC_TRY(gemm(oo, na * v, vv, 1.0, A2, imap1(vv), imap1(1), Xc, imap2(v, 1, vv), imap2(v, v, v3), 1.0,
                    R2 + a0 * v, imap1(vv), imap1(1)));
    }
    return GFCC_OK;
  }

  // ---------------------------------------------------------------- T residual at t = [t1 | t2]
  int t_residual(const double *t, double *res) {
    const double *t1 = t, *t2 = t + ov;
    double *r1 = res, *r2 = res + ov;
    (void)t1;
    GFCC_TRY(rotate(t));
    // r1 = f'_ai + f'_me t_im^ae
    {
      const long long d[4] = {1, 1, o, v}, is[4] = {0, 0, 1, n}, os[4] = {0, 0, v, 1};
      GFCC_TRY(permute4(st, d, fp + (long long)o * n, is, r1, os, 1.0, 0.0));
    }
    GFCC_TRY(gemm(ov, 1, ov, 1.0, t2, imap2(v, v, ov2), imap2(v, 1, vv), Fov, imap1(1), imap1(0), 1.0, r1, imap1(1),
                  imap1(0)));
    // + sum_K sum_e L'_ae Y[K][i][e],  Y[K][i][e] = sum_mf L'_mf t_im^ef
    GFCC_TRY(gemm(ov, L, ov, 1.0, t2, imap2(v, v, ov2), imap2(v, 1, vv), Lt + o, imap2(v, 1, n), imap1(nn), 0.0, Yk,
                  imap1(1), imap1(ov)));
    GFCC_TRY(gemm(v, o, (long long)L * v, 1.0, Lt + (long long)o * n + o, imap1(n), imap2(v, 1, nn), Yk,
                  imap2(v, 1, ov), imap1(v), 1.0, r1, imap1(1), imap1(v)));
    // + sum_K sum_n L'_ni Y2[K][n][a],  Y2[K][n][a] = sum_me L'_me t_mn^ae
    GFCC_TRY(gemm(ov, L, ov, 1.0, t2, imap2(v, v, vv), imap2(v, 1, ov2), Lt + o, imap2(v, 1, n), imap1(nn), 0.0, Yk,
                  imap1(1), imap1(ov)));
    GFCC_TRY(gemm(v, o, (long long)L * o, 1.0, Yk, imap1(1), imap2(o, v, ov), Lt, imap2(o, n, nn), imap1(1), 1.0, r1,
                  imap1(1), imap1(v)));

    // r2 = <ab||ij>' = (ai|bj)' - (aj|bi)'
    GFCC_TRY(eri(o, v, 0, o, o, v, 0, o, 1.0, 0.0, r2, imap2(o, ov2, v), imap2(o, vv, 1)));
    GFCC_TRY(eri(o, v, 0, o, o, v, 0, o, -1.0, 1.0, r2, imap2(o, vv, v), imap2(o, ov2, 1)));
    // + P(ab) Fbar_be t_ij^ae
    GFCC_TRY(gemm(oo * v, v, v, 1.0, t2, imap1(v), imap1(1), Fvv, imap1(1), imap1(v), 1.0, r2, imap1(v), imap1(1)));
    GFCC_TRY(gemm(oo * v, v, v, -1.0, t2, imap1(v), imap1(1), Fvv, imap1(1), imap1(v), 1.0, r2, imap2(v, 1, vv),
                  imap1(v)));
    // - P(ij) Fbar_mj t_im^ab  (batched over i)
    GFCC_TRY(gemm(o, vv, o, -1.0, Foo, imap1(1), imap1(o), t2, imap1(vv), imap1(1), 1.0, r2, imap1(vv), imap1(1), o, 0,
                  ov2, ov2));
    GFCC_TRY(gemm(o, vv, o, 1.0, Foo, imap1(1), imap1(o), t2, imap1(vv), imap1(1), 1.0, r2, imap1(ov2), imap1(1), o, 0,
                  ov2, vv));
    // + 1/2 (<mn||ij>' + 1/2 Z_mnij) t_mn^ab
    GFCC_TRY(gemm(oo, vv, oo, 0.5, Wmnij, imap1(1), imap1(oo), t2, imap1(vv), imap1(1), 1.0, r2, imap1(vv), imap1(1)));
    // + sum_ef (ae|bf)' t_ij^ef
    GFCC_TRY(ladder(t2, r2, false));
    // + P(ij) P(ab) W_mbej t_im^ae,  W_mbej = <mb||ej>' - 1/2 <mn||ef>' t_jn^fb
    GFCC_TRY(ring_matrix(t2, 0.5));
    GFCC_TRY(gemm(ov, ov, ov, 1.0, t2, imap2(v, v, ov2), imap2(v, 1, vv), Wr, imap1(1), imap1(ov), 0.0, tmp4,
                  imap2(v, v, ov2), imap2(v, 1, vv)));
    return antisym_add(r2, tmp4, 1.0);
  }

  // ---------------------------------------------------------------- Lambda: Hbar elements at fixed T
  int lambda_setup() {
    const double *t2 = tfix + ov;
    GFCC_TRY(rotate(tfix));
    GFCC_TRY(ring_matrix(t2, 1.0));   // Wbar_mbej
    // Wooov[m][n][i][e] = <mn||ie>' = (mi|ne)' - (me|ni)'
    GFCC_TRY(get(&Wooov, oo * ov));
    GFCC_TRY(eri(0, o, 0, o, 0, o, o, v, 1.0, 0.0, Wooov, imap2(o, v, o2v), imap2(v, 1, ov)));
    GFCC_TRY(eri(0, o, o, v, 0, o, 0, o, -1.0, 1.0, Wooov, imap2(v, 1, o2v), imap2(o, v, ov)));
    // Q[x][i][j][b] = Wbar_xbij = <xb||ij>' - f'_xe t_ij^be + 1/2 <xb||ef>' t_ij^ef + P(ij) <xn||ie>' t_jn^be
    GFCC_TRY(get(&Q, oo * ov));
    GFCC_TRY(eri(0, o, 0, o, o, v, 0, o, 1.0, 0.0, Q, imap2(o, ov, o2v), imap2(o, v, 1)));     // (xi|bj)
    GFCC_TRY(eri(0, o, 0, o, o, v, 0, o, -1.0, 1.0, Q, imap2(o, v, o2v), imap2(o, ov, 1)));    // -(xj|bi)
    GFCC_TRY(gemm(o, o2v, v, -1.0, Fov, imap1(v), imap1(1), t2, imap1(1), imap1(v), 1.0, Q, imap1(o2v), imap1(1)));
    GFCC_TRY(gemm(oo, ov, ov, 1.0, Wooov, imap2(o, v, o2v), imap2(v, 1, ov), t2, imap2(v, 1, vv), imap2(v, v, ov2), 1.0,
                  Q, imap2(o, ov, o2v), imap1(1)));
    GFCC_TRY(gemm(oo, ov, ov, -1.0, Wooov, imap2(o, v, o2v), imap2(v, 1, ov), t2, imap2(v, 1, vv), imap2(v, v, ov2),
                  1.0, Q, imap2(o, v, o2v), imap2(v, 1, ov)));
    // R3[a][m][e][f] = Wbar_efam = <ef||am>' - f'_na t_nm^ef + 1/2 <no||am>' t_no^ef - P(ef) <nf||ag>' t_nm^eg
    GFCC_TRY(get(&R3, ov2 * v));
    GFCC_TRY(eri(o, v, o, v, o, v, 0, o, 1.0, 0.0, R3, imap2(v, ov2, v), imap2(o, vv, 1)));    // (ea|fm)
    GFCC_TRY(eri(o, v, 0, o, o, v, o, v, -1.0, 1.0, R3, imap2(o, vv, v), imap2(v, ov2, 1)));   // -(em|fa)
    GFCC_TRY(gemm(v, ov2, o, -1.0, Fov, imap1(1), imap1(v), t2, imap1(ov2), imap1(1), 1.0, R3, imap1(ov2), imap1(1)));
    // <no||am>' = -<no||ma>' = -Wooov[n][o][m][a]
    GFCC_TRY(gemm(ov, vv, oo, -0.5, Wooov, imap1(1), imap1(ov), t2, imap1(vv), imap1(1), 1.0, R3, imap2(v, ov2, vv),
                  imap1(1)));
    // blocks of <nb||ef>' over n: vc[n][b][e][f]
    mc = std::max<long long>(1, std::min<long long>(o, (1LL << 29) / std::max<long long>(1, v3)));
    GFCC_TRY(get(&vc, mc * v3));
    for (long long n0 = 0; n0 < o; n0 += mc) {
      const long long nm = std::min<long long>(mc, o - n0);
      GFCC_TRY(eri(n0, nm, o, v, o, v, o, v, 1.0, 0.0, vc, imap2(v, v, v3), imap2(v, 1, vv)));
      GFCC_TRY(eri(n0, nm, o, v, o, v, o, v, -1.0, 1.0, vc, imap2(v, 1, v3), imap2(v, v, vv)));
      // Q[x][ij][b] += 1/2 sum_ef vc[x][b][ef] t2[ij][ef]
      GFCC_TRY(gemm(nm * v, oo, vv, 0.5, vc, imap1(vv), imap1(1), t2, imap1(1), imap1(vv), 1.0, Q + n0 * o2v,
                    imap2(v, 1, o2v), imap1(v)));
      // T5(f, a, m, e) = sum_{n in block, g} vc[n][f][a][g] t2[n][m][e][g]:  R3[a][m][e][f] -= T5, R3[a][m][f][e] += T5
      GFCC_TRY(gemm(vv, ov, nm * v, -1.0, vc, imap1(v), imap2(v, 1, v3), t2 + n0 * ov2, imap2(v, 1, ov2), imap1(v),
                    1.0, R3, imap2(v, ov2, 1), imap2(v, v, vv)));
      GFCC_TRY(gemm(vv, ov, nm * v, 1.0, vc, imap1(v), imap2(v, 1, v3), t2 + n0 * ov2, imap2(v, 1, ov2), imap1(v),
                    1.0, R3, imap2(v, ov2, v), imap2(v, 1, vv)));
    }
    GFCC_TRY(get(&Gvv, vv));
    GFCC_TRY(get(&Goo, oo));
    GFCC_TRY(get(&gK, L));
    return GFCC_OK;
  }

  // ---------------------------------------------------------------- Lambda residual at l = [l1 | l2]
  int lambda_residual(const double *l, double *res) {
    const double *l1 = l, *l2 = l + ov, *t2 = tfix + ov;
    double *r1 = res, *r2 = res + ov;
    // G_ae = -1/2 t_mn^ef l_mnaf  (Gvv[a][e]);  G_mi = 1/2 t_mn^ef l_inef  (Goo[m][i])
    GFCC_TRY(gemm(v, v, oo * v, -0.5, l2, imap1(v), imap2(v, 1, vv), t2, imap2(v, 1, vv), imap1(v), 0.0, Gvv, imap1(v),
                  imap1(1)));
    GFCC_TRY(gemm(o, o, ov2, 0.5, t2, imap1(ov2), imap1(1), l2, imap1(1), imap1(ov2), 0.0, Goo, imap1(o), imap1(1)));

    // ---- singles
    GFCC_TRY(copy(Fov, ov, r1));
    GFCC_TRY(gemm(o, v, v, 1.0, l1, imap1(v), imap1(1), Fvv, imap1(v), imap1(1), 1.0, r1, imap1(v), imap1(1)));
    GFCC_TRY(gemm(o, v, o, -1.0, Foo, imap1(o), imap1(1), l1, imap1(v), imap1(1), 1.0, r1, imap1(v), imap1(1)));
    // + l_me Wbar_ieam = sum_(m,e) l1[(m,e)] Wr[(m,e)][(i,a)]
    GFCC_TRY(gemm(ov, 1, ov, 1.0, Wr, imap1(1), imap1(ov), l1, imap1(1), imap1(0), 1.0, r1, imap1(1), imap1(0)));
    // + 1/2 l_imef Wbar_efam
    GFCC_TRY(gemm(o, v, ov2, 0.5, l2, imap1(ov2), imap1(1), R3, imap1(1), imap1(ov2), 1.0, r1, imap1(v), imap1(1)));
    // - 1/2 l_mnae Wbar_iemn
    GFCC_TRY(gemm(o, v, o2v, -0.5, Q, imap1(o2v), imap1(1), l2, imap2(v, 1, vv), imap1(v), 1.0, r1, imap1(v),
                  imap1(1)));
    // - G_ef <ei||fa>' = - sum_K g[K] L'_ia + sum_K sum_e L'_ea H[K][i][e],  g[K] = G_ef L'_ef, H = L'_if G_ef
    GFCC_TRY(gemm(L, 1, vv, 1.0, Lt + (long long)o * n + o, imap1(nn), imap2(v, 1, n), Gvv, imap1(1), imap1(0), 0.0, gK,
                  imap1(1), imap1(0)));
    GFCC_TRY(gemm(ov, 1, L, -1.0, Lt + o, imap2(v, 1, n), imap1(nn), gK, imap1(1), imap1(0), 1.0, r1, imap1(1),
                  imap1(0)));
    GFCC_TRY(gemm((long long)L * o, v, v, 1.0, Lt + o, imap2(o, n, nn), imap1(1), Gvv, imap1(1), imap1(v), 0.0, Yk,
                  imap1(v), imap1(1)));
    GFCC_TRY(gemm(v, o, (long long)L * v, 1.0, Lt + (long long)o * n + o, imap1(1), imap2(v, n, nn), Yk,
                  imap2(v, 1, ov), imap1(v), 1.0, r1, imap1(1), imap1(v)));
    // - G_mn <mi||na>' = - sum_mn Goo[m][n] Wooov[m][i][n][a]
    GFCC_TRY(gemm(ov, 1, oo, -1.0, Wooov, imap2(v, 1, ov), imap2(o, v, o2v), Goo, imap1(1), imap1(0), 1.0, r1, imap1(1),
                  imap1(0)));

    // ---- doubles
    GFCC_TRY(copy(voovv, oo * vv, r2));
    // + P(ab) l_ijae Fbar_eb
    GFCC_TRY(gemm(oo * v, v, v, 1.0, l2, imap1(v), imap1(1), Fvv, imap1(v), imap1(1), 1.0, r2, imap1(v), imap1(1)));
    GFCC_TRY(gemm(oo * v, v, v, -1.0, l2, imap1(v), imap1(1), Fvv, imap1(v), imap1(1), 1.0, r2, imap2(v, 1, vv),
                  imap1(v)));
    // - P(ij) l_imab Fbar_jm  (batched over i)
    GFCC_TRY(gemm(o, vv, o, -1.0, Foo, imap1(o), imap1(1), l2, imap1(vv), imap1(1), 1.0, r2, imap1(vv), imap1(1), o, 0,
                  ov2, ov2));
    GFCC_TRY(gemm(o, vv, o, 1.0, Foo, imap1(o), imap1(1), l2, imap1(vv), imap1(1), 1.0, r2, imap1(ov2), imap1(1), o, 0,
                  ov2, vv));
    // + 1/2 l_mnab Wbar_ijmn
    GFCC_TRY(gemm(oo, vv, oo, 0.5, Wmnij, imap1(oo), imap1(1), l2, imap1(vv), imap1(1), 1.0, r2, imap1(vv), imap1(1)));
    // + 1/2 l_ijef Wbar_efab = sum_ef l_ijef (ea|fb)' + 1/4 (l_ijef t_mn^ef) <mn||ab>'
    GFCC_TRY(ladder(l2, r2, true));
    GFCC_TRY(gemm(oo, oo, vv, 1.0, l2, imap1(vv), imap1(1), t2, imap1(1), imap1(vv), 0.0, Zm, imap1(oo), imap1(1)));
    GFCC_TRY(gemm(oo, vv, oo, 0.25, Zm, imap1(oo), imap1(1), voovv, imap1(vv), imap1(1), 1.0, r2, imap1(vv), imap1(1)));
    // - P(ab) l_ma <ij||mb>'
    GFCC_TRY(gemm(v, oo * v, o, -1.0, l1, imap1(1), imap1(v), Wooov, imap1(v), imap2(v, 1, ov), 1.0, r2, imap1(v),
                  imap2(v, 1, vv)));
    GFCC_TRY(gemm(v, oo * v, o, 1.0, l1, imap1(1), imap1(v), Wooov, imap1(v), imap2(v, 1, ov), 1.0, r2, imap1(1),
                  imap2(v, v, vv)));
    // + P(ab) <ij||ae>' G_be - P(ij) <im||ab>' G_mj
    GFCC_TRY(gemm(oo * v, v, v, 1.0, voovv, imap1(v), imap1(1), Gvv, imap1(1), imap1(v), 1.0, r2, imap1(v), imap1(1)));
    GFCC_TRY(gemm(oo * v, v, v, -1.0, voovv, imap1(v), imap1(1), Gvv, imap1(1), imap1(v), 1.0, r2, imap2(v, 1, vv),
                  imap1(v)));
    GFCC_TRY(gemm(o, vv, o, -1.0, Goo, imap1(1), imap1(o), voovv, imap1(vv), imap1(1), 1.0, r2, imap1(vv), imap1(1), o,
                  0, ov2, ov2));
    GFCC_TRY(gemm(o, vv, o, 1.0, Goo, imap1(1), imap1(o), voovv, imap1(vv), imap1(1), 1.0, r2, imap1(ov2), imap1(1), o,
                  0, ov2, vv));
    // P(ij) P(ab) of: l_imae Wbar_jebm + l_ia Fbar_jb + sum_K (l_ie L'_ea) L'_jb  (the last is P(ij) l_ie <ej||ab>')
    GFCC_TRY(gemm(ov, ov, ov, 1.0, l2, imap2(v, v, ov2), imap2(v, 1, vv), Wr, imap1(ov), imap1(1), 0.0, tmp4,
                  imap2(v, v, ov2), imap2(v, 1, vv)));
    GFCC_TRY(gemm(ov, ov, 1, 1.0, l1, imap1(1), imap1(0), Fov, imap1(0), imap1(1), 1.0, tmp4, imap2(v, v, ov2),
                  imap2(v, 1, vv)));
    GFCC_TRY(gemm((long long)L * v, o, v, 1.0, Lt + (long long)o * n + o, imap2(v, 1, nn), imap1(n), l1, imap1(1),
                  imap1(v), 0.0, Yk, imap2(v, 1, ov), imap1(v)));
    GFCC_TRY(gemm(ov, ov, L, 1.0, Yk, imap1(1), imap1(ov), Lt + o, imap1(nn), imap2(v, 1, n), 1.0, tmp4,
                  imap2(v, v, ov2), imap2(v, 1, vv)));
    return antisym_add(r2, tmp4, 1.0);
  }

  // ---------------------------------------------------------------- reductions and the DIIS loop
  int maxabs(const double *p, long long count, double *out) {
    reduce_kernel<1><<<RED_BLOCKS, RED_THREADS, 0, st>>>(nullptr, count, 1, p, part);
    GFCC_LAUNCH_CHECK();
    double h[RED_BLOCKS];
    GFCC_CUDA(cudaMemcpyAsync(h, part, sizeof(h), cudaMemcpyDeviceToHost, st));
    GFCC_CUDA(cudaStreamSynchronize(st));
    double m = 0.0;
    for (int b = 0; b < RED_BLOCKS; b++) m = std::max(m, h[b]);
    *out = m;
    return GFCC_OK;
  }

  int energy(const double *t, double *out) {
    energy_kernel<<<RED_BLOCKS, RED_THREADS, 0, st>>>(fock, V0, t, t + ov, o, v, part);
    GFCC_LAUNCH_CHECK();
    double h[RED_BLOCKS];
    GFCC_CUDA(cudaMemcpyAsync(h, part, sizeof(h), cudaMemcpyDeviceToHost, st));
    GFCC_CUDA(cudaStreamSynchronize(st));
    double s = 0.0;
    for (int b = 0; b < RED_BLOCKS; b++) s += h[b];
    *out = s;
    return GFCC_OK;
  }

  // Iterate x (in place) on the T (lam = false) or Lambda equations; iterations and the final max
  // |residual| are returned.  GFCC_WARN_NOT_CONVERGED after max_iter iterations without tol.
  int iterate(bool lam, double tol, int max_iter, int *iters, double *rmax, double *flops_per_iter) {
    double B[DIIS_CAP][DIIS_CAP] = {};
    int cnt = 0, slot = 0;
    for (int it = 1; it <= max_iter; it++) {
      flops = 0.0;
      GFCC_TRY(lam ? lambda_residual(x, r) : t_residual(x, r));
      if (flops_per_iter) *flops_per_iter = flops;
      GFCC_TRY(maxabs(r, N, rmax));
      *iters = it;
      if (!std::isfinite(*rmax)) {
        set_error("gfcc_ccsd: the %s iterations diverged (non-finite residual at iteration %d)", lam ? "Lambda" : "T",
                  it);
        return GFCC_ERR_ARG;
      }
      if (*rmax <= tol) return GFCC_OK;
      double *e = he + (long long)slot * N, *xn = hx + (long long)slot * N;
      jacobi_kernel<<<grid1d(N), 256, 0, st>>>(x, r, eps, o, v, e, xn);
      GFCC_LAUNCH_CHECK();
      cnt = std::min(cnt + 1, DIIS_CAP);
      // the new row of B: e . e_j for the stored slots j < cnt
      reduce_kernel<0><<<RED_BLOCKS, RED_THREADS, 0, st>>>(he, N, cnt, e, part);
      GFCC_LAUNCH_CHECK();
      std::vector<double> h((size_t)cnt * RED_BLOCKS);
      GFCC_CUDA(cudaMemcpyAsync(h.data(), part, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
      GFCC_CUDA(cudaStreamSynchronize(st));
      for (int j = 0; j < cnt; j++) {
        double s = 0.0;
        for (int b = 0; b < RED_BLOCKS; b++) s += h[(size_t)j * RED_BLOCKS + b];
        B[slot][j] = B[j][slot] = s;
      }
      Coef cf{};
      bool mixed = false;
      if (cnt >= 2) mixed = diis_solve(B, cnt, cf.c);
      if (mixed) {
        combine_kernel<<<grid1d(N), 256, 0, st>>>(hx, N, cnt, cf, x);
        GFCC_LAUNCH_CHECK();
      } else {
        GFCC_TRY(copy(xn, N, x));
      }
      slot = (slot + 1) % DIIS_CAP;
    }
    return GFCC_WARN_NOT_CONVERGED;
  }
};

double seconds_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

int ccsd_impl(int o, int v, int L, const double *fock, const double *chol, double tol, int max_iter, int flags,
              double *t1, double *t2, double *lambda, double *info) {
  if (o < 1 || v < 1 || L < 1 || fock == nullptr || chol == nullptr || t1 == nullptr || t2 == nullptr) {
    set_error("gfcc_ccsd: need o >= 1, v >= 1, L >= 1 and non-NULL fock, chol, t1, t2");
    return GFCC_ERR_ARG;
  }
  if (!(tol > 0.0) || max_iter < 1 || (flags & ~(GFCC_CCSD_EMULATE | GFCC_CCSD_GUESS))) {
    set_error("gfcc_ccsd: need tol > 0, max_iter >= 1 and known flags (got tol %g, max_iter %d, flags %d)", tol,
              max_iter, flags);
    return GFCC_ERR_ARG;
  }
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    set_error("gfcc_ccsd: cannot create a CUDA stream (no usable GPU?)");
    return GFCC_ERR_CUDA;
  }
  const bool prev_emulate = g_emulate_big;
  const double prev_min = g_emulate_min_flops_local;
  g_emulate_big = (flags & GFCC_CCSD_EMULATE) != 0;
  // the iteration's large contractions (the vvvv blocks and their ladder products, the ring, the
  // Cholesky sums of the singles) are 1e11-1e12 flops each at medium sizes: below the setup threshold
  if (g_emulate_big) g_emulate_min_flops_local = std::min(g_emulate_min_flops, CCSD_EMULATE_MIN_FLOPS);
  auto run = [&](Ccsd &C) -> int {
    GFCC_TRY(C.init(o, v, L, fock, chol));
    const long long ov = C.ov, N = C.N;
    double it_info[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (flags & GFCC_CCSD_GUESS) {
      GFCC_CUDA(cudaMemcpyAsync(C.x, t1, sizeof(double) * ov, cudaMemcpyHostToDevice, st));
      GFCC_CUDA(cudaMemcpyAsync(C.x + ov, t2, sizeof(double) * ov * ov, cudaMemcpyHostToDevice, st));
      GFCC_TRY(check_input_tensor(st, C.x + ov, o, o, v, v, 1, 0, -1.0, 1e-12, "t2 (i<->j)"));
      GFCC_TRY(check_input_tensor(st, C.x + ov, o, o, v, v, 0, 1, -1.0, 1e-12, "t2 (a<->b)"));
    } else {
      GFCC_TRY(fill_f64(st, C.x, N, 0.0));
    }
    GFCC_CUDA(cudaStreamSynchronize(st));
    auto t0 = std::chrono::steady_clock::now();
    int it = 0;
    double rmax = 0.0, fl = 0.0;
    const int st_t = C.iterate(false, tol, max_iter, &it, &rmax, &fl);
    GFCC_TRY(st_t);
    GFCC_CUDA(cudaStreamSynchronize(st));
    it_info[5] = seconds_since(t0);
    it_info[1] = it;
    it_info[2] = rmax;
    it_info[7] = fl;
    GFCC_TRY(C.energy(C.x, &it_info[0]));
    GFCC_CUDA(cudaMemcpyAsync(t1, C.x, sizeof(double) * ov, cudaMemcpyDeviceToHost, st));
    GFCC_CUDA(cudaMemcpyAsync(t2, C.x + ov, sizeof(double) * ov * ov, cudaMemcpyDeviceToHost, st));
    GFCC_CUDA(cudaStreamSynchronize(st));
    int status = st_t;
    if (lambda != nullptr) {
      GFCC_TRY(C.copy(C.x, N, C.tfix));
      if (flags & GFCC_CCSD_GUESS) {
        GFCC_CUDA(cudaMemcpyAsync(C.x, lambda, sizeof(double) * N, cudaMemcpyHostToDevice, st));
        GFCC_TRY(check_input_tensor(st, C.x + ov, o, o, v, v, 1, 0, -1.0, 1e-12, "lambda2 (i<->j)"));
        GFCC_TRY(check_input_tensor(st, C.x + ov, o, o, v, v, 0, 1, -1.0, 1e-12, "lambda2 (a<->b)"));
      }   // else Lambda starts from T (already in x)
      t0 = std::chrono::steady_clock::now();
      GFCC_TRY(C.lambda_setup());
      int lit = 0;
      double lr = 0.0;
      const int st_l = C.iterate(true, tol, max_iter, &lit, &lr, nullptr);
      GFCC_TRY(st_l);
      GFCC_CUDA(cudaStreamSynchronize(st));
      it_info[6] = seconds_since(t0);
      it_info[3] = lit;
      it_info[4] = lr;
      if (st_l != GFCC_OK) status = st_l;
      GFCC_CUDA(cudaMemcpyAsync(lambda, C.x, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
      GFCC_CUDA(cudaStreamSynchronize(st));
    }
    if (info) memcpy(info, it_info, sizeof(it_info));
    return status;
  };
  int s;
  {
    Ccsd C;   // device memory freed at the end of this scope, before the stream goes
    C.st = st;
    s = run(C);
    cudaStreamSynchronize(st);
  }
  g_emulate_big = prev_emulate;
  g_emulate_min_flops_local = prev_min;
  cudaGetLastError();
  cudaStreamDestroy(st);
  return s;
}

}  // namespace

}  // namespace gfcc

extern "C" int gfcc_ccsd(int o, int v, int L, const double *fock, const double *chol, double tol, int max_iter,
                         int flags, double *t1, double *t2, double *lambda, double *info) {
  return gfcc::ccsd_impl(o, v, L, fock, chol, tol, max_iter, flags, t1, t2, lambda, info);
}
