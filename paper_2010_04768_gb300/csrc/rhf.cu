// Closed-shell spin-adapted GFCCSD-IP (FP64): the paper's closed-shell IP code keeps the alpha
// amplitudes only (Table 2).  For a closed-shell reference, removing an alpha electron from spatial
// orbital p keeps the IP vector in the doublet subspace with coordinates r_i = R_{i alpha} and
// r_ij^a = R_{i alpha, j beta}^{a beta} (all i, j, a), R_{i alpha, j alpha}^{a alpha} = r_ij^a - r_ji^a.
// Summing the spin-orbital IP-EOM-CCSD equations over the spins gives, with u_mnef = (me|nf)' and
// (pq|rs)' = sum_K L'^K_pq L'^K_rs over the T1-rotated spatial Cholesky vectors (t_ij^ab =
// T_{i alpha, j beta}^{a alpha, b beta}):
//   Fbar_mi = f'_mi + (2 u_mnef - u_mnfe) t_in^ef,  Fbar_ae = f'_ae - (2 u_mnef - u_mnfe) t_mn^af,
//   Fbar_me = f'_me,  W_mnij = (mi|nj)' + u_mnef t_ij^ef,
//   W_maij = (mi|aj)' + Fbar_me t_ij^ea + (me|af)' t_ij^ef + (2 (mi|ne)' - (me|ni)') t_jn^ae
//            - (mi|ne)' t_jn^ea - (me|nj)' t_in^ea,
//   X_maej = (me|aj)' + (2 u_mnef - u_mnfe) t_jn^af - u_mnef t_jn^fa,
//   Y_maie = (mi|ae)' - u_mnfe t_in^fa,
//   sigma_i   = -Fbar_mi r_m + Fbar_me (2 r_im^e - r_mi^e) + (W_nmie - 2 W_mnie) r_mn^e,
//   sigma_ija = -W_maij r_m + Fbar_ae r_ij^e - Fbar_mi r_mj^a - Fbar_mj r_im^a + W_mnij r_mn^a
//               - Y_maie r_mj^e + (2 X_maej - Y_maje) r_im^e - X_maej r_mi^e - z_e t_ij^ea,
//   z_e = (2 u_mnef - u_mnfe) r_mn^f,   W_mnie = (mi|ne)'.
// Layout of the operator: the three ring sums are (ov) x (ov) contractions against the three
// orderings r[m][j][e], r[i][m][e], r[m][i][e] of the same unpacked vector (the Fock terms of the
// doubles block folded into the first two), the W_maij and three-body terms one contraction over
// K = v + o, the oooo term one over (m,n), the 1h row one over K = o + o^2 v.  The vector needs no
// packing: the GMRES coordinates are the contraction layout.
#include <algorithm>

#include "ctx.cuh"
#include "kernels.cuh"
#include "ozaki.cuh"
#include "sigma.cuh"

namespace gfcc {

// Contractions of at least this many flops run on the FP64-accurate digit-plane path when the
// context's emulation option is on (the ring sums and the oooo term at useful sizes; the narrow ones
// stay on the FP64 units); the digit planes of the ring matrices are cut once at setup with the
// digit count and pair level of the setup's emulated contractions
constexpr double RHF_EMULATE_MIN_FLOPS = 1e9;
constexpr int RHF_EMU_DIGITS = 8, RHF_EMU_LEVEL = 9;

namespace {

// M[(j,a)][(m,a)] += cF * Foo[m][j];  M[(j,a)][(j,e)] += cV * Fvv[a][e]
__global__ void rhf_fold_kernel(double *M, int o, int v, const double *Foo, const double *Fvv, double cF, double cV) {
  const long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long ov = (long long)o * v;
  if (row >= ov) return;
  const int j = (int)(row / v), a = (int)(row % v);
  double *w = M + row * ov;
  if (cF != 0.0)
    for (int m = 0; m < o; m++) w[(long long)m * v + a] += cF * Foo[(long long)m * o + j];
  if (cV != 0.0)
    for (int e = 0; e < v; e++) w[(long long)j * v + e] += cV * Fvv[(long long)a * v + e];
}

// out[r] = [A[r][0..ka) | B[r][0..kb)]
__global__ void rhf_concat_kernel(const double *A, long long ka, const double *B, long long kb, long long rows,
                                  double alpha, double *out) {
  const long long K = ka + kb, tot = rows * K;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < tot; x += (long long)gridDim.x * blockDim.x) {
    const long long r = x / K, c = x - r * K;
    out[x] = alpha * (c < ka ? A[r * ka + c] : B[r * kb + (c - ka)]);
  }
}

__global__ void rhf_diag_kernel(const double *Foo, const double *Fvv, int o, int v, double *d) {
  const long long dim = o + (long long)o * o * v;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < dim; x += (long long)gridDim.x * blockDim.x) {
    if (x < o) {
      d[x] = -Foo[x * o + x];
      continue;
    }
    const long long r = x - o;
    const int a = (int)(r % v);
    const int j = (int)((r / v) % o);
    const int i = (int)(r / ((long long)o * v));
    d[x] = Fvv[(long long)a * v + a] - Foo[(long long)i * o + i] - Foo[(long long)j * o + j];
  }
}

// [P rows k][c = 2 s + re/im] = u_k of system s (u = x / D_s with the preconditioner)
__global__ void rhf_unpack_kernel(SysBatch b, long long dim, long long C2, double *P) {
  const long long tot = dim * b.nsys;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(t % b.nsys);
    const long long k = t / b.nsys;
    const long long q = 2 * ((long long)sysv(b, s) * b.ldx + k);
    double ur = b.x[q], ui = b.x[q + 1];
    if (b.diag != nullptr && b.omega != nullptr) {
      const double dr = b.omega[sysv(b, s)] + b.dsign * b.diag[k], di = b.zsign * b.eta;
      const double den = dr * dr + di * di;
      const double nr = (ur * dr + ui * di) / den, ni = (ui * dr - ur * di) / den;
      ur = nr;
      ui = ni;
    }
    P[k * C2 + 2 * s] = ur;
    P[k * C2 + 2 * s + 1] = ui;
  }
}

// y_s[k] = z_s u_k + sigma_k  (z_s = omega_s + i zsign eta; y = sigma without omega)
__global__ void rhf_epilogue_kernel(SysBatch b, long long dim, long long C2, const double *U, const double *Sg) {
  const long long tot = dim * b.nsys;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(t % b.nsys);
    if (!sys_stores(b, s)) continue;
    const long long k = t / b.nsys;
    double yr = Sg[k * C2 + 2 * s], yi = Sg[k * C2 + 2 * s + 1];
    if (b.omega != nullptr) {
      const double zr = b.omega[sysv(b, s)], zi = b.zsign * b.eta;
      const double ur = U[k * C2 + 2 * s], ui = U[k * C2 + 2 * s + 1];
      yr += zr * ur - zi * ui;
      yi += zr * ui + zi * ur;
    }
    const long long q = 2 * ((long long)sysv(b, s) * b.ldy + k);
    b.y[q] = yr;
    b.y[q + 1] = yi;
  }
}

// b_p: p occupied: r_i = d_ip; p = o + b: r_i = t_i^b, r_ij^a = t_ij^ba
__global__ void rhf_rhs_kernel(double *B, long long n, int nsys, const int *porb, int o, int v, const double *t1,
                               const double *t2, const int *mask) {
  const long long tot = n * nsys;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(t / n);
    if (mask != nullptr && !mask[s]) continue;
    const long long mu = t - (long long)s * n;
    const int p = porb[s];
    double val = 0.0;
    if (mu < o) {
      val = p < o ? (mu == p ? 1.0 : 0.0) : t1[mu * v + (p - o)];
    } else if (p >= o) {
      const long long r = mu - o;
      const long long a = r % v, ij = r / v;
      val = t2[(ij * v + (p - o)) * v + a];
    }
    B[2 * t] = val;
    B[2 * t + 1] = 0.0;
  }
}

// left vector 1h part of an occupied q = m: d_mi - t_m^c l_i^c - (2 t_ml^cd - t_ml^dc) l_il^cd
// (one block per (q, i)); virtual q = b: l_i^b
__global__ void rhf_left_1h_kernel(double *C, long long n, int nq, const int *qorb, int o, int v, const double *t1,
                                   const double *t2, const double *l1, const double *l2) {
  const int qi = blockIdx.x / o, i = blockIdx.x % o;
  const int q = qorb[qi];
  __shared__ double sh[256];
  double acc = 0.0;
  if (q < o) {
    const int m = q;
    const long long ov2 = (long long)o * v * v, vv = (long long)v * v;
    for (long long x = threadIdx.x; x < ov2; x += blockDim.x) {   // x = (l, c, d)
      const long long l = x / vv, cd = x % vv, c = cd / v, d = cd % v;
      const double tt = 2.0 * t2[(long long)m * ov2 + x] - t2[(long long)m * ov2 + l * vv + d * v + c];
      acc -= tt * l2[(long long)i * ov2 + x];
    }
    for (long long c = threadIdx.x; c < v; c += blockDim.x) acc -= t1[(long long)m * v + c] * l1[(long long)i * v + c];
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double val = sh[0];
    if (q < o) {
      if (i == q) val += 1.0;
    } else {
      val = l1[(long long)i * v + (q - o)];
    }
    C[(long long)qi * n + i] = val;
  }
}

// left vector 2h1p part: q = b: 2 l_ij^ba - l_ij^ab;  q = m: 2 d_im l_j^a - d_jm l_i^a
// - 2 t_m^c l_ij^ca + t_m^c l_ij^ac
__global__ void rhf_left_2h1p_kernel(double *C, long long n, int nq, const int *qorb, int o, int v, const double *t1,
                                     const double *l1, const double *l2) {
  const long long m2 = n - o, tot = m2 * nq;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int qi = (int)(t / m2);
    const long long r = t - (long long)qi * m2;
    const int q = qorb[qi];
    const int a = (int)(r % v);
    const long long ij = r / v;
    const int j = (int)(ij % o), i = (int)(ij / o);
    const double *L = l2 + ij * v * v;
    double val;
    if (q >= o) {
      const int b = q - o;
      val = 2.0 * L[(long long)b * v + a] - L[(long long)a * v + b];
    } else {
      const int m = q;
      val = (i == m ? 2.0 * l1[(long long)j * v + a] : 0.0) - (j == m ? l1[(long long)i * v + a] : 0.0);
      for (int c = 0; c < v; c++)
        val += t1[(long long)m * v + c] * (L[(long long)a * v + c] - 2.0 * L[(long long)c * v + a]);
    }
    C[(long long)qi * n + o + r] = val;
  }
}

struct Tmp {
  std::vector<double *> ptrs;
  ~Tmp() {
    for (double *p : ptrs) dfree(p);
  }
  int get(double **p, long long count) {
    int s = dev_alloc_tmp(p, count);
    if (s == GFCC_OK) ptrs.push_back(*p);
    return s;
  }
};

}  // namespace

long long rhf_work_doubles(const gfcc_ctx *c, int nsys) {
  const long long o = c->o, v = c->v, o2v = o * o * v;
  return (v + o + o2v + o + o2v) * 2LL * nsys;
}

double rhf_sigma_flops(const gfcc_ctx *c) {
  const double o = c->o, v = c->v;
  // per real vector: three ring sums 6 o^3 v^2, oooo 2 o^4 v, [three-body | ovoo] 2 o^2 v (v + o),
  // z 2 o^2 v^2, 1h row 2 o (o + o^2 v); a complex vector is two real ones
  return 2.0 * (6.0 * o * o * o * v * v + 2.0 * o * o * o * o * v + 2.0 * o * o * v * (v + o) + 2.0 * o * o * v * v +
                2.0 * o * (o + o * o * v));
}

int build_hbar_rhf(gfcc_ctx *c, const double *d_fock, const double *d_chol) {
  cudaStream_t st = c->stream;
  const int o = c->o, v = c->v, n = c->n, L = c->L;
  const long long ov = (long long)o * v, oo = (long long)o * o, vv = (long long)v * v, nn = (long long)n * n;
  const long long ov2 = (long long)o * vv, o2v = oo * v, v3 = vv * v;
  const double *t2 = c->t2;
  Tmp tmp;
  // ---- T1-rotated Cholesky vectors; h = f - 2J + K; f' = h' + 2J' - K'
  double *Lt, *fp;
  GFCC_TRY(tmp.get(&Lt, (long long)L * nn));
  GFCC_CUDA(cudaMemcpyAsync(Lt, d_chol, sizeof(double) * L * nn, cudaMemcpyDeviceToDevice, st));
  GFCC_TRY(t1_dress(st, c->t1, o, v, Lt, L, nn));
  GFCC_TRY(tmp.get(&fp, nn));
  GFCC_CUDA(cudaMemcpyAsync(fp, d_fock, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st));
  GFCC_TRY(chol_coulomb_exchange(st, d_chol, n, o, L, fp, -2.0, 1.0));
  GFCC_TRY(t1_dress(st, c->t1, o, v, fp, 1, nn));
  GFCC_TRY(chol_coulomb_exchange(st, Lt, n, o, L, fp, 2.0, -1.0));
  auto eri = [&](long long P0, long long np, long long R0, long long nr, long long Q0, long long nq, long long S0,
                 long long ns, double alpha, double beta, double *C, IMap cm, IMap cn) {
    return chol_eri(st, Lt, n, L, P0, np, R0, nr, Q0, nq, S0, ns, alpha, beta, C, cm, cn);
  };

  // ---- u[m][n][e][f] = (me|nf)';  u2 = 2 u_mnef - u_mnfe
  double *u, *u2;
  GFCC_TRY(tmp.get(&u, oo * vv));
  GFCC_TRY(tmp.get(&u2, oo * vv));
  GFCC_TRY(eri(0, o, o, v, 0, o, o, v, 1.0, 0.0, u, imap2(v, v, ov2), imap2(v, 1, vv)));
  {
    const long long d[4] = {o, o, v, v}, is[4] = {ov2, vv, v, 1}, os[4] = {ov2, vv, v, 1}, os2[4] = {ov2, vv, 1, v};
    GFCC_TRY(permute4(st, d, u, is, u2, os, 2.0, 0.0));
    GFCC_TRY(permute4(st, d, u, is, u2, os2, -1.0, 1.0));   // u2[m][n][f][e] -= u[m][n][e][f]
  }

  // ---- Fbar
  GFCC_TRY(dev_alloc(c, &c->Foo, oo));
  GFCC_TRY(dev_alloc(c, &c->Fvv, vv));
  GFCC_TRY(dev_alloc(c, &c->Fov, ov));
  {
    const long long d[4] = {1, 1, o, o}, is[4] = {0, 0, n, 1}, os[4] = {0, 0, o, 1};
    GFCC_TRY(permute4(st, d, fp, is, c->Foo, os, 1.0, 0.0));
    const long long d2[4] = {1, 1, v, v}, os2[4] = {0, 0, v, 1};
    GFCC_TRY(permute4(st, d2, fp + (long long)o * n + o, is, c->Fvv, os2, 1.0, 0.0));
    const long long d3[4] = {1, 1, o, v};
    GFCC_TRY(permute4(st, d3, fp + o, is, c->Fov, os2, 1.0, 0.0));
  }
  // Foo[m][i] += u2[m][(n,e,f)] t2[i][(n,e,f)];  Fvv[a][e] -= t2[(m,n)][a][f] u2[(m,n)][e][f]
  GFCC_TRY(gemm_f64(st, o, o, ov2, 1.0, u2, imap1(ov2), imap1(1), t2, imap1(1), imap1(ov2), 1.0, c->Foo, imap1(o),
                    imap1(1)));
  GFCC_TRY(gemm_f64(st, v, v, oo * v, -1.0, t2, imap1(v), imap2(v, 1, vv), u2, imap2(v, 1, vv), imap1(v), 1.0, c->Fvv,
                    imap1(v), imap1(1)));

  // ---- Woooo[m][n][i][j] = (mi|nj)' + u[m][n][e][f] t2[i][j][e][f]
  GFCC_TRY(dev_alloc(c, &c->Woooo, oo * oo));
  GFCC_TRY(eri(0, o, 0, o, 0, o, 0, o, 1.0, 0.0, c->Woooo, imap2(o, o, oo * o), imap2(o, 1, oo)));
  GFCC_TRY(gemm_f64(st, oo, oo, vv, 1.0, u, imap1(vv), imap1(1), t2, imap1(1), imap1(vv), 1.0, c->Woooo, imap1(oo),
                    imap1(1)));

  // ---- B1[m][i][n][e] = (mi|ne)',  C1[m][i][n][e] = (me|ni)'
  double *B1, *C1;
  GFCC_TRY(tmp.get(&B1, oo * ov));
  GFCC_TRY(tmp.get(&C1, oo * ov));
  GFCC_TRY(eri(0, o, 0, o, 0, o, o, v, 1.0, 0.0, B1, imap2(o, ov, o2v), imap1(1)));
  GFCC_TRY(eri(0, o, o, v, 0, o, 0, o, 1.0, 0.0, C1, imap2(v, 1, o2v), imap2(o, ov, v)));

  // ---- W1r[(i,j,a)][m] = W_maij
  double *W1r;
  GFCC_TRY(tmp.get(&W1r, o2v * o));
  GFCC_TRY(eri(0, o, 0, o, o, v, 0, o, 1.0, 0.0, W1r, imap2(o, o2v, 1), imap2(o, ov, o)));           // (mi|aj)'
  GFCC_TRY(gemm_f64(st, o2v, o, v, 1.0, t2, imap2(v, 1, vv), imap1(v), c->Fov, imap1(1), imap1(v), 1.0, W1r, imap1(o),
                    imap1(1)));                                                                        // Fbar_me t_ij^ea
  {
    // A1 = 2 B1 - C1 against t_jn^ae, then -B1 against t_jn^ea, -(me|nj)' against t_in^ea
    double *A1;
    GFCC_TRY(tmp.get(&A1, oo * ov));
    const long long d[4] = {1, 1, 1, oo * ov}, is[4] = {0, 0, 0, 1};
    GFCC_TRY(permute4(st, d, B1, is, A1, is, 2.0, 0.0));
    GFCC_TRY(permute4(st, d, C1, is, A1, is, -1.0, 1.0));
    GFCC_TRY(gemm_f64(st, oo, ov, ov, 1.0, A1, imap1(ov), imap1(1), t2, imap2(v, 1, vv), imap2(v, v, ov2), 1.0, W1r,
                      imap2(o, o2v, 1), imap2(v, o, ov)));
    GFCC_TRY(gemm_f64(st, oo, ov, ov, -1.0, B1, imap1(ov), imap1(1), t2, imap2(v, v, vv), imap2(v, 1, ov2), 1.0, W1r,
                      imap2(o, o2v, 1), imap2(v, o, ov)));
    GFCC_TRY(gemm_f64(st, oo, ov, ov, -1.0, C1, imap1(ov), imap1(1), t2, imap2(v, v, vv), imap2(v, 1, ov2), 1.0, W1r,
                      imap2(o, ov, 1), imap2(v, o, o2v)));
  }
  // + (me|af)' t_ij^ef over blocks of m: vc[m][e][a][f]
  {
    const long long mc = std::max<long long>(1, std::min<long long>(o, (1LL << 29) / std::max<long long>(1, v3)));
    double *vc;
    GFCC_TRY(tmp.get(&vc, mc * v3));
    for (long long m0 = 0; m0 < o; m0 += mc) {
      const long long nm = std::min<long long>(mc, o - m0);
      GFCC_TRY(eri(m0, nm, o, v, o, v, o, v, 1.0, 0.0, vc, imap2(v, vv, v3), imap1(1)));
      GFCC_TRY(gemm_f64(st, nm * v, oo, vv, 1.0, vc, imap2(v, v, v3), imap2(v, 1, vv), t2, imap1(1), imap1(vv), 1.0,
                        W1r + m0, imap2(v, o, 1), imap1(v * o)));
    }
  }

  // ---- ring matrices: Xr[(j,a)][(m,e)] = X_maej, Yr[(i,a)][(m,e)] = Y_maie
  double *Xr, *Yr;
  GFCC_TRY(tmp.get(&Xr, ov * ov));
  GFCC_TRY(tmp.get(&Yr, ov * ov));
  GFCC_TRY(eri(0, o, o, v, o, v, 0, o, 1.0, 0.0, Xr, imap1(1), imap2(o, ov * v, ov)));               // (me|aj)'
  GFCC_TRY(gemm_f64(st, ov, ov, ov, 1.0, t2, imap2(v, v, ov2), imap2(v, 1, vv), u2, imap2(v, 1, vv), imap2(v, v, ov2),
                    1.0, Xr, imap1(ov), imap1(1)));                                                   // u2 t_jn^af
  GFCC_TRY(gemm_f64(st, ov, ov, ov, -1.0, t2, imap2(v, 1, ov2), imap2(v, v, vv), u, imap2(v, 1, vv), imap2(v, v, ov2),
                    1.0, Xr, imap1(ov), imap1(1)));                                                   // -u t_jn^fa
  GFCC_TRY(eri(0, o, 0, o, o, v, o, v, 1.0, 0.0, Yr, imap2(o, ov * v, v), imap2(v, 1, ov)));         // (mi|ae)'
  GFCC_TRY(gemm_f64(st, ov, ov, ov, -1.0, t2, imap2(v, 1, ov2), imap2(v, v, vv), u, imap2(v, v, vv), imap2(v, 1, ov2),
                    1.0, Yr, imap1(ov), imap1(1)));                                                   // -u_mnfe t_in^fa
  // M1 = -Yr - d_ae Foo[m][i];  M2 = 2 Xr - Yr - d_ae Foo[m][j] + d_mj Fvv[a][e];  M3 = -Xr
  GFCC_TRY(dev_alloc(c, &c->rM1, ov * ov));
  GFCC_TRY(dev_alloc(c, &c->rM2, ov * ov));
  GFCC_TRY(dev_alloc(c, &c->rM3, ov * ov));
  {
    const long long d[4] = {1, 1, 1, ov * ov}, is[4] = {0, 0, 0, 1};
    GFCC_TRY(permute4(st, d, Yr, is, c->rM1, is, -1.0, 0.0));
    GFCC_TRY(permute4(st, d, Xr, is, c->rM2, is, 2.0, 0.0));
    GFCC_TRY(permute4(st, d, Yr, is, c->rM2, is, -1.0, 1.0));
    GFCC_TRY(permute4(st, d, Xr, is, c->rM3, is, -1.0, 0.0));
  }
  rhf_fold_kernel<<<cdiv(ov, 128), 128, 0, st>>>(c->rM1, o, v, c->Foo, c->Fvv, -1.0, 0.0);
  GFCC_LAUNCH_CHECK();
  rhf_fold_kernel<<<cdiv(ov, 128), 128, 0, st>>>(c->rM2, o, v, c->Foo, c->Fvv, -1.0, 1.0);
  GFCC_LAUNCH_CHECK();
  // digit planes of the three ring matrices, sliced once here for the digit-plane operator (when the
  // three together take at most a quarter of the free device memory)
  {
    const long long eb = emu_operand_bytes(ov, ov, RHF_EMU_DIGITS);
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      fr = 0;
    }
    if (3.0 * (double)eb <= 0.25 * (double)fr) {
      gfcc::EmuOperand *ops[3] = {&c->rM1e, &c->rM2e, &c->rM3e};
      double *mats[3] = {c->rM1, c->rM2, c->rM3};
      for (int k = 0; k < 3; k++) {
        double *mem;
        GFCC_TRY(dev_alloc(c, &mem, eb / 8 + 1));
        GFCC_TRY(emu_slice(st, mats[k], ov, ov, ov, RHF_EMU_DIGITS, mem, *ops[k]));
      }
    }
  }

  // ---- [(i,j,a)][e | m] = [-t_ij^ea | -W_maij]
  {
    double *T3;
    GFCC_TRY(tmp.get(&T3, o2v * v));
    const long long d[4] = {1, oo, v, v}, is[4] = {0, vv, 1, v}, os[4] = {0, vv, v, 1};   // (-, ij, a, e)
    GFCC_TRY(permute4(st, d, t2, is, T3, os, 1.0, 0.0));
    GFCC_TRY(dev_alloc(c, &c->rWT, o2v * (v + o)));
    rhf_concat_kernel<<<grid1d(o2v * (v + o)), 256, 0, st>>>(T3, v, W1r, o, o2v, -1.0, c->rWT);
    GFCC_LAUNCH_CHECK();
  }
  // ---- Vz[e][(m,n,f)] = u2[m][n][e][f]
  GFCC_TRY(dev_alloc(c, &c->rVz, v * o2v));
  {
    const long long d[4] = {oo, v, v, 1}, is[4] = {vv, v, 1, 0}, os[4] = {v, o2v, 1, 0};   // (mn, e, f)
    GFCC_TRY(permute4(st, d, u2, is, c->rVz, os, 1.0, 0.0));
  }
  // ---- the 1h row U1[i][m | (m,n,e)] = [-Foo[m][i] | B1[n][i][m][e] - 2 B1[m][i][n][e] + 2 d_mi Fov[n][e]
  //      - d_ni Fov[m][e]]
  {
    const long long K1 = o + o2v;
    GFCC_TRY(dev_alloc(c, &c->rU1, o * K1));
    GFCC_TRY(fill_f64(st, c->rU1, o * K1, 0.0));
    const long long d0[4] = {1, 1, o, o}, is0[4] = {0, 0, 1, o}, os0[4] = {0, 0, K1, 1};     // (i, m)
    GFCC_TRY(permute4(st, d0, c->Foo, is0, c->rU1, os0, -1.0, 1.0));
    const long long d[4] = {o, o, o, v};                                                    // (i, m, n, e)
    const long long isa[4] = {ov, v, o2v, 1}, isb[4] = {ov, o2v, v, 1}, os[4] = {K1, ov, v, 1};
    GFCC_TRY(permute4(st, d, B1, isa, c->rU1 + o, os, 1.0, 1.0));
    GFCC_TRY(permute4(st, d, B1, isb, c->rU1 + o, os, -2.0, 1.0));
    const long long df[4] = {1, o, o, v}, isf[4] = {0, 0, v, 1};                             // (-, i, n|m, e)
    const long long osm[4] = {0, K1 + ov, v, 1}, osn[4] = {0, K1 + v, ov, 1};
    GFCC_TRY(permute4(st, df, c->Fov, isf, c->rU1 + o, osm, 2.0, 1.0));                   // m = i
    GFCC_TRY(permute4(st, df, c->Fov, isf, c->rU1 + o, osn, -1.0, 1.0));                  // n = i
  }
  GFCC_TRY(dev_alloc(c, &c->diag_ip, c->dim_ip));
  rhf_diag_kernel<<<grid1d(c->dim_ip), 256, 0, st>>>(c->Foo, c->Fvv, o, v, c->diag_ip);
  GFCC_LAUNCH_CHECK();
  GFCC_CUDA(cudaStreamSynchronize(st));
  return GFCC_OK;
}

namespace {
struct EmulateScope {
  bool prev_big;
  double prev_min;
  explicit EmulateScope(bool on) : prev_big(g_emulate_big), prev_min(g_emulate_min_flops_local) {
    g_emulate_big = on;
    g_emulate_min_flops_local = on ? RHF_EMULATE_MIN_FLOPS : prev_min;
  }
  ~EmulateScope() {
    g_emulate_big = prev_big;
    g_emulate_min_flops_local = prev_min;
  }
};
}  // namespace

int apply_ip_rhf(gfcc_ctx *c, const SysBatch &b, double *work) {
  cudaStream_t st = c->stream;
  EmulateScope emu(c->rhf_emulate != 0);
  const long long o = c->o, v = c->v, ov = o * v, oo = o * o, o2v = oo * v, C2 = 2LL * b.nsys, dim = c->dim_ip;
  double *P = work;                    // [z (v rows) | r1u (o) | r2u (o^2 v)] x C2
  double *r1u = P + v * C2;
  double *r2u = r1u + o * C2;
  double *S1 = r2u + o2v * C2;         // [S1 (o) | S2 (o^2 v)] x C2
  double *S2 = S1 + o * C2;
  PhaseTimer tsig(c, PH_SIGMA, b.nsys * rhf_sigma_flops(c));
  rhf_unpack_kernel<<<grid1d(dim * b.nsys), 256, 0, st>>>(b, dim, C2, r1u);
  GFCC_LAUNCH_CHECK();
  // z[e][c] = Vz[e][(m,n,f)] r2u[(m,n,f)][c];  S2 = [-t | -W_maij] [z; r1u]
  GFCC_TRY(gemm_f64(st, v, C2, o2v, 1.0, c->rVz, imap1(o2v), imap1(1), r2u, imap1(C2), imap1(1), 0.0, P, imap1(C2),
                    imap1(1)));
  GFCC_TRY(gemm_f64(st, o2v, C2, v + o, 1.0, c->rWT, imap1(v + o), imap1(1), P, imap1(C2), imap1(1), 0.0, S2, imap1(C2),
                    imap1(1)));
  // + W_mnij r_mn^a
  GFCC_TRY(gemm_f64(st, oo, v * C2, oo, 1.0, c->Woooo, imap1(1), imap1(oo), r2u, imap1(v * C2), imap1(1), 1.0, S2,
                    imap1(v * C2), imap1(1)));
  {
    const double rflops = 2.0 * (double)ov * (double)ov * (double)(o * C2);
    PhaseTimer tr(c, PH_RING, 3.0 * rflops);
    // the ring matrix k times the B operand (maps bk, bn) into S2 (maps cm, cn): from its digit
    // planes cut at setup when the operator runs on digit planes, else through gemm_f64
    auto ring = [&](const double *Mk, const EmuOperand &Ek, IMap bk, IMap bn, IMap cm, IMap cn) -> int {
      if (c->rhf_emulate && Ek.dig != nullptr && rflops >= RHF_EMULATE_MIN_FLOPS)
        return gemm_f64_emulated_pre(st, Ek, o * C2, r2u, bk, bn, 1.0, 1.0, S2, cm, cn, RHF_EMU_LEVEL);
      return gemm_f64(st, ov, o * C2, ov, 1.0, Mk, imap1(ov), imap1(1), r2u, bk, bn, 1.0, S2, cm, cn);
    };
    // + M1[(i,a)][(m,e)] r[m][j][e]
    GFCC_TRY(ring(c->rM1, c->rM1e, imap2(v, C2, ov * C2), imap2(C2, 1, v * C2), imap2(v, C2, ov * C2),
                  imap2(C2, 1, v * C2)));
    // + M2[(j,a)][(m,e)] r[i][m][e] + M3[(j,a)][(m,e)] r[m][i][e]
    GFCC_TRY(ring(c->rM2, c->rM2e, imap1(C2), imap2(C2, 1, ov * C2), imap1(C2), imap2(C2, 1, ov * C2)));
    GFCC_TRY(ring(c->rM3, c->rM3e, imap2(v, C2, ov * C2), imap2(C2, 1, v * C2), imap1(C2), imap2(C2, 1, ov * C2)));
  }
  // S1 = U1 [r1u; r2u]
  GFCC_TRY(gemm_f64(st, o, C2, o + o2v, 1.0, c->rU1, imap1(o + o2v), imap1(1), r1u, imap1(C2), imap1(1), 0.0, S1,
                    imap1(C2), imap1(1)));
  rhf_epilogue_kernel<<<grid1d(dim * b.nsys), 256, 0, st>>>(b, dim, C2, r1u, S1);
  GFCC_LAUNCH_CHECK();
  return GFCC_OK;
}

int build_rhs_rhf(gfcc_ctx *c, int nsys, const int *d_porb, const int *d_mask, double *B, cudaStream_t st) {
  rhf_rhs_kernel<<<grid1d(c->dim_ip * nsys), 256, 0, st>>>(B, c->dim_ip, nsys, d_porb, c->o, c->v, c->t1, c->t2,
                                                           d_mask);
  GFCC_LAUNCH_CHECK();
  return GFCC_OK;
}

int build_left_rhf(gfcc_ctx *c, int nq, const int *d_orb, double *C, cudaStream_t st) {
  const long long n = c->dim_ip;
  rhf_left_1h_kernel<<<nq * c->o, 256, 0, st>>>(C, n, nq, d_orb, c->o, c->v, c->t1, c->t2, c->l1, c->l2);
  GFCC_LAUNCH_CHECK();
  if (n > c->o) {
    rhf_left_2h1p_kernel<<<grid1d((n - c->o) * nq), 256, 0, st>>>(C, n, nq, d_orb, c->o, c->v, c->t1, c->l1, c->l2);
    GFCC_LAUNCH_CHECK();
  }
  return GFCC_OK;
}

}  // namespace gfcc
