// FP64 sigma product and shifted operator of eq. xplin, batched over systems.
//
// A batch holds nsys packed complex vectors.  They are expanded into unpacked,
// antisymmetric, real "planar" columns (column c = 2 s + {0: Re, 1: Im}; the
// Hbar elements are real, so sigma(x) = sigma(Re x) + i sigma(Im x)), the sigma
// terms are evaluated as real contractions over all 2 nsys columns at once, and
// an epilogue antisymmetrises, adds the shift and packs the result:
//
//   IP:  y = (omega_s - i eta) u + sigma(u),   u = x / D_s   (D_s = 1 without preconditioner)
//   EA:  y = (omega_s + i eta) u - sigma(u)
//
// IP sigma (1h r1, 2h1p r2[i,j,a] antisymmetric in ij):
//   s1_i     = -Fbar_mi r1_m - Fbar_me r2_mie + 1/2 Wbar_nmie r2_mne
//   s2_ija   = Wbar_maji r1_m + Fbar_ae r2_ije - P(ij) Fbar_mi r2_mja + 1/2 Wbar_mnij r2_mna
//              + P(ij) Wbar_maei r2_mje + (1/2 <mn||ef>' r2_mnf) t_ij^ae
// EA sigma (1p y1, 2p1h y2[i,a,b] antisymmetric in ab):
//   s1_a     = Fbar_ae y1_e + Fbar_me y2_mae + 1/2 Wbar_amef y2_mef
//   s2_iab   = Wbar_abei y1_e - Fbar_mi y2_mab + P(ab) Fbar_be y2_iae + 1/2 Wbar_abef y2_ief
//              + P(ab) Wbar_mbei y2_mae - (1/2 <mn||ef>' y2_nef) t_mi^ab
// The Fbar_vv / Fbar_oo terms of the doubles block are folded into the ring
// matrices (see ctx.cuh), so one (ov) x (ov) contraction carries ring + Fock terms.
#include "ctx.cuh"
#include "kernels.cuh"
#include "sigma.cuh"
#include "epilogue.cuh"

namespace gfcc {

namespace {

struct Cplx {
  double r, i;
};
__device__ __forceinline__ Cplx cmul(Cplx a, Cplx b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__device__ __forceinline__ Cplx cdivz(Cplx a, Cplx b) {
  const double d = b.r * b.r + b.i * b.i;
  return {(a.r * b.r + a.i * b.i) / d, (a.i * b.r - a.r * b.i) / d};
}

// u = x / D_s(mu) for system s at packed index mu (sign = +1 IP: D = z + d, -1 EA: D = z - d)
__device__ __forceinline__ Cplx precond_in(const double *x, long long idx, const SysBatch &b, int s, long long mu) {
  Cplx u{x[2 * idx], x[2 * idx + 1]};
  if (b.diag != nullptr && b.omega != nullptr) {
    const Cplx D{b.omega[sysv(b, s)] + b.dsign * b.diag[mu], b.zsign * b.eta};
    u = cdivz(u, D);
  }
  return u;
}

// ---------------------------------------------------------------- IP
__global__ void unpack_ip_kernel(SysBatch b, int o, int v, long long C2, double *r1u, double *r2u) {
  const int ns = b.nsys;
  const long long tot2 = (long long)o * v * o * ns;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot2 + (long long)o * ns;
       t += (long long)gridDim.x * blockDim.x) {
    if (t < tot2) {
      const int s = (int)(t % ns);
      long long r = t / ns;
      const int j = (int)(r % o); r /= o;
      const int e = (int)(r % v);
      const int m = (int)(r / v);
      Cplx u{0.0, 0.0};
      if (m != j) {
        const long long lo = m < j ? m : j, hi = m < j ? j : m;
        const long long mu = o + pair_index(lo, hi, o) * v + e;
        u = precond_in(b.x, (long long)sysv(b, s) * b.ldx + mu, b, s, mu);
        if (m > j) { u.r = -u.r; u.i = -u.i; }
      }
      double *dst = r2u + (((long long)m * v + e) * o + j) * C2 + 2 * s;
      dst[0] = u.r;
      dst[1] = u.i;
    } else {
      const long long q = t - tot2;
      const int s = (int)(q % ns);
      const int m = (int)(q / ns);
      const Cplx u = precond_in(b.x, (long long)sysv(b, s) * b.ldx + m, b, s, m);
      r1u[(long long)m * C2 + 2 * s] = u.r;
      r1u[(long long)m * C2 + 2 * s + 1] = u.i;
    }
  }
}

// ---------------------------------------------------------------- EA
__global__ void unpack_ea_kernel(SysBatch b, int o, int v, long long Pv, long long C2, double *y1u, double *y2u,
                                 double *y2p) {
  const int ns = b.nsys;
  const long long totu = (long long)o * v * v * ns;
  const long long totp = Pv * o * ns;
  const long long tot1 = (long long)v * ns;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < totu + totp + tot1;
       t += (long long)gridDim.x * blockDim.x) {
    if (t < totu) {
      // y2u[m][e][a] = y2[m, a, e]
      const int s = (int)(t % ns);
      long long r = t / ns;
      const int a = (int)(r % v); r /= v;
      const int e = (int)(r % v);
      const int m = (int)(r / v);
      Cplx u{0.0, 0.0};
      if (a != e) {
        const long long lo = a < e ? a : e, hi = a < e ? e : a;
        const long long mu = v + (long long)m * Pv + pair_index(lo, hi, v);
        u = precond_in(b.x, (long long)sysv(b, s) * b.ldx + mu, b, s, mu);
        if (a > e) { u.r = -u.r; u.i = -u.i; }
      }
      double *dst = y2u + (((long long)m * v + e) * v + a) * C2 + 2 * s;
      dst[0] = u.r;
      dst[1] = u.i;
    } else if (t < totu + totp) {
      // y2p[(e<f)][i] = y2[i, e, f]
      const long long q = t - totu;
      const int s = (int)(q % ns);
      long long r = q / ns;
      const long long i = r % o;
      const long long ef = r / o;
      const long long mu = v + i * Pv + ef;
      const Cplx u = precond_in(b.x, (long long)sysv(b, s) * b.ldx + mu, b, s, mu);
      double *dst = y2p + (ef * o + i) * C2 + 2 * s;
      dst[0] = u.r;
      dst[1] = u.i;
    } else {
      const long long q = t - totu - totp;
      const int s = (int)(q % ns);
      const int a = (int)(q / ns);
      const Cplx u = precond_in(b.x, (long long)sysv(b, s) * b.ldx + a, b, s, a);
      y1u[(long long)a * C2 + 2 * s] = u.r;
      y1u[(long long)a * C2 + 2 * s + 1] = u.i;
    }
  }
}

}  // namespace

int launch_epilogue_ip(gfcc_ctx *c, const SysBatch &b, const double *S1, const double *T, const double *Q,
                       const double *U, const double *diag) {
  if (diag != nullptr)
    return epi::launch_ip<double, epi::MODE_OFFDIAG>(c->stream, b, c->o, c->v, S1, T, Q, U, diag);
  return epi::launch_ip<double, epi::MODE_FULL>(c->stream, b, c->o, c->v, S1, T, Q, U, nullptr);
}

int launch_epilogue_ea(gfcc_ctx *c, const SysBatch &b, const double *S1, const double *T, const double *Qp,
                       const double *U, const double *diag) {
  if (diag != nullptr)
    return epi::launch_ea<double, epi::MODE_OFFDIAG>(c->stream, b, c->o, c->v, c->Pv, S1, T, Qp, U, diag);
  return epi::launch_ea<double, epi::MODE_FULL>(c->stream, b, c->o, c->v, c->Pv, S1, T, Qp, U, nullptr);
}

double sigma_flops(const gfcc_ctx *c, int sector) {
  if (c->rhf) return rhf_sigma_flops(c);
  const double o = c->o, v = c->v;
  if (sector == GFCC_SECTOR_IP)
    return 2.0 * (2 * o * o * o * v * v + 0.5 * o * o * o * o * v + 3 * o * o * v * v + 4 * o * o * o * v +
                  2 * o * o * v + 2 * o * o);
  return 2.0 * (2 * o * o * v * v * v + 0.5 * o * v * v * v * v + 3 * o * v * v * v + 3 * o * o * v * v);
}

long long sigma_work_doubles(const gfcc_ctx *c, int sector, int nsys) {
  const long long o = c->o, v = c->v, C2 = 2LL * nsys;
  if (c->rhf) return rhf_work_doubles(c, nsys) + 64;
  if (sector == GFCC_SECTOR_IP) return (o + 4 * o * o * v + v + o) * C2 + 64;
  const long long Pv = c->Pv;
  return (v + 3 * o * v * v + 2 * Pv * o + o + v) * C2 + 64;
}

int apply_ip(gfcc_ctx *c, const SysBatch &b, double *work) {
  if (c->rhf) return apply_ip_rhf(c, b, work);
  cudaStream_t st = c->stream;
  const long long o = c->o, v = c->v, ov = o * v, C2 = 2LL * b.nsys;
  double *r1u = work;
  double *r2u = r1u + o * C2;
  double *T = r2u + o * v * o * C2;
  double *Q = T + o * v * o * C2;
  double *U = Q + o * o * v * C2;
  double *Z = U + o * v * o * C2;
  double *S1 = Z + v * C2;
  PhaseTimer tsig(c, PH_SIGMA, b.nsys * sigma_flops(c, GFCC_SECTOR_IP));
  unpack_ip_kernel<<<grid1d((o * v * o + o) * b.nsys), 256, 0, st>>>(b, (int)o, (int)v, C2, r1u, r2u);
  GFCC_LAUNCH_CHECK();
  // ring + Fock terms: T[(i,a)][(j,c)] = Wr[(i,a)][(m,e)] r2u[(m,e)][(j,c)]
  {
    PhaseTimer tr(c, PH_RING, 2.0 * (double)ov * (double)ov * (double)(o * C2));
    GFCC_TRY(gemm_f64(st, ov, o * C2, ov, 1.0, c->Wr_ip, imap1(ov), imap1(1), r2u, imap1(o * C2), imap1(1), 0.0, T,
                      imap1(o * C2), imap1(1)));
  }
  // Q[(i,j)][(a,c)] = 1/2 sum_mn Woooo[m][n][i][j] r2u[m][a][n][c]
  GFCC_TRY(gemm_f64(st, o * o, v * C2, o * o, 0.5, c->Woooo, imap1(1), imap1(o * o), r2u,
                    imap2(o, C2, v * o * C2), imap2(C2, 1, o * C2), 0.0, Q, imap1(v * C2), imap1(1)));
  // U[(i,a,j)][c] = W1 r1u + T3 Z,  Z[e][c] = V3[e][(m,f,n)] r2u[(m,f,n)][c]
  GFCC_TRY(gemm_f64(st, o * v * o, C2, o, 1.0, c->W1, imap1(o), imap1(1), r1u, imap1(C2), imap1(1), 0.0, U,
                    imap1(C2), imap1(1)));
  GFCC_TRY(gemm_f64(st, v, C2, o * v * o, 1.0, c->V3, imap1(o * v * o), imap1(1), r2u, imap1(C2), imap1(1), 0.0, Z,
                    imap1(C2), imap1(1)));
  GFCC_TRY(gemm_f64(st, o * v * o, C2, v, 1.0, c->T3, imap1(v), imap1(1), Z, imap1(C2), imap1(1), 1.0, U, imap1(C2),
                    imap1(1)));
  // S1[i][c] = -Foo[m][i] r1u[m][c] + U1[i][(m,e,n)] r2u[(m,e,n)][c]
  GFCC_TRY(gemm_f64(st, o, C2, o, -1.0, c->Foo, imap1(1), imap1(o), r1u, imap1(C2), imap1(1), 0.0, S1, imap1(C2),
                    imap1(1)));
  GFCC_TRY(gemm_f64(st, o, C2, o * v * o, 1.0, c->U1, imap1(o * v * o), imap1(1), r2u, imap1(C2), imap1(1), 1.0, S1,
                    imap1(C2), imap1(1)));
  GFCC_TRY((epi::launch_ip<double, epi::MODE_FULL>(st, b, (int)o, (int)v, S1, T, Q, U, nullptr)));
  return GFCC_OK;
}

int apply_ea(gfcc_ctx *c, const SysBatch &b, double *work) {
  cudaStream_t st = c->stream;
  const long long o = c->o, v = c->v, ov = o * v, C2 = 2LL * b.nsys, Pv = c->Pv;
  double *y1u = work;
  double *y2u = y1u + v * C2;
  double *T = y2u + o * v * v * C2;
  double *U = T + o * v * v * C2;
  double *y2p = U + o * v * v * C2;
  double *Qp = y2p + Pv * o * C2;
  double *Z = Qp + Pv * o * C2;
  double *S1 = Z + o * C2;
  PhaseTimer tsig(c, PH_SIGMA, b.nsys * sigma_flops(c, GFCC_SECTOR_EA));
  unpack_ea_kernel<<<grid1d((o * v * v + Pv * o + v) * b.nsys), 256, 0, st>>>(b, (int)o, (int)v, Pv, C2, y1u, y2u,
                                                                              y2p);
  GFCC_LAUNCH_CHECK();
  // T[(i,b)][(a,c)] = Wr_ea[(i,b)][(m,e)] y2u[(m,e)][(a,c)]
  {
    PhaseTimer tr(c, PH_RING, 2.0 * (double)ov * (double)ov * (double)(v * C2));
    GFCC_TRY(gemm_f64(st, ov, v * C2, ov, 1.0, c->Wr_ea, imap1(ov), imap1(1), y2u, imap1(v * C2), imap1(1), 0.0, T,
                      imap1(v * C2), imap1(1)));
  }
  // Qp[(a<b)][(i,c)] = Wp[(ab)][(ef)] y2p[(ef)][(i,c)]
  if (Pv > 0) {
    PhaseTimer tv(c, PH_VVVV, 2.0 * (double)Pv * (double)Pv * (double)(o * C2));
    GFCC_TRY(gemm_f64(st, Pv, o * C2, Pv, 1.0, c->Wp, imap1(Pv), imap1(1), y2p, imap1(o * C2), imap1(1), 0.0, Qp,
                      imap1(o * C2), imap1(1)));
  }
  // U[(i,b,a)][c] = W3 y1u + T3e Z,  Z[m][c] = V3e[m][(n,f,e)] y2u[(n,f,e)][c]
  GFCC_TRY(gemm_f64(st, o * v * v, C2, v, 1.0, c->W3, imap1(v), imap1(1), y1u, imap1(C2), imap1(1), 0.0, U,
                    imap1(C2), imap1(1)));
  GFCC_TRY(gemm_f64(st, o, C2, o * v * v, 1.0, c->V3e, imap1(o * v * v), imap1(1), y2u, imap1(C2), imap1(1), 0.0, Z,
                    imap1(C2), imap1(1)));
  GFCC_TRY(gemm_f64(st, o * v * v, C2, o, 1.0, c->T3e, imap1(o), imap1(1), Z, imap1(C2), imap1(1), 1.0, U,
                    imap1(C2), imap1(1)));
  // S1[a][c] = Fvv[a][e] y1u[e][c] + U1e[a][(m,x,y)] y2u[(m,x,y)][c]
  GFCC_TRY(gemm_f64(st, v, C2, v, 1.0, c->Fvv, imap1(v), imap1(1), y1u, imap1(C2), imap1(1), 0.0, S1, imap1(C2),
                    imap1(1)));
  GFCC_TRY(gemm_f64(st, v, C2, o * v * v, 1.0, c->U1e, imap1(o * v * v), imap1(1), y2u, imap1(C2), imap1(1), 1.0, S1,
                    imap1(C2), imap1(1)));
  GFCC_TRY((epi::launch_ea<double, epi::MODE_FULL>(st, b, (int)o, (int)v, Pv, S1, T, Qp, U, nullptr)));
  return GFCC_OK;
}

}  // namespace gfcc
