// Construction of the Hbar elements on the device (FP64), once per context.
//
// Implementation Details section of the paper: the contractions are arranged so
// that constant intermediates of size <= O(O^2 V^2) are precomputed before the
// frequency loop; the EA sector additionally keeps the vvvv block (packed over
// a<b, e<f).  The two-electron integrals are used only through Cholesky vectors.
//
// Route.  T1 enters as an orbital rotation: L'^K = (1-t) L^K (1+t) and
// h' = (1-t) h (1+t) with t[a][i] = t_i^a, so e^-T1 H e^T1 is again a two-body
// Hamiltonian; f' = h' + sum_j <pj||qj>' is its Fock matrix.  The T2 similarity
// transformation then gives the standard spin-orbital EOM-CCSD elements at T1 = 0:
//   Fbar_oo[m,i] = f'_mi + 1/2 <mn||ef>' t_in^ef        Fbar_vv[a,e] = f'_ae - 1/2 <mn||ef>' t_mn^af
//   Wbar_oooo    = <mn||ij>' + 1/2 <mn||ef>' t_ij^ef     Wbar_ooov    = <mn||ie>'
//   Wbar_ovvo    = <mb||ej>' - <mn||ef>' t_jn^fb
//   Wbar_ovoo    = <mb||ij>' - Fbar_me t_ij^be + 1/2 <mb||ef>' t_ij^ef + P(ij) <mn||ie>' t_jn^be
//   Wbar_vvvv    = <ab||ef>' + 1/2 <mn||ef>' t_mn^ab
//   Wbar_vvvo    = <ab||ei>' - Fbar_me t_mi^ab + 1/2 <mn||ei>' t_mn^ab - P(ab) <mb||ef>' t_mi^af
// with <pq||rs>' = (pr|qs)' - (ps|qr)', (pr|qs)' = sum_K L'^K_pr L'^K_qs.
// Every contraction below is one call of the strided FP64 contraction kernel; the
// index maps place the result directly in the layout the sigma product reads.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <initializer_list>
#include <vector>


#include "ctx.cuh"
#include "kernels.cuh"
#include "ozaki.cuh"

namespace gfcc {

namespace {

__global__ void permute4_kernel(long long d0, long long d1, long long d2, long long d3, const double *in,
                                long long i0s, long long i1s, long long i2s, long long i3s, double *out,
                                long long o0s, long long o1s, long long o2s, long long o3s, double alpha,
                                double beta) {
  const long long total = d0 * d1 * d2 * d3;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
       x += (long long)gridDim.x * blockDim.x) {
    long long r = x;
    const long long k3 = r % d3; r /= d3;
    const long long k2 = r % d2; r /= d2;
    const long long k1 = r % d1;
    const long long k0 = r / d1;
    const long long oo = k0 * o0s + k1 * o1s + k2 * o2s + k3 * o3s;
    double val = alpha * in[k0 * i0s + k1 * i1s + k2 * i2s + k3 * i3s];
    if (beta != 0.0) val += beta * out[oo];
    out[oo] = val;
  }
}

__global__ void fill_kernel(double *p, long long n, double value) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x)
    p[x] = value;
}

// d[K] = sum_{j<o} L[K][j][j]
__global__ void chol_trace_kernel(const double *Lc, int L, int n, int o, double *d) {
  const int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= L) return;
  const double *p = Lc + (long long)K * n * n;
  double s = 0.0;
  for (int j = 0; j < o; j++) s += p[(long long)j * (n + 1)];
  d[K] = s;
}

// Wr[(i,a)][(i,e)] += cvv * Fvv[a][e];  Wr[(i,a)][(m,a)] += coo * Foo[m][i]
__global__ void ring_diag_kernel(double *Wr, int o, int v, const double *Foo, const double *Fvv, double cvv,
                                 double coo) {
  const long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long ov = (long long)o * v;
  if (row >= ov) return;
  const int i = (int)(row / v), a = (int)(row % v);
  double *w = Wr + row * ov;
  for (int e = 0; e < v; e++) w[(long long)i * v + e] += cvv * Fvv[(long long)a * v + e];
  for (int m = 0; m < o; m++) w[(long long)m * v + a] += coo * Foo[(long long)m * o + i];
}

// Wp[(a<b)][(e<f)] = X[a-a0][e][b][f] - X[a-a0][f][b][e] for a in [a0, a0+na)
__global__ void pack_vvvv_kernel(const double *X, int v, int a0, int na, double *Wp, long long Pv) {
  const long long tot = (long long)na * v * Pv;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < tot; x += (long long)gridDim.x * blockDim.x) {
    const long long ef = x % Pv;
    const long long r = x / Pv;
    const int b = (int)(r % v);
    const int al = (int)(r / v);
    const int a = a0 + al;
    if (b <= a) continue;
    long long e, f;
    pair_decode(ef, v, e, f);
    const long long vv = (long long)v * v;
    const double val = X[((long long)al * v + e) * vv + (long long)b * v + f] - X[((long long)al * v + f) * vv + (long long)b * v + e];
    Wp[pair_index(a, b, v) * Pv + ef] = val;
  }
}

// out[mn][(a<b)] = in[mn][a][b]
__global__ void pack_pairs_kernel(const double *in, long long rows, int v, long long Pv, double *out) {
  const long long tot = rows * Pv;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < tot; x += (long long)gridDim.x * blockDim.x) {
    const long long ab = x % Pv, r = x / Pv;
    long long a, b;
    pair_decode(ab, v, a, b);
    out[x] = in[r * v * v + a * v + b];
  }
}

// packed Fock-like diagonals
__global__ void diag_ip_kernel(const double *Foo, const double *Fvv, int o, int v, double *d) {
  const long long dim = o + (long long)o * (o - 1) / 2 * v;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < dim; x += (long long)gridDim.x * blockDim.x) {
    if (x < o) {
      d[x] = -Foo[x * o + x];
      continue;
    }
    const long long r = x - o;
    const int a = (int)(r % v);
    long long i, j;
    pair_decode(r / v, o, i, j);
    d[x] = Fvv[(long long)a * v + a] - Foo[i * o + i] - Foo[j * o + j];
  }
}

__global__ void diag_ea_kernel(const double *Foo, const double *Fvv, int o, int v, double *d) {
  const long long Pv = (long long)v * (v - 1) / 2;
  const long long dim = v + (long long)o * Pv;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < dim; x += (long long)gridDim.x * blockDim.x) {
    if (x < v) {
      d[x] = Fvv[x * v + x];
      continue;
    }
    const long long r = x - v;
    const long long i = r / Pv;
    long long a, b;
    pair_decode(r % Pv, v, a, b);
    d[x] = Fvv[a * v + a] + Fvv[b * v + b] - Foo[i * o + i];
  }
}

// out[r][c] = bf16(scale * in[r * ld_in + c]) for c < cols (columns up to ld_out are zeroed)
__global__ void to_bf16_kernel(const double *in, long long rows, long long cols, long long ld_in, double scale,
                               __nv_bfloat16 *out, long long ld_out) {
  const long long tot = rows * ld_out;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < tot; x += (long long)gridDim.x * blockDim.x) {
    const long long r = x / ld_out, c = x - r * ld_out;
    out[x] = __double2bfloat16(c < cols ? scale * in[r * ld_in + c] : 0.0);
  }
}

// out[r] = [in1[r][0..k1) | in2[r][0..k2)] (rows of k1 + k2)
__global__ void concat_f64_kernel(const double *in1, long long k1, const double *in2, long long k2, long long rows,
                                  double *out) {
  const long long K = k1 + k2, tot = rows * K;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < tot; x += (long long)gridDim.x * blockDim.x) {
    const long long r = x / K, c = x - r * K;
    out[x] = c < k1 ? in1[r * k1 + c] : in2[r * k2 + (c - k1)];
  }
}

// out[r] = [bf16(in1[r][0..k1)) | bf16(in2[r][0..k2)) | 0 ...] (ld_out >= k1 + k2)
__global__ void concat_bf16_kernel(const double *in1, long long k1, const double *in2, long long k2, long long rows,
                                   __nv_bfloat16 *out, long long ld_out) {
  const long long tot = rows * ld_out;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < tot; x += (long long)gridDim.x * blockDim.x) {
    const long long r = x / ld_out, c = x - r * ld_out;
    const double val = c < k1 ? in1[r * k1 + c] : c < k1 + k2 ? in2[r * k2 + (c - k1)] : 0.0;
    out[x] = __double2bfloat16(val);
  }
}

// remove the Fock-like diagonal element of the folded ring matrix: Wr[(i,a)][(i,a)] -= cvv Fvv[a][a] + coo Foo[i][i]
__global__ void ring_undiag_kernel(double *Wr, int o, int v, const double *Foo, const double *Fvv, double cvv,
                                   double coo) {
  const long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long ov = (long long)o * v;
  if (row >= ov) return;
  const int i = (int)(row / v), a = (int)(row % v);
  Wr[row * ov + row] -= cvv * Fvv[(long long)a * v + a] + coo * Foo[(long long)i * o + i];
}

// p[k * stride] = 0 for k < count (zeroes a diagonal)
__global__ void diag_zero_kernel(double *p, int count, long long stride) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < count) p[(long long)k * stride] = 0.0;
}

// U1x[i][o2v + m] = -Foo[m][i] for m != i (the off-diagonal part of the 1h row)
__global__ void u1_foo_kernel(double *U1x, int o, long long o2v, long long ld, const double *Foo) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= o * o) return;
  const int i = t / o, m = t % o;
  U1x[(long long)i * ld + o2v + m] = (m == i) ? 0.0 : -Foo[(long long)m * o + i];
}

// Digit-level drops of a sector's digit-plane operands (see emu_level_drop): the smallest magnitude of
// the Fock-like diagonal entries cvv Fvv[a][a] + coo Foo[i][i] that the ring rows carried before the
// diagonal was taken out, against each operand's largest row scale.
int set_level_drops(gfcc_ctx *c, double cvv, double coo, std::initializer_list<EmuOperand *> ops) {
  const int o = c->o, v = c->v;
  std::vector<double> foo((size_t)o * o), fvv((size_t)v * v);
  GFCC_CUDA(cudaMemcpyAsync(foo.data(), c->Foo, sizeof(double) * o * o, cudaMemcpyDeviceToHost, c->stream));
  GFCC_CUDA(cudaMemcpyAsync(fvv.data(), c->Fvv, sizeof(double) * v * v, cudaMemcpyDeviceToHost, c->stream));
  GFCC_CUDA(cudaStreamSynchronize(c->stream));
  double mn = HUGE_VAL;
  for (int i = 0; i < o; i++)
    for (int a = 0; a < v; a++)
      mn = std::min(mn, std::fabs(cvv * fvv[(size_t)a * v + a] + coo * foo[(size_t)i * o + i]));
  for (EmuOperand *e : ops) {
    if (e->dig == nullptr || e->rows <= 0) continue;
    int emax = 0;
    GFCC_TRY(emu_max_exponent(c->stream, *e, &emax));
    e->drop = emu_level_drop(emax, mn);
  }
  return GFCC_OK;
}

}  // namespace

static inline long long round8(long long x) { return (x + 7) / 8 * 8; }

int permute4(cudaStream_t st, const long long d[4], const double *in, const long long is[4], double *out,
             const long long os[4], double alpha, double beta) {
  const long long total = d[0] * d[1] * d[2] * d[3];
  if (total <= 0) return GFCC_OK;
  long long hi_in = 0, hi_out = 0;
  for (int k = 0; k < 4; k++) {
    hi_in += (d[k] - 1) * is[k];
    hi_out += (d[k] - 1) * os[k];
  }
  GFCC_TRY(check_extent(in, 0, hi_in, "permute4 input"));
  GFCC_TRY(check_extent(out, 0, hi_out, "permute4 output"));
  permute4_kernel<<<grid1d(total), 256, 0, st>>>(d[0], d[1], d[2], d[3], in, is[0], is[1], is[2], is[3], out,
                                                   os[0], os[1], os[2], os[3], alpha, beta);
  GFCC_LAUNCH_CHECK();
  return GFCC_OK;
}

int fill_f64(cudaStream_t st, double *p, long long n, double value) {
  if (n <= 0) return GFCC_OK;
  fill_kernel<<<grid1d(n), 256, 0, st>>>(p, n, value);
  GFCC_LAUNCH_CHECK();
  return GFCC_OK;
}

int dev_alloc(gfcc_ctx *c, double **p, long long count) {
  *p = nullptr;
  if (count <= 0) count = 1;
  cudaError_t e = dmalloc((void **)p, (size_t)count * sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("device allocation of %lld doubles failed: %s", count, cudaGetErrorString(e));
    *p = nullptr;
    return GFCC_ERR_OOM;
  }
  c->allocs.push_back(*p);
  return GFCC_OK;
}

int dev_alloc_tmp(double **p, long long count) {
  *p = nullptr;
  if (count <= 0) count = 1;
  cudaError_t e = dmalloc((void **)p, (size_t)count * sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("device allocation of %lld doubles failed: %s", count, cudaGetErrorString(e));
    *p = nullptr;
    return GFCC_ERR_OOM;
  }
  return GFCC_OK;
}

int chol_eri(cudaStream_t st, const double *Lt, int n, int L, long long P0, long long np, long long R0, long long nr,
             long long Q0, long long nq, long long S0, long long ns, double alpha, double beta, double *C, IMap cm,
             IMap cn) {
  const long long nn = (long long)n * n;
  return gemm_f64(st, np * nr, nq * ns, L, alpha, Lt + P0 * n + R0, imap2(nr, 1, n), imap1(nn), Lt + Q0 * n + S0,
                  imap1(nn), imap2(ns, 1, n), beta, C, cm, cn);
}

int t1_dress(cudaStream_t st, const double *t1, int o, int v, double *M, long long batch, long long stride) {
  const int n = o + v;
  // M[p][i] += sum_a M[p][o+a] t1[i][a]
  GFCC_TRY(gemm_f64(st, n, o, v, 1.0, M + o, imap1(n), imap1(1), t1, imap1(1), imap1(v), 1.0, M, imap1(n), imap1(1),
                    batch, stride, 0, stride));
  // M[o+a][q] -= sum_i t1[i][a] M[i][q]
  GFCC_TRY(gemm_f64(st, v, n, o, -1.0, t1, imap1(1), imap1(v), M, imap1(n), imap1(1), 1.0, M + (long long)o * n,
                    imap1(n), imap1(1), batch, 0, stride, stride));
  return GFCC_OK;
}

int chol_coulomb_exchange(cudaStream_t st, const double *M, int n, int o, int L, double *F, double aj, double ak) {
  double *d;
  GFCC_TRY(dev_alloc_tmp(&d, L));
  chol_trace_kernel<<<cdiv(L, 128), 128, 0, st>>>(M, L, n, o, d);
  int s = cudaGetLastError() == cudaSuccess ? GFCC_OK : GFCC_ERR_CUDA;
  count_launch();
  const long long nn = (long long)n * n;
  if (s == GFCC_OK)
    s = gemm_f64(st, nn, 1, L, aj, M, imap1(1), imap1(nn), d, imap1(1), imap1(0), 1.0, F, imap1(1), imap1(0));
  if (s == GFCC_OK)
    s = gemm_f64(st, n, n, (long long)L * o, ak, M, imap1(n), imap2(o, 1, nn), M, imap2(o, n, nn), imap1(1), 1.0, F,
                 imap1(n), imap1(1));
  if (s == GFCC_ERR_CUDA) set_error("Coulomb/exchange build: %s", cudaGetErrorString(cudaGetLastError()));
  dfree(d);   // cudaFree waits for the launches above
  return s;
}

namespace {

int alloc_bf16(gfcc_ctx *c, __nv_bfloat16 **p, long long count) {
  double *d = nullptr;
  GFCC_TRY(dev_alloc(c, &d, (count + 3) / 4));
  *p = reinterpret_cast<__nv_bfloat16 *>(d);
  return GFCC_OK;
}

int to_bf16(cudaStream_t st, const double *in, long long rows, long long cols, long long ld_in, double scale,
            __nv_bfloat16 *out, long long ld_out) {
  GFCC_TRY(check_extent(in, 0, (rows - 1) * ld_in + cols - 1, "bf16 conversion input"));
  GFCC_TRY(check_extent_bytes(out, rows * ld_out * 2, "bf16 conversion output"));
  to_bf16_kernel<<<grid1d(rows * ld_out), 256, 0, st>>>(in, rows, cols, ld_in, scale, out, ld_out);
  GFCC_LAUNCH_CHECK();
  return GFCC_OK;
}

// RAII holder of setup temporaries.
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

struct Builder {
  gfcc_ctx *c;
  cudaStream_t st;
  int o, v, n, L;
  long long ov, oo, vv;
  double *Lt = nullptr;   // [K][p][q] T1-transformed Cholesky vectors
  double *fp = nullptr;   // [p][q] f'

  // Row map of a fused pair (p, r) of an Lt block: index p*|R| + r.
  IMap lt_pair(long long nr) const { return imap2(nr, 1, n); }
  const double *lt_block(long long p0, long long r0) const { return Lt + p0 * n + r0; }

  // C((p,r),(q,s)) (+)= alpha * sum_K L'[K][P0+p][R0+r] L'[K][Q0+q][S0+s]
  int eri(long long P0, long long np, long long R0, long long nr, long long Q0, long long nq, long long S0,
          long long ns, double alpha, double beta, double *C, IMap cm, IMap cn) {
    return chol_eri(st, Lt, n, L, P0, np, R0, nr, Q0, nq, S0, ns, alpha, beta, C, cm, cn);
  }

  // M <- (1 - t) M (1 + t) in place for `batch` n x n matrices spaced `stride` apart.
  int dress(double *M, long long batch, long long stride) { return t1_dress(st, c->t1, o, v, M, batch, stride); }

  // F[p][q] += alpha_j * sum_K M[K][p][q] tr_o(M[K]) + alpha_k * sum_K sum_j M[K][p][j] M[K][j][q]
  int coulomb_exchange(const double *M, double *F, double aj, double ak, Tmp &) {
    return chol_coulomb_exchange(st, M, n, o, L, F, aj, ak);
  }

  int copy_block(const double *src, long long ld_src, long long rows, long long cols, double *dst, double alpha,
                 double beta) {
    const long long d[4] = {1, 1, rows, cols};
    const long long is[4] = {0, 0, ld_src, 1};
    const long long os[4] = {0, 0, cols, 1};
    return permute4(st, d, src, is, dst, os, alpha, beta);
  }
};

}  // namespace

int build_hbar(gfcc_ctx *c, const double *d_fock, const double *d_chol) {
  Builder B;
  B.c = c;
  B.st = c->stream;
  B.o = c->o; B.v = c->v; B.n = c->n; B.L = c->L;
  const int o = c->o, v = c->v, n = c->n, L = c->L;
  const long long ov = (long long)o * v, oo = (long long)o * o, vv = (long long)v * v, nn = (long long)n * n;
  const long long ov2 = (long long)o * vv, o2v = oo * v;
  B.ov = ov; B.oo = oo; B.vv = vv;
  cudaStream_t st = c->stream;
  const bool want_ip = c->sectors & GFCC_SECTOR_IP, want_ea = c->sectors & GFCC_SECTOR_EA;
  Tmp tmp;

  // ---- T1-transformed Cholesky vectors and Fock matrix
  GFCC_TRY(tmp.get(&B.Lt, (long long)L * nn));
  GFCC_CUDA(cudaMemcpyAsync(B.Lt, d_chol, sizeof(double) * L * nn, cudaMemcpyDeviceToDevice, st));
  GFCC_TRY(B.dress(B.Lt, L, nn));
  double *h;
  GFCC_TRY(tmp.get(&h, nn));
  GFCC_CUDA(cudaMemcpyAsync(h, d_fock, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st));
  GFCC_TRY(B.coulomb_exchange(d_chol, h, -1.0, 1.0, tmp));    // h = f - J + K
  GFCC_TRY(B.dress(h, 1, nn));                                  // h' = (1-t) h (1+t)
  B.fp = h;
  GFCC_TRY(B.coulomb_exchange(B.Lt, B.fp, 1.0, -1.0, tmp));   // f' = h' + J' - K'
  const double *fp = B.fp;

  // ---- <mn||ef>' as [m][n][e][f]
  double *voovv;
  GFCC_TRY(tmp.get(&voovv, oo * vv));
  GFCC_TRY(B.eri(0, o, o, v, 0, o, o, v, 1.0, 0.0, voovv, imap2(v, v, ov2), imap2(v, 1, vv)));      // (me|nf)
  GFCC_TRY(B.eri(0, o, o, v, 0, o, o, v, -1.0, 1.0, voovv, imap2(v, 1, ov2), imap2(v, v, vv)));     // -(mf|ne)

  // ---- Fbar
  GFCC_TRY(dev_alloc(c, &c->Foo, oo));
  GFCC_TRY(dev_alloc(c, &c->Fvv, vv));
  GFCC_TRY(dev_alloc(c, &c->Fov, ov));
  GFCC_TRY(B.copy_block(fp, n, o, o, c->Foo, 1.0, 0.0));
  GFCC_TRY(B.copy_block(fp + (long long)o * n + o, n, v, v, c->Fvv, 1.0, 0.0));
  GFCC_TRY(B.copy_block(fp + o, n, o, v, c->Fov, 1.0, 0.0));
  // Foo[m][i] += 1/2 sum_{nef} v[m][n][e][f] t2[i][n][e][f]
  GFCC_TRY(gemm_f64(st, o, o, ov2, 0.5, voovv, imap1(ov2), imap1(1), c->t2, imap1(1), imap1(ov2), 1.0, c->Foo,
                    imap1(o), imap1(1)));
  // Fvv[a][e] -= 1/2 sum_{mn f} t2[mn][a][f] v[mn][e][f]
  GFCC_TRY(gemm_f64(st, v, v, oo * v, -0.5, c->t2, imap1(v), imap2(v, 1, vv), voovv, imap2(v, 1, vv), imap1(v), 1.0,
                    c->Fvv, imap1(v), imap1(1)));

  // ---- Wooov[m][n][i][e] = (mi|ne) - (me|ni)   (temporary)
  double *wooov;
  GFCC_TRY(tmp.get(&wooov, oo * ov));
  GFCC_TRY(B.eri(0, o, 0, o, 0, o, o, v, 1.0, 0.0, wooov, imap2(o, v, o2v), imap2(v, 1, ov)));
  GFCC_TRY(B.eri(0, o, o, v, 0, o, 0, o, -1.0, 1.0, wooov, imap2(v, 1, o2v), imap2(o, v, ov)));

  // ---- ring matrix core: Wr[(j,b)][(m,e)] = Wovvo[m,b,e,j]
  double *wr_core;
  GFCC_TRY(tmp.get(&wr_core, ov * ov));
  GFCC_TRY(B.eri(0, o, o, v, o, v, 0, o, 1.0, 0.0, wr_core, imap1(1), imap2(o, ov2, ov)));          // (me|bj)
  GFCC_TRY(B.eri(0, o, 0, o, o, v, o, v, -1.0, 1.0, wr_core, imap2(o, ov2, v), imap2(v, 1, ov)));   // -(mj|be)
  // - sum_{nf} t2[j][n][f][b] v[m][n][e][f]
  GFCC_TRY(gemm_f64(st, ov, ov, ov, -1.0, c->t2, imap2(v, 1, ov2), imap2(v, v, vv), voovv, imap2(v, 1, vv),
                    imap2(v, v, ov2), 1.0, wr_core, imap1(ov), imap1(1)));

  // ---- chunked <mb||ef>' = (me|bf) - (mf|be) as [m][b][e][f], shared by Wovoo (IP) and Wvvvo / Wvovv (EA)
  const long long v3 = vv * v;
  long long mc = std::max<long long>(1, std::min<long long>(o, (1LL << 29) / std::max<long long>(1, v3)));
  double *vc = nullptr;
  GFCC_TRY(tmp.get(&vc, mc * v3));

  if (want_ip) {
    GFCC_TRY(dev_alloc(c, &c->Wr_ip, ov * ov));
    GFCC_CUDA(cudaMemcpyAsync(c->Wr_ip, wr_core, sizeof(double) * ov * ov, cudaMemcpyDeviceToDevice, st));
    ring_diag_kernel<<<cdiv(ov, 128), 128, 0, st>>>(c->Wr_ip, o, v, c->Foo, c->Fvv, 0.5, -1.0);
    GFCC_LAUNCH_CHECK();

    // Woooo[m][n][i][j] = (mi|nj) - (mj|ni) + 1/2 v[mn][ef] t2[ij][ef]
    GFCC_TRY(dev_alloc(c, &c->Woooo, oo * oo));
    const long long o3 = oo * o;
    GFCC_TRY(B.eri(0, o, 0, o, 0, o, 0, o, 1.0, 0.0, c->Woooo, imap2(o, o, o3), imap2(o, 1, oo)));
    GFCC_TRY(B.eri(0, o, 0, o, 0, o, 0, o, -1.0, 1.0, c->Woooo, imap2(o, 1, o3), imap2(o, o, oo)));
    GFCC_TRY(gemm_f64(st, oo, oo, vv, 0.5, voovv, imap1(vv), imap1(1), c->t2, imap1(1), imap1(vv), 1.0, c->Woooo,
                      imap1(oo), imap1(1)));

    // W1[(y,b,x)][m] = Wovoo[m,b,x,y]: offset ((y v + b) o + x) o + m
    GFCC_TRY(dev_alloc(c, &c->W1, o2v * o));
    const long long vo2 = (long long)v * oo;
    GFCC_TRY(B.eri(0, o, 0, o, o, v, 0, o, 1.0, 0.0, c->W1, imap2(o, o, 1), imap2(o, vo2, oo)));      // (mx|by)
    GFCC_TRY(B.eri(0, o, 0, o, o, v, 0, o, -1.0, 1.0, c->W1, imap2(o, vo2, 1), imap2(o, o, oo)));     // -(my|bx)
    // - sum_e Fov[m][e] t2[x][y][b][e], batched over x
    GFCC_TRY(gemm_f64(st, o, ov, v, -1.0, c->Fov, imap1(v), imap1(1), c->t2, imap1(1), imap2(v, v, vv), 1.0, c->W1,
                      imap1(1), imap2(v, oo, vo2), o, 0, ov2, o));
    // + P(xy) sum_{ne} Wooov[m][n][x][e] t2[y][n][b][e]
    GFCC_TRY(gemm_f64(st, oo, ov, ov, 1.0, wooov, imap2(o, v, o2v), imap2(v, 1, ov), c->t2, imap2(v, 1, vv),
                      imap2(v, v, ov2), 1.0, c->W1, imap2(o, o, 1), imap2(v, oo, vo2)));
    GFCC_TRY(gemm_f64(st, oo, ov, ov, -1.0, wooov, imap2(o, v, o2v), imap2(v, 1, ov), c->t2, imap2(v, 1, vv),
                      imap2(v, v, ov2), 1.0, c->W1, imap2(o, vo2, 1), imap2(v, oo, o)));

    // V3[e][(m,f,n)] = 1/2 v[m][n][e][f];  T3[(i,a,j)][e] = t2[i][j][a][e]
    GFCC_TRY(dev_alloc(c, &c->V3, oo * vv));
    GFCC_TRY(dev_alloc(c, &c->T3, oo * vv));
    {
      const long long d[4] = {v, o, v, o};
      const long long is[4] = {v, ov2, 1, vv};
      const long long os[4] = {oo * v, ov, o, 1};
      GFCC_TRY(permute4(st, d, voovv, is, c->V3, os, 0.5, 0.0));
    }
    {
      const long long d[4] = {o, v, o, v};
      const long long is[4] = {ov2, v, vv, 1};
      const long long os[4] = {vv * o, ov, v, 1};
      GFCC_TRY(permute4(st, d, c->t2, is, c->T3, os, 1.0, 0.0));
    }
    // U1[i][(m,e,n)] = 1/2 Wooov[n][m][i][e] - d_in Fov[m][e]
    GFCC_TRY(dev_alloc(c, &c->U1, o * o2v));
    {
      const long long d[4] = {o, o, v, o};
      const long long is[4] = {v, ov, 1, o2v};
      const long long os[4] = {o2v, ov, o, 1};
      GFCC_TRY(permute4(st, d, wooov, is, c->U1, os, 0.5, 0.0));
      const long long d2[4] = {1, o, o, v};             // (-, i, m, e) -> U1[i][m][e][i]
      const long long is2[4] = {0, 0, v, 1};
      const long long os2[4] = {0, o2v + 1, ov, o};
      GFCC_TRY(permute4(st, d2, c->Fov, is2, c->U1, os2, -1.0, 1.0));
    }
    GFCC_TRY(dev_alloc(c, &c->diag_ip, c->dim_ip));
    diag_ip_kernel<<<grid1d(c->dim_ip), 256, 0, st>>>(c->Foo, c->Fvv, o, v, c->diag_ip);
    GFCC_LAUNCH_CHECK();

  }

  if (want_ea) {
    GFCC_TRY(dev_alloc(c, &c->Wr_ea, ov * ov));
    GFCC_CUDA(cudaMemcpyAsync(c->Wr_ea, wr_core, sizeof(double) * ov * ov, cudaMemcpyDeviceToDevice, st));
    ring_diag_kernel<<<cdiv(ov, 128), 128, 0, st>>>(c->Wr_ea, o, v, c->Foo, c->Fvv, 1.0, -0.5);
    GFCC_LAUNCH_CHECK();

    // Wp[(a<b)][(e<f)] = (ae|bf) - (af|be) + 1/2 sum_mn t2[mn][ab] v[mn][ef]
    const long long Pv = c->Pv;
    GFCC_TRY(dev_alloc(c, &c->Wp, std::max<long long>(1, Pv * Pv)));
    if (Pv > 0) {
      long long ac = std::max<long long>(1, std::min<long long>(v, (1LL << 29) / std::max<long long>(1, v3)));
      double *x4;
      GFCC_TRY(tmp.get(&x4, ac * v3));
      for (long long a0 = 0; a0 < v; a0 += ac) {
        const long long na = std::min<long long>(ac, v - a0);
        GFCC_TRY(B.eri(o + a0, na, o, v, o, v, o, v, 1.0, 0.0, x4, imap1(vv), imap1(1)));
        pack_vvvv_kernel<<<grid1d(na * v * Pv), 256, 0, st>>>(x4, v, (int)a0, (int)na, c->Wp, Pv);
        GFCC_LAUNCH_CHECK();
      }
      double *t2p, *vp;
      GFCC_TRY(tmp.get(&t2p, oo * Pv));
      GFCC_TRY(tmp.get(&vp, oo * Pv));
      pack_pairs_kernel<<<grid1d(oo * Pv), 256, 0, st>>>(c->t2, oo, v, Pv, t2p);
      GFCC_LAUNCH_CHECK();
      pack_pairs_kernel<<<grid1d(oo * Pv), 256, 0, st>>>(voovv, oo, v, Pv, vp);
      GFCC_LAUNCH_CHECK();
      GFCC_TRY(gemm_f64(st, Pv, Pv, oo, 0.5, t2p, imap1(1), imap1(Pv), vp, imap1(Pv), imap1(1), 1.0, c->Wp,
                        imap1(Pv), imap1(1)));
    }

    // W3[(i,b,a)][e] = Wvvvo[a,b,e,i]: offset ((i v + b) v + a) v + e
    GFCC_TRY(dev_alloc(c, &c->W3, ov2 * v));
    GFCC_TRY(B.eri(o, v, o, v, o, v, 0, o, 1.0, 0.0, c->W3, imap1(1), imap2(o, v3, vv)));           // (ae|bi)
    GFCC_TRY(B.eri(o, v, 0, o, o, v, o, v, -1.0, 1.0, c->W3, imap2(o, v3, v), imap2(v, 1, vv)));    // -(ai|be)
    // - sum_m Fov[m][e] t2[m][i][a][b], batched over i
    GFCC_TRY(gemm_f64(st, vv, v, o, -1.0, c->t2, imap1(1), imap1(ov2), c->Fov, imap1(v), imap1(1), 1.0, c->W3,
                      imap2(v, vv, v), imap1(1), o, vv, 0, v3));
    // - 1/2 sum_mn Wooov[mn][i][e] t2[mn][a][b]
    GFCC_TRY(gemm_f64(st, vv, ov, oo, -0.5, c->t2, imap1(1), imap1(vv), wooov, imap1(ov), imap1(1), 1.0, c->W3,
                      imap2(v, vv, v), imap2(v, 1, v3)));

    // V3e[m][(n,f,e)] = 1/2 v[m][n][e][f];  T3e[(i,b,a)][m] = -t2[m][i][a][b]
    GFCC_TRY(dev_alloc(c, &c->V3e, oo * vv));
    GFCC_TRY(dev_alloc(c, &c->T3e, oo * vv));
    {
      const long long d[4] = {o, o, v, v};
      const long long is[4] = {ov2, vv, 1, v};
      const long long os[4] = {ov2, vv, v, 1};
      GFCC_TRY(permute4(st, d, voovv, is, c->V3e, os, 0.5, 0.0));
    }
    {
      const long long d[4] = {o, v, v, o};
      const long long is[4] = {vv, 1, v, ov2};
      const long long os[4] = {v * v * o, v * o, o, 1};
      GFCC_TRY(permute4(st, d, c->t2, is, c->T3e, os, -1.0, 0.0));
    }
    // U1e[a][(m,x,y)]: Fov[m][e] at [a][m][e][a]; -1/2 <ma||ef>' at [a][m][f][e] (below, per m chunk)
    GFCC_TRY(dev_alloc(c, &c->U1e, (long long)v * ov2));
    GFCC_TRY(fill_f64(st, c->U1e, (long long)v * ov2, 0.0));
    {
      const long long d[4] = {1, v, o, v};               // (-, a, m, e)
      const long long is[4] = {0, 0, v, 1};
      const long long os[4] = {0, ov2 + 1, vv, v};
      GFCC_TRY(permute4(st, d, c->Fov, is, c->U1e, os, 1.0, 1.0));
    }
    GFCC_TRY(dev_alloc(c, &c->diag_ea, c->dim_ea));
    diag_ea_kernel<<<grid1d(c->dim_ea), 256, 0, st>>>(c->Foo, c->Fvv, o, v, c->diag_ea);
    GFCC_LAUNCH_CHECK();
  }

  // ---- terms that need <mb||ef>' (o v^3), computed in chunks of m
  for (long long m0 = 0; m0 < o; m0 += mc) {
    const long long nm = std::min<long long>(mc, o - m0);
    // vc[m][b][e][f] = (me|bf) - (mf|be)
    GFCC_TRY(B.eri(m0, nm, o, v, o, v, o, v, 1.0, 0.0, vc, imap2(v, v, v3), imap2(v, 1, vv)));
    GFCC_TRY(B.eri(m0, nm, o, v, o, v, o, v, -1.0, 1.0, vc, imap2(v, 1, v3), imap2(v, v, vv)));
    if (want_ip) {
      // W1[(y,b,x)][m] += 1/2 sum_ef vc[m][b][e][f] t2[x][y][e][f]
      const long long vo2 = (long long)v * oo;
      GFCC_TRY(gemm_f64(st, nm * v, oo, vv, 0.5, vc, imap1(vv), imap1(1), c->t2, imap1(1), imap1(vv), 1.0,
                        c->W1 + m0, imap2(v, oo, 1), imap2(o, vo2, o)));
    }
    if (want_ea) {
      // Wvvvo[a,b,e,i] -= T5[a,b,e,i] - T5[b,a,e,i],  T5 = sum_{mf} vc[m][b][e][f] t2[m][i][a][f]
      GFCC_TRY(gemm_f64(st, vv, ov, nm * v, -1.0, vc, imap1(v), imap2(v, 1, v3), c->t2 + m0 * ov2,
                        imap2(v, 1, ov2), imap1(v), 1.0, c->W3, imap2(v, 1, vv), imap2(v, v, v3)));
      GFCC_TRY(gemm_f64(st, vv, ov, nm * v, 1.0, vc, imap1(v), imap2(v, 1, v3), c->t2 + m0 * ov2,
                        imap2(v, 1, ov2), imap1(v), 1.0, c->W3, imap2(v, 1, v), imap2(v, vv, v3)));
      // U1e[a][m][f][e] += -1/2 vc[m][a][e][f]
      const long long d[4] = {nm, v, v, v};              // (m, a, e, f)
      const long long is[4] = {v3, vv, v, 1};
      const long long os[4] = {vv, ov2, 1, v};
      GFCC_TRY(permute4(st, d, vc, is, c->U1e + m0 * vv, os, -0.5, 1.0));
    }
  }
  // BF16 operands of the mixed-precision sigma, after every FP64 term is in place
  if (want_ip && c->precision == GFCC_PREC_MIXED_BF16) {
    // BF16 operands of the mixed-precision sigma (the Fock-like diagonal stays in FP64)
    c->ld_ov = round8(ov);
    c->ld_o2 = round8(oo);
    c->ld_o = round8(o);
    c->ld_o2v = round8(o2v);
    c->ld_v = round8(v);
    c->ld_k1 = round8(o2v + o);
    double *t;
    GFCC_TRY(tmp.get(&t, std::max(ov * ov, o * (o2v + o))));
    GFCC_CUDA(cudaMemcpyAsync(t, wr_core, sizeof(double) * ov * ov, cudaMemcpyDeviceToDevice, st));
    ring_diag_kernel<<<cdiv(ov, 128), 128, 0, st>>>(t, o, v, c->Foo, c->Fvv, 0.5, -1.0);
    GFCC_LAUNCH_CHECK();
    ring_undiag_kernel<<<cdiv(ov, 128), 128, 0, st>>>(t, o, v, c->Foo, c->Fvv, 0.5, -1.0);
    GFCC_LAUNCH_CHECK();
    GFCC_TRY(alloc_bf16(c, &c->Wr_bf, ov * c->ld_ov));
    GFCC_TRY(to_bf16(st, t, ov, ov, ov, 1.0, c->Wr_bf, c->ld_ov));
    // Digit planes of the FP64 operands for the FP64-accurate residual: the same couplings as the BF16
    // operands (the exact Fock-like diagonal is applied in FP64 by the epilogue), so that each row's
    // scale, and with it the truncation error of the digit pairs, is set by the couplings
    const int S = c->emu_S;
    auto slice = [&](const double *A, long long rows, long long K, long long lda, EmuOperand &e) -> int {
      double *mem;
      GFCC_TRY(dev_alloc(c, &mem, emu_operand_bytes(rows, K, S) / 8 + 1));
      return emu_slice(st, A, rows, K, lda, S, mem, e);
    };
    GFCC_TRY(slice(t, ov, ov, ov, c->eWr));
    // Wq[(i,j)][(m,n)] = 1/2 Woooo[m][n][i][j]
    {
      const long long d[4] = {o, o, o, o};          // (i, j, m, n)
      const long long is[4] = {o, 1, o * oo, oo};
      const long long os[4] = {o * oo, oo, o, 1};
      GFCC_TRY(permute4(st, d, c->Woooo, is, t, os, 1.0, 0.0));
    }
    GFCC_TRY(alloc_bf16(c, &c->Wq_bf, oo * c->ld_o2));
    GFCC_TRY(to_bf16(st, t, oo, oo, oo, 0.5, c->Wq_bf, c->ld_o2));
    // [W1 | T3]: the ovoo and three-body terms of U share one contraction over K = o + v
    c->ld_ot = round8(o + v);
    GFCC_TRY(alloc_bf16(c, &c->WT_bf, o2v * c->ld_ot));
    concat_bf16_kernel<<<grid1d(o2v * c->ld_ot), 256, 0, st>>>(c->W1, o, c->T3, v, o2v, c->WT_bf, c->ld_ot);
    GFCC_LAUNCH_CHECK();
    GFCC_TRY(alloc_bf16(c, &c->V3_bf, v * c->ld_o2v));
    GFCC_TRY(to_bf16(st, c->V3, v, o2v, o2v, 1.0, c->V3_bf, c->ld_o2v));
    // U1x[i] = [U1[i][(m,e,n)] | -Foo_offdiag[m][i]]
    {
      const long long d[4] = {1, 1, o, o2v};
      const long long is[4] = {0, 0, o2v, 1};
      const long long os[4] = {0, 0, o2v + o, 1};
      GFCC_TRY(permute4(st, d, c->U1, is, t, os, 1.0, 0.0));
    }
    u1_foo_kernel<<<cdiv(oo, 128), 128, 0, st>>>(t, o, o2v, o2v + o, c->Foo);
    GFCC_LAUNCH_CHECK();
    GFCC_TRY(alloc_bf16(c, &c->U1_bf, o * c->ld_k1));
    GFCC_TRY(to_bf16(st, t, o, o2v + o, o2v + o, 1.0, c->U1_bf, c->ld_k1));

    // the other digit-plane operands (oooo, [ovoo | three-body], three-body Z, 1h row)
    {
      const long long d[4] = {o, o, o, o};          // (i, j, m, n)
      const long long is[4] = {o, 1, o * oo, oo};
      const long long os[4] = {o * oo, oo, o, 1};
      GFCC_TRY(permute4(st, d, c->Woooo, is, t, os, 0.5, 0.0));
    }
    GFCC_TRY(slice(t, oo, oo, oo, c->eWq));
    {
      // [W1 | T3] with one exponent per row over K = o + v (one product with [r1 | Z])
      double *wt;
      GFCC_TRY(tmp.get(&wt, o2v * (o + v)));
      concat_f64_kernel<<<grid1d(o2v * (o + v)), 256, 0, st>>>(c->W1, o, c->T3, v, o2v, wt);
      GFCC_LAUNCH_CHECK();
      GFCC_TRY(slice(wt, o2v, o + v, o + v, c->eWT));
    }
    double *t2x;
    GFCC_TRY(tmp.get(&t2x, std::max(v, o) * (o2v + o)));
    {
      // [V3 | 0]: V3 padded to the K of the 1h row
      GFCC_TRY(fill_f64(st, t2x, v * (o2v + o), 0.0));
      const long long d[4] = {1, 1, v, o2v};
      const long long is[4] = {0, 0, o2v, 1};
      const long long os[4] = {0, 0, o2v + o, 1};
      GFCC_TRY(permute4(st, d, c->V3, is, t2x, os, 1.0, 0.0));
    }
    GFCC_TRY(slice(t2x, v, o2v + o, o2v + o, c->eV3));
    {
      // [U1 | -Fbar_oo^T off the diagonal]: the 1h row without its diagonal -Fbar_oo[i][i]
      const long long d[4] = {1, 1, o, o2v};
      const long long is[4] = {0, 0, o2v, 1};
      const long long os[4] = {0, 0, o2v + o, 1};
      GFCC_TRY(permute4(st, d, c->U1, is, t2x, os, 1.0, 0.0));
      u1_foo_kernel<<<cdiv(oo, 128), 128, 0, st>>>(t2x, o, o2v, o2v + o, c->Foo);
      GFCC_LAUNCH_CHECK();
    }
    GFCC_TRY(slice(t2x, o, o2v + o, o2v + o, c->eU1));
    GFCC_TRY(set_level_drops(c, 0.5, -1.0, {&c->eWr, &c->eWq, &c->eWT, &c->eV3, &c->eU1}));
  }
  if (want_ea && c->precision == GFCC_PREC_MIXED_BF16) {
    // BF16 EA operands (the Fock-like diagonal stays in FP64) and their FP64 digit planes
    const long long Pv = c->Pv;
    c->ld_ov = round8(ov);
    c->ld_o = round8(o);
    c->ld_v = round8(v);
    c->ld_pv = round8(std::max<long long>(Pv, 1));
    c->ld_ov2 = round8(ov2);
    c->ld_k1e = round8(ov2 + v);
    const int S = c->emu_S;
    auto slice = [&](const double *A, long long rows, long long K, long long lda, EmuOperand &e) -> int {
      double *mem;
      GFCC_TRY(dev_alloc(c, &mem, emu_operand_bytes(rows, K, S) / 8 + 1));
      return emu_slice(st, A, rows, K, lda, S, mem, e);
    };
    double *t;
    GFCC_TRY(tmp.get(&t, std::max(ov * ov, std::max<long long>(o, v) * (ov2 + v))));
    // ring: Wr_ea without the diagonal entries Fbar_vv[b][b] - 1/2 Fbar_oo[i][i]
    GFCC_CUDA(cudaMemcpyAsync(t, c->Wr_ea, sizeof(double) * ov * ov, cudaMemcpyDeviceToDevice, st));
    ring_undiag_kernel<<<cdiv(ov, 128), 128, 0, st>>>(t, o, v, c->Foo, c->Fvv, 1.0, -0.5);
    GFCC_LAUNCH_CHECK();
    GFCC_TRY(alloc_bf16(c, &c->Wre_bf, ov * c->ld_ov));
    GFCC_TRY(to_bf16(st, t, ov, ov, ov, 1.0, c->Wre_bf, c->ld_ov));
    // digit planes of the same couplings (the exact diagonal is applied in FP64 by the epilogue)
    GFCC_TRY(slice(t, ov, ov, ov, c->eWre));
    if (Pv > 0) {
      GFCC_TRY(alloc_bf16(c, &c->Wp_bf, Pv * c->ld_pv));
      GFCC_TRY(to_bf16(st, c->Wp, Pv, Pv, Pv, 1.0, c->Wp_bf, c->ld_pv));
      GFCC_TRY(slice(c->Wp, Pv, Pv, Pv, c->eWp));
    }
    // [W3 | T3e]: one contraction over K = v + o for U
    c->ld_ot = round8(o + v);
    GFCC_TRY(alloc_bf16(c, &c->WTe_bf, ov2 * c->ld_ot));
    concat_bf16_kernel<<<grid1d(ov2 * c->ld_ot), 256, 0, st>>>(c->W3, v, c->T3e, o, ov2, c->WTe_bf, c->ld_ot);
    GFCC_LAUNCH_CHECK();
    {
      // [W3 | T3e] with one exponent per row over K = v + o
      double *wt;
      GFCC_TRY(tmp.get(&wt, ov2 * (v + o)));
      concat_f64_kernel<<<grid1d(ov2 * (v + o)), 256, 0, st>>>(c->W3, v, c->T3e, o, ov2, wt);
      GFCC_LAUNCH_CHECK();
      GFCC_TRY(slice(wt, ov2, v + o, v + o, c->eWTe));
    }
    GFCC_TRY(alloc_bf16(c, &c->V3e_bf, o * c->ld_ov2));
    GFCC_TRY(to_bf16(st, c->V3e, o, ov2, ov2, 1.0, c->V3e_bf, c->ld_ov2));
    // [V3e | 0]: padded to the K of the 1p row
    {
      const long long d[4] = {1, 1, o, ov2};
      const long long is[4] = {0, 0, ov2, 1};
      const long long os[4] = {0, 0, ov2 + v, 1};
      GFCC_TRY(fill_f64(st, t, o * (ov2 + v), 0.0));
      GFCC_TRY(permute4(st, d, c->V3e, is, t, os, 1.0, 0.0));
    }
    GFCC_TRY(slice(t, o, ov2 + v, ov2 + v, c->eV3e));
    // 1p row: [U1e | Fbar_vv off the diagonal] (the diagonal Fbar_vv[a][a] is applied in FP64), for the
    // digit planes and the BF16 operand
    {
      const long long d[4] = {1, 1, v, ov2};
      const long long is[4] = {0, 0, ov2, 1};
      const long long os[4] = {0, 0, ov2 + v, 1};
      GFCC_TRY(permute4(st, d, c->U1e, is, t, os, 1.0, 0.0));
      const long long d2[4] = {1, 1, v, v};             // t[a][ov2 + e] = Fvv[a][e]
      const long long is2[4] = {0, 0, v, 1};
      const long long os2[4] = {0, 0, ov2 + v, 1};
      GFCC_TRY(permute4(st, d2, c->Fvv, is2, t + ov2, os2, 1.0, 0.0));
    }
    diag_zero_kernel<<<cdiv(v, 128), 128, 0, st>>>(t + ov2, v, ov2 + v + 1);
    GFCC_LAUNCH_CHECK();
    GFCC_TRY(slice(t, v, ov2 + v, ov2 + v, c->eU1e));
    GFCC_TRY(set_level_drops(c, 1.0, -0.5, {&c->eWre, &c->eWp, &c->eWTe, &c->eV3e, &c->eU1e}));
    GFCC_TRY(alloc_bf16(c, &c->U1e_bf, v * c->ld_k1e));
    GFCC_TRY(to_bf16(st, t, v, ov2 + v, ov2 + v, 1.0, c->U1e_bf, c->ld_k1e));
  }
  GFCC_CUDA(cudaStreamSynchronize(st));
  return GFCC_OK;
}

}  // namespace gfcc
