// FP64-accurate IP operator y = (omega - i eta) x + sigma(x) evaluated from base-64 digit
// planes on the BF16 tensor cores (ozaki.cu), for the residuals of the mixed-precision
// refinement.  Same contractions, layouts and operator couplings as the BF16 operator of
// sigma_mixed.cu: the exact Fock-like diagonal and the shift are applied in FP64 by the epilogue,
// and every coupling product is FP64-accurate, so the refinement converges to the FP64 solution.
// Leaving the diagonal (orbital energies, order 1 Hartree) out of the digit planes lets each row's
// power-of-two scale follow its couplings (about three orders of magnitude smaller on the synthetic
// workloads), which lowers the truncation error of a given digit level by the same factor.
//
// Each vector plane (system s, re/im) shares one power-of-two scale: its packed entries are
// written as digits of x 2^-e_c directly by the unpack kernels, so no FP64 copy of the
// unpacked layouts is made.  Systems are processed in sub-batches that fit the workspace.
#include <cuda_bf16.h>

#include "ctx.cuh"
#include "kernels.cuh"
#include "ozaki.cuh"
#include "sigma.cuh"
#include "umma.cuh"

namespace gfcc {

namespace {

// e[c] (c = 2 s + re/im) with max_mu |x_s| * 2^-e in [1/4, 1/2)
__global__ void plane_exp_kernel(const double *x, long long ldx, long long n, int *e) {
  __shared__ double sh[32];
  const int c = blockIdx.x, s = c >> 1, t = c & 1;
  double mx = 0.0;
  for (long long mu = threadIdx.x; mu < n; mu += blockDim.x) mx = fmax(mx, fabs(x[2 * (s * ldx + mu) + t]));
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) mx = fmax(mx, sh[w]);
    int E = 0;
    if (mx > 0.0) frexp(mx, &E);
    e[c] = mx > 0.0 ? E + 1 : 0;
  }
}

__device__ __forceinline__ double packed_r2(const double *x, long long ldx, int o, int v, int c, int m, int j, int e) {
  if (m == j) return 0.0;
  const long long lo = m < j ? m : j, hi = m < j ? j : m;
  const long long mu = o + pair_index(lo, hi, o) * v + e;
  const double val = x[2 * ((long long)(c >> 1) * ldx + mu) + (c & 1)];
  return m > j ? -val : val;
}

__device__ __forceinline__ void put_digits(double val, int ex, int S, __nv_bfloat16 *dst, long long plane) {
  long long Y = fixed_point(val, ex, 6 * S);
  for (int i = 0; i < S; i++) {
    const int sh = 6 * (S - 1 - i);
    const long long d = sh > 0 ? (Y + (1LL << (sh - 1))) >> sh : Y;
    Y -= d << sh;
    dst[i * plane] = __float2bfloat16((float)(int)d);
  }
}

// digit planes of r2b[(j,c)][(m,e)] = r2[m,j,e]; exp2[row] = e_c
__global__ void digits_ring_kernel(const double *x, long long ldx, int C2, int o, int v, const int *ec, int S,
                                   long long ld, __nv_bfloat16 *dig, int *rexp) {
  const long long K = (long long)o * v, rows = (long long)o * C2, plane = rows * ld;
  const long long tot = rows * ld;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const long long row = t / ld, k = t - row * ld;
    const int c = (int)(row % C2), j = (int)(row / C2);
    double val = 0.0;
    if (k < K) val = packed_r2(x, ldx, o, v, c, (int)(k / v), j, (int)(k % v));
    put_digits(val, ec[c], S, dig + t, plane);
    if (k == 0) rexp[row] = ec[c];
  }
}

// digit planes of r2o[(a,c)][(m,n)] = r2[m,n,a]: 32 x 32 tile transpose (reads along a, writes
// along (m,n)); grid (ld/32, v/32, C2), block (32, 8); exp2[row] = e_c
__global__ void digits_oooo_kernel(const double *x, long long ldx, int C2, int o, int v, const int *ec, int S,
                                   long long ld, __nv_bfloat16 *dig, int *rexp) {
  __shared__ double tile[32][33];
  const long long K = (long long)o * o, rows = (long long)v * C2, plane = rows * ld;
  const int c = blockIdx.z;
  const long long k0 = (long long)blockIdx.x * 32;
  const int a0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const long long k = k0 + r;
    const int a = a0 + threadIdx.x;
    tile[r][threadIdx.x] = (k < K && a < v) ? packed_r2(x, ldx, o, v, c, (int)(k / o), (int)(k % o), a) : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int a = a0 + r;
    const long long k = k0 + threadIdx.x;
    if (a < v && k < ld) {
      const long long row = (long long)a * C2 + c;
      put_digits(tile[threadIdx.x][r], ec[c], S, dig + row * ld + k, plane);
      if (k == 0) rexp[row] = ec[c];
    }
  }
}

// digit planes of rk[c][(m,e,n)] = r2[m,n,e] (tile transpose over (e, n) for fixed m, c);
// grid (o/32, v/32, o * C2), block (32, 8)
__global__ void digits_k2_kernel(const double *x, long long ldx, int C2, int o, int v, const int *ec, int S,
                                 long long ldk, __nv_bfloat16 *digk) {
  __shared__ double tile[32][33];
  const long long planek = (long long)C2 * ldk;
  const int c = blockIdx.z % C2, m = blockIdx.z / C2;
  const int n0 = blockIdx.x * 32, e0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int n = n0 + r, e = e0 + threadIdx.x;
    tile[r][threadIdx.x] = (n < o && e < v) ? packed_r2(x, ldx, o, v, c, m, n, e) : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int e = e0 + r, n = n0 + threadIdx.x;
    if (e < v && n < o)
      put_digits(tile[threadIdx.x][r], ec[c], S, digk + (long long)c * ldk + ((long long)m * v + e) * o + n, planek);
  }
}

// digit planes of the r1 part: rk[c][o2v + m] (and the zero padding of rk up to ldk) and, when ld1 > 0,
// r1b[c][m] (zero up to ld1); exponents of the operands written
__global__ void digits_k1_kernel(const double *x, long long ldx, int C2, int o, int v, const int *ec, int S,
                                 long long ldk, __nv_bfloat16 *digk, int *rexpk, long long ld1, __nv_bfloat16 *dig1,
                                 int *rexp1) {
  const long long o2v = (long long)o * o * v;
  const long long planek = (long long)C2 * ldk, plane1 = (long long)C2 * ld1;
  const long long tail = ldk - o2v;   // r1 values plus padding
  const long long tot = (long long)C2 * (tail > ld1 ? tail : ld1);
  const long long span = tail > ld1 ? tail : ld1;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t / span);
    const long long q = t % span;
    const double val = q < o ? x[2 * ((long long)(c >> 1) * ldx + q) + (c & 1)] : 0.0;
    if (q < tail) put_digits(val, ec[c], S, digk + (long long)c * ldk + o2v + q, planek);
    if (q < ld1) put_digits(val, ec[c], S, dig1 + (long long)c * ld1 + q, plane1);
    if (q == 0) {
      rexpk[c] = ec[c];
      if (rexp1 != nullptr) rexp1[c] = ec[c];
    }
  }
}

// Rz[c] = [plane c of x[s][0..k1) | Z[0..k2)[c]]: the B rows of the concatenated product
// [W1 | T3] (IP: x's 1h block, then Z over v) or [W3 | T3e] (EA: x's 1p block, then Z over o)
__global__ void rz_fill_kernel(const double *x, long long ldx, int C2, int k1, const double *Z, int k2, double *Rz) {
  const long long K = (long long)k1 + k2, tot = (long long)C2 * K;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t / K);
    const long long k = t - (long long)c * K;
    Rz[t] = k < k1 ? x[2 * ((long long)(c >> 1) * ldx + k) + (c & 1)] : Z[(k - k1) * C2 + c];
  }
}

// ---------------------------------------------------------------------------------------- EA
__device__ __forceinline__ double packed_y2(const double *x, long long ldx, int v, long long Pv, int c, int m, int a,
                                            int e) {
  if (a == e) return 0.0;
  const long long lo = a < e ? a : e, hi = a < e ? e : a;
  const long long mu = v + (long long)m * Pv + pair_index(lo, hi, v);
  const double val = x[2 * ((long long)(c >> 1) * ldx + mu) + (c & 1)];
  return a > e ? -val : val;
}

// digit planes of r2e[(a,c)][(m,e)] = y2[m,a,e]
__global__ void digits_ea_ring_kernel(const double *x, long long ldx, int C2, int o, int v, long long Pv,
                                      const int *ec, int S, long long ld, __nv_bfloat16 *dig, int *rexp) {
  const long long K = (long long)o * v, rows = (long long)v * C2, plane = rows * ld;
  const long long tot = rows * ld;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const long long row = t / ld, k = t - row * ld;
    const int c = (int)(row % C2), a = (int)(row / C2);
    const double val = k < K ? packed_y2(x, ldx, v, Pv, c, (int)(k / v), a, (int)(k % v)) : 0.0;
    put_digits(val, ec[c], S, dig + t, plane);
    if (k == 0) rexp[row] = ec[c];
  }
}

// digit planes of r2p[(i,c)][(e<f)] = y2[i,e,f]
__global__ void digits_ea_vvvv_kernel(const double *x, long long ldx, int C2, int o, int v, long long Pv,
                                      const int *ec, int S, long long ld, __nv_bfloat16 *dig, int *rexp) {
  const long long rows = (long long)o * C2, plane = rows * ld;
  const long long tot = rows * ld;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const long long row = t / ld, k = t - row * ld;
    const int c = (int)(row % C2), i = (int)(row / C2);
    const double val = k < Pv ? x[2 * ((long long)(c >> 1) * ldx + v + (long long)i * Pv + k) + (c & 1)] : 0.0;
    put_digits(val, ec[c], S, dig + t, plane);
    if (k == 0) rexp[row] = ec[c];
  }
}

// digit planes of rk[c][(m,x,y)] = y2[m,y,x], rk[c][o v v + e] = y1[e] (zero padding to ldk), and,
// when ld1 > 0, r1[c][e] = y1[e] (zero padding to ld1); exponents of the operands written
__global__ void digits_ea_k_kernel(const double *x, long long ldx, int C2, int o, int v, long long Pv, const int *ec,
                                   int S, long long ldk, __nv_bfloat16 *digk, int *rexpk, long long ld1,
                                   __nv_bfloat16 *dig1, int *rexp1) {
  const long long ov2 = (long long)o * v * v;
  const long long planek = (long long)C2 * ldk, plane1 = (long long)C2 * ld1;
  const long long span = ldk > ld1 ? ldk : ld1;
  const long long tot = (long long)C2 * span;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t / span);
    const long long k = t % span;
    if (k < ldk) {
      double val = 0.0;
      if (k < ov2) {
        const int y = (int)(k % v);
        const long long r = k / v;
        val = packed_y2(x, ldx, v, Pv, c, (int)(r / v), y, (int)(r % v));
      } else if (k < ov2 + v) {
        val = x[2 * ((long long)(c >> 1) * ldx + (k - ov2)) + (c & 1)];
      }
      put_digits(val, ec[c], S, digk + (long long)c * ldk + k, planek);
    }
    if (k < ld1) {
      const double val = k < v ? x[2 * ((long long)(c >> 1) * ldx + k) + (c & 1)] : 0.0;
      put_digits(val, ec[c], S, dig1 + (long long)c * ld1 + k, plane1);
    }
    if (k == 0) {
      rexpk[c] = ec[c];
      if (rexp1 != nullptr) rexp1[c] = ec[c];
    }
  }
}

struct EmuWorkEA {
  EmuOperand r2e, r2p, rk, Zo;
  int *ec;
  double *T, *Qp, *U, *S1, *Z, *Zt;
  void *gw;
  long long bytes;
};

EmuWorkEA emu_layout_ea(const gfcc_ctx *c, int nsub, void *base) {
  const long long o = c->o, v = c->v, C2 = 2LL * nsub, S = c->emu_S, Pv = c->Pv;
  const long long ov = o * v, ov2 = ov * v;
  EmuWorkEA w;
  unsigned char *p = static_cast<unsigned char *>(base);
  auto take = [&](long long bytes) {
    unsigned char *q = p;
    p += (bytes + 255) / 256 * 256;
    return q;
  };
  auto op = [&](EmuOperand &e, long long rows, long long K) {
    e.rows = rows;
    e.K = K;
    e.ld = (K + 7) / 8 * 8;
    e.S = (int)S;
    e.dig = reinterpret_cast<__nv_bfloat16 *>(take(S * rows * e.ld * 2));
    e.exp2 = reinterpret_cast<int *>(take(rows * 4));
  };
  op(w.r2e, v * C2, ov);
  op(w.r2p, o * C2, std::max<long long>(Pv, 1));
  op(w.rk, C2, ov2 + v);
  op(w.Zo, C2, v + o);
  w.ec = reinterpret_cast<int *>(take(C2 * 4));
  w.T = reinterpret_cast<double *>(take(ov * v * C2 * 8));
  w.Qp = reinterpret_cast<double *>(take(std::max<long long>(Pv, 1) * o * C2 * 8));
  w.U = reinterpret_cast<double *>(take(ov2 * C2 * 8));
  w.S1 = reinterpret_cast<double *>(take(v * C2 * 8));
  w.Z = reinterpret_cast<double *>(take(o * C2 * 8));
  w.Zt = reinterpret_cast<double *>(take((v + o) * C2 * 8));
  long long g = 0;
  g = std::max(g, emu_gemm_work_bytes(ov, v * C2, ov));
  g = std::max(g, emu_gemm_work_bytes(std::max<long long>(Pv, 1), o * C2, std::max<long long>(Pv, 1)));
  g = std::max(g, emu_gemm_work_bytes(ov2, C2, v + o));
  g = std::max(g, emu_gemm_work_bytes(o, C2, ov2 + v));
  g = std::max(g, emu_gemm_work_bytes(v, C2, ov2 + v));
  w.gw = take(g);
  w.bytes = p - static_cast<unsigned char *>(base);
  return w;
}

struct EmuWork {
  EmuOperand r2b, r2o, rk, Zo;
  int *ec;
  double *T, *Q, *U, *S1, *Z, *Zt;
  void *gw;     // emu_gemm workspace
  long long bytes;
};

EmuWork emu_layout(const gfcc_ctx *c, int nsub, void *base) {
  const long long o = c->o, v = c->v, C2 = 2LL * nsub, S = c->emu_S;
  const long long o2v = o * o * v;
  EmuWork w;
  unsigned char *p = static_cast<unsigned char *>(base);
  auto take = [&](long long bytes) {
    unsigned char *q = p;
    p += (bytes + 255) / 256 * 256;
    return q;
  };
  auto op = [&](EmuOperand &e, long long rows, long long K) {
    e.rows = rows;
    e.K = K;
    e.ld = (K + 7) / 8 * 8;
    e.S = (int)S;
    e.dig = reinterpret_cast<__nv_bfloat16 *>(take(S * rows * e.ld * 2));
    e.exp2 = reinterpret_cast<int *>(take(rows * 4));
  };
  op(w.r2b, o * C2, o * v);
  op(w.r2o, v * C2, o * o);
  op(w.rk, C2, o2v + o);
  op(w.Zo, C2, o + v);
  w.ec = reinterpret_cast<int *>(take(C2 * 4));
  w.T = reinterpret_cast<double *>(take(o * v * o * C2 * 8));
  w.Q = reinterpret_cast<double *>(take(o * o * v * C2 * 8));
  w.U = reinterpret_cast<double *>(take(o * v * o * C2 * 8));
  w.S1 = reinterpret_cast<double *>(take(o * C2 * 8));
  w.Z = reinterpret_cast<double *>(take(v * C2 * 8));
  w.Zt = reinterpret_cast<double *>(take((o + v) * C2 * 8));
  long long g = 0;
  g = std::max(g, emu_gemm_work_bytes(o * v, o * C2, o * v));
  g = std::max(g, emu_gemm_work_bytes(o * o, v * C2, o * o));
  g = std::max(g, emu_gemm_work_bytes(o2v, C2, o + v));
  g = std::max(g, emu_gemm_work_bytes(v, C2, o2v + o));
  g = std::max(g, emu_gemm_work_bytes(o, C2, o2v + o));
  w.gw = take(g);
  w.bytes = p - static_cast<unsigned char *>(base);
  return w;
}

}  // namespace

long long sigma_emu_work_doubles(const gfcc_ctx *c, int nsub) {
  long long b = 0;
  if (c->eWr.dig != nullptr) b = std::max(b, emu_layout(c, nsub, nullptr).bytes);
  if (c->eWre.dig != nullptr) b = std::max(b, emu_layout_ea(c, nsub, nullptr).bytes);
  return b / 8 + 64;
}

int apply_ip_emu(gfcc_ctx *c, const SysBatch &b, double *work, long long work_doubles, int level) {
  if (c->eWr.dig == nullptr) {
    set_error("FP64-emulated residual requested but its digit planes were not built");
    return GFCC_ERR_STATE;
  }
  cudaStream_t st = c->stream;
  const long long o = c->o, v = c->v, oo = o * o, o2v = oo * v, n = c->dim_ip;
  // largest sub-batch whose workspace fits
  int nsub = b.nsys;
  while (nsub > 1 && sigma_emu_work_doubles(c, nsub) > work_doubles) nsub = (nsub + 1) / 2;
  if (sigma_emu_work_doubles(c, nsub) > work_doubles) {
    set_error("apply_ip_emu: workspace too small for one system");
    return GFCC_ERR_OOM;
  }
  const int S = c->emu_S, P = level > 0 ? std::min(level, c->emu_P) : c->emu_P;
  PhaseTimer tsig(c, PH_SIGMA, b.nsys * sigma_flops(c, GFCC_SECTOR_IP));
  for (int s0 = 0; s0 < b.nsys; s0 += nsub) {
    const int ns = std::min(nsub, b.nsys - s0);
    const int C2 = 2 * ns;
    EmuWork w = emu_layout(c, ns, work);
    const double *x = b.x + 2 * (long long)s0 * b.ldx;
    {
    PhaseTimer tu(c, PH_UNPACK);
    plane_exp_kernel<<<C2, 256, 0, st>>>(x, b.ldx, n, w.ec);
    GFCC_LAUNCH_CHECK();
    digits_ring_kernel<<<grid1d(w.r2b.rows * w.r2b.ld), 256, 0, st>>>(x, b.ldx, C2, (int)o, (int)v, w.ec, S, w.r2b.ld,
                                                                       w.r2b.dig, w.r2b.exp2);
    GFCC_LAUNCH_CHECK();
    digits_oooo_kernel<<<dim3(cdiv(w.r2o.ld, 32), cdiv(v, 32), C2), dim3(32, 8), 0, st>>>(
        x, b.ldx, C2, (int)o, (int)v, w.ec, S, w.r2o.ld, w.r2o.dig, w.r2o.exp2);
    GFCC_LAUNCH_CHECK();
    digits_k2_kernel<<<dim3(cdiv(o, 32), cdiv(v, 32), o * C2), dim3(32, 8), 0, st>>>(x, b.ldx, C2, (int)o, (int)v,
                                                                                    w.ec, S, w.rk.ld, w.rk.dig);
    GFCC_LAUNCH_CHECK();
    // (the 1h block also enters [r1 | Z] of the concatenated ovoo / three-body product, sliced there)
    digits_k1_kernel<<<grid1d((long long)C2 * (w.rk.ld - o2v)), 256, 0, st>>>(
        x, b.ldx, C2, (int)o, (int)v, w.ec, S, w.rk.ld, w.rk.dig, w.rk.exp2, 0, nullptr, nullptr);
    GFCC_LAUNCH_CHECK();
    }
    {
      // tensor-core work: one BF16 GEMM per digit pair (i, j), i + j <= P
      int pairs = 0;
      const int Pr = std::max(2, P - c->eWr.drop);
      for (int L = 2; L <= Pr; L++)
        for (int i = 1; i <= S; i++)
          if (L - i >= 1 && L - i <= S) pairs++;
      const double prod = 2.0 * (double)(o * v) * (double)(o * v) * (double)(o * C2);
      PhaseTimer tr(c, PH_RING_EMU, prod);
      PhaseTimer tw(c, PH_RING_EMU_WORK, pairs * prod);
      GFCC_TRY(emu_gemm(st, c->eWr, w.r2b, P, 1.0, 0.0, w.T, imap1(o * C2), imap1(1), w.gw));
    }
    {
      // oooo, three-body Z, [ovoo | three-body] U and the 1h row, one FP64 product each
      PhaseTimer te(c, PH_EMU_OTHER, 2.0 * C2 * ((double)oo * oo * v + (double)v * o2v + (double)o2v * (o + v) +
                                                 (double)o * (o2v + o)));
      GFCC_TRY(emu_gemm(st, c->eWq, w.r2o, P, 1.0, 0.0, w.Q, imap1(v * C2), imap1(1), w.gw));
      // three-body Z = V3 rk, then U = [W1 | T3] [r1 | Z] in one product over K = o + v
      GFCC_TRY(emu_gemm(st, c->eV3, w.rk, P, 1.0, 0.0, w.Z, imap1(C2), imap1(1), w.gw));
      rz_fill_kernel<<<grid1d(C2 * (o + v)), 256, 0, st>>>(x, b.ldx, C2, (int)o, w.Z, (int)v, w.Zt);
      GFCC_LAUNCH_CHECK();
      GFCC_TRY(emu_slice(st, w.Zt, C2, o + v, o + v, S, w.Zo.dig, w.Zo));
      GFCC_TRY(emu_gemm(st, c->eWT, w.Zo, P, 1.0, 0.0, w.U, imap1(C2), imap1(1), w.gw));
      GFCC_TRY(emu_gemm(st, c->eU1, w.rk, P, 1.0, 0.0, w.S1, imap1(C2), imap1(1), w.gw));
    }
    SysBatch bb = b;
    bb.nsys = ns;
    bb.x = x;
    bb.y = b.y + 2 * (long long)s0 * b.ldy;
    bb.omega = b.omega ? b.omega + s0 : nullptr;
    bb.diag = nullptr;
    {
      PhaseTimer tp(c, PH_EPILOGUE, 8.0 * C2 * (3.0 * o2v + o) + 32.0 * ns * n);
      GFCC_TRY(launch_epilogue_ip(c, bb, w.S1, w.T, w.Q, w.U, c->diag_ip));
    }
  }
  return GFCC_OK;
}


int apply_ea_emu(gfcc_ctx *c, const SysBatch &b, double *work, long long work_doubles, int level) {
  if (c->eWre.dig == nullptr) {
    set_error("FP64-emulated EA residual requested but its digit planes were not built");
    return GFCC_ERR_STATE;
  }
  cudaStream_t st = c->stream;
  const long long o = c->o, v = c->v, ov = o * v, ov2 = ov * v, Pv = c->Pv, n = c->dim_ea;
  int nsub = b.nsys;
  while (nsub > 1 && emu_layout_ea(c, nsub, nullptr).bytes / 8 + 64 > work_doubles) nsub = (nsub + 1) / 2;
  if (emu_layout_ea(c, nsub, nullptr).bytes / 8 + 64 > work_doubles) {
    set_error("apply_ea_emu: workspace too small for one system");
    return GFCC_ERR_OOM;
  }
  const int S = c->emu_S, P = level > 0 ? std::min(level, c->emu_P) : c->emu_P;
  PhaseTimer tsig(c, PH_SIGMA, b.nsys * sigma_flops(c, GFCC_SECTOR_EA));
  for (int s0 = 0; s0 < b.nsys; s0 += nsub) {
    const int ns = std::min(nsub, b.nsys - s0);
    const int C2 = 2 * ns;
    EmuWorkEA w = emu_layout_ea(c, ns, work);
    const double *x = b.x + 2 * (long long)s0 * b.ldx;
    {
      PhaseTimer tu(c, PH_UNPACK);
      plane_exp_kernel<<<C2, 256, 0, st>>>(x, b.ldx, n, w.ec);
      GFCC_LAUNCH_CHECK();
      digits_ea_ring_kernel<<<grid1d(w.r2e.rows * w.r2e.ld), 256, 0, st>>>(x, b.ldx, C2, (int)o, (int)v, Pv, w.ec, S,
                                                                            w.r2e.ld, w.r2e.dig, w.r2e.exp2);
      GFCC_LAUNCH_CHECK();
      digits_ea_vvvv_kernel<<<grid1d(w.r2p.rows * w.r2p.ld), 256, 0, st>>>(x, b.ldx, C2, (int)o, (int)v, Pv, w.ec, S,
                                                                            w.r2p.ld, w.r2p.dig, w.r2p.exp2);
      GFCC_LAUNCH_CHECK();
      // (the 1p block also enters [y1 | Z] of the concatenated product, sliced there)
      digits_ea_k_kernel<<<grid1d((long long)C2 * w.rk.ld), 256, 0, st>>>(
          x, b.ldx, C2, (int)o, (int)v, Pv, w.ec, S, w.rk.ld, w.rk.dig, w.rk.exp2, 0, nullptr, nullptr);
      GFCC_LAUNCH_CHECK();
    }
    {
      int pairs = 0;
      const int Pr = std::max(2, P - c->eWre.drop);
      for (int L = 2; L <= Pr; L++)
        for (int i = 1; i <= S; i++)
          if (L - i >= 1 && L - i <= S) pairs++;
      const double prod = 2.0 * (double)ov * (double)ov * (double)(v * C2);
      PhaseTimer tr(c, PH_RING_EMU, prod);
      PhaseTimer tw(c, PH_RING_EMU_WORK, pairs * prod);
      GFCC_TRY(emu_gemm(st, c->eWre, w.r2e, P, 1.0, 0.0, w.T, imap1(v * C2), imap1(1), w.gw));
    }
    {
      // vvvv, three-body Z, [vvvo | three-body] U and the 1p row, one FP64 product each
      PhaseTimer te(c, PH_EMU_OTHER, 2.0 * C2 * ((double)Pv * Pv * o + (double)o * ov2 + (double)ov2 * (v + o) +
                                                 (double)v * (ov2 + v)));
      if (Pv > 0) GFCC_TRY(emu_gemm(st, c->eWp, w.r2p, P, 1.0, 0.0, w.Qp, imap1(o * C2), imap1(1), w.gw));
      // Z = V3e rk, then U = [W3 | T3e] [y1 | Z] in one product over K = v + o
      GFCC_TRY(emu_gemm(st, c->eV3e, w.rk, P, 1.0, 0.0, w.Z, imap1(C2), imap1(1), w.gw));
      rz_fill_kernel<<<grid1d(C2 * (v + o)), 256, 0, st>>>(x, b.ldx, C2, (int)v, w.Z, (int)o, w.Zt);
      GFCC_LAUNCH_CHECK();
      GFCC_TRY(emu_slice(st, w.Zt, C2, v + o, v + o, S, w.Zo.dig, w.Zo));
      GFCC_TRY(emu_gemm(st, c->eWTe, w.Zo, P, 1.0, 0.0, w.U, imap1(C2), imap1(1), w.gw));
      GFCC_TRY(emu_gemm(st, c->eU1e, w.rk, P, 1.0, 0.0, w.S1, imap1(C2), imap1(1), w.gw));
    }
    SysBatch bb = b;
    bb.nsys = ns;
    bb.x = x;
    bb.y = b.y + 2 * (long long)s0 * b.ldy;
    bb.omega = b.omega ? b.omega + s0 : nullptr;
    bb.diag = nullptr;
    {
      PhaseTimer tp(c, PH_EPILOGUE, 8.0 * C2 * (2.0 * ov2 + (double)Pv * o + v) + 32.0 * ns * n);
      GFCC_TRY(launch_epilogue_ea(c, bb, w.S1, w.T, w.Qp, w.U, c->diag_ea));
    }
  }
  return GFCC_OK;
}

}  // namespace gfcc
