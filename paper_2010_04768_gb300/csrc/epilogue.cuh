// Tiled epilogues of the batched sigma product: antisymmetrise the contraction outputs, add the
// shift of eq. xplin and pack into y[s][mu].
//
// The contraction outputs are column-major in the systems (the planar column c = 2 s + re/im is
// the fastest index: T[(i,a)][(j,c)], Q[(i,j)][(a,c)], U[(i,a,j)][c] for IP; T[(i,b)][(a,c)],
// Qp[(a<b)][(i,c)], U[(i,b,a)][c] for EA), while y is row-major in the systems.  A block therefore
// handles a run of consecutive packed elements of one (i<j) pair (IP) or one i (EA): it reads the
// contraction outputs along c (coalesced), stages sigma in shared memory, and writes y along mu
// (coalesced).
//
// MODE_FULL: the outputs contain the whole operator (FP64 and FP64-accurate products):
//   IP y = z u + sigma(u), EA y = z u - sigma(u), u = x / D_s (right preconditioner) or x;
//   without omega y = sigma(x).
// MODE_OFFDIAG: the outputs contain the couplings only (BF16 products); the Fock-like diagonal d
//   is applied here in FP64: IP y = x + sigma_off(u) (preconditioned), (z + d) x + sigma_off(x);
//   EA y = x - sigma_off(u), (z - d) x - sigma_off(x); without omega y = d x + sigma_off(x).
#pragma once
#include "sigma.cuh"

namespace gfcc {
namespace epi {

constexpr int MODE_FULL = 0, MODE_OFFDIAG = 1;
constexpr int THREADS = 256;

template <typename TIn>
constexpr int run_len() {
  return sizeof(TIn) == 4 ? 16 : 8;   // packed elements per block
}
// systems per launch: the shared tile run_len x (2 ns + 1) stays below 33 KB
template <typename TIn>
constexpr int max_systems() {
  return 256;
}

__device__ __forceinline__ void load_x(const SysBatch &b, int s, long long mu, double &xr, double &xi) {
  s = sysv(b, s);
  if (b.xf != nullptr) {
    const float2 t = reinterpret_cast<const float2 *>(b.xf)[s * b.ldx + mu];
    xr = t.x;
    xi = t.y;
  } else {
    const double2 t = reinterpret_cast<const double2 *>(b.x)[s * b.ldx + mu];
    xr = t.x;
    xi = t.y;
  }
}

__device__ __forceinline__ void store_y(const SysBatch &b, int s, long long mu, double yr, double yi) {
  if (!sys_stores(b, s)) return;
  s = sysv(b, s);
  if (b.yf != nullptr)
    reinterpret_cast<float2 *>(b.yf)[s * b.ldy + mu] = make_float2((float)yr, (float)yi);
  else
    reinterpret_cast<double2 *>(b.y)[s * b.ldy + mu] = make_double2(yr, yi);
}

// sgn = +1 IP, -1 EA; diag = the operator's Fock-like diagonal (MODE_OFFDIAG)
template <int MODE>
__device__ __forceinline__ void combine(const SysBatch &b, int s, long long mu, double sr, double si,
                                        const double *diag, double sgn) {
  double xr, xi;
  load_x(b, s, mu, xr, xi);
  double yr, yi;
  if (MODE == MODE_FULL) {
    if (b.omega == nullptr) {
      yr = sr;
      yi = si;
    } else {
      double ur = xr, ui = xi;
      if (b.diag != nullptr) {
        const double dr = b.omega[sysv(b, s)] + b.dsign * b.diag[mu], di = b.zsign * b.eta;
        const double d2 = dr * dr + di * di;
        ur = (xr * dr + xi * di) / d2;
        ui = (xi * dr - xr * di) / d2;
      }
      const double zr = b.omega[sysv(b, s)], zi = b.zsign * b.eta;
      yr = zr * ur - zi * ui + sgn * sr;
      yi = zr * ui + zi * ur + sgn * si;
    }
  } else {
    const double d = diag[mu];
    if (b.omega == nullptr) {
      yr = d * xr + sr;
      yi = d * xi + si;
    } else if (b.diag != nullptr) {
      yr = xr + sgn * sr;
      yi = xi + sgn * si;
    } else {
      const double dr = b.omega[sysv(b, s)] + sgn * d, di = b.zsign * b.eta;
      yr = dr * xr - di * xi + sgn * sr;
      yi = dr * xi + di * xr + sgn * si;
    }
  }
  store_y(b, s, mu, yr, yi);
}

// IP 2h1p block: one block per (pair p = (i<j), run of a); grid (Po, cdiv(v, run)), dynamic shared
// memory run * (C2 + 1) * sizeof(TIn)
template <typename TIn, int MODE>
__global__ __launch_bounds__(THREADS) void ip2_kernel(SysBatch b, int o, int v, long long C2, int s0, int ns,
                                                       const TIn *T, const TIn *Q, const TIn *U, const double *diag) {
  extern __shared__ __align__(16) unsigned char smem[];
  TIn *tile = reinterpret_cast<TIn *>(smem);
  constexpr int A = run_len<TIn>();
  const long long p = blockIdx.x;
  const int a0 = blockIdx.y * A;
  long long i, j;
  pair_decode(p, o, i, j);
  const long long Cl = 2LL * ns, ld = Cl + 1, c0 = 2LL * s0;
  const int cl = (int)Cl;   // at most 2 max_systems()
  for (int t = threadIdx.x; t < A * cl; t += THREADS) {
    const int al = t / cl;
    const long long c = t - al * cl;
    const long long a = a0 + al;
    if (a >= v) continue;
    const long long tij = ((i * v + a) * o + j) * C2 + c0 + c;
    const long long tji = ((j * v + a) * o + i) * C2 + c0 + c;
    const long long qij = ((i * o + j) * v + a) * C2 + c0 + c;
    tile[al * ld + c] = T[tij] - T[tji] + Q[qij] + U[tij];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < A * ns; t += THREADS) {
    const int s = t / A, al = t - s * A;
    const long long a = a0 + al;
    if (a >= v) continue;
    const long long mu = o + p * v + a;
    combine<MODE>(b, s0 + s, mu, (double)tile[al * ld + 2 * s], (double)tile[al * ld + 2 * s + 1], diag, 1.0);
  }
}

// EA 2p1h block: one block per (i, run of pairs a<b); grid (o, cdiv(Pv, run))
template <typename TIn, int MODE>
__global__ __launch_bounds__(THREADS) void ea2_kernel(SysBatch b, int o, int v, long long Pv, long long C2, int s0,
                                                       int ns, const TIn *T, const TIn *Qp, const TIn *U,
                                                       const double *diag) {
  extern __shared__ __align__(16) unsigned char smem[];
  TIn *tile = reinterpret_cast<TIn *>(smem);
  constexpr int A = run_len<TIn>();
  __shared__ int pa[A], pb[A];   // the block's pairs (a < b), decoded once
  const long long i = blockIdx.x;
  const long long ab0 = (long long)blockIdx.y * A;
  const long long Cl = 2LL * ns, ld = Cl + 1, c0 = 2LL * s0;
  if (threadIdx.x < A && ab0 + threadIdx.x < Pv) {
    long long a, bb;
    pair_decode(ab0 + threadIdx.x, v, a, bb);
    pa[threadIdx.x] = (int)a;
    pb[threadIdx.x] = (int)bb;
  }
  __syncthreads();
  const int cl = (int)Cl;   // at most 2 max_systems()
  for (int t = threadIdx.x; t < A * cl; t += THREADS) {
    const int al = t / cl;
    const long long c = t - al * cl;
    const long long ab = ab0 + al;
    if (ab >= Pv) continue;
    const long long a = pa[al], bb = pb[al];
    const long long tiba = ((i * v + bb) * v + a) * C2 + c0 + c;
    const long long tiab = ((i * v + a) * v + bb) * C2 + c0 + c;
    const long long qq = (ab * o + i) * C2 + c0 + c;
    tile[al * ld + c] = T[tiba] - T[tiab] + Qp[qq] + U[tiba];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < A * ns; t += THREADS) {
    const int s = t / A, al = t - s * A;
    const long long ab = ab0 + al;
    if (ab >= Pv) continue;
    const long long mu = v + i * Pv + ab;
    combine<MODE>(b, s0 + s, mu, (double)tile[al * ld + 2 * s], (double)tile[al * ld + 2 * s + 1], diag, -1.0);
  }
}

// the one-index block (IP 1h: n1 = o, sgn +1; EA 1p: n1 = v, sgn -1): S1[m][c]
template <typename TIn, int MODE>
__global__ void one_kernel(SysBatch b, int n1, long long C2, const TIn *S1, const double *diag, double sgn) {
  const long long tot = (long long)n1 * b.nsys;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(t / n1);
    const long long m = t - (long long)s * n1;
    combine<MODE>(b, s, m, (double)S1[m * C2 + 2 * s], (double)S1[m * C2 + 2 * s + 1], diag, sgn);
  }
}

template <typename TIn, int MODE>
int launch_ip(cudaStream_t st, const SysBatch &b, int o, int v, const TIn *S1, const TIn *T, const TIn *Q,
              const TIn *U, const double *diag) {
  const long long C2 = 2LL * b.nsys, Po = (long long)o * (o - 1) / 2;
  constexpr int A = run_len<TIn>();
  one_kernel<TIn, MODE><<<grid1d((long long)o * b.nsys), THREADS, 0, st>>>(b, o, C2, S1, diag, 1.0);
  GFCC_LAUNCH_CHECK();
  for (int s0 = 0; Po > 0 && v > 0 && s0 < b.nsys; s0 += max_systems<TIn>()) {
    const int ns = b.nsys - s0 < max_systems<TIn>() ? b.nsys - s0 : max_systems<TIn>();
    const size_t sm = (size_t)A * (2 * ns + 1) * sizeof(TIn);
    ip2_kernel<TIn, MODE><<<dim3((unsigned)Po, cdiv(v, A)), THREADS, sm, st>>>(b, o, v, C2, s0, ns, T, Q, U, diag);
    GFCC_LAUNCH_CHECK();
  }
  return GFCC_OK;
}

template <typename TIn, int MODE>
int launch_ea(cudaStream_t st, const SysBatch &b, int o, int v, long long Pv, const TIn *S1, const TIn *T,
              const TIn *Qp, const TIn *U, const double *diag) {
  const long long C2 = 2LL * b.nsys;
  constexpr int A = run_len<TIn>();
  one_kernel<TIn, MODE><<<grid1d((long long)v * b.nsys), THREADS, 0, st>>>(b, v, C2, S1, diag, -1.0);
  GFCC_LAUNCH_CHECK();
  for (int s0 = 0; Pv > 0 && o > 0 && s0 < b.nsys; s0 += max_systems<TIn>()) {
    const int ns = b.nsys - s0 < max_systems<TIn>() ? b.nsys - s0 : max_systems<TIn>();
    const size_t sm = (size_t)A * (2 * ns + 1) * sizeof(TIn);
    ea2_kernel<TIn, MODE><<<dim3((unsigned)o, cdiv(Pv, A)), THREADS, sm, st>>>(b, o, v, Pv, C2, s0, ns, T, Qp, U,
                                                                                diag);
    GFCC_LAUNCH_CHECK();
  }
  return GFCC_OK;
}

}  // namespace epi
}  // namespace gfcc
