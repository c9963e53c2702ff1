// Batched restarted GMRES (Saad & Schultz 1986) for the GFCCSD linear systems, FP64.
//
// GFCC Workflow and Bottlenecks section: the systems (omega - i eta + Hbar_N) X = b
// are solved by GMRES, whose residual norm decreases monotonically; its cost grows
// as O(n^2 O^2 V) in the iteration count n, which is the Arnoldi work here.
//
// All systems of a batch advance in lock step through the Arnoldi steps of a
// restart cycle.  Orthogonalisation is classical Gram-Schmidt applied twice
// (CGS2): both passes are batched dot products / vector updates that stream the
// Krylov basis once each, which suits HBM better than the sequential modified
// Gram-Schmidt of the oracle and is as stable.  The (m+1) x m Hessenberg matrix
// of each system is reduced by complex Givens rotations on the device, one thread
// per system; a system leaves its cycle when the rotated residual estimate
// reaches tol ||b|| (or on breakdown), and every cycle ends with the true
// residual b - A x recomputed by the operator.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ctx.cuh"
#include "gmres.cuh"
#include "kernels.cuh"
#include "sigma.cuh"

namespace gfcc {

namespace {

constexpr int ST_PENDING = 0, ST_IN_CYCLE = 1, ST_CYCLE_DONE = 2, ST_CONVERGED = 3, ST_FAILED = 4;
constexpr int DOT_THREADS = 256, DOT_PER_THREAD = 8, DOT_CHUNK = DOT_THREADS * DOT_PER_THREAD;

__device__ __forceinline__ double2 ld2(const double *p, long long i) { return reinterpret_cast<const double2 *>(p)[i]; }
__device__ __forceinline__ void st2(double *p, long long i, double2 v) { reinterpret_cast<double2 *>(p)[i] = v; }

// Krylov vectors are complex interleaved arrays of T = double (FP64 solves) or T = float (the inner
// solves of mixed-precision refinement).  Arithmetic on vector elements runs in T; sums across
// elements are reduced in double.
template <typename T>
struct Cplx;
template <>
struct Cplx<double> {
  using type = double2;
};
template <>
struct Cplx<float> {
  using type = float2;
};
template <typename T>
using CT = typename Cplx<T>::type;
template <typename T>
__device__ __forceinline__ CT<T> ldc(const T *p, long long i) {
  return reinterpret_cast<const CT<T> *>(p)[i];
}
template <typename T>
__device__ __forceinline__ void stc(T *p, long long i, CT<T> v) {
  reinterpret_cast<CT<T> *>(p)[i] = v;
}
template <typename T>
__device__ __forceinline__ CT<T> mkc(double x, double y) {
  CT<T> r;
  r.x = (T)x;
  r.y = (T)y;
  return r;
}

// Block-wide sum of a complex value; result valid in thread 0.
__device__ __forceinline__ double2 block_sum(double2 v, double2 *sh) {
  for (int off = 16; off > 0; off >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, off);
    v.y += __shfl_down_sync(0xffffffffu, v.y, off);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < (int)(blockDim.x >> 5) ? sh[lane] : make_double2(0.0, 0.0);
    for (int off = 16; off > 0; off >>= 1) {
      v.x += __shfl_down_sync(0xffffffffu, v.x, off);
      v.y += __shfl_down_sync(0xffffffffu, v.y, off);
    }
  }
  return v;
}

// partial[(s*NV + i)*nch + chunk] = sum_{mu in chunk} conj(Vs_i[mu]) w_s[mu]   (systems with state == want)
template <typename T>
__global__ __launch_bounds__(DOT_THREADS) void mdot_partial_kernel(const T *V, long long vs_stride,
                                                                   long long vi_stride, int nv, const T *w,
                                                                   long long ws_stride, long long n, int nch,
                                                                   const int *state, int want, double *partial,
                                                                   int NV) {
  __shared__ double2 sh[32];
  const int s = blockIdx.y, chunk = blockIdx.x;
  if (state != nullptr && state[s] != want) return;
  const long long base = (long long)chunk * DOT_CHUNK;
  CT<T> wv[DOT_PER_THREAD];
  const T *ws = w + 2 * s * ws_stride;
#pragma unroll
  for (int r = 0; r < DOT_PER_THREAD; r++) {
    const long long mu = base + threadIdx.x + (long long)r * DOT_THREADS;
    wv[r] = mu < n ? ldc(ws, mu) : mkc<T>(0.0, 0.0);
  }
  for (int i = 0; i < nv; i++) {
    const T *vi = V + 2 * (s * vs_stride + i * vi_stride);
    CT<T> a2 = mkc<T>(0.0, 0.0);
#pragma unroll
    for (int r = 0; r < DOT_PER_THREAD; r++) {
      const long long mu = base + threadIdx.x + (long long)r * DOT_THREADS;
      if (mu < n) {
        const CT<T> a = ldc(vi, mu);
        a2.x += a.x * wv[r].x + a.y * wv[r].y;
        a2.y += a.x * wv[r].y - a.y * wv[r].x;
      }
    }
    double2 acc = make_double2((double)a2.x, (double)a2.y);
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) reinterpret_cast<double2 *>(partial)[((long long)s * NV + i) * nch + chunk] = acc;
  }
}

// out[s*NV + i] (+)= sum_chunk partial  (one warp per (s, i))
__global__ void mdot_final_kernel(const double *partial, int nsys, int nv, int NV, int nch, const int *state,
                                  int want, double *out, int accumulate) {
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (gw >= nsys * nv) return;
  const int s = gw / nv, i = gw % nv;
  if (state != nullptr && state[s] != want) return;
  double2 acc = make_double2(0.0, 0.0);
  const double2 *p = reinterpret_cast<const double2 *>(partial) + ((long long)s * NV + i) * nch;
  for (int c = lane; c < nch; c += 32) {
    acc.x += p[c].x;
    acc.y += p[c].y;
  }
  for (int off = 16; off > 0; off >>= 1) {
    acc.x += __shfl_down_sync(0xffffffffu, acc.x, off);
    acc.y += __shfl_down_sync(0xffffffffu, acc.y, off);
  }
  if (lane == 0) {
    double2 *o = reinterpret_cast<double2 *>(out) + (long long)s * NV + i;
    if (accumulate) {
      o->x += acc.x;
      o->y += acc.y;
    } else {
      *o = acc;
    }
  }
}

// w_s[mu] += sign * sum_{i<nv_s} coef[s*NV + i] Vs_i[mu]   (systems with state == want;
// nv_s = nvs[s] when nvs != nullptr, else nv)
template <typename T>
__global__ void vupdate_kernel(const T *V, long long vs_stride, long long vi_stride, int nv, const int *nvs,
                               const double *coef, int NV, double sign, T *w, long long ws_stride, long long n,
                               int nsys, const int *state, int want) {
  const long long tot = n * nsys;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(t / n);
    const long long mu = t - (long long)s * n;
    if (state != nullptr && state[s] != want) continue;
    CT<T> acc = mkc<T>(0.0, 0.0);
    const double2 *cf = reinterpret_cast<const double2 *>(coef) + (long long)s * NV;
    const int nvv = nvs != nullptr ? nvs[s] : nv;
    for (int i = 0; i < nvv; i++) {
      const CT<T> a = ldc(V + 2 * (s * vs_stride + i * vi_stride), mu);
      const T cx = (T)cf[i].x, cy = (T)cf[i].y;
      acc.x += cx * a.x - cy * a.y;
      acc.y += cx * a.y + cy * a.x;
    }
    CT<T> x = ldc(w + 2 * s * ws_stride, mu);
    x.x += (T)sign * acc.x;
    x.y += (T)sign * acc.y;
    stc(w + 2 * s * ws_stride, mu, x);
  }
}

// w_s *= 1 / scale[s] (real scale stored as the real part of a complex entry scale[s*NV + idx]).
// Grid (cdiv(2n, VSCALE_PER_BLOCK), nsys): the factor is formed once per thread; each thread scales
// VSCALE_UNROLL reals with independent loads.
constexpr int VSCALE_UNROLL = 4, VSCALE_PER_BLOCK = 256 * VSCALE_UNROLL;
template <typename T>
__global__ void vscale_kernel(T *w, long long ws_stride, long long n, const double *nrm2, int NV, int idx,
                              const int *state, int want) {
  const int s = blockIdx.y;
  if (state != nullptr && state[s] != want) return;
  const double nn = nrm2[2 * ((long long)s * NV + idx)];
  if (!(nn > 0.0)) return;
  const T inv = (T)(1.0 / sqrt(nn));
  T *ws = w + 2 * s * ws_stride;
  const long long n2 = 2 * n, t0 = (long long)blockIdx.x * VSCALE_PER_BLOCK + threadIdx.x;
  T x[VSCALE_UNROLL];
#pragma unroll
  for (int u = 0; u < VSCALE_UNROLL; u++) {
    const long long t = t0 + (long long)u * blockDim.x;
    x[u] = t < n2 ? ws[t] : (T)0;
  }
#pragma unroll
  for (int u = 0; u < VSCALE_UNROLL; u++) {
    const long long t = t0 + (long long)u * blockDim.x;
    if (t < n2) ws[t] = x[u] * inv;
  }
}
static inline dim3 vscale_grid(long long n, int nsys) {
  return dim3((unsigned)std::max<long long>(1, (2 * n + VSCALE_PER_BLOCK - 1) / VSCALE_PER_BLOCK), (unsigned)nsys);
}

// r_s = b_s - w_s for systems that are not finished
template <typename T>
__global__ void resid_form_kernel(const T *B, const T *W, T *R, long long r_stride, long long n, int nsys,
                                  const int *state) {
  const long long tot = n * nsys;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(t / n);
    const long long mu = t - (long long)s * n;
    if (state[s] != ST_PENDING) continue;
    const CT<T> b = ldc(B, t), w = ldc(W, t);
    stc(R + 2 * s * r_stride, mu, mkc<T>(b.x - w.x, b.y - w.y));
  }
}

// Decide per system after the true residual: converged, failed (budget) or start a new cycle.
__global__ void cycle_start_kernel(int nsys, const double *nrm2, int NV, const double *bnorm, double tol, int max_iters,
                                   int m1, int *state, int *iters, double *relres, double *g, double *H) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsys || state[s] != ST_PENDING) return;
  const double beta = sqrt(fmax(nrm2[2 * ((long long)s * NV)], 0.0));
  const double bn = bnorm[s];
  relres[s] = bn > 0.0 ? beta / bn : 0.0;
  if (bn == 0.0 || beta <= tol * bn) {
    state[s] = ST_CONVERGED;
    return;
  }
  if (iters[s] >= max_iters) {
    state[s] = ST_FAILED;
    return;
  }
  double2 *gs = reinterpret_cast<double2 *>(g) + (long long)s * m1;
  for (int i = 0; i < m1; i++) gs[i] = make_double2(0.0, 0.0);
  gs[0] = make_double2(beta, 0.0);
  (void)H;
  state[s] = ST_IN_CYCLE;
}

// Givens update of column k for systems in cycle.
//   h[s*NV + i], i <= k: Gram-Schmidt coefficients (pass 1 + pass 2); h[s*NV + k+1]: ||w||^2 (real part)
__global__ void givens_kernel(int nsys, int k, int m, const double *h, int NV, double *H, double *cs, double *sn,
                              double *g, const double *bnorm, double tol, int *state, int *kcyc, int *iters,
                              double *est) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsys || state[s] != ST_IN_CYCLE) return;
  const double2 *hs = reinterpret_cast<const double2 *>(h) + (long long)s * NV;
  double2 *Hs = reinterpret_cast<double2 *>(H) + (long long)s * (m + 1) * m;   // column-major [col][row], ld m+1
  double2 *css = reinterpret_cast<double2 *>(cs) + (long long)s * m;
  double2 *sns = reinterpret_cast<double2 *>(sn) + (long long)s * m;
  double2 *gs = reinterpret_cast<double2 *>(g) + (long long)s * (m + 1);
  double2 col[65];
  for (int i = 0; i <= k; i++) col[i] = hs[i];
  const double hk1 = sqrt(fmax(hs[k + 1].x, 0.0));
  col[k + 1] = make_double2(hk1, 0.0);
  for (int i = 0; i < k; i++) {   // previous rotations: [c, s; -conj(s), conj(c)]
    const double2 c = css[i], sv = sns[i], a = col[i], b = col[i + 1];
    const double2 t = make_double2(c.x * a.x - c.y * a.y + sv.x * b.x - sv.y * b.y,
                                   c.x * a.y + c.y * a.x + sv.x * b.y + sv.y * b.x);
    const double2 u = make_double2(-(sv.x * a.x + sv.y * a.y) + (c.x * b.x + c.y * b.y),
                                   -(sv.x * a.y - sv.y * a.x) + (c.x * b.y - c.y * b.x));
    col[i] = t;
    col[i + 1] = u;
  }
  const double2 a = col[k], b = col[k + 1];
  const double den = sqrt(a.x * a.x + a.y * a.y + b.x * b.x + b.y * b.y);
  double2 c, sv;
  if (den > 0.0) {
    c = make_double2(a.x / den, -a.y / den);    // conj(a) / den
    sv = make_double2(b.x / den, -b.y / den);   // conj(b) / den
  } else {
    c = make_double2(1.0, 0.0);
    sv = make_double2(0.0, 0.0);
  }
  css[k] = c;
  sns[k] = sv;
  col[k] = make_double2(den, 0.0);
  col[k + 1] = make_double2(0.0, 0.0);
  const double2 gk = gs[k];
  gs[k + 1] = make_double2(-(sv.x * gk.x + sv.y * gk.y), -(sv.x * gk.y - sv.y * gk.x));   // -conj(s) g_k
  gs[k] = make_double2(c.x * gk.x - c.y * gk.y, c.x * gk.y + c.y * gk.x);                  // c g_k
  for (int i = 0; i <= k; i++) Hs[(long long)k * (m + 1) + i] = col[i];
  iters[s] += 1;
  const double res = sqrt(gs[k + 1].x * gs[k + 1].x + gs[k + 1].y * gs[k + 1].y);
  est[s] = bnorm[s] > 0.0 ? res / bnorm[s] : 0.0;
  const bool breakdown = !(hk1 > 1e-14 * den);
  if (res <= tol * bnorm[s] || breakdown || k + 1 == m || den == 0.0) {
    state[s] = ST_CYCLE_DONE;
    kcyc[s] = k + 1;
  }
}

// y = R^-1 g (back substitution on the rotated Hessenberg), stored in y[s*NV + i]
__global__ void backsolve_kernel(int nsys, int m, const double *H, const double *g, const int *state, const int *kcyc,
                                 double *y, int NV) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsys || state[s] != ST_CYCLE_DONE) return;
  const double2 *Hs = reinterpret_cast<const double2 *>(H) + (long long)s * (m + 1) * m;
  const double2 *gs = reinterpret_cast<const double2 *>(g) + (long long)s * (m + 1);
  double2 *ys = reinterpret_cast<double2 *>(y) + (long long)s * NV;
  const int k = kcyc[s];
  for (int i = k - 1; i >= 0; i--) {
    double2 acc = gs[i];
    for (int j = i + 1; j < k; j++) {
      const double2 r = Hs[(long long)j * (m + 1) + i], yj = ys[j];
      acc.x -= r.x * yj.x - r.y * yj.y;
      acc.y -= r.x * yj.y + r.y * yj.x;
    }
    const double2 d = Hs[(long long)i * (m + 1) + i];
    const double dd = d.x * d.x + d.y * d.y;
    ys[i] = dd > 0.0 ? make_double2((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd)
                     : make_double2(0.0, 0.0);
  }
  for (int i = k; i < NV; i++) ys[i] = make_double2(0.0, 0.0);
}

__global__ void coef_add_kernel(int nsys, int nv, double *h, const double *h2, int NV, const int *state, int want) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)nsys * nv) return;
  const int s = (int)(t / nv), i = (int)(t % nv);
  if (state[s] != want) return;
  const long long q = 2 * ((long long)s * NV + i);
  h[q] += h2[q];
  h[q + 1] += h2[q + 1];
}


// ---------------------------------------------------------------- fused Gram-Schmidt passes
// Both passes stream the Krylov basis of a system once per chunk of CGS_CHUNK elements.  They are
// HBM-bound, so what matters is the number of independent loads each thread has in flight:
// * dots: each warp of a block owns whole basis vectors (i = warp, warp + 8, ...; i = nv is w
//   itself, for ||w||^2) and sweeps the chunk with CGS_UNROLL independent loads per lane; w is
//   re-read by every warp from L1.  No block-level reduction: one warp shuffle per vector.
// * update: every thread owns two elements and accumulates sum_i c_i V_i over batches of
//   CGS_BATCH vectors whose loads are predicated (not branched), so they issue together.
constexpr int CGS_THREADS = 256, CGS_CHUNK = 4096, CGS_UNROLL = 8, CGS_BATCH = 8;
constexpr double REORTH_THETA_F32 = 0.01;   // FP32 Krylov vectors: second pass where ||w'|| < 0.1 ||w||

template <typename T>
__global__ __launch_bounds__(CGS_THREADS) void cgs_dots_kernel(const T *V, long long vs, long long vi, int nv,
                                                               const T *w, long long n, int nch, const int *state,
                                                               int want, double *partial, int NV) {
  const int s = blockIdx.y, chunk = blockIdx.x;
  if (state[s] != want) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long e0 = (long long)chunk * CGS_CHUNK;
  const long long e1 = e0 + CGS_CHUNK < n ? e0 + CGS_CHUNK : n;
  const T *ws = w + 2 * s * vs;
  const T *Vs = V + 2 * s * vs;
  for (int i = warp; i <= nv; i += CGS_THREADS / 32) {
    const T *vp = i < nv ? Vs + 2 * i * vi : ws;   // slot nv: ||w||^2
    T ar = T(0), ai = T(0);
    long long e = e0 + lane;
    // full rounds: CGS_UNROLL unconditional loads of the basis vector and of w in flight per lane
    for (; e + 32 * (CGS_UNROLL - 1) < e1; e += 32 * CGS_UNROLL) {
      CT<T> a[CGS_UNROLL], x[CGS_UNROLL];
#pragma unroll
      for (int u = 0; u < CGS_UNROLL; u++) {
        a[u] = ldc(vp, e + 32 * u);
        x[u] = ldc(ws, e + 32 * u);
      }
#pragma unroll
      for (int u = 0; u < CGS_UNROLL; u++) {
        ar += a[u].x * x[u].x + a[u].y * x[u].y;
        ai += a[u].x * x[u].y - a[u].y * x[u].x;
      }
    }
    for (; e < e1; e += 32) {
      const CT<T> a = ldc(vp, e), x = ldc(ws, e);
      ar += a.x * x.x + a.y * x.y;
      ai += a.x * x.y - a.y * x.x;
    }
    double2 acc = make_double2((double)ar, (double)ai);
    for (int off = 16; off > 0; off >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
    }
    if (lane == 0) reinterpret_cast<double2 *>(partial)[((long long)s * NV + i) * nch + chunk] = acc;
  }
}

// w -= V h2 (in place), then the partial squared norm of w (slot 0)
template <typename T>
__global__ __launch_bounds__(CGS_THREADS) void cgs_update_norm_kernel(const T *V, long long vs, long long vi, int nv,
                                                                      T *w, long long n, int nch, const int *state,
                                                                      int want, const double *h2, double *partial,
                                                                      int NV) {
  __shared__ CT<T> hh[72];
  __shared__ double sh[CGS_THREADS / 32];
  const int s = blockIdx.y, chunk = blockIdx.x;
  if (state[s] != want) return;
  for (int i = threadIdx.x; i < nv; i += CGS_THREADS) {
    const double2 c = reinterpret_cast<const double2 *>(h2)[(long long)s * NV + i];
    hh[i] = mkc<T>(c.x, c.y);
  }
  __syncthreads();
  const long long e0 = (long long)chunk * CGS_CHUNK;
  const long long e1 = e0 + CGS_CHUNK < n ? e0 + CGS_CHUNK : n;
  T *ws = w + 2 * s * vs;
  const T *Vs = V + 2 * s * vs;
  T nn = T(0);
  for (long long e = e0 + threadIdx.x; e < e1; e += 2 * CGS_THREADS) {
    const long long f = e + CGS_THREADS;
    const bool inf = f < e1;
    CT<T> acc0 = mkc<T>(0.0, 0.0), acc1 = mkc<T>(0.0, 0.0);
    // element f: the second element of the thread, or (past the chunk) a repeat of e whose result is
    // not stored, so that every load below is unconditional
    const long long fl = inf ? f : e;
    int i0 = 0;
    for (; i0 + CGS_BATCH <= nv; i0 += CGS_BATCH) {
      CT<T> a0[CGS_BATCH], a1[CGS_BATCH];
#pragma unroll
      for (int j = 0; j < CGS_BATCH; j++) {
        const T *vp = Vs + 2 * (long long)(i0 + j) * vi;
        a0[j] = ldc(vp, e);
        a1[j] = ldc(vp, fl);
      }
#pragma unroll
      for (int j = 0; j < CGS_BATCH; j++) {
        const CT<T> c = hh[i0 + j];
        acc0.x += c.x * a0[j].x - c.y * a0[j].y;
        acc0.y += c.x * a0[j].y + c.y * a0[j].x;
        acc1.x += c.x * a1[j].x - c.y * a1[j].y;
        acc1.y += c.x * a1[j].y + c.y * a1[j].x;
      }
    }
    for (; i0 < nv; i0++) {
      const T *vp = Vs + 2 * (long long)i0 * vi;
      const CT<T> a0 = ldc(vp, e), a1 = ldc(vp, fl), c = hh[i0];
      acc0.x += c.x * a0.x - c.y * a0.y;
      acc0.y += c.x * a0.y + c.y * a0.x;
      acc1.x += c.x * a1.x - c.y * a1.y;
      acc1.y += c.x * a1.y + c.y * a1.x;
    }
    CT<T> x0 = ldc(ws, e);
    x0.x -= acc0.x;
    x0.y -= acc0.y;
    stc(ws, e, x0);
    nn += x0.x * x0.x + x0.y * x0.y;
    if (inf) {
      CT<T> x1 = ldc(ws, f);
      x1.x -= acc1.x;
      x1.y -= acc1.y;
      stc(ws, f, x1);
      nn += x1.x * x1.x + x1.y * x1.y;
    }
  }
  double t = (double)nn;
  for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int k = 0; k < CGS_THREADS / 32; k++) tot += sh[k];
    reinterpret_cast<double2 *>(partial)[((long long)s * NV) * nch + chunk] = make_double2(tot, 0.0);
  }
}

// Selective reorthogonalisation (Daniel, Gragg, Kaufman & Stewart 1976): a second Gram-Schmidt
// pass only where the first one cancelled more than half of w (||w'||^2 < ||w||^2 / 2).
__global__ void reorth_flag_kernel(int nsys, const int *state, int want, const double *h, const double *w2, int NV,
                                   int nv, double theta, int *flag) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsys) return;
  const double before = h[2 * ((long long)s * NV + nv)];    // ||w||^2 from the first pass
  const double after = w2[2 * ((long long)s * NV)];          // ||w'||^2
  flag[s] = (state[s] == want && after < theta * before) ? 1 : 0;
}

// h[s][i] += h2[s][i] (i < nv) and h[s][nv] = ||w||^2 for the flagged systems; copy the final norm
__global__ void reorth_merge_kernel(int nsys, int nv, double *h, const double *h2, const double *n1, const double *n2,
                                    int NV, const int *state, int want, const int *flag) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsys || state[s] != want) return;
  double2 *hs = reinterpret_cast<double2 *>(h) + (long long)s * NV;
  const double2 *h2s = reinterpret_cast<const double2 *>(h2) + (long long)s * NV;
  if (flag[s]) {
    for (int i = 0; i < nv; i++) {
      hs[i].x += h2s[i].x;
      hs[i].y += h2s[i].y;
    }
    hs[nv] = make_double2(n2[2 * (long long)s * NV], 0.0);
  } else {
    hs[nv] = make_double2(n1[2 * (long long)s * NV], 0.0);
  }
}

__global__ void set_state_kernel(int nsys, int *state, int from, int to) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < nsys && state[s] == from) state[s] = to;
}

// x_s = u_s / D_s (final solution from the preconditioned iterate)
template <typename T>
__global__ void unprecondition_kernel(T *U, long long n, int nsys, const double *omega, double eta, double zsign,
                                      const double *diag, double dsign) {
  const long long tot = n * nsys;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(t / n);
    const long long mu = t - (long long)s * n;
    const double dr = omega[s] + dsign * diag[mu], di = zsign * eta;
    const double d2 = dr * dr + di * di;
    const CT<T> u = ldc(U, t);
    const double ux = u.x, uy = u.y;
    stc(U, t, mkc<T>((ux * dr + uy * di) / d2, (uy * dr - ux * di) / d2));
  }
}

// u_s = D_s x_s (an initial iterate into the preconditioned coordinates)
template <typename T>
__global__ void precondition_kernel(T *U, long long n, int nsys, const double *omega, double eta, double zsign,
                                    const double *diag, double dsign) {
  const long long tot = n * nsys;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(t / n);
    const long long mu = t - (long long)s * n;
    const double dr = omega[s] + dsign * diag[mu], di = zsign * eta;
    const CT<T> x = ldc(U, t);
    const double xx = x.x, xy = x.y;
    stc(U, t, mkc<T>(xx * dr - xy * di, xx * di + xy * dr));
  }
}

__global__ void norm_from_partial_kernel(int nsys, const double *nrm2, int NV, double *out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < nsys) out[s] = sqrt(fmax(nrm2[2 * (long long)s * NV], 0.0));
}

}  // namespace

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------

namespace {
// doubles occupied by `count` elements of type T
template <typename T>
long long dbl_of(long long count) {
  return (count * (long long)sizeof(T) + 7) / 8;
}
}  // namespace

long long gmres_work_doubles(const gfcc_ctx *c, int sector, long long n, int nsys, int m, bool mixed) {
  const long long NV = m + 2;
  const long long nch = (n + DOT_CHUNK - 1) / DOT_CHUNK;   // the finer of the two chunkings
  const bool f32 = mixed && c->inner_fp64 == 0;
  long long w = 0;
  const long long vb = 2LL * nsys * (m + 1) * n, vv = 2LL * nsys * n;
  w += f32 ? dbl_of<float>(vb) : vb;            // V
  w += 3 * (f32 ? dbl_of<float>(vv) : vv);      // U, B, W
  w += 2LL * nsys * NV * nch;               // dot partials
  w += 2LL * nsys * NV * 5;                 // h, h2, y, nrm (two slots)
  w += 2LL * nsys * (m + 1) * m;            // H
  w += 2LL * nsys * (2 * m + (m + 1));      // cs, sn, g
  w += 9LL * nsys + 512;                    // bnorm, relres, relres0, est, omega, int state/kcyc/iters/rflag/act,
                                            // alignment
  w += sigma_work_doubles(c, sector, nsys);
  if (mixed) {
    w += 5 * 2LL * nsys * n + nsys + 64;     // X, R, B0, D, A D, ||b0||
    w += sigma_mixed_work_doubles(c, nsys);
    if (c->eWr.dig != nullptr || c->eWre.dig != nullptr)
      w += sigma_emu_work_doubles(c, std::min(nsys, EMU_SUB_MAX));
  }
  return w;
}

int Gmres::init(gfcc_ctx *ctx, int sec, long long dim, int ns, int mm, double *work, bool mx) {
  c = ctx;
  mixed = mx;
  f32 = mixed && c->inner_fp64 == 0;
  sector = sec;
  n = dim;
  nsys = ns;
  m = mm;
  NV = m + 2;
  nch = (int)((n + DOT_CHUNK - 1) / DOT_CHUNK);
  const long long nch_alloc = (n + DOT_CHUNK - 1) / DOT_CHUNK;
  double *p = work;
  auto take = [&](double *&dst, long long cnt) {
    dst = p;
    p += (cnt + 7) & ~7LL;
  };
  const long long vb = 2LL * nsys * (m + 1) * n, vv = 2LL * nsys * n;
  take(V, f32 ? dbl_of<float>(vb) : vb);
  take(U, f32 ? dbl_of<float>(vv) : vv);
  take(B, f32 ? dbl_of<float>(vv) : vv);
  take(W, f32 ? dbl_of<float>(vv) : vv);
  take(partial, 2LL * nsys * NV * nch_alloc);
  take(h, 2LL * nsys * NV);
  take(h2, 2LL * nsys * NV);
  take(y, 2LL * nsys * NV);
  take(nrm, 2LL * 2 * nsys * NV);
  take(H, 2LL * nsys * (m + 1) * m);
  take(cs, 2LL * nsys * m);
  take(sn, 2LL * nsys * m);
  take(g, 2LL * nsys * (m + 1));
  take(bnorm, nsys);
  take(relres, nsys);
  take(relres0, nsys);
  take(est, nsys);
  take(omega, nsys);
  double *ip;
  take(ip, 5LL * nsys);
  state = reinterpret_cast<int *>(ip);
  kcyc = state + nsys;
  iters = kcyc + nsys;
  rflag = iters + nsys;
  act = rflag + nsys;
  if (mixed) {
    take(X, 2LL * nsys * n);
    take(R, 2LL * nsys * n);
    take(B0, 2LL * nsys * n);
    take(D, 2LL * nsys * n);
    take(Yd, 2LL * nsys * n);
    take(b0norm, nsys);
  }
  sigma_work = p;
  long long used = (p - work) + sigma_work_doubles(c, sector, nsys);
  if (mixed) used += sigma_mixed_work_doubles(c, nsys) + 64;
  if (used > gmres_work_doubles(c, sector, n, nsys, m, mixed)) {
    set_error("internal: GMRES workspace layout (%lld doubles) exceeds its size", used);
    return GFCC_ERR_ARG;
  }
  return GFCC_OK;
}

int Gmres::op_fp64(const double *x, long long ldx, double *yout, long long ldy, int level) {
  const bool ip = sector == GFCC_SECTOR_IP;
  if (mixed && c->residual_emulated && (ip ? c->eWr.dig : c->eWre.dig) != nullptr) {
    SysBatch b;
    b.nsys = nsys;
    b.x = x;
    b.ldx = ldx;
    b.y = yout;
    b.ldy = ldy;
    b.omega = omega;
    b.eta = eta;
    b.dsign = ip ? 1.0 : -1.0;
    b.zsign = ip ? -1.0 : 1.0;
    double *ew = sigma_work + sigma_work_doubles(c, sector, nsys) + sigma_mixed_work_doubles(c, nsys);
    const long long ewd = sigma_emu_work_doubles(c, std::min(nsys, EMU_SUB_MAX));
    return ip ? apply_ip_emu(c, b, ew, ewd, level) : apply_ea_emu(c, b, ew, ewd, level);
  }
  SysBatch b;
  b.nsys = nsys;
  b.x = x;
  b.ldx = ldx;
  b.y = yout;
  b.ldy = ldy;
  b.omega = omega;
  b.eta = eta;
  b.diag = nullptr;
  b.dsign = sector == GFCC_SECTOR_IP ? 1.0 : -1.0;
  b.zsign = sector == GFCC_SECTOR_IP ? -1.0 : 1.0;
  return sector == GFCC_SECTOR_IP ? apply_ip(c, b, sigma_work) : apply_ea(c, b, sigma_work);
}

template <typename T>
int Gmres::op_t(const T *x, long long ldx, T *yout, long long ldy, int nact, const int *idx) {
  SysBatch b;
  b.nsys = nact > 0 ? nact : nsys;
  b.idx = nact > 0 ? idx : nullptr;
  if constexpr (sizeof(T) == sizeof(float)) {
    b.xf = x;
    b.yf = yout;
  } else {
    b.x = x;
    b.y = yout;
  }
  b.ldx = ldx;
  b.ldy = ldy;
  b.omega = omega;
  b.eta = eta;
  b.diag = use_precond ? (sector == GFCC_SECTOR_IP ? c->diag_ip : c->diag_ea) : nullptr;
  b.dsign = sector == GFCC_SECTOR_IP ? 1.0 : -1.0;
  b.zsign = sector == GFCC_SECTOR_IP ? -1.0 : 1.0;
  if (mixed) {
    double *mw = sigma_work + sigma_work_doubles(c, sector, nsys);
    return sector == GFCC_SECTOR_IP ? apply_ip_mixed(c, b, mw) : apply_ea_mixed(c, b, mw);
  }
  if constexpr (sizeof(T) == sizeof(float)) {
    set_error("internal: FP32 Krylov vectors need the mixed-precision IP operator");
    return GFCC_ERR_STATE;
  } else {
    return sector == GFCC_SECTOR_IP ? apply_ip(c, b, sigma_work) : apply_ea(c, b, sigma_work);
  }
}

// dots of vectors [0, nv) of each system's basis (V + s*vs + i*vi) with w (w + s*ws) -> out
template <typename T>
int Gmres::mdot_t(const T *Vb, long long vs, long long vi, int nv, const T *w, long long ws, double *out, int want,
                  int accumulate) {
  cudaStream_t st = c->stream;
  dim3 grid(nch, nsys);
  const int *filt = want < 0 ? nullptr : state;   // want < 0: every system
  mdot_partial_kernel<T><<<grid, DOT_THREADS, 0, st>>>(Vb, vs, vi, nv, w, ws, n, nch, filt, want, partial, NV);
  GFCC_LAUNCH_CHECK();
  const int warps = nsys * nv;
  mdot_final_kernel<<<cdiv(warps * 32LL, 256), 256, 0, st>>>(partial, nsys, nv, NV, nch, filt, want, out, accumulate);
  GFCC_LAUNCH_CHECK();
  return GFCC_OK;
}

int Gmres::mdot(const double *Vb, long long vs, long long vi, int nv, const double *w, long long ws, double *out,
                int want, int accumulate) {
  return mdot_t<double>(Vb, vs, vi, nv, w, ws, out, want, accumulate);
}

template <typename T>
int Gmres::cgs2_t(const T *Vb, long long vs, int nv, T *w, cudaStream_t st) {
  const int nchc = (int)((n + CGS_CHUNK - 1) / CGS_CHUNK);   // partial holds nch_alloc >= nchc chunks
  dim3 grid(nchc, nsys);
  const int TH = 256;
  // pass p (0: dots and norm, 2: update and norm) over the systems whose filter array equals `want`
  auto pass = [&](int p, const double *coef, const int *filt, int want) -> int {
    if (p == 0)
      cgs_dots_kernel<T><<<grid, CGS_THREADS, 0, st>>>(Vb, vs, n, nv, w, n, nchc, filt, want, partial, NV);
    else
      cgs_update_norm_kernel<T><<<grid, CGS_THREADS, 0, st>>>(Vb, vs, n, nv, w, n, nchc, filt, want, coef, partial,
                                                             NV);
    GFCC_LAUNCH_CHECK();
    return GFCC_OK;
  };
  auto final = [&](int nvv, double *out, const int *filt, int want) -> int {
    mdot_final_kernel<<<cdiv(nsys * (long long)nvv * 32, 256), 256, 0, st>>>(partial, nsys, nvv, NV, nchc, filt, want,
                                                                             out, 0);
    GFCC_LAUNCH_CHECK();
    return GFCC_OK;
  };
  int *flag = rflag;
  // pass 1: h = V^H w and ||w||^2 (slot nv)
  GFCC_TRY(pass(0, nullptr, state, ST_IN_CYCLE));
  GFCC_TRY(final(nv + 1, h, state, ST_IN_CYCLE));
  // pass 2: w -= V h, ||w'||^2
  GFCC_TRY(pass(2, h, state, ST_IN_CYCLE));
  GFCC_TRY(final(1, nrm, state, ST_IN_CYCLE));
  // passes 3-4 only where the first pass cancelled most of w
  // Second pass where ||w'||^2 < theta ||w||^2.  The orthogonality lost by the new vector is about
  // the relative rounding error of the pass times ||w|| / ||w'||: FP64 solves reorthogonalise below
  // 1/sqrt(2) (the usual twice-is-enough test); the FP32 inner solves of the refinement, which stop
  // at a relative residual of 3e-4 and are corrected by the FP64-accurate outer residual, only where
  // the first pass cancelled more than 90% of w (orthogonality loss <= 10 x about 1e-6 per vector).
  const double theta = sizeof(T) == sizeof(float) ? REORTH_THETA_F32 : 0.5;
  reorth_flag_kernel<<<cdiv(nsys, TH), TH, 0, st>>>(nsys, state, ST_IN_CYCLE, h, nrm, NV, nv, theta, flag);
  GFCC_LAUNCH_CHECK();
  GFCC_TRY(pass(0, nullptr, flag, 1));
  GFCC_TRY(final(nv, h2, flag, 1));
  GFCC_TRY(pass(2, h2, flag, 1));
  GFCC_TRY(final(1, nrm + 2 * NV * (long long)nsys, flag, 1));
  reorth_merge_kernel<<<cdiv(nsys, TH), TH, 0, st>>>(nsys, nv, h, h2, nrm, nrm + 2 * NV * (long long)nsys, NV, state,
                                                     ST_IN_CYCLE, flag);
  GFCC_LAUNCH_CHECK();
  vscale_kernel<T><<<vscale_grid(n, nsys), 256, 0, st>>>(w, vs, n, h, NV, nv, state, ST_IN_CYCLE);
  GFCC_LAUNCH_CHECK();
  return GFCC_OK;
}

Gmres::~Gmres() { drop_graphs(); }

void Gmres::drop_graphs() {
  for (cudaGraphExec_t &g : gexec)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

int Gmres::solve(double tol, int max_iters, int *h_state, int max_cycles, bool use_x0) {
  return f32 ? solve_t<float>(tol, max_iters, h_state, max_cycles, use_x0)
             : solve_t<double>(tol, max_iters, h_state, max_cycles, use_x0);
}

template <typename T>
int Gmres::solve_t(double tol, int max_iters, int *h_state, int max_cycles, bool use_x0) {
  cudaStream_t st = c->stream;
  const long long vs = (long long)(m + 1) * n;   // basis stride per system (complex elements)
  const int TH = 256;
  T *Vt = reinterpret_cast<T *>(V), *Ut = reinterpret_cast<T *>(U), *Bt = reinterpret_cast<T *>(B);
  T *Wt = reinterpret_cast<T *>(W);
  const double dsg = sector == GFCC_SECTOR_IP ? 1.0 : -1.0, zsg = sector == GFCC_SECTOR_IP ? -1.0 : 1.0;
  const double *dg = sector == GFCC_SECTOR_IP ? c->diag_ip : c->diag_ea;
  // CUDA graphs for the inner solves of the refinement (FP32 Krylov vectors) on a created stream,
  // not while profiling (the phase timers are stream events); the contraction shapes of the current
  // number of systems must have been seen (and tuned) before a capture
  const bool use_graphs =
      sizeof(T) == sizeof(float) && mixed && c->use_graphs && graphs_ok && !c->prof && st != nullptr;
  if (use_graphs) {
    if (gnsys != nsys) {
      drop_graphs();
      gexec.assign(m, nullptr);
      glaunch.assign(m, 0);
      gnsys = nsys;
      gseen = 0;
    }
    gseen++;
  }
  if (!use_x0) {
    GFCC_CUDA(cudaMemsetAsync(Ut, 0, sizeof(T) * 2 * nsys * n, st));
  } else if (use_precond) {
    precondition_kernel<T><<<grid1d(n * nsys), TH, 0, st>>>(Ut, n, nsys, omega, eta, zsg, dg, dsg);
    GFCC_LAUNCH_CHECK();
  }
  GFCC_CUDA(cudaMemsetAsync(Vt, 0, sizeof(T) * 2 * nsys * (m + 1) * n, st));
  GFCC_CUDA(cudaMemsetAsync(iters, 0, sizeof(int) * nsys, st));
  GFCC_CUDA(cudaMemsetAsync(state, 0, sizeof(int) * nsys, st));   // ST_PENDING
  // ||b||
  GFCC_TRY(mdot_t<T>(Bt, n, 0, 1, Bt, n, nrm, ST_PENDING, 0));
  norm_from_partial_kernel<<<cdiv(nsys, TH), TH, 0, st>>>(nsys, nrm, NV, bnorm);
  GFCC_LAUNCH_CHECK();
  bool first = !use_x0;
  for (int cycle = 0;; cycle++) {
    if (max_cycles > 0 && cycle >= max_cycles) {
      // cycle budget spent: the systems still pending keep their iterate (state 4)
      set_state_kernel<<<cdiv(nsys, TH), TH, 0, st>>>(nsys, state, ST_PENDING, ST_FAILED);
      GFCC_LAUNCH_CHECK();
      break;
    }
    // true residual r = b - A x into V_0 (x = 0 on the first cycle)
    if (first) {
      GFCC_CUDA(cudaMemsetAsync(Wt, 0, sizeof(T) * 2 * nsys * n, st));
    } else {
      GFCC_TRY(op_t<T>(Ut, n, Wt, n));
    }
    resid_form_kernel<T><<<grid1d(n * nsys), TH, 0, st>>>(Bt, Wt, Vt, vs, n, nsys, state);
    GFCC_LAUNCH_CHECK();
    GFCC_TRY(mdot_t<T>(Vt, vs, 0, 1, Vt, vs, nrm, ST_PENDING, 0));
    cycle_start_kernel<<<cdiv(nsys, TH), TH, 0, st>>>(nsys, nrm, NV, bnorm, tol, max_iters, m + 1, state, iters,
                                                      relres, g, H);
    GFCC_LAUNCH_CHECK();
    vscale_kernel<T><<<vscale_grid(n, nsys), 256, 0, st>>>(Vt, vs, n, nrm, NV, 0, state, ST_IN_CYCLE);
    GFCC_LAUNCH_CHECK();
    if (cycle == 0) GFCC_CUDA(cudaMemcpyAsync(relres0, relres, sizeof(double) * nsys, cudaMemcpyDeviceToDevice, st));
    first = false;
    GFCC_CUDA(cudaMemcpyAsync(h_state, state, sizeof(int) * nsys, cudaMemcpyDeviceToHost, st));
    GFCC_CUDA(cudaStreamSynchronize(st));
    bool any = false;
    for (int s = 0; s < nsys; s++) any |= h_state[s] == ST_IN_CYCLE;
    if (!any) break;
    // Arnoldi steps
    int active = 0;
    for (int s = 0; s < nsys; s++) active += h_state[s] == ST_IN_CYCLE;
    // Systems whose cycle has ended stay in the batch until the cycle of every system has: the
    // operator then runs on the systems in cycle only (their list, padded to a multiple of 4 with
    // entries that read an active system and store nothing, so that the contraction widths repeat)
    int nact = -1;
    std::vector<int> h_act;
    auto plan_active = [&]() -> int {
      nact = -1;
      if (active >= nsys || active == 0) return GFCC_OK;
      h_act.clear();
      for (int s = 0; s < nsys; s++)
        if (h_state[s] == ST_IN_CYCLE) h_act.push_back(s);
      const int padded = std::min(nsys, (active + 3) / 4 * 4);
      while ((int)h_act.size() < padded) h_act.push_back(-1 - h_act[0]);
      if (padded >= nsys) return GFCC_OK;   // no narrower than the batch: run it whole
      GFCC_CUDA(cudaMemcpyAsync(act, h_act.data(), sizeof(int) * padded, cudaMemcpyHostToDevice, st));
      nact = padded;
      return GFCC_OK;
    };
    GFCC_TRY(plan_active());
    for (int k = 0; k < m; k++) {
      T *vk = Vt + 2 * (long long)k * n;
      T *w = Vt + 2 * (long long)(k + 1) * n;
      auto step = [&]() -> int {
        GFCC_TRY(op_t<T>(vk, vs, w, vs, nact, act));
        // Gram-Schmidt against the basis: one classical pass (dots with ||w||^2, then update with
        // ||w'||^2), a second pass only where needed, then w /= ||w||.  Algorithmic bytes of one
        // classical pass per system: dots read k+1 basis vectors and w, the update reads k+1 basis
        // vectors and reads / writes w, the scaling reads / writes w.
        {
          const double bytes = (double)active * (2.0 * (k + 1) + 5.0) * (double)n * 2.0 * sizeof(T);
          PhaseTimer ta(c, PH_ARNOLDI, bytes);
          GFCC_TRY(cgs2_t<T>(Vt, vs, k + 1, w, st));
        }
        {
          PhaseTimer tl(c, PH_LSQ);
          givens_kernel<<<cdiv(nsys, TH), TH, 0, st>>>(nsys, k, m, h, NV, H, cs, sn, g, bnorm, tol, state, kcyc,
                                                       iters, est);
          GFCC_LAUNCH_CHECK();
        }
        return GFCC_OK;
      };
      bool done_step = false;
      if (use_graphs && gseen > 1 && !gbroken && nact < 0) {
        if (!gexec[k]) {
          // capture the step once (its launches are counted as they are recorded; the launch right
          // after the capture runs them), replay it afterwards.  A capture that fails leaves the
          // graphs off for this solver and the step runs directly.
          const long long l0 = thread_launch_count();   // other threads may launch meanwhile
          cudaGraph_t gr = nullptr;
          cudaError_t ec = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
          int rc = GFCC_ERR_CUDA;
          if (ec == cudaSuccess) {
            rc = step();
            ec = cudaStreamEndCapture(st, &gr);
          }
          if (rc == GFCC_OK && ec == cudaSuccess && gr != nullptr &&
              cudaGraphInstantiate(&gexec[k], gr, 0) == cudaSuccess) {
            glaunch[k] = thread_launch_count() - l0;
            GFCC_CUDA(cudaGraphLaunch(gexec[k], st));
            done_step = true;
          } else {
            cudaGetLastError();
            gexec[k] = nullptr;
            gbroken = true;
            count_launches(l0 - thread_launch_count());   // nothing of the failed capture ran
          }
          if (gr) cudaGraphDestroy(gr);
        } else {
          GFCC_CUDA(cudaGraphLaunch(gexec[k], st));
          count_launches(glaunch[k]);
          done_step = true;
        }
      }
      if (!done_step) GFCC_TRY(step());
      GFCC_CUDA(cudaMemcpyAsync(h_state, state, sizeof(int) * nsys, cudaMemcpyDeviceToHost, st));
      GFCC_CUDA(cudaStreamSynchronize(st));
      active = 0;
      for (int s = 0; s < nsys; s++) active += h_state[s] == ST_IN_CYCLE;
      if (active == 0) break;
      GFCC_TRY(plan_active());
    }
    // x += V y
    backsolve_kernel<<<cdiv(nsys, TH), TH, 0, st>>>(nsys, m, H, g, state, kcyc, y, NV);
    GFCC_LAUNCH_CHECK();
    vupdate_kernel<T><<<grid1d(n * nsys), TH, 0, st>>>(Vt, vs, n, m, kcyc, y, NV, 1.0, Ut, n, n, nsys, state,
                                                       ST_CYCLE_DONE);
    GFCC_LAUNCH_CHECK();
    set_state_kernel<<<cdiv(nsys, TH), TH, 0, st>>>(nsys, state, ST_CYCLE_DONE, ST_PENDING);
    GFCC_LAUNCH_CHECK();
  }
  if (use_precond) {
    unprecondition_kernel<T><<<grid1d(n * nsys), TH, 0, st>>>(Ut, n, nsys, omega, eta, zsg, dg, dsg);
    GFCC_LAUNCH_CHECK();
  }
  return GFCC_OK;
}

namespace {
// y = a - y (all systems, contiguous [s][n] complex)
__global__ void rsub_kernel(const double *a, double *y, long long tot) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x)
    y[t] = a[t] - y[t];
}
// y = x rounded to FP32
__global__ void to_f32_kernel(const double *x, float *y, long long tot) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x)
    y[t] = (float)x[t];
}
// D = d (FP64 copy of the inner correction) and x += d (all systems)
template <typename T>
__global__ void add_keep_kernel(double *x, double *D, const T *d, long long tot) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const double v = (double)d[t];
    D[t] = v;
    x[t] += v;
  }
}
// y -= a (all systems)
__global__ void sub_kernel(double *y, const double *a, long long tot) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x)
    y[t] -= a[t];
}
// amax[s] = max |v_s| over both planes of system s ([s][n] complex); grid (blocks, nsys), amax
// zeroed by the caller.  Non-negative doubles order like their bit patterns, so the maximum is
// an integer atomicMax.
__global__ void absmax_kernel(const double *v, long long n, unsigned long long *amax) {
  const int s = blockIdx.y;
  const double *vs = v + 2 * (long long)s * n;
  double m = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 2 * n; t += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(vs[t]));
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(&amax[s], (unsigned long long)__double_as_longlong(m));
}
// per system: relres = ||r|| / ||b0||; done systems get r = 0 so that the inner solve leaves them alone
__global__ void refine_check_kernel(int nsys, const double *nrm2, int NV, const double *b0norm, double tol, int *done,
                                    double *relres) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsys) return;
  const double r = sqrt(fmax(nrm2[2 * (long long)s * NV], 0.0));
  relres[s] = b0norm[s] > 0.0 ? r / b0norm[s] : 0.0;
  done[s] = (b0norm[s] == 0.0 || r <= tol * b0norm[s]) ? 1 : 0;
}
__global__ void zero_done_kernel(double *R, long long n, int nsys, const int *done) {
  const long long tot = n * nsys;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x)
    if (done[t / n]) {
      R[2 * t] = 0.0;
      R[2 * t + 1] = 0.0;
    }
}
}  // namespace

namespace {
__global__ void reset_slots_kernel(double *X, double *R, const double *B0, long long n, int nsys, const int *mask) {
  const long long tot = n * nsys;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    if (!mask[t / n]) continue;
    reinterpret_cast<double2 *>(X)[t] = make_double2(0.0, 0.0);
    reinterpret_cast<double2 *>(R)[t] = reinterpret_cast<const double2 *>(B0)[t];
  }
}
}  // namespace

namespace {
// dst[q] = src[perm[q]] for q < na (rows of n complex)
__global__ void gather_rows_kernel(const double *src, double *dst, long long n, int na, const int *perm) {
  const long long tot = n * na;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(t / n);
    const long long i = t - (long long)q * n;
    reinterpret_cast<double2 *>(dst)[t] = reinterpret_cast<const double2 *>(src)[(long long)perm[q] * n + i];
  }
}
}  // namespace

int Gmres::compact_slots(const int *d_perm, int na) {
  cudaStream_t st = c->stream;
  if (na <= 0 || na > nsys) {
    set_error("internal: compact_slots(%d) with %d slots", na, nsys);
    return GFCC_ERR_ARG;
  }
  // Yd (free between refinement steps) is the staging buffer
  for (double *a : {X, B0, R, D}) {
    gather_rows_kernel<<<grid1d(n * na), 256, 0, st>>>(a, Yd, n, na, d_perm);
    GFCC_LAUNCH_CHECK();
    GFCC_CUDA(cudaMemcpyAsync(a, Yd, sizeof(double) * 2 * na * n, cudaMemcpyDeviceToDevice, st));
  }
  nsys = na;
  return GFCC_OK;
}

int Gmres::refine_norms() {
  GFCC_TRY(mdot(B0, n, 0, 1, B0, n, nrm, -1, 0));
  norm_from_partial_kernel<<<cdiv(nsys, 256), 256, 0, c->stream>>>(nsys, nrm, NV, b0norm);
  GFCC_LAUNCH_CHECK();
  return GFCC_OK;
}

int Gmres::reset_slots(const int *d_mask) {
  reset_slots_kernel<<<grid1d(n * nsys), 256, 0, c->stream>>>(X, R, B0, n, nsys, d_mask);
  GFCC_LAUNCH_CHECK();
  return GFCC_OK;
}

int Gmres::refine_residual(int *h_done, double *h_relres) {
  GFCC_TRY(residual_update());
  return refine_residual_free(h_done, h_relres);
}

int Gmres::residual_update() {
  cudaStream_t st = c->stream;
  const long long tot = 2LL * nsys * n;
  const bool emu = c->residual_emulated && (sector == GFCC_SECTOR_IP ? c->eWr.dig : c->eWre.dig) != nullptr;
  if (c->incremental && have_d && emu) {
    // R = B0 - A (X - D) already; R -= A D.  The digit-plane product of D at level P - k has the
    // error bound of the level-P product of X when 2^(6k) <= max|X| / max|D| (the planes of a
    // vector are sliced relative to its own largest entry), so k comes from the worst live slot.
    have_d = false;
    unsigned long long *am = reinterpret_cast<unsigned long long *>(partial);
    GFCC_CUDA(cudaMemsetAsync(am, 0, sizeof(unsigned long long) * 2 * nsys, st));
    const dim3 gr((unsigned)std::min<long long>(64, std::max<long long>(1, (2 * n + 2047) / 2048)), (unsigned)nsys);
    absmax_kernel<<<gr, 256, 0, st>>>(X, n, am);
    GFCC_LAUNCH_CHECK();
    absmax_kernel<<<gr, 256, 0, st>>>(D, n, am + nsys);
    GFCC_LAUNCH_CHECK();
    std::vector<unsigned long long> h(2 * (size_t)nsys);
    GFCC_CUDA(cudaMemcpyAsync(h.data(), am, sizeof(unsigned long long) * 2 * nsys, cudaMemcpyDeviceToHost, st));
    GFCC_CUDA(cudaStreamSynchronize(st));
    int drop = 1 << 20;
    bool any = false;
    for (int s = 0; s < nsys; s++) {
      double dx, dd;
      std::memcpy(&dx, &h[s], sizeof(double));
      std::memcpy(&dd, &h[nsys + s], sizeof(double));
      if (!(dd > 0.0)) continue;   // no correction in this slot (done or empty)
      any = true;
      int ex = 0, ed = 0;
      std::frexp(dx, &ex);
      std::frexp(dd, &ed);
      const int gap = ex - ed - 1;   // log2(max|X| / max|D|) >= gap
      drop = std::min(drop, gap > 0 ? gap / 6 : 0);
    }
    if (any) {
      const int level = std::max(2, c->emu_P - drop);
      GFCC_TRY(op_fp64(D, n, Yd, n, level));
      sub_kernel<<<grid1d(tot), 256, 0, st>>>(R, Yd, tot);
      GFCC_LAUNCH_CHECK();
      c->res_inc++;
      c->res_inc_levels += level;
    }
    return GFCC_OK;
  }
  have_d = false;
  GFCC_TRY(op_fp64(X, n, R, n));
  rsub_kernel<<<grid1d(tot), 256, 0, st>>>(B0, R, tot);
  GFCC_LAUNCH_CHECK();
  c->res_full++;
  return GFCC_OK;
}

int Gmres::refine_residual_free(int *h_done, double *h_relres) {
  cudaStream_t st = c->stream;
  GFCC_TRY(mdot(R, n, 0, 1, R, n, nrm, -1, 0));
  refine_check_kernel<<<cdiv(nsys, 256), 256, 0, st>>>(nsys, nrm, NV, b0norm, tol_outer, kcyc, relres);
  GFCC_LAUNCH_CHECK();
  GFCC_CUDA(cudaMemcpyAsync(h_done, kcyc, sizeof(int) * nsys, cudaMemcpyDeviceToHost, st));
  GFCC_CUDA(cudaMemcpyAsync(h_relres, relres, sizeof(double) * nsys, cudaMemcpyDeviceToHost, st));
  GFCC_CUDA(cudaStreamSynchronize(st));
  return GFCC_OK;
}

int Gmres::refine_correct(const int *h_done, int *h_state, int *h_iters) {
  cudaStream_t st = c->stream;
  const long long tot = 2LL * nsys * n;
  int *done = kcyc;
  GFCC_CUDA(cudaMemcpyAsync(done, h_done, sizeof(int) * nsys, cudaMemcpyHostToDevice, st));
  zero_done_kernel<<<grid1d(n * nsys), 256, 0, st>>>(R, n, nsys, done);
  GFCC_LAUNCH_CHECK();
  if (f32) {
    to_f32_kernel<<<grid1d(tot), 256, 0, st>>>(R, reinterpret_cast<float *>(B), tot);
    GFCC_LAUNCH_CHECK();
  } else {
    GFCC_CUDA(cudaMemcpyAsync(B, R, sizeof(double) * tot, cudaMemcpyDeviceToDevice, st));
  }
  GFCC_TRY(solve(c->inner_tol, c->max_iters, h_state, c->inner_cycles));
  std::vector<int> it(nsys);
  GFCC_CUDA(cudaMemcpyAsync(it.data(), iters, sizeof(int) * nsys, cudaMemcpyDeviceToHost, st));
  if (f32)
    add_keep_kernel<float><<<grid1d(tot), 256, 0, st>>>(X, D, reinterpret_cast<const float *>(U), tot);
  else
    add_keep_kernel<double><<<grid1d(tot), 256, 0, st>>>(X, D, U, tot);
  GFCC_LAUNCH_CHECK();
  have_d = true;
  GFCC_CUDA(cudaStreamSynchronize(st));
  for (int s = 0; s < nsys; s++) h_iters[s] += it[s];
  return GFCC_OK;
}

int Gmres::solve_refined(double tol, double inner_tol, int max_iters, int *h_state, int *h_iters, bool use_x0,
                         int *h_outer) {
  cudaStream_t st = c->stream;
  const long long tot = 2LL * nsys * n;
  const int TH = 256;
  std::vector<int> h_done(nsys, 0), it(nsys, 0);
  for (int s = 0; s < nsys; s++) h_iters[s] = 0;
  if (h_outer)
    for (int s = 0; s < nsys; s++) h_outer[s] = 0;
  // B0 holds the right-hand sides (FP64), X the initial iterate when use_x0
  have_d = false;
  if (!use_x0) GFCC_CUDA(cudaMemsetAsync(X, 0, sizeof(double) * tot, st));
  GFCC_TRY(mdot(B0, n, 0, 1, B0, n, nrm, -1, 0));
  int *done = kcyc;   // reused: per-system done flags between inner solves
  norm_from_partial_kernel<<<cdiv(nsys, TH), TH, 0, st>>>(nsys, nrm, NV, b0norm);
  GFCC_LAUNCH_CHECK();
  const int max_outer = 400;
  bool all_done = false;
  for (int outer = 0; outer <= max_outer; outer++) {
    // FP64-accurate residual r = b - A x (after a correction: r -= A d, see residual_update)
    if (outer == 0 && !use_x0) {
      GFCC_CUDA(cudaMemcpyAsync(R, B0, sizeof(double) * tot, cudaMemcpyDeviceToDevice, st));
    } else {
      GFCC_TRY(residual_update());
    }
    GFCC_TRY(mdot(R, n, 0, 1, R, n, nrm, -1, 0));
    refine_check_kernel<<<cdiv(nsys, TH), TH, 0, st>>>(nsys, nrm, NV, b0norm, tol, done, relres);
    GFCC_LAUNCH_CHECK();
    if (outer == 0) GFCC_CUDA(cudaMemcpyAsync(relres0, relres, sizeof(double) * nsys, cudaMemcpyDeviceToDevice, st));
    GFCC_CUDA(cudaMemcpyAsync(h_done.data(), done, sizeof(int) * nsys, cudaMemcpyDeviceToHost, st));
    GFCC_CUDA(cudaStreamSynchronize(st));
    all_done = true;
    bool any_active = false;
    for (int s = 0; s < nsys; s++) {
      if (h_outer && h_outer[s] == outer) h_outer[s] = outer + 1;   // still active before this check
      all_done &= h_done[s] != 0;
      // a system over its iteration budget stops here (not converged); the others go on
      if (!h_done[s] && h_iters[s] >= max_iters) h_done[s] = 2;
      any_active |= h_done[s] == 0;
    }
    if (all_done || !any_active || outer == max_outer) break;
    GFCC_CUDA(cudaMemcpyAsync(done, h_done.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, st));
    zero_done_kernel<<<grid1d(n * nsys), TH, 0, st>>>(R, n, nsys, done);
    GFCC_LAUNCH_CHECK();
    // inner correction A d = r on the BF16 operator (FP32 or FP64 Krylov vectors), x += d
    if (f32) {
      to_f32_kernel<<<grid1d(tot), TH, 0, st>>>(R, reinterpret_cast<float *>(B), tot);
      GFCC_LAUNCH_CHECK();
    } else {
      GFCC_CUDA(cudaMemcpyAsync(B, R, sizeof(double) * tot, cudaMemcpyDeviceToDevice, st));
    }
    GFCC_TRY(solve(inner_tol, max_iters, h_state, c->inner_cycles));
    GFCC_CUDA(cudaMemcpyAsync(it.data(), iters, sizeof(int) * nsys, cudaMemcpyDeviceToHost, st));
    GFCC_CUDA(cudaStreamSynchronize(st));
    for (int s = 0; s < nsys; s++) h_iters[s] += it[s];
    if (f32)
      add_keep_kernel<float><<<grid1d(tot), TH, 0, st>>>(X, D, reinterpret_cast<const float *>(U), tot);
    else
      add_keep_kernel<double><<<grid1d(tot), TH, 0, st>>>(X, D, U, tot);
    GFCC_LAUNCH_CHECK();
    have_d = true;
  }
  // final state: converged where the FP64 residual met tol; the solution stays in X
  for (int s = 0; s < nsys; s++) h_state[s] = h_done[s] == 1 ? 3 : 4;
  GFCC_CUDA(cudaMemcpyAsync(state, h_state, sizeof(int) * nsys, cudaMemcpyHostToDevice, st));
  GFCC_CUDA(cudaMemcpyAsync(iters, h_iters, sizeof(int) * nsys, cudaMemcpyHostToDevice, st));
  return GFCC_OK;
}

}  // namespace gfcc
