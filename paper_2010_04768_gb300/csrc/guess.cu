// Initial guesses from converged solutions at nearby frequencies (Algorithm 1: "compute initial
// guess"), scored through the Gram matrix of (b, delta_k X_k); see guess.cuh for the identity.
//
// Kernels: the batched 9 x 9 Gram matrices (HBM-bound: one pass over b and the 8 kept neighbours
// of every system), the per-system choice of coefficients (learned or minimal residual, with the
// zero-guess fallback), the combination x0 = sum_k c_k X_k and the FP32 copy of a converged
// solution into the kept-solution store.
#include <algorithm>
#include <cmath>
#include <vector>

#include "guess.cuh"

namespace gfcc {

namespace {

constexpr int GT = 256;                  // threads of the Gram kernel (one element per thread per tile)
constexpr int GCHUNK = 16 * GT;          // elements per block
constexpr int NPAIR = (GUESS_K + 1) * (GUESS_K + 2) / 2;   // 45 pairs j <= l
constexpr double MINRES_REG = 1e-12;     // Tikhonov shift of the normal equations, relative to their largest diagonal

__constant__ unsigned char c_pair_j[NPAIR], c_pair_l[NPAIR];

__device__ __forceinline__ double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// partial[(s * nch + chunk) * 2 * NPAIR + 2 * pair + (re, im)] = sum over the chunk of conj(u_j) u_l
// for u_0 = b_s, u_k = X_{nbr[s][k-1]} (raw, not delta-scaled).  Pair p is handled by the four
// adjacent threads 4p..4p+3, each over every fourth element of a tile.
__global__ __launch_bounds__(GT) void gram_partial_kernel(const double *B, long long ldb, const float2 *store,
                                                          const int *nbr, long long n, int nch, double *partial) {
  __shared__ double2 u[GUESS_K + 1][GT];
  __shared__ int slot[GUESS_K];
  const int s = blockIdx.y, ch = blockIdx.x, tid = threadIdx.x;
  if (tid < GUESS_K) slot[tid] = nbr[s * GUESS_K + tid];
  __syncthreads();
  const int pair = tid >> 2, q = tid & 3;
  const int pj = pair < NPAIR ? c_pair_j[pair] : 0, pl = pair < NPAIR ? c_pair_l[pair] : 0;
  double2 acc = make_double2(0.0, 0.0);
  const long long e0 = (long long)ch * GCHUNK, e1 = std::min<long long>(n, e0 + GCHUNK);
  const double2 *b = reinterpret_cast<const double2 *>(B) + (long long)s * ldb;
  for (long long t0 = e0; t0 < e1; t0 += GT) {
    const long long i = t0 + tid;
    const bool in = i < e1;
    u[0][tid] = in ? b[i] : make_double2(0.0, 0.0);
#pragma unroll
    for (int k = 0; k < GUESS_K; k++) {
      const int sl = slot[k];
      if (in && sl >= 0) {
        const float2 x = store[(long long)sl * n + i];
        u[k + 1][tid] = make_double2((double)x.x, (double)x.y);
      } else {
        u[k + 1][tid] = make_double2(0.0, 0.0);
      }
    }
    __syncthreads();
    if (pair < NPAIR) {
#pragma unroll 4
      for (int e = q; e < GT; e += 4) {
        const double2 a = u[pj][e], c = u[pl][e];
        acc.x = fma(a.x, c.x, fma(a.y, c.y, acc.x));
        acc.y = fma(a.x, c.y, fma(-a.y, c.x, acc.y));
      }
    }
    __syncthreads();
  }
  acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
  acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
  acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
  acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
  if (pair < NPAIR && q == 0) {
    double *p = partial + ((long long)s * nch + ch) * 2 * NPAIR + 2 * pair;
    p[0] = acc.x;
    p[1] = acc.y;
  }
}

// One block per system: raw pair sums over the chunks, then the delta-scaled Gram matrix (both
// triangles) and the feature vector.
__global__ void gram_final_kernel(const double *partial, int nch, const double *delta, const double *omega,
                                  double eta, const double *pfrac, double *Gm, double *feat) {
  __shared__ double2 raw[NPAIR];
  const int s = blockIdx.x, tid = threadIdx.x;
  if (tid < NPAIR) {
    double2 a = make_double2(0.0, 0.0);
    for (int ch = 0; ch < nch; ch++) {
      const double *p = partial + ((long long)s * nch + ch) * 2 * NPAIR + 2 * tid;
      a.x += p[0];
      a.y += p[1];
    }
    raw[tid] = a;
  }
  __syncthreads();
  const double *d = delta + (long long)s * GUESS_K;
  if (tid < NPAIR) {
    const int j = c_pair_j[tid], l = c_pair_l[tid];
    const double sc = (j == 0 ? 1.0 : d[j - 1]) * (l == 0 ? 1.0 : d[l - 1]);
    double2 *G = reinterpret_cast<double2 *>(Gm) + (long long)s * GUESS_G;
    const double2 v = make_double2(sc * raw[tid].x, sc * raw[tid].y);
    G[j * (GUESS_K + 1) + l] = v;
    G[l * (GUESS_K + 1) + j] = make_double2(v.x, -v.y);
  }
  if (tid == 0) {
    double *f = feat + (long long)s * GUESS_NF;
    const double bb = raw[0].x;
    const double sc = bb > 0.0 ? eta / bb : 0.0;
    f[0] = omega[s];
    f[1] = eta;
    f[2] = pfrac[s];
    for (int k = 0; k < GUESS_K; k++) {
      f[3 + k] = d[k];
      // pair (0, k+1) is pair index k+1 (row 0 of the upper triangle)
      f[3 + GUESS_K + k] = raw[k + 1].x * sc;
      f[3 + 2 * GUESS_K + k] = raw[k + 1].y * sc;
    }
  }
}

// ||(1 - sum c) b - sum c_k delta_k X_k||^2 / ||b||^2 = a^H Gm a / Gm_00 with a = (sum c - 1, c).
__device__ double quad_loss(const double2 *G, const double2 *c) {
  double2 a[GUESS_K + 1];
  double2 sum = make_double2(-1.0, 0.0);
  for (int k = 0; k < GUESS_K; k++) {
    a[k + 1] = c[k];
    sum.x += c[k].x;
    sum.y += c[k].y;
  }
  a[0] = sum;
  double num = 0.0;
  for (int j = 0; j <= GUESS_K; j++) {
    double2 ga = make_double2(0.0, 0.0);
    for (int l = 0; l <= GUESS_K; l++) {
      const double2 t = cmul(G[j * (GUESS_K + 1) + l], a[l]);
      ga.x += t.x;
      ga.y += t.y;
    }
    num += a[j].x * ga.x + a[j].y * ga.y;   // Re(conj(a_j) (G a)_j)
  }
  return num / G[0].x;
}

// Minimiser of the residual over the first K neighbours: (P^T Gm P + lambda I) c = P^T Gm e_0 with
// P = [1^T; I] (columns e_0 + e_k), solved by Gaussian elimination with partial pivoting.
__device__ void minres_coef(const double2 *G, int K, double2 *c) {
  double2 A[GUESS_K][GUESS_K + 1];
  constexpr int W = GUESS_K + 1;
  double dmax = 0.0;
  for (int j = 0; j < K; j++) {
    for (int k = 0; k < K; k++) {
      const double2 g00 = G[0], g0k = G[k + 1], gj0 = G[(j + 1) * W], gjk = G[(j + 1) * W + k + 1];
      A[j][k] = make_double2(g00.x + g0k.x + gj0.x + gjk.x, g00.y + g0k.y + gj0.y + gjk.y);
    }
    const double2 g00 = G[0], gj0 = G[(j + 1) * W];
    A[j][K] = make_double2(g00.x + gj0.x, g00.y + gj0.y);
    dmax = fmax(dmax, A[j][j].x);
  }
  const double lam = MINRES_REG * dmax;
  for (int j = 0; j < K; j++) A[j][j].x += lam;
  for (int col = 0; col < K; col++) {
    int piv = col;
    double best = A[col][col].x * A[col][col].x + A[col][col].y * A[col][col].y;
    for (int r = col + 1; r < K; r++) {
      const double m2 = A[r][col].x * A[r][col].x + A[r][col].y * A[r][col].y;
      if (m2 > best) {
        best = m2;
        piv = r;
      }
    }
    if (!(best > 0.0)) {
      for (int k = 0; k < GUESS_K; k++) c[k] = make_double2(0.0, 0.0);
      return;
    }
    if (piv != col)
      for (int k = col; k <= K; k++) {
        const double2 t = A[col][k];
        A[col][k] = A[piv][k];
        A[piv][k] = t;
      }
    const double2 p = A[col][col];
    const double2 pinv = make_double2(p.x / best, -p.y / best);
    for (int r = col + 1; r < K; r++) {
      const double2 f = cmul(A[r][col], pinv);
      for (int k = col; k <= K; k++) {
        const double2 t = cmul(f, A[col][k]);
        A[r][k].x -= t.x;
        A[r][k].y -= t.y;
      }
    }
  }
  for (int k = 0; k < GUESS_K; k++) c[k] = make_double2(0.0, 0.0);
  for (int r = K - 1; r >= 0; r--) {
    double2 acc = A[r][K];
    for (int k = r + 1; k < K; k++) {
      const double2 t = cmul(A[r][k], c[k]);
      acc.x -= t.x;
      acc.y -= t.y;
    }
    const double2 p = A[r][r];
    const double m2 = p.x * p.x + p.y * p.y;
    c[r] = cmul(acc, make_double2(p.x / m2, -p.y / m2));
  }
}

__global__ void choose_kernel(int nsys, int mode, const double *Gm, const double *y, const int *navail, double *coef,
                              double *pred, int *kind) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsys) return;
  const double2 *G = reinterpret_cast<const double2 *>(Gm) + (long long)s * GUESS_G;
  double2 c[GUESS_K];
  for (int k = 0; k < GUESS_K; k++) c[k] = make_double2(0.0, 0.0);
  const int K = navail[s];
  bool ok = G[0].x > 0.0;
  if (mode == GFCC_GUESS_LEARNED) {
    ok = ok && K == GUESS_K;
    if (ok)
      for (int k = 0; k < GUESS_K; k++) c[k] = make_double2(y[(long long)s * GUESS_NO + 2 * k], y[(long long)s * GUESS_NO + 2 * k + 1]);
  } else {
    ok = ok && K >= 1;
    if (ok) minres_coef(G, K, c);
  }
  double loss = 1.0;
  if (ok) {
    loss = quad_loss(G, c);
    ok = loss < 1.0;   // no worse than the zero guess (||r(x0)|| < ||b||)
  }
  double2 *co = reinterpret_cast<double2 *>(coef) + (long long)s * GUESS_K;
  for (int k = 0; k < GUESS_K; k++) co[k] = ok ? c[k] : make_double2(0.0, 0.0);
  pred[s] = ok ? fmax(loss, 0.0) : 1.0;
  kind[s] = ok ? mode : GFCC_GUESS_ZERO;
}

__global__ void losses_kernel(int nsys, const double *Gm, const double *y, double *loss_model, double *loss_minres) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsys) return;
  const double2 *G = reinterpret_cast<const double2 *>(Gm) + (long long)s * GUESS_G;
  double2 c[GUESS_K];
  if (!(G[0].x > 0.0)) {
    loss_model[s] = 0.0;
    loss_minres[s] = 0.0;
    return;
  }
  for (int k = 0; k < GUESS_K; k++) c[k] = make_double2(y[(long long)s * GUESS_NO + 2 * k], y[(long long)s * GUESS_NO + 2 * k + 1]);
  loss_model[s] = quad_loss(G, c);
  minres_coef(G, GUESS_K, c);
  loss_minres[s] = quad_loss(G, c);
}

__global__ void combine_kernel(int nsys, long long n, const float2 *store, const int *nbr, const double *coef,
                               const int *kind, double *X0, long long ldx) {
  const long long tot = n * nsys;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(t / n);
    const long long i = t - (long long)s * n;
    double2 acc = make_double2(0.0, 0.0);
    if (kind[s] != GFCC_GUESS_ZERO) {
      const double2 *co = reinterpret_cast<const double2 *>(coef) + (long long)s * GUESS_K;
#pragma unroll
      for (int k = 0; k < GUESS_K; k++) {
        const int sl = nbr[s * GUESS_K + k];
        if (sl < 0) continue;
        const float2 x = store[(long long)sl * n + i];
        const double2 c = co[k];
        acc.x += c.x * (double)x.x - c.y * (double)x.y;
        acc.y += c.x * (double)x.y + c.y * (double)x.x;
      }
    }
    reinterpret_cast<double2 *>(X0)[(long long)s * ldx + i] = acc;
  }
}

__global__ void store_put_kernel(int nsys, long long n, const double *U, long long ldu, const int *slot,
                                 float2 *store) {
  const long long tot = n * nsys;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(t / n);
    const long long i = t - (long long)s * n;
    const int sl = slot[s];
    if (sl < 0) continue;
    const double2 u = reinterpret_cast<const double2 *>(U)[(long long)s * ldu + i];
    store[(long long)sl * n + i] = make_float2((float)u.x, (float)u.y);
  }
}

int upload_pairs() {
  static bool done[128] = {false};
  int dev = 0;
  GFCC_CUDA(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 128 && done[dev]) return GFCC_OK;
  unsigned char j[NPAIR], l[NPAIR];
  int p = 0;
  // row-major upper triangle: (0,0), (0,1), ..., (0,8), (1,1), ...; pair k+1 is (0, k+1)
  for (int a = 0; a <= GUESS_K; a++)
    for (int b = a; b <= GUESS_K; b++) {
      j[p] = (unsigned char)a;
      l[p] = (unsigned char)b;
      p++;
    }
  GFCC_CUDA(cudaMemcpyToSymbol(c_pair_j, j, sizeof(j)));
  GFCC_CUDA(cudaMemcpyToSymbol(c_pair_l, l, sizeof(l)));
  if (dev >= 0 && dev < 128) done[dev] = true;
  return GFCC_OK;
}

}  // namespace

long long guess_gram_work_doubles(int nsys, long long n) {
  return (long long)nsys * cdiv(std::max<long long>(n, 1), GCHUNK) * 2 * NPAIR;
}

int guess_gram(cudaStream_t st, int nsys, long long n, const double *B, long long ldb, const float2 *store,
               const int *nbr, const double *delta, const double *omega, double eta, const double *pfrac, double *Gm,
               double *feat, double *work) {
  if (nsys <= 0) return GFCC_OK;
  GFCC_TRY(upload_pairs());
  const int nch = (int)cdiv(std::max<long long>(n, 1), GCHUNK);
  gram_partial_kernel<<<dim3(nch, nsys), GT, 0, st>>>(B, ldb, store, nbr, n, nch, work);
  GFCC_LAUNCH_CHECK();
  gram_final_kernel<<<nsys, 64, 0, st>>>(work, nch, delta, omega, eta, pfrac, Gm, feat);
  GFCC_LAUNCH_CHECK();
  return GFCC_OK;
}

int guess_choose(cudaStream_t st, int nsys, int mode, const double *Gm, const double *y, const int *navail,
                 double *coef, double *pred, int *kind) {
  if (nsys <= 0) return GFCC_OK;
  choose_kernel<<<cdiv(nsys, 64), 64, 0, st>>>(nsys, mode, Gm, y, navail, coef, pred, kind);
  GFCC_LAUNCH_CHECK();
  return GFCC_OK;
}

int guess_losses(cudaStream_t st, int nsys, const double *Gm, const double *y, double *loss_model,
                 double *loss_minres) {
  if (nsys <= 0) return GFCC_OK;
  losses_kernel<<<cdiv(nsys, 64), 64, 0, st>>>(nsys, Gm, y, loss_model, loss_minres);
  GFCC_LAUNCH_CHECK();
  return GFCC_OK;
}

int guess_combine(cudaStream_t st, int nsys, long long n, const float2 *store, const int *nbr, const double *coef,
                  const int *kind, double *X0, long long ldx) {
  if (nsys <= 0 || n <= 0) return GFCC_OK;
  combine_kernel<<<grid1d(n * nsys), 256, 0, st>>>(nsys, n, store, nbr, coef, kind, X0, ldx);
  GFCC_LAUNCH_CHECK();
  return GFCC_OK;
}

int guess_store_put(cudaStream_t st, int nsys, long long n, const double *U, long long ldu, const int *slot,
                    float2 *store) {
  if (nsys <= 0 || n <= 0) return GFCC_OK;
  store_put_kernel<<<grid1d(n * nsys), 256, 0, st>>>(nsys, n, U, ldu, slot, store);
  GFCC_LAUNCH_CHECK();
  return GFCC_OK;
}

std::vector<int> guess_frequency_order(const std::vector<double> &omega) {
  const int nw = (int)omega.size();
  std::vector<int> order;
  if (nw == 0) return order;
  std::vector<char> taken(nw, 0);
  std::vector<double> dist(nw, INFINITY);
  auto take = [&](int w) {
    order.push_back(w);
    taken[w] = 1;
    for (int j = 0; j < nw; j++) dist[j] = std::min(dist[j], std::fabs(omega[j] - omega[w]));
  };
  int lo = 0, hi = 0;
  for (int w = 1; w < nw; w++) {
    if (omega[w] < omega[lo]) lo = w;
    if (omega[w] > omega[hi]) hi = w;
  }
  take(lo);
  if (hi != lo) take(hi);
  while ((int)order.size() < nw) {
    int best = -1;
    for (int j = 0; j < nw; j++)
      if (!taken[j] && (best < 0 || dist[j] > dist[best])) best = j;
    take(best);
  }
  return order;
}

int guess_neighbours(const std::vector<double> &omega, const char *done, long long done_stride, int w, int k,
                     int *out) {
  const int nw = (int)omega.size();
  int cnt = 0;
  // insertion into a sorted list of at most k candidates
  std::vector<int> best;
  for (int j = 0; j < nw; j++) {
    if (j == w || !done[(long long)j * done_stride]) continue;
    const double dj = std::fabs(omega[j] - omega[w]);
    int pos = (int)best.size();
    while (pos > 0 && std::fabs(omega[best[pos - 1]] - omega[w]) > dj) pos--;
    if (pos >= k) continue;
    best.insert(best.begin() + pos, j);
    if ((int)best.size() > k) best.pop_back();
  }
  cnt = (int)best.size();
  for (int i = 0; i < cnt; i++) out[i] = best[i];
  return cnt;
}

}  // namespace gfcc
