// Model-order reduction of the GFCCSD linear systems (Theory section, eq. model; Algorithm 1: the
// Gram-Schmidt, projection and spectral-function steps after the frequency loop of a level), and the
// adaptive frequency levels of the Implementation Details section (eq. Lmax).
//
// A gfcc_mor object holds, for one sector of a context, a real orthonormal subspace S = {v_1 .. v_m}
// of the packed space (the columns of S are stored as rows v_k[mu]), W = Hbar_N S (the sigma product
// of every basis vector) and the projected operator Hhat = S^T Hbar_N S (m x m, real).  Hbar, the
// right-hand sides and the left vectors are real, so S is spanned by the real and imaginary parts of
// the complex solutions X_p(omega_k); its complex span contains every sampled solution, and the model
//     IP: (omega - i eta + Hhat) Xhat = S^T b_p,   G_pq = (S^T c_q)^T Xhat
//     EA: (omega + i eta - Hhat) Yhat = S^T b_q,   G_pq = (S^T c_p)^T Yhat
// reproduces the full G at every sampled frequency.
//
// Gram-Schmidt: every new real vector is orthogonalised against the basis by two classical passes
// (batched dots, then one update; HBM-bound streams of the basis) and kept when the norm that remains
// exceeds drop_tol times its norm before.  Projection: the new basis vectors are paired as the real and
// imaginary planes of complex vectors and sent through the context's sigma product (FP64, or the
// FP64-accurate digit-plane product in mixed-precision contexts), Hhat = S W^T by an FP64 contraction.
// Model solves: one CTA per frequency builds z I +/- Hhat in global memory and runs Gaussian
// elimination with partial pivoting on it for all right-hand sides at once (O(N_omega m^3), the cost
// the paper states for this step).  The model residual b - A(omega) S Xhat = b - z S Xhat -/+ W Xhat
// of a model solution needs no sigma product (the driver's error indicator).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ctx.cuh"
#include "kernels.cuh"
#include "sigma.cuh"

struct gfcc_mor {
  gfcc_ctx *c = nullptr;
  int sector = GFCC_SECTOR_IP;
  long long n = 0;
  int m = 0, cap = 0;
  double drop_tol = 1e-10;
  double *S = nullptr;   // [cap][n]
  double *W = nullptr;   // [cap][n]
  double *H = nullptr;   // [cap][cap], H[i][j] = v_i . W_j
  double *work = nullptr;
  size_t work_bytes = 0;
  std::vector<double> sampled;   // frequencies whose solutions entered the subspace
};

namespace gfcc {

int solve_for_sink(gfcc_ctx *c, int sector, int n_omega, const double *h_om, double eta, int n_orb,
                   const int *h_orb, double tol, double *d_sink, double *h_G);
int build_left_vectors(gfcc_ctx *c, int sector, int nq, const int *d_orb, double *C, cudaStream_t st);
int build_rhs(gfcc_ctx *c, int sector, int nsys, const int *d_porb, double *B, cudaStream_t st);

namespace {

constexpr int MT = 256;

// dots[k][chunk] = sum_{mu in chunk} S[k][mu] v[mu] for k < m; dots[m][chunk] = ||v||^2 over the chunk.
// grid (nchunk, m + 1)
constexpr int MOR_CHUNK = 8192;
__global__ void mor_dots_kernel(const double *S, long long n, int m, const double *v, int nchunk, double *part) {
  __shared__ double sh[MT / 32];
  const int k = blockIdx.y, ch = blockIdx.x;
  const double *a = k < m ? S + (long long)k * n : v;
  const long long e0 = (long long)ch * MOR_CHUNK, e1 = min(n, e0 + MOR_CHUNK);
  double acc = 0.0;
  for (long long e = e0 + threadIdx.x; e < e1; e += MT) acc += a[e] * v[e];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < MT / 32; w++) t += sh[w];
    part[(long long)k * nchunk + ch] = t;
  }
}

// out[k] = sum_chunk part[k][chunk], k <= m (one warp per k)
__global__ void mor_dots_final_kernel(const double *part, int m1, int nchunk, double *out) {
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (k >= m1) return;
  double acc = 0.0;
  for (int c = lane; c < nchunk; c += 32) acc += part[(long long)k * nchunk + c];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) out[k] = acc;
}

// v -= sum_{k<m} h[k] S[k]
__global__ void mor_update_kernel(const double *S, long long n, int m, const double *h, double *v) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int k = 0; k < m; k++) acc += h[k] * S[(long long)k * n + e];
    v[e] -= acc;
  }
}

// dst = src * scale[0] (scale = 1 / ||v||, from the device)
__global__ void mor_scale_kernel(const double *src, long long n, const double *nrm2, double *dst) {
  const double inv = 1.0 / sqrt(nrm2[0]);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    dst[e] = src[e] * inv;
}

// real plane p (0 re, 1 im) of complex vector x [n] -> v [n]
__global__ void mor_plane_kernel(const double *x, long long n, int p, double *v) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    v[e] = x[2 * e + p];
}

// complex vectors [np][n] from pairs of real rows: z_s = S[k0 + 2s] + i S[k0 + 2s + 1] (the imaginary
// plane zero past k1)
__global__ void mor_pack_kernel(const double *S, long long n, int k0, int k1, int np, double *z) {
  const long long tot = (long long)np * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(t / n);
    const long long e = t - (long long)s * n;
    const int kr = k0 + 2 * s, ki = kr + 1;
    z[2 * t] = S[(long long)kr * n + e];
    z[2 * t + 1] = ki < k1 ? S[(long long)ki * n + e] : 0.0;
  }
}

// W rows from the complex sigma products: W[k0 + 2s] = Re y_s, W[k0 + 2s + 1] = Im y_s (below k1)
__global__ void mor_unpack_kernel(const double *y, long long n, int k0, int k1, int np, double *W) {
  const long long tot = (long long)np * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(t / n);
    const long long e = t - (long long)s * n;
    const int kr = k0 + 2 * s, ki = kr + 1;
    W[(long long)kr * n + e] = y[2 * t];
    if (ki < k1) W[(long long)ki * n + e] = y[2 * t + 1];
  }
}

// real parts of complex vectors: out[r][mu] = Re z[r][mu]
__global__ void mor_real_kernel(const double *z, long long n, int rows, double *out) {
  const long long tot = (long long)rows * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x)
    out[t] = z[2 * t];
}

// Model solves: one CTA per frequency w.  A = z_w I + s Hhat (complex, m x m, row-major in work
// [w][m][m]), right-hand sides bh [m][nb] (real), solution X [w][m][nb] complex; then
// G[w][a][b] (IP: a over rhs, b over left; EA: a over left, b over rhs) = sum_k ch[k][left] X[k][rhs].
// Gaussian elimination with partial pivoting by rows; threads split the trailing updates.
__global__ __launch_bounds__(MT) void mor_model_solve_kernel(const double *Hh, int m, const double *omegas, double eta,
                                                             double zsign, double hsign, const double *bh, int nb,
                                                             const double *ch, int nl, int is_ip, double2 *Aw,
                                                             double2 *Xw, double *G) {
  __shared__ int piv;
  __shared__ double pval[MT];
  __shared__ int pidx[MT];
  const int w = blockIdx.x;
  double2 *A = Aw + (long long)w * m * m;
  double2 *X = Xw + (long long)w * m * nb;
  const double om = omegas[w];
  for (long long t = threadIdx.x; t < (long long)m * m; t += MT) {
    const int i = (int)(t / m), j = (int)(t % m);
    A[t] = make_double2(hsign * Hh[t] + (i == j ? om : 0.0), i == j ? zsign * eta : 0.0);
  }
  for (long long t = threadIdx.x; t < (long long)m * nb; t += MT) X[t] = make_double2(bh[t], 0.0);
  __syncthreads();
  for (int k = 0; k < m; k++) {
    // pivot: largest |A[i][k]| over i >= k
    double best = -1.0;
    int bi = k;
    for (int i = k + threadIdx.x; i < m; i += MT) {
      const double2 a = A[(long long)i * m + k];
      const double mag = a.x * a.x + a.y * a.y;
      if (mag > best) {
        best = mag;
        bi = i;
      }
    }
    pval[threadIdx.x] = best;
    pidx[threadIdx.x] = bi;
    __syncthreads();
    if (threadIdx.x == 0) {
      double b = -1.0;
      int idx = k;
      for (int t = 0; t < MT; t++)
        if (pval[t] > b) {
          b = pval[t];
          idx = pidx[t];
        }
      piv = idx;
    }
    __syncthreads();
    const int p = piv;
    if (p != k) {
      for (int j = threadIdx.x; j < m; j += MT) {
        const double2 t = A[(long long)k * m + j];
        A[(long long)k * m + j] = A[(long long)p * m + j];
        A[(long long)p * m + j] = t;
      }
      for (int j = threadIdx.x; j < nb; j += MT) {
        const double2 t = X[(long long)k * nb + j];
        X[(long long)k * nb + j] = X[(long long)p * nb + j];
        X[(long long)p * nb + j] = t;
      }
    }
    __syncthreads();
    const double2 d = A[(long long)k * m + k];
    const double dd = d.x * d.x + d.y * d.y;
    const double2 inv = dd > 0.0 ? make_double2(d.x / dd, -d.y / dd) : make_double2(0.0, 0.0);
    // eliminate below: row i -= l_i row k, l_i = A[i][k] / A[k][k] (columns > k and the right-hand sides)
    const int rows = m - k - 1, cols = m - k - 1 + nb;
    for (long long t = threadIdx.x; t < (long long)rows * cols; t += MT) {
      const int i = k + 1 + (int)(t / cols), jj = (int)(t % cols);
      const double2 a = A[(long long)i * m + k];
      const double2 l = make_double2(a.x * inv.x - a.y * inv.y, a.x * inv.y + a.y * inv.x);
      double2 *dst;
      double2 src;
      if (jj < m - k - 1) {
        dst = &A[(long long)i * m + k + 1 + jj];
        src = A[(long long)k * m + k + 1 + jj];
      } else {
        dst = &X[(long long)i * nb + (jj - (m - k - 1))];
        src = X[(long long)k * nb + (jj - (m - k - 1))];
      }
      double2 v = *dst;
      v.x -= l.x * src.x - l.y * src.y;
      v.y -= l.x * src.y + l.y * src.x;
      *dst = v;
    }
    __syncthreads();
  }
  // back substitution, one right-hand side per thread
  for (int r = threadIdx.x; r < nb; r += MT) {
    for (int i = m - 1; i >= 0; i--) {
      double2 acc = X[(long long)i * nb + r];
      for (int j = i + 1; j < m; j++) {
        const double2 a = A[(long long)i * m + j], x = X[(long long)j * nb + r];
        acc.x -= a.x * x.x - a.y * x.y;
        acc.y -= a.x * x.y + a.y * x.x;
      }
      const double2 d = A[(long long)i * m + i];
      const double dd = d.x * d.x + d.y * d.y;
      X[(long long)i * nb + r] =
          dd > 0.0 ? make_double2((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd)
                   : make_double2(0.0, 0.0);
    }
  }
  __syncthreads();
  if (G == nullptr) return;
  for (int t = threadIdx.x; t < nb * nl; t += MT) {
    const int r = t / nl, q = t % nl;   // rhs r, left q
    double gr = 0.0, gi = 0.0;
    for (int k = 0; k < m; k++) {
      const double cq = ch[(long long)k * nl + q];
      const double2 x = X[(long long)k * nb + r];
      gr += cq * x.x;
      gi += cq * x.y;
    }
    const long long idx = is_ip ? ((long long)w * nb + r) * nl + q : ((long long)w * nl + q) * nb + r;
    G[2 * idx] = gr;
    G[2 * idx + 1] = gi;
  }
}

// Model residuals: for the nr (frequency, rhs) pairs of a block of frequencies, r = b - z S^T xh -/+ W^T xh,
// out[2 r] += ||r||^2 over this block of mu, out[2 r + 1] += ||b||^2.  xh = X[w][k][rhs] complex.
// grid (cdiv(n, MT), nw * nb) -- one (frequency, rhs) pair per blockIdx.y.
__global__ __launch_bounds__(MT) void mor_residual_kernel(const double *S, const double *W, long long n, int m,
                                                          const double2 *Xw, int nb, const double *omegas, double eta,
                                                          double zsign, double wsign, const double *B, double *out) {
  __shared__ double2 xs[1024];
  __shared__ double sh[2][MT / 32];
  const int pr = blockIdx.y, w = pr / nb, r = pr % nb;
  for (int k = threadIdx.x; k < m; k += MT) xs[k] = Xw[((long long)w * m + k) * nb + r];
  __syncthreads();
  const long long e = (long long)blockIdx.x * MT + threadIdx.x;
  double rr = 0.0, bb = 0.0;
  if (e < n) {
    double sr = 0.0, si = 0.0, wr = 0.0, wi = 0.0;
    for (int k = 0; k < m; k++) {
      const double s = S[(long long)k * n + e], q = W[(long long)k * n + e];
      sr += s * xs[k].x;
      si += s * xs[k].y;
      wr += q * xs[k].x;
      wi += q * xs[k].y;
    }
    const double zr = omegas[w], zi = zsign * eta;
    const double b = B[(long long)r * n + e];
    const double ar = zr * sr - zi * si + wsign * wr, ai = zr * si + zi * sr + wsign * wi;
    rr = (b - ar) * (b - ar) + ai * ai;
    bb = b * b;
  }
  for (int off = 16; off > 0; off >>= 1) {
    rr += __shfl_xor_sync(0xffffffffu, rr, off);
    bb += __shfl_xor_sync(0xffffffffu, bb, off);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = rr;
    sh[1][threadIdx.x >> 5] = bb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int t = 0; t < MT / 32; t++) {
      a += sh[0][t];
      c += sh[1][t];
    }
    atomicAdd(&out[2 * pr], a);
    atomicAdd(&out[2 * pr + 1], c);
  }
}

int grow(gfcc_mor *M, size_t bytes) {
  if (M->work_bytes >= bytes) return GFCC_OK;
  if (M->work) dfree(M->work);
  M->work = nullptr;
  M->work_bytes = 0;
  if (dmalloc(reinterpret_cast<void **>(&M->work), bytes) != cudaSuccess) {
    cudaGetLastError();
    set_error("model-order reduction: cannot allocate %.3f GB of workspace", bytes / 1e9);
    return GFCC_ERR_OOM;
  }
  M->work_bytes = bytes;
  return GFCC_OK;
}

int ensure_cap(gfcc_mor *M, int need) {
  if (need <= M->cap) return GFCC_OK;
  const int cap = std::max(need, std::max(64, 2 * M->cap));
  double *S = nullptr, *W = nullptr, *H = nullptr;
  const size_t vb = sizeof(double) * (size_t)cap * (size_t)M->n;
  if (dmalloc(reinterpret_cast<void **>(&S), vb) != cudaSuccess ||
      dmalloc(reinterpret_cast<void **>(&W), vb) != cudaSuccess ||
      dmalloc(reinterpret_cast<void **>(&H), sizeof(double) * (size_t)cap * cap) != cudaSuccess) {
    cudaGetLastError();
    dfree(S);
    dfree(W);
    dfree(H);
    set_error("model-order reduction: cannot allocate a subspace of %d vectors (%.3f GB)", cap, 2.0 * vb / 1e9);
    return GFCC_ERR_OOM;
  }
  cudaStream_t st = M->c->stream;
  if (M->m > 0) {
    GFCC_CUDA(cudaMemcpyAsync(S, M->S, sizeof(double) * (size_t)M->m * M->n, cudaMemcpyDeviceToDevice, st));
    GFCC_CUDA(cudaMemcpyAsync(W, M->W, sizeof(double) * (size_t)M->m * M->n, cudaMemcpyDeviceToDevice, st));
    GFCC_CUDA(cudaMemcpy2DAsync(H, sizeof(double) * cap, M->H, sizeof(double) * M->cap, sizeof(double) * M->m, M->m,
                                cudaMemcpyDeviceToDevice, st));
    GFCC_CUDA(cudaStreamSynchronize(st));
  }
  dfree(M->S);
  dfree(M->W);
  dfree(M->H);
  M->S = S;
  M->W = W;
  M->H = H;
  M->cap = cap;
  return GFCC_OK;
}

// Gram-Schmidt of one real vector v (device, n) against the basis; appended when it survives.
int gs_append(gfcc_mor *M, double *v, double *part, double *h, bool &added) {
  cudaStream_t st = M->c->stream;
  const long long n = M->n;
  const int nchunk = (int)((n + MOR_CHUNK - 1) / MOR_CHUNK);
  double nrm0 = 0.0;
  added = false;
  for (int pass = 0; pass < 2; pass++) {
    mor_dots_kernel<<<dim3(nchunk, M->m + 1), MT, 0, st>>>(M->S, n, M->m, v, nchunk, part);
    GFCC_LAUNCH_CHECK();
    mor_dots_final_kernel<<<cdiv((long long)(M->m + 1) * 32, MT), MT, 0, st>>>(part, M->m + 1, nchunk, h);
    GFCC_LAUNCH_CHECK();
    if (pass == 0) {
      GFCC_CUDA(cudaMemcpyAsync(&nrm0, h + M->m, sizeof(double), cudaMemcpyDeviceToHost, st));
      GFCC_CUDA(cudaStreamSynchronize(st));
      if (!(nrm0 > 0.0)) return GFCC_OK;
    }
    if (M->m > 0) {
      mor_update_kernel<<<grid1d(n), MT, 0, st>>>(M->S, n, M->m, h, v);
      GFCC_LAUNCH_CHECK();
    }
  }
  // remaining norm
  mor_dots_kernel<<<dim3(nchunk, 1), MT, 0, st>>>(M->S, n, 0, v, nchunk, part);
  GFCC_LAUNCH_CHECK();
  mor_dots_final_kernel<<<1, MT, 0, st>>>(part, 1, nchunk, h);
  GFCC_LAUNCH_CHECK();
  double nrm = 0.0;
  GFCC_CUDA(cudaMemcpyAsync(&nrm, h, sizeof(double), cudaMemcpyDeviceToHost, st));
  GFCC_CUDA(cudaStreamSynchronize(st));
  if (!(nrm > M->drop_tol * M->drop_tol * nrm0)) return GFCC_OK;
  GFCC_TRY(ensure_cap(M, M->m + 1));
  mor_scale_kernel<<<grid1d(n), MT, 0, st>>>(v, n, h, M->S + (long long)M->m * n);
  GFCC_LAUNCH_CHECK();
  M->m++;
  added = true;
  return GFCC_OK;
}

// W rows [k0, k1) = sigma(S rows [k0, k1)), then Hhat = S W^T over the whole basis
int project_new(gfcc_mor *M, int k0) {
  gfcc_ctx *c = M->c;
  cudaStream_t st = c->stream;
  const long long n = M->n;
  const bool ip = M->sector == GFCC_SECTOR_IP;
  const bool emu = (ip ? c->eWr.dig : c->eWre.dig) != nullptr;
  const int k1 = M->m;
  const int pairs = (k1 - k0 + 1) / 2;
  const int chunk = std::max(1, std::min(pairs, emu ? 16 : 8));   // complex vectors per sigma call
  const long long sw = sigma_work_doubles(c, M->sector, chunk);
  const long long ew = emu ? sigma_emu_work_doubles(c, chunk) : 0;
  const size_t bytes = sizeof(double) * (size_t)(4LL * chunk * n + sw + ew + 64);
  GFCC_TRY(grow(M, bytes));
  double *z = M->work, *y = z + 2LL * chunk * n, *w = y + 2LL * chunk * n;
  for (int p0 = 0; p0 < pairs; p0 += chunk) {
    const int np = std::min(chunk, pairs - p0);
    const int ka = k0 + 2 * p0;
    const int kb = std::min(k1, ka + 2 * np);
    mor_pack_kernel<<<grid1d(np * n), MT, 0, st>>>(M->S, n, ka, kb, np, z);
    GFCC_LAUNCH_CHECK();
    SysBatch b;
    b.nsys = np;
    b.x = z;
    b.ldx = n;
    b.y = y;
    b.ldy = n;
    b.dsign = ip ? 1.0 : -1.0;
    b.zsign = ip ? -1.0 : 1.0;
    if (emu)
      GFCC_TRY(ip ? apply_ip_emu(c, b, w, ew) : apply_ea_emu(c, b, w, ew));
    else
      GFCC_TRY(ip ? apply_ip(c, b, w) : apply_ea(c, b, w));
    mor_unpack_kernel<<<grid1d(np * n), MT, 0, st>>>(y, n, ka, kb, np, M->W);
    GFCC_LAUNCH_CHECK();
  }
  // Hhat[i][j] = sum_mu S[i][mu] W[j][mu]  (row stride cap)
  GFCC_TRY(gemm_f64(st, k1, k1, n, 1.0, M->S, imap1(n), imap1(1), M->W, imap1(1), imap1(n), 0.0, M->H,
                    imap1(M->cap), imap1(1)));
  return GFCC_OK;
}

}  // namespace

// Model Green's function on a frequency grid (the sector of the object): rows / columns as gfcc_solve_block.
int mor_green_impl(gfcc_mor *M, int n_omega, const double *h_om, double eta, int nP, const int *h_P, int nQ,
                   const int *h_Q, double *h_G, double *h_relres) {
  gfcc_ctx *c = M->c;
  cudaStream_t st = c->stream;
  const long long n = M->n;
  const int m = M->m;
  const bool ip = M->sector == GFCC_SECTOR_IP;
  if (m < 1) {
    set_error("gfcc_mor_green: the subspace is empty (gfcc_mor_expand first)");
    return GFCC_ERR_STATE;
  }
  if (m > 1024 && h_relres != nullptr) {
    set_error("gfcc_mor_green: model residuals need m <= 1024 (m = %d)", m);
    return GFCC_ERR_ARG;
  }
  const int nb = ip ? nP : nQ, nl = ip ? nQ : nP;   // right-hand sides, left vectors
  const int *h_b = ip ? h_P : h_Q, *h_l = ip ? h_Q : h_P;
  // host lists -> device, right-hand sides (complex, real part only) and left vectors
  int *d_lists = nullptr;
  double *buf = nullptr;
  // frequencies per model launch: their dense model matrices and solutions within about 4 GB
  const long long per_w = 16LL * m * (m + nb);
  const long long wb = std::max<long long>(1, std::min<long long>({(long long)n_omega, 256LL, (4LL << 30) / per_w}));
  const size_t need = sizeof(double) * (size_t)(2LL * nb * n + (long long)nb * n + (long long)nl * n +
                                                (long long)m * (nb + nl) + 2LL * wb * m * m + 2LL * wb * m * nb +
                                                2LL * n_omega * nb * nl + n_omega + 2LL * wb * nb + 64);
  GFCC_TRY(grow(M, need));
  if (dmalloc(reinterpret_cast<void **>(&d_lists), sizeof(int) * (nb + nl) + 16) != cudaSuccess) {
    cudaGetLastError();
    set_error("gfcc_mor_green: allocation failed");
    return GFCC_ERR_OOM;
  }
  buf = M->work;
  double *Bc = buf;                          // [nb][n] complex
  double *Br = Bc + 2LL * nb * n;            // [nb][n] real
  double *Cl = Br + (long long)nb * n;       // [nl][n]
  double *bh = Cl + (long long)nl * n;       // [m][nb]
  double *ch = bh + (long long)m * nb;       // [m][nl]
  double2 *Aw = reinterpret_cast<double2 *>(ch + (long long)m * nl);
  double2 *Xw = Aw + wb * m * m;
  double *Gd = reinterpret_cast<double *>(Xw + wb * m * nb);
  double *om = Gd + 2LL * n_omega * nb * nl;
  double *res = om + n_omega;
  int s = GFCC_OK;
  auto done = [&](int code) {
    dfree(d_lists);
    return code;
  };
  if (cudaMemcpyAsync(d_lists, h_b, sizeof(int) * nb, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(d_lists + nb, h_l, sizeof(int) * nl, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(om, h_om, sizeof(double) * n_omega, cudaMemcpyHostToDevice, st) != cudaSuccess) {
    set_error("gfcc_mor_green: host-to-device copy failed");
    return done(GFCC_ERR_CUDA);
  }
  if ((s = build_rhs(c, M->sector, nb, d_lists, Bc, st)) < 0) return done(s);
  mor_real_kernel<<<grid1d((long long)nb * n), MT, 0, st>>>(Bc, n, nb, Br);
  GFCC_LAUNCH_CHECK();
  if ((s = build_left_vectors(c, M->sector, nl, d_lists + nb, Cl, st)) < 0) return done(s);
  // bh[k][r] = S_k . b_r, ch[k][q] = S_k . c_q
  if ((s = gemm_f64(st, m, nb, n, 1.0, M->S, imap1(n), imap1(1), Br, imap1(1), imap1(n), 0.0, bh, imap1(nb),
                    imap1(1))) < 0)
    return done(s);
  if ((s = gemm_f64(st, m, nl, n, 1.0, M->S, imap1(n), imap1(1), Cl, imap1(1), imap1(n), 0.0, ch, imap1(nl),
                    imap1(1))) < 0)
    return done(s);
  // Hhat packed with row stride m for the model kernel
  double *Hm = nullptr;
  if (dmalloc(reinterpret_cast<void **>(&Hm), sizeof(double) * (size_t)m * m) != cudaSuccess) {
    cudaGetLastError();
    set_error("gfcc_mor_green: allocation failed");
    return done(GFCC_ERR_OOM);
  }
  if (cudaMemcpy2DAsync(Hm, sizeof(double) * m, M->H, sizeof(double) * M->cap, sizeof(double) * m, m,
                        cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
    dfree(Hm);
    set_error("gfcc_mor_green: copy failed");
    return done(GFCC_ERR_CUDA);
  }
  const double zsign = ip ? -1.0 : 1.0, hsign = ip ? 1.0 : -1.0;
  std::vector<double> hres(2 * wb * nb);
  for (int w0 = 0; w0 < n_omega; w0 += (int)wb) {
    const int nw = std::min<int>((int)wb, n_omega - w0);
    mor_model_solve_kernel<<<nw, MT, 0, st>>>(Hm, m, om + w0, eta, zsign, hsign, bh, nb, ch, nl, ip ? 1 : 0, Aw, Xw,
                                              Gd + 2LL * w0 * nb * nl);
    GFCC_LAUNCH_CHECK();
    if (h_relres) {
      GFCC_CUDA(cudaMemsetAsync(res, 0, sizeof(double) * 2 * nw * nb, st));
      mor_residual_kernel<<<dim3(cdiv(n, MT), (unsigned)(nw * nb)), MT, 0, st>>>(
          M->S, M->W, n, m, Xw, nb, om + w0, eta, zsign, ip ? 1.0 : -1.0, Br, res);
      GFCC_LAUNCH_CHECK();
      GFCC_CUDA(cudaMemcpyAsync(hres.data(), res, sizeof(double) * 2 * nw * nb, cudaMemcpyDeviceToHost, st));
      GFCC_CUDA(cudaStreamSynchronize(st));
      for (int t = 0; t < nw * nb; t++)
        h_relres[(long long)w0 * nb + t] = hres[2 * t + 1] > 0.0 ? std::sqrt(hres[2 * t] / hres[2 * t + 1]) : 0.0;
    }
  }
  dfree(Hm);
  if (h_G) {
    GFCC_CUDA(cudaMemcpyAsync(h_G, Gd, sizeof(double) * 2 * n_omega * nb * nl, cudaMemcpyDeviceToHost, st));
  }
  GFCC_CUDA(cudaStreamSynchronize(st));
  return done(GFCC_OK);
}

int mor_expand_impl(gfcc_mor *M, int n_omega, const double *h_om, double eta, int n_orb, const int *h_orb, double tol,
                    double *h_G) {
  gfcc_ctx *c = M->c;
  cudaStream_t st = c->stream;
  const long long n = M->n;
  const long long ntasks = (long long)n_omega * n_orb;
  // solutions of the full systems (the hot path), then Gram-Schmidt of their real and imaginary parts
  double *sink = nullptr;
  if (dmalloc(reinterpret_cast<void **>(&sink), sizeof(double) * 2 * (size_t)ntasks * n) != cudaSuccess) {
    cudaGetLastError();
    set_error("gfcc_mor_expand: cannot allocate %.3f GB for the solutions", 16.0 * ntasks * n / 1e9);
    return GFCC_ERR_OOM;
  }
  int rc = solve_for_sink(c, M->sector, n_omega, h_om, eta, n_orb, h_orb, tol, sink, h_G);
  if (rc < 0) {
    dfree(sink);
    return rc;
  }
  std::vector<int> status(c->st_status);
  const int nchunk = (int)((n + MOR_CHUNK - 1) / MOR_CHUNK);
  int s = GFCC_OK;
  const int m0 = M->m;
  for (long long t = 0; t < ntasks && s == GFCC_OK; t++) {
    if (status[t] != GFCC_STATUS_CONVERGED) continue;   // only converged solutions span the model
    for (int p = 0; p < 2 && s == GFCC_OK; p++) {
      // capacity first (ensure_cap may move S), then the workspace view
      s = ensure_cap(M, M->m + 1);
      if (s < 0) break;
      s = grow(M, sizeof(double) * (size_t)(n + (long long)(M->cap + 1) * nchunk + M->cap + 64));
      if (s < 0) break;
      double *v = M->work, *part = v + n, *h = part + (long long)(M->cap + 1) * nchunk;
      mor_plane_kernel<<<grid1d(n), MT, 0, st>>>(sink + 2 * t * n, n, p, v);
      if (cudaGetLastError() != cudaSuccess) {
        s = GFCC_ERR_CUDA;
        break;
      }
      count_launch();
      bool added = false;
      s = gs_append(M, v, part, h, added);
    }
  }
  dfree(sink);
  if (s < 0) return s;
  for (int w = 0; w < n_omega; w++) M->sampled.push_back(h_om[w]);
  if (M->m > m0) GFCC_TRY(project_new(M, m0));
  GFCC_CUDA(cudaStreamSynchronize(st));
  return rc;
}

}  // namespace gfcc

using namespace gfcc;

extern "C" {

int gfcc_mor_create(gfcc_ctx *ctx, int sector, double drop_tol, gfcc_mor **out) {
  if (out == nullptr) {
    set_error("gfcc_mor_create: out is NULL");
    return GFCC_ERR_ARG;
  }
  *out = nullptr;
  if (ctx == nullptr || (sector != GFCC_SECTOR_IP && sector != GFCC_SECTOR_EA) || !(ctx->sectors & sector) ||
      !(drop_tol > 0.0 && drop_tol < 1.0)) {
    set_error("gfcc_mor_create: need a context with the sector built and 0 < drop_tol < 1");
    return GFCC_ERR_ARG;
  }
  if (ctx->rhf) {
    set_error("gfcc_mor_create: model-order reduction is not offered for closed-shell contexts");
    return GFCC_ERR_ARG;
  }
  gfcc_mor *M = new gfcc_mor();
  M->c = ctx;
  M->sector = sector;
  M->n = sector == GFCC_SECTOR_IP ? ctx->dim_ip : ctx->dim_ea;
  M->drop_tol = drop_tol;
  *out = M;
  return GFCC_OK;
}

void gfcc_mor_destroy(gfcc_mor *M) {
  if (M == nullptr) return;
  if (M->c && M->c->stream) cudaStreamSynchronize(M->c->stream);
  dfree(M->S);
  dfree(M->W);
  dfree(M->H);
  dfree(M->work);
  delete M;
}

int gfcc_mor_dim(gfcc_mor *M) { return M == nullptr ? -1 : M->m; }

int gfcc_mor_expand(gfcc_mor *M, int n_omega, const double *omegas, double eta, int n_orb, const int *orbitals,
                    double tol, double *G) {
  if (M == nullptr || n_omega < 1 || n_orb < 1 || omegas == nullptr || orbitals == nullptr || !(eta > 0.0) ||
      !(tol > 0.0)) {
    set_error("gfcc_mor_expand: bad arguments");
    return GFCC_ERR_ARG;
  }
  for (int a = 0; a < n_orb; a++)
    if (orbitals[a] < 0 || orbitals[a] >= M->c->n) {
      set_error("gfcc_mor_expand: orbital index %d out of range", orbitals[a]);
      return GFCC_ERR_ARG;
    }
  return mor_expand_impl(M, n_omega, omegas, eta, n_orb, orbitals, tol, G);
}

int gfcc_mor_green(gfcc_mor *M, int n_omega, const double *omegas, double eta, int n_p, const int *p_orbitals,
                   int n_q, const int *q_orbitals, double *G, double *relres) {
  if (M == nullptr || n_omega < 1 || n_p < 1 || n_q < 1 || omegas == nullptr || p_orbitals == nullptr ||
      q_orbitals == nullptr || !(eta > 0.0)) {
    set_error("gfcc_mor_green: bad arguments");
    return GFCC_ERR_ARG;
  }
  for (int a = 0; a < n_p + n_q; a++) {
    const int x = a < n_p ? p_orbitals[a] : q_orbitals[a - n_p];
    if (x < 0 || x >= M->c->n) {
      set_error("gfcc_mor_green: orbital index %d out of range", x);
      return GFCC_ERR_ARG;
    }
  }
  return mor_green_impl(M, n_omega, omegas, eta, n_p, p_orbitals, n_q, q_orbitals, G, relres);
}

int gfcc_mor_projected(gfcc_mor *M, double *Hhat, double *S_rows, int row_count) {
  if (M == nullptr) {
    set_error("gfcc_mor_projected: NULL object");
    return GFCC_ERR_ARG;
  }
  cudaStream_t st = M->c->stream;
  if (Hhat != nullptr && M->m > 0)
    GFCC_CUDA(cudaMemcpy2DAsync(Hhat, sizeof(double) * M->m, M->H, sizeof(double) * M->cap, sizeof(double) * M->m,
                                M->m, cudaMemcpyDeviceToHost, st));
  if (S_rows != nullptr && row_count > 0)
    GFCC_CUDA(cudaMemcpyAsync(S_rows, M->S, sizeof(double) * (size_t)std::min(row_count, M->m) * M->n,
                              cudaMemcpyDeviceToHost, st));
  GFCC_CUDA(cudaStreamSynchronize(st));
  return GFCC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Adaptive frequency levels and the spectral function (Implementation Details, eq. Lmax; eq. specfxn).
namespace gfcc {
namespace {
int n_max_level(int L) { return L == 1 ? 3 : (L >= 31 ? (1 << 30) : (1 << (L - 1))); }
}  // namespace
}  // namespace gfcc

extern "C" {

int gfcc_spectral_adaptive(gfcc_ctx *ctx, int sectors, double omega_min, double omega_max, double d_omega,
                           double eta, int n_orb, const int *orbitals, double tol, double level_tol, int max_levels,
                           int n_fine, const double *fine_omegas, double *A, int *n_levels, int *level_sizes,
                           double *sampled, int sampled_cap, int *mdim) {
  if (ctx == nullptr || sectors < 1 || sectors > 3 || (sectors & ~ctx->sectors) || !(omega_max > omega_min) ||
      !(d_omega > 0.0) || !(eta > 0.0) || n_orb < 1 || orbitals == nullptr || !(tol > 0.0) || !(level_tol > 0.0) ||
      max_levels < 1 || max_levels > 30 || n_fine < 0 || (n_fine > 0 && (fine_omegas == nullptr || A == nullptr))) {
    set_error("gfcc_spectral_adaptive: bad arguments");
    return GFCC_ERR_ARG;
  }
  gfcc_mor *mors[2] = {nullptr, nullptr};
  const int secs[2] = {GFCC_SECTOR_IP, GFCC_SECTOR_EA};
  int rc = GFCC_OK, warn = GFCC_OK;
  auto cleanup = [&]() {
    for (gfcc_mor *m : mors) gfcc_mor_destroy(m);
  };
  for (int k = 0; k < 2; k++)
    if (sectors & secs[k]) {
      if ((rc = gfcc_mor_create(ctx, secs[k], 1e-10, &mors[k])) < 0) {
        cleanup();
        return rc;
      }
    }
  std::vector<double> all;   // sampled frequencies, in sampling order
  std::vector<int> sizes;
  auto expand = [&](const std::vector<double> &w) -> int {
    for (gfcc_mor *m : mors) {
      if (m == nullptr) continue;
      const int r = gfcc_mor_expand(m, (int)w.size(), w.data(), eta, n_orb, orbitals, tol, nullptr);
      if (r < 0) return r;
      if (r == GFCC_WARN_NOT_CONVERGED) warn = GFCC_WARN_NOT_CONVERGED;
    }
    all.insert(all.end(), w.begin(), w.end());
    sizes.push_back((int)w.size());
    return GFCC_OK;
  };
  std::vector<double> lev = {omega_min, 0.5 * (omega_min + omega_max), omega_max};
  if ((rc = expand(lev)) < 0) {
    cleanup();
    return rc;
  }
  for (int L = 2; L <= max_levels; L++) {
    std::vector<double> s(all);
    std::sort(s.begin(), s.end());
    std::vector<double> cand;
    for (size_t i = 0; i + 1 < s.size(); i++)
      if ((s[i + 1] - s[i]) / 2 >= d_omega * (1 - 1e-12)) cand.push_back(0.5 * (s[i] + s[i + 1]));
    if (cand.empty()) break;
    // error indicator: the largest relative model residual over the sectors and orbitals
    std::vector<double> err(cand.size(), 0.0);
    std::vector<double> G(2 * cand.size() * (size_t)n_orb * n_orb), rr(cand.size() * (size_t)n_orb);
    for (gfcc_mor *m : mors) {
      if (m == nullptr) continue;
      if ((rc = gfcc_mor_green(m, (int)cand.size(), cand.data(), eta, n_orb, orbitals, n_orb, orbitals, G.data(),
                               rr.data())) < 0) {
        cleanup();
        return rc;
      }
      for (size_t w = 0; w < cand.size(); w++)
        for (int a = 0; a < n_orb; a++) err[w] = std::max(err[w], rr[w * n_orb + a]);
    }
    std::vector<std::pair<double, double>> over;   // (error, omega) above the tolerance
    for (size_t w = 0; w < cand.size(); w++)
      if (err[w] > level_tol) over.push_back({err[w], cand[w]});
    if (over.empty()) break;
    std::sort(over.begin(), over.end(), [](const std::pair<double, double> &a, const std::pair<double, double> &b) {
      return a.first > b.first;
    });
    if ((int)over.size() > n_max_level(L)) over.resize(n_max_level(L));
    lev.clear();
    for (auto &e : over) lev.push_back(e.second);
    std::sort(lev.begin(), lev.end());
    if ((rc = expand(lev)) < 0) {
      cleanup();
      return rc;
    }
  }
  // spectral function on the fine grid: A = (1/pi) sum_p (Im G^IP_pp - Im G^EA_pp)
  if (n_fine > 0) {
    for (int w = 0; w < n_fine; w++) A[w] = 0.0;
    std::vector<double> G(2 * (size_t)n_fine * n_orb * n_orb);
    for (int k = 0; k < 2; k++) {
      if (mors[k] == nullptr) continue;
      if ((rc = gfcc_mor_green(mors[k], n_fine, fine_omegas, eta, n_orb, orbitals, n_orb, orbitals, G.data(),
                               nullptr)) < 0) {
        cleanup();
        return rc;
      }
      const double sg = k == 0 ? 1.0 : -1.0;
      for (int w = 0; w < n_fine; w++)
        for (int a = 0; a < n_orb; a++) A[w] += sg * G[2 * (((size_t)w * n_orb + a) * n_orb + a) + 1] / M_PI;
    }
  }
  if (n_levels) *n_levels = (int)sizes.size();
  if (level_sizes)
    for (size_t i = 0; i < sizes.size(); i++) level_sizes[i] = sizes[i];
  if (sampled)
    for (int i = 0; i < (int)all.size() && i < sampled_cap; i++) sampled[i] = all[i];
  if (mdim) {
    mdim[0] = mors[0] ? mors[0]->m : 0;
    mdim[1] = mors[1] ? mors[1]->m : 0;
  }
  cleanup();
  return warn;
}

}  // extern "C"
