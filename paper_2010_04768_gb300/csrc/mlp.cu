// The learned initial-guess model (mlp.cuh): inference, forward / backward, Adam, sample
// collection from kept solutions, and the gfcc_mlp_* entry points.
//
// All layers are small (27 -> 256 -> 256 -> 16): the model is latency-bound, so the kernels are
// plain SIMT code: one 256-thread block per system for inference, a 32 x 32 tiled GEMM with fused
// bias / ReLU / ReLU-mask epilogues for training.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "mlp.cuh"

namespace gfcc {

namespace {

constexpr int MT = 256;   // threads of the inference kernel (>= hidden width)

struct Offsets {
  long long W1, b1, W2, b2, W3, b3, mu, sd, n;
};
__host__ __device__ Offsets offsets(int nin, int nh, int nout) {
  Offsets o;
  o.W1 = 0;
  o.b1 = o.W1 + (long long)nh * nin;
  o.W2 = o.b1 + nh;
  o.b2 = o.W2 + (long long)nh * nh;
  o.W3 = o.b2 + nh;
  o.b3 = o.W3 + (long long)nout * nh;
  o.mu = o.b3 + nout;
  o.sd = o.mu + nin;
  o.n = o.sd + nin;
  return o;
}

template <typename W, typename A>
struct InfView {
  const W *w1t, *w2t, *w3t;             // [nin][nh], [nh][nh], [nh][nout] (transposed)
  const A *b1, *b2, *b3, *mu, *sd;
};

__device__ __forceinline__ float to_acc(__half x, float) { return __half2float(x); }
__device__ __forceinline__ double to_acc(double x, double) { return x; }
template <typename W>
__device__ __forceinline__ W from_master(double x);
template <>
__device__ __forceinline__ __half from_master<__half>(double x) { return __float2half_rn((float)x); }
template <>
__device__ __forceinline__ double from_master<double>(double x) { return x; }

// One block per system (grid-stride over systems): the three layers with the inference copy.
template <typename W, typename A>
__global__ __launch_bounds__(MT) void mlp_infer_kernel(InfView<W, A> p, int nin, int nh, int nout, int nb,
                                                       const double *feat, double *y) {
  __shared__ A x[64], h1[MT], h2[MT];
  const int j = threadIdx.x;
  for (int s = blockIdx.x; s < nb; s += gridDim.x) {
    if (j < nin) x[j] = (A)((feat[(long long)s * nin + j] - (double)p.mu[j]) / (double)p.sd[j]);
    __syncthreads();
    if (j < nh) {
      A z = p.b1[j];
      for (int i = 0; i < nin; i++) z += to_acc(p.w1t[i * nh + j], A()) * x[i];
      h1[j] = z > A(0) ? z : A(0);
    }
    __syncthreads();
    if (j < nh) {
      A z = p.b2[j];
      for (int i = 0; i < nh; i++) z += to_acc(p.w2t[(long long)i * nh + j], A()) * h1[i];
      h2[j] = z > A(0) ? z : A(0);
    }
    __syncthreads();
    if (j < nout) {
      A z = p.b3[j];
      for (int i = 0; i < nh; i++) z += to_acc(p.w3t[i * nout + j], A()) * h2[i];
      y[(long long)s * nout + j] = (double)z;
    }
    __syncthreads();
  }
}

// master parameters -> inference copy (weights transposed)
template <typename T, typename W, typename A>
__global__ void mlp_refresh_kernel(const T *P, int nin, int nh, int nout, W *w1t, W *w2t, W *w3t, A *vec) {
  const Offsets o = offsets(nin, nh, nout);
  const long long n1 = (long long)nin * nh, n2 = (long long)nh * nh, n3 = (long long)nh * nout;
  const long long nv = 2LL * nh + nout + 2LL * nin;
  const long long tot = n1 + n2 + n3 + nv;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    if (t < n1) {
      const long long i = t / nh, j = t % nh;   // w1t[i][j] = W1[j][i]
      w1t[t] = from_master<W>((double)P[o.W1 + j * nin + i]);
    } else if (t < n1 + n2) {
      const long long u = t - n1, i = u / nh, j = u % nh;
      w2t[u] = from_master<W>((double)P[o.W2 + j * nh + i]);
    } else if (t < n1 + n2 + n3) {
      const long long u = t - n1 - n2, i = u / nout, j = u % nout;
      w3t[u] = from_master<W>((double)P[o.W3 + j * nh + i]);
    } else {
      // b1 | b2 | b3 | mu | sd
      const long long u = t - n1 - n2 - n3;
      long long src;
      if (u < nh) src = o.b1 + u;
      else if (u < 2 * nh) src = o.b2 + (u - nh);
      else if (u < 2 * nh + nout) src = o.b3 + (u - 2 * nh);
      else if (u < 2 * nh + nout + nin) src = o.mu + (u - 2 * nh - nout);
      else src = o.sd + (u - 2 * nh - nout - nin);
      vec[u] = (A)P[src];
    }
  }
}

// C[m][n] = sum_k A(m,k) B(k,n) (+ bias[n]); A(m,k) = A[m*as0 + k*as1], B(k,n) = B[k*bs0 + n*bs1].
// mask: C = 0 where mask[m][n] <= 0 (ReLU derivative); C2: relu(C) as well.
template <typename T>
__global__ __launch_bounds__(256) void mlp_gemm_kernel(int M, int N, int K, const T *A, long long as0, long long as1,
                                                       const T *B, long long bs0, long long bs1, const T *bias,
                                                       const T *mask, T *C, T *C2, long long ldc) {
  __shared__ T As[32][33];
  __shared__ T Bs[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int m0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
  T acc[4] = {T(0), T(0), T(0), T(0)};
  for (int k0 = 0; k0 < K; k0 += 32) {
    for (int r = ty; r < 32; r += 8) {
      const int m = m0 + r, k = k0 + tx;
      As[r][tx] = (m < M && k < K) ? A[(long long)m * as0 + (long long)k * as1] : T(0);
      const int kk = k0 + r, n = n0 + tx;
      Bs[r][tx] = (kk < K && n < N) ? B[(long long)kk * bs0 + (long long)n * bs1] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; k++) {
      const T b = Bs[k][tx];
#pragma unroll
      for (int r = 0; r < 4; r++) acc[r] += As[ty + 8 * r][k] * b;
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; r++) {
    const int m = m0 + ty + 8 * r, n = n0 + tx;
    if (m >= M || n >= N) continue;
    T v = acc[r] + (bias ? bias[n] : T(0));
    const long long idx = (long long)m * ldc + n;
    if (mask && !(mask[idx] > T(0))) v = T(0);
    C[idx] = v;
    if (C2) C2[idx] = v > T(0) ? v : T(0);
  }
}

// db[n] = sum_m D[m][n]
template <typename T>
__global__ void mlp_colsum_kernel(int M, int N, const T *D, T *db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  T s = T(0);
  for (int m = 0; m < M; m++) s += D[(long long)m * N + n];
  db[n] = s;
}

// Per sample: loss = a^H Gm a / Gm_00 (a = (sum c - 1, c), c_k = y_2k + i y_2k+1) and its gradient
// d loss / d y = 2 Re / Im ((Gm a)_0 + (Gm a)_k) / Gm_00, scaled by 1 / batch.
template <typename T>
__global__ void mlp_loss_kernel(int Bn, const T *Y, const double *Gm, double inv_b, T *dY, double *lossv) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Bn) return;
  const double2 *G = reinterpret_cast<const double2 *>(Gm) + (long long)s * GUESS_G;
  const T *y = Y + (long long)s * GUESS_NO;
  T *dy = dY + (long long)s * GUESS_NO;
  const double g00 = G[0].x;
  if (!(g00 > 0.0)) {
    for (int k = 0; k < GUESS_NO; k++) dy[k] = T(0);
    lossv[s] = 0.0;
    return;
  }
  double2 a[GUESS_K + 1];
  a[0] = make_double2(-1.0, 0.0);
  for (int k = 0; k < GUESS_K; k++) {
    a[k + 1] = make_double2((double)y[2 * k], (double)y[2 * k + 1]);
    a[0].x += a[k + 1].x;
    a[0].y += a[k + 1].y;
  }
  double2 ga[GUESS_K + 1];
  double num = 0.0;
  for (int j = 0; j <= GUESS_K; j++) {
    double2 t = make_double2(0.0, 0.0);
    for (int l = 0; l <= GUESS_K; l++) {
      const double2 g = G[j * (GUESS_K + 1) + l];
      t.x += g.x * a[l].x - g.y * a[l].y;
      t.y += g.x * a[l].y + g.y * a[l].x;
    }
    ga[j] = t;
    num += a[j].x * t.x + a[j].y * t.y;
  }
  lossv[s] = num / g00;
  const double sc = 2.0 * inv_b / g00;
  for (int k = 0; k < GUESS_K; k++) {
    dy[2 * k] = (T)(sc * (ga[0].x + ga[k + 1].x));
    dy[2 * k + 1] = (T)(sc * (ga[0].y + ga[k + 1].y));
  }
}

__global__ void sum_kernel(int n, const double *x, double *out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// Adam (Kingma & Ba 2015) on the trained prefix of the parameters.
template <typename T>
__global__ void mlp_adam_kernel(long long n, T *P, const T *G, T *Mo, T *Vo, double lr, double b1, double b2,
                                double eps, double bc1, double bc2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double g = (double)G[i];
    const double m = b1 * (double)Mo[i] + (1.0 - b1) * g;
    const double v = b2 * (double)Vo[i] + (1.0 - b2) * g * g;
    Mo[i] = (T)m;
    Vo[i] = (T)v;
    P[i] = (T)((double)P[i] - lr * (m / bc1) / (sqrt(v / bc2) + eps));
  }
}

// Xn[r] = (feat[ids[r]] - mu) / sd in the training precision, Gb[r] = gram[ids[r]].
template <typename T>
__global__ void mlp_gather_kernel(int Bn, const int *ids, const double *feat, const double *gram, const T *P,
                                  long long omu, long long osd, T *Xn, double *Gb) {
  const long long per = GUESS_NF + 2 * GUESS_G;
  const long long tot = per * Bn;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t / per);
    const int u = (int)(t - (long long)r * per);
    const long long id = ids[r];
    if (u < GUESS_NF) {
      Xn[(long long)r * GUESS_NF + u] = (T)((feat[id * GUESS_NF + u] - (double)P[omu + u]) / (double)P[osd + u]);
    } else {
      const int g = u - GUESS_NF;
      Gb[(long long)r * 2 * GUESS_G + g] = gram[id * 2 * GUESS_G + g];
    }
  }
}

// mu / sd of each feature over the samples (one block per feature; a constant feature gets sd = 1).
template <typename T>
__global__ void mlp_norm_kernel(long long ns, const double *feat, T *P, long long omu, long long osd) {
  __shared__ double sh[256];
  const int i = blockIdx.x;
  double s = 0.0;
  for (long long r = threadIdx.x; r < ns; r += blockDim.x) s += feat[r * GUESS_NF + i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  const double mean = sh[0] / (double)ns;
  __syncthreads();
  s = 0.0;
  for (long long r = threadIdx.x; r < ns; r += blockDim.x) {
    const double d = feat[r * GUESS_NF + i] - mean;
    s += d * d;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double sd = sqrt(sh[0] / (double)ns);
    P[omu + i] = (T)mean;
    P[osd + i] = (T)(sd > 1e-12 * fmax(1.0, fabs(mean)) ? sd : 1.0);
  }
}

// ---------------------------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------------------------

size_t tsize(const gfcc_mlp *m) { return m->precision == GFCC_MLP_FP64 ? sizeof(double) : sizeof(float); }

int ensure_ws(gfcc_mlp *m, size_t bytes) {
  if (m->ws_bytes >= bytes) return GFCC_OK;
  if (m->ws) dfree(m->ws);
  m->ws = nullptr;
  m->ws_bytes = 0;
  if (dmalloc(&m->ws, bytes) != cudaSuccess) {
    cudaGetLastError();
    set_error("gfcc_mlp: cannot allocate %.3f MB of workspace", bytes / 1e6);
    return GFCC_ERR_OOM;
  }
  m->ws_bytes = bytes;
  return GFCC_OK;
}

// Training workspace for a batch of Bn samples (T = training precision).
struct TrainWs {
  void *Xn, *Z1, *H1, *Z2, *H2, *Y, *dY, *dZ2, *dZ1;   // T arrays
  double *Gb, *lossv, *feat, *gram, *acc;
  int *ids;
  size_t bytes;
};
// base == nullptr: only the size (w.bytes) is meaningful
TrainWs train_layout(const gfcc_mlp *m, int Bn, void *base, long long nacc) {
  TrainWs w;
  const size_t ts = tsize(m);
  size_t off = 0;
  auto take = [&](size_t bytes) -> void * {
    void *r = base ? static_cast<void *>(static_cast<char *>(base) + off) : nullptr;
    off += (bytes + 255) & ~size_t(255);
    return r;
  };
  w.Xn = take(ts * Bn * m->nin);
  w.Z1 = take(ts * Bn * m->nh);
  w.H1 = take(ts * Bn * m->nh);
  w.Z2 = take(ts * Bn * m->nh);
  w.H2 = take(ts * Bn * m->nh);
  w.Y = take(ts * Bn * m->nout);
  w.dY = take(ts * Bn * m->nout);
  w.dZ2 = take(ts * Bn * m->nh);
  w.dZ1 = take(ts * Bn * m->nh);
  w.Gb = static_cast<double *>(take(sizeof(double) * Bn * 2 * GUESS_G));
  w.lossv = static_cast<double *>(take(sizeof(double) * Bn));
  w.feat = static_cast<double *>(take(sizeof(double) * Bn * GUESS_NF));
  w.gram = static_cast<double *>(take(sizeof(double) * Bn * 2 * GUESS_G));
  w.acc = static_cast<double *>(take(sizeof(double) * std::max<long long>(nacc, 1)));
  w.ids = static_cast<int *>(take(sizeof(int) * Bn));
  w.bytes = off;
  return w;
}

template <typename T>
int gemm(cudaStream_t st, int M, int N, int K, const T *A, long long as0, long long as1, const T *B, long long bs0,
         long long bs1, const T *bias, const T *mask, T *C, T *C2, long long ldc) {
  if (M <= 0 || N <= 0) return GFCC_OK;
  mlp_gemm_kernel<T><<<dim3(cdiv(N, 32), cdiv(M, 32)), 256, 0, st>>>(M, N, K, A, as0, as1, B, bs0, bs1, bias, mask, C,
                                                                    C2, ldc);
  GFCC_LAUNCH_CHECK();
  return GFCC_OK;
}

// Forward (training precision) of Bn gathered samples, loss per sample, and (want_grad) the
// gradient of the mean loss into m->Gr.
template <typename T>
int fwd_bwd(gfcc_mlp *m, const TrainWs &w, int Bn, bool want_grad) {
  cudaStream_t st = m->stream;
  const Offsets o = offsets(m->nin, m->nh, m->nout);
  const int nin = m->nin, nh = m->nh, nout = m->nout;
  T *P = static_cast<T *>(m->P), *G = static_cast<T *>(m->Gr);
  T *Xn = static_cast<T *>(w.Xn), *Z1 = static_cast<T *>(w.Z1), *H1 = static_cast<T *>(w.H1);
  T *Z2 = static_cast<T *>(w.Z2), *H2 = static_cast<T *>(w.H2), *Y = static_cast<T *>(w.Y);
  T *dY = static_cast<T *>(w.dY), *dZ2 = static_cast<T *>(w.dZ2), *dZ1 = static_cast<T *>(w.dZ1);
  // Z1 = Xn W1^T + b1, H1 = relu(Z1); Z2 = H1 W2^T + b2, H2 = relu(Z2); Y = H2 W3^T + b3
  GFCC_TRY(gemm<T>(st, Bn, nh, nin, Xn, nin, 1, P + o.W1, 1, nin, P + o.b1, nullptr, Z1, H1, nh));
  GFCC_TRY(gemm<T>(st, Bn, nh, nh, H1, nh, 1, P + o.W2, 1, nh, P + o.b2, nullptr, Z2, H2, nh));
  GFCC_TRY(gemm<T>(st, Bn, nout, nh, H2, nh, 1, P + o.W3, 1, nh, P + o.b3, nullptr, Y, nullptr, nout));
  mlp_loss_kernel<T><<<cdiv(Bn, 128), 128, 0, st>>>(Bn, Y, w.Gb, 1.0 / Bn, dY, w.lossv);
  GFCC_LAUNCH_CHECK();
  if (!want_grad) return GFCC_OK;
  // dW3 = dY^T H2, db3 = colsum dY; dZ2 = (dY W3) * [Z2 > 0]
  GFCC_TRY(gemm<T>(st, nout, nh, Bn, dY, 1, nout, H2, nh, 1, nullptr, nullptr, G + o.W3, nullptr, nh));
  mlp_colsum_kernel<T><<<cdiv(nout, 128), 128, 0, st>>>(Bn, nout, dY, G + o.b3);
  GFCC_LAUNCH_CHECK();
  GFCC_TRY(gemm<T>(st, Bn, nh, nout, dY, nout, 1, P + o.W3, nh, 1, nullptr, Z2, dZ2, nullptr, nh));
  // dW2 = dZ2^T H1, db2 = colsum dZ2; dZ1 = (dZ2 W2) * [Z1 > 0]
  GFCC_TRY(gemm<T>(st, nh, nh, Bn, dZ2, 1, nh, H1, nh, 1, nullptr, nullptr, G + o.W2, nullptr, nh));
  mlp_colsum_kernel<T><<<cdiv(nh, 128), 128, 0, st>>>(Bn, nh, dZ2, G + o.b2);
  GFCC_LAUNCH_CHECK();
  GFCC_TRY(gemm<T>(st, Bn, nh, nh, dZ2, nh, 1, P + o.W2, nh, 1, nullptr, Z1, dZ1, nullptr, nh));
  // dW1 = dZ1^T Xn, db1 = colsum dZ1
  GFCC_TRY(gemm<T>(st, nh, nin, Bn, dZ1, 1, nh, Xn, nin, 1, nullptr, nullptr, G + o.W1, nullptr, nin));
  mlp_colsum_kernel<T><<<cdiv(nh, 128), 128, 0, st>>>(Bn, nh, dZ1, G + o.b1);
  GFCC_LAUNCH_CHECK();
  return GFCC_OK;
}

int refresh(gfcc_mlp *m) {
  const int nin = m->nin, nh = m->nh, nout = m->nout;
  const long long n1 = (long long)nin * nh, n2 = (long long)nh * nh, n3 = (long long)nh * nout;
  const long long tot = n1 + n2 + n3 + 2LL * nh + nout + 2LL * nin;
  if (m->precision == GFCC_MLP_FP64) {
    double *w = static_cast<double *>(m->Pinf);
    mlp_refresh_kernel<double, double, double><<<grid1d(tot), 256, 0, m->stream>>>(
        static_cast<const double *>(m->P), nin, nh, nout, w, w + n1, w + n1 + n2, w + n1 + n2 + n3);
  } else {
    __half *w = static_cast<__half *>(m->Pinf);
    float *vec = reinterpret_cast<float *>(static_cast<char *>(m->Pinf) + (((n1 + n2 + n3) * sizeof(__half) + 255) & ~255LL));
    mlp_refresh_kernel<float, __half, float><<<grid1d(tot), 256, 0, m->stream>>>(
        static_cast<const float *>(m->P), nin, nh, nout, w, w + n1, w + n1 + n2, vec);
  }
  GFCC_LAUNCH_CHECK();
  return GFCC_OK;
}

size_t inf_bytes(const gfcc_mlp *m) {
  const long long nw = (long long)m->nin * m->nh + (long long)m->nh * m->nh + (long long)m->nh * m->nout;
  const long long nv = 2LL * m->nh + m->nout + 2LL * m->nin;
  if (m->precision == GFCC_MLP_FP64) return sizeof(double) * (nw + nv);
  return ((nw * sizeof(__half) + 255) & ~255LL) + sizeof(float) * nv;
}

// host parameter array (double) <-> master array (T)
int params_to_device(gfcc_mlp *m, const double *h, long long count) {
  if (m->precision == GFCC_MLP_FP64) {
    GFCC_CUDA(cudaMemcpyAsync(m->P, h, sizeof(double) * count, cudaMemcpyHostToDevice, m->stream));
  } else {
    std::vector<float> f(h, h + count);
    GFCC_CUDA(cudaMemcpyAsync(m->P, f.data(), sizeof(float) * count, cudaMemcpyHostToDevice, m->stream));
    GFCC_CUDA(cudaStreamSynchronize(m->stream));
  }
  return GFCC_OK;
}
int array_to_host(const gfcc_mlp *m, const void *d, long long count, double *h) {
  if (m->precision == GFCC_MLP_FP64) {
    GFCC_CUDA(cudaMemcpyAsync(h, d, sizeof(double) * count, cudaMemcpyDeviceToHost, m->stream));
    GFCC_CUDA(cudaStreamSynchronize(m->stream));
  } else {
    std::vector<float> f(count);
    GFCC_CUDA(cudaMemcpyAsync(f.data(), d, sizeof(float) * count, cudaMemcpyDeviceToHost, m->stream));
    GFCC_CUDA(cudaStreamSynchronize(m->stream));
    for (long long i = 0; i < count; i++) h[i] = f[i];
  }
  return GFCC_OK;
}

template <typename T>
int gather(gfcc_mlp *m, const TrainWs &w, int Bn, const int *ids, const double *feat, const double *gram) {
  const Offsets o = offsets(m->nin, m->nh, m->nout);
  mlp_gather_kernel<T><<<grid1d((long long)Bn * (GUESS_NF + 2 * GUESS_G)), 256, 0, m->stream>>>(
      Bn, ids, feat, gram, static_cast<const T *>(m->P), o.mu, o.sd, static_cast<T *>(w.Xn), w.Gb);
  GFCC_LAUNCH_CHECK();
  return GFCC_OK;
}

template <typename T>
int adam(gfcc_mlp *m, double lr) {
  m->step++;
  const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
  const double bc1 = 1.0 - std::pow(b1, (double)m->step), bc2 = 1.0 - std::pow(b2, (double)m->step);
  mlp_adam_kernel<T><<<grid1d(m->ntrain), 256, 0, m->stream>>>(m->ntrain, static_cast<T *>(m->P),
                                                               static_cast<const T *>(m->Gr), static_cast<T *>(m->Mo),
                                                               static_cast<T *>(m->Vo), lr, b1, b2, eps, bc1, bc2);
  GFCC_LAUNCH_CHECK();
  return GFCC_OK;
}

int check_mlp(const gfcc_mlp *m, const char *who) {
  if (m == nullptr) {
    set_error("%s: model is NULL", who);
    return GFCC_ERR_ARG;
  }
  return GFCC_OK;
}

// splitmix64 (Steele, Lea, Flood 2014): sampling of minibatches and neighbour subsets
struct SplitMix {
  unsigned long long x;
  unsigned long long next() {
    unsigned long long z = (x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  }
  double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};

int append_samples(gfcc_mlp *m, int cnt, const double *feat, const double *gram) {
  if (m->ns + cnt > m->cap) {
    const long long ncap = std::max<long long>(m->ns + cnt, std::max<long long>(1024, 2 * m->cap));
    double *nf = nullptr, *ng = nullptr;
    if (dmalloc(reinterpret_cast<void **>(&nf), sizeof(double) * ncap * GUESS_NF) != cudaSuccess ||
        dmalloc(reinterpret_cast<void **>(&ng), sizeof(double) * ncap * 2 * GUESS_G) != cudaSuccess) {
      cudaGetLastError();
      if (nf) dfree(nf);
      set_error("gfcc_mlp_collect: cannot grow the sample store to %lld samples", ncap);
      return GFCC_ERR_OOM;
    }
    if (m->ns > 0) {
      GFCC_CUDA(cudaMemcpyAsync(nf, m->feat, sizeof(double) * m->ns * GUESS_NF, cudaMemcpyDeviceToDevice, m->stream));
      GFCC_CUDA(cudaMemcpyAsync(ng, m->gram, sizeof(double) * m->ns * 2 * GUESS_G, cudaMemcpyDeviceToDevice, m->stream));
    }
    GFCC_CUDA(cudaStreamSynchronize(m->stream));
    if (m->feat) dfree(m->feat);
    if (m->gram) dfree(m->gram);
    m->feat = nf;
    m->gram = ng;
    m->cap = ncap;
  }
  GFCC_CUDA(cudaMemcpyAsync(m->feat + m->ns * GUESS_NF, feat, sizeof(double) * cnt * GUESS_NF, cudaMemcpyDeviceToDevice,
                            m->stream));
  GFCC_CUDA(cudaMemcpyAsync(m->gram + m->ns * 2 * GUESS_G, gram, sizeof(double) * cnt * 2 * GUESS_G,
                            cudaMemcpyDeviceToDevice, m->stream));
  m->ns += cnt;
  return GFCC_OK;
}

}  // namespace

int mlp_infer(gfcc_mlp *m, cudaStream_t st, int nb, const double *feat, double *y) {
  if (nb <= 0) return GFCC_OK;
  const int nin = m->nin, nh = m->nh, nout = m->nout;
  const long long n1 = (long long)nin * nh, n2 = (long long)nh * nh, n3 = (long long)nh * nout;
  const int grid = std::min(nb, 152 * 8);
  if (m->precision == GFCC_MLP_FP64) {
    const double *w = static_cast<const double *>(m->Pinf);
    const double *vec = w + n1 + n2 + n3;
    InfView<double, double> p{w, w + n1, w + n1 + n2, vec, vec + nh, vec + 2 * nh, vec + 2 * nh + nout,
                              vec + 2 * nh + nout + nin};
    mlp_infer_kernel<double, double><<<grid, MT, 0, st>>>(p, nin, nh, nout, nb, feat, y);
  } else {
    const __half *w = static_cast<const __half *>(m->Pinf);
    const float *vec = reinterpret_cast<const float *>(static_cast<const char *>(m->Pinf) +
                                                       (((n1 + n2 + n3) * sizeof(__half) + 255) & ~255LL));
    InfView<__half, float> p{w, w + n1, w + n1 + n2, vec, vec + nh, vec + 2 * nh, vec + 2 * nh + nout,
                             vec + 2 * nh + nout + nin};
    mlp_infer_kernel<__half, float><<<grid, MT, 0, st>>>(p, nin, nh, nout, nb, feat, y);
  }
  GFCC_LAUNCH_CHECK();
  return GFCC_OK;
}

}  // namespace gfcc

using namespace gfcc;

extern "C" {

int gfcc_mlp_create(int hidden, int precision, const double *init_params, gfcc_mlp **out) {
  if (out == nullptr || init_params == nullptr || hidden < 1 || hidden > MT ||
      (precision != GFCC_MLP_FP32 && precision != GFCC_MLP_FP64)) {
    set_error("gfcc_mlp_create: need 1 <= hidden <= %d, a precision GFCC_MLP_*, initial parameters and out", MT);
    return GFCC_ERR_ARG;
  }
  *out = nullptr;
  gfcc_mlp *m = new gfcc_mlp();
  m->nh = hidden;
  m->precision = precision;
  const Offsets o = offsets(m->nin, m->nh, m->nout);
  m->nparam = o.n;
  m->ntrain = o.mu;
  auto fail = [&](int rc) {
    gfcc_mlp_destroy(m);
    return rc;
  };
  if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    set_error("gfcc_mlp_create: cannot create a stream");
    delete m;
    return GFCC_ERR_CUDA;
  }
  const size_t pb = tsize(m) * m->nparam;
  if (dmalloc(&m->P, pb) != cudaSuccess || dmalloc(&m->Mo, pb) != cudaSuccess || dmalloc(&m->Vo, pb) != cudaSuccess ||
      dmalloc(&m->Gr, pb) != cudaSuccess || dmalloc(&m->Pinf, inf_bytes(m)) != cudaSuccess) {
    cudaGetLastError();
    set_error("gfcc_mlp_create: device allocation failed");
    return fail(GFCC_ERR_OOM);
  }
  if (cudaMemsetAsync(m->Mo, 0, pb, m->stream) != cudaSuccess || cudaMemsetAsync(m->Vo, 0, pb, m->stream) != cudaSuccess ||
      cudaMemsetAsync(m->Gr, 0, pb, m->stream) != cudaSuccess) {
    set_error("gfcc_mlp_create: memset failed");
    return fail(GFCC_ERR_CUDA);
  }
  // the normalisation entries start at mu = 0, sd = 1 (set from the samples at the first training)
  std::vector<double> h(init_params, init_params + m->nparam);
  for (int i = 0; i < m->nin; i++) {
    h[o.mu + i] = 0.0;
    h[o.sd + i] = 1.0;
  }
  int rc = params_to_device(m, h.data(), m->nparam);
  if (rc == GFCC_OK) rc = refresh(m);
  if (rc == GFCC_OK && cudaStreamSynchronize(m->stream) != cudaSuccess) rc = GFCC_ERR_CUDA;
  if (rc != GFCC_OK) return fail(rc);
  *out = m;
  return GFCC_OK;
}

void gfcc_mlp_destroy(gfcc_mlp *m) {
  if (m == nullptr) return;
  if (m->stream) cudaStreamSynchronize(m->stream);
  for (void *p : {m->P, m->Mo, m->Vo, m->Gr, m->Pinf, m->ws, static_cast<void *>(m->feat), static_cast<void *>(m->gram)})
    if (p) dfree(p);
  if (m->stream) cudaStreamDestroy(m->stream);
  delete m;
}

long long gfcc_mlp_num_params(const gfcc_mlp *m) { return m ? m->nparam : 0; }

long long gfcc_mlp_num_samples(const gfcc_mlp *m) { return m ? m->ns : 0; }

int gfcc_mlp_get_params(gfcc_mlp *m, double *params) {
  GFCC_TRY(check_mlp(m, "gfcc_mlp_get_params"));
  if (params == nullptr) {
    set_error("gfcc_mlp_get_params: params is NULL");
    return GFCC_ERR_ARG;
  }
  return array_to_host(m, m->P, m->nparam, params);
}

int gfcc_mlp_set_params(gfcc_mlp *m, const double *params) {
  GFCC_TRY(check_mlp(m, "gfcc_mlp_set_params"));
  if (params == nullptr) {
    set_error("gfcc_mlp_set_params: params is NULL");
    return GFCC_ERR_ARG;
  }
  const Offsets o = offsets(m->nin, m->nh, m->nout);
  for (int i = 0; i < m->nin; i++)
    if (!(params[o.sd + i] != 0.0)) {
      set_error("gfcc_mlp_set_params: normalisation sd[%d] is zero", i);
      return GFCC_ERR_ARG;
    }
  GFCC_TRY(params_to_device(m, params, m->nparam));
  GFCC_TRY(refresh(m));
  GFCC_CUDA(cudaStreamSynchronize(m->stream));
  m->norm_set = true;
  return GFCC_OK;
}

int gfcc_mlp_forward(gfcc_mlp *m, int nb, const double *features, double *y) {
  GFCC_TRY(check_mlp(m, "gfcc_mlp_forward"));
  if (nb < 0 || (nb > 0 && (features == nullptr || y == nullptr))) {
    set_error("gfcc_mlp_forward: bad arguments");
    return GFCC_ERR_ARG;
  }
  if (nb == 0) return GFCC_OK;
  const size_t fb = sizeof(double) * nb * GUESS_NF, yb = sizeof(double) * nb * GUESS_NO;
  GFCC_TRY(ensure_ws(m, fb + yb + 512));
  double *df = static_cast<double *>(m->ws);
  double *dy = reinterpret_cast<double *>(static_cast<char *>(m->ws) + ((fb + 255) & ~size_t(255)));
  GFCC_CUDA(cudaMemcpyAsync(df, features, fb, cudaMemcpyHostToDevice, m->stream));
  GFCC_TRY(mlp_infer(m, m->stream, nb, df, dy));
  GFCC_CUDA(cudaMemcpyAsync(y, dy, yb, cudaMemcpyDeviceToHost, m->stream));
  GFCC_CUDA(cudaStreamSynchronize(m->stream));
  return GFCC_OK;
}

// shared by gfcc_mlp_loss_grad and gfcc_mlp_train_batch
static int host_batch_step(gfcc_mlp *m, int nb, const double *features, const double *gram, double lr, double *loss,
                           double *grad, const char *who) {
  GFCC_TRY(check_mlp(m, who));
  if (nb < 1 || features == nullptr || gram == nullptr) {
    set_error("%s: need nb >= 1, features and gram", who);
    return GFCC_ERR_ARG;
  }
  const size_t need = train_layout(m, nb, nullptr, 1).bytes + 256;
  GFCC_TRY(ensure_ws(m, need));
  const TrainWs w = train_layout(m, nb, m->ws, 1);
  std::vector<int> ids(nb);
  for (int i = 0; i < nb; i++) ids[i] = i;
  GFCC_CUDA(cudaMemcpyAsync(w.feat, features, sizeof(double) * nb * GUESS_NF, cudaMemcpyHostToDevice, m->stream));
  GFCC_CUDA(cudaMemcpyAsync(w.gram, gram, sizeof(double) * nb * 2 * GUESS_G, cudaMemcpyHostToDevice, m->stream));
  GFCC_CUDA(cudaMemcpyAsync(w.ids, ids.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, m->stream));
  const bool f64 = m->precision == GFCC_MLP_FP64;
  GFCC_TRY(f64 ? gather<double>(m, w, nb, w.ids, w.feat, w.gram) : gather<float>(m, w, nb, w.ids, w.feat, w.gram));
  GFCC_TRY(f64 ? fwd_bwd<double>(m, w, nb, true) : fwd_bwd<float>(m, w, nb, true));
  sum_kernel<<<1, 256, 0, m->stream>>>(nb, w.lossv, w.acc);
  GFCC_LAUNCH_CHECK();
  double tot = 0.0;
  GFCC_CUDA(cudaMemcpyAsync(&tot, w.acc, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  if (grad) {
    GFCC_TRY(array_to_host(m, m->Gr, m->ntrain, grad));
    for (long long i = m->ntrain; i < m->nparam; i++) grad[i] = 0.0;
  }
  if (lr > 0.0) {
    GFCC_TRY(f64 ? adam<double>(m, lr) : adam<float>(m, lr));
    GFCC_TRY(refresh(m));
  }
  GFCC_CUDA(cudaStreamSynchronize(m->stream));
  if (loss) *loss = tot / nb;
  return GFCC_OK;
}

int gfcc_mlp_loss_grad(gfcc_mlp *m, int nb, const double *features, const double *gram, double *loss, double *grad) {
  return host_batch_step(m, nb, features, gram, 0.0, loss, grad, "gfcc_mlp_loss_grad");
}

int gfcc_mlp_train_batch(gfcc_mlp *m, int nb, const double *features, const double *gram, double lr, double *loss) {
  if (!(lr > 0.0)) {
    set_error("gfcc_mlp_train_batch: lr must be > 0");
    return GFCC_ERR_ARG;
  }
  return host_batch_step(m, nb, features, gram, lr, loss, nullptr, "gfcc_mlp_train_batch");
}

int gfcc_mlp_train(gfcc_mlp *m, int steps, int minibatch, double lr, unsigned long long seed, double *loss) {
  GFCC_TRY(check_mlp(m, "gfcc_mlp_train"));
  if (steps < 1 || minibatch < 1 || minibatch > 65536 || !(lr > 0.0)) {
    set_error("gfcc_mlp_train: need steps >= 1, 1 <= minibatch <= 65536, lr > 0");
    return GFCC_ERR_ARG;
  }
  if (m->ns < 1) {
    set_error("gfcc_mlp_train: no samples (call gfcc_mlp_collect first)");
    return GFCC_ERR_STATE;
  }
  const bool f64 = m->precision == GFCC_MLP_FP64;
  const Offsets o = offsets(m->nin, m->nh, m->nout);
  if (!m->norm_set) {
    if (f64)
      mlp_norm_kernel<double><<<m->nin, 256, 0, m->stream>>>(m->ns, m->feat, static_cast<double *>(m->P), o.mu, o.sd);
    else
      mlp_norm_kernel<float><<<m->nin, 256, 0, m->stream>>>(m->ns, m->feat, static_cast<float *>(m->P), o.mu, o.sd);
    GFCC_LAUNCH_CHECK();
    m->norm_set = true;
  }
  // minibatch indices of every step, drawn on the host (with replacement) and uploaded once
  std::vector<int> ids((size_t)steps * minibatch);
  SplitMix rng{seed};
  for (auto &x : ids) x = (int)(rng.next() % (unsigned long long)m->ns);
  const size_t idb = ((sizeof(int) * ids.size() + 255) & ~size_t(255));
  const size_t need = train_layout(m, minibatch, nullptr, steps).bytes + idb + 256;
  GFCC_TRY(ensure_ws(m, need));
  const TrainWs w = train_layout(m, minibatch, m->ws, steps);
  int *d_ids = reinterpret_cast<int *>(static_cast<char *>(m->ws) + w.bytes);
  GFCC_CUDA(cudaMemcpyAsync(d_ids, ids.data(), sizeof(int) * ids.size(), cudaMemcpyHostToDevice, m->stream));
  for (int s = 0; s < steps; s++) {
    const int *sid = d_ids + (size_t)s * minibatch;
    GFCC_TRY(f64 ? gather<double>(m, w, minibatch, sid, m->feat, m->gram)
                 : gather<float>(m, w, minibatch, sid, m->feat, m->gram));
    GFCC_TRY(f64 ? fwd_bwd<double>(m, w, minibatch, true) : fwd_bwd<float>(m, w, minibatch, true));
    sum_kernel<<<1, 256, 0, m->stream>>>(minibatch, w.lossv, w.acc + s);
    GFCC_LAUNCH_CHECK();
    GFCC_TRY(f64 ? adam<double>(m, lr) : adam<float>(m, lr));
  }
  GFCC_TRY(refresh(m));
  std::vector<double> acc(steps);
  GFCC_CUDA(cudaMemcpyAsync(acc.data(), w.acc, sizeof(double) * steps, cudaMemcpyDeviceToHost, m->stream));
  GFCC_CUDA(cudaStreamSynchronize(m->stream));
  if (loss) {
    // mean minibatch loss over the last (up to) 50 steps
    const int k = std::min(steps, 50);
    double t = 0.0;
    for (int s = steps - k; s < steps; s++) t += acc[s];
    *loss = t / ((double)k * minibatch);
  }
  return GFCC_OK;
}

int gfcc_mlp_get_samples(gfcc_mlp *m, long long start, int count, double *features, double *gram) {
  GFCC_TRY(check_mlp(m, "gfcc_mlp_get_samples"));
  if (start < 0 || count < 0 || start + count > m->ns) {
    set_error("gfcc_mlp_get_samples: samples [%lld, %lld) outside [0, %lld)", start, start + count, m->ns);
    return GFCC_ERR_ARG;
  }
  if (count == 0) return GFCC_OK;
  if (features)
    GFCC_CUDA(cudaMemcpyAsync(features, m->feat + start * GUESS_NF, sizeof(double) * count * GUESS_NF,
                              cudaMemcpyDeviceToHost, m->stream));
  if (gram)
    GFCC_CUDA(cudaMemcpyAsync(gram, m->gram + start * 2 * GUESS_G, sizeof(double) * count * 2 * GUESS_G,
                              cudaMemcpyDeviceToHost, m->stream));
  GFCC_CUDA(cudaStreamSynchronize(m->stream));
  return GFCC_OK;
}

int gfcc_mlp_eval(gfcc_mlp *m, double *out) {
  GFCC_TRY(check_mlp(m, "gfcc_mlp_eval"));
  if (out == nullptr) {
    set_error("gfcc_mlp_eval: out is NULL");
    return GFCC_ERR_ARG;
  }
  if (m->ns < 1) {
    set_error("gfcc_mlp_eval: no samples");
    return GFCC_ERR_STATE;
  }
  const int CB = 1024;
  const size_t yb = ((sizeof(double) * CB * GUESS_NO + 255) & ~size_t(255));
  GFCC_TRY(ensure_ws(m, yb + 2 * sizeof(double) * CB + 512));
  double *dy = static_cast<double *>(m->ws);
  double *lm = reinterpret_cast<double *>(static_cast<char *>(m->ws) + yb);
  double *lr = lm + CB;
  std::vector<double> hm(CB), hr(CB);
  double sm = 0.0, sf = 0.0, sr = 0.0, better = 0.0;
  for (long long s0 = 0; s0 < m->ns; s0 += CB) {
    const int nb = (int)std::min<long long>(CB, m->ns - s0);
    GFCC_TRY(mlp_infer(m, m->stream, nb, m->feat + s0 * GUESS_NF, dy));
    GFCC_TRY(guess_losses(m->stream, nb, m->gram + s0 * 2 * GUESS_G, dy, lm, lr));
    GFCC_CUDA(cudaMemcpyAsync(hm.data(), lm, sizeof(double) * nb, cudaMemcpyDeviceToHost, m->stream));
    GFCC_CUDA(cudaMemcpyAsync(hr.data(), lr, sizeof(double) * nb, cudaMemcpyDeviceToHost, m->stream));
    GFCC_CUDA(cudaStreamSynchronize(m->stream));
    for (int i = 0; i < nb; i++) {
      sm += hm[i];
      sf += hm[i] < 1.0 ? hm[i] : 1.0;
      sr += std::min(std::max(hr[i], 0.0), 1.0);
      better += hm[i] < 1.0 ? 1.0 : 0.0;
    }
  }
  out[0] = sm / m->ns;
  out[1] = sf / m->ns;
  out[2] = sr / m->ns;
  out[3] = better / m->ns;
  return GFCC_OK;
}

int gfcc_mlp_collect(gfcc_mlp *m, gfcc_ctx *c, int samples_per_system, unsigned long long seed, long long *added) {
  GFCC_TRY(check_mlp(m, "gfcc_mlp_collect"));
  if (c == nullptr || samples_per_system < 1) {
    set_error("gfcc_mlp_collect: need a context and samples_per_system >= 1");
    return GFCC_ERR_ARG;
  }
  const KeptSolutions &kp = c->kept;
  if (kp.X == nullptr || kp.nw == 0) {
    set_error("gfcc_mlp_collect: the context keeps no solutions (set GFCC_OPT_KEEP_SOLUTIONS or a guess, then solve)");
    return GFCC_ERR_STATE;
  }
  GFCC_CUDA(cudaStreamSynchronize(c->stream));
  const int CB = 128;
  const long long n = kp.n;
  // device temporaries: rhs [CB][n], Gram, features, gram work, nbr, delta, omega, pfrac, porb
  const long long gw = guess_gram_work_doubles(CB, n);
  const long long dbl = 2LL * CB * n + 2LL * CB * GUESS_G + (long long)CB * GUESS_NF + gw + CB * GUESS_K + 2LL * CB + 64;
  const long long ints = (long long)CB * GUESS_K + CB;
  void *tmp = nullptr;
  if (dmalloc(&tmp, sizeof(double) * dbl + sizeof(int) * ints + 1024) != cudaSuccess) {
    cudaGetLastError();
    set_error("gfcc_mlp_collect: cannot allocate %.3f GB of workspace", (sizeof(double) * dbl) / 1e9);
    return GFCC_ERR_OOM;
  }
  double *Bt = static_cast<double *>(tmp);
  double *Gm = Bt + 2LL * CB * n;
  double *feat = Gm + 2LL * CB * GUESS_G;
  double *work = feat + (long long)CB * GUESS_NF;
  double *delta = work + gw;
  double *om = delta + CB * GUESS_K;
  double *pf = om + CB;
  int *nbr = reinterpret_cast<int *>(pf + CB + 64);
  int *porb = nbr + CB * GUESS_K;
  std::vector<int> h_nbr(CB * GUESS_K), h_porb(CB);
  std::vector<double> h_delta(CB * GUESS_K), h_om(CB), h_pf(CB);
  std::vector<char> mask(kp.nw);
  SplitMix rng{seed};
  long long cnt_total = 0;
  int cnt = 0;
  int rc = GFCC_OK;
  auto flush = [&]() -> int {
    if (cnt == 0) return GFCC_OK;
    GFCC_CUDA(cudaMemcpyAsync(nbr, h_nbr.data(), sizeof(int) * cnt * GUESS_K, cudaMemcpyHostToDevice, c->stream));
    GFCC_CUDA(cudaMemcpyAsync(porb, h_porb.data(), sizeof(int) * cnt, cudaMemcpyHostToDevice, c->stream));
    GFCC_CUDA(cudaMemcpyAsync(delta, h_delta.data(), sizeof(double) * cnt * GUESS_K, cudaMemcpyHostToDevice, c->stream));
    GFCC_CUDA(cudaMemcpyAsync(om, h_om.data(), sizeof(double) * cnt, cudaMemcpyHostToDevice, c->stream));
    GFCC_CUDA(cudaMemcpyAsync(pf, h_pf.data(), sizeof(double) * cnt, cudaMemcpyHostToDevice, c->stream));
    GFCC_TRY(build_rhs(c, kp.sector, cnt, porb, Bt, c->stream));
    GFCC_TRY(guess_gram(c->stream, cnt, n, Bt, n, kp.X, nbr, delta, om, kp.eta, pf, Gm, feat, work));
    GFCC_CUDA(cudaStreamSynchronize(c->stream));
    GFCC_TRY(append_samples(m, cnt, feat, Gm));
    GFCC_CUDA(cudaStreamSynchronize(m->stream));
    cnt_total += cnt;
    cnt = 0;
    return GFCC_OK;
  };
  for (int w = 0; w < kp.nw && rc == GFCC_OK; w++)
    for (int a = 0; a < kp.norb && rc == GFCC_OK; a++) {
      if (!kp.done[(size_t)w * kp.norb + a]) continue;
      for (int r = 0; r < samples_per_system && rc == GFCC_OK; r++) {
        // neighbours: the 8 nearest among a random subset of the other converged frequencies
        // (keep probability drawn in [0.15, 1)), so that the samples span near and far neighbours
        const double keep = 0.15 + 0.85 * rng.uniform();
        for (int j = 0; j < kp.nw; j++) mask[j] = kp.done[(size_t)j * kp.norb + a] && rng.uniform() < keep;
        int idx[GUESS_K];
        const int k = guess_neighbours(kp.omega, mask.data(), 1, w, GUESS_K, idx);
        if (k < GUESS_K) continue;
        for (int q = 0; q < GUESS_K; q++) {
          h_nbr[cnt * GUESS_K + q] = idx[q] * kp.norb + a;
          h_delta[cnt * GUESS_K + q] = kp.omega[w] - kp.omega[idx[q]];
        }
        h_porb[cnt] = kp.orb[a];
        h_om[cnt] = kp.omega[w];
        h_pf[cnt] = (double)kp.orb[a] / (double)c->n;
        if (++cnt == CB) rc = flush();
      }
    }
  if (rc == GFCC_OK) rc = flush();
  cudaStreamSynchronize(c->stream);
  dfree(tmp);
  if (added) *added = cnt_total;
  return rc;
}

}  // extern "C"
