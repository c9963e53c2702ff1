// FP64-accurate matrix products on the BF16 tensor cores by exact digit splitting
// (the splitting scheme of Ozaki, Ogita, Oishi & Rump, Numer. Algorithms 59 (2012), with
// fixed-point digits per row).
//
// GB300 runs FP64 at about 1.1 TFLOP/s, three orders of magnitude below its BF16 tensor
// rate.  A row r of an FP64 operand is scaled by a power of two 2^-e_r so that its entries
// lie in (-1/2, 1/2), then written as S base-64 digits
//     a = 2^e_r * sum_{i=1..S} d_i 64^-i + rem,   d_i integer, |d_i| <= 32, |rem| <= 2^e_r 64^-S / 2.
// Digits are exact in BF16 (8 significant bits).  A digit product is an integer of magnitude
// <= 2^10, so a sum of up to 2^14 of them is an integer of magnitude <= 2^24 and the FP32
// accumulation of the tensor cores is exact.  The product of two operands is then
//     sum_k A[m][k] B[n][k] = 2^(e_m + f_n) sum_{i,j} 64^-(i+j) sum_k dA_i[m][k] dB_j[n][k]
// and the digit-pair products with i + j <= P are evaluated as BF16 GEMMs (K split into
// chunks of 2^14 with separate FP32 partial sums) and combined in FP64.  The truncation
// error per term is bounded by about 2^-(6P-4) of 2^(e_m + f_n); P = S + 1.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"
#include "ozaki.cuh"
#include "umma.cuh"

namespace gfcc {

// products with at most this many columns take the fused kernel (all digit pairs of a tile in one
// CTA, levels in TMEM); wider ones keep one GEMM per digit pair (256-column tiles)
long long g_fused_max_n = 512;

namespace {

constexpr int KCHUNK_BLOCKS = (1 << 14) / 64;   // K blocks (of 64) per exact partial sum

// e[r] such that max_k |A[r][k]| * 2^-e[r] lies in [1/4, 1/2); rows of zeros get 0
__global__ void rowexp_kernel(const double *A, long long rows, long long K, long long lda, int *e) {
  __shared__ double sh[32];
  const long long r = blockIdx.x;
  if (r >= rows) return;
  double mx = 0.0;
  for (long long k = threadIdx.x; k < K; k += blockDim.x) mx = fmax(mx, fabs(A[r * lda + k]));
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) mx = fmax(mx, sh[w]);
    int E = 0;
    if (mx > 0.0) frexp(mx, &E);   // mx = f 2^E, f in [1/2, 1)
    e[r] = mx > 0.0 ? E + 1 : 0;
  }
}

// dig[i][r][k] = i-th base-64 digit of A[r][k] 2^-e[r] (k < K), 0 for K <= k < ld
__global__ void slice_kernel(const double *A, long long rows, long long K, long long lda, const int *e, int S,
                             __nv_bfloat16 *dig, long long ld) {
  const long long tot = rows * ld;
  const long long plane = rows * ld;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const long long r = t / ld, k = t - r * ld;
    long long Y = k < K ? fixed_point(A[r * lda + k], e[r], 6 * S) : 0;
    for (int i = 0; i < S; i++) {
      const int sh = 6 * (S - 1 - i);
      const long long d = sh > 0 ? (Y + (1LL << (sh - 1))) >> sh : Y;
      Y -= d << sh;
      dig[i * plane + t] = __float2bfloat16((float)(int)d);
    }
  }
}

// Exact integer accumulation of digit-pair products: the FP32 partial sums are integers of
// magnitude <= 2^24, so they convert to int32 exactly; a pair of level L adds (sum_z part) shifted
// by 6 (Lhi - L) into the high accumulator (levels <= Lsplit) or by 6 (P - L) into the low one.
// The two int64 accumulators are separate planes, acc[t] = high and acc[tot + t] = low, so that a
// combine touches only its own; the first combine into a plane sets it.  No FP64 arithmetic.
__global__ void combine_int_kernel(const float *part, int nz, long long tot, int shift, int which, long long *acc,
                                   int first) {
  long long *a = acc + (which ? tot : 0);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    long long s = 0;
    for (int z = 0; z < nz; z++) s += (long long)__float2int_rn(part[(long long)z * tot + t]);
    s <<= shift;
    a[t] = first ? s : a[t] + s;
  }
}
// C = alpha * (high 2^(ex - 6 Lhi) + low 2^(ex - 6 P)) + beta C, ex = eA[m] + eB[n].  Grid
// (cdiv(N, 256), rows): a block walks rows m = blockIdx.y, blockIdx.y + gridDim.y, ...
__global__ void finalize_kernel(const long long *acc, long long M, long long N, const int *eA, const int *eB,
                                int Lhi, int P, double alpha, double beta, double *C, IMap cm, IMap cn, long long n0) {
  const long long tot = M * N;
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int eb = eB[n];
  const long long offn = imap_apply(cn, n0 + n);
  for (long long m = blockIdx.y; m < M; m += gridDim.y) {
    const long long t = m * N + n;
    const int ex = eA[m] + eb;
    double val = scalbn((double)acc[t], ex - 6 * Lhi);
    if (P > Lhi) val += scalbn((double)acc[tot + t], ex - 6 * P);
    const long long off = imap_apply(cm, m) + offn;
    const double v = alpha * val;
    C[off] = beta != 0.0 ? v + beta * C[off] : v;
  }
}

}  // namespace

long long emu_operand_bytes(long long rows, long long K, int S) {
  const long long ld = (K + 7) / 8 * 8;
  return (long long)S * rows * ld * 2 + ((rows * 4 + 255) / 256) * 256 + 256;
}

int emu_slice(cudaStream_t st, const double *A, long long rows, long long K, long long lda, int S, void *mem,
              EmuOperand &out) {
  out.rows = rows;
  out.K = K;
  out.ld = (K + 7) / 8 * 8;
  out.S = S;
  unsigned char *p = static_cast<unsigned char *>(mem);
  out.dig = reinterpret_cast<__nv_bfloat16 *>(p);
  p += ((long long)S * rows * out.ld * 2 + 255) / 256 * 256;
  out.exp2 = reinterpret_cast<int *>(p);
  if (rows <= 0 || K <= 0) return GFCC_OK;
  GFCC_TRY(check_extent(A, 0, (rows - 1) * lda + K - 1, "digit split input"));
  GFCC_TRY(check_extent_bytes(mem, emu_operand_bytes(rows, K, S), "digit split output"));
  if (rows > 0x7fffffffLL) {
    set_error("emu_slice: too many rows (%lld)", rows);
    return GFCC_ERR_ARG;
  }
  rowexp_kernel<<<(unsigned)rows, 256, 0, st>>>(A, rows, K, lda, out.exp2);
  GFCC_LAUNCH_CHECK();
  slice_kernel<<<grid1d(rows * out.ld), 256, 0, st>>>(A, rows, K, lda, out.exp2, S, out.dig, out.ld);
  GFCC_LAUNCH_CHECK();
  return GFCC_OK;
}

// The digit pairs of one level L = i + j share a weight, so several of them can accumulate in the
// same FP32 partial sums (beta = 1) while the sums stay exact integers: a partial over kbs K blocks
// of 64 holds up to KCHUNK_BLOCKS / kbs pairs (2^14 digit products of magnitude <= 2^10).  The K
// split is the one of a single pair; pairs are grouped within that bound, one integer combine per
// group.
long long emu_gemm_work_bytes(long long M, long long N, long long K) {
  const long long nk = (K + 63) / 64;
  const long long nz = (nk + KCHUNK_BLOCKS - 1) / KCHUNK_BLOCKS;
  return std::max(nz * M * N * 4 + M * N * 16 + 512, emu_fused_work_bytes(M, N, K));
}

void emu_set_fused_max_n(long long n) { g_fused_max_n = n; }

namespace {
__global__ void max_int_kernel(const int *x, long long n, int *out) {
  int m = -(1 << 30);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    m = max(m, x[t]);
  for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}
}  // namespace

int emu_max_exponent(cudaStream_t st, const EmuOperand &e, int *out) {
  int *d = nullptr;
  const int init = -(1 << 30);
  GFCC_CUDA(cudaMalloc(&d, sizeof(int)));
  GFCC_CUDA(cudaMemcpyAsync(d, &init, sizeof(int), cudaMemcpyHostToDevice, st));
  max_int_kernel<<<grid1d(e.rows), 256, 0, st>>>(e.exp2, e.rows, d);
  cudaError_t er = cudaGetLastError();
  count_launch();
  if (er == cudaSuccess) er = cudaMemcpyAsync(out, d, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (er == cudaSuccess) er = cudaStreamSynchronize(st);
  cudaFree(d);
  if (er != cudaSuccess) {
    set_error("emu_max_exponent: %s", cudaGetErrorString(er));
    return GFCC_ERR_CUDA;
  }
  return GFCC_OK;
}

int emu_gemm(cudaStream_t st, const EmuOperand &A, const EmuOperand &B, int P, double alpha, double beta, double *C,
             IMap cm, IMap cn, void *work, long long n0) {
  P = std::max(2, P - A.drop);
  const long long M = A.rows, N = B.rows, K = A.K;
  if (M <= 0 || N <= 0) return GFCC_OK;
  if (B.K != K || A.ld != B.ld) {
    set_error("emu_gemm: operands disagree in K (%lld vs %lld)", A.K, B.K);
    return GFCC_ERR_ARG;
  }
  if (N <= g_fused_max_n && A.S <= 8 && B.S <= 8 && P <= 9 && M <= (1LL << 31) - 1)
    return emu_gemm_fused(st, A.dig, A.rows * A.ld, A.S, A.exp2, B.dig, B.rows * B.ld, B.S, B.exp2, A.ld, (int)M,
                          (int)N, (int)K, P, alpha, beta, C, cm, cn, n0, static_cast<double *>(work));
  const long long nk = (K + 63) / 64;
  const int nz = (int)((nk + KCHUNK_BLOCKS - 1) / KCHUNK_BLOCKS);
  const long long kbs = (nk + nz - 1) / nz;
  const int group = (int)std::max<long long>(1, KCHUNK_BLOCKS / kbs);   // pairs per exact partial
  float *part = static_cast<float *>(work);
  long long *acc =
      reinterpret_cast<long long *>(static_cast<unsigned char *>(work) + ((nz * M * N * 4 + 255) / 256) * 256);
  GFCC_TRY(check_extent_bytes(work, emu_gemm_work_bytes(M, N, K), "digit GEMM workspace"));
  GFCC_TRY(check_extent(C, 0, imap_max(cm, M) + imap_max(cn, n0 + N), "digit GEMM output"));
  const long long plA = A.rows * A.ld, plB = B.rows * B.ld;
  // two exact int64 accumulators: levels 2..Lhi (weights 64^(Lhi-L)) and Lhi+1..P (64^(P-L));
  // a group sum is below nz 2^24 < 2^33 (and a level holds at most S groups), so 4 levels of 6-bit
  // shifts stay below 2^63
  const int Lhi = std::min(P, 5);
  if (P - Lhi > 4 || nz > (1 << 16)) {
    set_error("emu_gemm: level %d or K %lld beyond the exact integer accumulation", P, K);
    return GFCC_ERR_ARG;
  }
  bool first = true, first_plane[2] = {true, true};
  for (int L = P; L >= 2; L--) {
    const int which = L <= Lhi ? 0 : 1;
    const int shift = which == 0 ? 6 * (Lhi - L) : 6 * (P - L);
    int in_group = 0;
    for (int i = 1; i <= A.S; i++) {
      const int j = L - i;
      if (j < 1 || j > B.S) continue;
      GFCC_TRY(gemm_bf16_tn(st, A.dig + (long long)(i - 1) * plA, A.ld, B.dig + (long long)(j - 1) * plB, B.ld, part,
                            N, (int)M, (int)N, (int)K, 1.0f, in_group == 0 ? 0.0f : 1.0f, nz, M * N));
      in_group++;
      // last pair of the level or a full group: fold the partials into the integer accumulators
      bool last = true;
      for (int i2 = i + 1; i2 <= A.S; i2++)
        if (L - i2 >= 1 && L - i2 <= B.S) last = false;
      if (in_group == group || last) {
        combine_int_kernel<<<grid1d(M * N), 256, 0, st>>>(part, umma_splits((int)K, nz), M * N, shift, which, acc,
                                                           first_plane[which] ? 1 : 0);
        GFCC_LAUNCH_CHECK();
        first = false;
        first_plane[which] = false;
        in_group = 0;
      }
    }
  }
  if (first) GFCC_CUDA(cudaMemsetAsync(acc, 0, sizeof(long long) * 2 * M * N, st));
  finalize_kernel<<<dim3(cdiv(N, 256), (unsigned)std::min<long long>(M, 8192)), 256, 0, st>>>(
      acc, M, N, A.exp2, B.exp2, Lhi, P, alpha, beta, C, cm, cn, n0);
  GFCC_LAUNCH_CHECK();
  return GFCC_OK;
}

namespace {
// G[r][k] = X[imap(rm, r) + imap(km, k)] for k < K, 0 for K <= k < ld
__global__ void gather_kernel(const double *X, long long rows, long long K, long long ld, IMap rm, IMap km, long long r0,
                              double *G) {
  const long long tot = rows * ld;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const long long r = t / ld, k = t - r * ld;
    G[t] = k < K ? X[imap_apply(rm, r0 + r) + imap_apply(km, k)] : 0.0;
  }
}
}  // namespace

int gemm_f64_emulated(cudaStream_t st, long long M, long long N, long long K, double alpha, const double *A, IMap am,
                      IMap ak, const double *B, IMap bk, IMap bn, double beta, double *C, IMap cm, IMap cn, int S,
                      int P) {
  if (M <= 0 || N <= 0) return GFCC_OK;
  GFCC_TRY(check_extent(A, 0, imap_max(am, M) + imap_max(ak, K), "emulated contraction operand A"));
  GFCC_TRY(check_extent(B, 0, imap_max(bk, K) + imap_max(bn, N), "emulated contraction operand B"));
  GFCC_TRY(check_extent(C, 0, imap_max(cm, M) + imap_max(cn, N), "emulated contraction output C"));
  const long long ld = (K + 7) / 8 * 8;
  // column blocks of B / C sized so that one pass stays within about 12 GB of temporaries
  const long long budget = 12LL << 30;
  const long long nk = (K + 63) / 64, nz = (nk + KCHUNK_BLOCKS - 1) / KCHUNK_BLOCKS;
  const long long per_col = ld * 8 + (long long)S * ld * 2 + nz * M * 4 + M * 8;
  long long nb = std::max<long long>(256, budget / std::max<long long>(per_col, 1));
  nb = std::min(nb, N);
  void *ag = nullptr, *adig = nullptr, *bg = nullptr, *bdig = nullptr, *w = nullptr;
  int s = GFCC_OK;
  if (dmalloc(&ag, sizeof(double) * M * ld) != cudaSuccess || dmalloc(&adig, emu_operand_bytes(M, K, S)) != cudaSuccess ||
      dmalloc(&bg, sizeof(double) * nb * ld) != cudaSuccess || dmalloc(&bdig, emu_operand_bytes(nb, K, S)) != cudaSuccess ||
      dmalloc(&w, emu_gemm_work_bytes(M, nb, K)) != cudaSuccess) {
    cudaGetLastError();
    set_error("emulated contraction: cannot allocate its temporaries (M=%lld N-block=%lld K=%lld)", M, nb, K);
    s = GFCC_ERR_OOM;
  }
  EmuOperand ea, eb;
  if (s == GFCC_OK) {
    gather_kernel<<<grid1d(M * ld), 256, 0, st>>>(A, M, K, ld, am, ak, 0, static_cast<double *>(ag));
    if (cudaGetLastError() != cudaSuccess) s = GFCC_ERR_CUDA;
    count_launch();
  }
  if (s == GFCC_OK) s = emu_slice(st, static_cast<double *>(ag), M, K, ld, S, adig, ea);
  for (long long n0 = 0; n0 < N && s == GFCC_OK; n0 += nb) {
    const long long cols = std::min(nb, N - n0);
    gather_kernel<<<grid1d(cols * ld), 256, 0, st>>>(B, cols, K, ld, bn, bk, n0, static_cast<double *>(bg));
    count_launch();
    if (cudaGetLastError() != cudaSuccess) {
      s = GFCC_ERR_CUDA;
      break;
    }
    s = emu_slice(st, static_cast<double *>(bg), cols, K, ld, S, bdig, eb);
    if (s == GFCC_OK) s = emu_gemm(st, ea, eb, P, alpha, beta, C, cm, cn, w, n0);
  }
  if (s == GFCC_OK && cudaStreamSynchronize(st) != cudaSuccess) {
    set_error("emulated contraction failed: %s", cudaGetErrorString(cudaGetLastError()));
    s = GFCC_ERR_CUDA;
  }
  for (void *p : {ag, adig, bg, bdig, w}) dfree(p);
  return s;
}

int gemm_f64_emulated_pre(cudaStream_t st, const EmuOperand &A, long long N, const double *B, IMap bk, IMap bn,
                          double alpha, double beta, double *C, IMap cm, IMap cn, int P) {
  const long long M = A.rows, K = A.K, S = A.S;
  if (M <= 0 || N <= 0) return GFCC_OK;
  GFCC_TRY(check_extent(B, 0, imap_max(bk, K) + imap_max(bn, N), "emulated contraction operand B"));
  GFCC_TRY(check_extent(C, 0, imap_max(cm, M) + imap_max(cn, N), "emulated contraction output C"));
  const long long ld = (K + 7) / 8 * 8;
  if (A.ld != ld) {
    set_error("emulated contraction: the sliced operand's row stride %lld is not %lld", A.ld, ld);
    return GFCC_ERR_ARG;
  }
  const long long budget = 12LL << 30;
  const long long nk = (K + 63) / 64, nz = (nk + KCHUNK_BLOCKS - 1) / KCHUNK_BLOCKS;
  const long long per_col = ld * 8 + S * ld * 2 + nz * M * 4 + M * 8;
  long long nb = std::max<long long>(256, budget / std::max<long long>(per_col, 1));
  nb = std::min(nb, N);
  void *bg = nullptr, *bdig = nullptr, *w = nullptr;
  int s = GFCC_OK;
  if (dmalloc(&bg, sizeof(double) * nb * ld) != cudaSuccess || dmalloc(&bdig, emu_operand_bytes(nb, K, (int)S)) != cudaSuccess ||
      dmalloc(&w, emu_gemm_work_bytes(M, nb, K)) != cudaSuccess) {
    cudaGetLastError();
    set_error("emulated contraction: cannot allocate its temporaries (M=%lld N-block=%lld K=%lld)", M, nb, K);
    s = GFCC_ERR_OOM;
  }
  EmuOperand eb;
  for (long long n0 = 0; n0 < N && s == GFCC_OK; n0 += nb) {
    const long long cols = std::min(nb, N - n0);
    gather_kernel<<<grid1d(cols * ld), 256, 0, st>>>(B, cols, K, ld, bn, bk, n0, static_cast<double *>(bg));
    count_launch();
    if (cudaGetLastError() != cudaSuccess) {
      s = GFCC_ERR_CUDA;
      break;
    }
    s = emu_slice(st, static_cast<double *>(bg), cols, K, ld, (int)S, bdig, eb);
    if (s == GFCC_OK) s = emu_gemm(st, A, eb, P, alpha, beta, C, cm, cn, w, n0);
  }
  if (s == GFCC_OK && cudaStreamSynchronize(st) != cudaSuccess) {
    set_error("emulated contraction failed: %s", cudaGetErrorString(cudaGetLastError()));
    s = GFCC_ERR_CUDA;
  }
  for (void *q : {bg, bdig, w}) dfree(q);
  return s;
}

}  // namespace gfcc
