// Generic strided FP64 tensor contraction on CUDA cores (DFMA).
//
//   C(m, n) = alpha * sum_k A(m, k) B(k, n) + beta * C(m, n),   batched over blockIdx.z
//
// Each GEMM index may fuse two tensor indices through an IMap, so the setup of the
// Hbar elements and the FP64 sigma product are written as plain contractions
// without explicit transposes.  GB300 has about 1.1 TFLOP/s of FP64 (about two
// DFMA per SM and clock), so this kernel is bound by the DFMA pipe: a 64x64 tile
// per 256-thread block with 4x4 outputs per thread keeps the pipe fed while the
// tile loads stay in L1/L2.
#include <map>
#include <mutex>

#include "common.cuh"
#include <algorithm>

#include "kernels.cuh"
#include "ozaki.cuh"

namespace gfcc {

namespace {
constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

__global__ __launch_bounds__(NT) void contract_f64_kernel(Contract c) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const long long b = blockIdx.z / c.nsplit;
  const long long z = blockIdx.z - b * c.nsplit;
  const double *A = c.A + b * c.sab;
  const double *B = c.B + b * c.sbb;
  double *C = c.C + b * c.scb + z * c.scz;
  const long long kbeg = z * c.kchunk;
  const long long kend = min(c.K, kbeg + c.kchunk);
  const long long m0 = (long long)blockIdx.x * BM;
  const long long n0 = (long long)blockIdx.y * BN;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc[i][j] = 0.0;

  for (long long k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int r = 0; r < (BM * BK) / NT; r++) {
      const int e = threadIdx.x + NT * r;
      const int kl = e % BK, ml = e / BK;
      const long long m = m0 + ml, k = k0 + kl;
      As[kl][ml] = (m < c.M && k < kend) ? A[imap_apply(c.am, m) + imap_apply(c.ak, k)] : 0.0;
    }
#pragma unroll
    for (int r = 0; r < (BN * BK) / NT; r++) {
      const int e = threadIdx.x + NT * r;
      const int nl = e % BN, kl = e / BN;
      const long long n = n0 + nl, k = k0 + kl;
      Bs[kl][nl] = (n < c.N && k < kend) ? B[imap_apply(c.bk, k) + imap_apply(c.bn, n)] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk++) {
      double a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; i++) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; j++) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const long long m = m0 + ty + 16 * i;
    if (m >= c.M) continue;
    const long long om = imap_apply(c.cm, m);
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const long long n = n0 + tx + 16 * j;
      if (n >= c.N) continue;
      const long long off = om + imap_apply(c.cn, n);
      double val = c.alpha * acc[i][j];
      if (c.beta != 0.0) val += c.beta * C[off];
      C[off] = val;
    }
  }
}
}  // namespace

int contract_f64(const Contract &c, cudaStream_t st) {
  if (c.M <= 0 || c.N <= 0 || c.batch <= 0) return GFCC_OK;
  // K == 0 leaves acc = 0, so C = beta * C (the empty sum).
  const long long mt = (c.M + BM - 1) / BM, nt = (c.N + BN - 1) / BN;
  Contract cc = c;
  if (cc.nsplit < 1) cc.nsplit = 1;
  if (cc.nsplit == 1) cc.kchunk = cc.K > 0 ? cc.K : 1;
  if (cc.kchunk < 1 || cc.kchunk * cc.nsplit < cc.K) {
    set_error("contract_f64: split-K chunk %lld x %lld does not cover K=%lld", cc.kchunk, cc.nsplit, cc.K);
    return GFCC_ERR_ARG;
  }
  if (mt > 0x7fffffffLL || nt > 65535 || c.batch * cc.nsplit > 65535) {
    set_error("contract_f64: grid too large (M=%lld N=%lld batch=%lld)", c.M, c.N, c.batch);
    return GFCC_ERR_ARG;
  }
  {
    const long long ka = imap_max(c.am, c.M) + imap_max(c.ak, c.K) + (c.batch - 1) * c.sab;
    const long long kb = imap_max(c.bk, c.K) + imap_max(c.bn, c.N) + (c.batch - 1) * c.sbb;
    const long long kc = imap_max(c.cm, c.M) + imap_max(c.cn, c.N) + (c.batch - 1) * c.scb + (cc.nsplit - 1) * cc.scz;
    if (c.K > 0) {
      GFCC_TRY(check_extent(c.A, 0, ka, "contraction operand A"));
      GFCC_TRY(check_extent(c.B, 0, kb, "contraction operand B"));
    }
    GFCC_TRY(check_extent(c.C, 0, kc, "contraction output C"));
  }
  dim3 grid((unsigned)mt, (unsigned)nt, (unsigned)(c.batch * cc.nsplit));
  contract_f64_kernel<<<grid, NT, 0, st>>>(cc);
  GFCC_LAUNCH_CHECK();
  return GFCC_OK;
}

namespace {
// C = alpha * sum_z part[z] + beta * C
__global__ void splitk_reduce_kernel(const double *part, int nsplit, long long M, long long N, double alpha, double beta,
                                     double *C, IMap cm, IMap cn) {
  const long long tot = M * N;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < nsplit; z++) s += part[z * tot + t];
    const long long m = t / N, n = t - m * N;
    const long long off = imap_apply(cm, m) + imap_apply(cn, n);
    C[off] = alpha * s + (beta != 0.0 ? beta * C[off] : 0.0);
  }
}

// split-K partial sums, one buffer per stream (work on a stream is ordered, so a buffer is never
// shared by concurrent contractions)
struct SplitBuf {
  double *p = nullptr;
  long long cap = 0;
};
std::mutex g_splitk_mu;
std::map<cudaStream_t, SplitBuf> g_splitk;
}  // namespace

thread_local bool g_emulate_big = false;
double g_emulate_min_flops = 4e12;
thread_local double g_emulate_min_flops_local = -1.0;

int gemm_f64(cudaStream_t st, long long M, long long N, long long K, double alpha,
             const double *A, IMap am, IMap ak, const double *B, IMap bk, IMap bn, double beta,
             double *C, IMap cm, IMap cn, long long batch, long long sab, long long sbb, long long scb) {
  Contract c;
  c.A = A; c.B = B; c.C = C;
  c.M = M; c.N = N; c.K = K;
  c.am = am; c.ak = ak; c.bk = bk; c.bn = bn; c.cm = cm; c.cn = cn;
  c.batch = batch; c.sab = sab; c.sbb = sbb; c.scb = scb;
  c.alpha = alpha; c.beta = beta;
  // Large contractions (setup of big problems) go to the FP64-accurate digit-plane path on the
  // tensor cores when enabled: at ~1 TFLOP/s of FP64 they would take minutes.
  const double emu_min = g_emulate_min_flops_local >= 0.0 ? g_emulate_min_flops_local : g_emulate_min_flops;
  if (batch == 1 && g_emulate_big && 2.0 * (double)M * (double)N * (double)K >= emu_min)
    return gemm_f64_emulated(st, M, N, K, alpha, A, am, ak, B, bk, bn, beta, C, cm, cn, 8, 9);
  // Few output tiles and a long K would leave most SMs idle: split K into partial sums.
  const long long tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN) * batch;
  if (batch == 1 && tiles < 152 && K >= 8192) {
    long long nsplit = std::min<long long>(std::max<long long>(1, 304 / tiles), K / 2048);
    nsplit = std::min<long long>(nsplit, 512);
    if (nsplit >= 2) {
      const long long need = nsplit * M * N;
      double *buf = nullptr;
      {
        std::lock_guard<std::mutex> lk(g_splitk_mu);
        SplitBuf &sb = g_splitk[st];
        if (need > sb.cap) {
          if (sb.p) dfree(sb.p);   // cudaFree synchronises: earlier work on the buffer is done
          sb.p = nullptr;
          sb.cap = 0;
          if (dmalloc((void **)&sb.p, sizeof(double) * need) != cudaSuccess) {
            cudaGetLastError();
            set_error("gemm_f64: cannot allocate %lld doubles of split-K workspace", need);
            return GFCC_ERR_OOM;
          }
          sb.cap = need;
        }
        buf = sb.p;
      }
      Contract p = c;
      p.C = buf;
      p.cm = imap1(N);
      p.cn = imap1(1);
      p.alpha = 1.0;
      p.beta = 0.0;
      p.nsplit = nsplit;
      p.kchunk = (K + nsplit - 1) / nsplit;
      p.scz = M * N;
      GFCC_TRY(contract_f64(p, st));
      splitk_reduce_kernel<<<grid1d(M * N), 256, 0, st>>>(buf, (int)nsplit, M, N, alpha, beta, C, cm, cn);
      GFCC_LAUNCH_CHECK();
      return GFCC_OK;
    }
  }
  return contract_f64(c, st);
}

}  // namespace gfcc
