// Mixed-precision IP operator: the off-diagonal part of the sigma product on the BF16 tensor
// cores (FP32 accumulation), the Fock-like diagonal and the frequency shift in FP64.
//
//   sigma(u) = d * u + sigma_off(u),   d_i = -Fbar_ii,  d_ija = Fbar_aa - Fbar_ii - Fbar_jj
//   A u = (omega - i eta) u + sigma(u) = D u + sigma_off(u),   D = omega - i eta + d
//
// With right preconditioning by D (u = x / D) the operator is x + sigma_off(x / D).  The
// diagonal carries the orbital energies (order 1 Hartree); rounding it to BF16 would put an
// error of the size of eta on every resonant system, so it never leaves FP64.  The couplings
// (ring, oooo, ovoo, three-body, off-diagonal Fbar) are small and tolerate BF16 operands:
// the refinement loop recomputes the residual in FP64 and removes their rounding error.
//
// Contractions (all D[m][n] = A[m][k] B[n][k], BF16 K-major, FP32 out):
//   ring  T[(i,a)][(j,c)]  = Wr[(i,a)][(m,e)]   r2b[(j,c)][(m,e)],  r2b = r2[m,j,e]
//   oooo  Q[(i,j)][(a,c)]  = Wq[(i,j)][(m,n)]   r2o[(a,c)][(m,n)],  r2o = r2[m,n,a]
//   ovoo  U[(i,a,j)][c]    = W1[(i,a,j)][m]     r1b[c][m]
//   3-body Z[e][c]         = V3[e][(m,f,n)]     rk[c][(m,f,n)]       (split K)
//          U             += T3[(i,a,j)][e]     Zb[c][e]
//   1h    S1[i][c]         = U1x[i][(m,e,n)|m]  rk[c][(m,e,n)|m]     (split K)
#include <cuda_bf16.h>

#include "ctx.cuh"
#include "kernels.cuh"
#include "sigma.cuh"
#include "umma.cuh"

namespace gfcc {

namespace {

// The BF16 operands only need FP32 accuracy: the vector (and the preconditioner division) is
// handled in FP32 on the FP32 pipe.
struct Cz {
  float r, i;
};

__device__ __forceinline__ Cz load_u(const SysBatch &b, int s, long long mu) {
  Cz u{d2f_trunc(b.x[2 * (s * b.ldx + mu)]), d2f_trunc(b.x[2 * (s * b.ldx + mu) + 1])};
  if (b.diag != nullptr && b.omega != nullptr) {
    const float dr = d2f_trunc(b.omega[s]) + (float)b.dsign * d2f_trunc(b.diag[mu]);
    const float di = (float)b.zsign * d2f_trunc(b.eta);
    const float inv = 1.0f / (dr * dr + di * di);
    u = {(u.r * dr + u.i * di) * inv, (u.i * dr - u.r * di) * inv};
  }
  return u;
}

// r2[m, j, e] of system s as (re, im); zero on the diagonal m == j
__device__ __forceinline__ Cz r2_at(const SysBatch &b, int o, int v, int s, int m, int j, int e) {
  if (m == j) return {0.0f, 0.0f};
  const long long lo = m < j ? m : j, hi = m < j ? j : m;
  const long long mu = o + pair_index(lo, hi, o) * v + e;
  Cz u = load_u(b, s, mu);
  if (m > j) {
    u.r = -u.r;
    u.i = -u.i;
  }
  return u;
}

// r2b[(j, c)][(m, e)] = r2[m, j, e]
__global__ void unpack_ring_kernel(SysBatch b, int o, int v, long long ld, __nv_bfloat16 *out) {
  const int ns = b.nsys;
  const long long K = (long long)o * v;
  const long long tot = (long long)o * 2 * ns * K;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const long long k = t % K, row = t / K;
    const int c = (int)(row % (2 * ns)), j = (int)(row / (2 * ns));
    const int m = (int)(k / v), e = (int)(k % v);
    const Cz u = r2_at(b, o, v, c >> 1, m, j, e);
    out[row * ld + k] = __float2bfloat16((c & 1) ? u.i : u.r);
  }
}

// r2o[(a, c)][(m, n)] = r2[m, n, a]: a 32 x 32 tile transpose through shared memory (reads
// coalesced along a, writes coalesced along (m, n)).  grid (K/32, v/32, C2), block (32, 8).
__global__ void unpack_oooo_kernel(SysBatch b, int o, int v, long long ld, __nv_bfloat16 *out) {
  __shared__ float tile[32][33];
  const int C2 = 2 * b.nsys;
  const long long K = (long long)o * o;
  const int c = blockIdx.z, s = c >> 1;
  const long long k0 = (long long)blockIdx.x * 32;
  const int a0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const long long k = k0 + r;
    const int a = a0 + threadIdx.x;
    float val = 0.f;
    if (k < K && a < v) {
      const Cz u = r2_at(b, o, v, s, (int)(k / o), (int)(k % o), a);
      val = (c & 1) ? u.i : u.r;
    }
    tile[r][threadIdx.x] = val;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int a = a0 + r;
    const long long k = k0 + threadIdx.x;
    if (a < v && k < K) out[((long long)a * C2 + c) * ld + k] = __float2bfloat16(tile[threadIdx.x][r]);
  }
}

// rk[c][(m, e, n)] = r2[m, n, e] (tile transpose over (e, n) for fixed m, c: reads coalesced along
// e, writes along n); grid (o/32, v/32, o * C2), block (32, 8)
__global__ void unpack_k_tiled_kernel(SysBatch b, int o, int v, long long ldk, __nv_bfloat16 *rk) {
  __shared__ float tile[32][33];
  const int C2 = 2 * b.nsys;
  const int c = blockIdx.z % C2, m = blockIdx.z / C2, s = c >> 1;
  const int n0 = blockIdx.x * 32, e0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int n = n0 + r, e = e0 + threadIdx.x;
    float val = 0.f;
    if (n < o && e < v) {
      const Cz u = r2_at(b, o, v, s, m, n, e);
      val = (c & 1) ? u.i : u.r;
    }
    tile[r][threadIdx.x] = val;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int e = e0 + r, n = n0 + threadIdx.x;
    if (e < v && n < o) rk[(long long)c * ldk + ((long long)m * v + e) * o + n] = __float2bfloat16(tile[threadIdx.x][r]);
  }
}

// rk[c][o2v + m] = r1[m] and r1b[c][m] = r1[m]
__global__ void unpack_r1_kernel(SysBatch b, int o, int v, long long ldk, __nv_bfloat16 *rk, long long ld1,
                                 __nv_bfloat16 *r1b) {
  const long long o2v = (long long)o * o * v;
  const int C2 = 2 * b.nsys;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= C2 * o) return;
  const int c = t / o, m = t % o;
  const Cz u = load_u(b, c >> 1, m);
  const __nv_bfloat16 h = __float2bfloat16((c & 1) ? u.i : u.r);
  rk[(long long)c * ldk + o2v + m] = h;
  r1b[(long long)c * ld1 + m] = h;
}

// out[r][c] = sum_z part[z][r][c] (in place into part[0]); optional BF16 transposed copy outT[c][r]
__global__ void reduce_splits_kernel(float *part, int nsplit, long long rows, long long cols, long long zstride,
                                     __nv_bfloat16 *outT, long long ldT) {
  const long long tot = rows * cols;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    float s = part[t];
    for (int z = 1; z < nsplit; z++) s += part[z * zstride + t];
    part[t] = s;
    if (outT != nullptr) {
      const long long r = t / cols, c = t % cols;
      outT[c * ldT + r] = __float2bfloat16(s);
    }
  }
}

__global__ void epilogue_ip_mixed_kernel(SysBatch b, int o, int v, long long C2, long long dim, const double *diag,
                                         const float *S1, const float *T, const float *Q, const float *U) {
  const int ns = b.nsys;
  const long long tot = dim * ns;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const long long mu = t % dim;
    const int s = (int)(t / dim);
    double sr, si;
    if (mu < o) {
      sr = S1[mu * C2 + 2 * s];
      si = S1[mu * C2 + 2 * s + 1];
    } else {
      const long long r = mu - o;
      const long long a = r % v;
      long long i, j;
      pair_decode(r / v, o, i, j);
      const long long tij = ((i * v + a) * o + j) * C2 + 2 * s;
      const long long tji = ((j * v + a) * o + i) * C2 + 2 * s;
      const long long qij = ((i * o + j) * v + a) * C2 + 2 * s;
      sr = (double)T[tij] - (double)T[tji] + (double)Q[qij] + (double)U[tij];
      si = (double)T[tij + 1] - (double)T[tji + 1] + (double)Q[qij + 1] + (double)U[tij + 1];
    }
    const double xr = b.x[2 * (s * b.ldx + mu)], xi = b.x[2 * (s * b.ldx + mu) + 1];
    double yr, yi;
    if (b.omega == nullptr) {            // sigma(x) = d x + sigma_off(x)
      yr = diag[mu] * xr + sr;
      yi = diag[mu] * xi + si;
    } else if (b.diag != nullptr) {      // right-preconditioned: D u = x
      yr = xr + sr;
      yi = xi + si;
    } else {                             // (omega - i eta + d) x + sigma_off(x)
      const double dr = b.omega[s] + diag[mu], di = -b.eta;
      yr = dr * xr - di * xi + sr;
      yi = dr * xi + di * xr + si;
    }
    b.y[2 * (s * b.ldy + mu)] = yr;
    b.y[2 * (s * b.ldy + mu) + 1] = yi;
  }
}

constexpr int KSPLIT = 64;   // split of the long-K contractions (Z, 1h row) into partial sums

struct MixedWork {
  __nv_bfloat16 *r2b, *r2o, *rk, *r1b, *Zb;
  float *T, *Q, *U, *Zp, *S1p;
  long long bytes;
};

MixedWork layout(const gfcc_ctx *c, int nsys, void *base) {
  const long long o = c->o, v = c->v, C2 = 2LL * nsys;
  MixedWork w;
  unsigned char *p = static_cast<unsigned char *>(base);
  auto take = [&](long long bytes) {
    unsigned char *q = p;
    p += (bytes + 255) / 256 * 256;
    return q;
  };
  w.r2b = reinterpret_cast<__nv_bfloat16 *>(take(o * C2 * c->ld_ov * 2));
  w.r2o = reinterpret_cast<__nv_bfloat16 *>(take(v * C2 * c->ld_o2 * 2));
  w.rk = reinterpret_cast<__nv_bfloat16 *>(take(C2 * c->ld_k1 * 2));
  w.r1b = reinterpret_cast<__nv_bfloat16 *>(take(C2 * c->ld_o * 2));
  w.Zb = reinterpret_cast<__nv_bfloat16 *>(take(C2 * c->ld_v * 2));
  w.T = reinterpret_cast<float *>(take(o * v * o * C2 * 4));
  w.Q = reinterpret_cast<float *>(take(o * o * v * C2 * 4));
  w.U = reinterpret_cast<float *>(take(o * v * o * C2 * 4));
  w.Zp = reinterpret_cast<float *>(take(KSPLIT * v * C2 * 4));
  w.S1p = reinterpret_cast<float *>(take(KSPLIT * o * C2 * 4));
  w.bytes = p - static_cast<unsigned char *>(base);
  return w;
}

}  // namespace

long long sigma_mixed_work_doubles(const gfcc_ctx *c, int nsys) {
  return layout(c, nsys, nullptr).bytes / 8 + 64;
}

int apply_ip_mixed(gfcc_ctx *c, const SysBatch &b, double *work) {
  if (c->Wr_bf == nullptr) {
    set_error("mixed-precision sigma requested but the context was created in FP64");
    return GFCC_ERR_STATE;
  }
  cudaStream_t st = c->stream;
  const long long o = c->o, v = c->v, ov = o * v, oo = o * o, o2v = oo * v, C2 = 2LL * b.nsys;
  MixedWork w = layout(c, b.nsys, work);
  PhaseTimer tsig(c, PH_SIGMA, b.nsys * sigma_flops(c, GFCC_SECTOR_IP));
  {
  PhaseTimer tu(c, PH_UNPACK);
  unpack_ring_kernel<<<grid1d(o * C2 * ov), 256, 0, st>>>(b, (int)o, (int)v, c->ld_ov, w.r2b);
  GFCC_LAUNCH_CHECK();
  unpack_oooo_kernel<<<dim3(cdiv(oo, 32), cdiv(v, 32), C2), dim3(32, 8), 0, st>>>(b, (int)o, (int)v, c->ld_o2,
                                                                                   w.r2o);
  GFCC_LAUNCH_CHECK();
  unpack_k_tiled_kernel<<<dim3(cdiv(o, 32), cdiv(v, 32), o * C2), dim3(32, 8), 0, st>>>(b, (int)o, (int)v, c->ld_k1,
                                                                                        w.rk);
  GFCC_LAUNCH_CHECK();
  unpack_r1_kernel<<<cdiv(C2 * o, 128), 128, 0, st>>>(b, (int)o, (int)v, c->ld_k1, w.rk, c->ld_o, w.r1b);
  GFCC_LAUNCH_CHECK();
  }
  {
    PhaseTimer tr(c, PH_RING_BF16, 2.0 * (double)ov * (double)ov * (double)(o * C2));
    GFCC_TRY(gemm_bf16_tn(st, c->Wr_bf, c->ld_ov, w.r2b, c->ld_ov, w.T, o * C2, (int)ov, (int)(o * C2), (int)ov, 1.0f,
                          0.0f));
  }
  GFCC_TRY(gemm_bf16_tn(st, c->Wq_bf, c->ld_o2, w.r2o, c->ld_o2, w.Q, v * C2, (int)oo, (int)(v * C2), (int)oo, 1.0f,
                        0.0f));
  GFCC_TRY(gemm_bf16_tn(st, c->W1_bf, c->ld_o, w.r1b, c->ld_o, w.U, C2, (int)o2v, (int)C2, (int)o, 1.0f, 0.0f));
  // three-body: Z (split K) -> BF16 transposed -> U += T3 Z
  const int zs = umma_splits((int)o2v, KSPLIT);
  GFCC_TRY(gemm_bf16_tn(st, c->V3_bf, c->ld_o2v, w.rk, c->ld_k1, w.Zp, C2, (int)v, (int)C2, (int)o2v, 1.0f, 0.0f, zs,
                        v * C2));
  reduce_splits_kernel<<<grid1d(v * C2), 256, 0, st>>>(w.Zp, zs, v, C2, v * C2, w.Zb, c->ld_v);
  GFCC_LAUNCH_CHECK();
  GFCC_TRY(gemm_bf16_tn(st, c->T3_bf, c->ld_v, w.Zb, c->ld_v, w.U, C2, (int)o2v, (int)C2, (int)v, 1.0f, 1.0f));
  // 1h row (split K)
  const int ss = umma_splits((int)(o2v + o), KSPLIT);
  GFCC_TRY(gemm_bf16_tn(st, c->U1_bf, c->ld_k1, w.rk, c->ld_k1, w.S1p, C2, (int)o, (int)C2, (int)(o2v + o), 1.0f, 0.0f,
                        ss, o * C2));
  reduce_splits_kernel<<<grid1d(o * C2), 256, 0, st>>>(w.S1p, ss, o, C2, o * C2, nullptr, 0);
  GFCC_LAUNCH_CHECK();
  epilogue_ip_mixed_kernel<<<grid1d(c->dim_ip * b.nsys), 256, 0, st>>>(b, (int)o, (int)v, C2, c->dim_ip, c->diag_ip,
                                                                       w.S1p, w.T, w.Q, w.U);
  GFCC_LAUNCH_CHECK();
  return GFCC_OK;
}

}  // namespace gfcc
