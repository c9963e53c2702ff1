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
//   3-body Z[e][c]         = V3[e][(m,f,n)]     rk[c][(m,f,n)]       (split K)
//   ovoo + 3-body
//         U[(i,a,j)][c]    = [W1 | T3][(i,a,j)][m | e]  rz[c][m | e],  rz = [r1 | Z]
//   1h    S1[i][c]         = U1x[i][(m,e,n)|m]  rk[c][(m,e,n)|m]     (split K)
#include <cuda_bf16.h>

#include "ctx.cuh"
#include "kernels.cuh"
#include "sigma.cuh"
#include "umma.cuh"
#include "epilogue.cuh"

namespace gfcc {

namespace {

// The BF16 operands only need FP32 accuracy: the vector (and the preconditioner division) is
// handled in FP32 on the FP32 pipe.
struct Cz {
  float r, i;
};

__device__ __forceinline__ Cz load_u(const SysBatch &b, int s, long long mu) {
  s = sysv(b, s);
  Cz u;
  if (b.xf != nullptr) {
    const float2 t = reinterpret_cast<const float2 *>(b.xf)[s * b.ldx + mu];
    u = {t.x, t.y};
  } else {
    u = {d2f_trunc(b.x[2 * (s * b.ldx + mu)]), d2f_trunc(b.x[2 * (s * b.ldx + mu) + 1])};
  }
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

// All three 2h1p layouts in one pass.  One block per (e tile, m, system s): the tile r2[m, j, e]
// of system s for every j (each packed element is read by the blocks of its two occupied indices;
// the right preconditioner is applied once per read), then
//   ring   r2b[(j, c)][(m, e)]  rows of the tile's e range,
//   oooo   r2o[(e, c)][(m, j)]  rows of o consecutive columns,
//   long K rk[c][(m, e, j)]     one contiguous run of (e range) x o columns,
// for both planes c = 2 s + re/im.  Quotients by o come from a 32.32 fixed-point reciprocal
// (exact while the dividend stays below 2^32 / o; here below 2 UNPACK_ET o).
constexpr int UNPACK_ET = 32;   // e values per block (a power of two)
constexpr int UNPACK_MAX_O = 180;   // tile o x (UNPACK_ET + 1) float2 within the default 48 KB

__device__ __forceinline__ int quo(unsigned q, unsigned long long rcp) {
  return (int)(((unsigned long long)q * rcp) >> 32);
}

__global__ __launch_bounds__(256) void unpack_ip_kernel(SysBatch b, int o, int v, unsigned long long rcp_o,
                                                        long long ld_ov, long long ld_o2, long long ld_k1,
                                                        __nv_bfloat16 *r2b, __nv_bfloat16 *r2o, __nv_bfloat16 *rk) {
  extern __shared__ float2 tl[];   // [o][UNPACK_ET + 1]
  constexpr int LD = UNPACK_ET + 1;
  const int e0 = blockIdx.x * UNPACK_ET, m = blockIdx.y, s = blockIdx.z;
  const int et = min(UNPACK_ET, v - e0);
  const int C2 = 2 * b.nsys;
  for (int t = threadIdx.x; t < o * UNPACK_ET; t += blockDim.x) {
    const int j = t / UNPACK_ET, el = t % UNPACK_ET;
    float2 val = make_float2(0.f, 0.f);
    if (el < et) {
      const Cz u = r2_at(b, o, v, s, m, j, e0 + el);
      val = make_float2(u.r, u.i);
    }
    tl[j * LD + el] = val;
  }
  __syncthreads();
  // ring: rows (j, 2 s + p), columns m v + e0 .. m v + e0 + et
  for (int t = threadIdx.x; t < 2 * o * UNPACK_ET; t += blockDim.x) {
    const int el = t % UNPACK_ET, jp = t / UNPACK_ET, p = jp & 1, j = jp >> 1;
    if (el >= et) continue;
    const float2 u = tl[j * LD + el];
    r2b[((long long)j * C2 + 2 * s + p) * ld_ov + (long long)m * v + e0 + el] = __float2bfloat16(p ? u.y : u.x);
  }
  // oooo: rows (e, 2 s + p), columns m o + j
  for (int t = threadIdx.x; t < 2 * et * o; t += blockDim.x) {
    const int ep = quo((unsigned)t, rcp_o), j = t - ep * o, p = ep & 1, el = ep >> 1;
    const float2 u = tl[j * LD + el];
    r2o[((long long)(e0 + el) * C2 + 2 * s + p) * ld_o2 + (long long)m * o + j] = __float2bfloat16(p ? u.y : u.x);
  }
  // long K: row 2 s + p, columns (m v + e) o + j for the tile's e range
  for (int p = 0; p < 2; p++) {
    __nv_bfloat16 *dst = rk + (long long)(2 * s + p) * ld_k1 + ((long long)m * v + e0) * o;
    for (int t = threadIdx.x; t < et * o; t += blockDim.x) {
      const int el = quo((unsigned)t, rcp_o), j = t - el * o;
      const float2 u = tl[j * LD + el];
      dst[t] = __float2bfloat16(p ? u.y : u.x);
    }
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

// ---------------------------------------------------------------------------------------- EA
// y2[m, a, e] of system s (antisymmetric in a, e; zero for a == e) from the packed EA vector
// (1p a, then i-major 2p1h with pairs a < b)
__device__ __forceinline__ Cz y2_at(const SysBatch &b, int v, long long Pv, int s, int m, int a, int e) {
  if (a == e) return {0.0f, 0.0f};
  const long long lo = a < e ? a : e, hi = a < e ? e : a;
  const long long mu = v + (long long)m * Pv + pair_index(lo, hi, v);
  Cz u = load_u(b, s, mu);
  if (a > e) {
    u.r = -u.r;
    u.i = -u.i;
  }
  return u;
}

// The ring and long-K layouts of the 2p1h block in one pass: block (e tile, a tile, (m, s)) holds the
// 32 x 32 tile Y[a][e] = y2[m, a, e] of system s (antisymmetric: packed a < e, read along e above
// the diagonal and along a below it, so that reads stay coalesced), then writes, for both planes,
//   ring   r2e[(a, c)][(m, e)] =  Y[a][e]
//   long K rk[c][(m, a, e)]     = -Y[a][e]  (= y2[m, e, a])
// both along e.  grid (cdiv(v, 32), cdiv(v, 32), o * nsys), block (32, 8).
__global__ void unpack_ea_tile_kernel(SysBatch b, int o, int v, long long Pv, long long ld_ov, long long ldk,
                                      __nv_bfloat16 *r2e, __nv_bfloat16 *rk) {
  __shared__ float2 tile[32][33];
  const int e0 = blockIdx.x * 32, a0 = blockIdx.y * 32;
  const int m = (int)(blockIdx.z % (unsigned)o), s = (int)(blockIdx.z / (unsigned)o);
  const int C2 = 2 * b.nsys;
  const bool below = e0 + 31 < a0;   // every a > e: packed pairs (e, a) run along a
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int a = below ? a0 + threadIdx.x : a0 + r, e = below ? e0 + r : e0 + threadIdx.x;
    float2 val = make_float2(0.f, 0.f);
    if (a < v && e < v) {
      const Cz u = y2_at(b, v, Pv, s, m, a, e);
      val = make_float2(u.r, u.i);
    }
    if (below)
      tile[threadIdx.x][r] = val;
    else
      tile[r][threadIdx.x] = val;
  }
  __syncthreads();
  const int e = e0 + threadIdx.x;
  if (e >= v) return;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int a = a0 + r;
    if (a >= v) break;
    const float2 u = tile[r][threadIdx.x];
    const long long ring = ((long long)a * C2 + 2 * s) * ld_ov + (long long)m * v + e;
    r2e[ring] = __float2bfloat16(u.x);
    r2e[ring + ld_ov] = __float2bfloat16(u.y);
    const long long kk = (long long)(2 * s) * ldk + ((long long)m * v + a) * v + e;
    rk[kk] = __float2bfloat16(-u.x);
    rk[kk + ldk] = __float2bfloat16(-u.y);
  }
}

// r2p[(i, c)][ef] = y2[i, e < f] (row i of the packed 2p1h block), both planes; grid
// (cdiv(Pv, 256), o * nsys)
__global__ void unpack_ea_pairs_kernel(SysBatch b, int o, int v, long long Pv, long long ld, __nv_bfloat16 *out) {
  const int i = (int)(blockIdx.y % (unsigned)o), s = (int)(blockIdx.y / (unsigned)o);
  const long long ef = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (ef >= Pv) return;
  const Cz u = load_u(b, s, v + (long long)i * Pv + ef);
  const long long row = (long long)i * 2 * b.nsys + 2 * s;
  out[row * ld + ef] = __float2bfloat16(u.r);
  out[(row + 1) * ld + ef] = __float2bfloat16(u.i);
}

// rk[c][o v v + e] = y1[e] and r1[c][e] = y1[e], both planes; grid (cdiv(v, 256), nsys)
__global__ void unpack_ea_y1_kernel(SysBatch b, int o, int v, long long ldk, __nv_bfloat16 *rk, long long ld1,
                                    __nv_bfloat16 *r1) {
  const int s = blockIdx.y, e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= v) return;
  const long long ov2 = (long long)o * v * v;
  const Cz u = load_u(b, s, e);
  const __nv_bfloat16 hr = __float2bfloat16(u.r), hi = __float2bfloat16(u.i);
  rk[(long long)(2 * s) * ldk + ov2 + e] = hr;
  rk[(long long)(2 * s + 1) * ldk + ov2 + e] = hi;
  r1[(long long)(2 * s) * ld1 + e] = hr;
  r1[(long long)(2 * s + 1) * ld1 + e] = hi;
}

constexpr int KSPLIT = 64;   // split of the long-K contractions (Z, 1h row) into partial sums

struct MixedWork {
  __nv_bfloat16 *r2b, *r2o, *rk, *rz;
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
  w.rz = reinterpret_cast<__nv_bfloat16 *>(take(C2 * c->ld_ot * 2));
  w.T = reinterpret_cast<float *>(take(o * v * o * C2 * 4));
  w.Q = reinterpret_cast<float *>(take(o * o * v * C2 * 4));
  w.U = reinterpret_cast<float *>(take(o * v * o * C2 * 4));
  w.Zp = reinterpret_cast<float *>(take(KSPLIT * v * C2 * 4));
  w.S1p = reinterpret_cast<float *>(take(KSPLIT * o * C2 * 4));
  w.bytes = p - static_cast<unsigned char *>(base);
  return w;
}

}  // namespace

struct MixedWorkEA {
  __nv_bfloat16 *r2e, *r2p, *rk, *rz;
  float *T, *Qp, *U, *Zp, *S1p;
  long long bytes;
};

MixedWorkEA layout_ea(const gfcc_ctx *c, int nsys, void *base) {
  const long long o = c->o, v = c->v, C2 = 2LL * nsys, Pv = c->Pv, ov2 = o * v * v;
  MixedWorkEA w;
  unsigned char *p = static_cast<unsigned char *>(base);
  auto take = [&](long long bytes) {
    unsigned char *q = p;
    p += (bytes + 255) / 256 * 256;
    return q;
  };
  w.r2e = reinterpret_cast<__nv_bfloat16 *>(take(v * C2 * c->ld_ov * 2));
  w.r2p = reinterpret_cast<__nv_bfloat16 *>(take(o * C2 * c->ld_pv * 2));
  w.rk = reinterpret_cast<__nv_bfloat16 *>(take(C2 * c->ld_k1e * 2));
  w.rz = reinterpret_cast<__nv_bfloat16 *>(take(C2 * c->ld_ot * 2));
  w.T = reinterpret_cast<float *>(take(o * v * v * C2 * 4));
  w.Qp = reinterpret_cast<float *>(take(std::max<long long>(Pv, 1) * o * C2 * 4));
  w.U = reinterpret_cast<float *>(take(ov2 * C2 * 4));
  w.Zp = reinterpret_cast<float *>(take(KSPLIT * o * C2 * 4));
  w.S1p = reinterpret_cast<float *>(take(KSPLIT * v * C2 * 4));
  w.bytes = p - static_cast<unsigned char *>(base);
  return w;
}

long long sigma_mixed_work_doubles(const gfcc_ctx *c, int nsys) {
  long long b = 0;
  if (c->Wr_bf != nullptr) b = std::max(b, layout(c, nsys, nullptr).bytes);
  if (c->Wre_bf != nullptr) b = std::max(b, layout_ea(c, nsys, nullptr).bytes);
  return b / 8 + 64;
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
  if (v > 0 && o <= UNPACK_MAX_O) {
    const unsigned long long rcp_o = ((1ULL << 32) + (unsigned long long)o - 1) / (unsigned long long)o;
    const size_t sm = (size_t)o * (UNPACK_ET + 1) * sizeof(float2);
    unpack_ip_kernel<<<dim3(cdiv(v, UNPACK_ET), (unsigned)o, (unsigned)b.nsys), 256, sm, st>>>(
        b, (int)o, (int)v, rcp_o, c->ld_ov, c->ld_o2, c->ld_k1, w.r2b, w.r2o, w.rk);
    GFCC_LAUNCH_CHECK();
  } else {
    unpack_ring_kernel<<<grid1d(o * C2 * ov), 256, 0, st>>>(b, (int)o, (int)v, c->ld_ov, w.r2b);
    GFCC_LAUNCH_CHECK();
    unpack_oooo_kernel<<<dim3(cdiv(oo, 32), cdiv(v, 32), C2), dim3(32, 8), 0, st>>>(b, (int)o, (int)v, c->ld_o2,
                                                                                     w.r2o);
    GFCC_LAUNCH_CHECK();
    unpack_k_tiled_kernel<<<dim3(cdiv(o, 32), cdiv(v, 32), o * C2), dim3(32, 8), 0, st>>>(b, (int)o, (int)v,
                                                                                          c->ld_k1, w.rk);
    GFCC_LAUNCH_CHECK();
  }
  unpack_r1_kernel<<<cdiv(C2 * o, 128), 128, 0, st>>>(b, (int)o, (int)v, c->ld_k1, w.rk, c->ld_ot, w.rz);
  GFCC_LAUNCH_CHECK();
  }
  {
    PhaseTimer tr(c, PH_RING_BF16, 2.0 * (double)ov * (double)ov * (double)(o * C2));
    GFCC_TRY(gemm_bf16_tn(st, c->Wr_bf, c->ld_ov, w.r2b, c->ld_ov, w.T, o * C2, (int)ov, (int)(o * C2), (int)ov, 1.0f,
                          0.0f));
  }
  {
    PhaseTimer tob(c, PH_BF16_OTHER, 2.0 * C2 * ((double)oo * oo * v + (double)v * o2v + (double)o2v * (o + v) +
                                                 (double)o * (o2v + o)));
    GFCC_TRY(gemm_bf16_tn(st, c->Wq_bf, c->ld_o2, w.r2o, c->ld_o2, w.Q, v * C2, (int)oo, (int)(v * C2), (int)oo, 1.0f,
                          0.0f));
    // three-body: Z (split K) -> BF16 transposed into rz[c][o + e]; then U = [W1 | T3] [r1 | Z]
    const int zs = umma_splits((int)o2v, KSPLIT);
    GFCC_TRY(gemm_bf16_tn(st, c->V3_bf, c->ld_o2v, w.rk, c->ld_k1, w.Zp, C2, (int)v, (int)C2, (int)o2v, 1.0f, 0.0f, zs,
                          v * C2));
    reduce_splits_kernel<<<grid1d(v * C2), 256, 0, st>>>(w.Zp, zs, v, C2, v * C2, w.rz + o, c->ld_ot);
    GFCC_LAUNCH_CHECK();
    GFCC_TRY(gemm_bf16_tn(st, c->WT_bf, c->ld_ot, w.rz, c->ld_ot, w.U, C2, (int)o2v, (int)C2, (int)(o + v), 1.0f,
                          0.0f));
    // 1h row (split K)
    const int ss = umma_splits((int)(o2v + o), KSPLIT);
    GFCC_TRY(gemm_bf16_tn(st, c->U1_bf, c->ld_k1, w.rk, c->ld_k1, w.S1p, C2, (int)o, (int)C2, (int)(o2v + o), 1.0f, 0.0f,
                          ss, o * C2));
    reduce_splits_kernel<<<grid1d(o * C2), 256, 0, st>>>(w.S1p, ss, o, C2, o * C2, nullptr, 0);
    GFCC_LAUNCH_CHECK();
  }
  {
    PhaseTimer tp(c, PH_EPILOGUE, 4.0 * C2 * (3.0 * o2v + o) + (b.xf ? 16.0 : 32.0) * b.nsys * c->dim_ip);
    GFCC_TRY((epi::launch_ip<float, epi::MODE_OFFDIAG>(st, b, (int)o, (int)v, w.S1p, w.T, w.Q, w.U, c->diag_ip)));
  }
  return GFCC_OK;
}


int apply_ea_mixed(gfcc_ctx *c, const SysBatch &b, double *work) {
  if (c->Wre_bf == nullptr) {
    set_error("mixed-precision EA sigma requested but its BF16 operands were not built");
    return GFCC_ERR_STATE;
  }
  cudaStream_t st = c->stream;
  const long long o = c->o, v = c->v, ov = o * v, ov2 = ov * v, C2 = 2LL * b.nsys, Pv = c->Pv;
  MixedWorkEA w = layout_ea(c, b.nsys, work);
  PhaseTimer tsig(c, PH_SIGMA, b.nsys * sigma_flops(c, GFCC_SECTOR_EA));
  {
    PhaseTimer tu(c, PH_UNPACK);
    unpack_ea_tile_kernel<<<dim3(cdiv(v, 32), cdiv(v, 32), (unsigned)(o * b.nsys)), dim3(32, 8), 0, st>>>(
        b, (int)o, (int)v, Pv, c->ld_ov, c->ld_k1e, w.r2e, w.rk);
    GFCC_LAUNCH_CHECK();
    if (Pv > 0) {
      unpack_ea_pairs_kernel<<<dim3(cdiv(Pv, 256), (unsigned)(o * b.nsys)), 256, 0, st>>>(b, (int)o, (int)v, Pv,
                                                                                        c->ld_pv, w.r2p);
      GFCC_LAUNCH_CHECK();
    }
    unpack_ea_y1_kernel<<<dim3(cdiv(v, 256), (unsigned)b.nsys), 256, 0, st>>>(b, (int)o, (int)v, c->ld_k1e, w.rk,
                                                                              c->ld_ot, w.rz);
    GFCC_LAUNCH_CHECK();
  }
  // T[(i,b)][(a,c)] = Wr_ea[(i,b)][(m,e)] y2[m,a,e]
  {
    PhaseTimer tr(c, PH_RING_BF16, 2.0 * (double)ov * (double)ov * (double)(v * C2));
    GFCC_TRY(gemm_bf16_tn(st, c->Wre_bf, c->ld_ov, w.r2e, c->ld_ov, w.T, v * C2, (int)ov, (int)(v * C2), (int)ov, 1.0f,
                          0.0f));
  }
  // Qp[(a<b)][(i,c)] = Wp[(ab)][(ef)] y2[i,e,f]
  if (Pv > 0) {
    PhaseTimer tv(c, PH_VVVV, 2.0 * (double)Pv * (double)Pv * (double)(o * C2));
    GFCC_TRY(gemm_bf16_tn(st, c->Wp_bf, c->ld_pv, w.r2p, c->ld_pv, w.Qp, o * C2, (int)Pv, (int)(o * C2), (int)Pv,
                          1.0f, 0.0f));
  }
  {
    PhaseTimer tob(c, PH_BF16_OTHER, 2.0 * C2 * ((double)o * ov2 + (double)ov2 * (v + o) + (double)v * (ov2 + v)));
    // U[(i,b,a)][c] = [W3 | T3e] [y1 | Z],  Z[m][c] = V3e[m][(n,f,e)] y2[n,e,f] (split K, into rz[c][v + m])
    const int zs = umma_splits((int)ov2, KSPLIT);
    GFCC_TRY(gemm_bf16_tn(st, c->V3e_bf, c->ld_ov2, w.rk, c->ld_k1e, w.Zp, C2, (int)o, (int)C2, (int)ov2, 1.0f, 0.0f,
                          zs, o * C2));
    reduce_splits_kernel<<<grid1d(o * C2), 256, 0, st>>>(w.Zp, zs, o, C2, o * C2, w.rz + v, c->ld_ot);
    GFCC_LAUNCH_CHECK();
    GFCC_TRY(gemm_bf16_tn(st, c->WTe_bf, c->ld_ot, w.rz, c->ld_ot, w.U, C2, (int)ov2, (int)C2, (int)(v + o), 1.0f,
                          0.0f));
    // 1p row: S1[a][c] = [U1e | Fvv off-diagonal][a] . [y2 | y1](c) (split K)
    const int ss = umma_splits((int)(ov2 + v), KSPLIT);
    GFCC_TRY(gemm_bf16_tn(st, c->U1e_bf, c->ld_k1e, w.rk, c->ld_k1e, w.S1p, C2, (int)v, (int)C2, (int)(ov2 + v), 1.0f,
                          0.0f, ss, v * C2));
    reduce_splits_kernel<<<grid1d(v * C2), 256, 0, st>>>(w.S1p, ss, v, C2, v * C2, nullptr, 0);
    GFCC_LAUNCH_CHECK();
  }
  {
    PhaseTimer tp(c, PH_EPILOGUE, 4.0 * C2 * (2.0 * ov2 + (double)Pv * o + v) + (b.xf ? 16.0 : 32.0) * b.nsys * c->dim_ea);
    GFCC_TRY((epi::launch_ea<float, epi::MODE_OFFDIAG>(st, b, (int)o, (int)v, Pv, w.S1p, w.T, w.Qp, w.U,
                                                       c->diag_ea)));
  }
  return GFCC_OK;
}

}  // namespace gfcc
