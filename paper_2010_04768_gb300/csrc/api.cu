// The C ABI of libgfcc: context life cycle, option handling, the frequency x orbital
// task loop of gfcc_solve (Algorithm 1 of the paper: all (omega, p) tasks of a level are
// independent; here they are batched onto one GPU instead of process groups), the
// right-hand sides, left vectors and overlaps of eqs. gfxn2/gfxn3.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include "ctx.cuh"
#include "gmres.cuh"
#include "kernels.cuh"
#include "sigma.cuh"
#include "ozaki.cuh"
#include "umma.cuh"
#include "guess.cuh"
#include "mlp.cuh"

namespace gfcc {

static thread_local char g_err[1024] = "";

namespace {
struct AllocRec {
  uintptr_t base;
  size_t bytes;
};
std::mutex g_alloc_mu;
std::vector<AllocRec> g_allocs;
}  // namespace

void reg_alloc(const void *p, size_t bytes) {
  if (p == nullptr) return;
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_allocs.push_back({reinterpret_cast<uintptr_t>(p), bytes});
}

void unreg_alloc(const void *p) {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  for (size_t i = 0; i < g_allocs.size(); i++)
    if (g_allocs[i].base == reinterpret_cast<uintptr_t>(p)) {
      g_allocs[i] = g_allocs.back();
      g_allocs.pop_back();
      return;
    }
}

int check_extent(const double *p, long long lo, long long hi, const char *what) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p + lo), b = reinterpret_cast<uintptr_t>(p + hi + 1);
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  for (const AllocRec &r : g_allocs)
    if (a >= r.base && b <= r.base + r.bytes && lo <= hi) return GFCC_OK;
  set_error("internal extent check failed for %s: offsets [%lld, %lld] are outside every device allocation", what,
            lo, hi);
  return GFCC_ERR_ARG;
}

int check_extent_bytes(const void *p, long long bytes, const char *what) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p), b = a + (uintptr_t)bytes;
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  for (const AllocRec &r : g_allocs)
    if (a >= r.base && b <= r.base + r.bytes && bytes > 0) return GFCC_OK;
  set_error("internal extent check failed for %s: %lld bytes are outside every device allocation", what, bytes);
  return GFCC_ERR_ARG;
}

cudaError_t dmalloc(void **p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) reg_alloc(*p, bytes);
  return e;
}

void dfree(void *p) {
  if (p == nullptr) return;
  unreg_alloc(p);
  cudaFree(p);
}

static std::atomic<long long> g_launches{0};
static thread_local long long t_launches = 0;   // this thread's launches (graph capture bookkeeping)
void count_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  t_launches++;
}
void count_launches(long long n) {
  g_launches.fetch_add(n, std::memory_order_relaxed);
  t_launches += n;
}
long long launch_count() { return g_launches.load(); }
long long thread_launch_count() { return t_launches; }

static cudaEvent_t take_event(gfcc_ctx *c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

PhaseTimer::PhaseTimer(gfcc_ctx *ctx, int ph, double fl) : c(ctx), phase(ph), flops(fl) {
  if (c->prof) {
    a = take_event(c);
    if (a) cudaEventRecord(a, c->stream);
  }
}

PhaseTimer::~PhaseTimer() {
  if (!c->prof || a == nullptr) return;
  cudaEvent_t b = take_event(c);
  if (b == nullptr) {
    c->ev_pool.push_back(a);
    return;
  }
  cudaEventRecord(b, c->stream);
  c->pend.push_back({a, b, phase, flops});
}

void prof_resolve(gfcc_ctx *c) {
  for (auto &p : c->pend) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      c->prof_ms[p.phase] += ms;
      c->prof_n[p.phase] += 1;
      c->prof_flops[p.phase] += p.flops;
    } else {
      cudaGetLastError();
    }
    c->ev_pool.push_back(p.a);
    c->ev_pool.push_back(p.b);
  }
  c->pend.clear();
}

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

namespace {

// ---------------------------------------------------------------- input checks (device)
// out[0] = max |x|; out[1] = max |x - sign * x^P| over the permutation given by (swap01, swap23) of a 4-index tensor
// (per-thread maxima of the |value| bit patterns, which order like unsigned integers with NaN above
// +inf, reduced over the warp, one atomic per warp and quantity; launched with whole warps)
__global__ void symmetry_kernel(const double *x, long long d0, long long d1, long long d2, long long d3, int swap01,
                                int swap23, double sign, unsigned long long *out) {
  const long long tot = d0 * d1 * d2 * d3;
  unsigned long long m0 = 0, m1 = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    long long r = t;
    const long long k3 = r % d3; r /= d3;
    const long long k2 = r % d2; r /= d2;
    const long long k1 = r % d1;
    const long long k0 = r / d1;
    long long p0 = k0, p1 = k1, p2 = k2, p3 = k3;
    if (swap01) { p0 = k1; p1 = k0; }
    if (swap23) { p2 = k3; p3 = k2; }
    const double a = x[t];
    const double b = x[((p0 * d1 + p1) * d2 + p2) * d3 + p3];
    m0 = max(m0, (unsigned long long)__double_as_longlong(fabs(a)) & 0x7fffffffffffffffULL);
    m1 = max(m1, (unsigned long long)__double_as_longlong(fabs(a - sign * b)) & 0x7fffffffffffffffULL);
  }
  for (int w = 16; w > 0; w >>= 1) {
    m0 = max(m0, __shfl_xor_sync(0xffffffffu, m0, w));
    m1 = max(m1, __shfl_xor_sync(0xffffffffu, m1, w));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, m0);
    atomicMax(out + 1, m1);
  }
}

// ---------------------------------------------------------------- right-hand sides
// IP b_p: p occupied: unit 1h vector; p = o + b virtual: r1 = t1[:, b], r2[i<j, a] = t2[i][j][b][a]
__global__ void rhs_ip_kernel(double *B, long long n, int nsys, const int *porb, int o, int v, const double *t1,
                              const double *t2, const int *mask) {
  const long long tot = n * nsys;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(t / n);
    if (mask != nullptr && !mask[s]) continue;
    const long long mu = t - (long long)s * n;
    const int p = porb[s];
    double val = 0.0;
    if (mu < o) {
      val = p < o ? (mu == p ? 1.0 : 0.0) : t1[mu * v + (p - o)];
    } else if (p >= o) {
      const long long r = mu - o;
      const long long a = r % v;
      long long i, j;
      pair_decode(r / v, o, i, j);
      val = t2[((i * o + j) * v + (p - o)) * v + a];
    }
    B[2 * t] = val;
    B[2 * t + 1] = 0.0;
  }
}

// EA b_q: q virtual: unit 1p vector; q = m occupied: y1 = -t1[m, :], y2[i, a<b] = -t2[m][i][a][b]
__global__ void rhs_ea_kernel(double *B, long long n, int nsys, const int *qorb, int o, int v, long long Pv,
                              const double *t1, const double *t2, const int *mask) {
  const long long tot = n * nsys;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(t / n);
    if (mask != nullptr && !mask[s]) continue;
    const long long mu = t - (long long)s * n;
    const int q = qorb[s];
    double val = 0.0;
    if (mu < v) {
      val = q >= o ? (mu == q - o ? 1.0 : 0.0) : -t1[(long long)q * v + mu];
    } else if (q < o) {
      const long long r = mu - v;
      const long long i = r / Pv;
      long long a, b;
      pair_decode(r % Pv, v, a, b);
      val = -t2[(((long long)q * o + i) * v + a) * v + b];
    }
    B[2 * t] = val;
    B[2 * t + 1] = 0.0;
  }
}

// ---------------------------------------------------------------- left vectors (real), C[q][mu]
// IP c_q(mu) = <Phi|(1+Lambda) a_q^+-bar |mu>:
//   q = o + b: c(k) = l1[k][b], c(i<j, a) = l2[i][j][b][a]
//   q = m    : c(k) = d_mk - t1[m].l1[k] - 1/2 t2[m][l][c][d] l2[k][l][c][d];
//              c(i<j, a) = d_mi l1[j][a] - d_mj l1[i][a] - t1[m][c] l2[i][j][c][a]
__global__ void left_ip_2h1p_kernel(double *C, long long n, int nq, const int *qorb, int o, int v, const double *t1,
                                    const double *l1, const double *l2) {
  const long long n2 = n - o;
  const long long tot = n2 * nq;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int qi = (int)(t / n2);
    const long long r = t - (long long)qi * n2;
    const int q = qorb[qi];
    const long long a = r % v;
    long long i, j;
    pair_decode(r / v, o, i, j);
    double val;
    if (q >= o) {
      val = l2[((i * o + j) * v + (q - o)) * v + a];
    } else {
      const int m = q;
      val = (m == i ? l1[j * v + a] : 0.0) - (m == j ? l1[i * v + a] : 0.0);
      for (int c = 0; c < v; c++) val -= t1[(long long)m * v + c] * l2[((i * o + j) * v + c) * v + a];
    }
    C[(long long)qi * n + o + r] = val;
  }
}

__global__ void left_ip_1h_kernel(double *C, long long n, int nq, const int *qorb, int o, int v, const double *t1,
                                  const double *t2, const double *l1, const double *l2) {
  __shared__ double2 sh[32];
  const int qi = blockIdx.x / o, k = blockIdx.x % o;
  const int q = qorb[qi];
  double val;
  if (q >= o) {
    val = l1[(long long)k * v + (q - o)];
  } else {
    const int m = q;
    const long long ovv = (long long)o * v * v;
    double acc = 0.0;
    for (long long x = threadIdx.x; x < ovv; x += blockDim.x)   // x = (l, c, d)
      acc += t2[(long long)m * ovv + x] * l2[(long long)k * ovv + x];
    double acc1 = 0.0;
    for (int c = threadIdx.x; c < v; c += blockDim.x) acc1 += t1[(long long)m * v + c] * l1[(long long)k * v + c];
    double2 sum = make_double2(acc, acc1);
    for (int off = 16; off > 0; off >>= 1) {
      sum.x += __shfl_down_sync(0xffffffffu, sum.x, off);
      sum.y += __shfl_down_sync(0xffffffffu, sum.y, off);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = sum;
    __syncthreads();
    if (threadIdx.x != 0) return;
    sum = make_double2(0.0, 0.0);
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
      sum.x += sh[w].x;
      sum.y += sh[w].y;
    }
    val = (m == k ? 1.0 : 0.0) - sum.y - 0.5 * sum.x;
  }
  if (threadIdx.x == 0) C[(long long)qi * n + k] = val;
}

// EA c_p(mu) = <Phi|(1+Lambda) a_p-bar |mu>:
//   p = m    : c(c) = -l1[m][c], c(i, c<d) = l2[i][m][c][d]
//   p = o + e: c(c) = d_ec - t1[k][e] l1[k][c] + 1/2 t2[k][l][e][d] l2[k][l][d][c];
//              c(i, c<d) = d_ec l1[i][d] - d_ed l1[i][c] + t1[k][e] l2[i][k][c][d]
__global__ void left_ea_2p1h_kernel(double *C, long long n, int np, const int *porb, int o, int v, long long Pv,
                                    const double *t1, const double *l1, const double *l2) {
  const long long n2 = n - v;
  const long long tot = n2 * np;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int pi = (int)(t / n2);
    const long long r = t - (long long)pi * n2;
    const int p = porb[pi];
    const long long i = r / Pv;
    long long c, d;
    pair_decode(r % Pv, v, c, d);
    double val;
    if (p < o) {
      val = l2[((i * o + p) * v + c) * v + d];
    } else {
      const long long e = p - o;
      val = (e == c ? l1[i * v + d] : 0.0) - (e == d ? l1[i * v + c] : 0.0);
      for (int k = 0; k < o; k++) val += t1[(long long)k * v + e] * l2[((i * o + k) * v + c) * v + d];
    }
    C[(long long)pi * n + v + r] = val;
  }
}

__global__ void left_ea_1p_kernel(double *C, long long n, int np, const int *porb, int o, int v, const double *t1,
                                  const double *t2, const double *l1, const double *l2) {
  __shared__ double2 sh[32];
  const int pi = blockIdx.x / v, c = blockIdx.x % v;
  const int p = porb[pi];
  double val;
  if (p < o) {
    val = -l1[(long long)p * v + c];
  } else {
    const long long e = p - o;
    const long long oov = (long long)o * o * v;
    double acc = 0.0;
    for (long long x = threadIdx.x; x < oov; x += blockDim.x) {   // x = (k, l, d)
      const long long kl = x / v, d = x % v;
      acc += t2[(kl * v + e) * v + d] * l2[(kl * v + d) * v + c];
    }
    double acc1 = 0.0;
    for (int k = threadIdx.x; k < o; k += blockDim.x) acc1 += t1[(long long)k * v + e] * l1[(long long)k * v + c];
    double2 sum = make_double2(acc, acc1);
    for (int off = 16; off > 0; off >>= 1) {
      sum.x += __shfl_down_sync(0xffffffffu, sum.x, off);
      sum.y += __shfl_down_sync(0xffffffffu, sum.y, off);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = sum;
    __syncthreads();
    if (threadIdx.x != 0) return;
    sum = make_double2(0.0, 0.0);
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
      sum.x += sh[w].x;
      sum.y += sh[w].y;
    }
    val = (e == c ? 1.0 : 0.0) - sum.y + 0.5 * sum.x;
  }
  if (threadIdx.x == 0) C[(long long)pi * n + c] = val;
}

// ---------------------------------------------------------------- overlaps
// part[z][(s,t)][q] summed over z -> G ([omega][nP][nQ]): the IP system (w_s, a_s) of row orbital a_s
// gets row a_s, columns q < nl (nl = nQ left vectors); the EA system (w_s, a_s) of column orbital
// a_s gets column a_s, rows q < nl (nl = nP left vectors).  Systems s < count with tw[s] >= 0 of a
// batch of nsys systems, from the split-K partial overlaps.
__global__ void overlap_scatter_kernel(const double *part, int nsplit, int nsys, int count, int nl, const int *tw,
                                       const int *ta, int is_ip, int nP, int nQ, double *G) {
  const long long tot = (long long)count * nl;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(t / nl), q = (int)(t % nl);
    if (tw[s] < 0) continue;
    double re = 0.0, im = 0.0;
    const long long zs = 2LL * nsys * nl;
    for (int z = 0; z < nsplit; z++) {
      re += part[z * zs + (2LL * s) * nl + q];
      im += part[z * zs + (2LL * s + 1) * nl + q];
    }
    const long long w = tw[s], a = ta[s];
    const long long idx = is_ip ? (w * nP + a) * nQ + q : (w * nP + q) * nQ + a;
    G[2 * idx] += re;
    G[2 * idx + 1] += im;
  }
}

__global__ void gather_omega_kernel(const double *om, const int *tw, int nsys, double *out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < nsys) out[s] = om[tw[s]];
}

__global__ void gather_orb_kernel(const int *orbs, const int *ta, int nsys, int *out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < nsys) out[s] = orbs[ta[s]];
}

int check_tensor(cudaStream_t st, const double *x, long long d0, long long d1, long long d2, long long d3, int s01,
                 int s23, double sign, double rel, const char *name) {
  unsigned long long *d, h[2];
  GFCC_CUDA(cudaMalloc(&d, 2 * sizeof(unsigned long long)));
  cudaMemsetAsync(d, 0, 2 * sizeof(unsigned long long), st);
  symmetry_kernel<<<grid1d(d0 * d1 * d2 * d3), 256, 0, st>>>(x, d0, d1, d2, d3, s01, s23, sign, d);
  cudaError_t e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  if (e != cudaSuccess) {
    set_error("input check of %s: %s", name, cudaGetErrorString(e));
    return GFCC_ERR_CUDA;
  }
  double mx, dev;
  memcpy(&mx, &h[0], sizeof(double));
  memcpy(&dev, &h[1], sizeof(double));
  if (!std::isfinite(mx) || !std::isfinite(dev)) {
    set_error("%s contains non-finite values", name);
    return GFCC_ERR_ARG;
  }
  if (dev > rel * std::max(1.0, mx)) {
    set_error("%s violates its permutation symmetry (max deviation %.3e, max |value| %.3e)", name, dev, mx);
    return GFCC_ERR_ARG;
  }
  return GFCC_OK;
}

int upload(gfcc_ctx *c, double **dst, const double *src, long long count) {
  GFCC_TRY(dev_alloc(c, dst, count));
  GFCC_CUDA(cudaMemcpyAsync(*dst, src, sizeof(double) * count, cudaMemcpyHostToDevice, c->stream));
  return GFCC_OK;
}

int create_impl(int o, int v, int L, const double *fock, const double *chol, const double *t1, const double *t2,
                const double *lambda, int sectors, int precision, gfcc_ctx **out, int rhf = 0) {
  if (out == nullptr) {
    set_error("gfcc_create: out is NULL");
    return GFCC_ERR_ARG;
  }
  *out = nullptr;
  if (o < 1 || v < 1 || L < 1 || fock == nullptr || chol == nullptr || t1 == nullptr || t2 == nullptr) {
    set_error("gfcc_create: need o >= 1, v >= 1, L >= 1 and non-NULL fock, chol, t1, t2");
    return GFCC_ERR_ARG;
  }
  if (sectors < 1 || sectors > 3 || (precision != GFCC_PREC_FP64 && precision != GFCC_PREC_MIXED_BF16)) {
    set_error("gfcc_create: bad sectors (%d) or precision (%d)", sectors, precision);
    return GFCC_ERR_ARG;
  }
  gfcc_ctx *c = new gfcc_ctx();
  c->o = o; c->v = v; c->L = L; c->n = o + v;
  c->Po = (long long)o * (o - 1) / 2;
  c->Pv = (long long)v * (v - 1) / 2;
  c->dim_ip = o + c->Po * v;
  c->dim_ea = v + (long long)o * c->Pv;
  c->rhf = rhf;
  if (rhf) c->dim_ip = o + (long long)o * o * v;   // spatial 1h + 2h1p coordinates, no pair packing
  c->sectors = sectors;
  c->precision = precision;
  int s = GFCC_OK;
  auto fail = [&](int code) {
    gfcc_destroy(c);
    return code;
  };
  if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    set_error("gfcc_create: cannot create a CUDA stream (no usable GPU?)");
    return fail(GFCC_ERR_CUDA);
  }
  c->stream = c->own_stream;
  const long long n = c->n, nn = n * n, ov = (long long)o * v, oovv = ov * ov;
  double *d_fock = nullptr, *d_chol = nullptr;
  if ((s = dev_alloc_tmp(&d_fock, nn)) < 0) return fail(s);
  if ((s = dev_alloc_tmp(&d_chol, (long long)L * nn)) < 0) {
    dfree(d_fock);
    return fail(s);
  }
  auto free_tmp = [&]() {
    dfree(d_fock);
    dfree(d_chol);
  };
  if (cudaMemcpyAsync(d_fock, fock, sizeof(double) * nn, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(d_chol, chol, sizeof(double) * L * nn, cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
    set_error("gfcc_create: host-to-device copy failed: %s", cudaGetErrorString(cudaGetLastError()));
    free_tmp();
    return fail(GFCC_ERR_CUDA);
  }
  if ((s = upload(c, &c->t1, t1, ov)) < 0 || (s = upload(c, &c->t2, t2, oovv)) < 0) {
    free_tmp();
    return fail(s);
  }
  if (lambda != nullptr) {
    if ((s = upload(c, &c->l1, lambda, ov)) < 0 || (s = upload(c, &c->l2, lambda + ov, oovv)) < 0) {
      free_tmp();
      return fail(s);
    }
  } else {
    c->l1 = c->t1;
    c->l2 = c->t2;
  }
  // input checks: symmetric fock and Cholesky vectors, antisymmetric T2 / Lambda2, all finite
  if ((s = check_tensor(c->stream, d_fock, 1, 1, n, n, 0, 1, 1.0, 1e-12, "fock")) < 0 ||
      (s = check_tensor(c->stream, d_chol, 1, L, n, n, 0, 1, 1.0, 1e-12, "chol")) < 0 ||
      (s = check_tensor(c->stream, c->t1, 1, 1, o, v, 0, 0, 1.0, 1e300, "t1")) < 0 ||
      (!rhf && (s = check_tensor(c->stream, c->t2, o, o, v, v, 1, 0, -1.0, 1e-12, "t2 (i<->j)")) < 0) ||
      (!rhf && (s = check_tensor(c->stream, c->t2, o, o, v, v, 0, 1, -1.0, 1e-12, "t2 (a<->b)")) < 0) ||
      (rhf && (s = check_tensor(c->stream, c->t2, o, o, v, v, 1, 1, 1.0, 1e-12, "t2 (ia<->jb)")) < 0)) {
    free_tmp();
    return fail(s);
  }
  if (lambda != nullptr &&
      ((s = check_tensor(c->stream, c->l1, 1, 1, o, v, 0, 0, 1.0, 1e300, "lambda1")) < 0 ||
       (!rhf && (s = check_tensor(c->stream, c->l2, o, o, v, v, 1, 0, -1.0, 1e-12, "lambda2 (i<->j)")) < 0) ||
       (!rhf && (s = check_tensor(c->stream, c->l2, o, o, v, v, 0, 1, -1.0, 1e-12, "lambda2 (a<->b)")) < 0) ||
       (rhf && (s = check_tensor(c->stream, c->l2, o, o, v, v, 1, 1, 1.0, 1e-12, "lambda2 (ia<->jb)")) < 0))) {
    free_tmp();
    return fail(s);
  }
  {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const bool timed = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
    if (timed) cudaEventRecord(e0, c->stream);
    // mixed-precision contexts build their large FP64 intermediates from digit planes on the
    // tensor cores (FP64-accurate); FP64 contexts keep every contraction on the FP64 units
    g_emulate_big = precision == GFCC_PREC_MIXED_BF16;
    s = rhf ? build_hbar_rhf(c, d_fock, d_chol) : build_hbar(c, d_fock, d_chol);
    g_emulate_big = false;
    if (timed) {
      cudaEventRecord(e1, c->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
        c->prof_ms[PH_SETUP] = ms;
        c->prof_n[PH_SETUP] = 1;
      }
    }
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
  free_tmp();
  if (s < 0) return fail(s);
  *out = c;
  return GFCC_OK;
}

// The orbital lists of a solve: rows p of G run over P, columns q over Q.  IP systems are solved for
// the row orbitals (X_p, eq. xp) and overlapped with the left vectors of the columns; EA systems
// are solved for the column orbitals (Y_q, eq. yq) and overlapped with the left vectors of the rows.
struct OrbLists {
  int nP = 0, nQ = 0;
  const int *dP = nullptr, *dQ = nullptr;   // device
  const int *hP = nullptr, *hQ = nullptr;   // host copies of the same lists
  int n_sys(bool ip) const { return ip ? nP : nQ; }
  const int *sys(bool ip) const { return ip ? dP : dQ; }
  int n_left(bool ip) const { return ip ? nQ : nP; }
  const int *left(bool ip) const { return ip ? dQ : dP; }
  const int *left_host(bool ip) const { return ip ? hQ : hP; }
};

int solve_impl_inner(gfcc_ctx *c, int n_omega, const double *d_om, double eta, const OrbLists &ol, double tol,
                     double *d_G);

int choose_batch(gfcc_ctx *c, int sector, long long n, long long ntasks) {
  if (c->batch > 0) return (int)std::min<long long>(c->batch, ntasks);
  const bool mixed = c->precision == GFCC_PREC_MIXED_BF16 && (sector == GFCC_SECTOR_IP ? c->Wr_bf : c->Wre_bf) != nullptr;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    fr = 1ULL << 30;
  }
  const int m = mixed ? c->inner_restart : c->restart;
  const double per = 8.0 * (double)(gmres_work_doubles(c, sector, n, 2, m, mixed) -
                                   gmres_work_doubles(c, sector, n, 1, m, mixed));
  long long b = (long long)(0.6 * c->mem_share * (double)fr / std::max(per, 1.0));
  b = std::max<long long>(1, std::min<long long>(b, 256));
  return (int)std::min<long long>(b, ntasks);
}

int grow_scratch(gfcc_ctx *c, size_t bytes) {
  if (c->scratch_bytes >= bytes) return GFCC_OK;
  if (c->scratch) dfree(c->scratch);
  c->scratch = nullptr;
  c->scratch_bytes = 0;
  if (dmalloc(&c->scratch, bytes) != cudaSuccess) {
    cudaGetLastError();
    set_error("cannot allocate %.3f GB of solver workspace", bytes / 1e9);
    return GFCC_ERR_OOM;
  }
  c->scratch_bytes = bytes;
  return GFCC_OK;
}

int solve_impl(gfcc_ctx *c, int n_omega, const double *d_om, double eta, const OrbLists &ol, double tol,
               double *d_G) {
  cudaStream_t st = c->stream;
  int rc;
  {
    PhaseTimer tm(c, PH_SOLVE);
    rc = solve_impl_inner(c, n_omega, d_om, eta, ol, tol, d_G);
  }
  if (c->prof) {
    GFCC_CUDA(cudaStreamSynchronize(st));
    prof_resolve(c);
  }
  return rc;
}

// Kept-solution store of one sector: [omega][orbital][n] complex FP32, done flags cleared.
int prepare_kept(gfcc_ctx *c, int sector, long long n, int n_omega, int n_orb, const double *d_om, const int *d_orb,
                 double eta) {
  KeptSolutions &kp = c->kept;
  const size_t bytes = sizeof(float2) * (size_t)n_omega * n_orb * (size_t)n;
  if (kp.bytes < bytes) {
    if (kp.X) dfree(kp.X);
    kp.X = nullptr;
    kp.bytes = 0;
    if (dmalloc(reinterpret_cast<void **>(&kp.X), bytes) != cudaSuccess) {
      cudaGetLastError();
      set_error("cannot allocate %.3f GB for the kept solutions of the initial guesses", bytes / 1e9);
      return GFCC_ERR_OOM;
    }
    kp.bytes = bytes;
  }
  kp.sector = sector;
  kp.n = n;
  kp.nw = n_omega;
  kp.norb = n_orb;
  kp.eta = eta;
  kp.omega.resize(n_omega);
  kp.orb.resize(n_orb);
  kp.done.assign((size_t)n_omega * n_orb, 0);
  GFCC_CUDA(cudaMemcpyAsync(kp.omega.data(), d_om, sizeof(double) * n_omega, cudaMemcpyDeviceToHost, c->stream));
  GFCC_CUDA(cudaMemcpyAsync(kp.orb.data(), d_orb, sizeof(int) * n_orb, cudaMemcpyDeviceToHost, c->stream));
  GFCC_CUDA(cudaStreamSynchronize(c->stream));
  return GFCC_OK;
}

int solve_impl_inner(gfcc_ctx *c, int n_omega, const double *d_om, double eta, const OrbLists &ol, double tol,
                     double *d_G) {
  cudaStream_t st = c->stream;
  const int sectors[2] = {GFCC_SECTOR_IP, GFCC_SECTOR_EA};
  const int guess = c->guess;
  if (guess == GFCC_GUESS_LEARNED && c->mlp == nullptr) {
    set_error("gfcc_solve: GFCC_GUESS_LEARNED needs a model (gfcc_set_guess_model)");
    return GFCC_ERR_STATE;
  }
  const bool keep = guess != GFCC_GUESS_ZERO || c->keep_solutions;
  // statistics entries: the IP systems (omega-major over the row orbitals), then the EA systems
  // (omega-major over the column orbitals)
  long long nstat = 0;
  for (int sector : sectors)
    if (c->sectors & sector) nstat += (long long)n_omega * ol.n_sys(sector == GFCC_SECTOR_IP);
  c->st_iters.assign(nstat, 0);
  c->st_status.assign(nstat, GFCC_STATUS_NOT_CONVERGED);
  c->st_relres.assign(nstat, 0.0);
  c->st_guess.assign(nstat, GFCC_GUESS_ZERO);
  c->st_guess_pred.assign(nstat, 1.0);
  c->st_relres0.assign(nstat, 1.0);
  c->st_outer.assign(nstat, 0);
  c->res_full = c->res_inc = c->res_inc_levels = 0;
  GFCC_CUDA(cudaMemsetAsync(d_G, 0, sizeof(double) * 2 * n_omega * (long long)ol.nP * ol.nQ, st));
  long long stat_off = 0;   // first statistics entry of the current sector
  bool all_ok = true;
  for (int sector : sectors) {
    if (!(c->sectors & sector)) continue;
    const bool ip = sector == GFCC_SECTOR_IP;
    const long long n = ip ? c->dim_ip : c->dim_ea;
    const int n_orb = ol.n_sys(ip);     // orbitals of the systems solved in this sector
    const int *d_orb = ol.sys(ip);
    const int n_left = ol.n_left(ip);   // orbitals of the left vectors they are overlapped with
    const int *d_left = ol.left(ip);
    const long long ntasks = (long long)n_omega * n_orb;
    if (ntasks == 0) continue;
    // mixed precision: BF16 operator inside FP64-accurate refinement, in every sector whose BF16
    // operands were built
    const bool mixed = c->precision == GFCC_PREC_MIXED_BF16 && (ip ? c->Wr_bf : c->Wre_bf) != nullptr;
    if (keep) GFCC_TRY(prepare_kept(c, sector, n, n_omega, n_orb, d_om, d_orb, eta));
    const int nsys = choose_batch(c, sector, n, ntasks);
    const int m = mixed ? c->inner_restart : c->restart;
    const long long nsplit = (n + 8191) / 8192;
    const long long gw = gmres_work_doubles(c, sector, n, nsys, m, mixed);
    // guess workspace: Gram, features, model outputs, coefficients, predictions, deltas, p/n,
    // Gram partials; then the ints (neighbour slots, counts, kinds, store slots)
    const long long gq = keep ? 2LL * nsys * GUESS_G + (long long)nsys * (GUESS_NF + 2 * GUESS_NO + 1 + GUESS_K + 1) +
                                    guess_gram_work_doubles(nsys, n) + (long long)nsys * (GUESS_K + 3) / 2 + 64
                              : 0;
    const long long work = gw + nsplit * 2LL * nsys * n_left + 4LL * nsys + 64 + gq;
    GFCC_TRY(grow_scratch(c, sizeof(double) * work));
    double *base = static_cast<double *>(c->scratch);
    Gmres gm;
    GFCC_TRY(gm.init(c, sector, n, nsys, m, base, mixed));
    // left vectors: cached per sector and orbital list (computed on the first solve over the list)
    double *Cl = nullptr;
    bool left_ready = false;
    {
      gfcc_ctx::LeftCache &lc = c->left_cache[ip ? 0 : 1];
      const int *hl = ol.left_host(ip);
      const size_t lbytes = sizeof(double) * (size_t)n_left * (size_t)n;
      left_ready = lc.C != nullptr && (int)lc.orb.size() == n_left &&
                   std::equal(lc.orb.begin(), lc.orb.end(), hl);
      if (!left_ready) {
        lc.orb.clear();
        if (lc.bytes < lbytes) {
          if (lc.C) dfree(lc.C);
          lc.C = nullptr;
          lc.bytes = 0;
          if (lbytes > 0 && dmalloc(reinterpret_cast<void **>(&lc.C), lbytes) != cudaSuccess) {
            cudaGetLastError();
            set_error("cannot allocate %.3f GB for the left vectors", lbytes / 1e9);
            return GFCC_ERR_OOM;
          }
          lc.bytes = lbytes;
        }
      }
      Cl = lc.C;
    }
    double *part = base + gw;
    int *d_tw = reinterpret_cast<int *>(part + nsplit * 2LL * nsys * n_left);
    int *d_ta = d_tw + nsys;
    int *d_porb = d_ta + nsys;
    double *g_Gm = part + nsplit * 2LL * nsys * n_left + 4LL * nsys + 64;
    double *g_feat = g_Gm + 2LL * nsys * GUESS_G;
    double *g_y = g_feat + (long long)nsys * GUESS_NF;
    double *g_coef = g_y + (long long)nsys * GUESS_NO;
    double *g_pred = g_coef + (long long)nsys * GUESS_NO;
    double *g_delta = g_pred + nsys;
    double *g_pf = g_delta + (long long)nsys * GUESS_K;
    double *g_work = g_pf + nsys;
    int *g_nbr = reinterpret_cast<int *>(g_work + (keep ? guess_gram_work_doubles(nsys, n) : 0));
    int *g_navail = g_nbr + (long long)nsys * GUESS_K;
    int *g_kind = g_navail + nsys;
    int *g_slot = g_kind + nsys;
    gm.eta = eta;
    gm.use_precond = c->precond == GFCC_PRECOND_DIAG;
    // left vectors for all orbitals of the overlap list (unless cached from an earlier solve)
    if (n_left > 0 && !left_ready) {
    PhaseTimer tleft(c, PH_OVERLAP);
    GFCC_TRY(build_left_vectors(c, sector, n_left, d_left, Cl, st));
    const int *hl = ol.left_host(ip);
    c->left_cache[ip ? 0 : 1].orb.assign(hl, hl + n_left);
    }
    if (mixed && guess == GFCC_GUESS_ZERO) {
      // continuous batching: a slot whose system has converged (or spent its budget) after a
      // refinement step is finalised (G row, statistics, kept solution) and refilled with the next
      // task, so the batched contractions keep running on live systems; once the task list is
      // exhausted the live slots are compacted to the front and the batch shrinks with them
      int ns = nsys;   // slots in use (a prefix of the nsys slots)
      std::vector<long long> task(nsys, -1);
      std::vector<int> h_tw(nsys, 0), h_ta(nsys, 0), h_done(nsys, 0), h_state(nsys), sl_it(nsys, 0), sl_outer(nsys, 0);
      std::vector<int> h_twf(nsys, -1), h_mask(nsys, 0), h_slot(nsys, -1), perm;
      std::vector<double> h_rel(nsys, 0.0);
      int *d_twf = d_porb + nsys;   // within the 4 nsys doubles reserved after the partials
      int *d_mask = d_twf + nsys;
      long long next = 0;
      gm.tol_outer = tol;
      auto upload_tasks = [&]() -> int {
        for (int s = 0; s < ns; s++) {
          const long long t = task[s] >= 0 ? task[s] : 0;
          h_tw[s] = (int)(t / n_orb);
          h_ta[s] = (int)(t % n_orb);
        }
        GFCC_CUDA(cudaMemcpyAsync(d_tw, h_tw.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st));
        GFCC_CUDA(cudaMemcpyAsync(d_ta, h_ta.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st));
        gather_omega_kernel<<<cdiv(ns, 128), 128, 0, st>>>(d_om, d_tw, ns, gm.omega);
        GFCC_LAUNCH_CHECK();
        gather_orb_kernel<<<cdiv(ns, 128), 128, 0, st>>>(d_orb, d_ta, ns, d_porb);
        GFCC_LAUNCH_CHECK();
        return GFCC_OK;
      };
      auto load_slots = [&](bool all) -> int {
        // tasks of the (re)filled slots: omega, orbital, right-hand side, X = 0, R = B0
        for (int s = 0; s < ns; s++) h_mask[s] = all || h_mask[s] ? 1 : 0;
        GFCC_TRY(upload_tasks());
        GFCC_CUDA(cudaMemcpyAsync(d_mask, h_mask.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st));
        {
          PhaseTimer trhs(c, PH_OVERLAP);
          GFCC_TRY(build_rhs_masked(c, sector, ns, d_porb, d_mask, gm.rhs(), st));
        }
        for (int s = 0; s < ns; s++)
          if (h_mask[s] && task[s] < 0) {
            // an empty slot: zero right-hand side (inert: ||b|| = 0 counts as converged)
            GFCC_CUDA(cudaMemsetAsync(gm.rhs() + 2LL * s * n, 0, sizeof(double) * 2 * n, st));
          }
        GFCC_TRY(gm.reset_slots(d_mask));
        GFCC_TRY(gm.refine_norms());
        return GFCC_OK;
      };
      for (int s = 0; s < nsys; s++) task[s] = next < ntasks ? next++ : -1;
      GFCC_TRY(load_slots(true));
      GFCC_TRY(umma_error_reset(st));
      bool first = true;
      for (int step = 0;; step++) {
        if (first) {
          // X = 0: R = B0 already; only the norms and the checks
          GFCC_TRY(gm.refine_residual_free(h_done.data(), h_rel.data()));
          first = false;
        } else {
          GFCC_TRY(gm.refine_residual(h_done.data(), h_rel.data()));
        }
        bool any_fin = false, any_active = false;
        for (int s = 0; s < ns; s++) {
          h_twf[s] = -1;
          h_mask[s] = 0;
          if (task[s] < 0) continue;
          sl_outer[s]++;
          const bool conv = h_done[s] == 1;
          const bool fail = !conv && (sl_it[s] >= c->max_iters || sl_outer[s] > 400);
          if (!conv && !fail) {
            any_active = true;
            continue;
          }
          // finalise the slot
          const long long t = task[s];
          const long long idx = stat_off + t;
          c->st_iters[idx] = sl_it[s];
          c->st_relres[idx] = h_rel[s];
          c->st_relres0[idx] = 1.0;
          c->st_outer[idx] = sl_outer[s];
          c->st_status[idx] = conv ? GFCC_STATUS_CONVERGED : GFCC_STATUS_NOT_CONVERGED;
          all_ok &= conv;
          h_twf[s] = h_tw[s];
          any_fin = true;
        }
        if (any_fin && n_left > 0) {
          GFCC_CUDA(cudaMemcpyAsync(d_twf, h_twf.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st));
          {
            PhaseTimer tov(c, PH_OVERLAP);
            Contract k;
            k.A = gm.solution(); k.am = imap2(2, 1, 2 * n); k.ak = imap1(2);
            k.B = Cl; k.bk = imap1(1); k.bn = imap1(n);
            k.C = part; k.cm = imap1(n_left); k.cn = imap1(1);
            k.M = 2LL * ns; k.N = n_left; k.K = n;
            k.nsplit = nsplit; k.kchunk = 8192; k.scz = 2LL * ns * n_left;
            GFCC_TRY(contract_f64(k, st));
            overlap_scatter_kernel<<<grid1d((long long)ns * n_left), 256, 0, st>>>(
                part, (int)nsplit, ns, ns, n_left, d_twf, d_ta, ip ? 1 : 0, ol.nP, ol.nQ, d_G);
            GFCC_LAUNCH_CHECK();
          }
        }
        if (any_fin) {
          if (keep) {
            for (int s = 0; s < ns; s++) h_slot[s] = h_twf[s] >= 0 ? h_tw[s] * n_orb + h_ta[s] : -1;
            GFCC_CUDA(cudaMemcpyAsync(g_slot, h_slot.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st));
            GFCC_TRY(guess_store_put(st, ns, n, gm.solution(), n, g_slot, c->kept.X));
            for (int s = 0; s < ns; s++)
              if (h_twf[s] >= 0 && h_done[s] == 1) c->kept.done[(size_t)h_tw[s] * n_orb + h_ta[s]] = 1;
          }
          if (c->sink != nullptr) {
            for (int s = 0; s < ns; s++)
              if (h_twf[s] >= 0)
                GFCC_CUDA(cudaMemcpyAsync(c->sink + 2 * task[s] * n, gm.solution() + 2LL * s * n,
                                          sizeof(double) * 2 * n, cudaMemcpyDeviceToDevice, st));
          }
          // refill the finished slots while tasks remain
          bool refill = false;
          for (int s = 0; s < ns; s++) {
            if (h_twf[s] < 0) continue;
            task[s] = next < ntasks ? next++ : -1;
            sl_it[s] = 0;
            sl_outer[s] = 0;
            h_mask[s] = 1;
            refill = true;
            if (task[s] >= 0) any_active = true;
          }
          if (refill) {
            GFCC_TRY(load_slots(false));
            // the refilled slots start from X = 0: residual R = B0 (set by reset_slots), checked below
            GFCC_TRY(gm.refine_residual_free(h_done.data(), h_rel.data()));
            for (int s = 0; s < ns; s++)
              if (h_mask[s] && task[s] >= 0) sl_outer[s] = 1;
          }
        }
        if (!any_active) break;
        // inner correction for the live slots (done and empty slots have R = 0)
        for (int s = 0; s < ns; s++)
          if (task[s] < 0) h_done[s] = 1;
        // the batch size only stays put while tasks remain (the drain compacts it)
        gm.graphs_ok = next < ntasks;
        GFCC_TRY(gm.refine_correct(h_done.data(), h_state.data(), sl_it.data()));
        // drain: no task left to refill with, so move the live slots to the front and shrink the batch
        if (next >= ntasks) {
          perm.clear();
          for (int s = 0; s < ns; s++)
            if (task[s] >= 0) perm.push_back(s);
          const int na = (int)perm.size();
          if (na > 0 && na < ns) {
            GFCC_CUDA(cudaMemcpyAsync(d_mask, perm.data(), sizeof(int) * na, cudaMemcpyHostToDevice, st));
            GFCC_TRY(gm.compact_slots(d_mask, na));
            for (int q = 0; q < na; q++) {
              const int s = perm[q];
              task[q] = task[s];
              sl_it[q] = sl_it[s];
              sl_outer[q] = sl_outer[s];
            }
            ns = na;
            GFCC_TRY(upload_tasks());
            GFCC_TRY(gm.refine_norms());
          }
        }
      }
      GFCC_TRY(umma_error_check(st));
      gm.nsys = nsys;
      stat_off += ntasks;
      continue;
    }
    // task order: frequency-major; with initial guesses the frequencies go in the order of
    // guess_frequency_order so that later ones have converged neighbours on both sides
    std::vector<int> word(n_omega);
    for (int w = 0; w < n_omega; w++) word[w] = w;
    if (guess != GFCC_GUESS_ZERO) word = guess_frequency_order(c->kept.omega);
    std::vector<int> h_tw(nsys), h_ta(nsys), h_state(nsys), h_it(nsys), h_kind(nsys), h_nbr((size_t)nsys * GUESS_K),
        h_navail(nsys), h_slot(nsys), h_outer(nsys, 0);
    std::vector<double> h_rel(nsys), h_rel0(nsys), h_pred(nsys), h_delta((size_t)nsys * GUESS_K), h_pf(nsys);
    for (long long t0 = 0; t0 < ntasks; t0 += nsys) {
      const int nb = (int)std::min<long long>(nsys, ntasks - t0);
      // pad a short last batch by repeating its last task (results of the padding are dropped)
      for (int s = 0; s < nsys; s++) {
        const long long t = t0 + std::min(s, nb - 1);
        h_tw[s] = word[t / n_orb];
        h_ta[s] = (int)(t % n_orb);
      }
      GFCC_CUDA(cudaMemcpyAsync(d_tw, h_tw.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, st));
      GFCC_CUDA(cudaMemcpyAsync(d_ta, h_ta.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, st));
      gather_omega_kernel<<<cdiv(nsys, 128), 128, 0, st>>>(d_om, d_tw, nsys, gm.omega);
      GFCC_LAUNCH_CHECK();
      gather_orb_kernel<<<cdiv(nsys, 128), 128, 0, st>>>(d_orb, d_ta, nsys, d_porb);
      GFCC_LAUNCH_CHECK();
      {
      PhaseTimer trhs(c, PH_OVERLAP);
      GFCC_TRY(build_rhs(c, sector, nsys, d_porb, gm.rhs(), st));
      }
      bool use_x0 = false;
      if (guess != GFCC_GUESS_ZERO) {
        // neighbours among the converged solutions of earlier batches (same orbital)
        PhaseTimer tg(c, PH_GUESS);
        const KeptSolutions &kp = c->kept;
        for (int s = 0; s < nsys; s++) {
          int idx[GUESS_K];
          const int a = h_ta[s], w = h_tw[s];
          const int k = guess_neighbours(kp.omega, kp.done.data() + a, n_orb, w, GUESS_K, idx);
          h_navail[s] = k;
          for (int q = 0; q < GUESS_K; q++) {
            h_nbr[s * GUESS_K + q] = q < k ? idx[q] * n_orb + a : -1;
            h_delta[s * GUESS_K + q] = q < k ? kp.omega[w] - kp.omega[idx[q]] : 0.0;
          }
          h_pf[s] = (double)kp.orb[a] / (double)c->n;
        }
        GFCC_CUDA(cudaMemcpyAsync(g_nbr, h_nbr.data(), sizeof(int) * nsys * GUESS_K, cudaMemcpyHostToDevice, st));
        GFCC_CUDA(cudaMemcpyAsync(g_navail, h_navail.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, st));
        GFCC_CUDA(cudaMemcpyAsync(g_delta, h_delta.data(), sizeof(double) * nsys * GUESS_K, cudaMemcpyHostToDevice, st));
        GFCC_CUDA(cudaMemcpyAsync(g_pf, h_pf.data(), sizeof(double) * nsys, cudaMemcpyHostToDevice, st));
        GFCC_TRY(guess_gram(st, nsys, n, gm.rhs(), n, kp.X, g_nbr, g_delta, gm.omega, eta, g_pf, g_Gm, g_feat, g_work));
        if (guess == GFCC_GUESS_LEARNED) GFCC_TRY(mlp_infer(c->mlp, st, nsys, g_feat, g_y));
        GFCC_TRY(guess_choose(st, nsys, guess, g_Gm, g_y, g_navail, g_coef, g_pred, g_kind));
        GFCC_TRY(guess_combine(st, nsys, n, kp.X, g_nbr, g_coef, g_kind, gm.solution(), n));
        use_x0 = true;
      }
      if (mixed) {
        GFCC_TRY(umma_error_reset(st));
        GFCC_TRY(gm.solve_refined(tol, c->inner_tol, c->max_iters, h_state.data(), h_it.data(), use_x0,
                                  h_outer.data()));
        GFCC_TRY(umma_error_check(st));
      } else {
        GFCC_TRY(gm.solve(tol, c->max_iters, h_state.data(), 0, use_x0));
      }
      // overlaps: part[z][(s,t)][q] = sum_{mu in chunk z} x_s[mu] C[q][mu]
      if (n_left > 0) {
      PhaseTimer tov(c, PH_OVERLAP);
      Contract k;
      k.A = gm.solution(); k.am = imap2(2, 1, 2 * n); k.ak = imap1(2);
      k.B = Cl; k.bk = imap1(1); k.bn = imap1(n);
      k.C = part; k.cm = imap1(n_left); k.cn = imap1(1);
      k.M = 2LL * nsys; k.N = n_left; k.K = n;
      k.nsplit = nsplit; k.kchunk = 8192; k.scz = 2LL * nsys * n_left;
      GFCC_TRY(contract_f64(k, st));
      overlap_scatter_kernel<<<grid1d((long long)nb * n_left), 256, 0, st>>>(part, (int)nsplit, nsys, nb, n_left,
                                                                              d_tw, d_ta, ip ? 1 : 0, ol.nP, ol.nQ,
                                                                              d_G);
      GFCC_LAUNCH_CHECK();
      }
      if (c->sink != nullptr) {
        for (int s = 0; s < nb; s++)
          GFCC_CUDA(cudaMemcpyAsync(c->sink + 2 * ((long long)h_tw[s] * n_orb + h_ta[s]) * n,
                                    gm.solution() + 2LL * s * n, sizeof(double) * 2 * n, cudaMemcpyDeviceToDevice,
                                    st));
      }
      if (keep) {
        for (int s = 0; s < nsys; s++) h_slot[s] = s < nb ? h_tw[s] * n_orb + h_ta[s] : -1;
        GFCC_CUDA(cudaMemcpyAsync(g_slot, h_slot.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, st));
        GFCC_TRY(guess_store_put(st, nsys, n, gm.solution(), n, g_slot, c->kept.X));
      }
      GFCC_CUDA(cudaMemcpyAsync(h_it.data(), gm.iters, sizeof(int) * nsys, cudaMemcpyDeviceToHost, st));
      GFCC_CUDA(cudaMemcpyAsync(h_rel.data(), gm.relres, sizeof(double) * nsys, cudaMemcpyDeviceToHost, st));
      GFCC_CUDA(cudaMemcpyAsync(h_rel0.data(), gm.relres0, sizeof(double) * nsys, cudaMemcpyDeviceToHost, st));
      GFCC_CUDA(cudaMemcpyAsync(h_state.data(), gm.state, sizeof(int) * nsys, cudaMemcpyDeviceToHost, st));
      if (guess != GFCC_GUESS_ZERO) {
        GFCC_CUDA(cudaMemcpyAsync(h_kind.data(), g_kind, sizeof(int) * nsys, cudaMemcpyDeviceToHost, st));
        GFCC_CUDA(cudaMemcpyAsync(h_pred.data(), g_pred, sizeof(double) * nsys, cudaMemcpyDeviceToHost, st));
      }
      GFCC_CUDA(cudaStreamSynchronize(st));
      for (int s = 0; s < nb; s++) {
        // statistics in (omega, orbital) order of the request
        const long long idx = stat_off + (long long)h_tw[s] * n_orb + h_ta[s];
        c->st_iters[idx] = h_it[s];
        c->st_relres[idx] = h_rel[s];
        c->st_relres0[idx] = h_rel0[s];
        c->st_outer[idx] = mixed ? h_outer[s] : 0;
        c->st_status[idx] = h_state[s] == 3 ? GFCC_STATUS_CONVERGED : GFCC_STATUS_NOT_CONVERGED;
        if (guess != GFCC_GUESS_ZERO) {
          c->st_guess[idx] = h_kind[s];
          c->st_guess_pred[idx] = h_pred[s];
        }
        // only converged solutions serve as neighbours (the Gram identity assumes A X_k = b)
        if (keep && h_state[s] == 3) c->kept.done[(size_t)h_tw[s] * n_orb + h_ta[s]] = 1;
        all_ok &= h_state[s] == 3;
      }
    }
    stat_off += ntasks;
  }
  return all_ok ? GFCC_OK : GFCC_WARN_NOT_CONVERGED;
}

int check_solve_args(gfcc_ctx *c, int n_omega, double eta, int n_orb, double tol) {
  if (c == nullptr) {
    set_error("gfcc_solve: ctx is NULL");
    return GFCC_ERR_ARG;
  }
  if (n_omega < 0 || n_orb < 0 || !(eta > 0.0) || !(tol > 0.0)) {
    set_error("gfcc_solve: need n_omega >= 0, n_orb >= 0, eta > 0, tol > 0");
    return GFCC_ERR_ARG;
  }
  return GFCC_OK;
}

// gfcc_solve / gfcc_solve_block on host arrays: device copies of the frequencies, the two orbital
// lists and G around solve_impl
int solve_host(gfcc_ctx *c, int n_omega, const double *omegas, double eta, int nP, const int *P, int nQ, const int *Q,
               double tol, double *G) {
  // G == nullptr: the solve runs and G stays on the device (internal callers that only want the
  // solutions); the entry points reject a NULL G themselves
  if (omegas == nullptr || P == nullptr || Q == nullptr) {
    set_error("gfcc_solve: NULL omegas or orbitals");
    return GFCC_ERR_ARG;
  }
  for (int pass = 0; pass < 2; pass++) {
    const int cnt = pass ? nQ : nP;
    const int *lst = pass ? Q : P;
    for (int a = 0; a < cnt; a++)
      if (lst[a] < 0 || lst[a] >= c->n) {
        set_error("gfcc_solve: orbital index %d out of range [0, %d)", lst[a], c->n);
        return GFCC_ERR_ARG;
      }
  }
  for (int w = 0; w < n_omega; w++)
    if (!std::isfinite(omegas[w])) {
      set_error("gfcc_solve: omega[%d] is not finite", w);
      return GFCC_ERR_ARG;
    }
  double *d_om = nullptr, *d_G = nullptr;
  int *d_P = nullptr, *d_Q = nullptr;
  const size_t gbytes = sizeof(double) * 2 * (size_t)n_omega * nP * nQ;
  if (dmalloc((void **)&d_om, sizeof(double) * n_omega) != cudaSuccess ||
      dmalloc((void **)&d_P, sizeof(int) * nP) != cudaSuccess || dmalloc((void **)&d_Q, sizeof(int) * nQ) != cudaSuccess ||
      dmalloc((void **)&d_G, gbytes) != cudaSuccess) {
    cudaGetLastError();
    dfree(d_om);
    dfree(d_P);
    dfree(d_Q);
    dfree(d_G);
    set_error("gfcc_solve: cannot allocate the frequency / orbital / G buffers");
    return GFCC_ERR_OOM;
  }
  int s = GFCC_OK;
  if (cudaMemcpyAsync(d_om, omegas, sizeof(double) * n_omega, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(d_P, P, sizeof(int) * nP, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(d_Q, Q, sizeof(int) * nQ, cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
    set_error("gfcc_solve: host-to-device copy failed");
    s = GFCC_ERR_CUDA;
  }
  OrbLists ol;
  ol.nP = nP;
  ol.nQ = nQ;
  ol.dP = d_P;
  ol.dQ = d_Q;
  ol.hP = P;
  ol.hQ = Q;
  if (s == GFCC_OK) s = solve_impl(c, n_omega, d_om, eta, ol, tol, d_G);
  if (s >= 0) {
    if ((G != nullptr && cudaMemcpyAsync(G, d_G, gbytes, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess) ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
      set_error("gfcc_solve: device-to-host copy of G failed");
      s = GFCC_ERR_CUDA;
    }
  }
  dfree(d_om);
  dfree(d_P);
  dfree(d_Q);
  dfree(d_G);
  return s;
}

}  // namespace

int check_input_tensor(cudaStream_t st, const double *x, long long d0, long long d1, long long d2, long long d3,
                       int s01, int s23, double sign, double rel, const char *name) {
  return check_tensor(st, x, d0, d1, d2, d3, s01, s23, sign, rel, name);
}

int solve_rows_host(gfcc_ctx *c, int n_omega, const double *omegas, double eta, int n_orb, const int *orbitals,
                    double tol, double *G) {
  GFCC_TRY(check_solve_args(c, n_omega, eta, n_orb, tol));
  return solve_host(c, n_omega, omegas, eta, n_orb, orbitals, n_orb, orbitals, tol, G);
}

int build_rhs_masked(gfcc_ctx *c, int sector, int nsys, const int *d_porb, const int *d_mask, double *B,
                     cudaStream_t st) {
  if (nsys <= 0) return GFCC_OK;
  if (c->rhf) return build_rhs_rhf(c, nsys, d_porb, d_mask, B, st);
  if (sector == GFCC_SECTOR_IP) {
    rhs_ip_kernel<<<grid1d(c->dim_ip * nsys), 256, 0, st>>>(B, c->dim_ip, nsys, d_porb, c->o, c->v, c->t1, c->t2,
                                                            d_mask);
  } else {
    rhs_ea_kernel<<<grid1d(c->dim_ea * nsys), 256, 0, st>>>(B, c->dim_ea, nsys, d_porb, c->o, c->v, c->Pv, c->t1,
                                                            c->t2, d_mask);
  }
  GFCC_LAUNCH_CHECK();
  return GFCC_OK;
}

int build_rhs(gfcc_ctx *c, int sector, int nsys, const int *d_porb, double *B, cudaStream_t st) {
  return build_rhs_masked(c, sector, nsys, d_porb, nullptr, B, st);
}

// left vectors C[q][mu] (real, [nq][dim]) of the orbitals d_orb (device) of one sector (eq. gfxn2)
int build_left_vectors(gfcc_ctx *c, int sector, int nq, const int *d_orb, double *C, cudaStream_t st) {
  if (nq <= 0) return GFCC_OK;
  if (c->rhf) return build_left_rhf(c, nq, d_orb, C, st);
  if (sector == GFCC_SECTOR_IP) {
    const long long n = c->dim_ip;
    left_ip_1h_kernel<<<nq * c->o, 256, 0, st>>>(C, n, nq, d_orb, c->o, c->v, c->t1, c->t2, c->l1, c->l2);
    GFCC_LAUNCH_CHECK();
    if (n > c->o) {
      left_ip_2h1p_kernel<<<grid1d((n - c->o) * nq), 256, 0, st>>>(C, n, nq, d_orb, c->o, c->v, c->t1, c->l1, c->l2);
      GFCC_LAUNCH_CHECK();
    }
  } else {
    const long long n = c->dim_ea;
    left_ea_1p_kernel<<<nq * c->v, 256, 0, st>>>(C, n, nq, d_orb, c->o, c->v, c->t1, c->t2, c->l1, c->l2);
    GFCC_LAUNCH_CHECK();
    if (n > c->v) {
      left_ea_2p1h_kernel<<<grid1d((n - c->v) * nq), 256, 0, st>>>(C, n, nq, d_orb, c->o, c->v, c->Pv, c->t1, c->l1,
                                                                     c->l2);
      GFCC_LAUNCH_CHECK();
    }
  }
  return GFCC_OK;
}

// gfcc_solve over one sector (rows and columns over the same orbital list) with every finished
// system's FP64 solution copied to d_sink ([omega][orbital][dim] complex); G to the host if h_G.
// The statistics of the solve stay in the context.
int solve_for_sink(gfcc_ctx *c, int sector, int n_omega, const double *h_om, double eta, int n_orb,
                   const int *h_orb, double tol, double *d_sink, double *h_G) {
  const int saved = c->sectors;
  c->sectors = sector;
  c->sink = d_sink;
  const int rc = solve_host(c, n_omega, h_om, eta, n_orb, h_orb, n_orb, h_orb, tol, h_G);
  c->sink = nullptr;
  c->sectors = saved;
  return rc;
}

}  // namespace gfcc

using namespace gfcc;

extern "C" {

int gfcc_create(int o, int v, int L, const double *fock, const double *chol, const double *t1, const double *t2,
                const double *lambda, gfcc_ctx **out) {
  return create_impl(o, v, L, fock, chol, t1, t2, lambda, GFCC_SECTOR_BOTH, GFCC_PREC_FP64, out);
}

int gfcc_create_ex(int o, int v, int L, const double *fock, const double *chol, const double *t1, const double *t2,
                   const double *lambda, int sectors, int precision, gfcc_ctx **out) {
  return create_impl(o, v, L, fock, chol, t1, t2, lambda, sectors, precision, out);
}

int gfcc_create_rhf(int o, int v, int L, const double *fock, const double *chol, const double *t1, const double *t2,
                    const double *lambda, gfcc_ctx **out) {
  return create_impl(o, v, L, fock, chol, t1, t2, lambda, GFCC_SECTOR_IP, GFCC_PREC_FP64, out, 1);
}

int gfcc_set_option(gfcc_ctx *c, int key, double value) {
  if (c == nullptr) {
    set_error("gfcc_set_option: ctx is NULL");
    return GFCC_ERR_ARG;
  }
  const int iv = (int)value;
  switch (key) {
    case GFCC_OPT_SECTOR:
      if (iv < 1 || iv > 3 || (iv & ~c->sectors)) {
        set_error("gfcc_set_option: sector %d not built in this context", iv);
        return GFCC_ERR_ARG;
      }
      c->sectors = iv;
      return GFCC_OK;
    case GFCC_OPT_PRECISION:
      if (iv != GFCC_PREC_FP64 && iv != GFCC_PREC_MIXED_BF16) break;
      c->precision = iv;
      return GFCC_OK;
    case GFCC_OPT_RESTART:
      if (iv < 1 || iv > 64) break;
      c->restart = iv;
      return GFCC_OK;
    case GFCC_OPT_INNER_RESTART:
      if (iv < 1 || iv > 64) break;
      c->inner_restart = iv;
      return GFCC_OK;
    case GFCC_OPT_MAX_ITERS:
      if (iv < 1) break;
      c->max_iters = iv;
      return GFCC_OK;
    case GFCC_OPT_PRECOND:
      if (iv != GFCC_PRECOND_NONE && iv != GFCC_PRECOND_DIAG) break;
      c->precond = iv;
      return GFCC_OK;
    case GFCC_OPT_BATCH:
      if (iv < 0 || iv > 4096) break;
      c->batch = iv;
      return GFCC_OK;
    case GFCC_OPT_INNER_CYCLES:
      if (iv < 1 || iv > 1000) break;
      c->inner_cycles = iv;
      return GFCC_OK;
    case GFCC_OPT_EMU_LEVEL:
      if (iv < 2 || iv > 2 * c->emu_S) break;
      c->emu_P = iv;
      return GFCC_OK;
    case GFCC_OPT_RESIDUAL:
      if (iv != 0 && iv != 1) break;
      c->residual_emulated = iv;
      return GFCC_OK;
    case GFCC_OPT_INNER_TOL:
      if (!(value > 0.0 && value < 1.0)) break;
      c->inner_tol = value;
      return GFCC_OK;
    case GFCC_OPT_CLOSED_SHELL_EMULATE:
      if (!c->rhf || (iv != 0 && iv != 1)) break;
      c->rhf_emulate = iv;
      return GFCC_OK;
    case GFCC_OPT_GUESS:
      if (iv != GFCC_GUESS_ZERO && iv != GFCC_GUESS_LEARNED && iv != GFCC_GUESS_MINRES) break;
      if (c->rhf && iv != GFCC_GUESS_ZERO) {
        set_error("gfcc_set_option: closed-shell contexts solve from the zero guess only");
        return GFCC_ERR_ARG;
      }
      c->guess = iv;
      return GFCC_OK;
    case GFCC_OPT_INNER_KRYLOV:
      if (iv != 32 && iv != 64) break;
      c->inner_fp64 = iv == 64 ? 1 : 0;
      return GFCC_OK;
    case GFCC_OPT_AUTOTUNE:
      if (iv != 0 && iv != 1) break;
      umma_set_autotune(iv == 1);
      return GFCC_OK;
    case GFCC_OPT_INCREMENTAL:
      if (iv != 0 && iv != 1) break;
      c->incremental = iv;
      return GFCC_OK;
    case GFCC_OPT_EMU_FUSED_N:
      if (iv < 0) break;
      emu_set_fused_max_n(iv);
      return GFCC_OK;
    case GFCC_OPT_GRAPHS:
      if (iv != 0 && iv != 1) break;
      c->use_graphs = iv;
      return GFCC_OK;
    case GFCC_OPT_KEEP_SOLUTIONS:
      if (iv != 0 && iv != 1) break;
      c->keep_solutions = iv;
      return GFCC_OK;
    default:
      set_error("gfcc_set_option: unknown key %d", key);
      return GFCC_ERR_ARG;
  }
  set_error("gfcc_set_option: value %g out of range for key %d", value, key);
  return GFCC_ERR_ARG;
}

int gfcc_set_process_option(int key, double value) {
  switch (key) {
    case GFCC_OPT_AUTOTUNE:
      if (value != 0.0 && value != 1.0) break;
      umma_set_autotune(value == 1.0);
      return GFCC_OK;
    case GFCC_OPT_EMU_FUSED_N:
      if (!(value >= 0.0)) break;
      emu_set_fused_max_n((long long)value);
      return GFCC_OK;
    case GFCC_OPT_GEMM_PAIR:
      if (value != 0.0 && value != 1.0 && value != 2.0) break;
      umma_set_pair_mode((int)value);
      return GFCC_OK;
    case GFCC_OPT_GEMM_PERSIST:
      if (value != 0.0 && value != 1.0 && value != 2.0) break;
      umma_set_persist_mode((int)value);
      return GFCC_OK;
    case GFCC_OPT_SETUP_EMULATE_FLOPS:
      if (!(value >= 0.0)) break;
      g_emulate_min_flops = value;
      return GFCC_OK;
    case GFCC_OPT_WAIT_NS:
    case GFCC_OPT_TEST_NO_LOADS: {
      static unsigned long long wait_ns = 1000000000ULL;
      static bool no_loads = false;
      if (key == GFCC_OPT_WAIT_NS) {
        if (!(value >= 1.0 && value <= 1e11)) break;
        wait_ns = (unsigned long long)value;
      } else {
        if (value != 0.0 && value != 1.0) break;
        no_loads = value == 1.0;
      }
      umma_set_wait(wait_ns, no_loads);
      return GFCC_OK;
    }
    default:
      set_error("gfcc_set_process_option: unknown key %d", key);
      return GFCC_ERR_ARG;
  }
  set_error("gfcc_set_process_option: value %g out of range for key %d", value, key);
  return GFCC_ERR_ARG;
}

int gfcc_set_stream(gfcc_ctx *c, void *stream) {
  if (c == nullptr) {
    set_error("gfcc_set_stream: ctx is NULL");
    return GFCC_ERR_ARG;
  }
  c->stream = stream ? static_cast<cudaStream_t>(stream) : c->own_stream;
  return GFCC_OK;
}

int gfcc_solve_device(gfcc_ctx *c, int n_omega, const double *omegas_dev, double eta, int n_orb,
                      const int *orbitals_dev, double tol, double *G_dev) {
  GFCC_TRY(check_solve_args(c, n_omega, eta, n_orb, tol));
  if (n_omega == 0 || n_orb == 0) return GFCC_OK;
  // orbital range check on a host copy
  std::vector<int> h_orb(n_orb);
  GFCC_CUDA(cudaMemcpyAsync(h_orb.data(), orbitals_dev, sizeof(int) * n_orb, cudaMemcpyDeviceToHost, c->stream));
  GFCC_CUDA(cudaStreamSynchronize(c->stream));
  for (int x : h_orb)
    if (x < 0 || x >= c->n) {
      set_error("gfcc_solve: orbital index %d out of range [0, %d)", x, c->n);
      return GFCC_ERR_ARG;
    }
  OrbLists ol;
  ol.nP = ol.nQ = n_orb;
  ol.dP = ol.dQ = orbitals_dev;
  ol.hP = ol.hQ = h_orb.data();
  return solve_impl(c, n_omega, omegas_dev, eta, ol, tol, G_dev);
}


int gfcc_solve(gfcc_ctx *c, int n_omega, const double *omegas, double eta, int n_orb, const int *orbitals, double tol,
               double *G) {
  GFCC_TRY(check_solve_args(c, n_omega, eta, n_orb, tol));
  if (n_omega == 0 || n_orb == 0) return GFCC_OK;
  if (G == nullptr) {
    set_error("gfcc_solve: G is NULL");
    return GFCC_ERR_ARG;
  }
  return solve_host(c, n_omega, omegas, eta, n_orb, orbitals, n_orb, orbitals, tol, G);
}

int gfcc_solve_block(gfcc_ctx *c, int n_omega, const double *omegas, double eta, int n_p, const int *p_orbitals,
                     int n_q, const int *q_orbitals, double tol, double *G) {
  GFCC_TRY(check_solve_args(c, n_omega, eta, n_p, tol));
  if (n_q < 0) {
    set_error("gfcc_solve_block: need n_q >= 0");
    return GFCC_ERR_ARG;
  }
  if (n_omega == 0 || n_p == 0 || n_q == 0) return GFCC_OK;
  if (G == nullptr) {
    set_error("gfcc_solve_block: G is NULL");
    return GFCC_ERR_ARG;
  }
  return solve_host(c, n_omega, omegas, eta, n_p, p_orbitals, n_q, q_orbitals, tol, G);
}

int gfcc_last_stats(gfcc_ctx *c, int *count, int *iters, double *relres, int *status) {
  if (c == nullptr || count == nullptr) {
    set_error("gfcc_last_stats: NULL argument");
    return GFCC_ERR_ARG;
  }
  const int total = (int)c->st_iters.size();
  const int cap = *count;
  const int nout = std::min(cap, total);
  for (int i = 0; i < nout; i++) {
    if (iters) iters[i] = c->st_iters[i];
    if (relres) relres[i] = c->st_relres[i];
    if (status) status[i] = c->st_status[i];
  }
  *count = total;
  return GFCC_OK;
}

int gfcc_solve_batch(gfcc_ctx *const *ctxs, int n_ctx, const gfcc_request *reqs, int *codes) {
  if (n_ctx < 0 || (n_ctx > 0 && (ctxs == nullptr || reqs == nullptr))) {
    set_error("gfcc_solve_batch: bad arguments");
    return GFCC_ERR_ARG;
  }
  for (int i = 0; i < n_ctx; i++) {
    if (ctxs[i] == nullptr) {
      set_error("gfcc_solve_batch: context %d is NULL", i);
      return GFCC_ERR_ARG;
    }
    for (int j = 0; j < i; j++)
      if (ctxs[j] == ctxs[i]) {
        set_error("gfcc_solve_batch: context %d appears twice (contexts are not thread-safe)", i);
        return GFCC_ERR_ARG;
      }
  }
  if (n_ctx == 0) return GFCC_OK;
  int dev = 0;
  GFCC_CUDA(cudaGetDevice(&dev));
  const int nthreads = std::min(n_ctx, 8);
  std::vector<int> rc(n_ctx, GFCC_OK);
  std::vector<std::string> msg(n_ctx);
  std::vector<double> share(n_ctx);
  for (int i = 0; i < n_ctx; i++) {
    share[i] = ctxs[i]->mem_share;
    ctxs[i]->mem_share = share[i] / nthreads;   // concurrent solves split the free memory
  }
  std::atomic<int> next{0};
  auto worker = [&]() {
    if (cudaSetDevice(dev) != cudaSuccess) {
      cudaGetLastError();
    }
    for (int i = next++; i < n_ctx; i = next++) {
      const gfcc_request &r = reqs[i];
      rc[i] = gfcc_solve(ctxs[i], r.n_omega, r.omegas, r.eta, r.n_orb, r.orbitals, r.tol, r.G);
      if (rc[i] < 0) msg[i] = gfcc_last_error();
    }
  };
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; t++) th.emplace_back(worker);
  for (auto &t : th) t.join();
  for (int i = 0; i < n_ctx; i++) ctxs[i]->mem_share = share[i];
  int out = GFCC_OK;
  for (int i = 0; i < n_ctx; i++) {
    if (codes) codes[i] = rc[i];
    if (rc[i] < 0 && out >= 0) {
      set_error("gfcc_solve_batch: context %d: %s", i, msg[i].c_str());
      out = rc[i];
    } else if (rc[i] == GFCC_WARN_NOT_CONVERGED && out == GFCC_OK) {
      out = GFCC_WARN_NOT_CONVERGED;
    }
  }
  return out;
}

int gfcc_guess_stats(gfcc_ctx *c, int *count, int *kind, double *pred, double *relres0) {
  if (c == nullptr || count == nullptr) {
    set_error("gfcc_guess_stats: NULL argument");
    return GFCC_ERR_ARG;
  }
  const int total = (int)c->st_guess.size();
  const int nout = std::min(*count, total);
  for (int i = 0; i < nout; i++) {
    if (kind) kind[i] = c->st_guess[i];
    if (pred) pred[i] = c->st_guess_pred[i];
    if (relres0) relres0[i] = c->st_relres0[i];
  }
  *count = total;
  return GFCC_OK;
}

int gfcc_refine_stats(gfcc_ctx *c, int *count, int *outer) {
  if (c == nullptr || count == nullptr) {
    set_error("gfcc_refine_stats: NULL argument");
    return GFCC_ERR_ARG;
  }
  const int total = (int)c->st_outer.size();
  const int nout = std::min(*count, total);
  for (int i = 0; i < nout && outer; i++) outer[i] = c->st_outer[i];
  *count = total;
  return GFCC_OK;
}

int gfcc_residual_stats(gfcc_ctx *c, long long *full, long long *incremental, double *mean_level) {
  if (c == nullptr) {
    set_error("gfcc_residual_stats: ctx is NULL");
    return GFCC_ERR_ARG;
  }
  if (full) *full = c->res_full;
  if (incremental) *incremental = c->res_inc;
  if (mean_level) *mean_level = c->res_inc > 0 ? (double)c->res_inc_levels / (double)c->res_inc : 0.0;
  return GFCC_OK;
}

int gfcc_set_guess_model(gfcc_ctx *c, gfcc_mlp *m) {
  if (c == nullptr) {
    set_error("gfcc_set_guess_model: ctx is NULL");
    return GFCC_ERR_ARG;
  }
  c->mlp = m;
  return GFCC_OK;
}

int gfcc_sigma(gfcc_ctx *c, int sector, int n_vec, const double *x, double *y) {
  return gfcc_sigma_ex(c, sector, GFCC_PREC_FP64, n_vec, x, y);
}

int gfcc_sigma_ex(gfcc_ctx *c, int sector, int precision, int n_vec, const double *x, double *y) {
  if (c == nullptr || x == nullptr || y == nullptr || n_vec < 0 ||
      (sector != GFCC_SECTOR_IP && sector != GFCC_SECTOR_EA) || !(c->sectors & sector)) {
    set_error("gfcc_sigma: bad arguments or sector not built");
    return GFCC_ERR_ARG;
  }
  const bool mixed = precision == GFCC_PREC_MIXED_BF16;
  const bool emu = precision == GFCC_PREC_FP64_EMULATED;
  const bool ip = sector == GFCC_SECTOR_IP;
  if ((precision != GFCC_PREC_FP64 && !mixed && !emu) ||
      ((mixed || emu) && (ip ? c->Wr_bf : c->Wre_bf) == nullptr)) {
    set_error("gfcc_sigma_ex: mixed / emulated precision needs a context created with GFCC_PREC_MIXED_BF16");
    return GFCC_ERR_ARG;
  }
  if (n_vec == 0) return GFCC_OK;
  const long long n = sector == GFCC_SECTOR_IP ? c->dim_ip : c->dim_ea;
  const long long ew = emu ? sigma_emu_work_doubles(c, std::min(n_vec, EMU_SUB_MAX)) : 0;
  const long long work = sigma_work_doubles(c, sector, n_vec) + 4LL * n_vec * n +
                         (mixed ? sigma_mixed_work_doubles(c, n_vec) : 0) + ew;
  GFCC_TRY(grow_scratch(c, sizeof(double) * work));
  double *dx = static_cast<double *>(c->scratch);
  double *dy = dx + 2LL * n_vec * n;
  double *w = dy + 2LL * n_vec * n;
  GFCC_CUDA(cudaMemcpyAsync(dx, x, sizeof(double) * 2 * n_vec * n, cudaMemcpyHostToDevice, c->stream));
  SysBatch b;
  b.nsys = n_vec;
  b.x = dx; b.ldx = n;
  b.y = dy; b.ldy = n;
  if (mixed || emu) {
    GFCC_TRY(umma_error_reset(c->stream));
    if (ip)
      GFCC_TRY(mixed ? apply_ip_mixed(c, b, w) : apply_ip_emu(c, b, w, ew));
    else
      GFCC_TRY(mixed ? apply_ea_mixed(c, b, w) : apply_ea_emu(c, b, w, ew));
    GFCC_TRY(umma_error_check(c->stream));
  } else {
    GFCC_TRY(sector == GFCC_SECTOR_IP ? apply_ip(c, b, w) : apply_ea(c, b, w));
  }
  GFCC_CUDA(cudaMemcpyAsync(y, dy, sizeof(double) * 2 * n_vec * n, cudaMemcpyDeviceToHost, c->stream));
  GFCC_CUDA(cudaStreamSynchronize(c->stream));
  return GFCC_OK;
}

int gfcc_dims(gfcc_ctx *c, long long *dim_ip, long long *dim_ea) {
  if (c == nullptr) {
    set_error("gfcc_dims: ctx is NULL");
    return GFCC_ERR_ARG;
  }
  if (dim_ip) *dim_ip = c->dim_ip;
  if (dim_ea) *dim_ea = c->dim_ea;
  return GFCC_OK;
}

void gfcc_destroy(gfcc_ctx *c) {
  if (c == nullptr) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  prof_resolve(c);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  for (void *p : c->allocs) dfree(p);
  if (c->scratch) dfree(c->scratch);
  for (auto &lc : c->left_cache)
    if (lc.C) dfree(lc.C);
  if (c->kept.X) dfree(c->kept.X);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  delete c;
}

const char *gfcc_last_error(void) { return g_err; }

int gfcc_profile(gfcc_ctx *c, int enable) {
  if (c == nullptr) {
    set_error("gfcc_profile: ctx is NULL");
    return GFCC_ERR_ARG;
  }
  if (c->stream) cudaStreamSynchronize(c->stream);
  prof_resolve(c);
  for (int i = 0; i < PH_COUNT; i++) {
    if (i == PH_SETUP) continue;   // the setup time of gfcc_create is kept
    c->prof_ms[i] = 0.0;
    c->prof_n[i] = 0;
    c->prof_flops[i] = 0.0;
  }
  c->prof = enable != 0;
  return GFCC_OK;
}

int gfcc_profile_read(gfcc_ctx *c, int phase, double *ms, long long *count, double *flops) {
  if (c == nullptr || phase < 0 || phase >= PH_COUNT) {
    set_error("gfcc_profile_read: bad ctx or phase");
    return GFCC_ERR_ARG;
  }
  if (c->stream) cudaStreamSynchronize(c->stream);
  prof_resolve(c);
  if (ms) *ms = c->prof_ms[phase];
  if (count) *count = c->prof_n[phase];
  if (flops) *flops = c->prof_flops[phase];
  return GFCC_OK;
}

long long gfcc_launch_count(void) { return gfcc::g_launches.load(); }

int gfcc_selftest_gemm_f64emu(int M, int N, int K, const double *A, const double *B, int S, int P, double *C) {
  if (M <= 0 || N <= 0 || K <= 0 || S < 1 || S > 12 || P < 2 || A == nullptr || B == nullptr || C == nullptr) {
    set_error("gfcc_selftest_gemm_f64emu: bad arguments");
    return GFCC_ERR_ARG;
  }
  void *da = nullptr, *db = nullptr, *dc = nullptr, *sa = nullptr, *sb = nullptr, *w = nullptr;
  cudaStream_t st = nullptr;
  int s = GFCC_OK;
  if (dmalloc(&da, sizeof(double) * M * K) != cudaSuccess || dmalloc(&db, sizeof(double) * N * K) != cudaSuccess ||
      dmalloc(&dc, sizeof(double) * M * N) != cudaSuccess ||
      dmalloc(&sa, emu_operand_bytes(M, K, S)) != cudaSuccess ||
      dmalloc(&sb, emu_operand_bytes(N, K, S)) != cudaSuccess ||
      dmalloc(&w, emu_gemm_work_bytes(M, N, K)) != cudaSuccess || cudaStreamCreate(&st) != cudaSuccess) {
    cudaGetLastError();
    set_error("gfcc_selftest_gemm_f64emu: allocation failed");
    s = GFCC_ERR_OOM;
  }
  if (s == GFCC_OK && (cudaMemcpy(da, A, sizeof(double) * M * K, cudaMemcpyHostToDevice) != cudaSuccess ||
                       cudaMemcpy(db, B, sizeof(double) * N * K, cudaMemcpyHostToDevice) != cudaSuccess)) {
    set_error("gfcc_selftest_gemm_f64emu: copy failed");
    s = GFCC_ERR_CUDA;
  }
  EmuOperand ea, eb;
  if (s == GFCC_OK) s = umma_error_reset(st);
  if (s == GFCC_OK) s = emu_slice(st, static_cast<double *>(da), M, K, K, S, sa, ea);
  if (s == GFCC_OK) s = emu_slice(st, static_cast<double *>(db), N, K, K, S, sb, eb);
  if (s == GFCC_OK) s = emu_gemm(st, ea, eb, P, 1.0, 0.0, static_cast<double *>(dc), imap1(N), imap1(1), w);
  if (s == GFCC_OK) s = umma_error_check(st);
  if (s == GFCC_OK && cudaMemcpy(C, dc, sizeof(double) * M * N, cudaMemcpyDeviceToHost) != cudaSuccess) {
    set_error("gfcc_selftest_gemm_f64emu: copy back failed");
    s = GFCC_ERR_CUDA;
  }
  for (void *p : {da, db, dc, sa, sb, w}) dfree(p);
  if (st) cudaStreamDestroy(st);
  return s;
}

int gfcc_selftest_gemm_bf16(int M, int N, int K, const float *A, const float *B, float *D) {
  if (M <= 0 || N <= 0 || K <= 0 || A == nullptr || B == nullptr || D == nullptr) {
    set_error("gfcc_selftest_gemm_bf16: bad arguments");
    return GFCC_ERR_ARG;
  }
  const long long ld = (K + 7) / 8 * 8;
  std::vector<unsigned short> ha((size_t)M * ld, 0), hb((size_t)N * ld, 0);
  auto to_bf16 = [](float x) -> unsigned short {   // round to nearest even
    unsigned u;
    memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (unsigned short)(u >> 16);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (unsigned short)(u >> 16);
  };
  for (long long i = 0; i < M; i++)
    for (long long k = 0; k < K; k++) ha[i * ld + k] = to_bf16(A[i * K + k]);
  for (long long i = 0; i < N; i++)
    for (long long k = 0; k < K; k++) hb[i * ld + k] = to_bf16(B[i * K + k]);
  void *da = nullptr, *db = nullptr, *dd = nullptr;
  cudaStream_t st = nullptr;
  int s = GFCC_OK;
  if (dmalloc(&da, ha.size() * 2) != cudaSuccess || dmalloc(&db, hb.size() * 2) != cudaSuccess ||
      dmalloc(&dd, (size_t)M * N * 4) != cudaSuccess || cudaStreamCreate(&st) != cudaSuccess) {
    cudaGetLastError();
    set_error("gfcc_selftest_gemm_bf16: allocation failed");
    s = GFCC_ERR_OOM;
  }
  if (s == GFCC_OK && (cudaMemcpy(da, ha.data(), ha.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess ||
                       cudaMemcpy(db, hb.data(), hb.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess)) {
    set_error("gfcc_selftest_gemm_bf16: copy failed");
    s = GFCC_ERR_CUDA;
  }
  if (s == GFCC_OK) s = umma_error_reset(st);
  if (s == GFCC_OK)
    s = gemm_bf16_tn(st, static_cast<const __nv_bfloat16 *>(da), ld, static_cast<const __nv_bfloat16 *>(db), ld,
                     static_cast<float *>(dd), N, M, N, K, 1.0f, 0.0f);
  if (s == GFCC_OK) s = umma_error_check(st);
  if (s == GFCC_OK && cudaMemcpy(D, dd, (size_t)M * N * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
    set_error("gfcc_selftest_gemm_bf16: copy back failed");
    s = GFCC_ERR_CUDA;
  }
  dfree(da);
  dfree(db);
  dfree(dd);
  if (st) cudaStreamDestroy(st);
  return s;
}

}  // extern "C"
