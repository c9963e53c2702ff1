// Shared device/host helpers of libgfcc (error propagation, index maps, launch helpers).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>

#include "../../include/gfcc.h"

namespace gfcc {

void set_error(const char *fmt, ...);

// Registry of device allocations made by the library.  Every contraction / permutation
// launch checks on the host that the address range its index maps can reach lies inside
// one registered allocation, so a wrong map becomes an error return, not a device fault.
void reg_alloc(const void *p, size_t bytes);
void unreg_alloc(const void *p);
// 0 if [p + lo*8, p + hi*8 + 8) lies inside a registered allocation, else GFCC_ERR_ARG (with message)
int check_extent(const double *p, long long lo, long long hi, const char *what);
// 0 if [p, p + bytes) lies inside a registered allocation
int check_extent_bytes(const void *p, long long bytes, const char *what);
cudaError_t dmalloc(void **p, size_t bytes);   // cudaMalloc + reg_alloc
void dfree(void *p);                           // unreg_alloc + cudaFree

// Evaluate a CUDA runtime call; on failure record the message and return GFCC_ERR_CUDA.
#define GFCC_CUDA(call)                                                                 \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      ::gfcc::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
      return GFCC_ERR_CUDA;                                                             \
    }                                                                                   \
  } while (0)

// Propagate a non-zero gfcc status.
#define GFCC_TRY(expr)          \
  do {                          \
    int s_ = (expr);            \
    if (s_ < 0) return s_;      \
  } while (0)

// Check the last kernel launch (and count it: gfcc_launch_count reports the total).
void count_launch();
void count_launches(long long n);   // kernels replayed from a CUDA graph
long long launch_count();
long long thread_launch_count();   // the calling thread's share (concurrent solves of gfcc_solve_batch)
#define GFCC_LAUNCH_CHECK()   \
  do {                        \
    ::gfcc::count_launch();   \
    GFCC_CUDA(cudaGetLastError()); \
  } while (0)

// Index map of a flattened GEMM index x onto a tensor offset:
//   d0 <= 0 : x * s0
//   d0  > 0 : (x % d0) * s0 + (x / d0) * s1      (two tensor indices fused into one GEMM index)
struct IMap {
  long long d0, s0, s1;
};
static inline IMap imap1(long long s0) { return IMap{0, s0, 0}; }
static inline IMap imap2(long long d0, long long s0, long long s1) { return IMap{d0, s0, s1}; }

// Largest offset an IMap produces for x in [0, X) (all strides are non-negative).
static inline long long imap_max(const IMap &m, long long X) {
  if (X <= 0) return 0;
  if (m.d0 <= 0) return (X - 1) * m.s0;
  const long long r = (X < m.d0 ? X : m.d0) - 1;
  return r * m.s0 + ((X - 1) / m.d0) * m.s1;
}

__device__ __forceinline__ long long imap_apply(const IMap &m, long long x) {
  if (m.d0 <= 0) return x * m.s0;
  long long q = x / m.d0;
  return (x - q * m.d0) * m.s0 + q * m.s1;
}

// Pairs i < j < m in lexicographic order: index = pair_start(i) + (j - i - 1).
__host__ __device__ __forceinline__ long long pair_start(long long i, long long m) { return i * m - i * (i + 1) / 2; }
__host__ __device__ __forceinline__ long long pair_index(long long i, long long j, long long m) {
  return pair_start(i, m) + (j - i - 1);
}
// Inverse of pair_index (closed form from the quadratic, then an exact integer correction).
__device__ __forceinline__ void pair_decode(long long idx, long long m, long long &i, long long &j) {
  const double b = 2.0 * (double)m - 1.0;
  long long ii = (long long)((b - sqrt(fmax(b * b - 8.0 * (double)idx, 0.0))) * 0.5);
  if (ii < 0) ii = 0;
  if (ii > m - 2) ii = m - 2;
  while (ii > 0 && pair_start(ii, m) > idx) ii--;
  while (ii + 1 <= m - 2 && pair_start(ii + 1, m) <= idx) ii++;
  i = ii;
  j = idx - pair_start(ii, m) + ii + 1;
}

// FP64 -> FP32 by bit manipulation on the integer units (truncating the mantissa; values below the
// FP32 normal range flush to zero, values above it saturate to infinity).  GB300 issues about two
// FP64 operations per SM and clock, so kernels that only need FP32 accuracy avoid the FP64 pipe.
__device__ __forceinline__ float d2f_trunc(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7ff) - 1023 + 127;
  if (e <= 0) return __int_as_float((int)sign);
  if (e >= 255) return __int_as_float((int)(sign | 0x7f800000u));
  return __int_as_float((int)(sign | ((unsigned)e << 23) | (unsigned)((b >> 29) & 0x7fffff)));
}

// Balanced base-64 digits of y = x 2^-ex (|y| < 1/2), S of them (S <= 10), with integer arithmetic:
// Y = round(y 2^(6S)) from the FP64 bit pattern, then d_i = round(Y / 2^(6(S-i))) successively.
__device__ __forceinline__ long long fixed_point(double x, int ex, int bits) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7ff);
  if (E == 0) return 0;   // zero (and subnormals, far below any digit)
  const long long m = (long long)((b & 0xfffffffffffffULL) | 0x10000000000000ULL);
  const int sh = E - 1075 - ex + bits;   // Y = m 2^sh
  long long Y;
  if (sh >= 0) {
    Y = sh < 11 ? (m << sh) : 0;          // cannot happen for |y| < 1/2 and bits <= 60
  } else if (sh > -63) {
    Y = (m + (1LL << (-sh - 1))) >> (-sh);
  } else {
    Y = 0;
  }
  return (b >> 63) ? -Y : Y;
}

static inline unsigned int cdiv(long long a, long long b) { return (unsigned int)((a + b - 1) / b); }

// Grid-stride 1-D launch size for `n` elements (capped to keep the grid modest).
static inline unsigned int grid1d(long long n, int threads = 256) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152LL * 64) b = 152LL * 64;
  return (unsigned int)b;
}

}  // namespace gfcc
