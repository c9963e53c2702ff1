// Batched shifted operator of eq. xplin over packed complex vectors.
#pragma once
#include "ctx.cuh"

namespace gfcc {

// nsys packed complex vectors (interleaved re, im) in, nsys out.
//   x + 2*s*ldx (in), y + 2*s*ldy (out), s < nsys
// omega == nullptr: y = sigma(x) (no shift, no preconditioner).
// omega != nullptr: y = z_s u +/- sigma(u), u = x / D_s, with z_s = omega_s - i eta (IP) or
//   omega_s + i eta (EA) and D_s = z_s + d (IP) / z_s - d (EA) when diag != nullptr, else 1.
struct SysBatch {
  int nsys = 0;
  const double *x = nullptr;
  long long ldx = 0;
  double *y = nullptr;
  long long ldy = 0;
  const float *xf = nullptr;       // FP32 vectors instead of x / y (mixed-precision operator only)
  float *yf = nullptr;
  const double *omega = nullptr;   // device [nsys]
  double eta = 0.0;
  const double *diag = nullptr;    // device [dim] or nullptr
  double dsign = 1.0;              // +1 IP, -1 EA
  double zsign = -1.0;             // -1 IP, +1 EA (sign of i*eta in z_s)
  // optional (device, nsys entries): batch system s is vector idx[s] of x, y and omega; an entry
  // -1 - t reads vector t and stores nothing (padding of a subset to a convenient width)
  const int *idx = nullptr;
};

// vector of batch system s, and whether its result is stored
__device__ __forceinline__ int sysv(const SysBatch &b, int s) {
  if (b.idx == nullptr) return s;
  const int t = b.idx[s];
  return t >= 0 ? t : -1 - t;
}
__device__ __forceinline__ bool sys_stores(const SysBatch &b, int s) { return b.idx == nullptr || b.idx[s] >= 0; }

long long sigma_work_doubles(const gfcc_ctx *c, int sector, int nsys);
// algorithmic flops of one complex sigma product (two real vectors)
double sigma_flops(const gfcc_ctx *c, int sector);
long long sigma_mixed_work_doubles(const gfcc_ctx *c, int nsys);
// mixed precision (IP): BF16 tensor-core couplings + FP64 diagonal and shift (sigma_mixed.cu)
int apply_ip_mixed(gfcc_ctx *c, const SysBatch &b, double *work);
int apply_ip(gfcc_ctx *c, const SysBatch &b, double *work);
// closed-shell spin-adapted IP operator (rhf.cu; apply_ip dispatches to it for such contexts)
int apply_ip_rhf(gfcc_ctx *c, const SysBatch &b, double *work);
long long rhf_work_doubles(const gfcc_ctx *c, int nsys);
double rhf_sigma_flops(const gfcc_ctx *c);
// the FP64 epilogue of the IP operator on given S1 / T / Q / U (FP64, layouts of sigma.cu); with diag
// (the packed Fock-like diagonal) the outputs hold the couplings only and the diagonal is applied here
int launch_epilogue_ip(gfcc_ctx *c, const SysBatch &b, const double *S1, const double *T, const double *Q,
                       const double *U, const double *diag = nullptr);
// FP64-accurate IP operator from digit planes on the BF16 tensor cores (sigma_emu.cu); processes
// the systems in sub-batches that fit its workspace.  The solvers size that workspace for up to
// EMU_SUB_MAX systems: each sub-batch re-reads the operator's digit planes, so fewer and wider
// sub-batches cost less (about 0.3 GB per system at o=40 v=200 EA, 0.9 GB at o=90 v=450 IP)
constexpr int EMU_SUB_MAX = 64;
long long sigma_emu_work_doubles(const gfcc_ctx *c, int nsub);
// level > 0: digit pairs i + j <= min(level, the context's level) only (products of small corrections)
int apply_ip_emu(gfcc_ctx *c, const SysBatch &b, double *work, long long work_doubles, int level = 0);
int apply_ea(gfcc_ctx *c, const SysBatch &b, double *work);
// mixed precision (EA): BF16 tensor-core couplings + FP64 diagonal and shift (sigma_mixed.cu)
int apply_ea_mixed(gfcc_ctx *c, const SysBatch &b, double *work);
// FP64-accurate EA operator from digit planes (sigma_emu.cu)
int apply_ea_emu(gfcc_ctx *c, const SysBatch &b, double *work, long long work_doubles, int level = 0);
// the FP64 epilogue of the EA operator on given S1 / T / Qp / U (FP64, layouts of sigma.cu); diag as
// launch_epilogue_ip
int launch_epilogue_ea(gfcc_ctx *c, const SysBatch &b, const double *S1, const double *T, const double *Qp,
                       const double *U, const double *diag = nullptr);

}  // namespace gfcc
