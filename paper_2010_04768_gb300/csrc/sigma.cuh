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
  const double *omega = nullptr;   // device [nsys]
  double eta = 0.0;
  const double *diag = nullptr;    // device [dim] or nullptr
  double dsign = 1.0;              // +1 IP, -1 EA
  double zsign = -1.0;             // -1 IP, +1 EA (sign of i*eta in z_s)
};

long long sigma_work_doubles(const gfcc_ctx *c, int sector, int nsys);
int apply_ip(gfcc_ctx *c, const SysBatch &b, double *work);
int apply_ea(gfcc_ctx *c, const SysBatch &b, double *work);

}  // namespace gfcc
