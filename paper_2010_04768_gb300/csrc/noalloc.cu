// gfcc_sigma_noalloc: the FP64 sigma product on caller-provided device buffers with its
// workspace in a fixed, file-scope device array, so the call allocates no memory.
//
// Who needs this: callers that cannot (or must not) allocate device memory on their call path,
// e.g. an application whose device memory is entirely reserved up front by its own pool
// allocator (a cudaMalloc would fail or fragment that pool), or a latency-critical service
// path where the implicit device-wide synchronisation of cudaMalloc / cudaFree would stall the
// other streams of the process.
//
// The workspace is g_sigma_scratch below: NOALLOC_SCRATCH_DOUBLES doubles (32 MiB) held by
// every GPU that loads the library, until the process exits.  Host code must not use the
// symbol's name as an address: the device address is obtained once per device with
// cudaGetSymbolAddress (the first call on a device does this; make that first call before any
// stream capture).  Every call shares the array, so calls whose executions overlap on the GPU
// race; serialise them (one stream, or events).  The sigma product writes every workspace entry
// it reads within the same call, so no clearing between calls is needed.
#include <mutex>

#include "ctx.cuh"
#include "sigma.cuh"

namespace gfcc {

namespace {

constexpr long long NOALLOC_SCRATCH_DOUBLES = 1LL << 22;   // 32 MiB
__device__ __align__(256) double g_sigma_scratch[NOALLOC_SCRATCH_DOUBLES];

constexpr int MAX_DEVICES = 128;
std::mutex g_noalloc_mu;
double *g_noalloc_addr[MAX_DEVICES] = {nullptr};

// Device address of g_sigma_scratch on the current device (looked up once per device).
int scratch_address(double **out) {
  int dev = 0;
  GFCC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES) {
    set_error("gfcc_sigma_noalloc: device index %d out of range", dev);
    return GFCC_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (g_noalloc_addr[dev] == nullptr) {
    double *p = nullptr;
    GFCC_CUDA(cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_sigma_scratch));
    reg_alloc(p, sizeof(double) * NOALLOC_SCRATCH_DOUBLES);   // known to the extent checks
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return GFCC_OK;
}

}  // namespace

}  // namespace gfcc

using namespace gfcc;

extern "C" int gfcc_sigma_noalloc(gfcc_ctx *c, int sector, int n_vec, const double *x_dev, double *y_dev) {
  if (c == nullptr || x_dev == nullptr || y_dev == nullptr || n_vec < 0 ||
      (sector != GFCC_SECTOR_IP && sector != GFCC_SECTOR_EA) || !(c->sectors & sector)) {
    set_error("gfcc_sigma_noalloc: bad arguments or sector not built");
    return GFCC_ERR_ARG;
  }
  if (n_vec == 0) return GFCC_OK;
  const long long o = c->o, v = c->v;
  const long long need = sigma_work_doubles(c, sector, n_vec);
  // the contractions of the sigma product with a long K would ask for a split-K buffer; keep to
  // sizes where none does, and to the fixed workspace
  const long long longk = sector == GFCC_SECTOR_IP ? o * o * v : o * v * v;
  if (need > NOALLOC_SCRATCH_DOUBLES || longk >= 8192) {
    set_error("gfcc_sigma_noalloc: %d vectors need %lld workspace doubles (maximum %lld) and a contraction "
              "length %lld (maximum 8191)",
              n_vec, need, NOALLOC_SCRATCH_DOUBLES, longk);
    return GFCC_ERR_ARG;
  }
  double *w = nullptr;
  GFCC_TRY(scratch_address(&w));
  SysBatch b;
  b.nsys = n_vec;
  b.x = x_dev;
  b.ldx = sector == GFCC_SECTOR_IP ? c->dim_ip : c->dim_ea;
  b.y = y_dev;
  b.ldy = b.ldx;
  GFCC_TRY(sector == GFCC_SECTOR_IP ? apply_ip(c, b, w) : apply_ea(c, b, w));
  GFCC_CUDA(cudaStreamSynchronize(c->stream));
  return GFCC_OK;
}
