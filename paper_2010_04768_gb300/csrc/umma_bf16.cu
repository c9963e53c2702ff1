// BF16 x BF16 -> FP32 GEMM on the 5th-generation tensor cores (tcgen05, sm_103a).
//
//   D[m][n] = alpha * sum_k A[m][k] B[n][k] (+ beta * D[m][n])     (both operands K-major)
//
// This is the contraction engine of the mixed-precision sigma product: the ring
// matrix Wbar_ovvo (and the other Hbar blocks) are stored once in BF16, the Krylov
// vectors are rounded to BF16 when they are unpacked, products accumulate in FP32
// in tensor memory (TMEM).
//
// Structure (one 128 x 256 output tile per CTA, 4 warps):
//   * warp 0, one lane: TMA producer.  A tile 128 x 64 and B tile 256 x 64 (BF16,
//     128-byte swizzle) per stage into a 4-stage shared-memory ring, completion
//     tracked by mbarrier transaction counts.
//   * warp 1, one lane: MMA issuer.  Four tcgen05.mma (M=128, N=256, K=16) per stage,
//     accumulating in 256 TMEM columns; tcgen05.commit releases the stage.
//   * all 4 warps: epilogue.  tcgen05.ld of the warp's 32 TMEM lanes, scale, store.
// Every wait is bounded (about one second of %globaltimer); on time-out the CTA sets
// the error flag, stops issuing work, drains what it issued and frees its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"
#include "umma.cuh"

namespace gfcc {

namespace {

constexpr int BM = 128, BK = 64, THREADS = 128;
constexpr int RASTER_GM = 16;   // row tiles per rasterisation group
// BN (the N extent of a tile and of the TMEM accumulator) is a template parameter: 256 for wide
// operands, 128 / 64 when the contraction has few columns (a tile wider than N wastes MMA work).
// ST: pipeline stages (0: the default for BN).  Contractions with only a K block or two per CTA use
// 2 stages, so that several CTAs fit an SM and the per-CTA set-up overlaps.
template <int BN, int ST = 0>
struct Tile {
  static constexpr int STAGES = ST > 0 ? ST : (BN == 256 ? 4 : 6);
  static constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2, STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /* alignment */ + 256 /* barriers */;
};
// Bounded waits.  The limit of the pipeline waits is a launch parameter (default 1 s, settable
// process-wide so that a test can make a wait run out); the waits of the abort path, for work
// this CTA has already issued, always keep the fixed DRAIN_NS.
constexpr unsigned long long DRAIN_NS = 1000000000ULL;
// Launch-time control of the pipeline: wait limit, and (test only) a producer that issues no
// loads, so that the consumer's wait runs out with no asynchronous copy outstanding.
struct UmmaCtl {
  unsigned long long wait_ns;
  int skip_loads;
};
unsigned long long g_wait_ns = 1000000000ULL;
bool g_skip_loads = false;
UmmaCtl umma_ctl() { return UmmaCtl{g_wait_ns, g_skip_loads ? 1 : 0}; }

__device__ unsigned int g_umma_error = 0;

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(unsigned addr, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(unsigned addr, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(addr), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned addr, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait (limit_ns of %globaltimer) for the phase of the given parity; false on time-out or
// abort.
__device__ __forceinline__ bool mbar_wait(unsigned addr, unsigned parity, volatile int *abort_flag,
                                          unsigned long long limit_ns) {
  if (mbar_try_wait(addr, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (true) {
    if (mbar_try_wait(addr, parity)) return true;
    if (*abort_flag) return false;
    if (globaltimer() - t0 > limit_ns) {
      *abort_flag = 1;
      atomicOr(&g_umma_error, 1u);
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap *map, unsigned mbar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(mbar), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr) {
  unsigned long long d = 0;
  d |= (unsigned long long)((addr & 0x3FFFF) >> 4);       // start address
  d |= (unsigned long long)(16 >> 4) << 16;               // leading byte offset (unused for swizzled K-major)
  d |= (unsigned long long)(1024 >> 4) << 32;             // stride byte offset
  d |= 1ULL << 46;                                        // descriptor version
  d |= 2ULL << 61;                                        // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16: BF16 A and B, FP32 accumulator, K-major A and B, M x N.
__host__ __device__ constexpr unsigned idesc_bf16(int M, int N) {
  return (1u << 4)                      // D format: F32
         | (1u << 7)                    // A format: BF16
         | (1u << 10)                   // B format: BF16
         | ((unsigned)(N >> 3) << 17)   // N / 8
         | ((unsigned)(M >> 4) << 24);  // M / 16
}

__device__ __forceinline__ void umma_bf16(unsigned d_tmem, unsigned long long a, unsigned long long b, unsigned idesc,
                                          unsigned accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(unsigned mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void tmem_ld_32(unsigned taddr, float (&v)[32]) {
  unsigned r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

template <int BN, int ST>
__global__ void __launch_bounds__(THREADS, 1)
    umma_bf16_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, float *D,
                          long long ldd, int M, int N, int K, float alpha, float beta, int kb_per_split,
                          long long split_stride, UmmaCtl ctl) {
  constexpr int STAGES = Tile<BN, ST>::STAGES, A_BYTES = Tile<BN, ST>::A_BYTES,
                STAGE_BYTES = Tile<BN, ST>::STAGE_BYTES;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem + STAGES * STAGE_BYTES);
  unsigned long long *full = bars, *empty = bars + STAGES, *done = bars + 2 * STAGES;
  unsigned *tmem_slot = reinterpret_cast<unsigned *>(bars + 2 * STAGES + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  volatile int *issued = reinterpret_cast<volatile int *>(tmem_slot + 2);     // TMA stages issued
  volatile int *consumed = reinterpret_cast<volatile int *>(tmem_slot + 3);   // stages the MMA warp waited for

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // tile order: groups of RASTER_GM row tiles sweep all column tiles, row tile fastest, so the CTAs
  // in flight share a few A row panels and B column panels (L2 reuse on long-K products)
  int m_tile, n_tile;
  {
    const int nM = gridDim.x, nN = gridDim.y;
    const int id = blockIdx.y * nM + blockIdx.x;
    const int first_m = (id / (RASTER_GM * nN)) * RASTER_GM;
    const int gm = min(nM - first_m, RASTER_GM);
    const int r = id - first_m * nN;
    m_tile = first_m + r % gm;
    n_tile = r / gm;
  }
  const int m0 = m_tile * BM, n0 = n_tile * BN;
  // split-K: this CTA covers K blocks [kb0, kb1) and writes its partial sum to D + z * split_stride
  const int nk_all = (K + BK - 1) / BK;
  const int kb0 = blockIdx.z * kb_per_split;
  const int kb1 = min(nk_all, kb0 + kb_per_split);
  const int nk = kb1 - kb0;
  D += (long long)blockIdx.z * split_stride;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; s++) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(done), 1);
    *abort_flag = 0;
    *issued = 0;
    *consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {   // TMEM: 256 FP32 columns x 128 lanes for the accumulator
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    for (int kb = 0; kb < nk && !ctl.skip_loads; kb++) {
      const int s = kb % STAGES;
      const unsigned ph = (kb / STAGES) & 1;
      if (!mbar_wait(smem_u32(&empty[s]), ph ^ 1, abort_flag, ctl.wait_ns)) break;
      unsigned char *sa = smem + s * STAGE_BYTES;
      unsigned char *sb = sa + A_BYTES;
      mbar_expect_tx(smem_u32(&full[s]), STAGE_BYTES);
      tma_load_2d(smem_u32(sa), &tmA, smem_u32(&full[s]), (kb0 + kb) * BK, m0);
      tma_load_2d(smem_u32(sb), &tmB, smem_u32(&full[s]), (kb0 + kb) * BK, n0);
      *issued = kb + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    const unsigned idesc = idesc_bf16(BM, BN);
    bool ok = true;
    for (int kb = 0; kb < nk && ok; kb++) {
      const int s = kb % STAGES;
      const unsigned ph = (kb / STAGES) & 1;
      if (!mbar_wait(smem_u32(&full[s]), ph, abort_flag, ctl.wait_ns)) {
        ok = false;
        break;
      }
      *consumed = kb + 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned sa = smem_u32(smem + s * STAGE_BYTES);
      const unsigned sb = sa + A_BYTES;
#pragma unroll
      for (int k = 0; k < BK / 16; k++) {
        // advance 16 BF16 (32 bytes) along K inside the 128-byte swizzle atom
        umma_bf16(tmem, smem_desc(sa + 32 * k), smem_desc(sb + 32 * k), idesc, (kb > 0 || k > 0) ? 1u : 0u);
      }
      umma_commit(smem_u32(&empty[s]));
    }
    umma_commit(smem_u32(done));   // arrives when every MMA issued above has completed
  }
  __syncwarp();

  // ---------------- epilogue: all 4 warps
  const bool ready = mbar_wait(smem_u32(done), 0, abort_flag, ctl.wait_ns);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // tcgen05.ld is warp-collective: take the decision per warp
  if (__all_sync(0xffffffffu, ready && !*abort_flag)) {
    const int row = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
      float v[32];
      tmem_ld_32(tmem + ((unsigned)(warp * 32) << 16) + c0, v);
      if (row < M) {
        float *dst = D + (long long)row * ldd + n0 + c0;
        const int ncols = min(32, N - (n0 + c0));
        if (ncols == 32 && beta == 0.0f && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
#pragma unroll
          for (int i = 0; i < 32; i += 4)
            *reinterpret_cast<float4 *>(dst + i) = make_float4(alpha * v[i], alpha * v[i + 1], alpha * v[i + 2],
                                                               alpha * v[i + 3]);
        } else if (ncols == 32 && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
#pragma unroll
          for (int i = 0; i < 32; i += 4) {
            const float4 d = *reinterpret_cast<const float4 *>(dst + i);
            *reinterpret_cast<float4 *>(dst + i) =
                make_float4(alpha * v[i] + beta * d.x, alpha * v[i + 1] + beta * d.y, alpha * v[i + 2] + beta * d.z,
                            alpha * v[i + 3] + beta * d.w);
          }
        } else {
          for (int i = 0; i < ncols; i++) dst[i] = alpha * v[i] + (beta != 0.0f ? beta * dst[i] : 0.0f);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) {
    // after a time-out: the MMA warp always commits `done` once its issued products have completed
    // (wait for it, so that no tcgen05.mma still reads shared memory or writes TMEM when the TMEM is
    // freed), then let the TMA copies this CTA issued land before its shared memory goes away.
    // These waits keep the fixed DRAIN_NS limit; if one of them runs out as well, the CTA exits with
    // that work in flight (the error flag is already set).
    volatile int never = 0;
    mbar_wait(smem_u32(done), 0, &never, DRAIN_NS);
    for (int kb = *consumed; kb < *issued; kb++)
      mbar_wait(smem_u32(&full[kb % STAGES]), (kb / STAGES) & 1, &never, DRAIN_NS);
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
  }
}

// ---------------------------------------------------------------------------------------------
// The same product with a persistent tile loop: one CTA per SM walks the output tiles (and K splits)
// of the launch; six warps: warp 0 the TMA producer, warp 1 the MMA issuer, warps 2-5 the epilogue
// (warp w reads TMEM lanes 32 (w mod 4) .. + 31).  Two accumulators of BN columns in TMEM (ping-pong):
// the epilogue of a tile overlaps the main loop of the next, and the load pipeline runs on across
// tiles, so products with few K blocks per tile (the long thin contractions of the sigma product)
// no longer pay a pipeline fill, a TMEM allocation and an unoverlapped epilogue per tile.
constexpr int PERSIST_THREADS = 192;
template <int BN>
struct PTile {
  static constexpr int STAGES = BN == 256 ? 4 : 6;
  static constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2, STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 512;
};

template <int BN>
__global__ void __launch_bounds__(PERSIST_THREADS, 1)
    umma_persist_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                             float *D, long long ldd, int M, int N, int K, float alpha, float beta, int kb_per_split,
                             long long split_stride, int nM, int nN, int nsplit, UmmaCtl ctl) {
  constexpr int STAGES = PTile<BN>::STAGES, A_BYTES = PTile<BN>::A_BYTES, STAGE_BYTES = PTile<BN>::STAGE_BYTES;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem + STAGES * STAGE_BYTES);
  unsigned long long *full = bars, *empty = bars + STAGES;
  unsigned long long *accf = bars + 2 * STAGES, *acce = accf + 2, *drain = acce + 2;
  unsigned *tmem_slot = reinterpret_cast<unsigned *>(drain + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  volatile int *issued = reinterpret_cast<volatile int *>(tmem_slot + 2);
  volatile int *consumed = reinterpret_cast<volatile int *>(tmem_slot + 3);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk_all = (K + BK - 1) / BK;
  const int tiles = nM * nN * nsplit;
  // tile t: split z = t / (nM nN); within a split, groups of RASTER_GM row tiles sweep the column tiles
  auto tile_of = [&](int t, int &m0, int &n0, int &kb0, int &nk, long long &zoff) {
    const int z = t / (nM * nN), id = t - z * (nM * nN);
    const int first_m = (id / (RASTER_GM * nN)) * RASTER_GM;
    const int gm = min(nM - first_m, RASTER_GM);
    const int r = id - first_m * nN;
    m0 = (first_m + r % gm) * BM;
    n0 = (r / gm) * BN;
    kb0 = z * kb_per_split;
    nk = min(nk_all, kb0 + kb_per_split) - kb0;
    zoff = (long long)z * split_stride;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; s++) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < 2; b++) {
      mbar_init(smem_u32(&accf[b]), 1);
      mbar_init(smem_u32(&acce[b]), 4);   // one arrive per epilogue warp
    }
    mbar_init(smem_u32(drain), 1);
    *abort_flag = 0;
    *issued = 0;
    *consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {   // TMEM: two accumulators of BN FP32 columns x 128 lanes
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0 && !ctl.skip_loads) {
      // ---------------- TMA producer: K blocks of the CTA's tiles, one continuous pipeline
      int it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
        int m0, n0, kb0, nk;
        long long zoff;
        tile_of(t, m0, n0, kb0, nk, zoff);
        for (int kb = 0; kb < nk; kb++, it++) {
          const int s = it % STAGES;
          const unsigned ph = (it / STAGES) & 1;
          if (!mbar_wait(smem_u32(&empty[s]), ph ^ 1, abort_flag, ctl.wait_ns)) {
            ok = false;
            break;
          }
          unsigned char *sa = smem + s * STAGE_BYTES;
          mbar_expect_tx(smem_u32(&full[s]), STAGE_BYTES);
          tma_load_2d(smem_u32(sa), &tmA, smem_u32(&full[s]), (kb0 + kb) * BK, m0);
          tma_load_2d(smem_u32(sa + A_BYTES), &tmB, smem_u32(&full[s]), (kb0 + kb) * BK, n0);
          *issued = it + 1;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer: accumulator lt & 1 of the CTA's lt-th tile
      const unsigned idesc = idesc_bf16(BM, BN);
      int it = 0, lt = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x, lt++) {
        int m0, n0, kb0, nk;
        long long zoff;
        tile_of(t, m0, n0, kb0, nk, zoff);
        const int buf = lt & 1;
        if (!mbar_wait(smem_u32(&acce[buf]), ((lt >> 1) & 1) ^ 1, abort_flag, ctl.wait_ns)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const unsigned acc = tmem + (unsigned)(buf * BN);
        for (int kb = 0; kb < nk; kb++, it++) {
          const int s = it % STAGES;
          const unsigned ph = (it / STAGES) & 1;
          if (!mbar_wait(smem_u32(&full[s]), ph, abort_flag, ctl.wait_ns)) {
            ok = false;
            break;
          }
          *consumed = it + 1;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const unsigned sa = smem_u32(smem + s * STAGE_BYTES);
          const unsigned sb = sa + A_BYTES;
#pragma unroll
          for (int k = 0; k < BK / 16; k++)
            umma_bf16(acc, smem_desc(sa + 32 * k), smem_desc(sb + 32 * k), idesc, (kb > 0 || k > 0) ? 1u : 0u);
          umma_commit(smem_u32(&empty[s]));
        }
        if (ok) umma_commit(smem_u32(&accf[buf]));
      }
      umma_commit(smem_u32(drain));   // arrives once every MMA issued above has completed
    }
  } else {
    // ---------------- epilogue warps 2..5: rows 32 (warp mod 4) + lane of each tile
    const int q = warp & 3;
    int lt = 0;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x, lt++) {
      int m0, n0, kb0, nk;
      long long zoff;
      tile_of(t, m0, n0, kb0, nk, zoff);
      const int buf = lt & 1;
      const bool ready = mbar_wait(smem_u32(&accf[buf]), (lt >> 1) & 1, abort_flag, ctl.wait_ns);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (!__all_sync(0xffffffffu, ready && !*abort_flag)) break;
      const int row = m0 + q * 32 + lane;
      float *Dz = D + zoff;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        float v[32];
        tmem_ld_32(tmem + ((unsigned)(q * 32) << 16) + (unsigned)(buf * BN + c0), v);
        if (row < M && n0 + c0 < N) {
          float *dst = Dz + (long long)row * ldd + n0 + c0;
          const int ncols = min(32, N - (n0 + c0));
          if (ncols == 32 && beta == 0.0f && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
#pragma unroll
            for (int i = 0; i < 32; i += 4)
              *reinterpret_cast<float4 *>(dst + i) = make_float4(alpha * v[i], alpha * v[i + 1], alpha * v[i + 2],
                                                                 alpha * v[i + 3]);
          } else if (ncols == 32 && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
#pragma unroll
            for (int i = 0; i < 32; i += 4) {
              const float4 d = *reinterpret_cast<const float4 *>(dst + i);
              *reinterpret_cast<float4 *>(dst + i) =
                  make_float4(alpha * v[i] + beta * d.x, alpha * v[i + 1] + beta * d.y, alpha * v[i + 2] + beta * d.z,
                              alpha * v[i + 3] + beta * d.w);
            }
          } else {
            for (int i = 0; i < ncols; i++) dst[i] = alpha * v[i] + (beta != 0.0f ? beta * dst[i] : 0.0f);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce[buf])) : "memory");
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    // every MMA the issuer committed has completed (the drain barrier); after a time-out also the TMA
    // copies issued but not consumed land before the shared memory goes away (fixed DRAIN_NS limits)
    volatile int never = 0;
    mbar_wait(smem_u32(drain), 0, &never, DRAIN_NS);
    if (*abort_flag)
      for (int it = *consumed; it < *issued; it++)
        mbar_wait(smem_u32(&full[it % STAGES]), (it / STAGES) & 1, &never, DRAIN_NS);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN));
  }
}

// ---------------------------------------------------------------------------------------------
// The same product on CTA pairs (tcgen05 cta_group::2): a cluster of two CTAs on two SMs computes a
// 256 x 256 output tile with M = 256 MMAs.  Each CTA stages its own 128 rows of A and one half (128
// columns) of the B tile, so per SM the shared memory holds and the tensor core reads half of the B
// tile of the one-CTA kernel: with a 128 x 256 tile per SM the operand traffic through shared
// memory (TMA writes plus MMA reads, about 1.5x the shared-memory bandwidth at the full MMA rate in
// the one-CTA kernel) drops to about the bandwidth.  The leader CTA (cluster rank 0) issues the MMAs
// for the pair; both CTAs' loads complete on the leader's barriers; the MMA commits arrive on the
// barriers of both CTAs (multicast); each CTA's TMEM holds its own 128 rows of the accumulator and
// each CTA writes them.  Same bounded waits and abort path as the one-CTA kernel; the pair meets at a
// cluster barrier before either frees its TMEM and exits.
constexpr int PAIR_BN = 256, PAIR_HALF = 128, PAIR_STAGES = 6;
constexpr int PAIR_A_BYTES = BM * BK * 2, PAIR_B_BYTES = PAIR_HALF * BK * 2;
constexpr int PAIR_STAGE_BYTES = PAIR_A_BYTES + PAIR_B_BYTES;
constexpr int PAIR_SMEM_BYTES = PAIR_STAGES * PAIR_STAGE_BYTES + 1024 + 256;

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// shared::cluster address of a shared::cta address in CTA `rank` of the cluster
__device__ __forceinline__ unsigned map_to_rank(unsigned addr, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}

// TMA tile load into this CTA's shared memory, completion on an mbarrier of either CTA of the pair
__device__ __forceinline__ void tma_load_2d_pair(unsigned dst, const CUtensorMap *map, unsigned mbar_cluster, int x,
                                                 int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
      "%4}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(mbar_cluster), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void umma_bf16_pair(unsigned d_tmem, unsigned long long a, unsigned long long b,
                                               unsigned idesc, unsigned accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

// arrive (once all earlier MMAs of this thread have completed) on the mbarrier at this shared
// offset in both CTAs of the pair
__device__ __forceinline__ void umma_commit_pair(unsigned mbar) {
  const unsigned short mask = 0x3;
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(mbar),
      "h"(mask)
      : "memory");
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(THREADS, 1)
    umma_pair_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, float *D,
                          long long ldd, int M, int N, int K, float alpha, float beta, int kb_per_split,
                          long long split_stride, UmmaCtl ctl) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem + PAIR_STAGES * PAIR_STAGE_BYTES);
  unsigned long long *full = bars, *empty = bars + PAIR_STAGES, *done = bars + 2 * PAIR_STAGES;
  unsigned *tmem_slot = reinterpret_cast<unsigned *>(bars + 2 * PAIR_STAGES + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  volatile int *issued = reinterpret_cast<volatile int *>(tmem_slot + 2);
  volatile int *consumed = reinterpret_cast<volatile int *>(tmem_slot + 3);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned rank = cluster_rank();
  const bool leader = rank == 0;
  // pair tile order as in the one-CTA kernel, over 256-row pair tiles
  int mp_tile, n_tile;
  {
    const int nM = gridDim.x / 2, nN = gridDim.y;
    const int id = blockIdx.y * nM + (int)(blockIdx.x / 2);
    const int first_m = (id / (RASTER_GM * nN)) * RASTER_GM;
    const int gm = min(nM - first_m, RASTER_GM);
    const int r = id - first_m * nN;
    mp_tile = first_m + r % gm;
    n_tile = r / gm;
  }
  const int m0 = mp_tile * (2 * BM) + (int)rank * BM;        // this CTA's rows
  const int n0 = n_tile * PAIR_BN;                            // the pair's columns
  const int nb0 = n0 + (int)rank * PAIR_HALF;                 // this CTA's half of the B tile
  const int nk_all = (K + BK - 1) / BK;
  const int kb0 = blockIdx.z * kb_per_split;
  const int kb1 = min(nk_all, kb0 + kb_per_split);
  const int nk = kb1 - kb0;
  D += (long long)blockIdx.z * split_stride;

  if (threadIdx.x == 0) {
    for (int s = 0; s < PAIR_STAGES; s++) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(done), 1);
    *abort_flag = 0;
    *issued = 0;
    *consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {   // TMEM of both CTAs: 256 FP32 columns x 128 lanes each (one warp per CTA)
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(PAIR_BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  cluster_sync_all();   // both CTAs' barriers initialised and TMEM allocated before any remote arrive
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer (both CTAs): loads complete on the leader's full barriers
    for (int kb = 0; kb < nk && !ctl.skip_loads; kb++) {
      const int s = kb % PAIR_STAGES;
      const unsigned ph = (kb / PAIR_STAGES) & 1;
      if (!mbar_wait(smem_u32(&empty[s]), ph ^ 1, abort_flag, ctl.wait_ns)) break;
      unsigned char *sa = smem + s * PAIR_STAGE_BYTES;
      unsigned char *sb = sa + PAIR_A_BYTES;
      if (leader) mbar_expect_tx(smem_u32(&full[s]), 2 * PAIR_STAGE_BYTES);
      const unsigned fb = map_to_rank(smem_u32(&full[s]), 0);
      tma_load_2d_pair(smem_u32(sa), &tmA, fb, (kb0 + kb) * BK, m0);
      tma_load_2d_pair(smem_u32(sb), &tmB, fb, (kb0 + kb) * BK, nb0);
      *issued = kb + 1;
    }
  } else if (warp == 1 && lane == 0 && leader) {
    // ---------------- MMA issuer (leader only): M = 256 over the pair, N = 256
    const unsigned idesc = idesc_bf16(2 * BM, PAIR_BN);
    bool ok = true;
    for (int kb = 0; kb < nk && ok; kb++) {
      const int s = kb % PAIR_STAGES;
      const unsigned ph = (kb / PAIR_STAGES) & 1;
      if (!mbar_wait(smem_u32(&full[s]), ph, abort_flag, ctl.wait_ns)) {
        ok = false;
        break;
      }
      *consumed = kb + 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned sa = smem_u32(smem + s * PAIR_STAGE_BYTES);
      const unsigned sb = sa + PAIR_A_BYTES;
#pragma unroll
      for (int k = 0; k < BK / 16; k++)
        umma_bf16_pair(tmem, smem_desc(sa + 32 * k), smem_desc(sb + 32 * k), idesc, (kb > 0 || k > 0) ? 1u : 0u);
      umma_commit_pair(smem_u32(&empty[s]));
    }
    umma_commit_pair(smem_u32(done));   // both CTAs: every MMA issued above has completed
  }
  __syncwarp();

  // ---------------- epilogue: all 4 warps of each CTA, its own 128 rows (skipped once any CTA of the
  // launch has given up, so that a pair whose leader aborted writes nothing)
  const bool ready = mbar_wait(smem_u32(done), 0, abort_flag, ctl.wait_ns);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool failed = *reinterpret_cast<volatile unsigned *>(&g_umma_error) != 0;
  if (__all_sync(0xffffffffu, ready && !*abort_flag && !failed) && nk > 0) {
    const int row = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < PAIR_BN; c0 += 32) {
      float v[32];
      tmem_ld_32(tmem + ((unsigned)(warp * 32) << 16) + c0, v);
      if (row < M && n0 + c0 < N) {
        float *dst = D + (long long)row * ldd + n0 + c0;
        const int ncols = min(32, N - (n0 + c0));
        if (ncols == 32 && beta == 0.0f && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
#pragma unroll
          for (int i = 0; i < 32; i += 4)
            *reinterpret_cast<float4 *>(dst + i) = make_float4(alpha * v[i], alpha * v[i + 1], alpha * v[i + 2],
                                                               alpha * v[i + 3]);
        } else if (ncols == 32 && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
#pragma unroll
          for (int i = 0; i < 32; i += 4) {
            const float4 d = *reinterpret_cast<const float4 *>(dst + i);
            *reinterpret_cast<float4 *>(dst + i) =
                make_float4(alpha * v[i] + beta * d.x, alpha * v[i + 1] + beta * d.y, alpha * v[i + 2] + beta * d.z,
                            alpha * v[i + 3] + beta * d.w);
          }
        } else {
          for (int i = 0; i < ncols; i++) dst[i] = alpha * v[i] + (beta != 0.0f ? beta * dst[i] : 0.0f);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0 && leader && *abort_flag) {
    // leader after a time-out: the committed MMAs (done), then the loads it waited for of both CTAs
    // (the pair's copies complete on the leader's barriers), each with the fixed DRAIN_NS limit
    volatile int never = 0;
    mbar_wait(smem_u32(done), 0, &never, DRAIN_NS);
    for (int kb = *consumed; kb < *issued; kb++)
      mbar_wait(smem_u32(&full[kb % PAIR_STAGES]), (kb / PAIR_STAGES) & 1, &never, DRAIN_NS);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  cluster_sync_all();   // neither CTA frees its TMEM or shared memory while the pair's work is in flight
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(PAIR_BN));
  }
}

// ---------------------------------------------------------------------------------------------
// FP64-accurate product from digit planes with every digit pair of a tile in one CTA:
//   C = alpha 2^(eA[m] + eB[n]) sum_L 2^(-6L) sum_{i+j=L, L<=P} A_i B_j^T + beta C.
// The accumulator of each level L = i + j lives in its own 64-column block of TMEM (8 levels fill
// the 512 columns).  A stage holds the tile of one A plane i and the tiles of the B planes
// j = 1 .. min(SB, P - i), so every level of pair (i, j) is fed from the same stage.  A level
// accumulates at most 8 pairs x 32 K blocks x 64 = 2^14 products of magnitude <= 2^10, so its FP32
// sums are exact integers; the epilogue adds the levels exactly in two int64 accumulators, forms
// the FP64 value and writes the FP64 result (or, with a K split, an FP64 partial per split).
constexpr int EMU_BN = 64, EMU_STAGES = 2, EMU_MAXS = 8;
constexpr int EMU_A_BYTES = BM * BK * 2, EMU_B_BYTES = EMU_BN * BK * 2;
constexpr int EMU_STAGE_BYTES = EMU_A_BYTES + EMU_MAXS * EMU_B_BYTES;
constexpr int EMU_SMEM_BYTES = EMU_STAGES * EMU_STAGE_BYTES + 1024 + 256;

struct EmuMaps {
  CUtensorMap a[EMU_MAXS];
  CUtensorMap b[EMU_MAXS];
};

__global__ void __launch_bounds__(THREADS, 1)
    umma_emu_kernel(const __grid_constant__ EmuMaps maps, int SA, int SB, int P, int M, int N, int K,
                    int kb_per_split, const int *eA, const int *eB, double alpha, double beta, double *C, IMap cm,
                    IMap cn, long long n0g, double *part, UmmaCtl ctl) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem + EMU_STAGES * EMU_STAGE_BYTES);
  unsigned long long *full = bars, *empty = bars + EMU_STAGES, *done = bars + 2 * EMU_STAGES;
  unsigned *tmem_slot = reinterpret_cast<unsigned *>(bars + 2 * EMU_STAGES + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  volatile int *issued = reinterpret_cast<volatile int *>(tmem_slot + 2);
  volatile int *consumed = reinterpret_cast<volatile int *>(tmem_slot + 3);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * EMU_BN;
  const int nk_all = (K + BK - 1) / BK;
  const int kb0 = blockIdx.z * kb_per_split;
  const int kb1 = min(nk_all, kb0 + kb_per_split);
  const int nk = kb1 - kb0;
  const int SAe = min(SA, P - 1);            // A planes with at least one partner
  const int iters = nk * SAe;                // stages: (K block, A plane)

  if (threadIdx.x == 0) {
    for (int s = 0; s < EMU_STAGES; s++) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(done), 1);
    *abort_flag = 0;
    *issued = 0;
    *consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {   // TMEM: 8 level accumulators of 64 FP32 columns x 128 lanes
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer: stage t = (K block t / SAe, A plane t % SAe + 1)
    for (int t = 0; t < iters && !ctl.skip_loads; t++) {
      const int s = t % EMU_STAGES;
      const unsigned ph = (t / EMU_STAGES) & 1;
      if (!mbar_wait(smem_u32(&empty[s]), ph ^ 1, abort_flag, ctl.wait_ns)) break;
      const int kb = kb0 + t / SAe, i = t % SAe + 1;
      const int nb = min(SB, P - i);
      unsigned char *sa = smem + s * EMU_STAGE_BYTES;
      mbar_expect_tx(smem_u32(&full[s]), EMU_A_BYTES + nb * EMU_B_BYTES);
      tma_load_2d(smem_u32(sa), &maps.a[i - 1], smem_u32(&full[s]), kb * BK, m0);
      for (int j = 1; j <= nb; j++)
        tma_load_2d(smem_u32(sa + EMU_A_BYTES + (j - 1) * EMU_B_BYTES), &maps.b[j - 1], smem_u32(&full[s]), kb * BK,
                    n0);
      *issued = t + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    const unsigned idesc = idesc_bf16(BM, EMU_BN);
    unsigned started = 0;   // bit L: level L has received its first product
    bool ok = true;
    for (int t = 0; t < iters && ok; t++) {
      const int s = t % EMU_STAGES;
      const unsigned ph = (t / EMU_STAGES) & 1;
      if (!mbar_wait(smem_u32(&full[s]), ph, abort_flag, ctl.wait_ns)) {
        ok = false;
        break;
      }
      *consumed = t + 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int i = t % SAe + 1;
      const int nb = min(SB, P - i);
      const unsigned sa = smem_u32(smem + s * EMU_STAGE_BYTES);
      for (int j = 1; j <= nb; j++) {
        const int L = i + j;
        const unsigned acc_col = tmem + (unsigned)((L - 2) * EMU_BN);
        const unsigned sb = sa + EMU_A_BYTES + (j - 1) * EMU_B_BYTES;
#pragma unroll
        for (int k = 0; k < BK / 16; k++) {
          const unsigned acc = ((started >> L) & 1u) || k > 0 ? 1u : 0u;
          umma_bf16(acc_col, smem_desc(sa + 32 * k), smem_desc(sb + 32 * k), idesc, acc);
        }
        started |= 1u << L;
      }
      umma_commit(smem_u32(&empty[s]));
    }
    umma_commit(smem_u32(done));
  }
  __syncwarp();

  // ---------------- epilogue: all 4 warps, one row per thread
  const bool ready = mbar_wait(smem_u32(done), 0, abort_flag, ctl.wait_ns);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (__all_sync(0xffffffffu, ready && !*abort_flag) && nk > 0) {
    const int row = m0 + warp * 32 + lane;
    const int ea = row < M ? eA[row] : 0;
    // The level sums are exact integers below 2^24: they are added in two int64 accumulators,
    // levels Lhi+1..P with weights 64^(P-L) and 2..Lhi with 64^(Lhi-L) (below 2^45 each), on the
    // integer pipes; FP64 work is two conversions and one scaled add per output.
    const int Lhi = min(P, 5);
#pragma unroll 1
    for (int c0 = 0; c0 < EMU_BN; c0 += 32) {
      double acc[32];
      long long ia[32];
#pragma unroll
      for (int q = 0; q < 32; q++) ia[q] = 0;
#pragma unroll 1
      for (int L = P; L > Lhi; L--) {
        const int ilo = max(1, L - SB), ihi = min(SAe, L - 1);   // a level holds products if some i + j = L
        if (ilo > ihi) continue;
        float v[32];
        tmem_ld_32(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)((L - 2) * EMU_BN + c0), v);
        const int sh = 6 * (P - L);
#pragma unroll
        for (int q = 0; q < 32; q++) ia[q] += (long long)__float2int_rn(v[q]) << sh;
      }
      const double wlo = ldexp(1.0, -6 * P), whi = ldexp(1.0, -6 * Lhi);
#pragma unroll
      for (int q = 0; q < 32; q++) {
        acc[q] = (double)ia[q] * wlo;
        ia[q] = 0;
      }
#pragma unroll 1
      for (int L = Lhi; L >= 2; L--) {
        const int ilo = max(1, L - SB), ihi = min(SAe, L - 1);
        if (ilo > ihi) continue;
        float v[32];
        tmem_ld_32(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)((L - 2) * EMU_BN + c0), v);
        const int sh = 6 * (Lhi - L);
#pragma unroll
        for (int q = 0; q < 32; q++) ia[q] += (long long)__float2int_rn(v[q]) << sh;
      }
#pragma unroll
      for (int q = 0; q < 32; q++) acc[q] = fma((double)ia[q], whi, acc[q]);
      if (row < M) {
        const int ncols = min(32, N - (n0 + c0));
        if (part != nullptr) {
          double *dst = part + ((long long)blockIdx.z * M + row) * N + n0 + c0;
#pragma unroll
          for (int q = 0; q < 32; q++)
            if (q < ncols) dst[q] = acc[q];
        } else {
          const long long ro = imap_apply(cm, row);
#pragma unroll
          for (int q = 0; q < 32; q++) {
            if (q >= ncols) continue;
            const int col = n0 + c0 + q;
            const long long off = ro + imap_apply(cn, n0g + col);
            const double val = alpha * ldexp(acc[q], ea + eB[col]);
            C[off] = beta != 0.0 ? val + beta * C[off] : val;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) {
    // as in umma_bf16_gemm_kernel: the committed products, then the issued copies (fixed limit)
    volatile int never = 0;
    mbar_wait(smem_u32(done), 0, &never, DRAIN_NS);
    for (int t = *consumed; t < *issued; t++)
      mbar_wait(smem_u32(&full[t % EMU_STAGES]), (t / EMU_STAGES) & 1, &never, DRAIN_NS);
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// C = alpha 2^(eA + eB) sum_z part[z] + beta C (the K splits of umma_emu_kernel)
__global__ void emu_split_reduce_kernel(const double *part, int nz, int M, int N, const int *eA, const int *eB,
                                        double alpha, double beta, double *C, IMap cm, IMap cn, long long n0g) {
  const long long tot = (long long)M * N;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(t / N), n = (int)(t - (long long)m * N);
    double s = 0.0;
    for (int z = 0; z < nz; z++) s += part[(long long)z * tot + t];
    const long long off = imap_apply(cm, m) + imap_apply(cn, n0g + n);
    const double val = alpha * ldexp(s, eA[m] + eB[n]);
    C[off] = beta != 0.0 ? val + beta * C[off] : val;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (fn == nullptr) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// 2-D K-major BF16 tensor map: rows x K (row stride ld elements), box 64 (K) x box_rows, 128-byte swizzle
int make_map(CUtensorMap *map, const void *base, long long rows, long long K, long long ld, int box_rows) {
  auto fn = encode_fn();
  if (fn == nullptr) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return GFCC_ERR_CUDA;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d) for rows=%lld K=%lld ld=%lld", (int)r, rows, K, ld);
    return GFCC_ERR_ARG;
  }
  return GFCC_OK;
}

}  // namespace

int umma_splits(int K, int nsplit) {
  const int nk = (K + BK - 1) / BK;
  if (nsplit < 1) nsplit = 1;
  if (nsplit > nk) nsplit = nk;
  const int kbs = (nk + nsplit - 1) / nsplit;
  return (nk + kbs - 1) / kbs;
}

int umma_error_reset(cudaStream_t st) {
  const unsigned zero = 0;
  GFCC_CUDA(cudaMemcpyToSymbolAsync(g_umma_error, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, st));
  return GFCC_OK;
}

int umma_error_check(cudaStream_t st) {
  unsigned h = 0;
  GFCC_CUDA(cudaMemcpyFromSymbolAsync(&h, g_umma_error, sizeof(h), 0, cudaMemcpyDeviceToHost, st));
  GFCC_CUDA(cudaStreamSynchronize(st));
  if (h != 0) {
    set_error("a tensor-core GEMM wait timed out on the device");
    return GFCC_ERR_TIMEOUT;
  }
  return GFCC_OK;
}

namespace {
// tile autotuner state: (device, M, N, K, split) -> tile width
bool g_autotune = true;
// 0: the autotuner also times the CTA-pair tile; 1: the pair tile whenever it applies; 2: never
int g_pair_mode = 0;
constexpr int TILE_PAIR = 512;   // autotuner key of the 256 x 256 CTA-pair tile
constexpr int TILE_PERSIST = 1024;   // autotuner key offset of the persistent kernel (+ its tile width)
// 0: the autotuner also times the persistent kernel; 1: always the persistent kernel; 2: never
int g_persist_mode = 0;
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, int> g_tune;

template <int BN, int ST>
int launch_umma_st(cudaStream_t st, const __nv_bfloat16 *A, long long lda, const __nv_bfloat16 *B, long long ldb,
                   float *D, long long ldd, int M, int N, int K, float alpha, float beta, int nsplit, int kbs,
                   long long split_stride) {
  CUtensorMap ma, mb;
  GFCC_TRY(make_map(&ma, A, M, K, lda, BM));
  GFCC_TRY(make_map(&mb, B, N, K, ldb, BN));
  static bool attr[64] = {false};
  int dev = 0;
  GFCC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64 || !attr[dev]) {
    GFCC_CUDA(cudaFuncSetAttribute(umma_bf16_gemm_kernel<BN, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   Tile<BN, ST>::SMEM_BYTES));
    if (dev >= 0 && dev < 64) attr[dev] = true;
  }
  if ((N + BN - 1) / BN > 65535 || nsplit > 65535) {
    set_error("gemm_bf16_tn: grid too large (N=%d, nsplit=%d)", N, nsplit);
    return GFCC_ERR_ARG;
  }
  dim3 grid((M + BM - 1) / BM, (N + BN - 1) / BN, nsplit);
  umma_bf16_gemm_kernel<BN, ST><<<grid, THREADS, Tile<BN, ST>::SMEM_BYTES, st>>>(ma, mb, D, ldd, M, N, K, alpha, beta, kbs,
                                                                         split_stride, umma_ctl());
  GFCC_LAUNCH_CHECK();
  return GFCC_OK;
}

template <int BN>
int launch_umma_persist(cudaStream_t st, const __nv_bfloat16 *A, long long lda, const __nv_bfloat16 *B, long long ldb,
                        float *D, long long ldd, int M, int N, int K, float alpha, float beta, int nsplit, int kbs,
                        long long split_stride) {
  CUtensorMap ma, mb;
  GFCC_TRY(make_map(&ma, A, M, K, lda, BM));
  GFCC_TRY(make_map(&mb, B, N, K, ldb, BN));
  static bool attr[64] = {false};
  static int nsm[64] = {0};
  int dev = 0;
  GFCC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64 || !attr[dev]) {
    GFCC_CUDA(cudaFuncSetAttribute(umma_persist_gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   PTile<BN>::SMEM_BYTES));
    int sms = 0;
    GFCC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (dev >= 0 && dev < 64) {
      attr[dev] = true;
      nsm[dev] = sms;
    }
  }
  const int sms = (dev >= 0 && dev < 64 && nsm[dev] > 0) ? nsm[dev] : 152;
  const long long nM = (M + BM - 1) / BM, nN = (N + BN - 1) / BN, tiles = nM * nN * nsplit;
  if (tiles > 0x7fffffffLL) {
    set_error("gemm_bf16_tn: too many tiles (M=%d, N=%d, nsplit=%d)", M, N, nsplit);
    return GFCC_ERR_ARG;
  }
  const unsigned grid = (unsigned)std::min<long long>(tiles, sms);
  umma_persist_gemm_kernel<BN><<<grid, PERSIST_THREADS, PTile<BN>::SMEM_BYTES, st>>>(
      ma, mb, D, ldd, M, N, K, alpha, beta, kbs, split_stride, (int)nM, (int)nN, nsplit, umma_ctl());
  GFCC_LAUNCH_CHECK();
  return GFCC_OK;
}

int launch_umma_pair(cudaStream_t st, const __nv_bfloat16 *A, long long lda, const __nv_bfloat16 *B, long long ldb,
                     float *D, long long ldd, int M, int N, int K, float alpha, float beta, int nsplit, int kbs,
                     long long split_stride) {
  CUtensorMap ma, mb;
  GFCC_TRY(make_map(&ma, A, M, K, lda, BM));
  GFCC_TRY(make_map(&mb, B, N, K, ldb, PAIR_HALF));
  static bool attr[64] = {false};
  int dev = 0;
  GFCC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64 || !attr[dev]) {
    GFCC_CUDA(cudaFuncSetAttribute(umma_pair_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   PAIR_SMEM_BYTES));
    if (dev >= 0 && dev < 64) attr[dev] = true;
  }
  const long long mp = (M + 2 * BM - 1) / (2 * BM);
  if ((N + PAIR_BN - 1) / PAIR_BN > 65535 || nsplit > 65535 || 2 * mp > 0x7fffffffLL) {
    set_error("gemm_bf16_tn: grid too large (M=%d, N=%d, nsplit=%d)", M, N, nsplit);
    return GFCC_ERR_ARG;
  }
  dim3 grid((unsigned)(2 * mp), (N + PAIR_BN - 1) / PAIR_BN, nsplit);
  umma_pair_gemm_kernel<<<grid, THREADS, PAIR_SMEM_BYTES, st>>>(ma, mb, D, ldd, M, N, K, alpha, beta, kbs,
                                                                 split_stride, umma_ctl());
  GFCC_LAUNCH_CHECK();
  return GFCC_OK;
}

// few K blocks per CTA: two stages
template <int BN>
int launch_umma(cudaStream_t st, const __nv_bfloat16 *A, long long lda, const __nv_bfloat16 *B, long long ldb,
                float *D, long long ldd, int M, int N, int K, float alpha, float beta, int nsplit, int kbs,
                long long split_stride) {
  if (kbs <= 2)
    return launch_umma_st<BN, 2>(st, A, lda, B, ldb, D, ldd, M, N, K, alpha, beta, nsplit, kbs, split_stride);
  return launch_umma_st<BN, 0>(st, A, lda, B, ldb, D, ldd, M, N, K, alpha, beta, nsplit, kbs, split_stride);
}
}  // namespace

int gemm_bf16_tn(cudaStream_t st, const __nv_bfloat16 *A, long long lda, const __nv_bfloat16 *B, long long ldb,
                 float *D, long long ldd, int M, int N, int K, float alpha, float beta, int nsplit,
                 long long split_stride) {
  if (M <= 0 || N <= 0) return GFCC_OK;
  const int nk = (K + BK - 1) / BK;
  if (nsplit < 1) nsplit = 1;
  if (nsplit > nk) nsplit = nk;
  const int kbs = (nk + nsplit - 1) / nsplit;
  nsplit = (nk + kbs - 1) / kbs;   // every split gets at least one K block
  if (nsplit > 1 && split_stride < (long long)(M - 1) * ldd + N) {
    set_error("gemm_bf16_tn: split-K writes separate partial sums (stride >= one output)");
    return GFCC_ERR_ARG;
  }
  if (K <= 0 || (lda % 8) || (ldb % 8) || lda < K || ldb < K || ldd < N ||
      (reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15)) {
    set_error("gemm_bf16_tn: need K > 0, 16-byte aligned operands and row strides that are multiples of 8 "
              "(M=%d N=%d K=%d lda=%lld ldb=%lld)", M, N, K, lda, ldb);
    return GFCC_ERR_ARG;
  }
  GFCC_TRY(check_extent_bytes(A, (long long)(M - 1) * lda * 2 + (long long)K * 2, "bf16 GEMM operand A"));
  GFCC_TRY(check_extent_bytes(B, (long long)(N - 1) * ldb * 2 + (long long)K * 2, "bf16 GEMM operand B"));
  GFCC_TRY(check_extent_bytes(D, ((long long)(M - 1) * ldd + N + (long long)(nsplit - 1) * split_stride) * 4,
                              "bf16 GEMM output D"));
  // tile widths: 64 / 128 / 256 columns per CTA, TILE_PAIR (256 x 256 over a CTA pair), or
  // TILE_PERSIST + 64 / 128 / 256 (the persistent kernel with that width)
  auto run = [&](int bn) -> int {
    if (bn == 64) return launch_umma<64>(st, A, lda, B, ldb, D, ldd, M, N, K, alpha, beta, nsplit, kbs, split_stride);
    if (bn == 128) return launch_umma<128>(st, A, lda, B, ldb, D, ldd, M, N, K, alpha, beta, nsplit, kbs, split_stride);
    if (bn == TILE_PAIR)
      return launch_umma_pair(st, A, lda, B, ldb, D, ldd, M, N, K, alpha, beta, nsplit, kbs, split_stride);
    if (bn == TILE_PERSIST + 64)
      return launch_umma_persist<64>(st, A, lda, B, ldb, D, ldd, M, N, K, alpha, beta, nsplit, kbs, split_stride);
    if (bn == TILE_PERSIST + 128)
      return launch_umma_persist<128>(st, A, lda, B, ldb, D, ldd, M, N, K, alpha, beta, nsplit, kbs, split_stride);
    if (bn == TILE_PERSIST + 256)
      return launch_umma_persist<256>(st, A, lda, B, ldb, D, ldd, M, N, K, alpha, beta, nsplit, kbs, split_stride);
    return launch_umma<256>(st, A, lda, B, ldb, D, ldd, M, N, K, alpha, beta, nsplit, kbs, split_stride);
  };
  // the pair kernel needs two row tiles and pays off on wide products with a long K loop
  const bool pair_ok = g_pair_mode != 2 && M > BM && N > 128 && kbs >= 8;
  if (g_pair_mode == 1) return pair_ok ? run(TILE_PAIR) : run(N <= 64 ? 64 : (N <= 128 ? 128 : 256));
  const int narrow = N <= 64 ? 64 : (N <= 128 ? 128 : 256);
  if (g_persist_mode == 1) return run(TILE_PERSIST + narrow);
  // the persistent kernel pays off once a launch has several waves of tiles
  const long long tiles_narrow = ((M + BM - 1) / BM) * ((N + narrow - 1) / narrow) * (long long)nsplit;
  const bool persist_ok = g_persist_mode != 2 && tiles_narrow > 2 * 152;
  // default: the narrowest tile that covers N (wide N keeps the 256-column tile)
  int bn = N <= 64 ? 64 : (N <= 128 ? 128 : 256);
  if (g_autotune && beta != 0.0f) {
    // accumulating calls are not timed (they would change D); they reuse a tuned choice if any
    const int t = umma_tuned_tile(M, N, K, nsplit);
    if (t) bn = t;
  } else if (g_autotune) {
    int dev = 0;
    GFCC_CUDA(cudaGetDevice(&dev));
    const auto key = std::make_tuple(dev, M, N, K, nsplit);
    int best = 0;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune.find(key);
      if (it != g_tune.end()) best = it->second;
    }
    if (best == 0) {
      // first call of this shape: time every tile width (second of two launches each, CUDA events on
      // the stream; beta == 0, so the repeated launches leave the same D) and keep the fastest
      cudaEvent_t e0, e1;
      GFCC_CUDA(cudaEventCreate(&e0));
      GFCC_CUDA(cudaEventCreate(&e1));
      float best_ms = 0.0f;
      for (int cand : {64, 128, 256, TILE_PAIR, TILE_PERSIST + 64, TILE_PERSIST + 128, TILE_PERSIST + 256}) {
        const int w = cand > TILE_PERSIST ? cand - TILE_PERSIST : cand;
        if (cand == TILE_PAIR ? !pair_ok
                              : ((cand > TILE_PERSIST && !persist_ok) || (w > 64 && w / 2 >= N)))
          continue;   // never better
        GFCC_TRY(run(cand));
        GFCC_CUDA(cudaEventRecord(e0, st));
        GFCC_TRY(run(cand));
        GFCC_CUDA(cudaEventRecord(e1, st));
        GFCC_CUDA(cudaEventSynchronize(e1));
        float ms = 0.0f;
        GFCC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (best == 0 || ms < best_ms) {
          best = cand;
          best_ms = ms;
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune[key] = best;
    }
    bn = best;
  }
  return run(bn);
}

int emu_fused_splits(long long K) {
  const int nk = (int)((K + BK - 1) / BK);
  return (nk + 31) / 32;
}

long long emu_fused_work_bytes(long long M, long long N, long long K) {
  const int nz = emu_fused_splits(K);
  return nz > 1 ? (long long)nz * M * N * 8 + 256 : 0;
}

int emu_gemm_fused(cudaStream_t st, const __nv_bfloat16 *Adig, long long plA, int SA, const int *eA,
                   const __nv_bfloat16 *Bdig, long long plB, int SB, const int *eB, long long ld, int M, int N, int K,
                   int P, double alpha, double beta, double *C, IMap cm, IMap cn, long long n0, double *work) {
  if (M <= 0 || N <= 0) return GFCC_OK;
  if (SA < 1 || SB < 1 || SA > EMU_MAXS || SB > EMU_MAXS || P < 2 || P > 9 || K <= 0 || (ld % 8) ||
      (reinterpret_cast<uintptr_t>(Adig) & 15) || (reinterpret_cast<uintptr_t>(Bdig) & 15) || (plA % 8) ||
      (plB % 8)) {
    set_error("emu_gemm_fused: unsupported digits (SA=%d SB=%d P=%d) or alignment", SA, SB, P);
    return GFCC_ERR_ARG;
  }
  EmuMaps maps;
  for (int i = 0; i < SA; i++) GFCC_TRY(make_map(&maps.a[i], Adig + (long long)i * plA, M, K, ld, BM));
  for (int j = 0; j < SB; j++) GFCC_TRY(make_map(&maps.b[j], Bdig + (long long)j * plB, N, K, ld, EMU_BN));
  for (int i = SA; i < EMU_MAXS; i++) maps.a[i] = maps.a[0];
  for (int j = SB; j < EMU_MAXS; j++) maps.b[j] = maps.b[0];
  static bool attr[64] = {false};
  int dev = 0;
  GFCC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64 || !attr[dev]) {
    GFCC_CUDA(cudaFuncSetAttribute(umma_emu_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, EMU_SMEM_BYTES));
    if (dev >= 0 && dev < 64) attr[dev] = true;
  }
  const int nz = emu_fused_splits(K);
  double *part = nz > 1 ? work : nullptr;
  if (nz > 1) GFCC_TRY(check_extent_bytes(work, emu_fused_work_bytes(M, N, K), "fused digit GEMM partials"));
  GFCC_TRY(check_extent(C, 0, imap_max(cm, M) + imap_max(cn, n0 + N), "fused digit GEMM output"));
  dim3 grid((M + BM - 1) / BM, (N + EMU_BN - 1) / EMU_BN, nz);
  if (grid.y > 65535 || grid.z > 65535) {
    set_error("emu_gemm_fused: grid too large");
    return GFCC_ERR_ARG;
  }
  umma_emu_kernel<<<grid, THREADS, EMU_SMEM_BYTES, st>>>(maps, SA, SB, P, M, N, K, 32, eA, eB, alpha, beta, C, cm, cn,
                                                          n0, part, umma_ctl());
  GFCC_LAUNCH_CHECK();
  if (nz > 1) {
    emu_split_reduce_kernel<<<grid1d((long long)M * N), 256, 0, st>>>(part, nz, M, N, eA, eB, alpha, beta, C, cm, cn,
                                                                       n0);
    GFCC_LAUNCH_CHECK();
  }
  return GFCC_OK;
}

void umma_set_autotune(bool on) { g_autotune = on; }

void umma_set_pair_mode(int mode) { g_pair_mode = mode; }
void umma_set_persist_mode(int mode) { g_persist_mode = mode; }

void umma_set_wait(unsigned long long wait_ns, bool skip_loads) {
  g_wait_ns = wait_ns;
  g_skip_loads = skip_loads;
}

int umma_tuned_tile(int M, int N, int K, int nsplit) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(std::make_tuple(dev, M, N, K, nsplit));
  return it == g_tune.end() ? 0 : it->second;
}

}  // namespace gfcc
