// Tensor-core (tcgen05) contractions.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace gfcc {

// D[m][n] = alpha * sum_k A[m][k] B[n][k] + beta * D[m][n]; A: M x K, B: N x K (BF16, K-major,
// row strides lda / ldb multiples of 8 elements, 16-byte aligned), D: FP32 row-major.
// nsplit > 1 splits K: partial sum z goes to D + z * split_stride (with beta != 0 each partial
// accumulates onto its own previous contents); the caller reduces the partials.  The split count actually used is returned through *nsplit_used if given.
int gemm_bf16_tn(cudaStream_t st, const __nv_bfloat16 *A, long long lda, const __nv_bfloat16 *B, long long ldb,
                 float *D, long long ldd, int M, int N, int K, float alpha, float beta, int nsplit = 1,
                 long long split_stride = 0);
// number of partial sums gemm_bf16_tn writes for a requested split of K
int umma_splits(int K, int nsplit);
// FP64-accurate product from digit planes with all digit pairs of a tile in one kernel (levels in
// TMEM): C(m, n0 + n) = alpha 2^(eA[m] + eB[n]) sum_{i+j<=P} 64^-(i+j) A_i B_j^T + beta C(m, n0 + n).
// A planes: Adig + i * plA (M x K, row stride ld), B planes: Bdig + j * plB (N x K).  With K longer
// than 2048 the product is split over K and `work` holds emu_fused_work_bytes of FP64 partials.
int emu_gemm_fused(cudaStream_t st, const __nv_bfloat16 *Adig, long long plA, int SA, const int *eA,
                   const __nv_bfloat16 *Bdig, long long plB, int SB, const int *eB, long long ld, int M, int N, int K,
                   int P, double alpha, double beta, double *C, IMap cm, IMap cn, long long n0, double *work);
long long emu_fused_work_bytes(long long M, long long N, long long K);
// Tile autotuning (on by default): the first call of each GEMM shape with beta == 0 times the
// 64 / 128 / 256-column tiles and every later call of the shape uses the fastest.
void umma_set_autotune(bool on);
// CTA-pair tile (cta_group::2, 256 x 256 per pair): 0 timed by the autotuner beside the one-CTA tiles
// (default), 1 used whenever it applies, 2 never
void umma_set_pair_mode(int mode);
// persistent tile loop (one CTA per SM, two TMEM accumulators): 0 timed by the autotuner (default),
// 1 always, 2 never
void umma_set_persist_mode(int mode);
int umma_tuned_tile(int M, int N, int K, int nsplit);   // 0 if the shape was not tuned yet
// Limit of the bounded pipeline waits of the tensor-core kernels (process-wide; default 1 s) and a
// test-only switch under which their producers issue no loads (the wait then runs out with nothing
// in flight and the kernel returns the GFCC_ERR_TIMEOUT status).
void umma_set_wait(unsigned long long wait_ns, bool skip_loads);
int umma_error_reset(cudaStream_t st);
int umma_error_check(cudaStream_t st);   // GFCC_ERR_TIMEOUT if a bounded wait gave up

}  // namespace gfcc
