// FP64-accurate products from BF16 digit planes on the tensor cores (ozaki.cu).
#pragma once
#include <cuda_bf16.h>

#include <cmath>

#include "common.cuh"

namespace gfcc {

// An FP64 matrix (rows x K, K-major) split into S base-64 digit planes with a power-of-two
// scale per row: A[r][k] ~= 2^exp2[r] sum_i dig[i][r][k] 64^-(i+1).
struct EmuOperand {
  __nv_bfloat16 *dig = nullptr;   // [S][rows][ld]
  int *exp2 = nullptr;            // [rows]
  long long rows = 0, K = 0, ld = 0;
  int S = 0;
  // levels this operand's products may drop (as the A operand of emu_gemm) while keeping the error
  // bound of the level-P product of the operator with its Fock-like diagonal (set at setup: see
  // emu_level_drop)
  int drop = 0;
};
// Largest row scale exponent of an operand (max over rows of exp2[r]); host value, synchronises st.
int emu_max_exponent(cudaStream_t st, const EmuOperand &e, int *out);
// Levels an operand may drop: every product term of the operand is bounded by 2^-(6P-4) times its
// row scale (at most 2^e_max), while the bound of the level-P product of the ring operator with the
// diagonal folded in is at least 2^-(6P-4) times the smallest diagonal entry of its rows; one level
// (6 bits) may go when 2^(e_max + 6) <= min_diag.  At most one level is dropped.
static inline int emu_level_drop(int e_max, double min_diag) {
  return (min_diag > 0.0 && std::ldexp(1.0, e_max + 6) <= min_diag) ? 1 : 0;
}

long long emu_operand_bytes(long long rows, long long K, int S);
int emu_slice(cudaStream_t st, const double *A, long long rows, long long K, long long lda, int S, void *mem,
              EmuOperand &out);
long long emu_gemm_work_bytes(long long M, long long N, long long K);
void emu_set_fused_max_n(long long n);   // widest product (columns) for the fused digit kernel
// C(m, n) = alpha * sum_k A[m][k] B[n][k] + beta * C(m, n) with digit pairs i + j <= P
// (the output column index of B's row n is n0 + n)
int emu_gemm(cudaStream_t st, const EmuOperand &A, const EmuOperand &B, int P, double alpha, double beta, double *C,
             IMap cm, IMap cn, void *work, long long n0 = 0);
// A strided FP64 contraction (the index maps of gemm_f64) evaluated from digit planes: operands are
// gathered K-major, split into S digits, multiplied pairwise (i + j <= P) and combined in FP64.
int gemm_f64_emulated(cudaStream_t st, long long M, long long N, long long K, double alpha, const double *A, IMap am,
                      IMap ak, const double *B, IMap bk, IMap bn, double beta, double *C, IMap cm, IMap cn, int S,
                      int P);

// The same with A already split into digit planes (rows x K, K-major; emu_slice with S digits): only B
// (given through its index maps, N columns) is gathered and split per call.
int gemm_f64_emulated_pre(cudaStream_t st, const EmuOperand &A, long long N, const double *B, IMap bk, IMap bn,
                          double alpha, double beta, double *C, IMap cm, IMap cn, int P);

}  // namespace gfcc
