// The learned initial-guess model: a 3-layer perceptron (ReLU) from the features of a system
// (guess.cuh) to the 8 complex mixing coefficients of its kept neighbours.
//   x^ = (x - mu) / sd;  h1 = relu(W1 x^ + b1);  h2 = relu(W2 h1 + b2);  y = W3 h2 + b3
// Training minimises the predicted relative residual a^H Gm a / Gm_00 of the combination (guess.cuh)
// with Adam.  Precisions: FP32 master weights with an FP16 inference copy (GFCC_MLP_FP32), or FP64
// throughout (GFCC_MLP_FP64, for gradient checks).
#pragma once
#include "guess.cuh"

struct gfcc_mlp {
  int nin = gfcc::GUESS_NF, nh = 256, nout = gfcc::GUESS_NO;
  int precision = GFCC_MLP_FP32;
  long long nparam = 0;   // W1 b1 W2 b2 W3 b3 mu sd
  long long ntrain = 0;   // the trained prefix (all but mu, sd)
  void *P = nullptr, *Mo = nullptr, *Vo = nullptr, *Gr = nullptr;   // master parameters, Adam moments, gradient
  void *Pinf = nullptr;   // inference copy (transposed weights; FP16 weights + FP32 vectors, or FP64)
  long long step = 0;     // Adam step counter
  bool norm_set = false;  // mu / sd set (by gfcc_mlp_set_params or from the samples at the first training)
  double *feat = nullptr, *gram = nullptr;   // training samples: [cap][GUESS_NF], [cap][GUESS_G][2]
  long long ns = 0, cap = 0;
  void *ws = nullptr;     // training / inference workspace
  size_t ws_bytes = 0;
  cudaStream_t stream = nullptr;
};

namespace gfcc {
// y[s] = model(feat[s]) with the inference copy, s < nb (device arrays, FP64 in and out).
int mlp_infer(gfcc_mlp *m, cudaStream_t st, int nb, const double *feat, double *y);
// left vectors C[q][mu] (real, [nq][dim]) of the orbitals d_orb (device) of one sector (api.cu)
int build_left_vectors(gfcc_ctx *c, int sector, int nq, const int *d_orb, double *C, cudaStream_t st);
// Right-hand sides of orbitals porb[s] (device) of one sector into B ([s][n] complex).
int build_rhs(gfcc_ctx *c, int sector, int nsys, const int *d_porb, double *B, cudaStream_t st);
// the same for the systems with d_mask[s] != 0 only
int build_rhs_masked(gfcc_ctx *c, int sector, int nsys, const int *d_porb, const int *d_mask, double *B,
                     cudaStream_t st);
}  // namespace gfcc
