// Batched dense RK4 of same-shape small systems on the tensor cores (dense.cu).
#pragma once
#include <cuda_runtime.h>

struct DenseArgs {
  int B;                  // systems
  int D, Dp, S, K;        // dimension, dimension padded for the operands, columns, drives
  int R, G, N;            // operand rows per system (1 + K) Dp, systems per CTA, B-operand rows 2 S G
  int nsteps, frame;      // RK4 steps, SG_FRAME_*
  double dt;
  const double* A;        // B x R x Dp: [C; O_1; ...; O_K] of every system (real, FP64)
  const float* coef;      // B x 3 nsteps x K: f_k at every stage slot 3 n + j
  const double* E;        // B x D: composite ground-shifted energies
  const long long* cols;  // S initial basis rows (shared by the systems)
  double2* out;           // B x D x S lab-frame final states, column innermost
  int* err;               // set to 1 when a bounded wait ran out
  int wlim;               // polls of a bounded wait
};

// Operand shape of a system shape, or false when the tensor-core path does not take
// it: 2 S in {8, 16, 32}; Dp the least multiple of 8 >= D with (1 + K) Dp a multiple
// of 32 and <= 128; G = 128 / R systems per CTA; N = 2 S G in [16, 256].
bool dense_shape(int D, int S, int K, int* Dp, int* R, int* G, int* N);
size_t dense_smem_bytes(const DenseArgs& a);
cudaError_t dense_launch(const DenseArgs& a, cudaStream_t st);
