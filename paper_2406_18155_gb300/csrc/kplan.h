// Device-side description of the Kronecker-sum Hamiltonian of one system and the
// complex arithmetic helpers shared by the evolution kernels.
//
// H(t) = sum_i B_i(t) [acting on mode i] + sum_e L_e(t) [mode a_e] (x) R_e(t) [mode b_e]
// (Eq. 1: 1-body and 2-body local terms).  For every RK4 stage time the d x d
// matrices of all terms are one row of the stage table:
//   B_i(t) = sum_{drives k on i} f_k(t) O_k(t)  (+ diag(E_i) in the lab frame)
//   L_e(t) = J_e A_e(t),  R_e(t) = B_e(t),  X(t)_ab = X_ab exp(i (E_a - E_b) t).
#pragma once
#include <cuda_runtime.h>
#include "sg_internal.h"

struct KPlan {
  int nq, S;
  long long D;
  int dims[SG_MAXQ];
  long long st[SG_MAXQ];          // row stride of each mode's digit
  int n1;                         // number of 1-body slots
  int s1_mode[SG_MAXQ];
  int s1_off[SG_MAXQ];            // complex offset of B_i in a table row
  int ne;
  int e_a[SG_MAXEDGE], e_b[SG_MAXEDGE];
  int e_offL[SG_MAXEDGE], e_offR[SG_MAXEDGE];
  int row;                        // complex entries per table row
  int dl;                         // max levels over modes
  unsigned par1;                  // bit i: B slot i is parity-odd
  unsigned long long parL, parR;  // bit e: L_e / R_e parity-odd
};

template <typename R> struct CT;
template <> struct CT<float> { typedef float2 T; };
template <> struct CT<double> { typedef double2 T; };

template <typename C> __host__ __device__ __forceinline__ C cmk(double x, double y) {
  C c; c.x = x; c.y = y; return c;
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {   // a*b + c
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
// conj(a)*b + c
__device__ __forceinline__ float2 cjfma(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, fmaf(a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(-a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 cjfma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.x, b.y, fma(-a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ float2 to_c(float2 v, float) { return v; }
__device__ __forceinline__ float2 to_c(double2 v, float) { return make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ double2 to_c(double2 v, double) { return v; }
__device__ __forceinline__ double2 to_c(float2 v, double) { return make_double2(v.x, v.y); }
