// Fixed-step RK4 evolution of a slab of state columns under the Kronecker-sum
// Hamiltonian, fidelity reduction, and the exact discrete adjoint with segment
// checkpointing.
//
// Paper: Eq. 1 (local 1- and 2-body terms), App. B (the operator is applied by
// contracting one tensor mode at a time, never as a dense D x D matrix), Eq. 13 and
// Eq. D2 (fidelities), Sec. 2.5 / Eqs. 7-12 (adjoint: the co-state is pulled back
// through each step and the gradient accumulates a_i^T dU_i/dtheta psi_{i-1}).
//
// Arithmetic: SG_FP64 runs everything in complex128.  SG_MIXED runs the stage
// contractions in complex64 and keeps the state and co-state in complex128 across
// steps; each step's increment dt/6 (k1 + 2k2 + 2k3 + k4) is formed in FP32 and added
// to the FP64 state once per step.  Reductions (fidelity, gradient) finish in FP64.
//
// This file holds the generic "gather" path: one launch per RK4 stage, each thread
// computes one slab entry and reads its neighbours along every mode a term acts on.
// It is correct for any mode count and level counts up to SG_MAXD.
#include "sg_internal.h"
#include "kplan.h"
#include "onchip.h"
#include "grad.cuh"
#include "slab.h"
#include "dense.h"
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <mutex>

namespace {

constexpr int kT = 256;

// ---------------------------------------------------------------------------
// drives and stage tables
// ---------------------------------------------------------------------------
struct DriveDev {
  int mode, op, kind, nseg, mp, amps_off;
  double amp, sigma, t0, length, omega, phase;
};

struct TabArgs {
  KPlan p;
  int nq, K, N, frame;
  int dims[SG_MAXQ];
  int eoff[SG_MAXQ];          // offset of mode i's levels in the flat energy/phase arrays
  int sumd;
  const DriveDev* drives;
  const double* amps;
  const double* E;            // flat ground-shifted energies (sumd)
  const double2* opd;         // flat truncated operators: per mode 2 x d x d
  int opd_off[SG_MAXQ];
  int e_opa[SG_MAXEDGE], e_opb[SG_MAXEDGE];
  double J[SG_MAXEDGE];
  int e_zpart[SG_MAXEDGE];    // real-operator rows: coupling factors both real (0) or both imaginary (1)
  int drv_of_slot_start[SG_MAXQ + 1];
  int drv_list[SG_MAXDRIVE];
  double dt;
  double* coef;               // 3N x K
  double2* ph;                // 3N x sumd
  double2* tab;               // 3N x row (FP64)
  float2* tab32;              // 3N x row (FP32 copy) or null
  // Suzuki-Trotter schedule: nsub Q2 sub-steps per step, sub-step j of length sc[j] dt with
  // its time-dependent terms at t_n + tau[j] dt (complex for Q4j) and its coupling
  // unitaries from set set_of[j]; set s has length setc[s] dt
  int nsub, nset;
  int q1;                     // first-order product: full-step factors, each term once per step
  int set_of[3];
  double2 sc[3], tau[3], setc[3];
};

__device__ double envelope_dev(const DriveDev& dr, const double* amps, int n, int j, double t) {
  const int m = 2 * n + j;
  if (dr.kind == SG_ENV_GAUSSIAN) {
    double x = t - dr.t0;
    return dr.amp * exp(-(x * x) / (2.0 * dr.sigma * dr.sigma));
  }
  if (dr.kind == SG_ENV_COSINE) {
    if (m > dr.mp) return 0.0;
    return dr.amp * 0.5 * (1.0 - cos(2.0 * M_PI * t / dr.length));
  }
  const int mid = 2 * n + 1;                       // PWC: segment of the step midpoint
  if (mid >= dr.mp) return 0.0;
  int seg = (int)(((long long)mid * dr.nseg) / dr.mp);
  if (seg > dr.nseg - 1) seg = dr.nseg - 1;
  return amps[dr.amps_off + seg];
}

// One block per stage q = 3n + j: coefficients f_k, phases exp(i E_a t), then every
// term matrix of the stage row.
__global__ void k_tables(TabArgs a) {
  const int q = blockIdx.x;
  const int n = q / 3, j = q % 3;
  const double t = (double)(2 * n + j) * a.dt * 0.5;
  __shared__ double f[SG_MAXDRIVE];
  __shared__ double2 ph[SG_MAXQ * SG_MAXD];
  for (int k = threadIdx.x; k < a.K; k += blockDim.x) {
    const DriveDev dr = a.drives[k];
    double E = envelope_dev(dr, a.amps, n, j, t);
    double v = E * cos(dr.omega * t + dr.phase);
    f[k] = v;
    a.coef[(size_t)q * a.K + k] = v;
  }
  for (int i = threadIdx.x; i < a.sumd; i += blockDim.x) {
    double s, c;
    if (a.frame == SG_FRAME_INTERACTION) sincos(a.E[i] * t, &s, &c); else { s = 0.0; c = 1.0; }
    ph[i] = make_double2(c, s);
    a.ph[(size_t)q * a.sumd + i] = make_double2(c, s);
  }
  __syncthreads();
  double2* row = a.tab + (size_t)q * a.p.row;
  // 1-body slots
  for (int u = 0; u < a.p.n1; ++u) {
    const int i = a.p.s1_mode[u], d = a.dims[i];
    for (int ab = threadIdx.x; ab < d * d; ab += blockDim.x) {
      const int ia = ab / d, ib = ab % d;
      double2 pa = ph[a.eoff[i] + ia], pb = ph[a.eoff[i] + ib];
      double2 P = cmul(pa, cconj(pb));
      double2 acc = make_double2(0.0, 0.0);
      for (int x = a.drv_of_slot_start[u]; x < a.drv_of_slot_start[u + 1]; ++x) {
        const int k = a.drv_list[x];
        const int op = a.drives[k].op;
        double2 O = a.opd[a.opd_off[i] + op * d * d + ab];
        double2 v = cmul(O, P);
        acc.x += f[k] * v.x;
        acc.y += f[k] * v.y;
      }
      if (a.frame == SG_FRAME_LAB && ia == ib) acc.x += a.E[a.eoff[i] + ia];
      row[a.p.s1_off[u] + ab] = acc;
      if (a.tab32) a.tab32[(size_t)q * a.p.row + a.p.s1_off[u] + ab] = make_float2((float)acc.x, (float)acc.y);
    }
  }
  for (int e = 0; e < a.p.ne; ++e) {
    const int ia_ = a.p.e_a[e], ib_ = a.p.e_b[e];
    for (int side = 0; side < 2; ++side) {
      const int i = side == 0 ? ia_ : ib_;
      const int op = side == 0 ? a.e_opa[e] : a.e_opb[e];
      const int d = a.dims[i];
      const int off = side == 0 ? a.p.e_offL[e] : a.p.e_offR[e];
      for (int ab = threadIdx.x; ab < d * d; ab += blockDim.x) {
        const int x = ab / d, y = ab % d;
        double2 P = cmul(ph[a.eoff[i] + x], cconj(ph[a.eoff[i] + y]));
        double2 v = cmul(a.opd[a.opd_off[i] + op * d * d + ab], P);
        if (side == 0) { v.x *= a.J[e]; v.y *= a.J[e]; }
        row[off + ab] = v;
        if (a.tab32) a.tab32[(size_t)q * a.p.row + off + ab] = make_float2((float)v.x, (float)v.y);
      }
    }
  }
}

// exp(i theta) for large |theta|: reduction to [-pi, pi] in FP64 with a two-term
// 2 pi (Cody-Waite), then the FP32 sine and cosine.  The phase keeps an absolute
// error of a few 1e-8 where an FP32 product E t alone would lose ~1e-4 rad at
// E t ~ 1e4 rad.
__device__ __forceinline__ float2 cis32(double theta) {
  const double k = rint(theta * 0.15915494309189535);                // 1 / (2 pi)
  const double r = fma(-k, 6.283185307179586, theta) - k * 2.4492935982947064e-16;
  float sn, cs;
  sincosf((float)r, &sn, &cs);
  return make_float2(cs, sn);
}

// Stage tables in FP32 only (mixed precision on the on-chip kernels, which read
// nothing else): the same coefficients, phases and term rows as k_tables, with the
// FP64 work cut to the envelope and the argument reduction.
__global__ void k_tables32(TabArgs a, float* __restrict__ coef32, float2* __restrict__ ph32) {
  const int q = blockIdx.x;
  const int n = q / 3, j = q % 3;
  const double t = (double)(2 * n + j) * a.dt * 0.5;
  __shared__ float f[SG_MAXDRIVE];
  __shared__ float2 ph[SG_MAXQ * SG_MAXD];
  for (int k = threadIdx.x; k < a.K; k += blockDim.x) {
    const DriveDev dr = a.drives[k];
    const double E = envelope_dev(dr, a.amps, n, j, t);
    const float v = (float)E * cis32(dr.omega * t + dr.phase).x;
    f[k] = v;
    coef32[(size_t)q * a.K + k] = v;
  }
  for (int i = threadIdx.x; i < a.sumd; i += blockDim.x) {
    const float2 c = a.frame == SG_FRAME_INTERACTION ? cis32(a.E[i] * t) : make_float2(1.f, 0.f);
    ph[i] = c;
    ph32[(size_t)q * a.sumd + i] = c;
  }
  __syncthreads();
  float2* row = a.tab32 + (size_t)q * a.p.row;
  auto pmul = [&](int i, int x, int y) {          // exp(i (E_x - E_y) t)
    const float2 px = ph[a.eoff[i] + x], py = ph[a.eoff[i] + y];
    return make_float2(px.x * py.x + px.y * py.y, px.y * py.x - px.x * py.y);
  };
  for (int u = 0; u < a.p.n1; ++u) {
    const int i = a.p.s1_mode[u], d = a.dims[i];
    for (int ab = threadIdx.x; ab < d * d; ab += blockDim.x) {
      const int ia = ab / d, ib = ab % d;
      const float2 P = pmul(i, ia, ib);
      float2 acc = make_float2(0.f, 0.f);
      for (int x = a.drv_of_slot_start[u]; x < a.drv_of_slot_start[u + 1]; ++x) {
        const int k = a.drv_list[x];
        const double2 O = a.opd[a.opd_off[i] + a.drives[k].op * d * d + ab];
        const float ox = (float)O.x, oy = (float)O.y;
        acc.x += f[k] * (ox * P.x - oy * P.y);
        acc.y += f[k] * (ox * P.y + oy * P.x);
      }
      if (a.frame == SG_FRAME_LAB && ia == ib) acc.x += (float)a.E[a.eoff[i] + ia];
      row[a.p.s1_off[u] + ab] = acc;
    }
  }
  for (int e = 0; e < a.p.ne; ++e) {
    for (int side = 0; side < 2; ++side) {
      const int i = side == 0 ? a.p.e_a[e] : a.p.e_b[e];
      const int op = side == 0 ? a.e_opa[e] : a.e_opb[e];
      const int d = a.dims[i];
      const int off = side == 0 ? a.p.e_offL[e] : a.p.e_offR[e];
      const float sc = side == 0 ? (float)a.J[e] : 1.f;
      for (int ab = threadIdx.x; ab < d * d; ab += blockDim.x) {
        const float2 P = pmul(i, ab / d, ab % d);
        const double2 O = a.opd[a.opd_off[i] + op * d * d + ab];
        const float ox = (float)O.x, oy = (float)O.y;
        row[off + ab] = make_float2(sc * (ox * P.x - oy * P.y), sc * (ox * P.y + oy * P.x));
      }
    }
  }
}

// Stage rows of the real-operator tiled passes (slab_dev.cuh): per 1-body slot
// sum_k f_k(t) O_k (+ diag E in the lab frame) and per coupling J A (x) B, each as
// its real matrix in the truncated eigenbasis (the interaction-frame phases are
// applied to the state instead).  A coupling whose two factors are imaginary
// stores -J Im(A) and Im(B).  Rows are packed for the passes: FP32 duplicates each
// element into both lanes of a float2; with zpar every operator is parity-odd and
// row x keeps its columns c with x + c odd in its first d / 2 places.
template <typename Z> __device__ __forceinline__ Z zpack(double v);
template <> __device__ __forceinline__ float2 zpack<float2>(double v) { return make_float2((float)v, (float)v); }
template <> __device__ __forceinline__ double zpack<double>(double v) { return v; }

template <typename Z>
__global__ void k_tables_z(TabArgs a, Z* __restrict__ zt, int zpar) {
  const int q = blockIdx.x;
  const int n = q / 3, j = q % 3;
  const double t = (double)(2 * n + j) * a.dt * 0.5;
  __shared__ double f[SG_MAXDRIVE];
  for (int k = threadIdx.x; k < a.K; k += blockDim.x) {
    const DriveDev dr = a.drives[k];
    f[k] = envelope_dev(dr, a.amps, n, j, t) * cos(dr.omega * t + dr.phase);
  }
  __syncthreads();
  Z* row = zt + (size_t)q * a.p.row;
  for (int u = 0; u < a.p.n1; ++u) {
    const int i = a.p.s1_mode[u], d = a.dims[i];
    for (int el = threadIdx.x; el < d * d; el += blockDim.x) {
      const int x = el / d, kk = el % d;
      double v = 0.0;
      if (!zpar || kk < d / 2) {
        const int c = zpar ? ((x + 1) & 1) + 2 * kk : kk;
        for (int xx = a.drv_of_slot_start[u]; xx < a.drv_of_slot_start[u + 1]; ++xx) {
          const int k = a.drv_list[xx];
          v += f[k] * a.opd[a.opd_off[i] + a.drives[k].op * d * d + x * d + c].x;
        }
        if (a.frame == SG_FRAME_LAB && x == c) v += a.E[a.eoff[i] + x];
      }
      row[a.p.s1_off[u] + el] = zpack<Z>(v);
    }
  }
  for (int e = 0; e < a.p.ne; ++e) {
    const bool im = a.e_zpart[e] != 0;
    for (int side = 0; side < 2; ++side) {
      const int i = side == 0 ? a.p.e_a[e] : a.p.e_b[e];
      const int op = side == 0 ? a.e_opa[e] : a.e_opb[e];
      const int d = a.dims[i];
      const int off = side == 0 ? a.p.e_offL[e] : a.p.e_offR[e];
      const double sc = side == 0 ? (im ? -a.J[e] : a.J[e]) : 1.0;
      for (int el = threadIdx.x; el < d * d; el += blockDim.x) {
        const int x = el / d, kk = el % d;
        double v = 0.0;
        if (!zpar || kk < d / 2) {
          const int c = zpar ? ((x + 1) & 1) + 2 * kk : kk;
          const double2 O = a.opd[a.opd_off[i] + op * d * d + x * d + c];
          v = sc * (im ? O.y : O.x);
        }
        row[off + el] = zpack<Z>(v);
      }
    }
  }
}

// The drive operators themselves as real matrices in the truncated eigenbasis,
// packed like the stage rows (one DL x DL block per drive, DL the common level
// count): the pulse-gradient adjoint of the real-operator passes contracts drive k's
// operator with the rotated co-state and state.  One block per drive.
template <typename Z>
__global__ void k_ops_z(TabArgs a, Z* __restrict__ zo, int zpar, int DL) {
  const int k = blockIdx.x;
  const DriveDev dr = a.drives[k];
  const int i = dr.mode, d = a.dims[i];
  for (int el = threadIdx.x; el < DL * DL; el += blockDim.x) {
    const int x = el / DL, kk = el % DL;
    double v = 0.0;
    if (x < d && (zpar ? kk < d / 2 : kk < d)) {
      const int c = zpar ? ((x + 1) & 1) + 2 * kk : kk;
      v = a.opd[a.opd_off[i] + dr.op * d * d + x * d + c].x;
    }
    zo[(size_t)k * DL * DL + el] = zpack<Z>(v);
  }
}

// ---------------------------------------------------------------------------
// Suzuki-Trotter tables (Sec. 2.3, App. A), lab frame
// ---------------------------------------------------------------------------
// exp(A) of a small complex matrix (n x n, row-major) by scaling and squaring of
// the Taylor series (Moler and Van Loan's method 3): A / 2^s with |A / 2^s|_1 <= 1/2,
// 18 Taylor terms (remainder below 1e-22 of the norm), then s squarings.  Serial,
// one thread: R = exp(A); W1, W2 are n x n scratch.
__device__ void expm_serial(const double2* A, int n, double2* R, double2* W1, double2* W2) {
  double nrm = 0.0;
  for (int c = 0; c < n; ++c) {
    double col = 0.0;
    for (int r = 0; r < n; ++r) col += hypot(A[r * n + c].x, A[r * n + c].y);
    nrm = fmax(nrm, col);
  }
  int sq = 0;
  while (nrm > 0.5 && sq < 60) { nrm *= 0.5; ++sq; }
  const double sc = ldexp(1.0, -sq);
  for (int i = 0; i < n * n; ++i) {
    W1[i] = make_double2((i / n == i % n) ? 1.0 : 0.0, 0.0);    // current term
    R[i] = W1[i];
  }
  for (int k = 1; k <= 18; ++k) {
    for (int r = 0; r < n; ++r)                                 // W2 = W1 (A sc) / k
      for (int c = 0; c < n; ++c) {
        double2 acc = make_double2(0.0, 0.0);
        for (int m = 0; m < n; ++m) acc = cfma(W1[r * n + m], A[m * n + c], acc);
        W2[r * n + c] = make_double2(acc.x * sc / k, acc.y * sc / k);
      }
    for (int i = 0; i < n * n; ++i) {
      W1[i] = W2[i];
      R[i].x += W2[i].x;
      R[i].y += W2[i].y;
    }
  }
  for (int q = 0; q < sq; ++q) {
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) {
        double2 acc = make_double2(0.0, 0.0);
        for (int m = 0; m < n; ++m) acc = cfma(R[r * n + m], R[m * n + c], acc);
        W2[r * n + c] = acc;
      }
    for (int i = 0; i < n * n; ++i) R[i] = W2[i];
  }
}

// Drive coefficient f_k = E(t) cos(omega t + phase) at the complex time t = tr + i ti
// inside step n: Gaussian and cosine envelopes and the carrier continued analytically,
// a piecewise-constant envelope from the segment of the step's midpoint (R8).  For
// ti = 0 it equals envelope_dev(dr, amps, n, 1, tr) cos(omega tr + phase) exactly.
__device__ double2 coef_complex(const DriveDev& dr, const double* amps, int n, double tr, double ti) {
  double2 E;
  if (dr.kind == SG_ENV_GAUSSIAN) {
    const double x = tr - dr.t0, y = ti, s2 = dr.sigma * dr.sigma;
    const double mag = dr.amp * exp(-(x * x - y * y) / (2.0 * s2)), ang = -(x * y) / s2;
    E = make_double2(mag * cos(ang), mag * sin(ang));
  } else if (dr.kind == SG_ENV_COSINE) {
    if (2 * n + 1 > dr.mp) return make_double2(0.0, 0.0);
    const double a = 2.0 * M_PI * tr / dr.length, b = 2.0 * M_PI * ti / dr.length;
    E = make_double2(dr.amp * 0.5 * (1.0 - cos(a) * cosh(b)), dr.amp * 0.5 * (sin(a) * sinh(b)));
  } else {
    E = make_double2(envelope_dev(dr, amps, n, 1, tr), 0.0);
  }
  const double a = dr.omega * tr + dr.phase, b = dr.omega * ti;
  return cmul(E, make_double2(cos(a) * cosh(b), -(sin(a) * sinh(b))));
}

// U_i(m) = exp(A), A = -i c_j (dt/2) H_i(t_n + tau_j dt) for sub-step m = J n + j,
// H_i = diag(E) + sum_{drives k on i} f_k O_k.  A is left in A.
__device__ void q2_onebody(const TabArgs& a, int i, int m, double2* U, double2* A, double2* W1, double2* W2) {
  const int d = a.dims[i];
  const int n = m / a.nsub, j = m - n * a.nsub;
  const double tr = (double)(2 * n + 1) * a.dt * 0.5 + (a.tau[j].x - 0.5) * a.dt;
  const double ti = a.tau[j].y * a.dt;
  for (int x = 0; x < d * d; ++x) A[x] = make_double2(0.0, 0.0);
  for (int x = 0; x < d; ++x) A[x * d + x].x = a.E[a.eoff[i] + x];
  for (int k = 0; k < a.K; ++k) {
    const DriveDev& dr = a.drives[k];
    if (dr.mode != i) continue;
    const double2 f = coef_complex(dr, a.amps, n, tr, ti);
    const double2* O = a.opd + a.opd_off[i] + dr.op * d * d;
    for (int x = 0; x < d * d; ++x) A[x] = cfma(f, O[x], A[x]);
  }
  const double h = a.q1 ? a.dt : a.dt * 0.5;        // Q1: the full step
  for (int x = 0; x < d * d; ++x) {
    const double2 cH = cmul(a.sc[j], A[x]);
    A[x] = make_double2(h * cH.y, -h * cH.x);                                     // -i c H dt/2 (Q1: dt)
  }
  expm_serial(A, d, U, W1, W2);
}

// Row m < M - 1 (M = J N sub-steps): V_i(m) = U_i(m+1) U_i(m) (the second half of
// sub-step m followed by the first of sub-step m + 1); row M - 1: U_i(M - 1); row M:
// U_i(0).  One thread per (row, mode).
__global__ void k_q2_onebody(TabArgs a, int DL, double2* __restrict__ rows) {
  const int M = a.N * a.nsub, nrow = M + 1;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nrow * a.nq; x += gridDim.x * blockDim.x) {
    const int m = x / a.nq, i = x - m * a.nq, d = a.dims[i];
    double2 U0[SG_MAXD * SG_MAXD], U1[SG_MAXD * SG_MAXD], A[SG_MAXD * SG_MAXD];
    double2 W1[SG_MAXD * SG_MAXD], W2[SG_MAXD * SG_MAXD];
    double2* out = rows + ((size_t)m * a.nq + i) * DL * DL;
    if (m == M) {
      q2_onebody(a, i, 0, U0, A, W1, W2);
      for (int y = 0; y < d * d; ++y) out[y] = U0[y];
      continue;
    }
    if (a.q1) {
      // Q1: row M is step 0's 1-body factor, applied first; row m < M - 1 step m + 1's,
      // applied after step m's couplings; row M - 1 the identity
      if (m == M - 1) {
        for (int y = 0; y < d * d; ++y) out[y] = make_double2(y % (d + 1) == 0 ? 1.0 : 0.0, 0.0);
      } else {
        q2_onebody(a, i, m + 1, U0, A, W1, W2);
        for (int y = 0; y < d * d; ++y) out[y] = U0[y];
      }
      continue;
    }
    q2_onebody(a, i, m, U0, A, W1, W2);
    if (m == M - 1) {
      for (int y = 0; y < d * d; ++y) out[y] = U0[y];
      continue;
    }
    q2_onebody(a, i, m + 1, U1, A, W1, W2);
    for (int r = 0; r < d; ++r)
      for (int c = 0; c < d; ++c) {
        double2 acc = make_double2(0.0, 0.0);
        for (int q = 0; q < d; ++q) acc = cfma(U1[r * d + q], U0[q * d + c], acc);
        out[r * d + c] = acc;
      }
  }
}

// Per set s and coupling e: G_half = exp(-i c_s J A (x) B dt/2) and G_full = G_half^2 (the
// two middle half steps of the palindrome), d_a d_b x d_a d_b with row index x d_b + z,
// at matrices (s ne + e) 2 + {0, 1}; for the pull-back of the gradient, from matrix
// 2 ne nset on, per (s, e) four: the inverses G_half^-1, G_full^-1 (the states) and the
// adjoints G_half^dag, G_full^dag (the co-states), equal pairs when c_s is real.  One
// thread per (set, coupling).
__global__ void k_q2_edges(TabArgs a, int DL, double2* __restrict__ mats, double2* __restrict__ scratch) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int ne = a.p.ne;
  if (x >= ne * a.nset) return;
  const int sidx = x / ne, e = x - sidx * ne;
  const int ia = a.p.e_a[e], ib = a.p.e_b[e], da = a.dims[ia], db = a.dims[ib], n = da * db;
  const double2* Aop = a.opd + a.opd_off[ia] + a.e_opa[e] * da * da;
  const double2* Bop = a.opd + a.opd_off[ib] + a.e_opb[e] * db * db;
  double2* M = scratch + (size_t)x * 3 * n * n;
  double2* W1 = M + n * n;
  double2* W2 = W1 + n * n;
  const size_t D4 = (size_t)DL * DL * DL * DL;
  double2* Gh = mats + (size_t)x * 2 * D4;
  double2* Gf = Gh + D4;
  double2* Ghi = mats + ((size_t)2 * ne * a.nset + (size_t)x * 4) * D4;
  double2* Gfi = Ghi + D4;
  double2* Ghd = Gfi + D4;
  double2* Gfd = Ghd + D4;
  const double h = a.J[e] * a.dt * 0.5;
  const double2 c = a.setc[sidx];
  for (int xx = 0; xx < da; ++xx)
    for (int z = 0; z < db; ++z)
      for (int p = 0; p < da; ++p)
        for (int q = 0; q < db; ++q) {
          const double2 v = cmul(c, cmul(Aop[xx * da + p], Bop[z * db + q]));
          M[(xx * db + z) * n + p * db + q] = make_double2(h * v.y, -h * v.x);   // -i c J (A x B) dt/2
        }
  expm_serial(M, n, Gh, W1, W2);
  for (int r = 0; r < n; ++r)
    for (int q = 0; q < n; ++q) {
      double2 acc = make_double2(0.0, 0.0);
      for (int m = 0; m < n; ++m) acc = cfma(Gh[r * n + m], Gh[m * n + q], acc);
      Gf[r * n + q] = acc;
    }
  for (int r = 0; r < n; ++r)
    for (int q = 0; q < n; ++q) {
      Ghd[r * n + q] = cconj(Gh[q * n + r]);
      Gfd[r * n + q] = cconj(Gf[q * n + r]);
    }
  for (int i = 0; i < n * n; ++i) M[i] = make_double2(-M[i].x, -M[i].y);
  expm_serial(M, n, Ghi, W1, W2);                                                // exp(+i c J (A x B) dt/2)
  for (int r = 0; r < n; ++r)
    for (int q = 0; q < n; ++q) {
      double2 acc = make_double2(0.0, 0.0);
      for (int m = 0; m < n; ++m) acc = cfma(Ghi[r * n + m], Ghi[m * n + q], acc);
      Gfi[r * n + q] = acc;
    }
}

// Gradient tables (pulse parameters), rows [J N][2 nq + K][d^2]: per sub-step m the
// inverses U_i(m)^-1 = exp(-A) of each mode's (unmerged) 1-body half step (they pull the
// states back), their adjoints U_i(m)^dag (they pull the co-states back; equal to the
// inverses when the step length is real), then per drive k on mode i,
// M_k(m) = U_i(m)^-1 L_k(m) with L_k(m) = L(A, -i c_j (dt/2) O_k) the Frechet derivative
// of expm at A = -i c_j (dt/2) H_i(t_n + tau_j dt), the top-right block of
// exp([[A, E], [0, A]]) (Sec. 2.5: dU/df_k).  Q1: the step's full-step factor, dt for
// dt/2 throughout.  One thread per (m, row).
constexpr int kQ2MaxD = 5;
__global__ void k_q2_gradtabs(TabArgs a, int DL, double2* __restrict__ rows) {
  const int per = 2 * a.nq + a.K, M = a.N * a.nsub;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < M * per; x += gridDim.x * blockDim.x) {
    const int m = x / per, r = x - m * per;
    double2 U[SG_MAXD * SG_MAXD], A[SG_MAXD * SG_MAXD], W1[SG_MAXD * SG_MAXD], W2[SG_MAXD * SG_MAXD];
    double2 Ui[SG_MAXD * SG_MAXD];
    double2* out = rows + ((size_t)m * per + r) * DL * DL;
    if (r < 2 * a.nq) {
      const int i = r < a.nq ? r : r - a.nq, d = a.dims[i];
      q2_onebody(a, i, m, U, A, W1, W2);
      if (r >= a.nq) {
        for (int p = 0; p < d; ++p)
          for (int c = 0; c < d; ++c) out[p * d + c] = cconj(U[c * d + p]);
      } else {
        for (int p = 0; p < d * d; ++p) A[p] = make_double2(-A[p].x, -A[p].y);
        expm_serial(A, d, Ui, W1, W2);
        for (int p = 0; p < d * d; ++p) out[p] = Ui[p];
      }
      continue;
    }
    const DriveDev& dr = a.drives[r - 2 * a.nq];
    const int i = dr.mode, d = a.dims[i], mm = 2 * d;
    if (d > kQ2MaxD) continue;                      // the on-chip Suzuki-Trotter plan has d <= 5
    q2_onebody(a, i, m, U, A, W1, W2);              // U_i(m), and A = -i c (dt/2) H_i on return
    constexpr int MM = 4 * kQ2MaxD * kQ2MaxD;
    double2 Z[MM], RZ[MM], Z1[MM], Z2[MM];
    const double2* O = a.opd + a.opd_off[i] + dr.op * d * d;
    const double h = a.q1 ? a.dt : a.dt * 0.5;       // Q1: full-step factors
    const double2 c = a.sc[m % a.nsub];
    for (int p = 0; p < mm * mm; ++p) Z[p] = make_double2(0.0, 0.0);
    for (int p = 0; p < d; ++p)
      for (int q = 0; q < d; ++q) {
        Z[p * mm + q] = A[p * d + q];
        Z[(p + d) * mm + q + d] = A[p * d + q];
        const double2 cO = cmul(c, O[p * d + q]);
        Z[p * mm + q + d] = make_double2(h * cO.y, -h * cO.x);                 // -i c (dt/2) O (Q1: dt)
      }
    expm_serial(Z, mm, RZ, Z1, Z2);
    for (int p = 0; p < d * d; ++p) A[p] = make_double2(-A[p].x, -A[p].y);
    expm_serial(A, d, Ui, W1, W2);                  // U^-1 = exp(-A)
    // df_k/dtheta = z (a segment or amplitude indicator): z = carrier x envelope shape at
    // the sub-step time (complex for Q4j), folded in here so that the real part the
    // adjoint takes is Re(<psibar, L psi> df/dtheta)
    const int n = m / a.nsub, j = m - n * a.nsub;
    const double tr = (double)(2 * n + 1) * a.dt * 0.5 + (a.tau[j].x - 0.5) * a.dt, ti = a.tau[j].y * a.dt;
    double2 z;
    if (dr.kind == SG_ENV_GAUSSIAN) {
      const double xg = tr - dr.t0, s2 = dr.sigma * dr.sigma;
      const double mag = exp(-(xg * xg - ti * ti) / (2.0 * s2)), ang = -(xg * ti) / s2;
      z = make_double2(mag * cos(ang), mag * sin(ang));
    } else if (dr.kind == SG_ENV_COSINE) {
      const double ca = 2.0 * M_PI * tr / dr.length, cb = 2.0 * M_PI * ti / dr.length;
      z = 2 * n + 1 > dr.mp ? make_double2(0.0, 0.0)
                            : make_double2(0.5 * (1.0 - cos(ca) * cosh(cb)), 0.5 * (sin(ca) * sinh(cb)));
    } else {
      z = make_double2(2 * n + 1 < dr.mp ? 1.0 : 0.0, 0.0);
    }
    const double wa = dr.omega * tr + dr.phase, wb = dr.omega * ti;
    z = cmul(z, make_double2(cos(wa) * cosh(wb), -(sin(wa) * sinh(wb))));
    for (int p = 0; p < d; ++p)                     // M = z U^-1 L
      for (int q = 0; q < d; ++q) {
        double2 acc = make_double2(0.0, 0.0);
        for (int w = 0; w < d; ++w) acc = cfma(Ui[p * d + w], RZ[w * mm + q + d], acc);
        out[p * d + q] = cmul(z, acc);
      }
  }
}

// ---------------------------------------------------------------------------
// H y at one slab entry (gather form)
// ---------------------------------------------------------------------------
template <typename C>
__device__ __forceinline__ C apply_entry(const KPlan& p, const C* __restrict__ M,
                                         const C* __restrict__ X, long long e) {
  const int S = p.S;
  const long long r = e / S;
  const int s = (int)(e - r * S);
  C acc = cmk<C>(0.0, 0.0);
  for (int u = 0; u < p.n1; ++u) {
    const int i = p.s1_mode[u], d = p.dims[i];
    const long long st = p.st[i];
    const int l = (int)((r / st) % d);
    const C* Xb = X + (r - (long long)l * st) * S + s;
    const C* Mr = M + p.s1_off[u] + l * d;
    const long long stS = st * S;
    if ((p.par1 >> u) & 1) {
      for (int b = (l + 1) & 1; b < d; b += 2) acc = cfma(Mr[b], Xb[b * stS], acc);
    } else {
      for (int b = 0; b < d; ++b) acc = cfma(Mr[b], Xb[b * stS], acc);
    }
  }
  for (int q = 0; q < p.ne; ++q) {
    const int i = p.e_a[q], j = p.e_b[q];
    const int di = p.dims[i], dj = p.dims[j];
    const long long sti = p.st[i], stj = p.st[j];
    const int li = (int)((r / sti) % di), lj = (int)((r / stj) % dj);
    const C* Xb = X + (r - (long long)li * sti - (long long)lj * stj) * S + s;
    const C* L = M + p.e_offL[q] + li * di;
    const C* R = M + p.e_offR[q] + lj * dj;
    const bool pl = (p.parL >> q) & 1ull, pr = (p.parR >> q) & 1ull;
    const long long siS = sti * S, sjS = stj * S;
    for (int x = pl ? ((li + 1) & 1) : 0; x < di; x += pl ? 2 : 1) {
      C u = cmk<C>(0.0, 0.0);
      for (int y = pr ? ((lj + 1) & 1) : 0; y < dj; y += pr ? 2 : 1)
        u = cfma(R[y], Xb[x * siS + y * sjS], u);
      acc = cfma(L[x], u, acc);
    }
  }
  return acc;
}

template <typename C>
__device__ __forceinline__ void load_row(const C* __restrict__ tab, int row, C* sm) {
  for (int i = threadIdx.x; i < row; i += blockDim.x) sm[i] = tab[i];
  __syncthreads();
}

// Forward RK4 stage.  X = stage input y_s, k = -i H y_s.
//   STAGE 0: D = dt/6 k,  Xn = psi + dt/2 k      STAGE 1: D += dt/3 k, Xn = psi + dt/2 k
//   STAGE 2: D += dt/3 k, Xn = psi + dt k        STAGE 3: psi_out = psi_in + (D + dt/6 k), Xn = psi_out
// STORE: recompute mode of the adjoint (writes Xn only).
template <typename R, int STAGE, bool STORE>
__global__ void __launch_bounds__(kT) k_fwd(KPlan p, const typename CT<R>::T* __restrict__ X,
                                            const typename CT<R>::T* __restrict__ tabrow,
                                            const double2* __restrict__ psi_in, double2* psi_out,
                                            typename CT<R>::T* __restrict__ Xn,
                                            typename CT<R>::T* __restrict__ Dacc, double dt) {
  typedef typename CT<R>::T C;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* M = reinterpret_cast<C*>(smraw);
  load_row(tabrow, p.row, M);
  const long long total = p.D * p.S;
  const R h = (R)dt;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    C a = apply_entry(p, M, X, e);
    C k = cmk<C>(a.y, -a.x);                       // -i * H y
    const double2 ps = psi_in[e];
    const C pr = to_c(ps, R(0));
    if (STAGE == 0) {
      if (!STORE) Dacc[e] = cmk<C>(h / 6 * k.x, h / 6 * k.y);
      Xn[e] = cmk<C>(pr.x + h / 2 * k.x, pr.y + h / 2 * k.y);
    } else if (STAGE == 1) {
      if (!STORE) { C d = Dacc[e]; Dacc[e] = cmk<C>(d.x + h / 3 * k.x, d.y + h / 3 * k.y); }
      Xn[e] = cmk<C>(pr.x + h / 2 * k.x, pr.y + h / 2 * k.y);
    } else if (STAGE == 2) {
      if (!STORE) { C d = Dacc[e]; Dacc[e] = cmk<C>(d.x + h / 3 * k.x, d.y + h / 3 * k.y); }
      Xn[e] = cmk<C>(pr.x + h * k.x, pr.y + h * k.y);
    } else {
      C d = Dacc[e];
      R incx = d.x + h / 6 * k.x, incy = d.y + h / 6 * k.y;
      double2 pn = make_double2(ps.x + (double)incx, ps.y + (double)incy);
      psi_out[e] = pn;
      Xn[e] = to_c(pn, R(0));
    }
  }
}

// Adjoint RK4 stage (reverse order 3, 2, 1, 0).  X = kbar_s, ybar_s = A_s^dag kbar_s = i H kbar_s.
//   3: Db = yb, Xn = dt/3 pb + dt yb      2: Db += yb, Xn = dt/3 pb + dt/2 yb
//   1: Db += yb, Xn = dt/6 pb + dt/2 yb   0: pb <- pb + (Db + yb), Xn = dt/6 pb
template <typename R, int STAGE>
__global__ void __launch_bounds__(kT) k_adj(KPlan p, const typename CT<R>::T* __restrict__ X,
                                            const typename CT<R>::T* __restrict__ tabrow,
                                            double2* __restrict__ pbar,
                                            typename CT<R>::T* __restrict__ Xn,
                                            typename CT<R>::T* __restrict__ Db, double dt) {
  typedef typename CT<R>::T C;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* M = reinterpret_cast<C*>(smraw);
  load_row(tabrow, p.row, M);
  const long long total = p.D * p.S;
  const R h = (R)dt;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    C a = apply_entry(p, M, X, e);
    C yb = cmk<C>(-a.y, a.x);                      // i * H kbar
    const double2 pb = pbar[e];
    const C pr = to_c(pb, R(0));
    if (STAGE == 3) {
      Db[e] = yb;
      Xn[e] = cmk<C>(h / 3 * pr.x + h * yb.x, h / 3 * pr.y + h * yb.y);
    } else if (STAGE == 2) {
      C d = Db[e];
      Db[e] = cmk<C>(d.x + yb.x, d.y + yb.y);
      Xn[e] = cmk<C>(h / 3 * pr.x + h / 2 * yb.x, h / 3 * pr.y + h / 2 * yb.y);
    } else if (STAGE == 1) {
      C d = Db[e];
      Db[e] = cmk<C>(d.x + yb.x, d.y + yb.y);
      Xn[e] = cmk<C>(h / 6 * pr.x + h / 2 * yb.x, h / 6 * pr.y + h / 2 * yb.y);
    } else {
      C d = Db[e];
      double2 pn = make_double2(pb.x + (double)(d.x + yb.x), pb.y + (double)(d.y + yb.y));
      pbar[e] = pn;
      C q = to_c(pn, R(0));
      Xn[e] = cmk<C>(h / 6 * q.x, h / 6 * q.y);
    }
  }
}

// complex64 -> complex128, element-wise
__global__ void k_widen(const float2* __restrict__ src, double2* __restrict__ dst, long long n) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    dst[e] = make_double2((double)src[e].x, (double)src[e].y);
}

template <typename R>
__global__ void k_cast(const double2* __restrict__ src, typename CT<R>::T* __restrict__ dst,
                       long long n, double scale) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    double2 v = src[e];
    dst[e] = to_c(make_double2(v.x * scale, v.y * scale), R(0));
  }
}

__global__ void k_init_cols(double2* psi, long long D, int S, const long long* cols) {
  const long long total = D * S;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long r = e / S;
    int s = (int)(e - r * S);
    psi[e] = make_double2(cols[s] == r ? 1.0 : 0.0, 0.0);
  }
}

// ---------------------------------------------------------------------------
// frame epilogue and fidelity (Eq. 13, Eq. D2)
// ---------------------------------------------------------------------------
struct FrameArgs {
  int nq, S;
  long long D;
  int dims[SG_MAXQ];
  long long st[SG_MAXQ];
  int eoff[SG_MAXQ];
  const double* E;
  double T;
  double sign;                // -1: psi_lab = exp(-i Hd T) psi_I ; +1: the inverse
};

// x <- exp(sign * i * E_tot(r) * T) x
__global__ void k_frame(FrameArgs a, double2* x) {
  const long long total = a.D * a.S;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long r = e / a.S;
    double Et = 0.0;
    for (int i = 0; i < a.nq; ++i) Et += a.E[a.eoff[i] + (int)((r / a.st[i]) % a.dims[i])];
    double s, c;
    sincos(a.sign * Et * a.T, &s, &c);
    double2 v = x[e];
    x[e] = make_double2(c * v.x - s * v.y, c * v.y + s * v.x);
  }
}

struct FidArgs {
  int S, Dc, Sc, full, kind, nq;
  int qpos[SG_MAXQ];          // bit of mode i in a comp label (LSB = 0), -1 for a coupler mode
  const double2* Uc;          // Dc x S   (comp rows of the lab-frame columns)
  const double2* Tg;          // Dc x Dc
  const int* lab;             // S: comp label of each column or -1
  double* F;                  // [F_avg, F_state]
  double2* bar;               // Dc x S co-state (lab frame) or null
  double2* M;                 // Dc x Dc scratch (full only)
  double* ebar_frame;         // nq x SG_MAXD or null
  double T;
  int frame;
};

__device__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  double r = red[0];
  __syncthreads();
  return r;
}

// Single block, FP64, fixed-order reductions.
__global__ void k_fidelity(FidArgs a) {
  __shared__ double red[kT];
  __shared__ double2 zsh;
  const int tid = threadIdx.x, nt = blockDim.x;
  // z = sum over comp columns of <target_{lab(s)} | psi_s>
  double zr = 0.0, zi = 0.0;
  for (int i = tid; i < a.Dc * a.S; i += nt) {
    int r = i / a.S, s = i % a.S;
    int l = a.lab[s];
    if (l < 0) continue;
    double2 t = a.Tg[r * a.Dc + l], u = a.Uc[i];
    zr += t.x * u.x + t.y * u.y;
    zi += t.x * u.y - t.y * u.x;
  }
  double Zr = block_sum(zr, red), Zi = block_sum(zi, red);
  const double Sc = (double)a.Sc;
  double Fst = (Zr * Zr + Zi * Zi) / (Sc * Sc);
  double Favg = nan("");
  double2 trM = make_double2(Zr, Zi);
  if (a.full) {
    // M[x][l] = sum_r conj(T[r][x]) U[r][col(l)]
    const int Dc = a.Dc;
    double fro = 0.0;
    for (int i = tid; i < Dc * Dc; i += nt) {
      int x = i / Dc, l = i % Dc;
      int col = -1;
      for (int s = 0; s < a.S; ++s) if (a.lab[s] == l) { col = s; break; }
      double2 acc = make_double2(0.0, 0.0);
      for (int r = 0; r < Dc; ++r) {
        double2 t = a.Tg[r * Dc + x], u = a.Uc[r * a.S + col];
        acc.x += t.x * u.x + t.y * u.y;
        acc.y += t.x * u.y - t.y * u.x;
      }
      a.M[i] = acc;
      fro += acc.x * acc.x + acc.y * acc.y;
    }
    double Fro = block_sum(fro, red);
    Favg = (Fro + Zr * Zr + Zi * Zi) / ((double)Dc * (Dc + 1));
  }
  if (tid == 0) { a.F[0] = Favg; a.F[1] = Fst; }
  if (!a.bar) return;
  __syncthreads();
  // co-state dF/dRe psi + i dF/dIm psi on the comp rows
  for (int i = tid; i < a.Dc * a.S; i += nt) {
    int r = i / a.S, s = i % a.S;
    int l = a.lab[s];
    double2 b = make_double2(0.0, 0.0);
    if (l >= 0) {
      if (a.kind == SG_FID_STATE) {
        double2 t = a.Tg[r * a.Dc + l];
        double sc = 2.0 / (Sc * Sc);
        b = make_double2(sc * (trM.x * t.x - trM.y * t.y), sc * (trM.x * t.y + trM.y * t.x));
      } else {
        const int Dc = a.Dc;
        double2 acc = make_double2(0.0, 0.0);             // (T M)[r][l]
        for (int x = 0; x < Dc; ++x) {
          double2 t = a.Tg[r * Dc + x], m = a.M[x * Dc + l];
          acc.x += t.x * m.x - t.y * m.y;
          acc.y += t.x * m.y + t.y * m.x;
        }
        double2 t = a.Tg[r * Dc + l];
        acc.x += trM.x * t.x - trM.y * t.y;
        acc.y += trM.x * t.y + trM.y * t.x;
        double sc = 2.0 / ((double)Dc * (Dc + 1));
        b = make_double2(sc * acc.x, sc * acc.y);
      }
    }
    a.bar[i] = b;
  }
}

// Column-sharded fidelity (Sec. 4.2: the unitary's columns distributed over
// devices).  Both fidelities depend on the columns only through sums over them:
//   z = tr M = sum_s <t_l(s) | u_s>,  q = tr(M M^dag) = sum_s ||T^dag u_s||^2,  S_c,
// so a shard evolves its columns, contributes its partial sums, and after the sums
// over shards computes F and its columns' co-states exactly as the unsharded solve:
//   F_state = |z / S_c|^2,  F_avg = (q + |z|^2) / (D_c (D_c + 1)),
//   co-state of column s (label l):  F_state: 2 z / S_c^2 t_l,
//                                    F_avg:   2 (T (T^dag u_s) + z t_l) / (D_c (D_c + 1)).
// k_shard_partials writes M_loc[x][s] = (T^dag u_s)_x (D_c x S, the shard's columns)
// and part = {Re z, Im z, q, S_c} of this shard.
__global__ void k_shard_partials(FidArgs a, double* __restrict__ part) {
  __shared__ double red[kT];
  const int tid = threadIdx.x, nt = blockDim.x, Dc = a.Dc;
  double zr = 0.0, zi = 0.0, q = 0.0, sc = 0.0;
  for (int i = tid; i < Dc * a.S; i += nt) {
    const int x = i / a.S, s = i % a.S, l = a.lab[s];
    double2 acc = make_double2(0.0, 0.0);
    if (l >= 0) {
      for (int r = 0; r < Dc; ++r) {
        const double2 t = a.Tg[r * Dc + x], u = a.Uc[r * a.S + s];
        acc.x += t.x * u.x + t.y * u.y;
        acc.y += t.x * u.y - t.y * u.x;
      }
      q += acc.x * acc.x + acc.y * acc.y;
      if (x == l) { zr += acc.x; zi += acc.y; }
      if (x == 0) sc += 1.0;
    }
    a.M[i] = acc;
  }
  const double Zr = block_sum(zr, red), Zi = block_sum(zi, red);
  const double Q = block_sum(q, red), Sc = block_sum(sc, red);
  if (tid == 0) { part[0] = Zr; part[1] = Zi; part[2] = Q; part[3] = Sc; }
}

// F from the sums over every shard (glob = {Re z, Im z, q, S_c}) and the co-states
// of this shard's columns (lab frame, D_c x S).  F_avg is defined when the shards
// together evolved every computational state once (S_c = D_c; the caller's column
// partition guarantees they are distinct).
__global__ void k_shard_costate(FidArgs a, const double* __restrict__ glob) {
  const int tid = threadIdx.x, nt = blockDim.x, Dc = a.Dc;
  const double Zr = glob[0], Zi = glob[1], Q = glob[2], Sc = glob[3];
  const bool full = (int)llround(Sc) == Dc;
  if (tid == 0) {
    a.F[0] = full ? (Q + Zr * Zr + Zi * Zi) / ((double)Dc * (Dc + 1)) : nan("");
    a.F[1] = (Zr * Zr + Zi * Zi) / (Sc * Sc);
  }
  if (!a.bar) return;
  for (int i = tid; i < Dc * a.S; i += nt) {
    const int r = i / a.S, s = i % a.S, l = a.lab[s];
    double2 b = make_double2(0.0, 0.0);
    if (l >= 0) {
      const double2 t = a.Tg[r * Dc + l];
      if (a.kind == SG_FID_STATE) {
        const double f = 2.0 / (Sc * Sc);
        b = make_double2(f * (Zr * t.x - Zi * t.y), f * (Zr * t.y + Zi * t.x));
      } else {
        double2 acc = make_double2(Zr * t.x - Zi * t.y, Zr * t.y + Zi * t.x);
        for (int x = 0; x < Dc; ++x) {
          const double2 tt = a.Tg[r * Dc + x], m = a.M[x * a.S + s];
          acc.x += tt.x * m.x - tt.y * m.y;
          acc.y += tt.x * m.y + tt.y * m.x;
        }
        const double f = 2.0 / ((double)Dc * (Dc + 1));
        b = make_double2(f * acc.x, f * acc.y);
      }
    }
    a.bar[i] = b;
  }
}

// Virtual-Z compensation: phases a (rows) and b (columns) of diag(1, e^{i phase}) gates
// on the qubits maximising |tr M|, M = T^dag Z(a) U Z(b), tr M = sum_rl W[r][l]
// za[r] zb[l] with W = conj(T) o U and za[r] = exp(i sum_q a_q bit_q(r)).  Coordinate
// ascent from zero phases, a_1..a_n then b_1..b_n (qubit q on label bit n - 1 - q):
// with the other phases fixed tr M = X_0 + e^{i phi} X_1 over the labels whose bit is
// 0 / 1, largest in modulus at phi = arg X_0 - arg X_1.  Stops at the first sweep that
// does not raise |tr M|, at most 2000 sweeps.  Writes T_eff = conj(za) o T o conj(zb)
// (tr(T_eff^dag U) = tr M), whose plain fidelity and co-state are the compensated ones.
// One block; warp 0 runs the O(D_c) coordinate updates, all threads the O(D_c^2) sums.
struct VzArgs {
  int S, Dc, n;
  const double2* Uc;          // Dc x S
  const double2* Tg;          // Dc x Dc
  const int* lab;             // S
  double2* W;                 // Dc x Dc scratch
  double2* Teff;              // Dc x Dc out
};
__global__ void k_vz_comp(VzArgs a) {
  constexpr int MAXDC = 256;
  __shared__ double2 v[MAXDC], za[MAXDC], zb[MAXDC];
  __shared__ int colof[MAXDC];
  __shared__ double ph[2][8];
  __shared__ int stop;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, Dc = a.Dc, n = a.n;
  for (int s = tid; s < a.S; s += nt)
    if (a.lab[s] >= 0) colof[a.lab[s]] = s;
  if (tid < 16) ph[tid / 8][tid % 8] = 0.0;
  for (int r = tid; r < Dc; r += nt) { za[r] = make_double2(1.0, 0.0); zb[r] = make_double2(1.0, 0.0); }
  __syncthreads();
  for (int i = tid; i < Dc * Dc; i += nt) {
    const int r = i / Dc, l = i - r * Dc;
    a.W[i] = cmul(cconj(a.Tg[i]), a.Uc[(size_t)r * a.S + colof[l]]);
  }
  __syncthreads();
  // warp 0: sum over labels of z[r] w[r] split by bit (fixed lane order)
  auto wsum = [&](const double2* z, const double2* w, int bit, int want) {
    double2 acc = make_double2(0.0, 0.0);
    for (int r = lane; r < Dc; r += 32)
      if (bit < 0 || ((r >> bit) & 1) == want) acc = cfma(z[r], w[r], acc);
    for (int o = 16; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    return acc;
  };
  auto refresh = [&](double2* z, const double* p) {   // z[r] = exp(i sum_q p_q bit_q(r))
    for (int r = lane; r < Dc; r += 32) {
      double t = 0.0;
      for (int q = 0; q < n; ++q) t += ((r >> (n - 1 - q)) & 1) ? p[q] : 0.0;
      double sn, cs;
      sincos(t, &sn, &cs);
      z[r] = make_double2(cs, sn);
    }
    __syncwarp();
  };
  double best = 0.0;
  // |tr M| at zero phases: v = W 1, tr = sum v
  for (int r = tid; r < Dc; r += nt) {
    double2 acc = make_double2(0.0, 0.0);
    for (int l = 0; l < Dc; ++l) { acc.x += a.W[(size_t)r * Dc + l].x; acc.y += a.W[(size_t)r * Dc + l].y; }
    v[r] = acc;
  }
  __syncthreads();
  if (tid < 32) {
    const double2 t = wsum(za, v, -1, 0);
    best = hypot(t.x, t.y);
  }
  for (int sweep = 0; sweep < 2000; ++sweep) {
    for (int side = 0; side < 2; ++side) {
      double2* zs = side == 0 ? za : zb;                  // the side being updated
      const double2* zo = side == 0 ? zb : za;
      // v = W zo (rows, side 0) or W^T zo (columns, side 1)
      for (int r = tid; r < Dc; r += nt) {
        double2 acc = make_double2(0.0, 0.0);
        for (int l = 0; l < Dc; ++l)
          acc = cfma(side == 0 ? a.W[(size_t)r * Dc + l] : a.W[(size_t)l * Dc + r], zo[l], acc);
        v[r] = acc;
      }
      __syncthreads();
      if (tid < 32) {
        for (int q = 0; q < n; ++q) {
          const int bit = n - 1 - q;
          if (lane == 0) ph[side][q] = 0.0;
          __syncwarp();
          refresh(zs, ph[side]);
          const double2 x0 = wsum(zs, v, bit, 0), x1 = wsum(zs, v, bit, 1);
          const double m1 = hypot(x1.x, x1.y);
          if (lane == 0) ph[side][q] = m1 > 0.0 ? atan2(x0.y, x0.x) - atan2(x1.y, x1.x) : 0.0;
          __syncwarp();
          refresh(zs, ph[side]);
        }
      }
      __syncthreads();
    }
    if (tid < 32) {
      const double2 t = wsum(zb, v, -1, 0);              // v = W^T za from the column side
      const double now = hypot(t.x, t.y);
      if (lane == 0) stop = !(now > best);
      best = now;
    }
    __syncthreads();
    if (stop) break;
  }
  for (int i = tid; i < Dc * Dc; i += nt) {
    const int r = i / Dc, l = i - r * Dc;
    a.Teff[i] = cmul(cconj(za[r]), cmul(a.Tg[i], cconj(zb[l])));
  }
}

// Energy co-gradient of the frame epilogue psi_lab = exp(-i Hd T) psi_I:
// ebar[i][c] += sum over comp rows with digit_i = c of Re(conj(bar) (-i T) psi_lab).
// Comp rows only have digits 0 and 1.  Single block.
__global__ void k_frame_ebar(FidArgs a) {
  __shared__ double red[kT];
  for (int i = 0; i < a.nq; ++i) {
    for (int c = 0; c < 2; ++c) {
      double part = 0.0;
      for (int x = threadIdx.x; x < a.Dc * a.S; x += blockDim.x) {
        int r = x / a.S;
        int bit = a.qpos[i] >= 0 ? (r >> a.qpos[i]) & 1 : 0;      // a coupler sits in level 0
        if (bit != c) continue;
        double2 b = a.bar[x], u = a.Uc[x];
        // Re(conj(b) * (-i T) u) = T * (b.x*u.y - b.y*u.x)
        part += a.T * (b.x * u.y - b.y * u.x);
      }
      double tot = block_sum(part, red);
      if (threadIdx.x == 0) a.ebar_frame[i * SG_MAXD + c] += tot;
    }
  }
}

struct CompArgs {
  int nq, S, Dc;
  int dims[SG_MAXQ];
  int qpos[SG_MAXQ];          // bit of mode i in a comp label (LSB = 0), -1 for a coupler mode
};
// Flat row of computational state j: qubit mode i takes bit qpos[i] of j, a
// coupler mode level 0.
__device__ long long comp_row(const CompArgs& a, int j) {
  long long r = 0;
  for (int i = 0; i < a.nq; ++i) r = r * a.dims[i] + (a.qpos[i] >= 0 ? ((j >> a.qpos[i]) & 1) : 0);
  return r;
}
// Dressed basis: columns start in the dressed computational states, psi[r][s] =
// Vc[r][lab(s)]; the block is Uc[j][s] = <v_j|psi_s>; the co-state of the final states
// is pbar[r][s] = sum_j Vc[r][j] barc[j][s].  Vc is D x Dc, row-major.
__global__ void k_init_dressed(const double2* __restrict__ Vc, const int* __restrict__ lab, long long D, int S,
                               int Dc, double2* __restrict__ psi) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < D * S; i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / S;
    const int s = (int)(i - r * S);
    psi[i] = Vc[r * Dc + lab[s]];
  }
}
__global__ void k_gather_dressed(const double2* __restrict__ Vc, const double2* __restrict__ psi, long long D, int S,
                                 int Dc, double2* __restrict__ Uc) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Dc * S; i += gridDim.x * blockDim.x) {
    const int j = i / S, s = i - j * S;
    double2 acc = make_double2(0.0, 0.0);
    for (long long r = 0; r < D; ++r) acc = cfma(cconj(Vc[r * Dc + j]), psi[r * S + s], acc);
    Uc[i] = acc;
  }
}
__global__ void k_scatter_dressed(const double2* __restrict__ Vc, const double2* __restrict__ barc, long long D,
                                  int S, int Dc, double2* __restrict__ pbar) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < D * S; i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / S;
    const int s = (int)(i - r * S);
    double2 acc = make_double2(0.0, 0.0);
    for (int j = 0; j < Dc; ++j) acc = cfma(Vc[r * Dc + j], barc[(size_t)j * S + s], acc);
    pbar[i] = acc;
  }
}

__global__ void k_gather_comp(CompArgs a, const double2* psi, double2* Uc) {
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < a.Dc * a.S; x += gridDim.x * blockDim.x) {
    int j = x / a.S, s = x % a.S;
    Uc[x] = psi[comp_row(a, j) * a.S + s];
  }
}
__global__ void k_scatter_comp(CompArgs a, const double2* bar, double2* pbar) {
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < a.Dc * a.S; x += gridDim.x * blockDim.x) {
    int j = x / a.S, s = x % a.S;
    pbar[comp_row(a, j) * a.S + s] = bar[x];
  }
}

// ---------------------------------------------------------------------------
// gradient: cross-densities per stage and their contraction into co-gradients
// ---------------------------------------------------------------------------
template <typename C, int DL>
__device__ void block_reduce_store(C (&acc)[DL][DL], double2* out, double* red) {
  // warp reduce each element, then combine warps in order through shared memory
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int x = 0; x < DL; ++x)
    for (int y = 0; y < DL; ++y) {
      double vr = acc[x][y].x, vi = acc[x][y].y;
      for (int o = 16; o > 0; o >>= 1) {
        vr += __shfl_xor_sync(0xffffffffu, vr, o);
        vi += __shfl_xor_sync(0xffffffffu, vi, o);
      }
      if (lane == 0) { red[2 * (warp * DL * DL + x * DL + y)] = vr; red[2 * (warp * DL * DL + x * DL + y) + 1] = vi; }
    }
  __syncthreads();
  for (int i = threadIdx.x; i < DL * DL; i += blockDim.x) {
    double sr = 0.0, si = 0.0;
    for (int w = 0; w < nw; ++w) { sr += red[2 * (w * DL * DL + i)]; si += red[2 * (w * DL * DL + i) + 1]; }
    out[i] = make_double2(sr, si);
  }
  __syncthreads();
}

// Cross-densities of one stage: for every term slot the d x d matrix
//   C_ab = <kbar, (|a><b| on the slot's mode, other factor of the term applied) y>
// summed over the slab.  The last block to finish sums the block partials in
// block order and contracts them (W = -i C) into the co-gradient accumulators.
template <typename R, int DL>
__global__ void __launch_bounds__(kT) k_xdens(XArgs a, const typename CT<R>::T* __restrict__ X,
                                              const typename CT<R>::T* __restrict__ Y) {
  typedef typename CT<R>::T C;
  extern __shared__ __align__(16) unsigned char smraw[];
  double* red = reinterpret_cast<double*>(smraw);                       // 2 * (kT/32) * DL^2
  C* Mt = reinterpret_cast<C*>(red + 2 * (kT / 32) * DL * DL);           // stage row
  const KPlan& p = a.p;
  for (int i = threadIdx.x; i < p.row; i += blockDim.x) Mt[i] = to_c(a.tabrow[i], R(0));
  __syncthreads();
  const int S = p.S;
  const long long gstride = (long long)gridDim.x * blockDim.x;
  double2* mypart = a.partial + (size_t)blockIdx.x * a.nW * DL * DL;
  int w = 0;
  // ---- 1-body slots
  for (int u = 0; u < p.n1; ++u, ++w) {
    const int i = p.s1_mode[u], d = p.dims[i];
    const long long st = p.st[i];
    const long long nf = p.D / d * S;
    C acc[DL][DL];
#pragma unroll
    for (int x = 0; x < DL; ++x)
#pragma unroll
      for (int y = 0; y < DL; ++y) acc[x][y] = cmk<C>(0.0, 0.0);
    for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gstride) {
      const long long tt = f / S;
      const int s = (int)(f - tt * S);
      const long long rlo = tt % st, rhi = tt / st;
      const long long base = (rhi * d * st + rlo) * S + s;
      C xv[DL], yv[DL];
#pragma unroll
      for (int x = 0; x < DL; ++x) {
        xv[x] = x < d ? X[base + x * st * S] : cmk<C>(0.0, 0.0);
        yv[x] = x < d ? Y[base + x * st * S] : cmk<C>(0.0, 0.0);
      }
#pragma unroll
      for (int x = 0; x < DL; ++x)
#pragma unroll
        for (int y = 0; y < DL; ++y) acc[x][y] = cjfma(xv[x], yv[y], acc[x][y]);
    }
    block_reduce_store<C, DL>(acc, mypart + (size_t)w * DL * DL, red);
  }
  // ---- 2-body slots: L side (fibres along mode a with R applied on mode b), then R side
  for (int side = 0; side < (a.ham ? 2 : 0); ++side) {
    for (int q = 0; q < p.ne; ++q, ++w) {
      const int i = side == 0 ? p.e_a[q] : p.e_b[q];      // fibre mode
      const int j = side == 0 ? p.e_b[q] : p.e_a[q];      // mode of the other factor
      const int d = p.dims[i], dj = p.dims[j];
      const long long st = p.st[i], stj = p.st[j];
      const C* O = Mt + (side == 0 ? p.e_offR[q] : p.e_offL[q]);
      const long long nf = p.D / d * S;
      C acc[DL][DL];
#pragma unroll
      for (int x = 0; x < DL; ++x)
#pragma unroll
        for (int y = 0; y < DL; ++y) acc[x][y] = cmk<C>(0.0, 0.0);
      for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gstride) {
        const long long tt = f / S;
        const int s = (int)(f - tt * S);
        const long long rlo = tt % st, rhi = tt / st;
        const long long r0 = rhi * d * st + rlo;           // row with digit i = 0
        const int lj = (int)((r0 / stj) % dj);
        const long long base = r0 * S + s;
        const long long basej = (r0 - (long long)lj * stj) * S + s;
        C xv[DL], yv[DL];
#pragma unroll
        for (int x = 0; x < DL; ++x) {
          xv[x] = x < d ? X[base + x * st * S] : cmk<C>(0.0, 0.0);
          C u = cmk<C>(0.0, 0.0);
          if (x < d)
            for (int c = 0; c < dj; ++c) u = cfma(O[lj * dj + c], Y[basej + x * st * S + c * stj * S], u);
          yv[x] = u;
        }
#pragma unroll
        for (int x = 0; x < DL; ++x)
#pragma unroll
          for (int y = 0; y < DL; ++y) acc[x][y] = cjfma(xv[x], yv[y], acc[x][y]);
      }
      block_reduce_store<C, DL>(acc, mypart + (size_t)w * DL * DL, red);
    }
  }
  // ---- last block: fixed-order sum over blocks and contraction
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned tk = atomicAdd(a.ticket, 1u);
    last = (tk == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  double2* Wt = reinterpret_cast<double2*>(smraw);        // reuse: nW * DL^2 double2
  for (int i = threadIdx.x; i < a.nW * DL * DL; i += blockDim.x) {
    double sr = 0.0, si = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) {
      double2 v = __ldcg(a.partial + (size_t)b * a.nW * DL * DL + i);
      sr += v.x;
      si += v.y;
    }
    Wt[i] = make_double2(si, -sr);                         // W = -i C
  }
  __syncthreads();
  if (threadIdx.x == 0) *a.ticket = 0u;
  const int slot = threadIdx.x;
  if (slot < a.nW && (a.ham || slot < a.p.n1)) contract_slot(a, slot, Wt + slot * DL * DL, DL);
}

// Pulse-parameter chain, one block per drive: dF/dparam = sum over stages of
// dF/df * df/dparam, and the carrier-frequency co-gradient sum dF/df * E (-sin) t.
// J = 0: the 3N RK4 stage slots (stage j of step n at t = (2n + j) dt/2).  J >= 1: the
// J N Suzuki-Trotter sub-steps, whose gF already carries df/dtheta up to the parameter
// indicator (k_q2_gradtabs); a PWC sub-step feeds the segment of its step's midpoint
// (reading R8), and no carrier co-gradient is formed.
__global__ void k_pulse_chain(const DriveDev* drives, const double* amps, const double* gF,
                              int K, int N, double dt, const int* pulse_off, int n_pulse, double* grad_pulse,
                              double* omega_bar, int J) {
  const int k = blockIdx.x;
  const DriveDev dr = drives[k];
  const int np = dr.kind == SG_ENV_PWC ? dr.nseg : 1;
  extern __shared__ double part[];             // blockDim x (np + 1)
  const int tid = threadIdx.x;
  double* mine = part + tid * (np + 1);
  for (int x = 0; x <= np; ++x) mine[x] = 0.0;
  const int per = J > 0 ? J : 3;
  for (int q = tid; q < per * N; q += blockDim.x) {
    const int n = q / per, jq = q % per;
    if (J > 0) {
      // Suzuki-Trotter: the carrier and the envelope shape are already in gF (the
      // gradient tables carry them); only the parameter each sub-step feeds is left
      const double g = gF[(size_t)q * K + k];
      if (dr.kind != SG_ENV_PWC) {
        mine[0] += g;
      } else {
        int seg = (int)(((long long)(2 * n + 1) * dr.nseg) / dr.mp);
        if (seg > dr.nseg - 1) seg = dr.nseg - 1;
        if (2 * n + 1 < dr.mp) mine[seg] += g;
      }
      continue;
    }
    const int j = jq;
    const double t = (double)(2 * n + j) * dt * 0.5;
    const double g = gF[(size_t)q * K + k];
    const double c = cos(dr.omega * t + dr.phase);
    const double E = envelope_dev(dr, amps, n, j, t);
    mine[np] += g * E * (-sin(dr.omega * t + dr.phase)) * t;
    if (dr.kind == SG_ENV_GAUSSIAN) {
      double x = t - dr.t0;
      mine[0] += g * c * exp(-(x * x) / (2.0 * dr.sigma * dr.sigma));
    } else if (dr.kind == SG_ENV_COSINE) {
      if (2 * n + j <= dr.mp) mine[0] += g * c * 0.5 * (1.0 - cos(2.0 * M_PI * t / dr.length));
    } else {
      const int mid = 2 * n + 1;
      if (mid < dr.mp) {
        int seg = (int)(((long long)mid * dr.nseg) / dr.mp);
        if (seg > dr.nseg - 1) seg = dr.nseg - 1;
        mine[seg] += g * c;
      }
    }
  }
  __syncthreads();
  for (int x = tid; x <= np; x += blockDim.x) {
    double s = 0.0;
    for (int y = 0; y < (int)blockDim.x; ++y) s += part[y * (np + 1) + x];
    if (x < np) {
      const int o = pulse_off[k] + x;
      if (o >= 0 && o < n_pulse) grad_pulse[o] = s;               // offsets come from the host plan
    } else {
      omega_bar[k] = s;
    }
  }
}

struct AssembleArgs {
  int nq, n1, ne, K;
  int dims[SG_MAXQ];
  int s1_of_mode[SG_MAXQ];
  int drv_mode[SG_MAXDRIVE], drv_op[SG_MAXDRIVE], drv_omode[SG_MAXDRIVE];
  int e_a[SG_MAXEDGE], e_b[SG_MAXEDGE], e_opa[SG_MAXEDGE], e_opb[SG_MAXEDGE];
  GradAcc acc;
  const double* omega_bar;
  const double* ebar_frame;
  double2* opbar;      // nq x 2 x MAXD^2
  double* ebar;        // nq x MAXD
};

// Sums the per-term co-gradients into per-mode operator and energy co-gradients
// in a fixed order.  One block, thread per (mode, level pair).
__global__ void k_assemble(AssembleArgs a) {
  for (int x = threadIdx.x; x < a.nq * SG_MAXD * SG_MAXD; x += blockDim.x) {
    const int i = x / (SG_MAXD * SG_MAXD), ab = x % (SG_MAXD * SG_MAXD);
    // n and phi only: local operators have fixed matrix elements (no device-parameter chain)
    double2 o[2] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
    for (int k = 0; k < a.K; ++k)
      if (a.drv_mode[k] == i && a.drv_op[k] < 2) {
        double2 v = a.acc.obD[(size_t)k * SG_MAXD * SG_MAXD + ab];
        o[a.drv_op[k]].x += v.x; o[a.drv_op[k]].y += v.y;
      }
    for (int e = 0; e < a.ne; ++e) {
      if (a.e_a[e] == i && a.e_opa[e] < 2) { double2 v = a.acc.obL[(size_t)e * SG_MAXD * SG_MAXD + ab]; o[a.e_opa[e]].x += v.x; o[a.e_opa[e]].y += v.y; }
      if (a.e_b[e] == i && a.e_opb[e] < 2) { double2 v = a.acc.obR[(size_t)e * SG_MAXD * SG_MAXD + ab]; o[a.e_opb[e]].x += v.x; o[a.e_opb[e]].y += v.y; }
    }
    a.opbar[(i * 2 + 0) * SG_MAXD * SG_MAXD + ab] = o[0];
    a.opbar[(i * 2 + 1) * SG_MAXD * SG_MAXD + ab] = o[1];
  }
  for (int x = threadIdx.x; x < a.nq * SG_MAXD; x += blockDim.x) {
    const int i = x / SG_MAXD, c = x % SG_MAXD;
    double s = a.ebar_frame[x];
    if (a.s1_of_mode[i] >= 0) s += a.acc.ebB[a.s1_of_mode[i] * SG_MAXD + c];
    for (int e = 0; e < a.ne; ++e) {
      if (a.e_a[e] == i) s += a.acc.ebL[e * SG_MAXD + c];
      if (a.e_b[e] == i) s += a.acc.ebR[e * SG_MAXD + c];
    }
    if (c == 1)
      for (int k = 0; k < a.K; ++k)
        if (a.drv_omode[k] == i) s += a.omega_bar[k];
    a.ebar[x] = s;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
};

// Per-solve device buffers, stream-ordered (cudaMallocAsync / cudaFreeAsync on the
// solve's stream), so solves on different streams never synchronise the device
// through allocation.  The device's default pool keeps freed memory for reuse.
struct Arena {
  std::vector<void*> ptrs;
  size_t bytes = 0;
  cudaStream_t st = nullptr;
  ~Arena() { for (void* p : ptrs) cudaFreeAsync(p, st); }
  template <typename T> T* get(size_t n) {
    void* p = nullptr;
    size_t b = std::max<size_t>(n * sizeof(T), 16);
    if (cudaMallocAsync(&p, b, st) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    ptrs.push_back(p);
    bytes += b;
    return static_cast<T*>(p);
  }
};

// Keep freed pool memory cached in the process (released at exit), once per device.
void keep_pool_memory(int device) {
  static std::mutex mu;
  static bool done[64] = {};
  std::lock_guard<std::mutex> lk(mu);
  if (device < 0 || device >= 64 || done[device]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  done[device] = true;
}

struct Setup {
  KPlan p{};
  TabArgs ta{};
  int N = 0, K = 0, nq = 0, sumd = 0, Dc = 0;
  long long D = 0;
  int S = 0;
  double dt = 0, T = 0;
  std::vector<DriveDev> drives;
  std::vector<double> amps;
  std::vector<double> Eflat;
  std::vector<double2> opdflat;
  std::vector<int> s1_of_mode;
  std::vector<int> pulse_off;
  int n_pulse = 0;
  bool q2 = false;                // a Suzuki-Trotter solver (Q2, Q4, Q4j; lab frame)
  int solver = SG_SOLVER_RK4;
  int frame = SG_FRAME_INTERACTION;
  int nqb = 0;                    // qubit modes (the rest are couplers)
  int qpos[SG_MAXQ] = {0};        // bit of mode i in a comp label (LSB = 0), -1 for a coupler
};

// The Suzuki-Trotter schedules of App. A as Q2 sub-steps (c dt at t_n + tau dt):
// Q2 (1, 1/2); Q4 (p, p/2), (1 - 2p, 1/2), (p, 1 - p/2) with p = 1 / (2 - 2^(1/3));
// Q4j (p, p/2), (p*, p + p*/2) with p = (3 - i sqrt 3) / 6, the complex sub-step times
// of Q4j being where its drive coefficients are continued (coef_complex).
void set_schedule(int solver, TabArgs& ta) {
  const double p4 = 1.0 / (2.0 - std::cbrt(2.0));
  const double2 pj = make_double2(0.5, -std::sqrt(3.0) / 6.0);
  const double2 pjc = make_double2(pj.x, -pj.y);
  if (solver == SG_SOLVER_Q4) {
    ta.nsub = 3; ta.nset = 2;
    ta.sc[0] = ta.sc[2] = make_double2(p4, 0.0);
    ta.sc[1] = make_double2(1.0 - 2.0 * p4, 0.0);
    ta.tau[0] = make_double2(p4 / 2.0, 0.0);
    ta.tau[1] = make_double2(0.5, 0.0);
    ta.tau[2] = make_double2(1.0 - p4 / 2.0, 0.0);
    ta.set_of[0] = ta.set_of[2] = 0; ta.set_of[1] = 1;
    ta.setc[0] = ta.sc[0]; ta.setc[1] = ta.sc[1];
  } else if (solver == SG_SOLVER_Q4J) {
    ta.nsub = 2; ta.nset = 2;
    ta.sc[0] = pj; ta.sc[1] = pjc;
    ta.tau[0] = make_double2(pj.x / 2.0, pj.y / 2.0);
    ta.tau[1] = make_double2(pj.x + pjc.x / 2.0, pj.y + pjc.y / 2.0);
    ta.set_of[0] = 0; ta.set_of[1] = 1;
    ta.setc[0] = pj; ta.setc[1] = pjc;
  } else {
    ta.nsub = 1; ta.nset = 1;
    ta.sc[0] = ta.setc[0] = make_double2(1.0, 0.0);
    ta.tau[0] = make_double2(0.5, 0.0);
    ta.set_of[0] = 0;
  }
  ta.q1 = solver == SG_SOLVER_Q1 ? 1 : 0;
}

sg_status build_setup(sg_system* sys, const sg_evolve_opts* o, Setup& s) {
  sg_ctx* ctx = sys->ctx;
  if (!o) return sg_fail(ctx, SG_E_INVALID, "null options");
  if (!(o->dt > 0.0) || !(o->T > 0.0) || !std::isfinite(o->T) || !std::isfinite(o->dt))
    return sg_fail(ctx, SG_E_INVALID, "T and dt must be positive and finite");
  double x = o->T / o->dt;
  long long N = llround(x);
  if (N < 1 || std::fabs(x - (double)N) > 1e-9 * std::max(1.0, x))
    return sg_fail(ctx, SG_E_INVALID, "T/dt must be a whole number of steps");
  if (N > (1ll << 26)) return sg_fail(ctx, SG_E_INVALID, "too many steps");
  if (o->precision != SG_FP64 && o->precision != SG_MIXED)
    return sg_fail(ctx, SG_E_INVALID, "precision must be SG_FP64 or SG_MIXED");
  if (o->frame != SG_FRAME_INTERACTION && o->frame != SG_FRAME_LAB)
    return sg_fail(ctx, SG_E_INVALID, "frame must be SG_FRAME_INTERACTION or SG_FRAME_LAB");
  if (o->solver != SG_SOLVER_RK4 && o->solver != SG_SOLVER_Q1 && o->solver != SG_SOLVER_Q2 &&
      o->solver != SG_SOLVER_Q4 && o->solver != SG_SOLVER_Q4J)
    return sg_fail(ctx, SG_E_INVALID, "solver must be SG_SOLVER_RK4, SG_SOLVER_Q1, SG_SOLVER_Q2, SG_SOLVER_Q4 or "
                                      "SG_SOLVER_Q4J");
  s.solver = o->solver;
  s.q2 = o->solver != SG_SOLVER_RK4;
  s.frame = s.q2 ? SG_FRAME_LAB : o->frame;          // Suzuki-Trotter always runs in the lab frame
  if (o->ncols < 1) return sg_fail(ctx, SG_E_INVALID, "ncols must be >= 1");
  s.N = (int)N;
  s.dt = o->dt;
  s.T = (double)N * o->dt;
  s.nq = (int)sys->modes.size();
  s.S = o->ncols;
  KPlan& p = s.p;
  p.nq = s.nq;
  p.S = s.S;
  long long D = 1;
  int dl = 0;
  for (int i = 0; i < s.nq; ++i) { p.dims[i] = sys->modes[i].d; D *= p.dims[i]; dl = std::max(dl, p.dims[i]); }
  p.D = D;
  p.dl = dl;
  s.D = D;
  if (D * (long long)s.S > (1ll << 40)) return sg_fail(ctx, SG_E_INVALID, "slab too large");
  long long st = 1;
  for (int i = s.nq - 1; i >= 0; --i) { p.st[i] = st; st *= p.dims[i]; }
  s.nqb = 0;
  for (int i = 0; i < s.nq; ++i) s.nqb += sys->modes[i].coupler ? 0 : 1;
  for (int i = 0, b = s.nqb - 1; i < s.nq; ++i) s.qpos[i] = sys->modes[i].coupler ? -1 : b--;
  s.Dc = 1 << std::min(s.nqb, 20);
  // energies and operators, flattened
  s.sumd = 0;
  int eoff[SG_MAXQ], ooff[SG_MAXQ];
  s.Eflat.clear();
  s.opdflat.clear();
  for (int i = 0; i < s.nq; ++i) {
    eoff[i] = s.sumd;
    s.sumd += p.dims[i];
    for (double e : sys->E_host[i]) s.Eflat.push_back(e);
    ooff[i] = (int)s.opdflat.size();
    const std::vector<double>& od = sys->opd_host[i];
    for (size_t k = 0; k + 1 < od.size(); k += 2) s.opdflat.push_back(make_double2(od[k], od[k + 1]));
  }
  // drives
  s.K = (int)sys->drives.size();
  if (s.K > SG_MAXDRIVE) return sg_fail(ctx, SG_E_UNSUPPORTED, "too many drives");
  s.drives.clear();
  s.amps.clear();
  s.pulse_off.clear();
  s.n_pulse = 0;
  for (const HostDrive& hd : sys->drives) {
    DriveDev dd{};
    dd.mode = hd.mode; dd.op = hd.op; dd.kind = hd.kind; dd.nseg = hd.nseg;
    double xm = 2.0 * hd.length / o->dt;
    long long mp = llround(xm);
    if (hd.kind != SG_ENV_GAUSSIAN && (mp < 1 || std::fabs(xm - (double)mp) > 1e-9 * std::max(1.0, xm)))
      return sg_fail(ctx, SG_E_INVALID, "pulse length must be a whole number of half steps");
    dd.mp = (int)mp;
    dd.amps_off = (int)s.amps.size();
    for (double v : hd.amps) s.amps.push_back(v);
    dd.amp = hd.amp; dd.sigma = hd.sigma; dd.t0 = hd.t0; dd.length = hd.length;
    dd.phase = hd.phase;
    dd.omega = hd.omega_mode >= 0 ? sys->E_host[hd.omega_mode][1] : hd.omega_d;
    s.drives.push_back(dd);
    s.pulse_off.push_back(s.n_pulse);
    s.n_pulse += hd.kind == SG_ENV_PWC ? hd.nseg : 1;
  }
  // slots
  TabArgs& ta = s.ta;
  ta = TabArgs{};
  int row = 0;
  p.n1 = 0;
  p.par1 = 0;
  s.s1_of_mode.assign(s.nq, -1);
  int ndl = 0;
  for (int i = 0; i < s.nq; ++i) {
    bool has = s.frame == SG_FRAME_LAB;
    bool par = s.frame == SG_FRAME_INTERACTION;
    for (const HostDrive& hd : sys->drives)
      if (hd.mode == i) { has = true; if (!sys->parity_odd[SG_MAXOP * i + hd.op]) par = false; }
    if (!has) continue;
    const int u = p.n1++;
    s.s1_of_mode[i] = u;
    p.s1_mode[u] = i;
    p.s1_off[u] = row;
    row += p.dims[i] * p.dims[i];
    if (par) p.par1 |= 1u << u;
    ta.drv_of_slot_start[u] = ndl;
    for (int k = 0; k < s.K; ++k)
      if (sys->drives[k].mode == i) ta.drv_list[ndl++] = k;
  }
  ta.drv_of_slot_start[p.n1] = ndl;
  p.ne = (int)sys->couplings.size();
  if (p.ne > SG_MAXEDGE) return sg_fail(ctx, SG_E_UNSUPPORTED, "too many couplings");
  p.parL = p.parR = 0;
  for (int e = 0; e < p.ne; ++e) {
    const HostCoupling& c = sys->couplings[e];
    p.e_a[e] = c.a; p.e_b[e] = c.b;
    p.e_offL[e] = row; row += p.dims[c.a] * p.dims[c.a];
    p.e_offR[e] = row; row += p.dims[c.b] * p.dims[c.b];
    if (sys->parity_odd[SG_MAXOP * c.a + c.op_a]) p.parL |= 1ull << e;
    if (sys->parity_odd[SG_MAXOP * c.b + c.op_b]) p.parR |= 1ull << e;
    ta.e_opa[e] = c.op_a; ta.e_opb[e] = c.op_b; ta.J[e] = c.J;
  }
  p.row = std::max(row, 1);
  {
    // stage rows and the cross-density scratch live in shared memory (<= 48 KB)
    const size_t nW = (size_t)p.n1 + 2 * p.ne;
    const size_t need = std::max<size_t>((size_t)p.row * sizeof(double2) + 2 * (256 / 32) * dl * dl * sizeof(double),
                                         nW * dl * dl * sizeof(double2));
    if (need > 48 * 1024) return sg_fail(ctx, SG_E_UNSUPPORTED, "too many terms for the stage kernels");
  }
  ta.p = p;
  ta.nq = s.nq; ta.K = s.K; ta.N = s.N; ta.frame = s.frame;
  for (int i = 0; i < s.nq; ++i) { ta.dims[i] = p.dims[i]; ta.eoff[i] = eoff[i]; ta.opd_off[i] = ooff[i]; }
  ta.sumd = s.sumd;
  ta.dt = o->dt;
  set_schedule(s.solver, ta);
  return SG_OK;
}

int grid_for(long long n) {
  long long g = (n + kT - 1) / kT;
  return (int)std::max<long long>(1, std::min<long long>(g, 152ll * 16));
}

template <typename R>
struct Bufs {
  typedef typename CT<R>::T C;
  C *X0 = nullptr, *X1 = nullptr, *Dacc = nullptr;
};

// Everything a solve needs on the device.
// CUDA-event brackets around the launches of every 16th step, per kernel family
// (0 forward stage passes, 1 adjoint passes, 2 recompute passes), enabled by
// SG_KTIMING=1.
struct KTimer {
  bool on = false;
  cudaStream_t st = nullptr;
  std::vector<cudaEvent_t> ev[3];
  std::vector<int> nl[3];
  long long total[3] = {0, 0, 0};
  template <typename F> void run(int k, int step, F&& f) {
    if (on && step % 16 == 0) {
      cudaEvent_t a, b;
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      cudaEventRecord(a, st);
      int n = f();
      cudaEventRecord(b, st);
      ev[k].push_back(a);
      ev[k].push_back(b);
      nl[k].push_back(n);
      total[k] += n;
    } else {
      total[k] += f();
    }
  }
  void finish(double* out) {
    for (int k = 0; k < 3; ++k) {
      double ms = 0.0, nb = 0.0;
      for (size_t i = 0; i + 1 < ev[k].size(); i += 2) {
        float x = 0.f;
        cudaEventSynchronize(ev[k][i + 1]);
        cudaEventElapsedTime(&x, ev[k][i], ev[k][i + 1]);
        ms += x;
        nb += nl[k][i / 2];
        cudaEventDestroy(ev[k][i]);
        cudaEventDestroy(ev[k][i + 1]);
      }
      ev[k].clear();
      nl[k].clear();
      out[3 * k] = ms;
      out[3 * k + 1] = nb;
      out[3 * k + 2] = (double)total[k];
    }
  }
};

struct Solve {
  KTimer kt;
  Setup s;
  Arena ar;
  DriveDev* drives_dev = nullptr;
  double* amps_dev = nullptr;
  double* E_dev = nullptr;
  double2* opd_dev = nullptr;
  double* coef = nullptr;
  double2* ph = nullptr;
  double2* tab = nullptr;
  float2* tab32 = nullptr;
  float* coef32 = nullptr;        // FP32-only tables (mixed on-chip solves): coef32, ph32, tab32
  float2* ph32 = nullptr;
  double2* psi = nullptr;
  int launches = 0;
  bool mixed = false;
  SlabPlanHost* slab = nullptr;
  OnchipPlan* oc = nullptr;
  bool want_ham = true;           // Hamiltonian-parameter gradient requested
  const void* q2rows = nullptr;   // Q2: 1-body unitaries and coupling unitaries (stage precision)
  const void* q2edges = nullptr;
  const void* q2grad = nullptr;   // Q2 pulse gradient: per step U_i(n)^dag and U_i(n)^dag L_k(n)
  // stage rows the adjoint passes apply, when they are not the forward rows (the open
  // evolution's non-Hermitian generator: rows of H_eff^dag); null: the forward rows
  const double2* adj_tab = nullptr;
  const float2* adj_tab32 = nullptr;
  double* J_dev = nullptr;        // coupling strengths (batched on-chip adjoint launches)
  // the generic gather kernels only: their cross-densities read the forward rows
  // (xa.tabrow) while the apply reads adj_tab; the tiled and on-chip adjoints contract
  // the coupling cross-densities with the rows they apply
  bool force_gather = false;
  ~Solve() {
    slab_plan_destroy(slab);
    onchip_plan_destroy(oc);
  }
  // the on-chip kernels evolve this solve (gradient solves need the adjoint to fit too)
  bool onchip(bool grad) const { return oc && (grad ? onchip_adjoint_ok(oc) : onchip_forward_ok(oc)); }
};

// Kernel family, a test knob: SG_PATH=gather forces the generic gather kernels,
// SG_PATH=slab the tiled HBM kernels; otherwise the on-chip kernels run whenever
// the columns fit in shared memory, else the tiled kernels when they handle the
// plan, else the gather kernels.
int path_choice() {
  const char* e = std::getenv("SG_PATH");
  const std::string v = e ? e : "";
  return v == "gather" ? 2 : (v == "slab" ? 1 : 0);
}

// Which part of a stored operator is its real matrix: 0 real, 1 imaginary, -1 a
// genuinely complex operator (the truncated eigenvectors are real, so n and phi are
// one or the other; a user's local operator may be neither).
int op_part(const sg_system* sys, int mode, int op) {
  const std::vector<double>& od = sys->opd_host[mode];
  const int d = sys->modes[mode].d;
  double mr = 0.0, mi = 0.0;
  for (int ab = 0; ab < d * d; ++ab) {
    const size_t k = 2 * ((size_t)op * d * d + ab);
    if (k + 1 >= od.size()) return -1;
    mr = std::max(mr, std::fabs(od[k]));
    mi = std::max(mi, std::fabs(od[k + 1]));
  }
  if (mi <= 1e-12 * mr) return 0;
  if (mr <= 1e-12 * mi) return 1;
  return -1;
}

// Every term real in the eigenbasis up to the frame phases: 1-body slots of real
// operators, couplings of two real or two imaginary factors (ta.e_zpart set).
bool real_terms(const sg_system* sys, const Setup& s, TabArgs& ta) {
  for (const HostDrive& hd : sys->drives)
    if (op_part(sys, hd.mode, hd.op) != 0) return false;
  for (int e = 0; e < s.p.ne; ++e) {
    const HostCoupling& c = sys->couplings[e];
    const int pa = op_part(sys, c.a, c.op_a), pb = op_part(sys, c.b, c.op_b);
    if (pa < 0 || pa != pb) return false;
    ta.e_zpart[e] = pa;
  }
  return true;
}

sg_status upload_and_tables(sg_system* sys, const sg_evolve_opts* o, Solve& sv, bool grad) {
  sg_ctx* ctx = sys->ctx;
  Setup& s = sv.s;
  cudaStream_t st = ctx->stream;
  // plans first: they upload their offset tables, and every host-to-device copy of
  // a solve goes before its first kernel (see dcopy)
  sv.mixed = o->precision == SG_MIXED;
  const int pc = sv.force_gather ? 2 : path_choice();
  if (pc == 0) sv.oc = onchip_plan_create(s.p, sv.mixed, s.K, s.sumd, st);
  if (pc <= 1 && !(sv.oc && onchip_adjoint_ok(sv.oc))) sv.slab = slab_plan_create(s.p, sv.mixed, st);
  // mixed precision on the on-chip kernels reads only FP32 tables
  const bool f32only = sv.mixed && sv.onchip(grad);
  sv.drives_dev = sv.ar.get<DriveDev>(std::max(1, s.K));
  sv.amps_dev = sv.ar.get<double>(std::max<size_t>(1, s.amps.size()));
  sv.E_dev = sv.ar.get<double>(s.sumd);
  sv.opd_dev = sv.ar.get<double2>(s.opdflat.size());
  const size_t nst = s.q2 ? 0 : 3ull * s.N;
  if (s.q2) {
    // Q2 reads no RK4 tables; it runs on the on-chip kernels, or beyond them on the
    // tiles of a two-pass plan
    if (!sv.oc && !(sv.slab && slab_q2_ok(sv.slab, s.p, sv.mixed)))
      return sg_fail(ctx, SG_E_UNSUPPORTED, "the Suzuki-Trotter solvers run on the on-chip kernels (every mode with "
                                            "the same level count 2..5 and D <= 4096) or on the tiles of a two-pass "
                                            "plan whose first pass holds the first couplings");
  } else if (f32only) {
    sv.coef32 = sv.ar.get<float>(nst * std::max(1, s.K));
    sv.ph32 = sv.ar.get<float2>(nst * s.sumd);
  } else {
    sv.coef = sv.ar.get<double>(nst * std::max(1, s.K));
    sv.ph = sv.ar.get<double2>(nst * s.sumd);
    sv.tab = sv.ar.get<double2>(nst * s.p.row);
  }
  if (sv.mixed && !s.q2) sv.tab32 = sv.ar.get<float2>(nst * s.p.row);
  if (!sv.drives_dev || !sv.amps_dev || !sv.E_dev || !sv.opd_dev ||
      (!s.q2 && ((sv.mixed && !sv.tab32) || (f32only ? (!sv.coef32 || !sv.ph32) : (!sv.coef || !sv.ph || !sv.tab)))))
    return sg_fail(ctx, SG_E_NOMEM, "device allocation of the stage tables failed");
  if (s.K) SG_CUDA_TRY(ctx, cudaMemcpyAsync(sv.drives_dev, s.drives.data(), s.K * sizeof(DriveDev), cudaMemcpyHostToDevice, st));
  if (!s.amps.empty()) SG_CUDA_TRY(ctx, cudaMemcpyAsync(sv.amps_dev, s.amps.data(), s.amps.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  SG_CUDA_TRY(ctx, cudaMemcpyAsync(sv.E_dev, s.Eflat.data(), s.sumd * sizeof(double), cudaMemcpyHostToDevice, st));
  SG_CUDA_TRY(ctx, cudaMemcpyAsync(sv.opd_dev, s.opdflat.data(), s.opdflat.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
  sv.J_dev = sv.ar.get<double>(std::max(1, s.p.ne));
  if (!sv.J_dev) return sg_fail(ctx, SG_E_NOMEM, "device allocation failed");
  if (s.p.ne) SG_CUDA_TRY(ctx, cudaMemcpyAsync(sv.J_dev, s.ta.J, s.p.ne * sizeof(double), cudaMemcpyHostToDevice, st));
  TabArgs ta = s.ta;
  ta.drives = sv.drives_dev;
  ta.amps = sv.amps_dev;
  ta.E = sv.E_dev;
  ta.opd = sv.opd_dev;
  ta.coef = sv.coef;
  ta.ph = sv.ph;
  ta.tab = sv.tab;
  ta.tab32 = sv.tab32;
  s.ta = ta;
  if (s.q2) {
    const int DL = sv.oc ? onchip_dl(sv.oc) : slab_dl(sv.slab);
    const long long M = (long long)s.N * ta.nsub;                  // Q2 sub-steps
    const int nset = ta.nset, ne1 = std::max(1, s.p.ne);
    const size_t D4 = (size_t)DL * DL * DL * DL;
    const size_t nrow = (size_t)(M + 1) * s.nq * DL * DL, nedge = (size_t)6 * ne1 * nset * D4;
    double2* rows = sv.ar.get<double2>(nrow);
    double2* edges = sv.ar.get<double2>(nedge);
    double2* scratch = sv.ar.get<double2>((size_t)ne1 * nset * 3 * D4);
    if (!rows || !edges || !scratch) return sg_fail(ctx, SG_E_NOMEM, "device allocation of the Q2 tables failed");
    k_q2_onebody<<<grid_for((M + 1) * s.nq), kT, 0, st>>>(ta, DL, rows);
    if (s.p.ne) k_q2_edges<<<(s.p.ne * nset + 31) / 32, 32, 0, st>>>(ta, DL, edges, scratch);
    sv.launches += 2;
    sv.q2rows = rows;
    sv.q2edges = edges;
    const size_t ngr = grad ? (size_t)M * (2 * s.nq + s.K) * DL * DL : 0;
    double2* gtab = nullptr;
    if (grad) {
      gtab = sv.ar.get<double2>(ngr);
      if (!gtab) return sg_fail(ctx, SG_E_NOMEM, "device allocation of the Q2 gradient tables failed");
      k_q2_gradtabs<<<grid_for(M * (2 * s.nq + s.K)), 64, 0, st>>>(ta, DL, gtab);
      ++sv.launches;
      sv.q2grad = gtab;
    }
    if (sv.mixed) {
      float* r32 = sv.ar.get<float>(2 * nrow);
      float* e32 = sv.ar.get<float>(2 * nedge);
      if (!r32 || !e32) return sg_fail(ctx, SG_E_NOMEM, "device allocation of the Q2 tables failed");
      onchip_to_f32(reinterpret_cast<const double*>(rows), r32, 2 * (long long)nrow, st);
      onchip_to_f32(reinterpret_cast<const double*>(edges), e32, 2 * (long long)nedge, st);
      sv.launches += 2;
      sv.q2rows = r32;
      sv.q2edges = e32;
      if (grad) {
        float* g32 = sv.ar.get<float>(2 * ngr);
        if (!g32) return sg_fail(ctx, SG_E_NOMEM, "device allocation of the Q2 gradient tables failed");
        onchip_to_f32(reinterpret_cast<const double*>(gtab), g32, 2 * (long long)ngr, st);
        ++sv.launches;
        sv.q2grad = g32;
      }
    }
  } else if (f32only) {
    k_tables32<<<(unsigned)nst, 64, 0, st>>>(ta, sv.coef32, sv.ph32);
  } else {
    k_tables<<<(unsigned)nst, 64, 0, st>>>(ta);
  }
  ++sv.launches;
  SG_CUDA_TRY(ctx, cudaGetLastError());
  // real-operator forward passes on the tiled kernels (SG_SLAB_REAL=0 keeps the
  // complex rows, a test knob)
  if (sv.slab && !s.q2 && slab_real_shape_ok(sv.slab) && real_terms(sys, s, ta)) {
    const char* e = std::getenv("SG_SLAB_REAL");
    if (!(e && e[0] == '0')) {
      const int zpar = slab_allpar(sv.slab) ? 1 : 0;
      void* zt = sv.ar.get<double>(nst * (size_t)s.p.row);      // 8-byte elements in both precisions
      if (!zt) return sg_fail(ctx, SG_E_NOMEM, "device allocation of the stage tables failed");
      if (sv.mixed) k_tables_z<float2><<<(unsigned)nst, 64, 0, st>>>(ta, (float2*)zt, zpar);
      else k_tables_z<double><<<(unsigned)nst, 64, 0, st>>>(ta, (double*)zt, zpar);
      ++sv.launches;
      // the drive operators for the pulse-gradient adjoint
      void* zo = nullptr;
      if (grad && s.K > 0) {
        zo = sv.ar.get<double>((size_t)s.K * s.p.dl * s.p.dl);
        if (!zo) return sg_fail(ctx, SG_E_NOMEM, "device allocation of the stage tables failed");
        if (sv.mixed) k_ops_z<float2><<<(unsigned)s.K, 32, 0, st>>>(ta, (float2*)zo, zpar, s.p.dl);
        else k_ops_z<double><<<(unsigned)s.K, 32, 0, st>>>(ta, (double*)zo, zpar, s.p.dl);
        ++sv.launches;
      }
      SG_CUDA_TRY(ctx, cudaGetLastError());
      slab_bind_real(sv.slab, zt, sv.ph, s.sumd, zo, ta.drv_of_slot_start, ta.drv_list);
      s.ta = ta;
    }
  }
  {
    const char* e = std::getenv("SG_KTIMING");
    sv.kt.on = e && e[0] == '1';
    sv.kt.st = st;
  }
  SG_CUDA_TRY(ctx, cudaGetLastError());
  return SG_OK;
}

template <typename R, int STAGE, bool STORE>
void launch_fwd(const Solve& sv, cudaStream_t st, const typename CT<R>::T* X, int n,
                const double2* pin, double2* pout, typename CT<R>::T* Xn,
                typename CT<R>::T* Dacc) {
  typedef typename CT<R>::T C;
  const Setup& s = sv.s;
  const int j = STAGE == 0 ? 0 : (STAGE == 3 ? 2 : 1);
  const size_t q = 3ull * n + j;
  const C* row;
  if (sizeof(R) == 4) row = reinterpret_cast<const C*>(sv.tab32 + q * s.p.row);
  else row = reinterpret_cast<const C*>(sv.tab + q * s.p.row);
  k_fwd<R, STAGE, STORE><<<grid_for(s.D * s.S), kT, s.p.row * sizeof(C), st>>>(
      s.p, X, row, pin, pout, Xn, Dacc, s.dt);
}

template <typename R, int STAGE>
void launch_adj(const Solve& sv, cudaStream_t st, const typename CT<R>::T* X, int n,
                double2* pbar, typename CT<R>::T* Xn, typename CT<R>::T* Db) {
  typedef typename CT<R>::T C;
  const Setup& s = sv.s;
  const int j = STAGE == 0 ? 0 : (STAGE == 3 ? 2 : 1);
  const size_t q = 3ull * n + j;
  const C* row;
  if (sizeof(R) == 4) row = reinterpret_cast<const C*>((sv.adj_tab32 ? sv.adj_tab32 : sv.tab32) + q * s.p.row);
  else row = reinterpret_cast<const C*>((sv.adj_tab ? sv.adj_tab : sv.tab) + q * s.p.row);
  k_adj<R, STAGE><<<grid_for(s.D * s.S), kT, s.p.row * sizeof(C), st>>>(s.p, X, row, pbar, Xn, Db, s.dt);
}

// One forward RK4 step from pin to pout (may alias).  X holds (R)psi on entry and on exit.
template <typename R>
void fwd_step(Solve& sv, cudaStream_t st, int n, const double2* pin, double2* pout,
              typename CT<R>::T*& X, typename CT<R>::T*& Xo, typename CT<R>::T* Dacc) {
  launch_fwd<R, 0, false>(sv, st, X, n, pin, nullptr, Xo, Dacc); std::swap(X, Xo);
  launch_fwd<R, 1, false>(sv, st, X, n, pin, nullptr, Xo, Dacc); std::swap(X, Xo);
  launch_fwd<R, 2, false>(sv, st, X, n, pin, nullptr, Xo, Dacc); std::swap(X, Xo);
  launch_fwd<R, 3, false>(sv, st, X, n, pin, pout, Xo, Dacc); std::swap(X, Xo);
  sv.launches += 4;
}

// Device-to-device copy as a kernel.  (A cudaMemcpyAsync waiting behind this
// stream's kernels would sit in a copy-engine queue shared with other streams and
// hold back their copies until those kernels end.)
void dcopy(double2* dst, const double2* src, long long n, cudaStream_t st) {
  k_cast<double><<<grid_for(n), kT, 0, st>>>(src, dst, n, 1.0);
}

template <typename R>
sg_status run_forward(sg_system* sys, Solve& sv, const long long* cols_dev, bool init_from_psi,
                      int ckpt_every, std::vector<double2*>* ckpts) {
  typedef typename CT<R>::T C;
  sg_ctx* ctx = sys->ctx;
  cudaStream_t st = ctx->stream;
  Setup& s = sv.s;
  const long long n = s.D * s.S;
  if (!init_from_psi) {
    k_init_cols<<<grid_for(n), kT, 0, st>>>(sv.psi, s.D, s.S, cols_dev);
    ++sv.launches;
  }
  // on-chip: the whole evolution in one launch, checkpoints as state images
  // (ckpts[c] = ckpts[0] + c * onchip_state_elems)
  if (sv.onchip(ckpts != nullptr)) {
    const void* tab = sizeof(R) == 4 ? (const void*)sv.tab32 : (const void*)sv.tab;
    sv.launches += onchip_forward(sv.oc, tab, sv.psi, nullptr, sv.psi, ckpts ? (*ckpts)[0] : nullptr,
                                  ckpt_every, 0, s.N, s.dt, nullptr, st);
    SG_CUDA_TRY(ctx, cudaGetLastError());
    return SG_OK;
  }
  C* X = sv.ar.get<C>(n);
  C* Xo = sv.ar.get<C>(n);
  C* Dacc = sv.ar.get<C>(n);
  if (!X || !Xo || !Dacc) return sg_fail(ctx, SG_E_NOMEM, "device allocation of stage buffers failed");
  if (sv.slab) {
    C* kA = sv.ar.get<C>(slab_passes(sv.slab) > 1 ? n : 1);
    double2* pint = sv.ar.get<double2>(n);
    if (!kA || !pint) return sg_fail(ctx, SG_E_NOMEM, "device allocation of stage buffers failed");
    slab_to_internal(sv.slab, sv.psi, pint, st);
    k_cast<R><<<grid_for(n), kT, 0, st>>>(pint, X, n, 1.0);
    sv.launches += 2;
    const void* tab = sizeof(R) == 4 ? (const void*)sv.tab32 : (const void*)sv.tab;
    void* Xv = X;
    void* Xov = Xo;
    for (int step = 0; step < s.N; ++step) {
      if (ckpts && step % ckpt_every == 0) dcopy((*ckpts)[step / ckpt_every], pint, n, st);
      sv.kt.run(0, step, [&] { return slab_fwd_step(sv.slab, sv.mixed, tab, step, pint, pint, Xv, Xov, Dacc, kA, s.dt, st); });
    }
    slab_from_internal(sv.slab, pint, sv.psi, st);
    ++sv.launches;
    SG_CUDA_TRY(ctx, cudaGetLastError());
    return SG_OK;
  }
  k_cast<R><<<grid_for(n), kT, 0, st>>>(sv.psi, X, n, 1.0);
  ++sv.launches;
  for (int step = 0; step < s.N; ++step) {
    if (ckpts && step % ckpt_every == 0) dcopy((*ckpts)[step / ckpt_every], sv.psi, n, st);
    fwd_step<R>(sv, st, step, sv.psi, sv.psi, X, Xo, Dacc);
  }
  SG_CUDA_TRY(ctx, cudaGetLastError());
  return SG_OK;
}

FrameArgs frame_args(const Setup& s, const double* E_dev, double sign) {
  FrameArgs f{};
  f.nq = s.nq; f.S = s.S; f.D = s.D;
  for (int i = 0; i < s.nq; ++i) { f.dims[i] = s.p.dims[i]; f.st[i] = s.p.st[i]; f.eoff[i] = s.ta.eoff[i]; }
  f.E = E_dev;
  f.T = s.T;
  f.sign = sign;
  return f;
}

CompArgs comp_args(const Setup& s) {
  CompArgs c{};
  c.nq = s.nq; c.S = s.S; c.Dc = s.Dc;
  for (int i = 0; i < s.nq; ++i) { c.dims[i] = s.p.dims[i]; c.qpos[i] = s.qpos[i]; }
  return c;
}

// Constant part of the cross-density contraction arguments of a solve.
XArgs make_xargs(const Solve& sv, GradAcc acc) {
  const Setup& s = sv.s;
  XArgs xa{};
  xa.p = s.p;
  xa.K = s.K;
  xa.nW = s.p.n1 + 2 * s.p.ne;
  xa.frame = s.ta.frame;
  xa.opd = sv.opd_dev;
  for (int i = 0; i < s.nq; ++i) { xa.opd_off[i] = s.ta.opd_off[i]; xa.eoff[i] = s.ta.eoff[i]; }
  xa.E = sv.E_dev;
  for (int i = 0; i <= s.p.n1; ++i) xa.drv_of_slot_start[i] = s.ta.drv_of_slot_start[i];
  for (int i = 0; i < SG_MAXDRIVE; ++i) xa.drv_list[i] = s.ta.drv_list[i];
  for (int k = 0; k < s.K; ++k) xa.drv_op[k] = s.drives[k].op;
  for (int e = 0; e < s.p.ne; ++e) { xa.e_opa[e] = s.ta.e_opa[e]; xa.e_opb[e] = s.ta.e_opb[e]; xa.J[e] = s.ta.J[e]; }
  xa.acc = acc;
  xa.ham = sv.want_ham ? 1 : 0;
  xa.Jdev = sv.J_dev;
  return xa;
}

// Adjoint on the on-chip kernels: per checkpoint segment one recompute launch that
// stores every stage input, one adjoint launch; per-CTA accumulators summed at the end.
template <typename R>
sg_status run_backward_onchip(sg_system* sys, Solve& sv, std::vector<double2*>& ckpts, int K,
                              double2* pbar, GradAcc acc) {
  typedef typename CT<R>::T C;
  sg_ctx* ctx = sys->ctx;
  cudaStream_t st = ctx->stream;
  Setup& s = sv.s;
  const OnchipPlan* oc = sv.oc;
  const XArgs xa = make_xargs(sv, acc);
  const long long ns = onchip_state_elems(oc);
  const long long nstage = onchip_stage_elems(oc);
  const int ncta = onchip_ctas(oc);
  const long long nst = 3ll * s.N;
  const int Kd = std::max(1, s.K);
  double2* pimg = sv.ar.get<double2>(ns);
  C* segY = sv.ar.get<C>((size_t)4 * K * nstage);
  double* gFc = sv.ar.get<double>((size_t)ncta * nst * Kd);
  double* accc = sv.ar.get<double>((size_t)ncta * onchip_acc_doubles(oc));
  int* err = sv.ar.get<int>(1);
  void* colow = onchip_colow_global(oc) ? (void*)sv.ar.get<float2>(ns) : nullptr;
  if (!pimg || !segY || !gFc || !accc || !err || (onchip_colow_global(oc) && !colow))
    return sg_fail(ctx, SG_E_NOMEM, "device allocation of the on-chip adjoint buffers failed");
  SG_CUDA_TRY(ctx, cudaMemsetAsync(gFc, 0, (size_t)ncta * nst * Kd * sizeof(double), st));
  SG_CUDA_TRY(ctx, cudaMemsetAsync(accc, 0, (size_t)ncta * onchip_acc_doubles(oc) * sizeof(double), st));
  SG_CUDA_TRY(ctx, cudaMemsetAsync(err, 0, sizeof(int), st));
  onchip_to_image(oc, pbar, pimg, st);
  ++sv.launches;
  const void* tab = sizeof(R) == 4 ? (const void*)sv.tab32 : (const void*)sv.tab;
  const void* atab = sizeof(R) == 4 ? (sv.adj_tab32 ? (const void*)sv.adj_tab32 : tab)
                                    : (sv.adj_tab ? (const void*)sv.adj_tab : tab);
  OnchipTables tb{atab, sv.coef, sv.ph, sv.opd_dev};
  if (sizeof(R) == 4) {
    // FP32 tables (k_tables32) and an FP32 copy of the operators
    const long long nop = 2 * (long long)s.opdflat.size();
    float* op32 = sv.ar.get<float>(nop);
    if (!op32 || !sv.coef32 || !sv.ph32) return sg_fail(ctx, SG_E_NOMEM, "FP32 tables missing");
    onchip_to_f32(reinterpret_cast<const double*>(sv.opd_dev), op32, nop, st);
    ++sv.launches;
    tb = OnchipTables{atab, sv.coef32, sv.ph32, op32};
  }
  const int nseg = (int)ckpts.size();
  for (int c = nseg - 1; c >= 0; --c) {
    const int n0 = c * K, n1 = std::min(s.N, n0 + K);
    sv.launches += onchip_forward(oc, tab, nullptr, ckpts[c], nullptr, nullptr, K, n0, n1, s.dt, segY, st);
    sv.launches += onchip_adjoint(oc, tb, segY, pimg, n0, n1, s.dt, xa, (int)nst, gFc, accc, err, colow, st);
  }
  onchip_batcher_release();                       // the solve's last on-chip launch is issued
  onchip_reduce(oc, gFc, accc, nst, s.K, s.p.n1, s.p.ne, acc, st);
  ++sv.launches;
  SG_CUDA_TRY(ctx, cudaGetLastError());
  int herr = 0;
  SG_CUDA_TRY(ctx, cudaStreamSynchronize(st));     // reads only from an idle stream (see dcopy)
  SG_CUDA_TRY(ctx, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  SG_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  if (herr) return sg_fail(ctx, SG_E_TIMEOUT, "on-chip adjoint: a bounded wait for a stage input's bulk copy ran out");
  return SG_OK;
}

template <typename R>
sg_status run_backward(sg_system* sys, Solve& sv, std::vector<double2*>& ckpts, int K,
                       double2* pbar, GradAcc acc) {
  typedef typename CT<R>::T C;
  sg_ctx* ctx = sys->ctx;
  cudaStream_t st = ctx->stream;
  Setup& s = sv.s;
  const long long n = s.D * s.S;
  if (sv.onchip(true)) return run_backward_onchip<R>(sys, sv, ckpts, K, pbar, acc);
  const bool slab = sv.slab != nullptr;
  // buffers of the gather path only (the slab path keeps a segment store instead)
  C* X = slab ? nullptr : sv.ar.get<C>(n);
  C* Xo = slab ? nullptr : sv.ar.get<C>(n);
  C* Dacc = sv.ar.get<C>(n);
  C* Y[4] = {nullptr, nullptr, nullptr, nullptr};
  if (!slab) for (int i = 0; i < 4; ++i) Y[i] = sv.ar.get<C>(n);
  C* KB = sv.ar.get<C>(n);
  C* KB2 = sv.ar.get<C>(n);
  C* Db = sv.ar.get<C>(n);
  std::vector<double2*> seg(slab ? 0 : K + 1);
  for (auto& b : seg) b = sv.ar.get<double2>(n);
  const int nW = s.p.n1 + 2 * s.p.ne;
  const int DL = s.p.dl;
  const int xgrid = (int)std::max<long long>(1, std::min<long long>((n / 2 + kT - 1) / kT, 152ll * 2));
  double2* partial = slab ? nullptr : sv.ar.get<double2>((size_t)xgrid * std::max(1, nW) * DL * DL);
  unsigned* ticket = sv.ar.get<unsigned>(1);
  for (C* c : {Dacc, KB, KB2, Db})
    if (!c) return sg_fail(ctx, SG_E_NOMEM, "device allocation of adjoint buffers failed");
  if (!slab) {
    for (C* c : {X, Xo, Y[0], Y[1], Y[2], Y[3]})
      if (!c) return sg_fail(ctx, SG_E_NOMEM, "device allocation of adjoint buffers failed");
    for (double2* c : seg) if (!c) return sg_fail(ctx, SG_E_NOMEM, "device allocation of the segment buffer failed");
    if (!partial) return sg_fail(ctx, SG_E_NOMEM, "device allocation failed");
  }
  if (!ticket) return sg_fail(ctx, SG_E_NOMEM, "device allocation failed");
  SG_CUDA_TRY(ctx, cudaMemsetAsync(ticket, 0, sizeof(unsigned), st));
  XArgs xa = make_xargs(sv, acc);
  xa.partial = partial;
  xa.ticket = ticket;
  const size_t xsm = std::max<size_t>(2 * (kT / 32) * DL * DL * sizeof(double) + s.p.row * sizeof(C),
                                      (size_t)std::max(1, nW) * DL * DL * sizeof(double2));
  auto xdens = [&](const C* Xk, const C* Yk, int step, int j) {
    xa.q = 3 * step + j;
    xa.t = (double)(2 * step + j) * s.dt * 0.5;
    xa.tabrow = sv.tab + (size_t)xa.q * s.p.row;
    xa.coef = sv.coef + (size_t)xa.q * s.K;
    xa.ph = sv.ph + (size_t)xa.q * s.sumd;
    switch (DL) {
      case 2: k_xdens<R, 2><<<xgrid, kT, xsm, st>>>(xa, Xk, Yk); break;
      case 3: k_xdens<R, 3><<<xgrid, kT, xsm, st>>>(xa, Xk, Yk); break;
      case 4: k_xdens<R, 4><<<xgrid, kT, xsm, st>>>(xa, Xk, Yk); break;
      case 5: k_xdens<R, 5><<<xgrid, kT, xsm, st>>>(xa, Xk, Yk); break;
      case 6: k_xdens<R, 6><<<xgrid, kT, xsm, st>>>(xa, Xk, Yk); break;
      case 7: k_xdens<R, 7><<<xgrid, kT, xsm, st>>>(xa, Xk, Yk); break;
      default: k_xdens<R, 8><<<xgrid, kT, xsm, st>>>(xa, Xk, Yk); break;
    }
    ++sv.launches;
  };
  if (sv.slab) {
    // segment store: every stage input y1..y4 of every step of one segment, so the
    // adjoint needs no in-step recompute; one working psi
    C* kA = sv.ar.get<C>(slab_passes(sv.slab) > 1 ? n : 1);
    C* yA = sv.ar.get<C>(slab_passes(sv.slab) > 1 ? n : 1);
    double2* pint = sv.ar.get<double2>(n);
    double2* spart = sv.ar.get<double2>(slab_partial_elems(sv.slab));
    double2* pwork = sv.ar.get<double2>(n);
    if (!kA || !yA || !pint || !spart || !pwork) return sg_fail(ctx, SG_E_NOMEM, "device allocation of adjoint buffers failed");
    std::vector<C*> segY(4 * (size_t)K + 1);
    for (auto& b : segY) {
      b = sv.ar.get<C>(n);
      if (!b) return sg_fail(ctx, SG_E_NOMEM, "device allocation of the segment store failed");
    }
    xa.partial = spart;
    slab_to_internal(sv.slab, pbar, pint, st);
    k_cast<R><<<grid_for(n), kT, 0, st>>>(pint, KB, n, s.dt / 6.0);
    sv.launches += 2;
    const void* tab = sizeof(R) == 4 ? (const void*)sv.tab32 : (const void*)sv.tab;
    const void* atab = sizeof(R) == 4 ? (sv.adj_tab32 ? (const void*)sv.adj_tab32 : tab)
                                      : (sv.adj_tab ? (const void*)sv.adj_tab : tab);
    void* KBv = KB;
    void* KB2v = KB2;
    const int nseg = (int)ckpts.size();
    for (int c = nseg - 1; c >= 0; --c) {
      const int n0 = c * K, n1 = std::min(s.N, n0 + K);
      dcopy(pwork, ckpts[c], n, st);
      k_cast<R><<<grid_for(n), kT, 0, st>>>(pwork, segY[0], n, 1.0);
      ++sv.launches;
      for (int step = n0; step < n1; ++step) {
        void* Yk[4] = {segY[4 * (step - n0)], segY[4 * (step - n0) + 1], segY[4 * (step - n0) + 2],
                       segY[4 * (step - n0) + 3]};
        if (step < n1 - 1)
          sv.kt.run(0, step, [&] {
            return slab_fwd_step_keep(sv.slab, sv.mixed, tab, step, pwork, pwork, Yk, segY[4 * (step - n0 + 1)],
                                      Dacc, kA, s.dt, st);
          });
        else
          sv.kt.run(2, step, [&] { return slab_fwd_store(sv.slab, sv.mixed, tab, step, pwork, Yk, kA, s.dt, st); });
      }
      for (int step = n1 - 1; step >= n0; --step) {
        void* Yv[4] = {segY[4 * (step - n0)], segY[4 * (step - n0) + 1], segY[4 * (step - n0) + 2],
                       segY[4 * (step - n0) + 3]};
        sv.kt.run(1, step, [&] {
          return slab_adj_step(sv.slab, sv.mixed, atab, step, Yv, pint, KBv, KB2v, Db, yA, s.dt, xa, sv.tab,
                               sv.coef, sv.ph, s.sumd, s.K, st);
        });
      }
      SG_CUDA_TRY(ctx, cudaGetLastError());
    }
    return SG_OK;
  }
  // kbar_4 of the last step = dt/6 psibar_N
  k_cast<R><<<grid_for(n), kT, 0, st>>>(pbar, KB, n, s.dt / 6.0);
  ++sv.launches;
  const int nseg = (int)ckpts.size();
  for (int c = nseg - 1; c >= 0; --c) {
    const int n0 = c * K, n1 = std::min(s.N, n0 + K);
    dcopy(seg[0], ckpts[c], n, st);
    k_cast<R><<<grid_for(n), kT, 0, st>>>(seg[0], X, n, 1.0);
    ++sv.launches;
    for (int step = n0; step < n1 - 1; ++step)
      fwd_step<R>(sv, st, step, seg[step - n0], seg[step - n0 + 1], X, Xo, Dacc);
    for (int step = n1 - 1; step >= n0; --step) {
      const double2* ps = seg[step - n0];
      k_cast<R><<<grid_for(n), kT, 0, st>>>(ps, Y[0], n, 1.0);
      launch_fwd<R, 0, true>(sv, st, Y[0], step, ps, nullptr, Y[1], nullptr);
      launch_fwd<R, 1, true>(sv, st, Y[1], step, ps, nullptr, Y[2], nullptr);
      launch_fwd<R, 2, true>(sv, st, Y[2], step, ps, nullptr, Y[3], nullptr);
      sv.launches += 4;
      xdens(KB, Y[3], step, 2);
      launch_adj<R, 3>(sv, st, KB, step, pbar, KB2, Db);
      xdens(KB2, Y[2], step, 1);
      launch_adj<R, 2>(sv, st, KB2, step, pbar, KB, Db);
      xdens(KB, Y[1], step, 1);
      launch_adj<R, 1>(sv, st, KB, step, pbar, KB2, Db);
      xdens(KB2, Y[0], step, 0);
      launch_adj<R, 0>(sv, st, KB2, step, pbar, KB, Db);
      sv.launches += 4;
    }
    SG_CUDA_TRY(ctx, cudaGetLastError());
  }
  return SG_OK;
}

}  // namespace

// Q2 evolution (on-chip) of the solve's columns, lab frame, in place in sv.psi.
sg_status run_q2(sg_system* sys, Solve& sv, const long long* cols_dev, bool init_from_psi) {
  sg_ctx* ctx = sys->ctx;
  cudaStream_t st = ctx->stream;
  Setup& s = sv.s;
  if (!init_from_psi) {
    k_init_cols<<<grid_for(s.D * s.S), kT, 0, st>>>(sv.psi, s.D, s.S, cols_dev);
    ++sv.launches;
  }
  if (!sv.oc) {
    // tiled: the internal layout in the stage precision, evolved in place
    const long long n = s.D * s.S;
    double2* pint = sv.ar.get<double2>(n);
    float2* X32 = sv.mixed ? sv.ar.get<float2>(n) : nullptr;
    if (!pint || (sv.mixed && !X32)) return sg_fail(ctx, SG_E_NOMEM, "device allocation of the state failed");
    slab_to_internal(sv.slab, sv.psi, pint, st);
    void* X = pint;
    if (sv.mixed) {
      k_cast<float><<<grid_for(n), kT, 0, st>>>(pint, X32, n, 1.0);
      X = X32;
    }
    sv.launches += slab_q2_run(sv.slab, sv.mixed, sv.q2rows, sv.q2edges, X, s.N * s.ta.nsub, s.ta.nsub,
                               s.ta.set_of, s.ta.q1 != 0, st);
    if (sv.mixed) k_widen<<<grid_for(n), kT, 0, st>>>(X32, pint, n);
    slab_from_internal(sv.slab, pint, sv.psi, st);
    sv.launches += sv.mixed ? 4 : 2;
    SG_CUDA_TRY(ctx, cudaGetLastError());
    return SG_OK;
  }
  sg_status rc = onchip_q2_forward(sv.oc, s.p, sv.q2rows, sv.q2edges, sv.psi, sv.psi, s.N * s.ta.nsub, s.ta.nsub,
                                   s.ta.set_of, s.ta.nset, st, &sv.launches, s.ta.q1 != 0);
  if (rc != SG_OK) return sg_fail(ctx, rc, "the Suzuki-Trotter solvers support at most 16 modes and 32 couplings");
  SG_CUDA_TRY(ctx, cudaGetLastError());
  return SG_OK;
}

// Q2 pulse gradient: the co-state pbar of the final lab-frame columns in sv.psi is
// pulled back through every factor with the state (Sec. 2.5 applied to the product
// of unitaries of Sec. 2.3); dF/df_k(n) lands at stage slot 3n + 1 of acc.gF.
sg_status run_backward_q2(sg_system* sys, Solve& sv, double2* pbar, GradAcc acc) {
  sg_ctx* ctx = sys->ctx;
  cudaStream_t st = ctx->stream;
  Setup& s = sv.s;
  if (!sv.oc) {
    // tiled: the final states and co-states in the internal layout and stage precision,
    // pulled back pass by pass
    const long long n = s.D * s.S;
    double2* pi = sv.ar.get<double2>(n);
    double2* li = sv.ar.get<double2>(n);
    float2* X32 = sv.mixed ? sv.ar.get<float2>(n) : nullptr;
    float2* L32 = sv.mixed ? sv.ar.get<float2>(n) : nullptr;
    double* gpart = sv.ar.get<double>(slab_q2_grad_part(sv.slab));
    unsigned* ticket = sv.ar.get<unsigned>(1);
    if (!pi || !li || (sv.mixed && (!X32 || !L32)) || !gpart || !ticket)
      return sg_fail(ctx, SG_E_NOMEM, "device allocation of the Q2 adjoint buffers failed");
    SG_CUDA_TRY(ctx, cudaMemsetAsync(ticket, 0, sizeof(unsigned), st));
    slab_to_internal(sv.slab, sv.psi, pi, st);
    slab_to_internal(sv.slab, pbar, li, st);
    sv.launches += 2;
    void* X = pi;
    void* L = li;
    if (sv.mixed) {
      k_cast<float><<<grid_for(n), kT, 0, st>>>(pi, X32, n, 1.0);
      k_cast<float><<<grid_for(n), kT, 0, st>>>(li, L32, n, 1.0);
      sv.launches += 2;
      X = X32;
      L = L32;
    }
    int drv_mode[SG_MAXDRIVE];
    for (int k = 0; k < s.K; ++k) drv_mode[k] = s.drives[k].mode;
    const size_t es = sv.mixed ? sizeof(float2) : sizeof(double2);
    const int DL = slab_dl(sv.slab);
    const void* edges_pb = static_cast<const char*>(sv.q2edges) +
                           (size_t)2 * std::max(1, s.p.ne) * s.ta.nset * DL * DL * DL * DL * es;
    const int nl = slab_q2_grad_run(sv.slab, sv.mixed, sv.q2grad, edges_pb, X, L, s.N * s.ta.nsub, s.ta.nsub,
                                    s.ta.set_of, s.ta.q1 != 0, s.K, drv_mode, acc.gF, gpart, ticket, st);
    if (nl < 0) return sg_fail(ctx, SG_E_UNSUPPORTED, "a drive's mode has no 1-body factor in the tiled plan");
    sv.launches += nl;
    SG_CUDA_TRY(ctx, cudaGetLastError());
    return SG_OK;
  }
  const int ncta = onchip_ctas(sv.oc);
  const long long nst = 3ll * s.N;
  const int Kd = std::max(1, s.K);
  double* gFc = sv.ar.get<double>((size_t)ncta * nst * Kd);
  if (!gFc) return sg_fail(ctx, SG_E_NOMEM, "device allocation of the Q2 adjoint buffers failed");
  SG_CUDA_TRY(ctx, cudaMemsetAsync(gFc, 0, (size_t)ncta * nst * Kd * sizeof(double), st));
  int drv_mode[SG_MAXDRIVE];
  for (int k = 0; k < s.K; ++k) drv_mode[k] = s.drives[k].mode;
  // the adjoint coupling unitaries follow the forward ones (2 ne nset matrices)
  const size_t es = sv.mixed ? sizeof(float2) : sizeof(double2);
  const int DL = onchip_dl(sv.oc);
  const void* adj_edges = static_cast<const char*>(sv.q2edges) +
                          (size_t)2 * std::max(1, s.p.ne) * s.ta.nset * DL * DL * DL * DL * es;
  sg_status rc = onchip_q2_pulse_adjoint(sv.oc, s.p, drv_mode, s.K, sv.q2grad, adj_edges, sv.psi, pbar,
                                         s.N * s.ta.nsub, s.ta.nsub, s.ta.set_of, s.ta.nset, nst * Kd, gFc, st,
                                         &sv.launches, s.ta.q1 != 0);
  if (rc != SG_OK)
    return sg_fail(ctx, rc, "the Q2 gradient needs 2..16 modes, <= 32 couplings, <= 16 drives and its buffers "
                            "in shared memory");
  onchip_reduce(sv.oc, gFc, nullptr, nst, s.K, s.p.n1, s.p.ne, acc, st);
  ++sv.launches;
  SG_CUDA_TRY(ctx, cudaGetLastError());
  return SG_OK;
}

// ---------------------------------------------------------------------------
// entry points used by the C ABI
// ---------------------------------------------------------------------------
sg_status sg_evolve_impl(sg_system* sys, const sg_evolve_opts* o, void* psi_dev) {
  sg_ctx* ctx = sys->ctx;
  if (!sys->prepared) return sg_fail(ctx, SG_E_STATE, "system is not prepared (call sg_prepare)");
  if (!psi_dev) return sg_fail(ctx, SG_E_INVALID, "psi_dev is NULL");
  Solve sv;
  sv.ar.st = ctx->stream;
  sg_status rc = build_setup(sys, o, sv.s);
  if (rc != SG_OK) return rc;
  SG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  keep_pool_memory(ctx->device);
  cudaStream_t st = ctx->stream;
  Setup& s = sv.s;
  long long* cols_dev = nullptr;
  if (o->col_index) {
    for (int c = 0; c < s.S; ++c)
      if (o->col_index[c] < 0 || o->col_index[c] >= s.D) return sg_fail(ctx, SG_E_INVALID, "col_index out of range");
    cols_dev = sv.ar.get<long long>(s.S);
    if (!cols_dev) return sg_fail(ctx, SG_E_NOMEM, "allocation failed");
    SG_CUDA_TRY(ctx, cudaMemcpyAsync(cols_dev, o->col_index, s.S * sizeof(long long), cudaMemcpyHostToDevice, st));
  }
  rc = upload_and_tables(sys, o, sv, false);
  if (rc != SG_OK) return rc;
  sv.psi = static_cast<double2*>(psi_dev);
  if (s.q2) rc = run_q2(sys, sv, cols_dev, !o->col_index);
  else rc = o->precision == SG_MIXED ? run_forward<float>(sys, sv, cols_dev, !o->col_index, 0, nullptr)
                                     : run_forward<double>(sys, sv, cols_dev, !o->col_index, 0, nullptr);
  if (rc != SG_OK) return rc;
  if (s.frame == SG_FRAME_INTERACTION) {
    k_frame<<<grid_for(s.D * s.S), kT, 0, st>>>(frame_args(s, sv.E_dev, -1.0), sv.psi);
    SG_CUDA_TRY(ctx, cudaGetLastError());
  }
  SG_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  sv.kt.finish(sys->ktimes);
  sv.launches += (int)(sv.kt.total[0] + sv.kt.total[1] + sv.kt.total[2]);
  sys->last_stats[4] = sv.launches;
  return SG_OK;
}

sg_status sg_fidelity_impl(sg_system* sys, const sg_evolve_opts* o, const double* target, int kind,
                           double* F_out, double* Ucomp_out, bool grad, double* grad_pulse,
                           double* grad_ham, int ckpt, sg_allreduce_fn red, void* red_user) {
  sg_ctx* ctx = sys->ctx;
  const bool shard = red != nullptr;    // this call evolves one shard of the columns
  if (!sys->prepared) return sg_fail(ctx, SG_E_STATE, "system is not prepared (call sg_prepare)");
  if (!target) return sg_fail(ctx, SG_E_INVALID, "target is NULL");
  if (!o || !o->col_index) return sg_fail(ctx, SG_E_INVALID, "fidelity needs opts->col_index");
  if (kind != SG_FID_AVG && kind != SG_FID_STATE) return sg_fail(ctx, SG_E_INVALID, "bad fidelity kind");
  Solve sv;
  sv.ar.st = ctx->stream;
  sv.want_ham = grad_ham != nullptr;     // no Hamiltonian gradient: skip the coupling slots
  sg_status rc = build_setup(sys, o, sv.s);
  if (rc != SG_OK) return rc;
  Setup& s = sv.s;
  if (s.nqb < 1 || s.nqb > 12) return sg_fail(ctx, SG_E_UNSUPPORTED, "fidelity needs 1..12 qubit (non-coupler) modes");
  if (s.q2 && grad && grad_ham)
    return sg_fail(ctx, SG_E_UNSUPPORTED, "the Suzuki-Trotter solvers compute the pulse-parameter gradient only "
                                          "(grad_ham = NULL)");
  for (int i = 0; i < s.nq; ++i)
    if (s.qpos[i] >= 0 && s.p.dims[i] < 2)
      return sg_fail(ctx, SG_E_INVALID, "computational states need >= 2 levels per qubit mode");
  SG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  keep_pool_memory(ctx->device);
  cudaStream_t st = ctx->stream;
  // comp labels of the columns
  std::vector<int> lab(s.S, -1);
  std::vector<int> seen(s.Dc, 0);
  int Sc = 0;
  for (int c = 0; c < s.S; ++c) {
    long long r = o->col_index[c];
    if (r < 0 || r >= s.D) return sg_fail(ctx, SG_E_INVALID, "col_index out of range");
    int j = 0;
    bool comp = true;
    for (int i = 0; i < s.nq; ++i) {
      int l = (int)((r / s.p.st[i]) % s.p.dims[i]);
      if (l > (s.qpos[i] >= 0 ? 1 : 0)) { comp = false; break; }     // couplers in level 0
      if (s.qpos[i] >= 0) j = (j << 1) | l;
    }
    if (comp) { lab[c] = j; ++Sc; ++seen[j]; }
  }
  if (Sc == 0) return sg_fail(ctx, SG_E_INVALID, "no evolved column is a computational state");
  bool full = true;
  for (int j = 0; j < s.Dc; ++j) if (seen[j] != 1) full = false;
  if (full && s.Dc > 256) full = false;
  if (shard) {
    for (int j = 0; j < s.Dc; ++j)
      if (seen[j] > 1) return sg_fail(ctx, SG_E_INVALID, "a computational state is evolved twice in this shard");
    if (o->compensation != SG_COMP_NONE || o->basis != SG_BASIS_PRODUCT)
      return sg_fail(ctx, SG_E_UNSUPPORTED, "a sharded solve takes the product basis without compensation");
    if (kind == SG_FID_AVG && s.Dc > 256)
      return sg_fail(ctx, SG_E_INVALID, "F_avg needs Dc <= 256");
    full = false;
  } else if (grad && kind == SG_FID_AVG && !full) {
    return sg_fail(ctx, SG_E_INVALID, "F_avg needs every computational state evolved exactly once (Dc <= 256)");
  }
  if (o->compensation != SG_COMP_NONE && o->compensation != SG_COMP_VZ)
    return sg_fail(ctx, SG_E_INVALID, "compensation must be SG_COMP_NONE or SG_COMP_VZ");
  const bool vz = o->compensation == SG_COMP_VZ;
  if (vz && (!full || s.nqb > 8))
    return sg_fail(ctx, SG_E_INVALID, "virtual-Z compensation needs every computational state evolved exactly once "
                                      "(Dc <= 256)");
  if (o->basis != SG_BASIS_PRODUCT && o->basis != SG_BASIS_DRESSED)
    return sg_fail(ctx, SG_E_INVALID, "basis must be SG_BASIS_PRODUCT or SG_BASIS_DRESSED");
  const bool dressed = o->basis == SG_BASIS_DRESSED;
  if (dressed && (s.D > kMaxDressedLarge || !full || Sc != s.S))
    return sg_fail(ctx, SG_E_INVALID, "the dressed basis needs D <= 1024 and the evolved columns to be the "
                                      "computational states, each once");
  if (dressed && grad && grad_ham)
    return sg_fail(ctx, SG_E_UNSUPPORTED, "the dressed basis computes the pulse-parameter gradient only "
                                          "(grad_ham = NULL)");
  auto t0 = std::chrono::steady_clock::now();
  long long* cols_dev = sv.ar.get<long long>(s.S);
  int* lab_dev = sv.ar.get<int>(s.S);
  double2* Tg = sv.ar.get<double2>((size_t)s.Dc * s.Dc);
  double2* Uc = sv.ar.get<double2>((size_t)s.Dc * s.S);
  double2* barc = sv.ar.get<double2>((size_t)s.Dc * s.S);
  double2* Mbuf = sv.ar.get<double2>(shard ? (size_t)s.Dc * s.S : (full ? (size_t)s.Dc * s.Dc : 1));
  double* Fd = sv.ar.get<double>(2);
  const long long n = s.D * s.S;
  sv.psi = sv.ar.get<double2>(n);
  if (!cols_dev || !lab_dev || !Tg || !Uc || !barc || !Mbuf || !Fd || !sv.psi)
    return sg_fail(ctx, SG_E_NOMEM, "device allocation failed");
  SG_CUDA_TRY(ctx, cudaMemcpyAsync(cols_dev, o->col_index, s.S * sizeof(long long), cudaMemcpyHostToDevice, st));
  SG_CUDA_TRY(ctx, cudaMemcpyAsync(lab_dev, lab.data(), s.S * sizeof(int), cudaMemcpyHostToDevice, st));
  SG_CUDA_TRY(ctx, cudaMemcpyAsync(Tg, target, (size_t)s.Dc * s.Dc * sizeof(double2), cudaMemcpyHostToDevice, st));
  int* poff = nullptr;
  if (grad) {
    poff = sv.ar.get<int>(std::max(1, s.K));
    if (!poff) return sg_fail(ctx, SG_E_NOMEM, "device allocation failed");
    if (s.K) SG_CUDA_TRY(ctx, cudaMemcpyAsync(poff, s.pulse_off.data(), s.K * sizeof(int), cudaMemcpyHostToDevice, st));
  }
  rc = upload_and_tables(sys, o, sv, grad);
  if (rc != SG_OK) return rc;
  if (grad && s.q2 && !sv.oc && (!slab_q2_grad_ok(sv.slab) || s.K > 16))
    return sg_fail(ctx, SG_E_UNSUPPORTED, "the Suzuki-Trotter gradient on the tiled kernels needs <= 16 drives "
                                          "and its pull-back lists in shared memory");
  double2* Vc = nullptr;
  if (dressed) {
    // dressed computational states of the idle Hamiltonian (FP64 Jacobi)
    DressArgs da{};
    da.D = (int)s.D; da.nq = s.nq; da.ne = s.p.ne; da.Dc = s.Dc;
    for (int i = 0; i < s.nq; ++i) {
      da.dims[i] = s.p.dims[i]; da.st[i] = s.p.st[i]; da.eoff[i] = s.ta.eoff[i]; da.opd_off[i] = s.ta.opd_off[i];
    }
    for (int e = 0; e < s.p.ne; ++e) {
      da.e_a[e] = s.p.e_a[e]; da.e_b[e] = s.p.e_b[e];
      da.e_opa[e] = s.ta.e_opa[e]; da.e_opb[e] = s.ta.e_opb[e]; da.J[e] = s.ta.J[e];
    }
    std::vector<long long> comp(s.Dc);
    for (int j = 0; j < s.Dc; ++j) {
      long long r = 0;
      for (int i = 0; i < s.nq; ++i) r += (long long)(s.qpos[i] >= 0 ? (j >> s.qpos[i]) & 1 : 0) * s.p.st[i];
      comp[j] = r;
    }
    long long* comp_dev = sv.ar.get<long long>(s.Dc);
    int* derr = sv.ar.get<int>(1);
    Vc = sv.ar.get<double2>((size_t)s.D * s.Dc);
    da.work = sv.ar.get<double>(dressed_work_doubles((int)s.D));
    if (!comp_dev || !derr || !Vc || !da.work) return sg_fail(ctx, SG_E_NOMEM, "device allocation failed");
    SG_CUDA_TRY(ctx, cudaMemcpyAsync(comp_dev, comp.data(), s.Dc * sizeof(long long), cudaMemcpyHostToDevice, st));
    da.E = sv.E_dev; da.opd = sv.opd_dev; da.comp = comp_dev; da.Vc = Vc; da.err = derr;
    SG_CUDA_TRY(ctx, launch_dressed(da, st, &sv.launches));
    int herr = 0;
    SG_CUDA_TRY(ctx, cudaStreamSynchronize(st));     // reads only from an idle stream (see dcopy)
    SG_CUDA_TRY(ctx, cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, st));
    SG_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    if (herr == 1) return sg_fail(ctx, SG_E_UNSUPPORTED, "the dressed basis needs a real idle Hamiltonian");
    if (herr == 2) return sg_fail(ctx, SG_E_INVALID, "two computational states share a dressed state");
    if (herr == 3) return sg_fail(ctx, SG_E_INVALID, "a dressed computational level is degenerate");
  }
  // checkpoints
  int K = 0;
  std::vector<double2*> ckpts;
  if (grad && !s.q2) {             // the Q2 adjoint recomputes the states by inverse factors
    K = ckpt > 0 ? ckpt : std::max(1, (int)std::lround(std::sqrt((double)s.N)));
    K = std::min(K, s.N);
    const int nck = (s.N + K - 1) / K;
    if (sv.onchip(true)) {
      // one block of state images, ckpts[c] = ckpts[0] + c * image size
      const long long ns = onchip_state_elems(sv.oc);
      double2* p = sv.ar.get<double2>((size_t)nck * ns);
      if (!p) return sg_fail(ctx, SG_E_NOMEM, "device allocation of checkpoints failed");
      for (int c = 0; c < nck; ++c) ckpts.push_back(p + (size_t)c * ns);
    } else {
      for (int c = 0; c < nck; ++c) {
        double2* p = sv.ar.get<double2>(n);
        if (!p) return sg_fail(ctx, SG_E_NOMEM, "device allocation of checkpoints failed");
        ckpts.push_back(p);
      }
    }
  }
  cudaEvent_t ev0, ev1, ev2;
  cudaEventCreate(&ev0); cudaEventCreate(&ev1); cudaEventCreate(&ev2);
  cudaEventRecord(ev0, st);
  if (dressed) {
    k_init_dressed<<<grid_for(n), kT, 0, st>>>(Vc, lab_dev, s.D, s.S, s.Dc, sv.psi);
    ++sv.launches;
  }
  if (s.q2) rc = run_q2(sys, sv, cols_dev, dressed);
  else rc = o->precision == SG_MIXED ? run_forward<float>(sys, sv, cols_dev, dressed, K, grad ? &ckpts : nullptr)
                                     : run_forward<double>(sys, sv, cols_dev, dressed, K, grad ? &ckpts : nullptr);
  if (!grad || rc != SG_OK) onchip_batcher_release();    // no further on-chip launch of this solve
  if (rc != SG_OK) { cudaEventDestroy(ev0); cudaEventDestroy(ev1); cudaEventDestroy(ev2); return rc; }
  if (s.frame == SG_FRAME_INTERACTION)
    k_frame<<<grid_for(n), kT, 0, st>>>(frame_args(s, sv.E_dev, -1.0), sv.psi);
  CompArgs ca = comp_args(s);
  if (dressed) k_gather_dressed<<<grid_for((long long)s.Dc * s.S), kT, 0, st>>>(Vc, sv.psi, s.D, s.S, s.Dc, Uc);
  else k_gather_comp<<<grid_for((long long)s.Dc * s.S), kT, 0, st>>>(ca, sv.psi, Uc);
  const double2* Tfid = Tg;
  if (vz) {
    // the compensated fidelity is the plain one against the effective target
    VzArgs va{};
    va.S = s.S; va.Dc = s.Dc; va.n = s.nqb; va.Uc = Uc; va.Tg = Tg; va.lab = lab_dev;
    va.W = sv.ar.get<double2>((size_t)s.Dc * s.Dc);
    va.Teff = sv.ar.get<double2>((size_t)s.Dc * s.Dc);
    if (!va.W || !va.Teff) return sg_fail(ctx, SG_E_NOMEM, "device allocation failed");
    k_vz_comp<<<1, kT, 0, st>>>(va);
    ++sv.launches;
    Tfid = va.Teff;
  }
  FidArgs fa{};
  fa.S = s.S; fa.Dc = s.Dc; fa.Sc = Sc; fa.full = full ? 1 : 0; fa.kind = kind; fa.nq = s.nq;
  for (int i = 0; i < s.nq; ++i) fa.qpos[i] = s.qpos[i];
  fa.Uc = Uc; fa.Tg = Tfid; fa.lab = lab_dev; fa.F = Fd; fa.bar = grad ? barc : nullptr; fa.M = Mbuf;
  fa.T = s.T;
  fa.frame = s.frame;
  if (shard) {
    // this shard's partial sums, summed over the shards by the caller, then F and the
    // co-states from the totals
    double* part = sv.ar.get<double>(4);
    if (!part) return sg_fail(ctx, SG_E_NOMEM, "device allocation failed");
    k_shard_partials<<<1, kT, 0, st>>>(fa, part);
    SG_CUDA_TRY(ctx, cudaGetLastError());
    double hp[4];
    SG_CUDA_TRY(ctx, cudaStreamSynchronize(st));    // reads only from an idle stream (see dcopy)
    SG_CUDA_TRY(ctx, cudaMemcpyAsync(hp, part, sizeof hp, cudaMemcpyDeviceToHost, st));
    SG_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    if (red(hp, 4, red_user) != 0) return sg_fail(ctx, SG_E_STATE, "the caller's all-reduce of the fidelity sums failed");
    if (!(hp[3] >= 1.0)) return sg_fail(ctx, SG_E_INVALID, "no shard evolved a computational state");
    if (grad && kind == SG_FID_AVG && (int)std::llround(hp[3]) != s.Dc)
      return sg_fail(ctx, SG_E_INVALID, "F_avg needs the shards to evolve every computational state exactly once");
    SG_CUDA_TRY(ctx, cudaMemcpyAsync(part, hp, sizeof hp, cudaMemcpyHostToDevice, st));
    k_shard_costate<<<1, kT, 0, st>>>(fa, part);
  } else {
    k_fidelity<<<1, kT, 0, st>>>(fa);
  }
  sv.launches += 3;
  SG_CUDA_TRY(ctx, cudaGetLastError());
  cudaEventRecord(ev1, st);
  double Fh[2];
  size_t peak = sv.ar.bytes;
  if (grad) {
    // accumulators
    const int ne = s.p.ne, n1 = s.p.n1;
    const size_t MD2 = SG_MAXD * SG_MAXD;
    GradAcc acc{};
    acc.gF = sv.ar.get<double>(3ull * s.N * std::max(1, s.K));
    acc.obD = sv.ar.get<double2>(std::max(1, s.K) * MD2);
    acc.obL = sv.ar.get<double2>(std::max(1, ne) * MD2);
    acc.obR = sv.ar.get<double2>(std::max(1, ne) * MD2);
    acc.ebB = sv.ar.get<double>(std::max(1, n1) * SG_MAXD);
    acc.ebL = sv.ar.get<double>(std::max(1, ne) * SG_MAXD);
    acc.ebR = sv.ar.get<double>(std::max(1, ne) * SG_MAXD);
    acc.jb = sv.ar.get<double>(std::max(1, ne));
    double* ebar_frame = sv.ar.get<double>(s.nq * SG_MAXD);
    double* omega_bar = sv.ar.get<double>(std::max(1, s.K));
    double2* opbar = sv.ar.get<double2>(s.nq * 2 * MD2);
    double* ebar = sv.ar.get<double>(s.nq * SG_MAXD);
    double* gpulse = sv.ar.get<double>(std::max(1, s.n_pulse));
    double* gdev = sv.ar.get<double>(3 * s.nq);
    double2* pbar = sv.ar.get<double2>(n);
    if (!acc.gF || !acc.obD || !acc.obL || !acc.obR || !acc.ebB || !acc.ebL || !acc.ebR || !acc.jb ||
        !ebar_frame || !omega_bar || !opbar || !ebar || !gpulse || !gdev || !poff || !pbar)
      return sg_fail(ctx, SG_E_NOMEM, "device allocation of gradient accumulators failed");
    SG_CUDA_TRY(ctx, cudaMemsetAsync(acc.gF, 0, 3ull * s.N * std::max(1, s.K) * sizeof(double), st));
    SG_CUDA_TRY(ctx, cudaMemsetAsync(acc.obD, 0, std::max(1, s.K) * MD2 * sizeof(double2), st));
    SG_CUDA_TRY(ctx, cudaMemsetAsync(acc.obL, 0, std::max(1, ne) * MD2 * sizeof(double2), st));
    SG_CUDA_TRY(ctx, cudaMemsetAsync(acc.obR, 0, std::max(1, ne) * MD2 * sizeof(double2), st));
    SG_CUDA_TRY(ctx, cudaMemsetAsync(acc.ebB, 0, std::max(1, n1) * SG_MAXD * sizeof(double), st));
    SG_CUDA_TRY(ctx, cudaMemsetAsync(acc.ebL, 0, std::max(1, ne) * SG_MAXD * sizeof(double), st));
    SG_CUDA_TRY(ctx, cudaMemsetAsync(acc.ebR, 0, std::max(1, ne) * SG_MAXD * sizeof(double), st));
    SG_CUDA_TRY(ctx, cudaMemsetAsync(acc.jb, 0, std::max(1, ne) * sizeof(double), st));
    SG_CUDA_TRY(ctx, cudaMemsetAsync(ebar_frame, 0, s.nq * SG_MAXD * sizeof(double), st));
    SG_CUDA_TRY(ctx, cudaMemsetAsync(pbar, 0, n * sizeof(double2), st));
    // co-state of the lab-frame columns, its frame-phase energy term, pull back to the frame
    if (dressed) k_scatter_dressed<<<grid_for(n), kT, 0, st>>>(Vc, barc, s.D, s.S, s.Dc, pbar);
    else k_scatter_comp<<<grid_for((long long)s.Dc * s.S), kT, 0, st>>>(ca, barc, pbar);
    if (s.frame == SG_FRAME_INTERACTION) {
      fa.ebar_frame = ebar_frame;
      if (!dressed) k_frame_ebar<<<1, kT, 0, st>>>(fa);    // energy co-gradient: Hamiltonian gradient only
      k_frame<<<grid_for(n), kT, 0, st>>>(frame_args(s, sv.E_dev, +1.0), pbar);
    }
    sv.launches += 3;
    if (s.q2) rc = run_backward_q2(sys, sv, pbar, acc);
    else rc = o->precision == SG_MIXED ? run_backward<float>(sys, sv, ckpts, K, pbar, acc)
                                       : run_backward<double>(sys, sv, ckpts, K, pbar, acc);
    onchip_batcher_release();
    if (rc != SG_OK) { cudaEventDestroy(ev0); cudaEventDestroy(ev1); cudaEventDestroy(ev2); return rc; }
    // chains
    if (s.K) {
      int np_max = 1;
      for (auto& d : s.drives) np_max = std::max(np_max, d.kind == SG_ENV_PWC ? d.nseg : 1);
      const int pt = 64;
      k_pulse_chain<<<s.K, pt, pt * (np_max + 1) * sizeof(double), st>>>(
          sv.drives_dev, sv.amps_dev, acc.gF, s.K, s.N, s.dt, poff, s.n_pulse, gpulse, omega_bar, s.q2 ? s.ta.nsub : 0);
    } else {
      SG_CUDA_TRY(ctx, cudaMemsetAsync(omega_bar, 0, sizeof(double), st));
    }
    AssembleArgs aa{};
    aa.nq = s.nq; aa.n1 = n1; aa.ne = ne; aa.K = s.K;
    for (int i = 0; i < s.nq; ++i) { aa.dims[i] = s.p.dims[i]; aa.s1_of_mode[i] = s.s1_of_mode[i]; }
    for (int k = 0; k < s.K; ++k) {
      aa.drv_mode[k] = sys->drives[k].mode; aa.drv_op[k] = sys->drives[k].op;
      aa.drv_omode[k] = sys->drives[k].omega_mode;
    }
    for (int e = 0; e < ne; ++e) {
      aa.e_a[e] = s.p.e_a[e]; aa.e_b[e] = s.p.e_b[e]; aa.e_opa[e] = s.ta.e_opa[e]; aa.e_opb[e] = s.ta.e_opb[e];
    }
    aa.acc = acc; aa.omega_bar = omega_bar; aa.ebar_frame = ebar_frame; aa.opbar = opbar; aa.ebar = ebar;
    ++sv.launches;
    if (grad_ham) {
      k_assemble<<<1, kT, 0, st>>>(aa);
      ++sv.launches;
      SG_CUDA_TRY(ctx, cudaGetLastError());
      rc = sg_chain_device_params(sys, opbar, ebar, gdev);
      if (rc != SG_OK) return rc;
      ++sv.launches;
    }
    cudaEventRecord(ev2, st);
    SG_CUDA_TRY(ctx, cudaStreamSynchronize(st));   // reads only from an idle stream (see dcopy)
    SG_CUDA_TRY(ctx, cudaMemcpyAsync(Fh, Fd, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    std::vector<double> gd(3 * s.nq), jb(std::max(1, ne));
    if (s.n_pulse && grad_pulse)
      SG_CUDA_TRY(ctx, cudaMemcpyAsync(grad_pulse, gpulse, s.n_pulse * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (grad_ham) {
      SG_CUDA_TRY(ctx, cudaMemcpyAsync(gd.data(), gdev, 3 * s.nq * sizeof(double), cudaMemcpyDeviceToHost, st));
      SG_CUDA_TRY(ctx, cudaMemcpyAsync(jb.data(), acc.jb, std::max(1, ne) * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    SG_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    if (grad_ham) {
      for (int i = 0; i < s.nq; ++i) {
        grad_ham[3 * i + 0] = gd[3 * i + 0];
        grad_ham[3 * i + 1] = gd[3 * i + 1];
        grad_ham[3 * i + 2] = sys->modes[i].kind == 0 ? 0.0 : gd[3 * i + 2];
      }
      for (int e = 0; e < ne; ++e) grad_ham[3 * s.nq + e] = jb[e];
    }
    if (shard) {
      // the gradient is linear in the co-states: the sum of the shards' gradients
      const int nh = grad_ham ? 3 * s.nq + ne : 0;
      std::vector<double> g((size_t)s.n_pulse + nh + 1, 0.0);
      if (grad_pulse) for (int k = 0; k < s.n_pulse; ++k) g[k] = grad_pulse[k];
      for (int k = 0; k < nh; ++k) g[s.n_pulse + k] = grad_ham[k];
      if (red(g.data(), s.n_pulse + nh, red_user) != 0)
        return sg_fail(ctx, SG_E_STATE, "the caller's all-reduce of the gradient failed");
      if (grad_pulse) for (int k = 0; k < s.n_pulse; ++k) grad_pulse[k] = g[k];
      for (int k = 0; k < nh; ++k) grad_ham[k] = g[s.n_pulse + k];
    }
    peak = sv.ar.bytes;
  } else {
    cudaEventRecord(ev2, st);
    SG_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    SG_CUDA_TRY(ctx, cudaMemcpyAsync(Fh, Fd, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  if (Ucomp_out)
    SG_CUDA_TRY(ctx, cudaMemcpyAsync(Ucomp_out, Uc, (size_t)s.Dc * s.S * sizeof(double2), cudaMemcpyDeviceToHost, st));
  SG_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  float fwd_ms = 0.f, bwd_ms = 0.f;
  cudaEventElapsedTime(&fwd_ms, ev0, ev1);
  cudaEventElapsedTime(&bwd_ms, ev1, ev2);
  cudaEventDestroy(ev0); cudaEventDestroy(ev1); cudaEventDestroy(ev2);
  (void)t0;
  if (F_out) { F_out[0] = Fh[0]; F_out[1] = Fh[1]; }
  sys->last_stats[0] = fwd_ms;
  sys->last_stats[1] = bwd_ms;
  sys->last_stats[2] = (double)peak;
  sys->last_stats[3] = K;
  sv.kt.finish(sys->ktimes);
  sys->last_stats[4] = sv.launches + (double)(sv.kt.total[0] + sv.kt.total[1] + sv.kt.total[2]);
  return SG_OK;
}

// ---------------------------------------------------------------------------
// Gradient of the open-system gate fidelity (sg_gate_fidelity_open_grad)
// ---------------------------------------------------------------------------
// The Dc^2 inputs |c_j><c_k| evolve as columns of the doubled system (lindblad.cu);
// the channel fidelity is linear in the evolved columns, so its co-state is fixed by
// the target (k_open_costate).  The discrete adjoint of the non-Hermitian generator
// A = -i H_eff pulls the co-state back with A^dag = i H_eff^dag, i.e. the adjoint passes
// apply the stage rows of the conjugate-transposed doubled system, while the drive
// terms of dF/df contract the forward operators (Sec. 2.5 on the vectorised equation,
// App. C last paragraph).  A drive of the open system appears twice in the doubled
// one, on the ket mode with its parameters and on the bra mode with their negatives,
// so its gradient is the ket copy's minus the bra copy's.  The Hamiltonian-parameter
// gradient (grad_ham) folds the doubled modes' operator and energy co-gradients onto
// the open system's modes (a bra mode carries the operators transposed and the energies
// negated, k_open_fold) before the eigen-derivative chain, and a coupling's gradient
// is its ket copy's minus its bra copy's (strength -J).
sg_status sg_gate_fidelity_open_grad_impl(sg_system* sys, const sg_evolve_opts* o, const double* target, int kind,
                                          double* F_out, double* grad_pulse, double* grad_ham, int ckpt) {
  sg_ctx* ctx = sys->ctx;
  if (!sys->prepared) return sg_fail(ctx, SG_E_STATE, "system is not prepared (call sg_prepare)");
  if (!o || !target || !F_out || !grad_pulse)
    return sg_fail(ctx, SG_E_INVALID, "the open gate fidelity gradient needs opts, target, F_out and grad_pulse");
  if (kind != SG_FID_AVG && kind != SG_FID_STATE) return sg_fail(ctx, SG_E_INVALID, "bad fidelity kind");
  if (o->solver != SG_SOLVER_RK4) return sg_fail(ctx, SG_E_UNSUPPORTED, "the open evolution runs RK4");
  const int nq = (int)sys->modes.size();
  int nqb = 0;
  for (const HostMode& m : sys->modes) nqb += m.coupler ? 0 : 1;
  if (nqb < 1 || nqb > 6) return sg_fail(ctx, SG_E_UNSUPPORTED, "the open gate fidelity takes 1..6 qubit modes");
  const int Dc = 1 << nqb;
  long long D = 1;
  std::vector<long long> stv(nq);
  for (int i = nq - 1; i >= 0; --i) { stv[i] = D; D *= sys->modes[i].d; }
  std::vector<long long> comp(Dc), cols((size_t)Dc * Dc);
  for (int j = 0; j < Dc; ++j) {
    long long r = 0;
    for (int i = 0, b = nqb - 1; i < nq; ++i) r += (long long)(sys->modes[i].coupler ? 0 : (j >> b--) & 1) * stv[i];
    comp[j] = r;
  }
  for (int j = 0; j < Dc; ++j)
    for (int k = 0; k < Dc; ++k) cols[(size_t)j * Dc + k] = comp[j] * D + comp[k];
  sg_system dsys, dadj;
  sg_status rc = lindblad_doubled(sys, o->T, dsys);
  if (rc != SG_OK) return rc;
  lindblad_adjoint_rows(dsys, dadj);
  sg_evolve_opts od = *o;
  od.ncols = Dc * Dc;
  od.col_index = cols.data();
  od.compensation = SG_COMP_NONE;
  od.basis = SG_BASIS_PRODUCT;
  Solve sv, sva;
  sv.ar.st = sva.ar.st = ctx->stream;
  sv.want_ham = sva.want_ham = grad_ham != nullptr;
  // the Hamiltonian gradient contracts the coupling and energy terms with the forward
  // rows of the non-Hermitian generator: the gather kernels keep them apart from the
  // applied (conjugate-transposed) rows
  sv.force_gather = sva.force_gather = grad_ham != nullptr;
  rc = build_setup(&dsys, &od, sv.s);
  if (rc != SG_OK) return rc;
  rc = build_setup(&dadj, &od, sva.s);
  if (rc != SG_OK) return rc;
  Setup& s = sv.s;
  if (sva.s.p.row != s.p.row || sva.s.N != s.N)
    return sg_fail(ctx, SG_E_STATE, "adjoint rows of the open evolution do not match its plan");
  SG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  keep_pool_memory(ctx->device);
  cudaStream_t st = ctx->stream;
  const long long n = s.D * s.S;
  long long* cols_dev = sv.ar.get<long long>(s.S);
  long long* comp_dev = sv.ar.get<long long>(Dc);
  double2* Tg = sv.ar.get<double2>((size_t)Dc * Dc);
  double* Fd = sv.ar.get<double>(2);
  int* poff = sv.ar.get<int>(std::max(1, s.K));
  sv.psi = sv.ar.get<double2>(n);
  if (!cols_dev || !comp_dev || !Tg || !Fd || !poff || !sv.psi) return sg_fail(ctx, SG_E_NOMEM, "device allocation failed");
  SG_CUDA_TRY(ctx, cudaMemcpyAsync(cols_dev, cols.data(), s.S * sizeof(long long), cudaMemcpyHostToDevice, st));
  SG_CUDA_TRY(ctx, cudaMemcpyAsync(comp_dev, comp.data(), Dc * sizeof(long long), cudaMemcpyHostToDevice, st));
  SG_CUDA_TRY(ctx, cudaMemcpyAsync(Tg, target, (size_t)Dc * Dc * sizeof(double2), cudaMemcpyHostToDevice, st));
  if (s.K) SG_CUDA_TRY(ctx, cudaMemcpyAsync(poff, s.pulse_off.data(), s.K * sizeof(int), cudaMemcpyHostToDevice, st));
  rc = upload_and_tables(&dsys, &od, sv, true);
  if (rc != SG_OK) return rc;
  rc = upload_and_tables(&dadj, &od, sva, true);
  if (rc != SG_OK) return rc;
  sv.adj_tab = sva.tab;
  sv.adj_tab32 = sva.tab32;
  if ((o->precision == SG_MIXED ? (const void*)sv.adj_tab32 : (const void*)sv.adj_tab) == nullptr)
    return sg_fail(ctx, SG_E_STATE, "adjoint rows of the open evolution missing");
  // checkpoints
  int K = ckpt > 0 ? ckpt : std::max(1, (int)std::lround(std::sqrt((double)s.N)));
  K = std::min(K, s.N);
  const int nck = (s.N + K - 1) / K;
  std::vector<double2*> ckpts;
  if (sv.onchip(true)) {
    const long long ns = onchip_state_elems(sv.oc);
    double2* p = sv.ar.get<double2>((size_t)nck * ns);
    if (!p) return sg_fail(ctx, SG_E_NOMEM, "device allocation of checkpoints failed");
    for (int c = 0; c < nck; ++c) ckpts.push_back(p + (size_t)c * ns);
  } else {
    for (int c = 0; c < nck; ++c) {
      double2* p = sv.ar.get<double2>(n);
      if (!p) return sg_fail(ctx, SG_E_NOMEM, "device allocation of checkpoints failed");
      ckpts.push_back(p);
    }
  }
  cudaEvent_t ev0, ev1, ev2;
  cudaEventCreate(&ev0); cudaEventCreate(&ev1); cudaEventCreate(&ev2);
  auto done = [&](sg_status r) { cudaEventDestroy(ev0); cudaEventDestroy(ev1); cudaEventDestroy(ev2); return r; };
  cudaEventRecord(ev0, st);
  rc = o->precision == SG_MIXED ? run_forward<float>(&dsys, sv, cols_dev, false, K, &ckpts)
                                : run_forward<double>(&dsys, sv, cols_dev, false, K, &ckpts);
  if (rc != SG_OK) return done(rc);
  if (s.frame == SG_FRAME_INTERACTION) k_frame<<<grid_for(n), kT, 0, st>>>(frame_args(s, sv.E_dev, -1.0), sv.psi);
  launch_open_fidelity(sv.psi, comp_dev, Tg, D, Dc, Fd, st);
  sv.launches += 2;
  cudaEventRecord(ev1, st);
  // accumulators (the pulse gradient reads gF; the adjoint kernels also write the
  // per-term operator and energy co-gradients of the 1-body slots)
  const int ne = s.p.ne, n1 = s.p.n1;
  const size_t MD2 = SG_MAXD * SG_MAXD;
  GradAcc acc{};
  acc.gF = sv.ar.get<double>(3ull * s.N * std::max(1, s.K));
  acc.obD = sv.ar.get<double2>(std::max(1, s.K) * MD2);
  acc.obL = sv.ar.get<double2>(std::max(1, ne) * MD2);
  acc.obR = sv.ar.get<double2>(std::max(1, ne) * MD2);
  acc.ebB = sv.ar.get<double>(std::max(1, n1) * SG_MAXD);
  acc.ebL = sv.ar.get<double>(std::max(1, ne) * SG_MAXD);
  acc.ebR = sv.ar.get<double>(std::max(1, ne) * SG_MAXD);
  acc.jb = sv.ar.get<double>(std::max(1, ne));
  double* omega_bar = sv.ar.get<double>(std::max(1, s.K));
  double* gpulse = sv.ar.get<double>(std::max(1, s.n_pulse));
  double2* pbar = sv.ar.get<double2>(n);
  if (!acc.gF || !acc.obD || !acc.obL || !acc.obR || !acc.ebB || !acc.ebL || !acc.ebR || !acc.jb || !omega_bar ||
      !gpulse || !pbar)
    return done(sg_fail(ctx, SG_E_NOMEM, "device allocation of gradient accumulators failed"));
  SG_CUDA_TRY(ctx, cudaMemsetAsync(acc.gF, 0, 3ull * s.N * std::max(1, s.K) * sizeof(double), st));
  SG_CUDA_TRY(ctx, cudaMemsetAsync(acc.obD, 0, std::max(1, s.K) * MD2 * sizeof(double2), st));
  SG_CUDA_TRY(ctx, cudaMemsetAsync(acc.obL, 0, std::max(1, ne) * MD2 * sizeof(double2), st));
  SG_CUDA_TRY(ctx, cudaMemsetAsync(acc.obR, 0, std::max(1, ne) * MD2 * sizeof(double2), st));
  SG_CUDA_TRY(ctx, cudaMemsetAsync(acc.ebB, 0, std::max(1, n1) * SG_MAXD * sizeof(double), st));
  SG_CUDA_TRY(ctx, cudaMemsetAsync(acc.ebL, 0, std::max(1, ne) * SG_MAXD * sizeof(double), st));
  SG_CUDA_TRY(ctx, cudaMemsetAsync(acc.ebR, 0, std::max(1, ne) * SG_MAXD * sizeof(double), st));
  SG_CUDA_TRY(ctx, cudaMemsetAsync(acc.jb, 0, std::max(1, ne) * sizeof(double), st));
  SG_CUDA_TRY(ctx, cudaMemsetAsync(pbar, 0, n * sizeof(double2), st));
  launch_open_costate(comp_dev, Tg, D, Dc, kind, pbar, st);
  double* ebar_frame = sv.ar.get<double>((size_t)s.nq * SG_MAXD);
  if (!ebar_frame) return done(sg_fail(ctx, SG_E_NOMEM, "device allocation failed"));
  SG_CUDA_TRY(ctx, cudaMemsetAsync(ebar_frame, 0, (size_t)s.nq * SG_MAXD * sizeof(double), st));
  if (grad_ham && s.frame == SG_FRAME_INTERACTION) {
    // energy cotangent of the frame epilogue, from the lab-frame states and co-state
    OpenModes om{};
    om.nq = nq;
    om.D = D;
    for (int i = 0; i < nq; ++i) { om.dims[i] = sys->modes[i].d; om.st[i] = stv[i]; }
    launch_open_frame_ebar(sv.psi, pbar, comp_dev, om, Dc, s.T, ebar_frame, st);
    ++sv.launches;
  }
  if (s.frame == SG_FRAME_INTERACTION) k_frame<<<grid_for(n), kT, 0, st>>>(frame_args(s, sv.E_dev, +1.0), pbar);
  sv.launches += 2;
  SG_CUDA_TRY(ctx, cudaGetLastError());
  rc = o->precision == SG_MIXED ? run_backward<float>(&dsys, sv, ckpts, K, pbar, acc)
                                : run_backward<double>(&dsys, sv, ckpts, K, pbar, acc);
  if (rc != SG_OK) return done(rc);
  if (s.K) {
    int np_max = 1;
    for (auto& d : s.drives) np_max = std::max(np_max, d.kind == SG_ENV_PWC ? d.nseg : 1);
    const int pt = 64;
    k_pulse_chain<<<s.K, pt, pt * (np_max + 1) * sizeof(double), st>>>(
        sv.drives_dev, sv.amps_dev, acc.gF, s.K, s.N, s.dt, poff, s.n_pulse, gpulse, omega_bar, 0);
    ++sv.launches;
  }
  double* gdev = nullptr;
  if (grad_ham) {
    // the doubled modes' co-gradients, folded onto the open system's modes, then the
    // eigen-derivative chain of the open system
    const size_t MD2 = SG_MAXD * SG_MAXD;
    double2* opbar_d = sv.ar.get<double2>((size_t)s.nq * 2 * MD2);
    double* ebar_d = sv.ar.get<double>((size_t)s.nq * SG_MAXD);
    double2* opbar = sv.ar.get<double2>((size_t)nq * 2 * MD2);
    double* ebar = sv.ar.get<double>((size_t)nq * SG_MAXD);
    gdev = sv.ar.get<double>(3 * nq);
    if (!opbar_d || !ebar_d || !opbar || !ebar || !gdev)
      return done(sg_fail(ctx, SG_E_NOMEM, "device allocation of gradient accumulators failed"));
    AssembleArgs aa{};
    aa.nq = s.nq; aa.n1 = n1; aa.ne = ne; aa.K = s.K;
    for (int i = 0; i < s.nq; ++i) { aa.dims[i] = s.p.dims[i]; aa.s1_of_mode[i] = s.s1_of_mode[i]; }
    for (int k = 0; k < s.K; ++k) {
      aa.drv_mode[k] = dsys.drives[k].mode; aa.drv_op[k] = dsys.drives[k].op;
      aa.drv_omode[k] = dsys.drives[k].omega_mode;
    }
    for (int e = 0; e < ne; ++e) {
      aa.e_a[e] = s.p.e_a[e]; aa.e_b[e] = s.p.e_b[e]; aa.e_opa[e] = s.ta.e_opa[e]; aa.e_opb[e] = s.ta.e_opb[e];
    }
    aa.acc = acc; aa.omega_bar = omega_bar; aa.ebar_frame = ebar_frame; aa.opbar = opbar_d; aa.ebar = ebar_d;
    if (!s.K) SG_CUDA_TRY(ctx, cudaMemsetAsync(omega_bar, 0, sizeof(double), st));
    k_assemble<<<1, kT, 0, st>>>(aa);
    launch_open_fold(nq, opbar_d, ebar_d, opbar, ebar, st);
    sv.launches += 2;
    SG_CUDA_TRY(ctx, cudaGetLastError());
    sg_status rc2 = sg_chain_device_params(sys, opbar, ebar, gdev);
    if (rc2 != SG_OK) return done(rc2);
    ++sv.launches;
  }
  SG_CUDA_TRY(ctx, cudaGetLastError());
  cudaEventRecord(ev2, st);
  double Fh[2] = {0.0, 0.0};
  std::vector<double> gd(std::max(1, s.n_pulse), 0.0);
  std::vector<double> gdh(3 * (size_t)nq), jbh(std::max(1, ne));
  SG_CUDA_TRY(ctx, cudaStreamSynchronize(st));    // reads only from an idle stream (see dcopy)
  SG_CUDA_TRY(ctx, cudaMemcpyAsync(Fh, Fd, sizeof Fh, cudaMemcpyDeviceToHost, st));
  if (s.n_pulse) SG_CUDA_TRY(ctx, cudaMemcpyAsync(gd.data(), gpulse, s.n_pulse * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (grad_ham) {
    SG_CUDA_TRY(ctx, cudaMemcpyAsync(gdh.data(), gdev, 3 * nq * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (ne) SG_CUDA_TRY(ctx, cudaMemcpyAsync(jbh.data(), acc.jb, ne * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  SG_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  if (grad_ham) {
    for (int i = 0; i < nq; ++i) {
      grad_ham[3 * i + 0] = gdh[3 * i + 0];
      grad_ham[3 * i + 1] = gdh[3 * i + 1];
      grad_ham[3 * i + 2] = sys->modes[i].kind == 0 ? 0.0 : gdh[3 * i + 2];
    }
    // the doubled couplings 2e (ket, J) and 2e + 1 (bra, -J) of coupling e
    for (size_t e = 0; e < sys->couplings.size(); ++e) grad_ham[3 * nq + e] = jbh[2 * e] - jbh[2 * e + 1];
  }
  // the doubled drives 2k (ket) and 2k + 1 (bra, negated parameters) of drive k
  int po = 0;
  for (size_t k = 0; k < sys->drives.size(); ++k) {
    const HostDrive& hd = sys->drives[k];
    const int np = hd.kind == SG_ENV_PWC ? hd.nseg : 1;
    for (int x = 0; x < np; ++x)
      grad_pulse[po + x] = gd[s.pulse_off[2 * k] + x] - gd[s.pulse_off[2 * k + 1] + x];
    po += np;
  }
  F_out[0] = Fh[0];
  F_out[1] = Fh[1];
  float fwd_ms = 0.f, bwd_ms = 0.f;
  cudaEventElapsedTime(&fwd_ms, ev0, ev1);
  cudaEventElapsedTime(&bwd_ms, ev1, ev2);
  sys->last_stats[0] = fwd_ms;
  sys->last_stats[1] = bwd_ms;
  sys->last_stats[2] = (double)(sv.ar.bytes + sva.ar.bytes);
  sys->last_stats[3] = K;
  sv.kt.finish(sys->ktimes);
  sys->last_stats[4] = sv.launches + (double)(sv.kt.total[0] + sv.kt.total[1] + sv.kt.total[2]);
  return done(SG_OK);
}

// ---------------------------------------------------------------------------
// Evolution without allocation (sg_evolve_noalloc)
// ---------------------------------------------------------------------------
// Some callers cannot allocate device memory when they evolve: a host program
// whose GPU memory is owned by another allocator (for example a framework's
// caching allocator that has reserved the device), or a latency-bound control
// loop that cannot afford cudaMalloc's implicit synchronisation.  For them this
// entry point keeps every per-call buffer (drive data, stage tables, stage slabs)
// in one fixed array compiled into the library.  Every GPU that loads the
// library holds the array until the process exits.
namespace {
constexpr size_t kNoAllocScratchBytes = 32ull << 20;   // 32 MiB
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the scratch array on the context's device.  The host-side
// symbol is only a stand-in, so the address is looked up once per device (with
// that device current) and cached.
static sg_status noalloc_scratch(sg_ctx* ctx, unsigned char** out) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  const int dev = ctx->device;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return sg_fail(ctx, SG_E_UNSUPPORTED, "device index beyond 63");
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return sg_fail(ctx, SG_E_CUDA, std::string("cudaGetSymbolAddress of the scratch array: ") + cudaGetErrorString(e));
    g_noalloc_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_noalloc_ptr[dev]);
  return SG_OK;
}

template <typename R>
static sg_status noalloc_run(sg_system* sys, const sg_evolve_opts* o, double2* psi) {
  typedef typename CT<R>::T C;
  sg_ctx* ctx = sys->ctx;
  Solve sv;
  sg_status rc = build_setup(sys, o, sv.s);
  if (rc != SG_OK) return rc;
  if (sv.s.q2) return sg_fail(ctx, SG_E_UNSUPPORTED, "sg_evolve_noalloc runs the RK4 solver only");
  Setup& s = sv.s;
  if (o->col_index)
    for (int c = 0; c < s.S; ++c)
      if (o->col_index[c] < 0 || o->col_index[c] >= s.D) return sg_fail(ctx, SG_E_INVALID, "col_index out of range");
  // layout of the scratch array
  size_t used = 0;
  auto carve = [&](size_t bytes) {
    const size_t at = used;
    used = (used + std::max<size_t>(bytes, 1) + 255) & ~(size_t)255;
    return at;
  };
  const size_t nst = 3ull * s.N;
  const long long n = s.D * s.S;
  const size_t o_drv = carve(std::max(1, s.K) * sizeof(DriveDev));
  const size_t o_amp = carve(std::max<size_t>(1, s.amps.size()) * sizeof(double));
  const size_t o_E = carve(s.sumd * sizeof(double));
  const size_t o_opd = carve(s.opdflat.size() * sizeof(double2));
  const size_t o_coef = carve(nst * std::max(1, s.K) * sizeof(double));
  const size_t o_ph = carve(nst * s.sumd * sizeof(double2));
  const size_t o_tab = carve(nst * s.p.row * sizeof(double2));
  const size_t o_tab32 = carve(sizeof(R) == 4 ? nst * s.p.row * sizeof(float2) : 1);
  const size_t o_cols = carve(s.S * sizeof(long long));
  const size_t o_X = carve(n * sizeof(C));
  const size_t o_Xo = carve(n * sizeof(C));
  const size_t o_D = carve(n * sizeof(C));
  if (used > kNoAllocScratchBytes) {
    char msg[200];
    std::snprintf(msg, sizeof msg,
                  "this evolution needs %.1f MiB of scratch; sg_evolve_noalloc has a fixed %zu MiB "
                  "(use sg_evolve, or fewer steps, columns or levels)",
                  used / 1048576.0, kNoAllocScratchBytes >> 20);
    return sg_fail(ctx, SG_E_INVALID, msg);
  }
  SG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  unsigned char* base = nullptr;
  rc = noalloc_scratch(ctx, &base);
  if (rc != SG_OK) return rc;
  cudaStream_t st = ctx->stream;
  sv.drives_dev = reinterpret_cast<DriveDev*>(base + o_drv);
  sv.amps_dev = reinterpret_cast<double*>(base + o_amp);
  sv.E_dev = reinterpret_cast<double*>(base + o_E);
  sv.opd_dev = reinterpret_cast<double2*>(base + o_opd);
  sv.coef = reinterpret_cast<double*>(base + o_coef);
  sv.ph = reinterpret_cast<double2*>(base + o_ph);
  sv.tab = reinterpret_cast<double2*>(base + o_tab);
  sv.tab32 = sizeof(R) == 4 ? reinterpret_cast<float2*>(base + o_tab32) : nullptr;
  long long* cols = reinterpret_cast<long long*>(base + o_cols);
  C* X = reinterpret_cast<C*>(base + o_X);
  C* Xo = reinterpret_cast<C*>(base + o_Xo);
  C* Dacc = reinterpret_cast<C*>(base + o_D);
  if (s.K) SG_CUDA_TRY(ctx, cudaMemcpyAsync(sv.drives_dev, s.drives.data(), s.K * sizeof(DriveDev), cudaMemcpyHostToDevice, st));
  if (!s.amps.empty()) SG_CUDA_TRY(ctx, cudaMemcpyAsync(sv.amps_dev, s.amps.data(), s.amps.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  SG_CUDA_TRY(ctx, cudaMemcpyAsync(sv.E_dev, s.Eflat.data(), s.sumd * sizeof(double), cudaMemcpyHostToDevice, st));
  SG_CUDA_TRY(ctx, cudaMemcpyAsync(sv.opd_dev, s.opdflat.data(), s.opdflat.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
  if (o->col_index)
    SG_CUDA_TRY(ctx, cudaMemcpyAsync(cols, o->col_index, s.S * sizeof(long long), cudaMemcpyHostToDevice, st));
  TabArgs ta = s.ta;
  ta.drives = sv.drives_dev; ta.amps = sv.amps_dev; ta.E = sv.E_dev; ta.opd = sv.opd_dev;
  ta.coef = sv.coef; ta.ph = sv.ph; ta.tab = sv.tab; ta.tab32 = sv.tab32;
  s.ta = ta;
  // every scratch buffer below is fully written before it is read, so nothing is cleared
  k_tables<<<(unsigned)nst, 64, 0, st>>>(ta);
  if (o->col_index) k_init_cols<<<grid_for(n), kT, 0, st>>>(psi, s.D, s.S, cols);
  sv.mixed = sizeof(R) == 4;
  sv.psi = psi;
  k_cast<R><<<grid_for(n), kT, 0, st>>>(psi, X, n, 1.0);
  for (int step = 0; step < s.N; ++step) fwd_step<R>(sv, st, step, psi, psi, X, Xo, Dacc);
  if (o->frame == SG_FRAME_INTERACTION)
    k_frame<<<grid_for(n), kT, 0, st>>>(frame_args(s, sv.E_dev, -1.0), psi);
  SG_CUDA_TRY(ctx, cudaGetLastError());
  SG_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  return SG_OK;
}

extern "C" sg_status sg_evolve_noalloc(sg_system* sys, const sg_evolve_opts* opts, void* psi_dev) {
  if (!sys) return SG_E_INVALID;
  std::lock_guard<std::mutex> lk(sys->ctx->mu);
  sg_ctx* ctx = sys->ctx;
  if (!sys->prepared) return sg_fail(ctx, SG_E_STATE, "system is not prepared (call sg_prepare)");
  if (!psi_dev) return sg_fail(ctx, SG_E_INVALID, "psi_dev is NULL");
  if (!opts) return sg_fail(ctx, SG_E_INVALID, "null options");
  double2* psi = static_cast<double2*>(psi_dev);
  return opts->precision == SG_MIXED ? noalloc_run<float>(sys, opts, psi) : noalloc_run<double>(sys, opts, psi);
}

// ---------------------------------------------------------------------------
// Batched dense evolution on the tensor cores (sg_evolve_batch, dense.cu)
// ---------------------------------------------------------------------------
namespace {

// f_k at every stage slot of every system (FP64 envelope and carrier, stored FP32).
__global__ void k_batch_coef(const DriveDev* __restrict__ drives, const double* __restrict__ amps, int B, int K,
                             int N, double dt, float* __restrict__ coef) {
  const long long total = (long long)B * 3 * N * K;
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < total;
       x += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(x % K);
    const long long bq = x / K;
    const int q = (int)(bq % (3ll * N));
    const int b = (int)(bq / (3ll * N));
    const int n = q / 3, j = q % 3;
    const double t = (double)(2 * n + j) * dt * 0.5;
    const DriveDev dr = drives[(size_t)b * K + k];
    coef[x] = (float)(envelope_dev(dr, amps, n, j, t) * cos(dr.omega * t + dr.phase));
  }
}

// Real part (part 0) or imaginary part (part 1) of element (x, y) of operator op of mode m.
double op_elem(const sg_system* sys, int m, int op, int x, int y, int part) {
  const int d = sys->modes[m].d;
  return sys->opd_host[m][2 * ((size_t)op * d * d + x * d + y) + part];
}

}  // namespace

sg_status sg_evolve_batch_impl(sg_system* const* systems, int B, const sg_evolve_opts* o, void* psi_dev) {
  if (!systems || B < 1 || !systems[0]) return SG_E_INVALID;
  sg_system* s0 = systems[0];
  sg_ctx* ctx = s0->ctx;
  if (!o || !o->col_index || !psi_dev) return sg_fail(ctx, SG_E_INVALID, "batch evolution needs col_index and psi_dev");
  if (o->precision != SG_MIXED)
    return sg_fail(ctx, SG_E_UNSUPPORTED, "the tensor-core batch runs 3xTF32 products (precision SG_MIXED)");
  if (o->solver != SG_SOLVER_RK4) return sg_fail(ctx, SG_E_UNSUPPORTED, "the tensor-core batch runs RK4");
  if (o->frame != SG_FRAME_INTERACTION && o->frame != SG_FRAME_LAB) return sg_fail(ctx, SG_E_INVALID, "bad frame");
  const int nq = (int)s0->modes.size(), K = (int)s0->drives.size();
  for (int b = 0; b < B; ++b) {
    const sg_system* sy = systems[b];
    if (!sy || !sy->prepared) return sg_fail(ctx, SG_E_STATE, "every system of a batch must be prepared");
    if (sy->ctx != ctx) return sg_fail(ctx, SG_E_INVALID, "the systems of a batch must share a context");
    if ((int)sy->modes.size() != nq || (int)sy->drives.size() != K)
      return sg_fail(ctx, SG_E_INVALID, "the systems of a batch must have the same modes and drive count");
    for (int m = 0; m < nq; ++m)
      if (sy->modes[m].d != s0->modes[m].d) return sg_fail(ctx, SG_E_INVALID, "the systems of a batch differ in levels");
  }
  Setup s;
  sg_status rc = build_setup(s0, o, s);
  if (rc != SG_OK) return rc;
  const int D = (int)s.D, S = s.S;
  int Dp = 0, R = 0, G = 0, Nn = 0;
  if (s.D > 64 || !dense_shape(D, S, K, &Dp, &R, &G, &Nn))
    return sg_fail(ctx, SG_E_UNSUPPORTED, "the tensor-core batch takes 2 S in {8, 16, 32} and (1 + drives) x D "
                                          "(padded) <= 128");
  for (int c = 0; c < S; ++c)
    if (o->col_index[c] < 0 || o->col_index[c] >= s.D) return sg_fail(ctx, SG_E_INVALID, "col_index out of range");
  SG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  keep_pool_memory(ctx->device);
  cudaStream_t st = ctx->stream;
  // per system: dense real [C; O_1..O_K] (R x Dp), composite energies, drives
  std::vector<double> A((size_t)B * R * Dp, 0.0), E((size_t)B * D, 0.0), amps;
  std::vector<DriveDev> drv((size_t)B * std::max(1, K));
  std::vector<int> dig((size_t)D * nq);
  for (int i = 0; i < D; ++i)
    for (int m = 0; m < nq; ++m) dig[(size_t)i * nq + m] = (int)((i / s.p.st[m]) % s.p.dims[m]);
  for (int b = 0; b < B; ++b) {
    sg_system* sy = systems[b];
    Setup sb;
    rc = b == 0 ? SG_OK : build_setup(sy, o, sb);
    if (rc != SG_OK) return rc;
    const Setup& ss = b == 0 ? s : sb;
    TabArgs ta = ss.ta;
    if (!real_terms(sy, ss, ta))
      return sg_fail(ctx, SG_E_UNSUPPORTED, "the tensor-core batch needs every term real in the eigenbasis up to the "
                                            "frame phases");
    double* Ab = A.data() + (size_t)b * R * Dp;
    for (int i = 0; i < D; ++i) {
      double e = 0.0;
      for (int m = 0; m < nq; ++m) e += sy->E_host[m][dig[(size_t)i * nq + m]];
      E[(size_t)b * D + i] = e;
      if (ss.frame == SG_FRAME_LAB) Ab[(size_t)i * Dp + i] += e;
    }
    // couplings: J A (x) B on modes (a, b), the other digits equal
    for (int e = 0; e < ss.p.ne; ++e) {
      const HostCoupling& c = sy->couplings[e];
      const int part = ta.e_zpart[e];
      const double J = part ? -c.J : c.J;
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
          bool same = true;
          for (int m = 0; m < nq && same; ++m)
            if (m != c.a && m != c.b) same = dig[(size_t)i * nq + m] == dig[(size_t)j * nq + m];
          if (!same) continue;
          const int ia = dig[(size_t)i * nq + c.a], ja = dig[(size_t)j * nq + c.a];
          const int ib = dig[(size_t)i * nq + c.b], jb = dig[(size_t)j * nq + c.b];
          Ab[(size_t)i * Dp + j] += J * op_elem(sy, c.a, c.op_a, ia, ja, part) * op_elem(sy, c.b, c.op_b, ib, jb, part);
        }
    }
    // drives: O_k on its mode
    for (int k = 0; k < K; ++k) {
      const HostDrive& hd = sy->drives[k];
      double* Ok = Ab + (size_t)(1 + k) * Dp * Dp;
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
          bool same = true;
          for (int m = 0; m < nq && same; ++m)
            if (m != hd.mode) same = dig[(size_t)i * nq + m] == dig[(size_t)j * nq + m];
          if (same)
            Ok[(size_t)i * Dp + j] = op_elem(sy, hd.mode, hd.op, dig[(size_t)i * nq + hd.mode],
                                             dig[(size_t)j * nq + hd.mode], 0);
        }
      DriveDev dd = ss.drives[k];
      dd.amps_off += (int)amps.size();
      drv[(size_t)b * K + k] = dd;
    }
    for (double v : ss.amps) amps.push_back(v);
  }
  Arena ar;
  ar.st = st;
  double* A_dev = ar.get<double>(A.size());
  double* E_dev = ar.get<double>(E.size());
  DriveDev* drv_dev = ar.get<DriveDev>(drv.size());
  double* amps_dev = ar.get<double>(std::max<size_t>(1, amps.size()));
  long long* cols_dev = ar.get<long long>(S);
  float* coef = ar.get<float>((size_t)B * 3 * s.N * std::max(1, K));
  int* err = ar.get<int>(1);
  if (!A_dev || !E_dev || !drv_dev || !amps_dev || !cols_dev || !coef || !err)
    return sg_fail(ctx, SG_E_NOMEM, "device allocation failed");
  SG_CUDA_TRY(ctx, cudaMemcpyAsync(A_dev, A.data(), A.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  SG_CUDA_TRY(ctx, cudaMemcpyAsync(E_dev, E.data(), E.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  SG_CUDA_TRY(ctx, cudaMemcpyAsync(drv_dev, drv.data(), drv.size() * sizeof(DriveDev), cudaMemcpyHostToDevice, st));
  if (!amps.empty())
    SG_CUDA_TRY(ctx, cudaMemcpyAsync(amps_dev, amps.data(), amps.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  SG_CUDA_TRY(ctx, cudaMemcpyAsync(cols_dev, o->col_index, S * sizeof(long long), cudaMemcpyHostToDevice, st));
  SG_CUDA_TRY(ctx, cudaMemsetAsync(err, 0, sizeof(int), st));
  if (K) k_batch_coef<<<grid_for((long long)B * 3 * s.N * K), kT, 0, st>>>(drv_dev, amps_dev, B, K, s.N, s.dt, coef);
  DenseArgs da{};
  da.B = B; da.D = D; da.Dp = Dp; da.S = S; da.K = K; da.R = R; da.G = G; da.N = Nn;
  da.nsteps = s.N; da.frame = s.frame; da.dt = s.dt;
  da.A = A_dev; da.coef = coef; da.E = E_dev; da.cols = cols_dev;
  da.out = static_cast<double2*>(psi_dev); da.err = err; da.wlim = 1 << 22;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0); cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  const cudaError_t le = dense_launch(da, st);
  cudaEventRecord(e1, st);
  if (le != cudaSuccess) { cudaEventDestroy(e0); cudaEventDestroy(e1); return sg_fail(ctx, SG_E_CUDA, cudaGetErrorString(le)); }
  int herr = 0;
  SG_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  SG_CUDA_TRY(ctx, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  SG_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0); cudaEventDestroy(e1);
  s0->last_stats[0] = ms;
  s0->last_stats[1] = 0;
  s0->last_stats[2] = (double)ar.bytes;
  s0->last_stats[3] = 0;
  s0->last_stats[4] = K ? 2 : 1;
  if (herr) return sg_fail(ctx, SG_E_TIMEOUT, "tensor-core batch: a bounded wait for the MMAs ran out");
  return SG_OK;
}
