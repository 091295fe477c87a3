// Device-side plan structures and the shared-memory tile machinery of the
// tiled evolution kernels (slab.cu: one launch per RK4 stage pass; onchip.cu: whole
// evolutions in one launch for single-tile plans).
#pragma once
#include "sg_internal.h"
#include "kplan.h"
#include "grad.cuh"

namespace {

constexpr int kST = 256;          // threads per block
constexpr int kTmax = 4096;       // entries per tile
constexpr int kMaxPass = 4;
constexpr int kSPW = 2;           // cross-density slots per warp
constexpr int kMaxX = kSPW * (kST / 32);
constexpr int kMaxPhase = 12;
constexpr int kMaxDrv = 8;
// Dynamic shared memory a tiled pass may take: the 227 KB opt-in limit of a block
// less 1 KB for the kernels' static shared variables.
constexpr size_t kSlabSmemMax = 226 * 1024;
// The lean passes' dynamic shared-memory limit (their static shared variables take up
// to ~1.5 KB).
constexpr size_t kLeanSmemMax = 200 * 1024;        // drives per pass of the real-operator pulse-gradient adjoint

// One phase of a pass: every thread owns d x d blocks over two tile digits
// (ka, kb) and applies the terms living on them in registers: the edge
// L(ka) (x) R(kb) and up to two 1-body matrices on ka and kb.
struct Phase {
  int ka, kb;
  int offL, offR, offA, offB;   // stage-row offsets (-1: absent)
  int ge, gA, gB;               // global edge index, global 1-body slots of A and B
  unsigned par;                 // bit 0 L, 1 R, 2 A, 3 B parity-odd
  int no;                       // other digits, in thread-mapping order
  int ost[SG_MAXQ];             // their tile strides
  int allpar;                   // every present term is parity-odd
  int psa, psb;                 // padded shared-memory strides of ka and kb
  int pst[SG_MAXQ];             // padded strides of the other digits (mapping order)
};

struct SlabPass {
  int ng, T, ntpc, row;
  int tsh[SG_MAXQ];               // tile stride of tile digit k
  int tlg[SG_MAXQ];               // log2 of tsh when the level count is a power of two
  int no;
  int odim[SG_MAXQ];
  long long ost[SG_MAXQ];
  long long D;
  int S;
  int n1;
  int s1_k[SG_MAXQ], s1_off[SG_MAXQ];
  unsigned par1;
  int ne;
  int e_ka[SG_MAXEDGE], e_kb[SG_MAXEDGE], e_offL[SG_MAXEDGE], e_offR[SG_MAXEDGE];
  unsigned long long parL, parR;
  int nx;                         // cross-density slots: phase, kind (0 A, 1 B, 2 L, 3 R), global id
  int x_ph[kMaxX], x_type[kMaxX], x_gslot[kMaxX];
  int nph;                        // register-blocked phases
  Phase ph[kMaxPhase];
  const int* off;                 // device tile offsets [T]
  int tphoff[SG_MAXQ];            // tile digit k: offset of its mode's levels in a stage's phase row
  int tmode[SG_MAXQ];             // tile digit k: its mode
  // drives whose 1-body slot lies in this pass (real-operator pulse-gradient adjoint):
  // the phase whose blocks carry the slot's digit, on its first (0) or second (1)
  // digit, and the global drive index
  int nd;
  int d_ph[kMaxDrv], d_type[kMaxDrv], d_k[kMaxDrv];
};

// Padded shared-memory position of tile entry t: one pad element per 16 and per
// 256 entries, so that a half-warp whose threads vary over one even-stride and
// one odd-stride base-4 digit touches 16 distinct 8-byte bank pairs.
// For power-of-two level counts the digits of a block base and of an in-block
// offset occupy disjoint bits, so spos(base + o) = spos(base) + spos(o).
template <int DL>
__host__ __device__ __forceinline__ int spos(int t) {
  return (DL == 2 || DL == 4 || DL == 8) ? t + (t >> 4) + (t >> 8) : t;
}
__host__ __device__ constexpr int spad(int T) { return T + (T >> 4) + (T >> 8) + 1; }

// Global -> shared tile copy with NB independent loads in flight per thread.
template <int DL, int NB, typename C>
__device__ __forceinline__ void load_tile(const SlabPass& sp, const C* __restrict__ X, long long base,
                                          const int* __restrict__ off, C* __restrict__ ys) {
  for (int t0 = threadIdx.x; t0 < sp.T; t0 += kST * NB) {
    C v[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const int t = t0 + j * kST;
      v[j] = t < sp.T ? X[base + __ldg(off + t)] : cmk<C>(0.0, 0.0);
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const int t = t0 + j * kST;
      if (t < sp.T) ys[spos<DL>(t)] = v[j];
    }
  }
}

// u[x][z] = sum_c R[z][c] y[x][c]      (apply along the block's second digit)
template <int DL, bool PAR, typename C>
__device__ __forceinline__ void blk_right(const C* __restrict__ Rm, const C (&y)[DL][DL], C (&u)[DL][DL]) {
#pragma unroll
  for (int z = 0; z < DL; ++z) {
    C r[DL];
#pragma unroll
    for (int c = 0; c < DL; ++c) r[c] = (!PAR || ((z + c) & 1)) ? Rm[z * DL + c] : cmk<C>(0.0, 0.0);
#pragma unroll
    for (int x = 0; x < DL; ++x) {
      C a = cmk<C>(0.0, 0.0);
#pragma unroll
      for (int c = 0; c < DL; ++c)
        if (!PAR || ((z + c) & 1)) a = cfma(r[c], y[x][c], a);
      u[x][z] = a;
    }
  }
}
// out[x][z] += sum_a L[x][a] u[a][z]    (apply along the block's first digit)
template <int DL, bool PAR, typename C>
__device__ __forceinline__ void blk_left_acc(const C* __restrict__ Lm, const C (&u)[DL][DL], C (&out)[DL][DL]) {
#pragma unroll
  for (int x = 0; x < DL; ++x) {
    C l[DL];
#pragma unroll
    for (int a = 0; a < DL; ++a) l[a] = (!PAR || ((x + a) & 1)) ? Lm[x * DL + a] : cmk<C>(0.0, 0.0);
#pragma unroll
    for (int z = 0; z < DL; ++z) {
      C acc = out[x][z];
#pragma unroll
      for (int a = 0; a < DL; ++a)
        if (!PAR || ((x + a) & 1)) acc = cfma(l[a], u[a][z], acc);
      out[x][z] = acc;
    }
  }
}
// out[x][z] += sum_c B[z][c] y[x][c]
template <int DL, bool PAR, typename C>
__device__ __forceinline__ void blk_right_acc(const C* __restrict__ Bm, const C (&y)[DL][DL], C (&out)[DL][DL]) {
#pragma unroll
  for (int z = 0; z < DL; ++z) {
    C r[DL];
#pragma unroll
    for (int c = 0; c < DL; ++c) r[c] = (!PAR || ((z + c) & 1)) ? Bm[z * DL + c] : cmk<C>(0.0, 0.0);
#pragma unroll
    for (int x = 0; x < DL; ++x) {
      C a = out[x][z];
#pragma unroll
      for (int c = 0; c < DL; ++c)
        if (!PAR || ((z + c) & 1)) a = cfma(r[c], y[x][c], a);
      out[x][z] = a;
    }
  }
}

// H (restricted to the phase's terms) applied to one d x d block in registers.
template <int DL, typename C>
__device__ __forceinline__ void blk_apply(const Phase& P, const C* __restrict__ M, const C (&y)[DL][DL],
                                          C (&out)[DL][DL]) {
#pragma unroll
  for (int x = 0; x < DL; ++x)
#pragma unroll
    for (int z = 0; z < DL; ++z) out[x][z] = cmk<C>(0.0, 0.0);
  if (P.offL >= 0) {
    C u[DL][DL];
    if (P.par & 2u) blk_right<DL, true>(M + P.offR, y, u);
    else blk_right<DL, false>(M + P.offR, y, u);
    if (P.par & 1u) blk_left_acc<DL, true>(M + P.offL, u, out);
    else blk_left_acc<DL, false>(M + P.offL, u, out);
  }
  if (P.offA >= 0) {
    if (P.par & 4u) blk_left_acc<DL, true>(M + P.offA, y, out);
    else blk_left_acc<DL, false>(M + P.offA, y, out);
  }
  if (P.offB >= 0) {
    if (P.par & 8u) blk_right_acc<DL, true>(M + P.offB, y, out);
    else blk_right_acc<DL, false>(M + P.offB, y, out);
  }
}

// o[x][z] = sum_{a,c} G[(x d + z), (a d + c)] y[a][c] over one block (digits ka, kb): a
// dense two-mode factor (the Suzuki-Trotter coupling unitaries).
template <int DL, typename C>
__device__ __forceinline__ void block_dense(const C* __restrict__ G, const C* __restrict__ ys, C* __restrict__ ks,
                                            int pb, int psa, int psb) {
  C y[DL][DL];
#pragma unroll
  for (int a = 0; a < DL; ++a)
#pragma unroll
    for (int c = 0; c < DL; ++c) y[a][c] = ys[pb + a * psa + c * psb];
  // one output per iteration (a runtime loop keeps the d^4 code small)
#pragma unroll 1
  for (int xz = 0; xz < DL * DL; ++xz) {
    const C* g = G + xz * DL * DL;
    C acc0 = cmk<C>(0.0, 0.0), acc1 = cmk<C>(0.0, 0.0);       // two chains for latency
#pragma unroll
    for (int a = 0; a < DL; ++a)
#pragma unroll
      for (int c = 0; c < DL; ++c) {
        if ((a * DL + c) & 1) acc1 = cfma(g[a * DL + c], y[a][c], acc1);
        else acc0 = cfma(g[a * DL + c], y[a][c], acc0);
      }
    const int x = xz / DL, z = xz - x * DL;
    ks[pb + x * psa + z * psb] = cmk<C>(acc0.x + acc1.x, acc0.y + acc1.y);
  }
}

// Padded shared-memory position of block b's (0, 0) entry: the other digits of b,
// in mapping order, times their padded strides.  For power-of-two level counts
// the padding is linear in each digit (spos(x s) = x spos(s) for a digit x of a
// stride s), so block offsets are x psa + z psb.
template <int DL>
__device__ __forceinline__ int blk_pos(const Phase& P, int b) {
  int pb = 0;
  for (int j = 0; j < P.no; ++j) {
    pb += (b % DL) * P.pst[j];
    b /= DL;
  }
  return pb;
}

// One block of one phase:
//   out[x][z] = sum_a L[x][a] sum_c R[z][c] y[a][c] + sum_a A[x][a] y[a][z] + sum_c B[z][c] y[x][c]
// computed one output column z at a time.  All loads (the y block and, after the
// first phase, the running sum) come first so none waits behind a store to a
// possibly aliasing address.  PAR: every present term is parity-odd, so only index
// pairs of odd sum are visited.
template <int DL, bool PAR, typename C>
__device__ __forceinline__ void phase_block(const Phase& P, const C* __restrict__ M, const C* __restrict__ ys,
                                            C* __restrict__ ks, int pb, const bool FIRST) {
  const int psa = P.psa, psb = P.psb;
  C y[DL][DL], o[DL][DL];
#pragma unroll
  for (int x = 0; x < DL; ++x)
#pragma unroll
    for (int z = 0; z < DL; ++z) {
      y[x][z] = ys[pb + x * psa + z * psb];
      o[x][z] = FIRST ? cmk<C>(0.0, 0.0) : ks[pb + x * psa + z * psb];
    }
  const C* Lm = M + P.offL;
  const C* Rm = M + P.offR;
  const C* Am = M + P.offA;
  const C* Bm = M + P.offB;
  const bool hasE = P.offL >= 0, hasA = P.offA >= 0, hasB = P.offB >= 0;
#pragma unroll
  for (int z = 0; z < DL; ++z) {
    if (hasE) {
      C u[DL];
#pragma unroll
      for (int a = 0; a < DL; ++a) {
        C acc = cmk<C>(0.0, 0.0);
#pragma unroll
        for (int c = 0; c < DL; ++c)
          if (!PAR || ((z + c) & 1)) acc = cfma(Rm[z * DL + c], y[a][c], acc);
        u[a] = acc;
      }
#pragma unroll
      for (int x = 0; x < DL; ++x)
#pragma unroll
        for (int a = 0; a < DL; ++a)
          if (!PAR || ((x + a) & 1)) o[x][z] = cfma(Lm[x * DL + a], u[a], o[x][z]);
    }
    if (hasA) {
#pragma unroll
      for (int x = 0; x < DL; ++x)
#pragma unroll
        for (int a = 0; a < DL; ++a)
          if (!PAR || ((x + a) & 1)) o[x][z] = cfma(Am[x * DL + a], y[a][z], o[x][z]);
    }
    if (hasB) {
#pragma unroll
      for (int x = 0; x < DL; ++x)
#pragma unroll
        for (int c = 0; c < DL; ++c)
          if (!PAR || ((z + c) & 1)) o[x][z] = cfma(Bm[z * DL + c], y[x][c], o[x][z]);
    }
  }
#pragma unroll
  for (int x = 0; x < DL; ++x)
#pragma unroll
    for (int z = 0; z < DL; ++z) ks[pb + x * psa + z * psb] = o[x][z];
}

// Applies every phase of the pass to the tile in ys, leaving H y (restricted to
// the pass's terms) in ks.  Ends with a barrier.
template <int DL, typename C>
__device__ __forceinline__ void pass_apply(const SlabPass& sp, const C* __restrict__ M,
                                           const C* __restrict__ ys, C* __restrict__ ks) {
  const int nb = sp.T / (DL * DL);
  for (int q = 0; q < sp.nph; ++q) {
    const Phase& P = sp.ph[q];
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
      const int pb = blk_pos<DL>(P, b);
      if (P.allpar) phase_block<DL, true>(P, M, ys, ks, pb, q == 0);
      else phase_block<DL, false>(P, M, ys, ks, pb, q == 0);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ long long tile_base(const SlabPass& sp, long long tile) {
  const long long col = tile / sp.ntpc;
  long long rest = tile - col * sp.ntpc;
  long long b = col * sp.D;
  for (int k = sp.no - 1; k >= 0; --k) {
    const int dk = sp.odim[k];
    b += (rest % dk) * sp.ost[k];
    rest /= dk;
  }
  return b;
}

template <typename C>
__device__ __forceinline__ void load_common(const SlabPass& sp, const C* __restrict__ tabrow, C* M) {
  for (int i = threadIdx.x; i < sp.row; i += blockDim.x) M[i] = tabrow[i];
  __syncthreads();
}

// Cross-density accumulators of one slot.  With PARX every operator of the plan is
// parity-odd and only entries with a + b odd are kept (the others multiply zeros in
// the contraction), packed in row-major order.
template <int DL, bool PARX> __host__ __device__ constexpr int xd_n() { return PARX ? (DL * DL) / 2 : DL * DL; }
template <int DL, bool PARX> __host__ __device__ constexpr int xd_i(int a, int b) {
  if (!PARX) return a * DL + b;
  int n = 0;
  for (int i = 0; i < a * DL + b; ++i) n += ((i / DL) + (i % DL)) & 1;
  return n;
}

// Cross-density of one slot over one d x d block (x = kbar block, y = y_s block),
// streamed from shared memory a column or a row at a time:
//   A (1-body on ka):  C[a][b] += sum_z conj(x[a][z]) y[b][z]
//   B (1-body on kb):  C[c][d] += sum_x conj(x[x][c]) y[x][d]
//   L (edge, ka):      C[a][b] += sum_z conj(x[a][z]) u[b][z],  u[b][z] = sum_c R[z][c] y[b][c]
//   R (edge, kb):      C[c][d] += sum_x conj(x[x][c]) v[x][d],  v[x][d] = sum_a L[x][a] y[a][d]
template <int DL, bool PARX, typename C>
__device__ __forceinline__ void xd_slot(const Phase& P, int type, const C* __restrict__ M,
                                        const C* __restrict__ xs, const C* __restrict__ ys, int pb,
                                        C (&acc)[xd_n<DL, PARX>()]) {
  const int psa = P.psa, psb = P.psb;
  if (type == 0 || type == 1) {
#pragma unroll
    for (int z = 0; z < DL; ++z) {
      C xc[DL], yc[DL];
#pragma unroll
      for (int a = 0; a < DL; ++a) {
        const int o = type == 0 ? a * psa + z * psb : z * psa + a * psb;
        xc[a] = xs[pb + o];
        yc[a] = ys[pb + o];
      }
#pragma unroll
      for (int a = 0; a < DL; ++a)
#pragma unroll
        for (int b = 0; b < DL; ++b) {
          if (PARX && !((a + b) & 1)) continue;
          acc[xd_i<DL, PARX>(a, b)] = cjfma(xc[a], yc[b], acc[xd_i<DL, PARX>(a, b)]);
        }
    }
    return;
  }
  C y[DL][DL];
#pragma unroll
  for (int a = 0; a < DL; ++a)
#pragma unroll
    for (int b = 0; b < DL; ++b) y[a][b] = ys[pb + a * psa + b * psb];
  if (type == 2) {
    const C* Rm = M + P.offR;
#pragma unroll
    for (int z = 0; z < DL; ++z) {
      C u[DL], xc[DL];
#pragma unroll
      for (int b = 0; b < DL; ++b) {
        C t = cmk<C>(0.0, 0.0);
#pragma unroll
        for (int c = 0; c < DL; ++c)
          if (!PARX || ((z + c) & 1)) t = cfma(Rm[z * DL + c], y[b][c], t);
        u[b] = t;
        xc[b] = xs[pb + b * psa + z * psb];
      }
#pragma unroll
      for (int a = 0; a < DL; ++a)
#pragma unroll
        for (int b = 0; b < DL; ++b) {
          if (PARX && !((a + b) & 1)) continue;
          acc[xd_i<DL, PARX>(a, b)] = cjfma(xc[a], u[b], acc[xd_i<DL, PARX>(a, b)]);
        }
    }
  } else {
    const C* Lm = M + P.offL;
#pragma unroll
    for (int x = 0; x < DL; ++x) {
      C v[DL], xr[DL];
#pragma unroll
      for (int d = 0; d < DL; ++d) {
        C t = cmk<C>(0.0, 0.0);
#pragma unroll
        for (int a = 0; a < DL; ++a)
          if (!PARX || ((x + a) & 1)) t = cfma(Lm[x * DL + a], y[a][d], t);
        v[d] = t;
        xr[d] = xs[pb + x * psa + d * psb];
      }
#pragma unroll
      for (int c = 0; c < DL; ++c)
#pragma unroll
        for (int d = 0; d < DL; ++d) {
          if (PARX && !((c + d) & 1)) continue;
          acc[xd_i<DL, PARX>(c, d)] = cjfma(xr[c], v[d], acc[xd_i<DL, PARX>(c, d)]);
        }
    }
  }
}

// Host: a phase over tile digits (ka, kb) of a single-pass plan with no terms set
// (offsets -1): the other digits in the bank-conflict-free mapping order (the lowest
// even-exponent digit, the lowest odd-exponent one, then the rest) and the padded
// shared-memory strides.  The tiled plans build their phases the same way.
inline Phase make_phase(const SlabPass& sp, int DL, int ka, int kb) {
  Phase P{};
  P.ka = ka;
  P.kb = kb;
  P.offL = P.offR = P.offA = P.offB = -1;
  P.ge = P.gA = P.gB = -1;
  P.par = 0;
  P.allpar = 0;
  int ord[SG_MAXQ], no = 0;
  const int ng = sp.ng;
  for (int pass = 0; pass < 3; ++pass)
    for (int k = ng - 1; k >= 0; --k) {
      if (k == ka || k == kb) continue;
      bool used = false;
      for (int j = 0; j < no; ++j) used = used || ord[j] == k;
      if (used) continue;
      const int ex = ng - 1 - k;
      if (pass == 0 && ex % 2 != 0) continue;
      if (pass == 1 && ex % 2 != 1) continue;
      ord[no++] = k;
      if (pass < 2) break;
    }
  const bool pw2 = DL == 2 || DL == 4;
  auto pad = [&](int o) { return pw2 ? o + (o >> 4) + (o >> 8) : o; };
  P.no = no;
  for (int j = 0; j < no; ++j) {
    P.ost[j] = sp.tsh[ord[j]];
    P.pst[j] = pad(P.ost[j]);
  }
  P.psa = pad(sp.tsh[ka]);
  P.psb = pad(sp.tsh[kb]);
  return P;
}

// ---------------------------------------------------------------------------
// Real-operator phases.  In the interaction frame a local operator is
// X(t) = P(t) X_r P(t)^dag with P = diag(exp(i E t)) on its mode; in the truncated
// eigenbasis X_r is real, or i times a real matrix, and the two factors of a
// coupling then multiply to a real term.  The terms of one pass act only on the
// pass's mode group G, so their sum is P_G(t) H_r(t) P_G(t)^dag with P_G the product
// of the group's phases (the other modes' phases cancel), and a pass computes
//     H y = P_G (H_r (P_G^dag y))
// with one phase rotation per tile entry on the way in and one on the way out, and
// real matrix elements times complex amplitudes in between: half the multiply-adds
// of the complex form, and in FP32 one packed two-lane FMA per element (the real
// element duplicated in both lanes, the amplitude's real and imaginary parts in the
// two lanes).
//
// Table layout (one stage row, the complex row's offsets): a d x d block per term,
// row x holding the stored elements of row x; a parity-odd operator stores only its
// columns c with x + c odd, in increasing order, in the first d/2 places of the row.
// ---------------------------------------------------------------------------
template <typename R> struct ZM;
template <> struct ZM<float> { typedef float2 T; };     // {m, m}
template <> struct ZM<double> { typedef double T; };

__device__ __forceinline__ float2 zfma(float2 m, float2 y, float2 o) { return __ffma2_rn(m, y, o); }
__device__ __forceinline__ double2 zfma(double m, double2 y, double2 o) {
  return make_double2(fma(m, y.x, o.x), fma(m, y.y, o.y));
}
template <bool PAR> __host__ __device__ constexpr int zcol(int x, int k) { return PAR ? ((x + 1) & 1) + 2 * k : k; }
template <int DL, bool PAR> __host__ __device__ constexpr int znz() { return PAR ? DL / 2 : DL; }

// The stored elements of one row (NZ consecutive elements, 16-byte aligned when
// the row offset is a multiple of the row length; FP32 loads them as float4 pairs).
template <int NZ>
__device__ __forceinline__ void zrow_ld(const float2* __restrict__ p, float2 (&r)[NZ]) {
  if constexpr (NZ % 2 == 0) {
#pragma unroll
    for (int k = 0; k < NZ; k += 2) {
      const float4 v = *reinterpret_cast<const float4*>(p + k);
      r[k] = make_float2(v.x, v.y);
      r[k + 1] = make_float2(v.z, v.w);
    }
  } else {
#pragma unroll
    for (int k = 0; k < NZ; ++k) r[k] = p[k];
  }
}
template <int NZ>
__device__ __forceinline__ void zrow_ld(const double* __restrict__ p, double (&r)[NZ]) {
#pragma unroll
  for (int k = 0; k < NZ; ++k) r[k] = p[k];
}

// One block of one phase with real matrices (the operation of phase_block):
//   out[x][z] (+)= sum_a L[x][a] sum_c R[z][c] y[a][c] + sum_a A[x][a] y[a][z] + sum_c B[z][c] y[x][c]
// FL: bit 0 edge L (x) R, bit 1 A on ka, bit 2 B on kb, bit 3 first phase (no running sum).
template <int DL, bool PAR, int FL, typename R>
__device__ __forceinline__ void zphase_block(const Phase& P, const typename ZM<R>::T* __restrict__ M,
                                             const typename CT<R>::T* __restrict__ ys,
                                             typename CT<R>::T* __restrict__ ks, int pb) {
  typedef typename CT<R>::T C;
  typedef typename ZM<R>::T Z;
  constexpr bool HE = FL & 1, HA = (FL >> 1) & 1, HB = (FL >> 2) & 1, FIRST = (FL >> 3) & 1;
  constexpr int NZ = znz<DL, PAR>();
  const int psa = P.psa, psb = P.psb;
  C y[DL][DL];
#pragma unroll
  for (int x = 0; x < DL; ++x)
#pragma unroll
    for (int z = 0; z < DL; ++z) y[x][z] = ys[pb + x * psa + z * psb];
  Z l[DL][NZ];
  if constexpr (HE) {
#pragma unroll
    for (int x = 0; x < DL; ++x) zrow_ld<NZ>(M + P.offL + x * DL, l[x]);
  }
#pragma unroll
  for (int z = 0; z < DL; ++z) {
    C o[DL];
#pragma unroll
    for (int x = 0; x < DL; ++x) o[x] = FIRST ? cmk<C>(0.0, 0.0) : ks[pb + x * psa + z * psb];
    if constexpr (HE) {
      Z r[NZ];
      zrow_ld<NZ>(M + P.offR + z * DL, r);
      C u[DL];
#pragma unroll
      for (int aa = 0; aa < DL; ++aa) {
        C t = cmk<C>(0.0, 0.0);
#pragma unroll
        for (int k = 0; k < NZ; ++k) t = zfma(r[k], y[aa][zcol<PAR>(z, k)], t);
        u[aa] = t;
      }
#pragma unroll
      for (int x = 0; x < DL; ++x)
#pragma unroll
        for (int k = 0; k < NZ; ++k) o[x] = zfma(l[x][k], u[zcol<PAR>(x, k)], o[x]);
    }
    if constexpr (HA) {
#pragma unroll
      for (int x = 0; x < DL; ++x) {
        Z a[NZ];
        zrow_ld<NZ>(M + P.offA + x * DL, a);
#pragma unroll
        for (int k = 0; k < NZ; ++k) o[x] = zfma(a[k], y[zcol<PAR>(x, k)][z], o[x]);
      }
    }
    if constexpr (HB) {
      Z b[NZ];
      zrow_ld<NZ>(M + P.offB + z * DL, b);
#pragma unroll
      for (int x = 0; x < DL; ++x)
#pragma unroll
        for (int k = 0; k < NZ; ++k) o[x] = zfma(b[k], y[x][zcol<PAR>(z, k)], o[x]);
    }
#pragma unroll
    for (int x = 0; x < DL; ++x) ks[pb + x * psa + z * psb] = o[x];
  }
}

template <int DL, bool PAR, int FL, typename R>
__device__ __forceinline__ void zphase_all(const Phase& P, const typename ZM<R>::T* __restrict__ M,
                                           const typename CT<R>::T* __restrict__ ys,
                                           typename CT<R>::T* __restrict__ ks, int nb, int nthr) {
  for (int b = threadIdx.x; b < nb; b += nthr) zphase_block<DL, PAR, FL, R>(P, M, ys, ks, blk_pos<DL>(P, b));
}

// Named barriers: bar.sync waits for `n` threads (arrivals included), bar.arrive
// counts this thread's warp without waiting; both order the shared-memory accesses
// before them for the threads the barrier completes.  id 0 is __syncthreads.
__device__ __forceinline__ void nb_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void nb_arrive(int id, int n) {
  asm volatile("bar.arrive %0, %1;\n" ::"r"(id), "r"(n) : "memory");
}

// ks = H_r ys over every phase of the pass (threads [0, nthr)); every phase ends
// with a barrier among those threads (__syncthreads when bar_id is 0).
template <int DL, bool PAR, typename R>
__device__ __forceinline__ void zpass_apply(const SlabPass& sp, const typename ZM<R>::T* __restrict__ M,
                                            const typename CT<R>::T* __restrict__ ys,
                                            typename CT<R>::T* __restrict__ ks, int nthr, int bar_id = 0) {
  const int nb = sp.T / (DL * DL);
  for (int q = 0; q < sp.nph; ++q) {
    const Phase& P = sp.ph[q];
    const int fl = (P.offL >= 0 ? 1 : 0) | (P.offA >= 0 ? 2 : 0) | (P.offB >= 0 ? 4 : 0) | (q == 0 ? 8 : 0);
    switch (fl) {
#define SG_ZCASE(F) case F: zphase_all<DL, PAR, F, R>(P, M, ys, ks, nb, nthr); break;
      SG_ZCASE(1) SG_ZCASE(2) SG_ZCASE(3) SG_ZCASE(4) SG_ZCASE(5) SG_ZCASE(6) SG_ZCASE(7)
      SG_ZCASE(9) SG_ZCASE(10) SG_ZCASE(11) SG_ZCASE(12) SG_ZCASE(13) SG_ZCASE(14) SG_ZCASE(15)
#undef SG_ZCASE
      default: break;
    }
    if (bar_id == 0) __syncthreads();
    else nb_sync(bar_id, nthr);
  }
}

// Phase factors of the tile entries at one stage: entry t = l + L h (L = min(T, 256))
// has P_G(t) = lo[l] hi[h], each the product of exp(i E t) over the group digits in
// that part of t.  Computed in FP64 from the stage's phase row, stored in R.
template <int DL, typename C>
__device__ __forceinline__ void zphase_tables(const SlabPass& sp, const double2* __restrict__ phrow, C* lo, C* hi) {
  const int L = sp.T < 256 ? sp.T : 256;
  for (int i = threadIdx.x; i < L + sp.T / L; i += blockDim.x) {
    const bool is_lo = i < L;
    const int v = is_lo ? i : (i - L) * L;       // tile index whose part this is
    double pr = 1.0, pi = 0.0;
    for (int k = 0; k < sp.ng; ++k) {
      if ((sp.tsh[k] < L) != is_lo) continue;
      const double2 e = phrow[sp.tphoff[k] + (v / sp.tsh[k]) % DL];
      const double nr = pr * e.x - pi * e.y, ni = pr * e.y + pi * e.x;
      pr = nr;
      pi = ni;
    }
    if (is_lo) lo[i] = cmk<C>(pr, pi); else hi[i - L] = cmk<C>(pr, pi);
  }
}
template <typename C> __device__ __forceinline__ C zcmul(C a, C b) {
  return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C zcmulc(C a, C b) {     // conj(a) b
  return cmk<C>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

struct PermArgs {
  int nq, S;
  long long D;
  int dims[SG_MAXQ];
  long long st_api[SG_MAXQ], st_int[SG_MAXQ];
};

}  // namespace

struct SlabPlanHost {
  int DL = 0, np = 0;
  bool allpar = false;             // every phase of every pass is parity-odd
  cudaStream_t st = nullptr;       // stream the offset tables were allocated on
  bool mixed = false;
  SlabPass pass[kMaxPass];
  int* off_dev[kMaxPass] = {nullptr, nullptr, nullptr, nullptr};
  PermArgs perm{};
  int grid_fwd = 0, grid_adj = 0;
  size_t sm_fwd[kMaxPass] = {0}, sm_adj[kMaxPass] = {0};
  // real-operator forward passes (bound by slab_bind_real)
  const void* ztab = nullptr;
  const double2* zph = nullptr;
  int zsumd = 0;
  int grid_zfwd = 0;
  size_t sm_zfwd[kMaxPass] = {0};
  size_t sm_zws[kMaxPass] = {0};   // warp-specialised FP32 pass (0: not usable for this pass)
  // real-operator pulse-gradient adjoint (bound by slab_bind_real when every pass has
  // at most kMaxDrv drives): the drive operators' real matrices, K x DL x DL
  const void* zop = nullptr;
  bool zadj = false;
  size_t sm_zadj[kMaxPass] = {0};
  // Suzuki-Trotter products on the tiles (slab_q2.cu): the factor lists of the two
  // passes of a sub-step (nullptr: not supported for this plan)
  struct SQPlan* q2 = nullptr;
  // lean FP32 passes (slab_lean.cuh): 4 levels, parity-odd, passes whose tiles hold
  // 4096 entries (each pass picks its kernel on its own)
  bool lean[kMaxPass] = {false, false, false, false};
  size_t sm_lean = 0, sm_lean_adj = 0;
};

// Byte offset of the real-operator row in the shared memory of k_zslab_fwd: after
// `ntile` tiles (2, or 4 for the double-buffered kernel) and the phase parts (256
// low, T / 256 high), 16-byte aligned.
__host__ __device__ inline size_t zrow_smem_off(int T, size_t csz, int ntile = 2) {
  const int nhi = T > 256 ? T / 256 : 1;
  return (((size_t)ntile * spad(T) + 256 + nhi) * csz + 15) & ~(size_t)15;
}

// Instantiates FN<R, DL> for the plan's precision and level count.
#define SLAB_DISPATCH(FN, ...)                                                              \
  do {                                                                                      \
    if (mixed) {                                                                            \
      switch (h->DL) {                                                                      \
        case 2: return FN<float, 2>(__VA_ARGS__);                                          \
        case 3: return FN<float, 3>(__VA_ARGS__);                                          \
        case 4: return FN<float, 4>(__VA_ARGS__);                                          \
        default: return FN<float, 5>(__VA_ARGS__);                                         \
      }                                                                                     \
    } else {                                                                                \
      switch (h->DL) {                                                                      \
        case 2: return FN<double, 2>(__VA_ARGS__);                                         \
        case 3: return FN<double, 3>(__VA_ARGS__);                                         \
        case 4: return FN<double, 4>(__VA_ARGS__);                                         \
        default: return FN<double, 5>(__VA_ARGS__);                                        \
      }                                                                                     \
    }                                                                                       \
  } while (0)
