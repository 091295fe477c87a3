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
};
