// Suzuki-Trotter products (Sec. 2.3, App. A) on the tiled kernels (see slab.h).
//
// Q2 over one sub-step applies, in order, the first half of every mode's 1-body factor,
// the couplings 0 .. ne-2 over half the sub-step, coupling ne-1 over the whole of it,
// the couplings ne-2 .. 0 over half again, and the second half of the 1-body factors
// (the on-chip kernel merges the second half of one sub-step with the first half of the
// next into one row of the table).  With two mode groups G1, G2 whose couplings E1 come
// before E2 in term order, factors on disjoint modes commute, so one sub-step m is two
// passes over the state:
//   pass A (tiles of G1):  E1 reversed (half, sub-step m-1), merged row of G1's modes,
//                          E1 forward (half, sub-step m)
//   pass B (tiles of G2):  merged row of the modes of G2 outside G1, E2 forward (half),
//                          coupling ne-1 (full), E2 reversed (half)
// and after the last sub-step pass A without E1 forward and pass B with the row alone.
// The first-order product Q1 (each term once per step, full-step factors; the tables'
// row m holds step m + 1's 1-body factors) is one pass of each kind per step:
//   pass A:  row of G1's modes, E1 (full step, term order)
//   pass B:  row of the modes of G2 outside G1, E2 (full step, term order)
// (G2's other modes' factors commute with E1, so this is the step's term order).
// Each pass loads a tile, applies its factors in shared memory (one block of d x d
// entries per thread and factor) and writes the tile back in place.
#include "sg_internal.h"
#include "kplan.h"
#include "grad.cuh"
#include "slab.h"
#include "slab_dev.cuh"
#include <algorithm>
#include <cstdlib>
#include <utility>
#include <vector>

namespace {

constexpr int kMaxSQ = 24;
struct SQFactor {
  Phase P;                  // block digits (ka, kb); kind 0: rows offL, offR; kind 1: offA
  int kind;                 // 0: two modes' 1-body factors L (x) R, 1: one mode's, 2: a coupling (dense)
  int mat;                  // kind 2: 2 e (half step) or 2 e + 1 (full step)
  int prev;                 // kind 2: from the previous sub-step's coupling set
  int spar;                 // kind 2: both factors parity-odd, so the unitary keeps the parity of
                            // the two levels' sum and half its entries are zero
};
struct SQList {
  int nf, ndense;
  SQFactor f[kMaxSQ];
};

// block_dense for a coupling unitary that keeps the parity of a + c (exp of A (x) B with
// A and B parity-odd): output (x, z) reads only the inputs (a, c) with a + c = x + z mod 2.
template <int DL, typename C>
__device__ __forceinline__ void block_dense_sp(const C* __restrict__ G, const C* __restrict__ ys,
                                               C* __restrict__ ks, int pb, int psa, int psb) {
  C y[DL][DL];
#pragma unroll
  for (int a = 0; a < DL; ++a)
#pragma unroll
    for (int c = 0; c < DL; ++c) y[a][c] = ys[pb + a * psa + c * psb];
#pragma unroll
  for (int par = 0; par < 2; ++par) {
#pragma unroll 1
    for (int xz = 0; xz < DL * DL; ++xz) {
      const int x = xz / DL, z = xz - x * DL;
      if (((x + z) & 1) != par) continue;
      const C* g = G + xz * DL * DL;
      C acc0 = cmk<C>(0.0, 0.0), acc1 = cmk<C>(0.0, 0.0);
#pragma unroll
      for (int a = 0; a < DL; ++a)
#pragma unroll
        for (int c = 0; c < DL; ++c) {
          if (((a + c) & 1) != par) continue;
          if (a & 1) acc1 = cfma(g[a * DL + c], y[a][c], acc1);
          else acc0 = cfma(g[a * DL + c], y[a][c], acc0);
        }
      ks[pb + x * psa + z * psb] = cmk<C>(acc0.x + acc1.x, acc0.y + acc1.y);
    }
  }
}

template <typename R, int DL>
__global__ void __launch_bounds__(kST, sizeof(R) == 4 ? 2 : 1)
k_slab_q2(SlabPass sp, SQList fl, const typename CT<R>::T* __restrict__ row,
          const typename CT<R>::T* __restrict__ edges, int so_prev, int so_cur, int nrow,
          typename CT<R>::T* __restrict__ X) {
  typedef typename CT<R>::T C;
  constexpr int D4 = DL * DL * DL * DL;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* ys = reinterpret_cast<C*>(smraw);
  C* ks = ys + spad(sp.T);
  C* M = ks + spad(sp.T);                         // the sub-step's merged 1-body row
  C* G = M + nrow;                                // the list's coupling factors, in list order
  for (int i = threadIdx.x; i < nrow; i += blockDim.x) M[i] = row[i];
  {
    int g = 0;
    for (int q = 0; q < fl.nf; ++q) {
      if (fl.f[q].kind != 2) continue;
      const C* src = edges + (size_t)(fl.f[q].mat + (fl.f[q].prev ? so_prev : so_cur)) * D4;
      for (int i = threadIdx.x; i < D4; i += blockDim.x) G[(size_t)g * D4 + i] = src[i];
      ++g;
    }
  }
  __syncthreads();
  const long long ntiles = (long long)sp.S * sp.ntpc;
  const int nb = sp.T / (DL * DL);
  const int* __restrict__ off = sp.off;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long base = tile_base(sp, tile);
    load_tile<DL, 8>(sp, X, base, off, ys);
    __syncthreads();
    int g = 0;
    for (int q = 0; q < fl.nf; ++q) {
      const SQFactor& F = fl.f[q];
      for (int b = threadIdx.x; b < nb; b += kST) {
        const int pb = blk_pos<DL>(F.P, b);
        if (F.kind == 2) {
          if (F.spar) block_dense_sp<DL>(G + (size_t)g * D4, ys, ks, pb, F.P.psa, F.P.psb);
          else block_dense<DL>(G + (size_t)g * D4, ys, ks, pb, F.P.psa, F.P.psb);
        }
        else phase_block<DL, false>(F.P, M, ys, ks, pb, true);
      }
      g += F.kind == 2 ? 1 : 0;
      __syncthreads();
      C* t = ys; ys = ks; ks = t;
    }
    for (int t = threadIdx.x; t < sp.T; t += kST) X[base + __ldg(off + t)] = ys[spos<DL>(t)];
    __syncthreads();
  }
}

// Pulse gradient on the tiles (Sec. 2.5 on the product): at a point of the backward
// sequence where the 1-body factors U_i(s) of a group's modes have just been undone
// (states psi <- U^-1 psi, co-states lambda <- U^dag lambda), every drive k on such a mode i
// adds Re <lambda, M_k(s) psi> = Re sum_ab M_k[a][b] sum conj(lambda[a, ..]) psi[b, ..] to
// dF/df_k(s), M_k(s) = U_i(s)^-1 L_k(s) from the gradient tables.  Each thread contracts
// its blocks' cross-densities at once; per drive the block sums in fixed order, the CTAs'
// partials in CTA order by the last CTA to finish (ticket), into gF[s K + k].
constexpr int kSQDrv = 16;
// dynamic shared memory of the contraction kernel: below the tiled kernels' cap by its
// static reduction buffer, so that the two together stay within a CTA's shared memory
constexpr size_t kXdSmemMax = kSlabSmemMax - 4096;
struct SQDList {
  int nd;
  int k[kSQDrv];                  // drive index
  Phase P[kSQDrv];                // block layout of the drive's mode: its digit first
};

template <typename R, int DL>
__global__ void __launch_bounds__(kST, 1)
k_slab_q2_xd(SlabPass sp, SQDList dl, const typename CT<R>::T* __restrict__ X,
             const typename CT<R>::T* __restrict__ Lb, const typename CT<R>::T* __restrict__ Mk, int nq,
             double* __restrict__ gpart, unsigned* __restrict__ ticket, double* __restrict__ gFs) {
  typedef typename CT<R>::T C;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* xs = reinterpret_cast<C*>(smraw);            // psi
  C* xb = xs + spad(sp.T);                        // lambda
  C* Ms = xb + spad(sp.T);                        // the drives' M_k, in list order
  __shared__ double red[kST / 32][kSQDrv];
  __shared__ bool last;
  const int tid = threadIdx.x;
  for (int i = tid; i < dl.nd * DL * DL; i += blockDim.x)
    Ms[i] = Mk[(size_t)(2 * nq + dl.k[i / (DL * DL)]) * DL * DL + i % (DL * DL)];
  R g[kSQDrv];
#pragma unroll
  for (int j = 0; j < kSQDrv; ++j) g[j] = R(0);
  __syncthreads();
  const long long ntiles = (long long)sp.S * sp.ntpc;
  const int nb = sp.T / (DL * DL);
  const int* __restrict__ off = sp.off;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long base = tile_base(sp, tile);
    load_tile<DL, 8>(sp, X, base, off, xs);
    load_tile<DL, 8>(sp, Lb, base, off, xb);
    __syncthreads();
    for (int j = 0; j < dl.nd; ++j) {
      const Phase& P = dl.P[j];
      const C* M = Ms + j * DL * DL;
      R v = R(0);
      for (int b = tid; b < nb; b += kST) {
        C acc[DL * DL];
#pragma unroll
        for (int a = 0; a < DL * DL; ++a) acc[a] = cmk<C>(0.0, 0.0);
        xd_slot<DL, false>(P, 0, M, xb, xs, blk_pos<DL>(P, b), acc);
#pragma unroll
        for (int ab = 0; ab < DL * DL; ++ab) v += M[ab].x * acc[ab].x - M[ab].y * acc[ab].y;
      }
#pragma unroll
      for (int i = 0; i < kSQDrv; ++i)
        if (i == j) g[i] += v;
    }
    __syncthreads();
  }
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int j = 0; j < kSQDrv; ++j) {
    if (j < dl.nd) {
      double v = (double)g[j];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][j] = v;
    }
  }
  __syncthreads();
  if (tid < dl.nd) {
    double v = 0.0;
    for (int w = 0; w < kST / 32; ++w) v += red[w][tid];
    gpart[(size_t)blockIdx.x * kSQDrv + tid] = v;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  if (tid < dl.nd) {
    double v = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) v += __ldcg(gpart + (size_t)b * kSQDrv + tid);
    gFs[dl.k[tid]] += v;
  }
  __syncthreads();
  if (tid == 0) *ticket = 0u;                     // ready for the next launch on the stream
}

// The backward of one pass of one sub-step in one launch: states and co-states tiled
// side by side, the pass's pull-back factors applied to both in shared memory (kind 0/1:
// 1-body rows of sub-step s0, or s1 when prev; kind 2: the pull-back set so0, or so1 when
// prev; states by the inverse, co-states by the adjoint) and at each contraction point
// (kind 3, mat = point 0 or 1) the drives' U^-1 L_k of sub-step s0 or s1 contracted with
// the cross-densities, so a pass reads and writes the two slabs once.  Reduction as in
// k_slab_q2_xd, into gF0 and gF1.
template <typename R, int DL>
__global__ void __launch_bounds__(kST, 1)
k_slab_q2_bwd(SlabPass sp, SQList fl, SQDList dl, const typename CT<R>::T* __restrict__ rows0,
              const typename CT<R>::T* __restrict__ rows1, const typename CT<R>::T* __restrict__ Ep, int so0,
              int so1, int nq, typename CT<R>::T* __restrict__ X, typename CT<R>::T* __restrict__ Lb,
              double* __restrict__ gpart, unsigned* __restrict__ ticket, double* __restrict__ gF0,
              double* __restrict__ gF1) {
  typedef typename CT<R>::T C;
  constexpr int D4 = DL * DL * DL * DL;
  constexpr int D2 = DL * DL;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int TP = spad(sp.T), nrow = nq * D2;
  C* ys = reinterpret_cast<C*>(smraw);            // states
  C* ks = ys + TP;
  C* yb = ks + TP;                                // co-states
  C* kb = yb + TP;
  C* Mr = kb + TP;                                // rows: s0 U^-1, s0 U^dag, s1 U^-1, s1 U^dag
  C* Mk = Mr + 4 * nrow;                          // M_k of the pass's drives: s0, then s1
  C* G = Mk + 2 * kSQDrv * D2;                    // per coupling factor: inverse, adjoint
  __shared__ double red[kST / 32][2 * kSQDrv];
  __shared__ bool last;
  const int tid = threadIdx.x;
  for (int i = tid; i < 2 * nrow; i += blockDim.x) {
    Mr[i] = rows0[i];
    Mr[2 * nrow + i] = rows1[i];
  }
  for (int i = tid; i < dl.nd * D2; i += blockDim.x) {
    const size_t o = (size_t)(2 * nq + dl.k[i / D2]) * D2 + i % D2;
    Mk[i] = rows0[o];
    Mk[kSQDrv * D2 + i] = rows1[o];
  }
  {
    int g = 0;
    for (int q = 0; q < fl.nf; ++q) {
      if (fl.f[q].kind != 2) continue;
      const C* src = Ep + (size_t)(fl.f[q].mat + (fl.f[q].prev ? so1 : so0)) * D4;
      for (int i = tid; i < D4; i += blockDim.x) {
        G[(size_t)(2 * g) * D4 + i] = src[i];
        G[(size_t)(2 * g + 1) * D4 + i] = src[2 * D4 + i];
      }
      ++g;
    }
  }
  R gv[2][kSQDrv];
#pragma unroll
  for (int pt = 0; pt < 2; ++pt)
#pragma unroll
    for (int j = 0; j < kSQDrv; ++j) gv[pt][j] = R(0);
  __syncthreads();
  const long long ntiles = (long long)sp.S * sp.ntpc;
  const int nb = sp.T / D2;
  const int* __restrict__ off = sp.off;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long base = tile_base(sp, tile);
    load_tile<DL, 8>(sp, X, base, off, ys);
    load_tile<DL, 8>(sp, Lb, base, off, yb);
    __syncthreads();
    int g = 0;
    for (int q = 0; q < fl.nf; ++q) {
      const SQFactor& F = fl.f[q];
      if (F.kind == 3) {
        const int pt = F.mat;
        for (int j = 0; j < dl.nd; ++j) {
          const Phase& P = dl.P[j];
          const C* M = Mk + (pt * kSQDrv + j) * D2;
          R v = R(0);
          for (int b = tid; b < nb; b += kST) {
            C acc[D2];
#pragma unroll
            for (int a = 0; a < D2; ++a) acc[a] = cmk<C>(0.0, 0.0);
            xd_slot<DL, false>(P, 0, M, yb, ys, blk_pos<DL>(P, b), acc);
#pragma unroll
            for (int ab = 0; ab < D2; ++ab) v += M[ab].x * acc[ab].x - M[ab].y * acc[ab].y;
          }
#pragma unroll
          for (int i = 0; i < kSQDrv; ++i) {
            if (i == j) {
              if (pt == 0) gv[0][i] += v;
              else gv[1][i] += v;
            }
          }
        }
        continue;                                 // read-only: the next factor's barrier orders it
      }
      const C* Mi = Mr + (F.prev ? 2 * nrow : 0);
      for (int b = tid; b < nb; b += kST) {
        const int pb = blk_pos<DL>(F.P, b);
        if (F.kind == 2) {
          const C* Gi = G + (size_t)(2 * g) * D4;
          if (F.spar) {
            block_dense_sp<DL>(Gi, ys, ks, pb, F.P.psa, F.P.psb);
            block_dense_sp<DL>(Gi + D4, yb, kb, pb, F.P.psa, F.P.psb);
          } else {
            block_dense<DL>(Gi, ys, ks, pb, F.P.psa, F.P.psb);
            block_dense<DL>(Gi + D4, yb, kb, pb, F.P.psa, F.P.psb);
          }
        } else {
          phase_block<DL, false>(F.P, Mi, ys, ks, pb, true);
          phase_block<DL, false>(F.P, Mi + nrow, yb, kb, pb, true);
        }
      }
      g += F.kind == 2 ? 1 : 0;
      __syncthreads();
      C* t = ys; ys = ks; ks = t;
      t = yb; yb = kb; kb = t;
    }
    for (int t = tid; t < sp.T; t += kST) {
      const long long o = base + __ldg(off + t);
      X[o] = ys[spos<DL>(t)];
      Lb[o] = yb[spos<DL>(t)];
    }
    __syncthreads();
  }
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int pt = 0; pt < 2; ++pt)
#pragma unroll
    for (int j = 0; j < kSQDrv; ++j) {
      if (j < dl.nd) {
        double v = (double)gv[pt][j];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][pt * kSQDrv + j] = v;
      }
    }
  __syncthreads();
  if (tid < 2 * kSQDrv && (tid % kSQDrv) < dl.nd) {
    double v = 0.0;
    for (int w = 0; w < kST / 32; ++w) v += red[w][tid];
    gpart[(size_t)blockIdx.x * 2 * kSQDrv + tid] = v;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  if (tid < 2 * kSQDrv && (tid % kSQDrv) < dl.nd) {
    double v = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) v += __ldcg(gpart + (size_t)b * 2 * kSQDrv + tid);
    if (tid < kSQDrv) gF0[dl.k[tid]] += v;
    else if (gF1) gF1[dl.k[tid - kSQDrv]] += v;
  }
  __syncthreads();
  if (tid == 0) *ticket = 0u;
}

}  // namespace

struct SQPlan {
  SQList a_first, a_mid, a_final, b_mid, b_final;
  SQList a_q1, b_q1;                              // the first-order product's step
  // backward (pull-back) lists of the gradient, couplings by their table index 4 e +
  // (0 half, 1 full) in the pull-back set (+2: the adjoint):
  //   b1: E2's palindrome, then G2's other modes;  b2: those modes alone
  //   a1: E1 in reverse term order, then G1's modes;  a2: G1's modes;  a3: E1 in term order
  //   a1q / b1q: Q1's couplings (full step) in reverse term order, then the modes
  SQList b1, b2, a1, a2, a3, a1q, b1q;
  int mgroup[SG_MAXQ];                            // pass of mode i's 1-body factors (0, 1)
  Phase mphase[SG_MAXQ];                          // its block layout in that pass, its digit first
  size_t sm_ga = 0, sm_gb = 0, sm_xa = 0, sm_xb = 0;
  bool grad_ok = false;
  // the same backward fused to one launch per pass and sub-step (k_slab_q2_bwd): factor
  // lists with contraction points (kind 3), prev = the earlier sub-step's rows and set
  SQList fb_mid, fb_0, fb_fin, fa_mid, fa_0, fa_fin, fbq, faq;
  size_t sm_fa = 0, sm_fb = 0;
  bool fused_ok = false;
  size_t sm_a = 0, sm_b = 0;
  int grid = 0;
};

namespace {

// 1-body factors of `modes` (tile digits of pass sp) as Kronecker pairs, an odd last one alone.
void add_onebody(const SlabPass& sp, int DL, const std::vector<int>& modes, SQList& L, bool& ok) {
  auto digit = [&](int m) {
    for (int k = 0; k < sp.ng; ++k) if (sp.tmode[k] == m) return k;
    return -1;
  };
  for (size_t j = 0; j < modes.size() && ok; j += 2) {
    if (L.nf >= kMaxSQ) { ok = false; return; }
    SQFactor& F = L.f[L.nf++];
    F = SQFactor{};
    const int ka = digit(modes[j]);
    if (j + 1 < modes.size()) {
      const int kb = digit(modes[j + 1]);
      F.P = make_phase(sp, DL, ka, kb);
      F.P.offL = modes[j] * DL * DL;
      F.P.offR = modes[j + 1] * DL * DL;
      F.kind = 0;
    } else {
      const int kb = ka == sp.ng - 1 ? sp.ng - 2 : sp.ng - 1;
      F.P = make_phase(sp, DL, ka, kb);
      F.P.offA = modes[j] * DL * DL;
      F.kind = 1;
    }
  }
}

void add_coupling(const Phase& E, int DL, int mat, int prev, SQList& L, bool& ok, int spar) {
  if (L.nf >= kMaxSQ) { ok = false; return; }
  SQFactor& F = L.f[L.nf++];
  F = SQFactor{};
  F.P = E;
  F.P.offL = F.P.offR = F.P.offA = F.P.offB = -1;
  F.kind = 2;
  F.mat = mat;
  F.prev = prev;
  F.spar = spar;
  ++L.ndense;
}

}  // namespace

bool slab_q2_ok(SlabPlanHost* h, const KPlan& p, bool mixed) {
  if (h->q2) return true;
  if (h->np != 2 || p.ne < 1) return false;
  const int DL = h->DL;
  // the couplings of each pass, in term order, with their block digits
  std::vector<std::pair<int, Phase>> E[2];
  for (int g = 0; g < 2; ++g)
    for (int q = 0; q < h->pass[g].nph; ++q)
      if (h->pass[g].ph[q].offL >= 0) E[g].push_back({h->pass[g].ph[q].ge, h->pass[g].ph[q]});
  if (E[0].empty() || E[1].empty()) return false;
  for (int g = 0; g < 2; ++g)
    std::sort(E[g].begin(), E[g].end(), [](const std::pair<int, Phase>& a, const std::pair<int, Phase>& b) {
      return a.first < b.first;
    });
  if (E[0].back().first >= E[1].front().first || E[1].back().first != p.ne - 1) return false;
  // modes of G1, and of G2 outside G1
  std::vector<int> m1, m2;
  for (int k = 0; k < h->pass[0].ng; ++k) m1.push_back(h->pass[0].tmode[k]);
  for (int k = 0; k < h->pass[1].ng; ++k) {
    const int m = h->pass[1].tmode[k];
    if (std::find(m1.begin(), m1.end(), m) == m1.end()) m2.push_back(m);
  }
  SQPlan* q = new SQPlan();
  bool ok = true;
  auto sp_of = [&](int e) { return (int)(((p.parL >> e) & 1ull) && ((p.parR >> e) & 1ull)); };
  const SlabPass& A = h->pass[0];
  const SlabPass& B = h->pass[1];
  auto e1_fwd = [&](SQList& L) { for (auto& e : E[0]) add_coupling(e.second, DL, 2 * e.first, 0, L, ok, sp_of(e.first)); };
  auto e1_rev = [&](SQList& L) {
    for (auto it = E[0].rbegin(); it != E[0].rend(); ++it) add_coupling(it->second, DL, 2 * it->first, 1, L, ok, sp_of(it->first));
  };
  q->a_first = SQList{};
  add_onebody(A, DL, m1, q->a_first, ok);
  e1_fwd(q->a_first);
  q->a_mid = SQList{};
  e1_rev(q->a_mid);
  add_onebody(A, DL, m1, q->a_mid, ok);
  e1_fwd(q->a_mid);
  q->a_final = SQList{};
  e1_rev(q->a_final);
  add_onebody(A, DL, m1, q->a_final, ok);
  q->b_mid = SQList{};
  add_onebody(B, DL, m2, q->b_mid, ok);
  for (size_t j = 0; j + 1 < E[1].size(); ++j) add_coupling(E[1][j].second, DL, 2 * E[1][j].first, 0, q->b_mid, ok, sp_of(E[1][j].first));
  add_coupling(E[1].back().second, DL, 2 * E[1].back().first + 1, 0, q->b_mid, ok, sp_of(E[1].back().first));
  for (int j = (int)E[1].size() - 2; j >= 0; --j)
    add_coupling(E[1][j].second, DL, 2 * E[1][j].first, 0, q->b_mid, ok, sp_of(E[1][j].first));
  q->b_final = SQList{};
  add_onebody(B, DL, m2, q->b_final, ok);
  q->a_q1 = SQList{};
  add_onebody(A, DL, m1, q->a_q1, ok);
  for (auto& e : E[0]) add_coupling(e.second, DL, 2 * e.first + 1, 0, q->a_q1, ok, sp_of(e.first));
  q->b_q1 = SQList{};
  add_onebody(B, DL, m2, q->b_q1, ok);
  for (auto& e : E[1]) add_coupling(e.second, DL, 2 * e.first + 1, 0, q->b_q1, ok, sp_of(e.first));
  // the gradient's pull-back lists (gok: they fit; the evolution does not need them)
  bool gok = true;
  auto pb = [&](const std::pair<int, Phase>& e, bool full, SQList& L) {
    add_coupling(e.second, DL, 4 * e.first + (full ? 1 : 0), 0, L, gok, sp_of(e.first));
  };
  q->b1 = SQList{};
  for (size_t j = 0; j + 1 < E[1].size(); ++j) pb(E[1][j], false, q->b1);
  pb(E[1].back(), true, q->b1);
  for (int j = (int)E[1].size() - 2; j >= 0; --j) pb(E[1][j], false, q->b1);
  add_onebody(B, DL, m2, q->b1, gok);
  q->b2 = SQList{};
  add_onebody(B, DL, m2, q->b2, gok);
  q->a1 = SQList{};
  for (auto it = E[0].rbegin(); it != E[0].rend(); ++it) pb(*it, false, q->a1);
  add_onebody(A, DL, m1, q->a1, gok);
  q->a2 = SQList{};
  add_onebody(A, DL, m1, q->a2, gok);
  q->a3 = SQList{};
  for (auto& e : E[0]) pb(e, false, q->a3);
  q->b1q = SQList{};
  for (auto it = E[1].rbegin(); it != E[1].rend(); ++it) pb(*it, true, q->b1q);
  add_onebody(B, DL, m2, q->b1q, gok);
  q->a1q = SQList{};
  for (auto it = E[0].rbegin(); it != E[0].rend(); ++it) pb(*it, true, q->a1q);
  add_onebody(A, DL, m1, q->a1q, gok);
  for (int i = 0; i < SG_MAXQ; ++i) q->mgroup[i] = -1;
  for (int g = 0; g < 2; ++g) {
    const SlabPass& sp = h->pass[g];
    for (int m : (g == 0 ? m1 : m2)) {
      int ka = -1;
      for (int k = 0; k < sp.ng; ++k) if (sp.tmode[k] == m) ka = k;
      if (ka < 0) { gok = false; continue; }
      q->mgroup[m] = g;
      q->mphase[m] = make_phase(sp, DL, ka, ka == sp.ng - 1 ? sp.ng - 2 : sp.ng - 1);
    }
  }
  const size_t csz = mixed ? sizeof(float2) : sizeof(double2);
  const size_t D4 = (size_t)DL * DL * DL * DL;
  const size_t nrow = (size_t)p.nq * DL * DL;
  auto need = [&](const SlabPass& sp, const SQList& L) {
    return (2 * (size_t)spad(sp.T) + nrow + (size_t)L.ndense * D4) * csz;
  };
  q->sm_a = std::max({need(A, q->a_first), need(A, q->a_mid), need(A, q->a_final), need(A, q->a_q1)});
  q->sm_b = std::max({need(B, q->b_mid), need(B, q->b_final), need(B, q->b_q1)});
  q->sm_ga = std::max({need(A, q->a1), need(A, q->a2), need(A, q->a3), need(A, q->a1q)});
  q->sm_gb = std::max({need(B, q->b1), need(B, q->b2), need(B, q->b1q)});
  q->sm_xa = (2 * (size_t)spad(A.T) + (size_t)kSQDrv * DL * DL) * csz;
  q->sm_xb = (2 * (size_t)spad(B.T) + (size_t)kSQDrv * DL * DL) * csz;
  q->grad_ok = gok && std::max(q->sm_ga, q->sm_gb) <= kSlabSmemMax && std::max(q->sm_xa, q->sm_xb) <= kXdSmemMax;
  bool fok = q->grad_ok;
  auto cat = [&](SQList& dst, const SQList& src, int prev) {
    for (int i = 0; i < src.nf; ++i) {
      if (dst.nf >= kMaxSQ) { fok = false; return; }
      dst.f[dst.nf] = src.f[i];
      dst.f[dst.nf].prev = prev;
      dst.ndense += src.f[i].kind == 2 ? 1 : 0;
      ++dst.nf;
    }
  };
  auto point = [&](SQList& dst, int pt) {
    if (dst.nf >= kMaxSQ) { fok = false; return; }
    SQFactor& F = dst.f[dst.nf++];
    F = SQFactor{};
    F.kind = 3;
    F.mat = pt;
  };
  q->fb_mid = SQList{}; cat(q->fb_mid, q->b1, 0); point(q->fb_mid, 0); cat(q->fb_mid, q->b2, 1); point(q->fb_mid, 1);
  q->fb_0 = SQList{};   cat(q->fb_0, q->b1, 0);   point(q->fb_0, 0);
  q->fb_fin = SQList{}; cat(q->fb_fin, q->b2, 0); point(q->fb_fin, 0);
  q->fa_mid = SQList{}; cat(q->fa_mid, q->a1, 0); point(q->fa_mid, 0); cat(q->fa_mid, q->a2, 1); point(q->fa_mid, 1);
  cat(q->fa_mid, q->a3, 1);
  q->fa_0 = SQList{};   cat(q->fa_0, q->a1, 0);   point(q->fa_0, 0);
  q->fa_fin = SQList{}; cat(q->fa_fin, q->a2, 0); point(q->fa_fin, 0); cat(q->fa_fin, q->a3, 0);
  q->fbq = SQList{};    cat(q->fbq, q->b1q, 0);   point(q->fbq, 0);
  q->faq = SQList{};    cat(q->faq, q->a1q, 0);   point(q->faq, 0);
  auto fneed = [&](const SlabPass& sp, const SQList& L) {
    return (4 * (size_t)spad(sp.T) + 4 * nrow + 2 * (size_t)kSQDrv * DL * DL + 2 * (size_t)L.ndense * D4) * csz;
  };
  q->sm_fa = std::max({fneed(A, q->fa_mid), fneed(A, q->fa_0), fneed(A, q->fa_fin), fneed(A, q->faq)});
  q->sm_fb = std::max({fneed(B, q->fb_mid), fneed(B, q->fb_0), fneed(B, q->fb_fin), fneed(B, q->fbq)});
  q->fused_ok = fok && std::max(q->sm_fa, q->sm_fb) <= kXdSmemMax;
  const long long ntiles = (long long)p.S * (p.D / h->pass[0].T);
  q->grid = (int)std::min<long long>(ntiles, 152ll * (mixed ? 2 : 1));
  if (!ok || q->sm_a > kSlabSmemMax || q->sm_b > kSlabSmemMax) {
    delete q;
    return false;
  }
  h->q2 = q;
  return true;
}

void slab_q2_free(SlabPlanHost* h) {
  delete h->q2;
  h->q2 = nullptr;
}

int slab_dl(const SlabPlanHost* h) { return h->DL; }

namespace {

template <typename R, int DL>
int q2_run_t(const SlabPlanHost* h, const void* rows, const void* edges, void* X, int M, int J, const int* set_of,
             bool q1, cudaStream_t st) {
  typedef typename CT<R>::T C;
  static const bool attr = [] {
    cudaFuncSetAttribute(k_slab_q2<R, DL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSlabSmemMax);
    return true;
  }();
  (void)attr;
  const SQPlan& q = *h->q2;
  const int nq = h->perm.nq;
  const int nrow = nq * DL * DL;
  const int ne = [&] {
    int n = 0;
    for (int g = 0; g < h->np; ++g) n += h->pass[g].ne;
    return n;
  }();
  const C* R0 = static_cast<const C*>(rows);
  const C* E = static_cast<const C*>(edges);
  C* Xc = static_cast<C*>(X);
  auto launch = [&](int g, const SQList& L, int rowidx, int so_prev, int so_cur) {
    if (L.nf == 0) return 0;
    k_slab_q2<R, DL><<<q.grid, kST, g == 0 ? q.sm_a : q.sm_b, st>>>(h->pass[g], L, R0 + (size_t)rowidx * nrow, E,
                                                                  so_prev, so_cur, nrow, Xc);
    return 1;
  };
  int n = 0;
  if (q1) {
    for (int m = 0; m < M; ++m) {
      const int so = 2 * ne * set_of[m % J];
      const int rowidx = m == 0 ? M : m - 1;        // step m's full-step 1-body factors
      n += launch(0, q.a_q1, rowidx, so, so);
      n += launch(1, q.b_q1, rowidx, so, so);
    }
    return n;
  }
  for (int m = 0; m < M; ++m) {
    const int so_cur = 2 * ne * set_of[m % J];
    const int so_prev = m > 0 ? 2 * ne * set_of[(m - 1) % J] : 0;
    const int rowidx = m == 0 ? M : m - 1;
    n += launch(0, m == 0 ? q.a_first : q.a_mid, rowidx, so_prev, so_cur);
    n += launch(1, q.b_mid, rowidx, so_cur, so_cur);
  }
  if (M > 0) {
    const int so_last = 2 * ne * set_of[(M - 1) % J];
    n += launch(0, q.a_final, M - 1, so_last, so_last);
    n += launch(1, q.b_final, M - 1, so_last, so_last);
  }
  return n;
}

// Backward of the tiled product for the pulse gradient: the reverse of the forward's
// factor sequence (per sub-step m, forward pass A: E1 reversed (m - 1), U_G1(m - 1) second
// half, U_G1(m) first half, E1 (m); pass B: U_G2'(m - 1) second half, U_G2'(m) first half,
// E2's palindrome (m); after the last sub-step E1 reversed and U_G1 second half, then
// U_G2' second half), each factor undone on the states by its inverse and on the
// co-states by its adjoint, a contribution point after every 1-body half step.  Q1: per
// step pass A U_G1(m), E1; pass B U_G2'(m), E2.
// SG_Q2_FUSE=0: the segmented backward (pull-back and contraction launches apart)
bool q2_fuse_on() {
  const char* e = std::getenv("SG_Q2_FUSE");
  return !(e && e[0] == '0');
}

template <typename R, int DL>
int q2_grad_t(const SlabPlanHost* h, const void* gtab, const void* edges_pb, void* X, void* Lb, int M, int J,
              const int* set_of, bool q1, int K, const int* drv_mode, double* gF, double* gpart, unsigned* ticket,
              cudaStream_t st) {
  typedef typename CT<R>::T C;
  static const bool attr = [] {
    cudaFuncSetAttribute(k_slab_q2<R, DL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSlabSmemMax);
    cudaFuncSetAttribute(k_slab_q2_xd<R, DL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kXdSmemMax);
    cudaFuncSetAttribute(k_slab_q2_bwd<R, DL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kXdSmemMax);
    return true;
  }();
  (void)attr;
  const SQPlan& q = *h->q2;
  const int nq = h->perm.nq;
  const int nrow = nq * DL * DL;
  const size_t rowblk = (size_t)(2 * nq + K) * DL * DL;
  const size_t D4 = (size_t)DL * DL * DL * DL;
  const int ne = [&] {
    int n = 0;
    for (int g = 0; g < h->np; ++g) n += h->pass[g].ne;
    return n;
  }();
  const C* G = static_cast<const C*>(gtab);
  const C* Ep = static_cast<const C*>(edges_pb);
  C* Xc = static_cast<C*>(X);
  C* Lc = static_cast<C*>(Lb);
  SQDList dl[2] = {};
  for (int k = 0; k < K; ++k) {
    const int g = q.mgroup[drv_mode[k]];
    if (g < 0 || dl[g].nd >= kSQDrv) return -1;
    dl[g].k[dl[g].nd] = k;
    dl[g].P[dl[g].nd++] = q.mphase[drv_mode[k]];
  }
  auto app = [&](int g, const SQList& L, int srow, int sigma) {
    if (L.nf == 0) return 0;
    const C* rows = G + (size_t)srow * rowblk;
    const int so = 4 * ne * sigma;
    const size_t sm = g == 0 ? q.sm_ga : q.sm_gb;
    k_slab_q2<R, DL><<<q.grid, kST, sm, st>>>(h->pass[g], L, rows, Ep, 0, so, nrow, Xc);           // U^-1
    k_slab_q2<R, DL><<<q.grid, kST, sm, st>>>(h->pass[g], L, rows + nrow, Ep + 2 * D4, 0, so, nrow, Lc);   // U^dag
    return 2;
  };
  auto xd = [&](int g, int srow) {
    if (dl[g].nd == 0) return 0;
    k_slab_q2_xd<R, DL><<<q.grid, kST, g == 0 ? q.sm_xa : q.sm_xb, st>>>(
        h->pass[g], dl[g], Xc, Lc, G + (size_t)srow * rowblk, nq, gpart, ticket, gF + (size_t)srow * K);
    return 1;
  };
  int n = 0;
  if (q.fused_ok && q2_fuse_on()) {
    auto fz = [&](int g, const SQList& L, int s0, int s1, int sg0, int sg1) {
      k_slab_q2_bwd<R, DL><<<q.grid, kST, g == 0 ? q.sm_fa : q.sm_fb, st>>>(
          h->pass[g], L, dl[g], G + (size_t)s0 * rowblk, G + (size_t)(s1 >= 0 ? s1 : s0) * rowblk, Ep,
          4 * ne * sg0, 4 * ne * sg1, nq, Xc, Lc, gpart, ticket, gF + (size_t)s0 * K,
          s1 >= 0 ? gF + (size_t)s1 * K : nullptr);
      return 1;
    };
    if (q1) {
      for (int m = M - 1; m >= 0; --m) {
        const int sg = set_of[m % J];
        n += fz(1, q.fbq, m, -1, sg, sg);
        n += fz(0, q.faq, m, -1, sg, sg);
      }
      return n;
    }
    if (M > 0) {
      const int sg = set_of[(M - 1) % J];
      n += fz(1, q.fb_fin, M - 1, -1, sg, sg);
      n += fz(0, q.fa_fin, M - 1, -1, sg, sg);
    }
    for (int m = M - 1; m >= 0; --m) {
      const int sg = set_of[m % J], sp = m > 0 ? set_of[(m - 1) % J] : sg;
      n += fz(1, m > 0 ? q.fb_mid : q.fb_0, m, m > 0 ? m - 1 : -1, sg, sp);
      n += fz(0, m > 0 ? q.fa_mid : q.fa_0, m, m > 0 ? m - 1 : -1, sg, sp);
    }
    return n;
  }
  if (q1) {
    for (int m = M - 1; m >= 0; --m) {
      const int sg = set_of[m % J];
      n += app(1, q.b1q, m, sg);
      n += xd(1, m);
      n += app(0, q.a1q, m, sg);
      n += xd(0, m);
    }
    return n;
  }
  if (M > 0) {
    const int s = M - 1, sg = set_of[s % J];
    n += app(1, q.b2, s, sg);                       // U_G2'(M - 1), second half
    n += xd(1, s);
    n += app(0, q.a2, s, sg);                       // U_G1(M - 1), second half
    n += xd(0, s);
    n += app(0, q.a3, s, sg);                       // E1 reversed (M - 1)
  }
  for (int m = M - 1; m >= 0; --m) {
    const int sg = set_of[m % J];
    n += app(1, q.b1, m, sg);                       // E2's palindrome, U_G2'(m) first half
    n += xd(1, m);
    if (m > 0) {
      n += app(1, q.b2, m - 1, set_of[(m - 1) % J]);   // U_G2'(m - 1) second half
      n += xd(1, m - 1);
    }
    n += app(0, q.a1, m, sg);                       // E1 (m), U_G1(m) first half
    n += xd(0, m);
    if (m > 0) {
      const int sp = set_of[(m - 1) % J];
      n += app(0, q.a2, m - 1, sp);                 // U_G1(m - 1) second half
      n += xd(0, m - 1);
      n += app(0, q.a3, m - 1, sp);                 // E1 reversed (m - 1)
    }
  }
  return n;
}

}  // namespace

bool slab_q2_grad_ok(const SlabPlanHost* h) { return h->q2 && h->q2->grad_ok; }

size_t slab_q2_grad_part(const SlabPlanHost* h) { return (size_t)std::max(1, h->q2 ? h->q2->grid : 1) * 2 * kSQDrv; }

int slab_q2_grad_run(const SlabPlanHost* h, bool mixed, const void* gtab, const void* edges_pb, void* X, void* Lb,
                     int M, int J, const int* set_of, bool q1, int K, const int* drv_mode, double* gF,
                     double* gpart, unsigned* ticket, cudaStream_t st) {
  SLAB_DISPATCH(q2_grad_t, h, gtab, edges_pb, X, Lb, M, J, set_of, q1, K, drv_mode, gF, gpart, ticket, st);
}

int slab_q2_run(const SlabPlanHost* h, bool mixed, const void* rows, const void* edges, void* X, int M, int J,
                const int* set_of, bool q1, cudaStream_t st) {
  SLAB_DISPATCH(q2_run_t, h, rows, edges, X, M, J, set_of, q1, st);
}
