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

}  // namespace

struct SQPlan {
  SQList a_first, a_mid, a_final, b_mid, b_final;
  SQList a_q1, b_q1;                              // the first-order product's step
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
  const size_t csz = mixed ? sizeof(float2) : sizeof(double2);
  const size_t D4 = (size_t)DL * DL * DL * DL;
  const size_t nrow = (size_t)p.nq * DL * DL;
  auto need = [&](const SlabPass& sp, const SQList& L) {
    return (2 * (size_t)spad(sp.T) + nrow + (size_t)L.ndense * D4) * csz;
  };
  q->sm_a = std::max({need(A, q->a_first), need(A, q->a_mid), need(A, q->a_final), need(A, q->a_q1)});
  q->sm_b = std::max({need(B, q->b_mid), need(B, q->b_final), need(B, q->b_q1)});
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

}  // namespace

int slab_q2_run(const SlabPlanHost* h, bool mixed, const void* rows, const void* edges, void* X, int M, int J,
                const int* set_of, bool q1, cudaStream_t st) {
  SLAB_DISPATCH(q2_run_t, h, rows, edges, X, M, J, set_of, q1, st);
}
