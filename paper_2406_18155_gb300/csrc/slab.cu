// Tiled RK4 stage kernels for HBM-resident slabs (see slab.h).
//
// Layout: internal slabs are column-major [S][D] with a permuted digit order
// chosen so that tiles read whole 128-byte lines (two-group plans put the
// modes shared by both groups lowest).  A tile is one column x all levels of the
// pass's mode group; its global offsets come from a per-pass table kept in shared
// memory.  Each thread computes the entries t = tid, tid + 256, ... of the tile,
// reading neighbours along each term's modes from shared memory; parity-odd
// operators (n and phi at n_g = 0, phi_ext = pi) skip their zero entries.
#include "sg_internal.h"
#include "kplan.h"
#include "grad.cuh"
#include "slab.h"
#include <algorithm>
#include <cstdlib>
#include <set>
#include <vector>

namespace {

constexpr int kST = 256;          // threads per block
constexpr int kTmax = 4096;       // entries per tile
constexpr int kMaxPass = 4;
constexpr int kSPW = 2;           // cross-density slots per warp
constexpr int kMaxX = kSPW * (kST / 32);

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
  int nx;                         // cross-density slots
  int x_k[kMaxX], x_k2[kMaxX], x_off2[kMaxX], x_gslot[kMaxX];
  const int* off;                 // device tile offsets [T]
};

template <int DL>
__device__ __forceinline__ int digit(const SlabPass& sp, int t, int k) {
  if (DL == 2 || DL == 4 || DL == 8) return (t >> sp.tlg[k]) & (DL - 1);
  return (t / sp.tsh[k]) % DL;
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

// H y at tile entry t, from the tile in shared memory.
template <int DL, typename C>
__device__ __forceinline__ C apply_tile(const SlabPass& sp, const C* __restrict__ M,
                                        const C* __restrict__ y, int t) {
  C acc = cmk<C>(0.0, 0.0);
  for (int u = 0; u < sp.n1; ++u) {
    const int k = sp.s1_k[u], sh = sp.tsh[k];
    const int l = digit<DL>(sp, t, k);
    const C* yb = y + (t - l * sh);
    const C* Mr = M + sp.s1_off[u] + l * DL;
    if ((sp.par1 >> u) & 1u) {
#pragma unroll
      for (int b = 0; b < DL; ++b)
        if (((b + l) & 1) == 1) acc = cfma(Mr[b], yb[b * sh], acc);
    } else {
#pragma unroll
      for (int b = 0; b < DL; ++b) acc = cfma(Mr[b], yb[b * sh], acc);
    }
  }
  for (int e = 0; e < sp.ne; ++e) {
    const int ka = sp.e_ka[e], kb = sp.e_kb[e];
    const int sa = sp.tsh[ka], sb = sp.tsh[kb];
    const int la = digit<DL>(sp, t, ka), lb = digit<DL>(sp, t, kb);
    const C* yb = y + (t - la * sa - lb * sb);
    const C* L = M + sp.e_offL[e] + la * DL;
    const C* R = M + sp.e_offR[e] + lb * DL;
    const bool pl = (sp.parL >> e) & 1ull, pr = (sp.parR >> e) & 1ull;
#pragma unroll
    for (int x = 0; x < DL; ++x) {
      if (pl && ((x + la) & 1) == 0) continue;
      C u = cmk<C>(0.0, 0.0);
#pragma unroll
      for (int z = 0; z < DL; ++z) {
        if (pr && ((z + lb) & 1) == 0) continue;
        u = cfma(R[z], yb[x * sa + z * sb], u);
      }
      acc = cfma(L[x], u, acc);
    }
  }
  return acc;
}

template <typename C>
__device__ __forceinline__ void load_common(const SlabPass& sp, const C* __restrict__ tabrow, C* M,
                                            int* off) {
  for (int i = threadIdx.x; i < sp.row; i += blockDim.x) M[i] = tabrow[i];
  for (int i = threadIdx.x; i < sp.T; i += blockDim.x) off[i] = sp.off[i];
  __syncthreads();
}

// KIND: 0 first partial pass (kA = k), 1 middle partial (kA += k), 2 last pass after
// partials (k += kA then the RK4 epilogue), 3 single pass (epilogue).
template <typename R, int DL, int STAGE, bool STORE, int KIND>
__global__ void __launch_bounds__(kST) k_slab_fwd(SlabPass sp, const typename CT<R>::T* __restrict__ X,
                                                  const typename CT<R>::T* __restrict__ tabrow,
                                                  const double2* __restrict__ psi_in, double2* psi_out,
                                                  typename CT<R>::T* __restrict__ Xn,
                                                  typename CT<R>::T* __restrict__ Dacc,
                                                  typename CT<R>::T* __restrict__ kA, double dt) {
  typedef typename CT<R>::T C;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* yt = reinterpret_cast<C*>(smraw);
  C* M = yt + sp.T;
  int* off = reinterpret_cast<int*>(M + sp.row);
  load_common(sp, tabrow, M, off);
  const long long ntiles = (long long)sp.S * sp.ntpc;
  const R h = (R)dt;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long base = tile_base(sp, tile);
    for (int t = threadIdx.x; t < sp.T; t += kST) yt[t] = X[base + off[t]];
    __syncthreads();
    for (int t = threadIdx.x; t < sp.T; t += kST) {
      const C a = apply_tile<DL>(sp, M, yt, t);
      C k = cmk<C>(a.y, -a.x);                     // -i H y
      const long long g = base + off[t];
      if (KIND == 0) { kA[g] = k; continue; }
      if (KIND == 1) { C p = kA[g]; kA[g] = cmk<C>(p.x + k.x, p.y + k.y); continue; }
      if (KIND == 2) { C p = kA[g]; k = cmk<C>(p.x + k.x, p.y + k.y); }
      const double2 ps = psi_in[g];
      const C pr = to_c(ps, R(0));
      if (STAGE == 0) {
        if (!STORE) Dacc[g] = cmk<C>(h / 6 * k.x, h / 6 * k.y);
        Xn[g] = cmk<C>(pr.x + h / 2 * k.x, pr.y + h / 2 * k.y);
      } else if (STAGE == 1) {
        if (!STORE) { C d = Dacc[g]; Dacc[g] = cmk<C>(d.x + h / 3 * k.x, d.y + h / 3 * k.y); }
        Xn[g] = cmk<C>(pr.x + h / 2 * k.x, pr.y + h / 2 * k.y);
      } else if (STAGE == 2) {
        if (!STORE) { C d = Dacc[g]; Dacc[g] = cmk<C>(d.x + h / 3 * k.x, d.y + h / 3 * k.y); }
        Xn[g] = cmk<C>(pr.x + h * k.x, pr.y + h * k.y);
      } else {
        C d = Dacc[g];
        R incx = d.x + h / 6 * k.x, incy = d.y + h / 6 * k.y;
        double2 pn = make_double2(ps.x + (double)incx, ps.y + (double)incy);
        psi_out[g] = pn;
        Xn[g] = to_c(pn, R(0));
      }
    }
    __syncthreads();
  }
}

// Adjoint pass: X = kbar_s tile, Y = y_s tile.  Applies A_s^dag = i H to kbar
// (partial or with the adjoint epilogue) and accumulates the cross-densities of
// this pass's slots, one warp per slot (kSPW slots per warp), persisting across
// tiles; one fixed-order reduction at the end.
template <typename R, int DL, int STAGE, int KIND>
__global__ void __launch_bounds__(kST) k_slab_adj(SlabPass sp, const typename CT<R>::T* __restrict__ X,
                                                  const typename CT<R>::T* __restrict__ Y,
                                                  const typename CT<R>::T* __restrict__ tabrow,
                                                  double2* __restrict__ pbar,
                                                  typename CT<R>::T* __restrict__ Xn,
                                                  typename CT<R>::T* __restrict__ Db,
                                                  typename CT<R>::T* __restrict__ yA, double dt,
                                                  XArgs xa) {
  typedef typename CT<R>::T C;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* xt = reinterpret_cast<C*>(smraw);
  C* yt = xt + sp.T;
  C* M = yt + sp.T;
  int* off = reinterpret_cast<int*>(M + sp.row);
  load_common(sp, tabrow, M, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  C acc[kSPW][DL][DL];
#pragma unroll
  for (int s = 0; s < kSPW; ++s)
#pragma unroll
    for (int a = 0; a < DL; ++a)
#pragma unroll
      for (int b = 0; b < DL; ++b) acc[s][a][b] = cmk<C>(0.0, 0.0);
  const long long ntiles = (long long)sp.S * sp.ntpc;
  const R h = (R)dt;
  const int nf = sp.T / DL;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long base = tile_base(sp, tile);
    for (int t = threadIdx.x; t < sp.T; t += kST) {
      const long long g = base + off[t];
      xt[t] = X[g];
      yt[t] = Y[g];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < sp.T; t += kST) {
      const C a = apply_tile<DL>(sp, M, xt, t);
      C yb = cmk<C>(-a.y, a.x);                     // i H kbar
      const long long g = base + off[t];
      if (KIND == 0) { yA[g] = yb; continue; }
      if (KIND == 1) { C p = yA[g]; yA[g] = cmk<C>(p.x + yb.x, p.y + yb.y); continue; }
      if (KIND == 2) { C p = yA[g]; yb = cmk<C>(p.x + yb.x, p.y + yb.y); }
      const double2 pb = pbar[g];
      const C pr = to_c(pb, R(0));
      if (STAGE == 3) {
        Db[g] = yb;
        Xn[g] = cmk<C>(h / 3 * pr.x + h * yb.x, h / 3 * pr.y + h * yb.y);
      } else if (STAGE == 2) {
        C d = Db[g];
        Db[g] = cmk<C>(d.x + yb.x, d.y + yb.y);
        Xn[g] = cmk<C>(h / 3 * pr.x + h / 2 * yb.x, h / 3 * pr.y + h / 2 * yb.y);
      } else if (STAGE == 1) {
        C d = Db[g];
        Db[g] = cmk<C>(d.x + yb.x, d.y + yb.y);
        Xn[g] = cmk<C>(h / 6 * pr.x + h / 2 * yb.x, h / 6 * pr.y + h / 2 * yb.y);
      } else {
        C d = Db[g];
        double2 pn = make_double2(pb.x + (double)(d.x + yb.x), pb.y + (double)(d.y + yb.y));
        pbar[g] = pn;
        C q = to_c(pn, R(0));
        Xn[g] = cmk<C>(h / 6 * q.x, h / 6 * q.y);
      }
    }
    // cross-densities of this warp's slots over the tile
#pragma unroll
    for (int s = 0; s < kSPW; ++s) {
      const int slot = warp + s * (kST / 32);
      if (slot >= sp.nx) continue;
      const int k = sp.x_k[slot], sh = sp.tsh[k];
      const int k2 = sp.x_k2[slot];
      for (int f = lane; f < nf; f += 32) {
        const int t0 = (f / sh) * (DL * sh) + (f % sh);
        C xv[DL], yv[DL];
        if (k2 < 0) {
#pragma unroll
          for (int a = 0; a < DL; ++a) { xv[a] = xt[t0 + a * sh]; yv[a] = yt[t0 + a * sh]; }
        } else {
          const int sh2 = sp.tsh[k2];
          const int l2 = digit<DL>(sp, t0, k2);
          const C* O2 = M + sp.x_off2[slot] + l2 * DL;
          const C* yb = yt + (t0 - l2 * sh2);
#pragma unroll
          for (int a = 0; a < DL; ++a) {
            xv[a] = xt[t0 + a * sh];
            C u = cmk<C>(0.0, 0.0);
#pragma unroll
            for (int c = 0; c < DL; ++c) u = cfma(O2[c], yb[a * sh + c * sh2], u);
            yv[a] = u;
          }
        }
#pragma unroll
        for (int a = 0; a < DL; ++a)
#pragma unroll
          for (int b = 0; b < DL; ++b) acc[s][a][b] = cjfma(xv[a], yv[b], acc[s][a][b]);
      }
    }
    __syncthreads();
  }
  // warp reductions -> block partials [block][slot][DL*DL]
#pragma unroll
  for (int s = 0; s < kSPW; ++s) {
    const int slot = warp + s * (kST / 32);
    if (slot >= sp.nx) continue;                    // warp-uniform
#pragma unroll
    for (int a = 0; a < DL; ++a)
#pragma unroll
      for (int b = 0; b < DL; ++b) {
        double vr = acc[s][a][b].x, vi = acc[s][a][b].y;
        for (int o = 16; o > 0; o >>= 1) {
          vr += __shfl_xor_sync(0xffffffffu, vr, o);
          vi += __shfl_xor_sync(0xffffffffu, vi, o);
        }
        if (lane == 0) xa.partial[((size_t)blockIdx.x * kMaxX + slot) * DL * DL + a * DL + b] = make_double2(vr, vi);
      }
  }
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(xa.ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  double2* Wt = reinterpret_cast<double2*>(smraw);   // nx * DL * DL
  for (int i = threadIdx.x; i < sp.nx * DL * DL; i += blockDim.x) {
    const int slot = i / (DL * DL), ab = i % (DL * DL);
    double sr = 0.0, si = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) {
      double2 v = __ldcg(xa.partial + ((size_t)b * kMaxX + slot) * DL * DL + ab);
      sr += v.x;
      si += v.y;
    }
    Wt[i] = make_double2(si, -sr);                     // W = -i C
  }
  __syncthreads();
  if (threadIdx.x == 0) *xa.ticket = 0u;
  if (threadIdx.x < sp.nx) contract_slot(xa, sp.x_gslot[threadIdx.x], Wt + threadIdx.x * DL * DL, DL);
}

struct PermArgs {
  int nq, S;
  long long D;
  int dims[SG_MAXQ];
  long long st_api[SG_MAXQ], st_int[SG_MAXQ];
};

// api [D][S] (digits in mode order) <-> internal [S][D] (permuted digits)
__global__ void k_perm(PermArgs a, const double2* __restrict__ src, double2* __restrict__ dst, int to_int) {
  const long long total = a.D * a.S;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / a.S;
    const int s = (int)(e - r * a.S);
    long long ri = 0;
    for (int i = 0; i < a.nq; ++i) ri += ((r / a.st_api[i]) % a.dims[i]) * a.st_int[i];
    const long long gi = (long long)s * a.D + ri;
    if (to_int) dst[gi] = src[e]; else dst[e] = src[gi];
  }
}

}  // namespace

struct SlabPlanHost {
  int DL = 0, np = 0;
  bool mixed = false;
  SlabPass pass[kMaxPass];
  int* off_dev[kMaxPass] = {nullptr, nullptr, nullptr, nullptr};
  PermArgs perm{};
  int grid_fwd = 0, grid_adj = 0;
  size_t sm_fwd[kMaxPass] = {0}, sm_adj[kMaxPass] = {0};
};

SlabPlanHost* slab_plan_create(const KPlan& p, bool mixed, cudaStream_t st) {
  const int nq = p.nq;
  const int DL = p.dims[0];
  for (int i = 0; i < nq; ++i) if (p.dims[i] != DL) return nullptr;
  if (DL < 2 || DL > 5) return nullptr;
  if (p.D >= (1ll << 31)) return nullptr;
  // SG_SLAB_TMAX lowers the tile budget so small systems exercise multi-pass plans (tests)
  long long tmax = kTmax;
  if (const char* e = std::getenv("SG_SLAB_TMAX")) tmax = std::max(1ll, std::min<long long>(kTmax, atoll(e)));
  // ---- mode groups: greedy cover of the 2-body terms, groups of <= kTmax entries
  auto size_of = [&](const std::set<int>& g) {
    long long s = 1;
    for (int m : g) s *= p.dims[m];
    return s;
  };
  std::vector<std::set<int>> groups;
  std::vector<int> edge_group(p.ne, -1), slot_group(p.n1, -1);
  if (p.D <= tmax) {
    std::set<int> all;
    for (int i = 0; i < nq; ++i) all.insert(i);
    groups.push_back(all);
    for (int e = 0; e < p.ne; ++e) edge_group[e] = 0;
    for (int u = 0; u < p.n1; ++u) slot_group[u] = 0;
  } else {
    std::set<int> cur;
    for (int e = 0; e < p.ne; ++e) {
      const int a = p.e_a[e], b = p.e_b[e];
      int found = -1;
      for (size_t g = 0; g < groups.size(); ++g)
        if (groups[g].count(a) && groups[g].count(b)) { found = (int)g; break; }
      if (found >= 0) { edge_group[e] = found; continue; }
      std::set<int> trial = cur;
      trial.insert(a);
      trial.insert(b);
      if (size_of(trial) <= tmax) {
        cur = trial;
        edge_group[e] = (int)groups.size();
      } else {
        if (!cur.empty()) groups.push_back(cur);
        cur = {a, b};
        edge_group[e] = (int)groups.size();
      }
    }
    if (!cur.empty()) groups.push_back(cur);
    // 1-body slots: the group holding the mode with the fewest terms so far
    for (int u = 0; u < p.n1; ++u) {
      const int m = p.s1_mode[u];
      int best = -1;
      size_t bestn = 1u << 30;
      for (size_t g = 0; g < groups.size(); ++g) {
        if (!groups[g].count(m)) continue;
        size_t n = 0;
        for (int e = 0; e < p.ne; ++e) n += edge_group[e] == (int)g;
        for (int v = 0; v < u; ++v) n += slot_group[v] == (int)g;
        if (n < bestn) { bestn = n; best = (int)g; }
      }
      if (best < 0) {
        for (size_t g = 0; g < groups.size() && best < 0; ++g) {
          std::set<int> trial = groups[g];
          trial.insert(m);
          if (size_of(trial) <= tmax) { groups[g] = trial; best = (int)g; }
        }
        if (best < 0) { groups.push_back({m}); best = (int)groups.size() - 1; }
      }
      slot_group[u] = best;
    }
  }
  const int np = (int)groups.size();
  if (np < 1 || np > kMaxPass) return nullptr;
  // ---- internal digit order (most significant first)
  std::vector<int> order;
  if (np == 2) {
    const std::set<int>& A = groups[0];
    const std::set<int>& B = groups[1];
    for (int i = 0; i < nq; ++i) if (!A.count(i) && !B.count(i)) order.push_back(i);
    for (int i = 0; i < nq; ++i) if (A.count(i) && !B.count(i)) order.push_back(i);
    for (int i = 0; i < nq; ++i) if (B.count(i) && !A.count(i)) order.push_back(i);
    for (int i = 0; i < nq; ++i) if (A.count(i) && B.count(i)) order.push_back(i);
  } else {
    for (int i = 0; i < nq; ++i) order.push_back(i);
  }
  long long st_int[SG_MAXQ];
  {
    long long s = 1;
    for (int k = nq - 1; k >= 0; --k) { st_int[order[k]] = s; s *= p.dims[order[k]]; }
  }
  SlabPlanHost* h = new SlabPlanHost();
  h->DL = DL;
  h->np = np;
  h->mixed = mixed;
  h->perm.nq = nq; h->perm.S = p.S; h->perm.D = p.D;
  for (int i = 0; i < nq; ++i) { h->perm.dims[i] = p.dims[i]; h->perm.st_api[i] = p.st[i]; h->perm.st_int[i] = st_int[i]; }
  const size_t csz = mixed ? sizeof(float2) : sizeof(double2);
  for (int g = 0; g < np; ++g) {
    SlabPass& sp = h->pass[g];
    sp = SlabPass{};
    std::vector<int> tm;                  // tile modes in internal order
    for (int m : order) if (groups[g].count(m)) tm.push_back(m);
    sp.ng = (int)tm.size();
    sp.T = 1;
    for (int m : tm) sp.T *= p.dims[m];
    int local[SG_MAXQ];
    for (int i = 0; i < nq; ++i) local[i] = -1;
    {
      int s = 1;
      for (int k = sp.ng - 1; k >= 0; --k) {
        sp.tsh[k] = s;
        int lg = 0;
        while ((1 << lg) < s) ++lg;
        sp.tlg[k] = lg;
        s *= p.dims[tm[k]];
        local[tm[k]] = k;
      }
    }
    sp.no = 0;
    for (int m : order)
      if (!groups[g].count(m)) { sp.odim[sp.no] = p.dims[m]; sp.ost[sp.no] = st_int[m]; ++sp.no; }
    sp.D = p.D;
    sp.S = p.S;
    sp.ntpc = (int)(p.D / sp.T);
    sp.row = p.row;
    sp.n1 = 0;
    sp.par1 = 0;
    sp.nx = 0;
    for (int u = 0; u < p.n1; ++u) {
      if (slot_group[u] != g) continue;
      const int j = sp.n1++;
      sp.s1_k[j] = local[p.s1_mode[u]];
      sp.s1_off[j] = p.s1_off[u];
      if ((p.par1 >> u) & 1u) sp.par1 |= 1u << j;
      if (sp.nx >= kMaxX) { delete h; return nullptr; }
      sp.x_k[sp.nx] = local[p.s1_mode[u]]; sp.x_k2[sp.nx] = -1; sp.x_off2[sp.nx] = 0; sp.x_gslot[sp.nx] = u;
      ++sp.nx;
    }
    sp.ne = 0;
    sp.parL = sp.parR = 0;
    for (int e = 0; e < p.ne; ++e) {
      if (edge_group[e] != g) continue;
      const int j = sp.ne++;
      sp.e_ka[j] = local[p.e_a[e]];
      sp.e_kb[j] = local[p.e_b[e]];
      sp.e_offL[j] = p.e_offL[e];
      sp.e_offR[j] = p.e_offR[e];
      if ((p.parL >> e) & 1ull) sp.parL |= 1ull << j;
      if ((p.parR >> e) & 1ull) sp.parR |= 1ull << j;
      if (sp.nx + 2 > kMaxX) { delete h; return nullptr; }
      sp.x_k[sp.nx] = local[p.e_a[e]]; sp.x_k2[sp.nx] = local[p.e_b[e]]; sp.x_off2[sp.nx] = p.e_offR[e];
      sp.x_gslot[sp.nx] = p.n1 + e;
      ++sp.nx;
      sp.x_k[sp.nx] = local[p.e_b[e]]; sp.x_k2[sp.nx] = local[p.e_a[e]]; sp.x_off2[sp.nx] = p.e_offL[e];
      sp.x_gslot[sp.nx] = p.n1 + p.ne + e;
      ++sp.nx;
    }
    // offsets of the tile entries
    std::vector<int> off(sp.T);
    for (int t = 0; t < sp.T; ++t) {
      long long o = 0;
      for (int k = 0; k < sp.ng; ++k) o += (long long)((t / sp.tsh[k]) % p.dims[tm[k]]) * st_int[tm[k]];
      off[t] = (int)o;
    }
    if (cudaMalloc(&h->off_dev[g], sp.T * sizeof(int)) != cudaSuccess) { slab_plan_destroy(h); return nullptr; }
    cudaMemcpyAsync(h->off_dev[g], off.data(), sp.T * sizeof(int), cudaMemcpyHostToDevice, st);
    sp.off = h->off_dev[g];
    h->sm_fwd[g] = sp.T * csz + p.row * csz + sp.T * sizeof(int);
    h->sm_adj[g] = std::max(2 * sp.T * csz + p.row * csz + sp.T * sizeof(int),
                            (size_t)kMaxX * DL * DL * sizeof(double2));
    if (h->sm_adj[g] > 200 * 1024) { slab_plan_destroy(h); return nullptr; }
  }
  long long ntiles = (long long)p.S * (p.D / h->pass[0].T);
  h->grid_fwd = (int)std::min<long long>(ntiles, 152ll * (mixed ? 3 : 2));
  h->grid_adj = (int)std::min<long long>(ntiles, 152ll * (mixed ? 2 : 1));
  cudaStreamSynchronize(st);
  return h;
}

void slab_plan_destroy(SlabPlanHost* h) {
  if (!h) return;
  for (int g = 0; g < kMaxPass; ++g) if (h->off_dev[g]) cudaFree(h->off_dev[g]);
  delete h;
}

int slab_passes(const SlabPlanHost* h) { return h->np; }

size_t slab_partial_elems(const SlabPlanHost* h) {
  return (size_t)std::max(h->grid_adj, 1) * kMaxX * h->DL * h->DL;
}

static int perm_grid(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152ll * 16)); }

void slab_to_internal(const SlabPlanHost* h, const double2* api, double2* in, cudaStream_t st) {
  k_perm<<<perm_grid(h->perm.D * h->perm.S), 256, 0, st>>>(h->perm, api, in, 1);
}
void slab_from_internal(const SlabPlanHost* h, const double2* in, double2* api, cudaStream_t st) {
  k_perm<<<perm_grid(h->perm.D * h->perm.S), 256, 0, st>>>(h->perm, in, api, 0);
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------
namespace {

template <typename R, int DL, int STAGE, bool STORE, int KIND>
void fwd_launch(const SlabPlanHost* h, int g, const void* X, const void* row, const double2* pin,
                double2* pout, void* Xn, void* Dacc, void* kA, double dt, cudaStream_t st) {
  typedef typename CT<R>::T C;
  auto kern = k_slab_fwd<R, DL, STAGE, STORE, KIND>;
  static bool attr = false;
  if (!attr) { cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024); attr = true; }
  kern<<<h->grid_fwd, kST, h->sm_fwd[g], st>>>(h->pass[g], (const C*)X, (const C*)row, pin, pout,
                                                 (C*)Xn, (C*)Dacc, (C*)kA, dt);
}

template <typename R, int DL, int STAGE, bool STORE>
void fwd_stage(const SlabPlanHost* h, const void* X, const void* row, const double2* pin, double2* pout,
               void* Xn, void* Dacc, void* kA, double dt, cudaStream_t st) {
  if (h->np == 1) {
    fwd_launch<R, DL, STAGE, STORE, 3>(h, 0, X, row, pin, pout, Xn, Dacc, kA, dt, st);
    return;
  }
  fwd_launch<R, DL, STAGE, STORE, 0>(h, 0, X, row, pin, pout, Xn, Dacc, kA, dt, st);
  for (int g = 1; g < h->np - 1; ++g) fwd_launch<R, DL, STAGE, STORE, 1>(h, g, X, row, pin, pout, Xn, Dacc, kA, dt, st);
  fwd_launch<R, DL, STAGE, STORE, 2>(h, h->np - 1, X, row, pin, pout, Xn, Dacc, kA, dt, st);
}

template <typename R, int DL, int STAGE, int KIND>
void adj_launch(const SlabPlanHost* h, int g, const void* X, const void* Y, const void* row,
                double2* pbar, void* Xn, void* Db, void* yA, double dt, const XArgs& xa, cudaStream_t st) {
  typedef typename CT<R>::T C;
  auto kern = k_slab_adj<R, DL, STAGE, KIND>;
  static bool attr = false;
  if (!attr) { cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024); attr = true; }
  kern<<<h->grid_adj, kST, h->sm_adj[g], st>>>(h->pass[g], (const C*)X, (const C*)Y, (const C*)row, pbar,
                                                 (C*)Xn, (C*)Db, (C*)yA, dt, xa);
}

template <typename R, int DL, int STAGE>
void adj_stage(const SlabPlanHost* h, const void* X, const void* Y, const void* row, double2* pbar,
               void* Xn, void* Db, void* yA, double dt, const XArgs& xa, cudaStream_t st) {
  if (h->np == 1) {
    adj_launch<R, DL, STAGE, 3>(h, 0, X, Y, row, pbar, Xn, Db, yA, dt, xa, st);
    return;
  }
  adj_launch<R, DL, STAGE, 0>(h, 0, X, Y, row, pbar, Xn, Db, yA, dt, xa, st);
  for (int g = 1; g < h->np - 1; ++g) adj_launch<R, DL, STAGE, 1>(h, g, X, Y, row, pbar, Xn, Db, yA, dt, xa, st);
  adj_launch<R, DL, STAGE, 2>(h, h->np - 1, X, Y, row, pbar, Xn, Db, yA, dt, xa, st);
}

template <typename R>
const void* row_of(const void* tab, int row, int step, int j) {
  typedef typename CT<R>::T C;
  return static_cast<const C*>(tab) + ((size_t)3 * step + j) * row;
}

template <typename R, int DL>
int fwd_step_t(const SlabPlanHost* h, const void* tab, int step, const double2* pin, double2* pout,
               void*& X, void*& Xo, void* Dacc, void* kA, double dt, cudaStream_t st) {
  const int row = h->pass[0].row;
  fwd_stage<R, DL, 0, false>(h, X, row_of<R>(tab, row, step, 0), pin, nullptr, Xo, Dacc, kA, dt, st); std::swap(X, Xo);
  fwd_stage<R, DL, 1, false>(h, X, row_of<R>(tab, row, step, 1), pin, nullptr, Xo, Dacc, kA, dt, st); std::swap(X, Xo);
  fwd_stage<R, DL, 2, false>(h, X, row_of<R>(tab, row, step, 1), pin, nullptr, Xo, Dacc, kA, dt, st); std::swap(X, Xo);
  fwd_stage<R, DL, 3, false>(h, X, row_of<R>(tab, row, step, 2), pin, pout, Xo, Dacc, kA, dt, st); std::swap(X, Xo);
  return 4 * h->np;
}

template <typename R, int DL>
int fwd_store_t(const SlabPlanHost* h, const void* tab, int step, const double2* psi, void* const Y[4],
                void* kA, double dt, cudaStream_t st) {
  const int row = h->pass[0].row;
  fwd_stage<R, DL, 0, true>(h, Y[0], row_of<R>(tab, row, step, 0), psi, nullptr, Y[1], nullptr, kA, dt, st);
  fwd_stage<R, DL, 1, true>(h, Y[1], row_of<R>(tab, row, step, 1), psi, nullptr, Y[2], nullptr, kA, dt, st);
  fwd_stage<R, DL, 2, true>(h, Y[2], row_of<R>(tab, row, step, 1), psi, nullptr, Y[3], nullptr, kA, dt, st);
  return 3 * h->np;
}

template <typename R, int DL>
int adj_step_t(const SlabPlanHost* h, const void* tab, int step, void* const Y[4], double2* pbar,
               void*& KB, void*& KB2, void* Db, void* yA, double dt, XArgs xa, const double2* tab64,
               const double* coef, const double2* ph, int sumd, int K, cudaStream_t st) {
  const int row = h->pass[0].row;
  auto set = [&](int j) {
    xa.q = 3 * step + j;
    xa.t = (double)(2 * step + j) * dt * 0.5;
    xa.tabrow = tab64 + (size_t)xa.q * row;
    xa.coef = coef + (size_t)xa.q * K;
    xa.ph = ph + (size_t)xa.q * sumd;
  };
  set(2);
  adj_stage<R, DL, 3>(h, KB, Y[3], row_of<R>(tab, row, step, 2), pbar, KB2, Db, yA, dt, xa, st); std::swap(KB, KB2);
  set(1);
  adj_stage<R, DL, 2>(h, KB, Y[2], row_of<R>(tab, row, step, 1), pbar, KB2, Db, yA, dt, xa, st); std::swap(KB, KB2);
  adj_stage<R, DL, 1>(h, KB, Y[1], row_of<R>(tab, row, step, 1), pbar, KB2, Db, yA, dt, xa, st); std::swap(KB, KB2);
  set(0);
  adj_stage<R, DL, 0>(h, KB, Y[0], row_of<R>(tab, row, step, 0), pbar, KB2, Db, yA, dt, xa, st); std::swap(KB, KB2);
  return 4 * h->np;
}

}  // namespace

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

int slab_fwd_step(const SlabPlanHost* h, bool mixed, const void* tab, int step, const double2* pin,
                  double2* pout, void*& X, void*& Xo, void* Dacc, void* kA, double dt, cudaStream_t st) {
  SLAB_DISPATCH(fwd_step_t, h, tab, step, pin, pout, X, Xo, Dacc, kA, dt, st);
}

int slab_fwd_store(const SlabPlanHost* h, bool mixed, const void* tab, int step, const double2* psi,
                   void* const Y[4], void* kA, double dt, cudaStream_t st) {
  SLAB_DISPATCH(fwd_store_t, h, tab, step, psi, Y, kA, dt, st);
}

int slab_adj_step(const SlabPlanHost* h, bool mixed, const void* tab, int step, void* const Y[4],
                  double2* pbar, void*& KB, void*& KB2, void* Db, void* yA, double dt, XArgs xa,
                  const double2* tab64, const double* coef, const double2* ph, int sumd, int K,
                  cudaStream_t st) {
  SLAB_DISPATCH(adj_step_t, h, tab, step, Y, pbar, KB, KB2, Db, yA, dt, xa, tab64, coef, ph, sumd, K, st);
}
