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
#include "slab_dev.cuh"
#include "slab_lean.cuh"
#include <algorithm>
#include <cstdlib>
#include <set>
#include <vector>

namespace {


// KIND: 0 first partial pass (kA = k), 1 middle partial (kA += k), 2 last pass after
// partials (k += kA then the RK4 epilogue), 3 single pass (epilogue).
template <typename R, int DL>
__global__ void __launch_bounds__(kST, sizeof(R) == 4 ? 3 : 1) k_slab_fwd(SlabPass sp, const typename CT<R>::T* __restrict__ X,
                                                     const typename CT<R>::T* __restrict__ tabrow,
                                                     const double2* __restrict__ psi_in, double2* psi_out,
                                                     typename CT<R>::T* __restrict__ Xn,
                                                     typename CT<R>::T* __restrict__ Dacc,
                                                     typename CT<R>::T* __restrict__ kA, double dt,
                                                     const int STAGE, const bool STORE, const int KIND) {
  typedef typename CT<R>::T C;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* ys = reinterpret_cast<C*>(smraw);
  C* ks = ys + spad(sp.T);
  C* M = ks + spad(sp.T);
  const int* __restrict__ off = sp.off;
  load_common(sp, tabrow, M);
  const long long ntiles = (long long)sp.S * sp.ntpc;
  const R h = (R)dt;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long base = tile_base(sp, tile);
    load_tile<DL, 8>(sp, X, base, off, ys);
    __syncthreads();
    pass_apply<DL>(sp, M, ys, ks);
    // epilogue, four entries per thread at a time so their loads are in flight together
    constexpr int EB = 4;
    for (int t0 = threadIdx.x; t0 < sp.T; t0 += kST * EB) {
      long long g[EB];
      C k[EB], pa[EB], dd[EB];
      double2 ps[EB];
      bool ok[EB];
#pragma unroll
      for (int j = 0; j < EB; ++j) {
        const int t = t0 + j * kST;
        ok[j] = t < sp.T;
        g[j] = ok[j] ? base + __ldg(off + t) : base;
        const C a = ok[j] ? ks[spos<DL>(t)] : cmk<C>(0.0, 0.0);
        k[j] = cmk<C>(a.y, -a.x);                   // -i H y
        pa[j] = (KIND == 1 || KIND == 2) && ok[j] ? kA[g[j]] : cmk<C>(0.0, 0.0);
        ps[j] = (KIND >= 2) && ok[j] ? psi_in[g[j]] : make_double2(0.0, 0.0);
        dd[j] = (KIND >= 2) && ok[j] && !STORE && STAGE > 0 ? Dacc[g[j]] : cmk<C>(0.0, 0.0);
      }
#pragma unroll
      for (int j = 0; j < EB; ++j) {
        if (!ok[j]) continue;
        C kk = k[j];
        if (KIND == 0) { kA[g[j]] = kk; continue; }
        if (KIND == 1) { kA[g[j]] = cmk<C>(pa[j].x + kk.x, pa[j].y + kk.y); continue; }
        if (KIND == 2) kk = cmk<C>(pa[j].x + kk.x, pa[j].y + kk.y);
        const C pr = to_c(ps[j], R(0));
        const C d = dd[j];
        if (STAGE == 0) {
          if (!STORE) Dacc[g[j]] = cmk<C>(h / 6 * kk.x, h / 6 * kk.y);
          Xn[g[j]] = cmk<C>(pr.x + h / 2 * kk.x, pr.y + h / 2 * kk.y);
        } else if (STAGE == 1) {
          if (!STORE) Dacc[g[j]] = cmk<C>(d.x + h / 3 * kk.x, d.y + h / 3 * kk.y);
          Xn[g[j]] = cmk<C>(pr.x + h / 2 * kk.x, pr.y + h / 2 * kk.y);
        } else if (STAGE == 2) {
          if (!STORE) Dacc[g[j]] = cmk<C>(d.x + h / 3 * kk.x, d.y + h / 3 * kk.y);
          Xn[g[j]] = cmk<C>(pr.x + h * kk.x, pr.y + h * kk.y);
        } else {
          R incx = d.x + h / 6 * kk.x, incy = d.y + h / 6 * kk.y;
          double2 pn = make_double2(ps[j].x + (double)incx, ps[j].y + (double)incy);
          psi_out[g[j]] = pn;
          Xn[g[j]] = to_c(pn, R(0));
        }
      }
    }
    __syncthreads();
  }
}

// Forward stage pass with real operators (slab_dev.cuh): the tile is loaded and
// rotated by the conjugate group phases, the phases apply real matrices, and the
// epilogue rotates back before the RK4 update of k_slab_fwd (same KIND / STAGE /
// STORE semantics).  Tile entry t = tid + 256 j has the phase lo[tid] hi[j].
template <typename R, int DL, bool PAR>
__global__ void __launch_bounds__(kST, sizeof(R) == 4 ? 2 : 1)
k_zslab_fwd(SlabPass sp, const typename CT<R>::T* __restrict__ X, const typename ZM<R>::T* __restrict__ zrow,
            const double2* __restrict__ phrow, const double2* __restrict__ psi_in, double2* psi_out,
            typename CT<R>::T* __restrict__ Xn, typename CT<R>::T* __restrict__ Dacc,
            typename CT<R>::T* __restrict__ kA, double dt, const int STAGE, const bool STORE, const int KIND) {
  typedef typename CT<R>::T C;
  typedef typename ZM<R>::T Z;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* ys = reinterpret_cast<C*>(smraw);
  C* ks = ys + spad(sp.T);
  C* plo = ks + spad(sp.T);                       // 256
  C* phi = plo + 256;                             // T / 256
  Z* M = reinterpret_cast<Z*>(smraw + zrow_smem_off(sp.T, sizeof(C)));
  const int* __restrict__ off = sp.off;
  for (int i = threadIdx.x; i < sp.row; i += blockDim.x) M[i] = zrow[i];
  zphase_tables<DL>(sp, phrow, plo, phi);
  __syncthreads();
  const int L = sp.T < 256 ? sp.T : 256;
  const C pl = threadIdx.x < L ? plo[threadIdx.x] : cmk<C>(1.0, 0.0);
  const long long ntiles = (long long)sp.S * sp.ntpc;
  const R h = (R)dt;
  constexpr int NB = 8;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long base = tile_base(sp, tile);
    // load, rotated into the real-operator basis: y_r = conj(P) y
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
        if (t < sp.T) ys[spos<DL>(t)] = zcmulc(zcmul(pl, phi[t / 256]), v[j]);
      }
    }
    __syncthreads();
    zpass_apply<DL, PAR, R>(sp, M, ys, ks, kST);
    constexpr int EB = 4;
    for (int t0 = threadIdx.x; t0 < sp.T; t0 += kST * EB) {
      long long g[EB];
      C k[EB], pa[EB], dd[EB];
      double2 ps[EB];
      bool ok[EB];
#pragma unroll
      for (int j = 0; j < EB; ++j) {
        const int t = t0 + j * kST;
        ok[j] = t < sp.T;
        g[j] = ok[j] ? base + __ldg(off + t) : base;
        const C a = ok[j] ? zcmul(zcmul(pl, phi[t / 256]), ks[spos<DL>(t)]) : cmk<C>(0.0, 0.0);
        k[j] = cmk<C>(a.y, -a.x);                   // -i H y
        pa[j] = (KIND == 1 || KIND == 2) && ok[j] ? kA[g[j]] : cmk<C>(0.0, 0.0);
        ps[j] = (KIND >= 2) && ok[j] ? psi_in[g[j]] : make_double2(0.0, 0.0);
        dd[j] = (KIND >= 2) && ok[j] && !STORE && STAGE > 0 ? Dacc[g[j]] : cmk<C>(0.0, 0.0);
      }
#pragma unroll
      for (int j = 0; j < EB; ++j) {
        if (!ok[j]) continue;
        C kk = k[j];
        if (KIND == 0) { kA[g[j]] = kk; continue; }
        if (KIND == 1) { kA[g[j]] = cmk<C>(pa[j].x + kk.x, pa[j].y + kk.y); continue; }
        if (KIND == 2) kk = cmk<C>(pa[j].x + kk.x, pa[j].y + kk.y);
        const C pr = to_c(ps[j], R(0));
        const C d = dd[j];
        if (STAGE == 0) {
          if (!STORE) Dacc[g[j]] = cmk<C>(h / 6 * kk.x, h / 6 * kk.y);
          Xn[g[j]] = cmk<C>(pr.x + h / 2 * kk.x, pr.y + h / 2 * kk.y);
        } else if (STAGE == 1) {
          if (!STORE) Dacc[g[j]] = cmk<C>(d.x + h / 3 * kk.x, d.y + h / 3 * kk.y);
          Xn[g[j]] = cmk<C>(pr.x + h / 2 * kk.x, pr.y + h / 2 * kk.y);
        } else if (STAGE == 2) {
          if (!STORE) Dacc[g[j]] = cmk<C>(d.x + h / 3 * kk.x, d.y + h / 3 * kk.y);
          Xn[g[j]] = cmk<C>(pr.x + h * kk.x, pr.y + h * kk.y);
        } else {
          R incx = d.x + h / 6 * kk.x, incy = d.y + h / 6 * kk.y;
          double2 pn = make_double2(ps[j].x + (double)incx, ps[j].y + (double)incy);
          psi_out[g[j]] = pn;
          Xn[g[j]] = to_c(pn, R(0));
        }
      }
    }
    __syncthreads();
  }
}

// Epilogue of the lean forward pass (slab_lean.cuh) for one pass kind and stage:
// thread tid's entries t = tid + 256 j, their H y rotated back to the frame basis,
// then the partial sum or the RK4 update of k_slab_fwd.
template <int KIND, int STAGE, bool STORE>
__device__ __forceinline__ void lepi_fwd(const float2* __restrict__ ks, const float2* __restrict__ phi, float2 pl,
                                         int s0, const int* __restrict__ ohi, long long bl,
                                         const double2* __restrict__ psi_in, double2* __restrict__ psi_out,
                                         float2* __restrict__ Xn, float2* __restrict__ Dacc,
                                         float2* __restrict__ kA, float h) {
  constexpr int EB = 8;
#pragma unroll
  for (int j0 = 0; j0 < lean::LJ; j0 += EB) {
    long long g[EB];
    float2 k[EB], pa[EB], dd[EB];
    double2 ps[EB];
#pragma unroll
    for (int jj = 0; jj < EB; ++jj) {
      const int j = j0 + jj;
      g[jj] = bl + ohi[j];
      const float2 a = zcmul(zcmul(pl, phi[j]), ks[s0 + 273 * j]);
      k[jj] = make_float2(a.y, -a.x);                 // -i H y
      if (KIND == 1 || KIND == 2) pa[jj] = kA[g[jj]];
      if (KIND >= 2) ps[jj] = psi_in[g[jj]];
      if (KIND >= 2 && !STORE && STAGE > 0) dd[jj] = Dacc[g[jj]];
    }
#pragma unroll
    for (int jj = 0; jj < EB; ++jj) {
      float2 kk = k[jj];
      if (KIND == 0) { kA[g[jj]] = kk; continue; }
      if (KIND == 1) { kA[g[jj]] = make_float2(pa[jj].x + kk.x, pa[jj].y + kk.y); continue; }
      if (KIND == 2) kk = make_float2(pa[jj].x + kk.x, pa[jj].y + kk.y);
      const float2 pr = make_float2((float)ps[jj].x, (float)ps[jj].y);
      if (STAGE == 0) {
        if (!STORE) Dacc[g[jj]] = make_float2(h / 6 * kk.x, h / 6 * kk.y);
        Xn[g[jj]] = make_float2(pr.x + h / 2 * kk.x, pr.y + h / 2 * kk.y);
      } else if (STAGE == 1) {
        if (!STORE) Dacc[g[jj]] = make_float2(dd[jj].x + h / 3 * kk.x, dd[jj].y + h / 3 * kk.y);
        Xn[g[jj]] = make_float2(pr.x + h / 2 * kk.x, pr.y + h / 2 * kk.y);
      } else if (STAGE == 2) {
        if (!STORE) Dacc[g[jj]] = make_float2(dd[jj].x + h / 3 * kk.x, dd[jj].y + h / 3 * kk.y);
        Xn[g[jj]] = make_float2(pr.x + h * kk.x, pr.y + h * kk.y);
      } else {
        const float incx = dd[jj].x + h / 6 * kk.x, incy = dd[jj].y + h / 6 * kk.y;
        const double2 pn = make_double2(ps[jj].x + (double)incx, ps[jj].y + (double)incy);
        psi_out[g[jj]] = pn;
        Xn[g[jj]] = make_float2((float)pn.x, (float)pn.y);
      }
    }
  }
}

// Lean forward stage pass: the operation of k_zslab_fwd<float, 4, true> on 4096-entry
// tiles, with the index work of slab_lean.cuh.  The next tile's entries stream into a
// dense shared-memory buffer by cp.async while the current tile's phases run; at the
// start of a tile they are rotated into the real-operator basis from there.
__global__ void __launch_bounds__(kST, 2)
k_lean_fwd(SlabPass sp, const float2* __restrict__ X, const float2* __restrict__ zrow,
           const double2* __restrict__ phrow, const double2* __restrict__ psi_in, double2* psi_out,
           float2* __restrict__ Xn, float2* __restrict__ Dacc, float2* __restrict__ kA, double dt,
           const int STAGE, const bool STORE, const int KIND) {
  using namespace lean;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ float2 phi[LJ];
  __shared__ int ohi[LJ];
  __shared__ int ohi2[LJ / 2];
  __shared__ int lph[kMaxPhase][kLph];
  float2* ys = reinterpret_cast<float2*>(smraw);
  float2* ks = ys + spad(LT);
  float2* raw = reinterpret_cast<float2*>(smraw + ((2 * spad(LT) * sizeof(float2) + 15) & ~(size_t)15));
  float2* M = raw + LT;
  const int tid = threadIdx.x;
  const long long ntiles = (long long)sp.S * sp.ntpc;
  const int olo2 = __ldg(sp.off + 2 * tid);
  if (tid < LJ / 2) ohi2[tid] = __ldg(sp.off + 2 * kST * tid);
  __syncthreads();
  if ((long long)blockIdx.x < ntiles) lprefetch(X, tile_base(sp, blockIdx.x) + olo2, ohi2, raw, tid);
  for (int i = tid; i < sp.row; i += blockDim.x) M[i] = zrow[i];
  float2 pl;
  int olo;
  lsetup(sp, phrow, phi, ohi, pl, olo);
  lphases_to_smem(sp, lph);
  const int s0 = tid + (tid >> 4);                  // spos(tid); spos(tid + 256 j) = s0 + 273 j
  const int nph = sp.nph;
  const float h = (float)dt;
  __shared__ LPf pf[3];
  __shared__ int npf;
  if (tid == 0) {
    int n = 0;
    if (KIND == 1 || KIND == 2) pf[n++] = LPf{reinterpret_cast<const char*>(kA), (int)sizeof(float2)};
    if (KIND >= 2) pf[n++] = LPf{reinterpret_cast<const char*>(psi_in), (int)sizeof(double2)};
    if (KIND >= 2 && !STORE && STAGE > 0) pf[n++] = LPf{reinterpret_cast<const char*>(Dacc), (int)sizeof(float2)};
    npf = n;
  }
  const bool contig = ltile_contig(sp, tid);        // (a barrier: pf and npf are visible after it)
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long tb = tile_base(sp, tile), bl = tb + olo;
    lprefetch_wait();
    __syncthreads();                                // every thread's copies of this tile landed
#pragma unroll
    for (int j = 0; j < LJ; ++j) ys[s0 + 273 * j] = zcmulc(zcmul(pl, phi[j]), raw[tid + kST * j]);
    __syncthreads();                                // raw is free again
    if (tile + gridDim.x < ntiles) lprefetch(X, tile_base(sp, tile + gridDim.x) + olo2, ohi2, raw, tid);
    // the epilogue's operands of this tile stream into L2 while its phases run
    lprefetch_l2(pf, npf, tb, bl, ohi, contig, tid);
    lpass(nph, lph, M, ys, ks, tid);
    if (KIND == 0) lepi_fwd<0, 0, false>(ks, phi, pl, s0, ohi, bl, psi_in, psi_out, Xn, Dacc, kA, h);
    else if (KIND == 1) lepi_fwd<1, 0, false>(ks, phi, pl, s0, ohi, bl, psi_in, psi_out, Xn, Dacc, kA, h);
    else {
      switch ((KIND == 3 ? 8 : 0) + 2 * STAGE + (STORE ? 1 : 0)) {
#define SG_LEPI(K, S, ST) case (K == 3 ? 8 : 0) + 2 * S + ST: \
        lepi_fwd<K, S, ST>(ks, phi, pl, s0, ohi, bl, psi_in, psi_out, Xn, Dacc, kA, h); break;
        SG_LEPI(2, 0, 0) SG_LEPI(2, 0, 1) SG_LEPI(2, 1, 0) SG_LEPI(2, 1, 1) SG_LEPI(2, 2, 0) SG_LEPI(2, 2, 1)
        SG_LEPI(2, 3, 0) SG_LEPI(3, 0, 0) SG_LEPI(3, 0, 1) SG_LEPI(3, 1, 0) SG_LEPI(3, 1, 1) SG_LEPI(3, 2, 0)
        SG_LEPI(3, 2, 1) SG_LEPI(3, 3, 0)
#undef SG_LEPI
        default: break;
      }
    }
    __syncthreads();
  }
  lprefetch_wait();
}

// The same forward pass, warp-specialised for FP32 tiles of >= 256 entries: 8
// compute warps run the phases of tile i while 8 memory warps write back tile
// i - 1 (epilogue) and load tile i + 1, two buffer pairs in shared memory.
// Protocol (named barriers, 512 arrivals each; b = i mod 2):
//   compute, per tile i:  sync LOADED[b] -> phases (barrier 1 among themselves)
//                         -> arrive COMPUTED[b]
//   memory:  load tiles 0, 1 -> arrive LOADED[0], LOADED[1]; per tile i: sync
//            COMPUTED[b] -> epilogue of tile i -> load tile i + 2 into buffer b ->
//            arrive LOADED[b]
// A buffer is reloaded only after its epilogue, and recomputed only after that
// load, so no barrier id ever has two generations pending.
constexpr int kWST = 512;
template <int DL, bool PAR>
__global__ void __launch_bounds__(kWST, 1)
k_zslab_fwd_ws(SlabPass sp, const float2* __restrict__ X, const float2* __restrict__ zrow,
               const double2* __restrict__ phrow, const double2* __restrict__ psi_in, double2* psi_out,
               float2* __restrict__ Xn, float2* __restrict__ Dacc, float2* __restrict__ kA, double dt,
               const int STAGE, const bool STORE, const int KIND) {
  typedef float2 C;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int TP = spad(sp.T);
  C* const tiles = reinterpret_cast<C*>(smraw);
  C* const plo = tiles + 4 * TP;                  // 256
  C* const phi = plo + 256;                       // T / 256
  float2* const M = reinterpret_cast<float2*>(smraw + zrow_smem_off(sp.T, sizeof(C), 4));
  for (int i = threadIdx.x; i < sp.row; i += blockDim.x) M[i] = zrow[i];
  zphase_tables<DL>(sp, phrow, plo, phi);
  __syncthreads();
  const long long ntiles = (long long)sp.S * sp.ntpc;
  const int n = blockIdx.x < ntiles ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
  if (threadIdx.x < kST) {
    // ---- compute warps
    for (int i = 0; i < n; ++i) {
      const int b = i & 1;
      nb_sync(2 + b, kWST);
      zpass_apply<DL, PAR, float>(sp, M, tiles + b * TP, tiles + (2 + b) * TP, kST, 1);
      __threadfence_block();
      nb_arrive(4 + b, kWST);
    }
    return;
  }
  // ---- memory warps: thread tm owns the tile entries t = tm + 256 j
  const int tm = threadIdx.x - kST;
  const C pl = plo[tm];
  const int* __restrict__ off = sp.off;
  const float h = (float)dt;
  auto load = [&](int i, C* ys) {
    const long long base = tile_base(sp, (long long)blockIdx.x + (long long)i * gridDim.x);
    constexpr int NB = 8;
    for (int t0 = tm; t0 < sp.T; t0 += kST * NB) {
      C v[NB];
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        const int t = t0 + j * kST;
        v[j] = t < sp.T ? X[base + __ldg(off + t)] : cmk<C>(0.0, 0.0);
      }
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        const int t = t0 + j * kST;
        if (t < sp.T) ys[spos<DL>(t)] = zcmulc(zcmul(pl, phi[t / 256]), v[j]);
      }
    }
    __threadfence_block();
  };
  auto epilogue = [&](int i, const C* ks) {
    const long long base = tile_base(sp, (long long)blockIdx.x + (long long)i * gridDim.x);
    constexpr int EB = 4;
    for (int t0 = tm; t0 < sp.T; t0 += kST * EB) {
      long long g[EB];
      C k[EB], pa[EB], dd[EB];
      double2 ps[EB];
      bool ok[EB];
#pragma unroll
      for (int j = 0; j < EB; ++j) {
        const int t = t0 + j * kST;
        ok[j] = t < sp.T;
        g[j] = ok[j] ? base + __ldg(off + t) : base;
        const C a = ok[j] ? zcmul(zcmul(pl, phi[t / 256]), ks[spos<DL>(t)]) : cmk<C>(0.0, 0.0);
        k[j] = cmk<C>(a.y, -a.x);                   // -i H y
        pa[j] = (KIND == 1 || KIND == 2) && ok[j] ? kA[g[j]] : cmk<C>(0.0, 0.0);
        ps[j] = (KIND >= 2) && ok[j] ? psi_in[g[j]] : make_double2(0.0, 0.0);
        dd[j] = (KIND >= 2) && ok[j] && !STORE && STAGE > 0 ? Dacc[g[j]] : cmk<C>(0.0, 0.0);
      }
#pragma unroll
      for (int j = 0; j < EB; ++j) {
        if (!ok[j]) continue;
        C kk = k[j];
        if (KIND == 0) { kA[g[j]] = kk; continue; }
        if (KIND == 1) { kA[g[j]] = cmk<C>(pa[j].x + kk.x, pa[j].y + kk.y); continue; }
        if (KIND == 2) kk = cmk<C>(pa[j].x + kk.x, pa[j].y + kk.y);
        const C pr = to_c(ps[j], 0.f);
        const C d = dd[j];
        if (STAGE == 0) {
          if (!STORE) Dacc[g[j]] = cmk<C>(h / 6 * kk.x, h / 6 * kk.y);
          Xn[g[j]] = cmk<C>(pr.x + h / 2 * kk.x, pr.y + h / 2 * kk.y);
        } else if (STAGE == 1) {
          if (!STORE) Dacc[g[j]] = cmk<C>(d.x + h / 3 * kk.x, d.y + h / 3 * kk.y);
          Xn[g[j]] = cmk<C>(pr.x + h / 2 * kk.x, pr.y + h / 2 * kk.y);
        } else if (STAGE == 2) {
          if (!STORE) Dacc[g[j]] = cmk<C>(d.x + h / 3 * kk.x, d.y + h / 3 * kk.y);
          Xn[g[j]] = cmk<C>(pr.x + h * kk.x, pr.y + h * kk.y);
        } else {
          const float incx = d.x + h / 6 * kk.x, incy = d.y + h / 6 * kk.y;
          const double2 pn = make_double2(ps[j].x + (double)incx, ps[j].y + (double)incy);
          psi_out[g[j]] = pn;
          Xn[g[j]] = to_c(pn, 0.f);
        }
      }
    }
  };
  if (n > 0) { load(0, tiles); nb_arrive(2, kWST); }
  if (n > 1) { load(1, tiles + TP); nb_arrive(3, kWST); }
  for (int i = 0; i < n; ++i) {
    const int b = i & 1;
    nb_sync(4 + b, kWST);
    epilogue(i, tiles + (2 + b) * TP);
    if (i + 2 < n) {
      load(i + 2, tiles + b * TP);
      nb_arrive(2 + b, kWST);
    }
  }
}

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


SlabPlanHost* slab_plan_create(const KPlan& p, bool mixed, cudaStream_t st, bool metadata_only) {
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
  h->st = st;
  h->DL = DL;
  h->np = np;
  h->mixed = mixed;
  h->perm.nq = nq; h->perm.S = p.S; h->perm.D = p.D;
  for (int i = 0; i < nq; ++i) { h->perm.dims[i] = p.dims[i]; h->perm.st_api[i] = p.st[i]; h->perm.st_int[i] = st_int[i]; }
  const size_t csz = mixed ? sizeof(float2) : sizeof(double2);
  int pass_low_mode[kMaxPass] = {0, 0, 0, 0};     // each pass's lowest tile digit
  for (int g = 0; g < np; ++g) {
    SlabPass& sp = h->pass[g];
    sp = SlabPass{};
    std::vector<int> tm;                  // tile modes in internal order
    for (int m : order) if (groups[g].count(m)) tm.push_back(m);
    pass_low_mode[g] = tm.back();
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
    {
      int eoff[SG_MAXQ], e = 0;                // offsets of each mode's levels in a phase row
      for (int i = 0; i < nq; ++i) { eoff[i] = e; e += p.dims[i]; }
      for (int k = 0; k < sp.ng; ++k) sp.tphoff[k] = eoff[tm[k]];
      for (int k = 0; k < sp.ng; ++k) sp.tmode[k] = tm[k];
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
    int s1_global[SG_MAXQ], e_global[SG_MAXEDGE];
    for (int u = 0; u < p.n1; ++u) {
      if (slot_group[u] != g) continue;
      const int j = sp.n1++;
      sp.s1_k[j] = local[p.s1_mode[u]];
      sp.s1_off[j] = p.s1_off[u];
      s1_global[j] = u;
      if ((p.par1 >> u) & 1u) sp.par1 |= 1u << j;
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
      e_global[j] = e;
    }
    // register-blocked phases: one per edge, 1-body terms fused into the first
    // phase holding their digit, or a phase of their own
    if (sp.ng < 2) { delete h; return nullptr; }
    sp.nph = 0;
    auto new_phase = [&](int ka, int kb) -> Phase* {
      if (sp.nph >= kMaxPhase) return nullptr;
      Phase& P = sp.ph[sp.nph++];
      P = Phase{};
      P.ka = ka; P.kb = kb;
      P.offL = P.offR = P.offA = P.offB = -1;
      P.ge = P.gA = P.gB = -1;
      P.par = 0;
      // other digits: the lowest even-exponent, the lowest odd-exponent, then the rest
      std::vector<int> others;
      for (int k = sp.ng - 1; k >= 0; --k) if (k != ka && k != kb) others.push_back(k);
      std::vector<int> ord;
      auto expo = [&](int k) { return sp.ng - 1 - k; };
      for (int k : others) if (expo(k) % 2 == 0) { ord.push_back(k); break; }
      for (int k : others) if (expo(k) % 2 == 1) { ord.push_back(k); break; }
      for (int k : others) if (std::find(ord.begin(), ord.end(), k) == ord.end()) ord.push_back(k);
      P.no = (int)ord.size();
      for (int j = 0; j < P.no; ++j) P.ost[j] = sp.tsh[ord[j]];
      return &P;
    };
    for (int j = 0; j < sp.ne; ++j) {
      Phase* P = new_phase(sp.e_ka[j], sp.e_kb[j]);
      if (!P) { delete h; return nullptr; }
      P->offL = sp.e_offL[j];
      P->offR = sp.e_offR[j];
      P->ge = e_global[j];
      if ((sp.parL >> j) & 1ull) P->par |= 1u;
      if ((sp.parR >> j) & 1ull) P->par |= 2u;
    }
    for (int j = 0; j < sp.n1; ++j) {
      const int k = sp.s1_k[j];
      const bool par = (sp.par1 >> j) & 1u;
      bool done = false;
      for (int q = 0; q < sp.nph && !done; ++q) {
        Phase& P = sp.ph[q];
        if (P.ka == k && P.offA < 0) { P.offA = sp.s1_off[j]; P.gA = s1_global[j]; if (par) P.par |= 4u; done = true; }
        else if (P.kb == k && P.offB < 0) { P.offB = sp.s1_off[j]; P.gB = s1_global[j]; if (par) P.par |= 8u; done = true; }
      }
      if (!done) {
        const int other = (k == sp.ng - 1) ? sp.ng - 2 : sp.ng - 1;
        Phase* P = new_phase(k, other);
        if (!P) { delete h; return nullptr; }
        P->offA = sp.s1_off[j];
        P->gA = s1_global[j];
        if (par) P->par |= 4u;
      }
    }
    for (int q = 0; q < sp.nph; ++q) {
      Phase& P = sp.ph[q];
      const bool pw2 = DL == 2 || DL == 4;
      auto pad = [&](int o) { return pw2 ? o + (o >> 4) + (o >> 8) : o; };
      P.psa = pad(sp.tsh[P.ka]);
      P.psb = pad(sp.tsh[P.kb]);
      for (int j = 0; j < P.no; ++j) P.pst[j] = pad(P.ost[j]);
      unsigned need = (P.offL >= 0 ? 3u : 0u) | (P.offA >= 0 ? 4u : 0u) | (P.offB >= 0 ? 8u : 0u);
      P.allpar = (P.par & need) == need ? 1 : 0;
    }
    // cross-density slots, phase by phase
    for (int q = 0; q < sp.nph; ++q) {
      const Phase& P = sp.ph[q];
      auto add = [&](int type, int gslot) {
        if (sp.nx >= kMaxX) return false;
        sp.x_ph[sp.nx] = q; sp.x_type[sp.nx] = type; sp.x_gslot[sp.nx] = gslot; ++sp.nx;
        return true;
      };
      bool ok = true;
      if (P.offL >= 0) { ok = ok && add(2, p.n1 + P.ge); ok = ok && add(3, p.n1 + p.ne + P.ge); }
      if (P.offA >= 0) ok = ok && add(0, P.gA);
      if (P.offB >= 0) ok = ok && add(1, P.gB);
      if (!ok) { delete h; return nullptr; }
    }
    // offsets of the tile entries
    std::vector<int> off(sp.T);
    for (int t = 0; t < sp.T; ++t) {
      long long o = 0;
      for (int k = 0; k < sp.ng; ++k) o += (long long)((t / sp.tsh[k]) % p.dims[tm[k]]) * st_int[tm[k]];
      off[t] = (int)o;
    }
    if (cudaMallocAsync(&h->off_dev[g], sp.T * sizeof(int), st) != cudaSuccess) { slab_plan_destroy(h); return nullptr; }
    cudaMemcpyAsync(h->off_dev[g], off.data(), sp.T * sizeof(int), cudaMemcpyHostToDevice, st);
    sp.off = h->off_dev[g];
    h->sm_fwd[g] = 2 * spad(sp.T) * csz + p.row * csz;
    h->sm_zfwd[g] = zrow_smem_off(sp.T, csz) + (size_t)p.row * 8;
    {
      const size_t ws = zrow_smem_off(sp.T, csz, 4) + (size_t)p.row * 8;
      h->sm_zws[g] = (mixed && sp.T >= 256 && ws <= kSlabSmemMax) ? ws : 0;
    }
    h->sm_adj[g] = std::max(3 * spad(sp.T) * csz + p.row * csz, (size_t)kMaxX * DL * DL * sizeof(double2));
    if (h->sm_adj[g] > kSlabSmemMax && !metadata_only) { slab_plan_destroy(h); return nullptr; }
  }
  h->allpar = true;
  for (int g = 0; g < np; ++g)
    for (int q = 0; q < h->pass[g].nph; ++q) h->allpar = h->allpar && h->pass[g].ph[q].allpar;
  h->sm_lean = ((2 * spad(lean::LT) * sizeof(float2) + 15) & ~(size_t)15) +
                (size_t)(lean::LT + p.row) * sizeof(float2);
  h->sm_lean_adj = ((3 * spad(lean::LT) * sizeof(float2) + 15) & ~(size_t)15) +
                   (size_t)(((p.row + 1) & ~1) + kMaxDrv * 16) * sizeof(float2);
  for (int g = 0; g < np; ++g)
    h->lean[g] = mixed && DL == 4 && h->allpar && h->pass[g].T == lean::LT && h->pass[g].ng == 6 &&
                 h->pass[g].nph <= kMaxPhase && h->sm_lean_adj <= kLeanSmemMax &&
                 h->sm_lean <= kLeanSmemMax && st_int[pass_low_mode[g]] == 1;
  long long ntiles = (long long)p.S * (p.D / h->pass[0].T);
  h->grid_fwd = (int)std::min<long long>(ntiles, 152ll * (mixed ? 3 : 1));
  h->grid_zfwd = (int)std::min<long long>(ntiles, 152ll * (mixed ? 2 : 1));
  h->grid_adj = (int)std::min<long long>(ntiles, 152ll * (mixed ? 2 : 1));
  cudaStreamSynchronize(st);
  return h;
}

void slab_plan_destroy(SlabPlanHost* h) {
  if (!h) return;
  slab_q2_free(h);
  for (int g = 0; g < kMaxPass; ++g) if (h->off_dev[g]) cudaFreeAsync(h->off_dev[g], h->st);
  delete h;
}

int slab_passes(const SlabPlanHost* h) { return h->np; }

bool slab_real_shape_ok(const SlabPlanHost* h) { return h->DL == 2 || h->DL == 4; }
bool slab_allpar(const SlabPlanHost* h) { return h->allpar; }
void slab_bind_real(SlabPlanHost* h, const void* ztab, const double2* ph, int sumd, const void* zop,
                    const int* drv_of_slot_start, const int* drv_list) {
  h->ztab = ztab;
  h->zph = ph;
  h->zsumd = sumd;
  h->zop = zop;
  h->zadj = zop != nullptr;
  const size_t csz = h->mixed ? sizeof(float2) : sizeof(double2);
  for (int g = 0; g < h->np && h->zadj; ++g) {
    SlabPass& sp = h->pass[g];
    sp.nd = 0;
    for (int x = 0; x < sp.nx && h->zadj; ++x) {
      if (sp.x_type[x] >= 2) continue;                 // coupling slots carry no drive
      const int u = sp.x_gslot[x];
      for (int i = drv_of_slot_start[u]; i < drv_of_slot_start[u + 1]; ++i) {
        if (sp.nd >= kMaxDrv) { h->zadj = false; break; }
        sp.d_ph[sp.nd] = sp.x_ph[x];
        sp.d_type[sp.nd] = sp.x_type[x];
        sp.d_k[sp.nd] = drv_list[i];
        ++sp.nd;
      }
    }
    h->sm_zadj[g] = zrow_smem_off(sp.T, csz, 3) + (size_t)(((sp.row + 1) & ~1) + sp.nd * h->DL * h->DL) * 8;
    if (h->sm_zadj[g] > kSlabSmemMax) h->zadj = false;
  }
}

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

// The warp-specialised real-operator forward pass runs only with SG_SLAB_WS=1: with
// 8 compute warps per SM its phases wait on dependencies and barriers (measured 25 %
// slower on the 10-fluxonium ring than the one-role kernel at 16 warps per SM).
bool zws_off() {
  const char* e = std::getenv("SG_SLAB_WS");
  return !(e && e[0] == '1');
}

// The lean FP32 passes run unless SG_SLAB_LEAN=0 (a test knob that keeps the
// general real-operator passes).
bool lean_on() {
  const char* e = std::getenv("SG_SLAB_LEAN");
  return !(e && e[0] == '0');
}

template <typename R, int DL>
void fwd_launch(const SlabPlanHost* h, int g, const void* X, const void* row, const double2* pin,
                double2* pout, void* Xn, void* Dacc, void* kA, double dt, cudaStream_t st, int stage,
                bool store, int kind, int q) {
  typedef typename CT<R>::T C;
  if constexpr (sizeof(R) == 4 && DL == 4) {
    if (h->ztab && h->lean[g] && zws_off() && lean_on() && ((uintptr_t)X & 15) == 0) {
      static const bool lattr = [] {
        cudaFuncSetAttribute(k_lean_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLeanSmemMax);
        return true;
      }();
      (void)lattr;
      k_lean_fwd<<<h->grid_zfwd, kST, h->sm_lean, st>>>(h->pass[g], (const float2*)X,
                                                        (const float2*)h->ztab + (size_t)q * h->pass[g].row,
                                                        h->zph + (size_t)q * h->zsumd, pin, pout, (float2*)Xn,
                                                        (float2*)Dacc, (float2*)kA, dt, stage, store, kind);
      return;
    }
  }
  if constexpr (DL == 2 || DL == 4) {
    if (h->ztab) {
      typedef typename ZM<R>::T Z;
      auto zk = h->allpar ? k_zslab_fwd<R, DL, true> : k_zslab_fwd<R, DL, false>;
      static const bool zattr = [] {
        cudaFuncSetAttribute(k_zslab_fwd<R, DL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSlabSmemMax);
        cudaFuncSetAttribute(k_zslab_fwd<R, DL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSlabSmemMax);
        return true;
      }();
      (void)zattr;
      if constexpr (sizeof(R) == 4) {
        if (h->sm_zws[g] && !zws_off()) {
          auto wk = h->allpar ? k_zslab_fwd_ws<DL, true> : k_zslab_fwd_ws<DL, false>;
          static const bool wattr = [] {
            cudaFuncSetAttribute(k_zslab_fwd_ws<DL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSlabSmemMax);
            cudaFuncSetAttribute(k_zslab_fwd_ws<DL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSlabSmemMax);
            return true;
          }();
          (void)wattr;
          const long long ntiles = (long long)h->pass[g].S * h->pass[g].ntpc;
          const int grid = (int)std::min<long long>(ntiles, 152);
          wk<<<grid, kWST, h->sm_zws[g], st>>>(h->pass[g], (const float2*)X,
                                              (const float2*)h->ztab + (size_t)q * h->pass[g].row,
                                              h->zph + (size_t)q * h->zsumd, pin, pout, (float2*)Xn,
                                              (float2*)Dacc, (float2*)kA, dt, stage, store, kind);
          return;
        }
      }
      zk<<<h->grid_zfwd, kST, h->sm_zfwd[g], st>>>(h->pass[g], (const C*)X,
                                                   (const Z*)h->ztab + (size_t)q * h->pass[g].row,
                                                   h->zph + (size_t)q * h->zsumd, pin, pout, (C*)Xn, (C*)Dacc,
                                                   (C*)kA, dt, stage, store, kind);
      return;
    }
  }
  auto kern = k_slab_fwd<R, DL>;
  // once per kernel, thread-safe (solves on several host threads launch the same kernels)
  static const bool attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSlabSmemMax) ==
                           cudaSuccess;
  (void)attr;
  kern<<<h->grid_fwd, kST, h->sm_fwd[g], st>>>(h->pass[g], (const C*)X, (const C*)row, pin, pout,
                                                 (C*)Xn, (C*)Dacc, (C*)kA, dt, stage, store, kind);
}

// One RK4 stage: the partial passes accumulate into kA, the last one applies the
// epilogue.  q: the stage slot 3 n + j of the stage's time.
template <typename R, int DL>
void fwd_stage(const SlabPlanHost* h, int stage, bool store, const void* X, const void* row,
               const double2* pin, double2* pout, void* Xn, void* Dacc, void* kA, double dt, cudaStream_t st,
               int q) {
  if (h->np == 1) {
    fwd_launch<R, DL>(h, 0, X, row, pin, pout, Xn, Dacc, kA, dt, st, stage, store, 3, q);
    return;
  }
  fwd_launch<R, DL>(h, 0, X, row, pin, pout, Xn, Dacc, kA, dt, st, stage, store, 0, q);
  for (int g = 1; g < h->np - 1; ++g)
    fwd_launch<R, DL>(h, g, X, row, pin, pout, Xn, Dacc, kA, dt, st, stage, store, 1, q);
  fwd_launch<R, DL>(h, h->np - 1, X, row, pin, pout, Xn, Dacc, kA, dt, st, stage, store, 2, q);
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
  const int q = 3 * step;
  fwd_stage<R, DL>(h, 0, false, X, row_of<R>(tab, row, step, 0), pin, nullptr, Xo, Dacc, kA, dt, st, q); std::swap(X, Xo);
  fwd_stage<R, DL>(h, 1, false, X, row_of<R>(tab, row, step, 1), pin, nullptr, Xo, Dacc, kA, dt, st, q + 1); std::swap(X, Xo);
  fwd_stage<R, DL>(h, 2, false, X, row_of<R>(tab, row, step, 1), pin, nullptr, Xo, Dacc, kA, dt, st, q + 1); std::swap(X, Xo);
  fwd_stage<R, DL>(h, 3, false, X, row_of<R>(tab, row, step, 2), pin, pout, Xo, Dacc, kA, dt, st, q + 2); std::swap(X, Xo);
  return 4 * h->np;
}

// Forward step that keeps every stage input: Yk[0..3] = y1..y4 of this step (Yk[0]
// holds y1 on entry), Ynext0 = y1 of the next step.
template <typename R, int DL>
int fwd_step_keep_t(const SlabPlanHost* h, const void* tab, int step, const double2* pin, double2* pout,
                    void* const Yk[4], void* Ynext0, void* Dacc, void* kA, double dt, cudaStream_t st) {
  const int row = h->pass[0].row;
  const int q = 3 * step;
  fwd_stage<R, DL>(h, 0, false, Yk[0], row_of<R>(tab, row, step, 0), pin, nullptr, Yk[1], Dacc, kA, dt, st, q);
  fwd_stage<R, DL>(h, 1, false, Yk[1], row_of<R>(tab, row, step, 1), pin, nullptr, Yk[2], Dacc, kA, dt, st, q + 1);
  fwd_stage<R, DL>(h, 2, false, Yk[2], row_of<R>(tab, row, step, 1), pin, nullptr, Yk[3], Dacc, kA, dt, st, q + 1);
  fwd_stage<R, DL>(h, 3, false, Yk[3], row_of<R>(tab, row, step, 2), pin, pout, Ynext0, Dacc, kA, dt, st, q + 2);
  return 4 * h->np;
}

template <typename R, int DL>
int fwd_store_t(const SlabPlanHost* h, const void* tab, int step, const double2* psi, void* const Y[4],
                void* kA, double dt, cudaStream_t st) {
  const int row = h->pass[0].row;
  const int q = 3 * step;
  fwd_stage<R, DL>(h, 0, true, Y[0], row_of<R>(tab, row, step, 0), psi, nullptr, Y[1], nullptr, kA, dt, st, q);
  fwd_stage<R, DL>(h, 1, true, Y[1], row_of<R>(tab, row, step, 1), psi, nullptr, Y[2], nullptr, kA, dt, st, q + 1);
  fwd_stage<R, DL>(h, 2, true, Y[2], row_of<R>(tab, row, step, 1), psi, nullptr, Y[3], nullptr, kA, dt, st, q + 1);
  return 3 * h->np;
}

}  // namespace


int slab_fwd_step(const SlabPlanHost* h, bool mixed, const void* tab, int step, const double2* pin,
                  double2* pout, void*& X, void*& Xo, void* Dacc, void* kA, double dt, cudaStream_t st) {
  SLAB_DISPATCH(fwd_step_t, h, tab, step, pin, pout, X, Xo, Dacc, kA, dt, st);
}

int slab_fwd_store(const SlabPlanHost* h, bool mixed, const void* tab, int step, const double2* psi,
                   void* const Y[4], void* kA, double dt, cudaStream_t st) {
  SLAB_DISPATCH(fwd_store_t, h, tab, step, psi, Y, kA, dt, st);
}

int slab_fwd_step_keep(const SlabPlanHost* h, bool mixed, const void* tab, int step, const double2* pin,
                       double2* pout, void* const Yk[4], void* Ynext0, void* Dacc, void* kA, double dt,
                       cudaStream_t st) {
  SLAB_DISPATCH(fwd_step_keep_t, h, tab, step, pin, pout, Yk, Ynext0, Dacc, kA, dt, st);
}

