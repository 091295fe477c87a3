// On-chip evolution kernels (see onchip.h).
//
// Shared-memory images: column c of a CTA's group starts at c * CS (CS = padded
// column stride, even, so every column and image is 16-byte aligned) and entry t of
// a column sits at spos(t), the bank-conflict-free padding of the tiled kernels.
// H is applied phase by phase with the register-blocked phases of the tiled kernels
// (slab_dev.cuh), one d x d block per thread.  (Splitting blocks into their d output
// columns to occupy more threads on small systems measured slower at every size:
// the extra loads and index arithmetic cost more than the added parallelism.)
//
// Mixed precision keeps the state (forward) and the co-state (adjoint) as
// float-float pairs (hi + lo, each FP32, renormalised after every addition), so the
// hot loop has no FP64 arithmetic, which runs at a small fraction of the FP32 rate
// on this part; the pair carries about 48 significant bits, more than the
// per-step FP32 increments it accumulates can use.  FP64 mode keeps complex128.
//
// Adjoint stage (reverse order 3, 2, 1, 0 of one RK4 step), warp-specialised:
//   phase warps:   ks = H kbar_s (phases, named barrier among them), then the
//                  epilogue: ybar = i ks, Db, pbar, next kbar (in place in ks);
//   density warps: the cross-densities of this stage's term slots between kbar_s
//                  and the stored stage input y_s, one warp per slot at a time,
//                  reduced across the warp and contracted by its lanes (one lane
//                  per level pair) into shared-memory accumulators.
// Both groups only read kbar_s, y_s and the stage row, so they run side by side;
// one CTA barrier ends the stage.  The next stage input arrives by a bulk copy
// (cp.async.bulk, completion on an mbarrier) and the next table rows by cp.async
// while the stage computes.
#include "sg_internal.h"
#include "kplan.h"
#include "grad.cuh"
#include "slab.h"
#include "slab_dev.cuh"
#include "onchip.h"
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <vector>
#include <algorithm>
#include <cstdint>
#include <cstdlib>

namespace {

// ---------------------------------------------------------------------------
// asynchronous copies and barriers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// cp.async of 4, 8 or 16 bytes global -> shared (no registers, completes at cp_wait_all)
__device__ __forceinline__ void cp4(void* s, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp8(void* s, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp16(void* s, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void cpv(float2* s, const float2* g) { cp8(s, g); }
__device__ __forceinline__ void cpv(double2* s, const double2* g) { cp16(s, g); }
__device__ __forceinline__ void cpv(float* s, const float* g) { cp4(s, g); }
__device__ __forceinline__ void cpv(double* s, const double* g) { cp8(s, g); }

__device__ __forceinline__ void mb_init(uint64_t* mb) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mb)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// One bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) into
// shared memory, completing a phase of mb.  Issued by one thread.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* mb) {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(mb)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(mb))
      : "memory");
}
__device__ __forceinline__ bool mb_try(uint64_t* mb, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(mb)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase `parity` of mb: true once the phase has completed,
// false after `limit` polls (about a second at the default limit).
__device__ __forceinline__ bool mb_wait_for(uint64_t* mb, unsigned parity, int limit) {
  for (int it = 0; it < limit; ++it) {
    if (mb_try(mb, parity)) return true;
    __nanosleep(64);
  }
  return false;
}
// Barrier among the first n threads of the CTA (n a multiple of 32); id 0 is __syncthreads.
__device__ __forceinline__ void bar_sub(int id, int n) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(n) : "memory");
}

// ---------------------------------------------------------------------------
// state: complex128, or float-float pairs in mixed precision
// ---------------------------------------------------------------------------
// hi + lo <- hi + lo + x with hi = fl(hi + lo) afterwards (TwoSum, then a fast
// renormalisation); exact up to the rounding of the low word.
__device__ __forceinline__ void ff_add(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bb = s - hi;
  const float e = (hi - (s - bb)) + (x - bb);
  const float l = lo + e;
  const float h2 = s + l;
  lo = l - (h2 - s);
  hi = h2;
}

template <typename R> struct StateArr;
template <> struct StateArr<double> {
  double2* p;
  __device__ void init(unsigned char* base, int n) { p = reinterpret_cast<double2*>(base); (void)n; }
  __device__ void set(int e, double2 v) { p[e] = v; }
  __device__ double2 get(int e) const { return p[e]; }
  __device__ double2 hi(int e) const { return p[e]; }
  __device__ void add(int e, double2 x) { p[e] = make_double2(p[e].x + x.x, p[e].y + x.y); }
};
template <> struct StateArr<float> {
  float2 *h, *l;
  __device__ void init(unsigned char* base, int n) {
    h = reinterpret_cast<float2*>(base);
    l = h + n;
  }
  // high words in shared memory, low words elsewhere (global memory when shared
  // memory is short: they are touched once per step)
  __device__ void init_split(unsigned char* base, float2* lo) {
    h = reinterpret_cast<float2*>(base);
    l = lo;
  }
  __device__ void set(int e, double2 v) {
    const float hx = __double2float_rn(v.x), hy = __double2float_rn(v.y);
    h[e] = make_float2(hx, hy);
    l[e] = make_float2(__double2float_rn(v.x - (double)hx), __double2float_rn(v.y - (double)hy));
  }
  __device__ double2 get(int e) const {
    return make_double2((double)h[e].x + (double)l[e].x, (double)h[e].y + (double)l[e].y);
  }
  __device__ float2 hi(int e) const { return h[e]; }
  __device__ void add(int e, float2 x) {
    float2 a = h[e], b = l[e];
    ff_add(a.x, b.x, x.x);
    ff_add(a.y, b.y, x.y);
    h[e] = a;
    l[e] = b;
  }
};

// ---------------------------------------------------------------------------
// plan arguments
// ---------------------------------------------------------------------------
struct OcArgs {
  int D, S, Sc, nbc, nbt, CS, CSP, ncta, row, K, sumd, n1, ne;
  int ent;               // Sc * D entries per CTA
  int npw;               // adjoint: phase warps (the rest compute cross-densities)
  int pblo_g;            // adjoint, mixed: co-state low words in global memory (shared memory short)
  // forward shared-memory byte offsets
  int f_ys, f_ks, f_ps, f_dl, f_M;
  // Q2 (products of local unitaries) shared-memory byte offsets: state, scratch, 1-body rows
  int q_ys, q_ks, q_M, q_G;
  // Q2 pulse-gradient backward: psi, psibar, two scratch images, rows (U^dag, L), warp
  // partials, then the coupling unitaries when they fit
  int b_x0, b_x1, b_x2, b_x3, b_rows, b_rowcap, b_red, b_G;
  // adjoint shared-memory byte offsets
  int a_xs, a_ks, a_ys, a_yn, a_db, a_pb, a_M, a_cf, a_ph, a_obD, a_obL, a_obR, a_ebB, a_ebL, a_ebR,
      a_jb, a_gs, a_sq;
  int rowA, Kp, sumdA;   // row, K and sumd rounded up to even counts
  long long accd;        // doubles per CTA accumulator block (global layout)
  // adjoint: polls of a bounded mbarrier wait, and a test knob (non-zero: CTA 0
  // skips the bulk copy of its first stage input, so that wait runs out)
  int wlim, skip_first;
};

// One solve of a batched launch: its tables, buffers and step range (the fields of
// the unbatched launch's arguments).  CTAs [b ncta, (b + 1) ncta) of a batched grid
// run solve b.
struct OcSys {
  const void* tab;
  const void* coef;
  const void* ph;
  const void* opd;
  const double2* psi_api;
  const double2* img_in;
  double2* psi_out;
  double2* ck_out;
  void* segY;
  double2* pbar_img;
  double* gF_cta;
  double* acc_cta;
  int* err;
  void* pblo;
  const double* J;       // coupling strengths of the solve (Hamiltonian-gradient contraction)
  long long nstK;
  int n0, n1, K;
};
constexpr int kOcMaxBatch = 24;
struct OcBatch {
  int nsys;              // 0: an unbatched launch (the kernel's own arguments)
  OcSys s[kOcMaxBatch];
};

template <int DL>
__device__ __forceinline__ int oc_pos(const OcArgs& oa, int e) {
  const int c = e / oa.D;
  const int t = e - c * oa.D;
  return c * oa.CS + spos<DL>(t);
}

// All phases over the CTA's Sc columns: ks = H ys, one d x d block per thread at a
// time (phase_block of the tiled kernels), by threads [0, nthr) with barrier `bar`
// among them after every phase.
template <int DL, typename C>
__device__ __forceinline__ void oc_apply(const SlabPass& sp, const OcArgs& oa, const C* __restrict__ M,
                                         const C* __restrict__ ys, C* __restrict__ ks, int nthr, int bar) {
  for (int q = 0; q < sp.nph; ++q) {
    const Phase& P = sp.ph[q];
    for (int b = threadIdx.x; b < oa.nbt; b += nthr) {
      const int c = b / oa.nbc;
      const int pb = blk_pos<DL>(P, b - c * oa.nbc) + c * oa.CS;
      if (P.allpar) phase_block<DL, true>(P, M, ys, ks, pb, q == 0);
      else phase_block<DL, false>(P, M, ys, ks, pb, q == 0);
    }
    if (bar == 0) __syncthreads();
    else bar_sub(bar, nthr);
  }
}

template <typename V>
__device__ __forceinline__ void issue_rows(const V* __restrict__ tab, int row, int q, V* dst, int tid, int nthr) {
  const V* src = tab + (size_t)q * row;
  for (int i = tid; i < row; i += nthr) cpv(dst + i, src + i);
}

__host__ __device__ __forceinline__ int stage_row(int s) { return s == 0 ? 0 : (s == 3 ? 2 : 1); }

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------
template <typename R, int DL>
__global__ void __launch_bounds__(kST, 1)
k_oc_fwd(SlabPass sp, OcArgs oa, const typename CT<R>::T* __restrict__ tab, const double2* __restrict__ psi_api,
         const double2* __restrict__ img_in, double2* __restrict__ psi_out, double2* __restrict__ ck_out, int K,
         int n0, int n1, double dt, typename CT<R>::T* __restrict__ segY, const __grid_constant__ OcBatch bt) {
  typedef typename CT<R>::T C;
  int cta = blockIdx.x;
  if (bt.nsys > 0) {
    const int b = blockIdx.x / oa.ncta;
    cta = blockIdx.x - b * oa.ncta;
    const OcSys& d = bt.s[b];
    tab = static_cast<const C*>(d.tab);
    psi_api = d.psi_api;
    img_in = d.img_in;
    psi_out = d.psi_out;
    ck_out = d.ck_out;
    K = d.K;
    n0 = d.n0;
    n1 = d.n1;
    segY = static_cast<C*>(d.segY);
  }
  extern __shared__ __align__(16) unsigned char sm[];
  C* ys = reinterpret_cast<C*>(sm + oa.f_ys);
  C* ks = reinterpret_cast<C*>(sm + oa.f_ks);
  StateArr<R> ps;
  ps.init(sm + oa.f_ps, oa.ent);
  C* dl = reinterpret_cast<C*>(sm + oa.f_dl);
  C* const M0 = reinterpret_cast<C*>(sm + oa.f_M);
  C* const M1 = M0 + oa.rowA;
  const R h = (R)dt;
  for (int e = threadIdx.x; e < oa.ent; e += blockDim.x) {
    const int c = e / oa.D, t = e - c * oa.D;
    const int col = cta * oa.Sc + c;
    double2 v = make_double2(0.0, 0.0);
    if (img_in) v = img_in[(size_t)cta * oa.ent + e];
    else if (col < oa.S) v = psi_api[(size_t)t * oa.S + col];
    ps.set(e, v);
    ys[oc_pos<DL>(oa, e)] = ps.hi(e);
  }
  if (n0 < n1) issue_rows<C>(tab, oa.row, 3 * n0, M0, threadIdx.x, blockDim.x);
  cp_wait_all();
  __syncthreads();
  int buf = 0;
  for (int step = n0; step < n1; ++step) {
    if (ck_out && (step - n0) % K == 0) {
      double2* ck = ck_out + ((size_t)((step - n0) / K) * oa.ncta + cta) * oa.ent;
      for (int e = threadIdx.x; e < oa.ent; e += blockDim.x) ck[e] = ps.get(e);
    }
#pragma unroll 1
    for (int s = 0; s < 4; ++s) {
      C* const Mc = buf ? M1 : M0;
      // next stage's table row
      const int nstep = s < 3 ? step : step + 1, ns = s < 3 ? s + 1 : 0;
      if (nstep < n1) issue_rows<C>(tab, oa.row, 3 * nstep + stage_row(ns), buf ? M0 : M1, threadIdx.x, blockDim.x);
      if (segY) {
        C* g = segY + ((size_t)(4 * (step - n0) + s) * oa.ncta + cta) * oa.CSP;
        for (int e = threadIdx.x; e < oa.ent; e += blockDim.x) {
          const int pos = oc_pos<DL>(oa, e);
          g[pos] = ys[pos];
        }
      }
      oc_apply<DL>(sp, oa, Mc, ys, ks, blockDim.x, 0);
      for (int e = threadIdx.x; e < oa.ent; e += blockDim.x) {
        const int pos = oc_pos<DL>(oa, e);
        const C a = ks[pos];
        const C kk = cmk<C>(a.y, -a.x);                 // -i H y
        const C pr = ps.hi(e);
        if (s == 0) {
          dl[e] = cmk<C>(h / 6 * kk.x, h / 6 * kk.y);
          ys[pos] = cmk<C>(pr.x + h / 2 * kk.x, pr.y + h / 2 * kk.y);
        } else if (s == 1) {
          const C d = dl[e];
          dl[e] = cmk<C>(d.x + h / 3 * kk.x, d.y + h / 3 * kk.y);
          ys[pos] = cmk<C>(pr.x + h / 2 * kk.x, pr.y + h / 2 * kk.y);
        } else if (s == 2) {
          const C d = dl[e];
          dl[e] = cmk<C>(d.x + h / 3 * kk.x, d.y + h / 3 * kk.y);
          ys[pos] = cmk<C>(pr.x + h * kk.x, pr.y + h * kk.y);
        } else {
          const C d = dl[e];
          ps.add(e, cmk<C>(d.x + h / 6 * kk.x, d.y + h / 6 * kk.y));
          ys[pos] = ps.hi(e);
        }
      }
      cp_wait_all();
      __syncthreads();
      buf ^= 1;
    }
  }
  if (psi_out) {
    for (int e = threadIdx.x; e < oa.ent; e += blockDim.x) {
      const int c = e / oa.D, t = e - c * oa.D;
      const int col = cta * oa.Sc + c;
      if (col < oa.S) psi_out[(size_t)t * oa.S + col] = ps.get(e);
    }
  }
}

// ---------------------------------------------------------------------------
// adjoint
// ---------------------------------------------------------------------------
template <typename C>
__device__ __forceinline__ C shfl_xor_c(C v, int o) {
  v.x = __shfl_xor_sync(0xffffffffu, v.x, o);
  v.y = __shfl_xor_sync(0xffffffffu, v.y, o);
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename C> __device__ __forceinline__ C cmulT(C a, C b) {
  return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cconjT(C a) { return cmk<C>(a.x, -a.y); }

// Shared-memory accumulators of one CTA and segment (level-pair stride DL * DL, level stride DL).
template <typename T>
struct OcAcc {
  typedef typename CT<T>::T C;
  C *obD, *obL, *obR;
  T *ebB, *ebL, *ebR, *jb, *gs;
};

// eb[a] += sum_b qv(a, b) - sum_b qv(b, a) from the lanes' qv (lane = a * DL + b).
template <int DL, typename T>
__device__ __forceinline__ void eb_rowcol(T qv, int lane, T* sq, T* eb) {
  sq[lane] = qv;
  __syncwarp();
  if (lane < DL) {
    T s = 0;
#pragma unroll
    for (int b = 0; b < DL; ++b) s += sq[lane * DL + b] - sq[b * DL + lane];
    eb[lane] += s;
  }
  __syncwarp();
}

// Contraction of one slot's W (lane = level pair a * DL + b, lanes >= DL^2 hold 0)
// into the co-gradients: the sums of contract_slot spread over the warp, in the
// stage precision T.
//   1-body slot, drive k:  gF[q][k] = Re sum W O_k(t),    obD[k] += f_k conj(W P)
//   edge side:             jb += Re sum W A(t) (side a),  obL += J conj(W P), obR += conj(W P)
//   interaction frame:     eb[a] += sum_b qv(a, b) - qv(b, a),  qv = -Im(W_ab X_ab(t)) t
//   lab frame, 1-body:     eb[a] += Re W_aa
// with P_ab = exp(i (E_a - E_b) t) and X the stage's term matrix (B, L or R).
template <int DL, typename T>
__device__ __forceinline__ void oc_contract(const XArgs& xa, const double* Jb, const typename CT<T>::T* __restrict__ opd,
                                            int slot,
                                            typename CT<T>::T w, int lane, const typename CT<T>::T* tabrow,
                                            const T* cf, const typename CT<T>::T* phs, T t, int q, int s,
                                            const OcAcc<T>& A, T* sq, double* gFc) {
  typedef typename CT<T>::T C;
  const KPlan& p = xa.p;
  const bool inter = xa.frame == SG_FRAME_INTERACTION;
  const bool on = lane < DL * DL;
  const int ia = on ? lane / DL : 0, ib = on ? lane - ia * DL : 0;
  if (slot < p.n1) {
    const int u = slot, i = p.s1_mode[u];
    const C P = on ? cmulT(phs[xa.eoff[i] + ia], cconjT(phs[xa.eoff[i] + ib])) : cmk<C>(0.0, 0.0);
    for (int x = xa.drv_of_slot_start[u]; x < xa.drv_of_slot_start[u + 1]; ++x) {
      const int k = xa.drv_list[x];
      T g = 0;
      if (on) {
        const C Ot = cmulT(opd[xa.opd_off[i] + xa.drv_op[k] * DL * DL + lane], P);
        g = w.x * Ot.x - w.y * Ot.y;
        const C cw = cmulT(cconjT(w), cconjT(P));
        const T fk = cf[k];
        C& ob = A.obD[k * DL * DL + lane];
        ob.x += fk * cw.x;
        ob.y += fk * cw.y;
      }
      g = warp_sum(g);
      if (lane == 0) {
        // stages 2 and 1 share the slot q = 3n + 1: hold stage 2's share, store once
        if (s == 2) A.gs[k] = g;
        else gFc[(size_t)q * xa.K + k] = s == 1 ? (double)A.gs[k] + (double)g : (double)g;
      }
    }
    T* eb = A.ebB + u * DL;
    if (inter) {
      T qv = 0;
      if (on) {
        const C v = cmulT(w, tabrow[p.s1_off[u] + lane]);
        qv = -v.y * t;
      }
      eb_rowcol<DL>(qv, lane, sq, eb);
    } else if (on && ia == ib) {
      eb[ia] += w.x;
    }
    return;
  }
  const int side = (slot - p.n1) / p.ne, qe = (slot - p.n1) % p.ne;
  const int i = side == 0 ? p.e_a[qe] : p.e_b[qe];
  const int op = side == 0 ? xa.e_opa[qe] : xa.e_opb[qe];
  const T sc = side == 0 ? (T)(Jb ? Jb[qe] : xa.J[qe]) : (T)1;
  T jg = 0;
  if (on) {
    const C P = cmulT(phs[xa.eoff[i] + ia], cconjT(phs[xa.eoff[i] + ib]));
    const C At = cmulT(opd[xa.opd_off[i] + op * DL * DL + lane], P);
    jg = w.x * At.x - w.y * At.y;
    const C cw = cmulT(cconjT(w), cconjT(P));
    C& ob = (side == 0 ? A.obL : A.obR)[qe * DL * DL + lane];
    ob.x += sc * cw.x;
    ob.y += sc * cw.y;
  }
  if (inter) {
    T qv = 0;
    if (on) {
      const C v = cmulT(w, tabrow[(side == 0 ? p.e_offL[qe] : p.e_offR[qe]) + lane]);
      qv = -v.y * t;
    }
    eb_rowcol<DL>(qv, lane, sq, (side == 0 ? A.ebL : A.ebR) + qe * DL);
  }
  if (side == 0) {
    jg = warp_sum(jg);
    if (lane == 0) A.jb[qe] += jg;
  }
}

template <typename R, int DL, bool PARX>
__global__ void __launch_bounds__(kST, 1)
k_oc_adj(SlabPass sp, OcArgs oa, const typename CT<R>::T* __restrict__ tab, const R* __restrict__ coef,
         const typename CT<R>::T* __restrict__ ph, const typename CT<R>::T* __restrict__ opd,
         const typename CT<R>::T* __restrict__ segY, double2* __restrict__ pbar_img, int n0, int n1, double dt,
         XArgs xa, double* __restrict__ gF_cta, double* __restrict__ acc_cta, long long nstK,
         int* __restrict__ err, float2* __restrict__ pblo, const __grid_constant__ OcBatch bt) {
  typedef typename CT<R>::T C;
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  int cta = blockIdx.x;
  const double* Jb = nullptr;                           // the solve's couplings (batched), else xa.J
  if (bt.nsys > 0) {
    const int b = blockIdx.x / oa.ncta;
    cta = blockIdx.x - b * oa.ncta;
    const OcSys& d = bt.s[b];
    tab = static_cast<const C*>(d.tab);
    coef = static_cast<const R*>(d.coef);
    ph = static_cast<const C*>(d.ph);
    opd = static_cast<const C*>(d.opd);
    segY = static_cast<const C*>(d.segY);
    pbar_img = d.pbar_img;
    n0 = d.n0;
    n1 = d.n1;
    gF_cta = d.gF_cta;
    acc_cta = d.acc_cta;
    nstK = d.nstK;
    err = d.err;
    pblo = static_cast<float2*>(d.pblo);
    Jb = d.J;
  }
  (void)pblo;
  C* xs = reinterpret_cast<C*>(sm + oa.a_xs);
  C* ks = reinterpret_cast<C*>(sm + oa.a_ks);
  C* ys = reinterpret_cast<C*>(sm + oa.a_ys);
  C* yn = reinterpret_cast<C*>(sm + oa.a_yn);
  C* db = reinterpret_cast<C*>(sm + oa.a_db);
  StateArr<R> pb;
  if constexpr (sizeof(R) == 4) {
    if (oa.pblo_g) pb.init_split(sm + oa.a_pb, pblo + (size_t)cta * oa.ent);
    else pb.init(sm + oa.a_pb, oa.ent);
  } else {
    pb.init(sm + oa.a_pb, oa.ent);
  }
  C* const M0 = reinterpret_cast<C*>(sm + oa.a_M);
  C* const M1 = M0 + oa.rowA;
  R* const cf0 = reinterpret_cast<R*>(sm + oa.a_cf);
  R* const cf1 = cf0 + oa.Kp;
  C* const ph0 = reinterpret_cast<C*>(sm + oa.a_ph);
  C* const ph1 = ph0 + oa.sumdA;
  OcAcc<R> A;
  A.obD = reinterpret_cast<C*>(sm + oa.a_obD);
  A.obL = reinterpret_cast<C*>(sm + oa.a_obL);
  A.obR = reinterpret_cast<C*>(sm + oa.a_obR);
  A.ebB = reinterpret_cast<R*>(sm + oa.a_ebB);
  A.ebL = reinterpret_cast<R*>(sm + oa.a_ebL);
  A.ebR = reinterpret_cast<R*>(sm + oa.a_ebR);
  A.jb = reinterpret_cast<R*>(sm + oa.a_jb);
  A.gs = reinterpret_cast<R*>(sm + oa.a_gs);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nphase = oa.npw * 32;                      // phase threads: [0, nphase)
  const int nxw = kST / 32 - oa.npw;                   // density warps: [npw, 8)
  R* sq = reinterpret_cast<R*>(sm + oa.a_sq) + warp * 32;
  const R h = (R)dt;
  const int DD = DL * DL;
  for (int i = threadIdx.x; i < oa.K * DD; i += blockDim.x) A.obD[i] = cmk<C>(0.0, 0.0);
  for (int i = threadIdx.x; i < oa.ne * DD; i += blockDim.x) A.obL[i] = A.obR[i] = cmk<C>(0.0, 0.0);
  for (int i = threadIdx.x; i < oa.n1 * DL; i += blockDim.x) A.ebB[i] = 0;
  for (int i = threadIdx.x; i < oa.ne * DL; i += blockDim.x) A.ebL[i] = A.ebR[i] = 0;
  for (int i = threadIdx.x; i < oa.ne; i += blockDim.x) A.jb[i] = 0;
  for (int i = threadIdx.x; i < oa.K; i += blockDim.x) A.gs[i] = 0;
  if (threadIdx.x == 0) mb_init(&mbar);
  // co-state, and kbar_4 = dt/6 pbar of the segment's last step (the epilogue's formula)
  for (int e = threadIdx.x; e < oa.ent; e += blockDim.x) {
    pb.set(e, pbar_img[(size_t)cta * oa.ent + e]);
    const C qv = pb.hi(e);
    xs[oc_pos<DL>(oa, e)] = cmk<C>(h / 6 * qv.x, h / 6 * qv.y);
  }
  __syncthreads();
  const unsigned img_bytes = (unsigned)(oa.CSP * sizeof(C));
  double* gFc = gF_cta + (size_t)cta * nstK;
  // prefetch of stage s of step n: its input into ydst, its rows into buffer b
  auto issue = [&](int n, int s, C* ydst, int b, bool skip) {
    if (threadIdx.x == 0 && !skip)
      bulk_load(ydst, segY + ((size_t)(4 * (n - n0) + s) * oa.ncta + cta) * oa.CSP, img_bytes, &mbar);
    const int q = 3 * n + stage_row(s);
    issue_rows<C>(tab, oa.row, q, b ? M1 : M0, threadIdx.x, blockDim.x);
    issue_rows<R>(coef, oa.K, q, b ? cf1 : cf0, threadIdx.x, blockDim.x);
    issue_rows<C>(ph, oa.sumd, q, b ? ph1 : ph0, threadIdx.x, blockDim.x);
  };
  // A wait that runs out sets *err and stops the CTA's bulk copies (the CTA computes
  // on to its end with what it has, every access in bounds); before it exits it
  // waits, again bounded, for the copy it gave up on.  The CTA agrees on each
  // outcome by a barrier vote, so `aborted` is uniform.
  unsigned parity = 0, lost_parity = 0;
  bool aborted = false;
  auto vote = [&](bool ok, unsigned par) {
    if (!__syncthreads_and(ok ? 1 : 0) && !aborted) {
      aborted = true;
      lost_parity = par;
      if (threadIdx.x == 0) atomicExch(err, 1);
    }
  };
  bool ok0 = true;
  if (n0 < n1) {
    issue(n1 - 1, 3, ys, 0, oa.skip_first != 0 && cta == 0);
    cp_wait_all();
    ok0 = mb_wait_for(&mbar, parity, oa.wlim);
    parity ^= 1;
  }
  vote(ok0, parity ^ 1);
  int buf = 0;
  constexpr int NA = xd_n<DL, PARX>();
  for (int step = n1 - 1; step >= n0; --step) {
#pragma unroll 1
    for (int s = 3; s >= 0; --s) {
      const int q = 3 * step + stage_row(s);
      const R tq = (R)((double)(2 * step + stage_row(s)) * dt * 0.5);
      const int pn = s > 0 ? step : step - 1, psn = s > 0 ? s - 1 : 3;
      const bool more = pn >= n0;
      const C* Mc = buf ? M1 : M0;
      if (more) issue(pn, psn, yn, buf ^ 1, aborted);
      if (warp < oa.npw) {
        // phase warps: ks = H kbar_s, then the adjoint epilogue
        oc_apply<DL>(sp, oa, Mc, xs, ks, nphase, 1);
        for (int e = threadIdx.x; e < oa.ent; e += nphase) {
          const int pos = oc_pos<DL>(oa, e);
          const C a = ks[pos];
          const C y = cmk<C>(-a.y, a.x);                 // ybar = i H kbar
          const C pr = pb.hi(e);
          if (s == 3) {
            db[e] = y;
            ks[pos] = cmk<C>(h / 3 * pr.x + h * y.x, h / 3 * pr.y + h * y.y);
          } else if (s == 2) {
            const C d = db[e];
            db[e] = cmk<C>(d.x + y.x, d.y + y.y);
            ks[pos] = cmk<C>(h / 3 * pr.x + h / 2 * y.x, h / 3 * pr.y + h / 2 * y.y);
          } else if (s == 1) {
            const C d = db[e];
            db[e] = cmk<C>(d.x + y.x, d.y + y.y);
            ks[pos] = cmk<C>(h / 6 * pr.x + h / 2 * y.x, h / 6 * pr.y + h / 2 * y.y);
          } else {
            const C d = db[e];
            pb.add(e, cmk<C>(d.x + y.x, d.y + y.y));
            const C qq = pb.hi(e);
            ks[pos] = cmk<C>(h / 6 * qq.x, h / 6 * qq.y);
          }
        }
      } else {
        // density warps: cross-densities of this stage, one slot per warp at a time
        const C* phs = buf ? ph1 : ph0;
        const R* cfs = buf ? cf1 : cf0;
#pragma unroll 1
        for (int slot = warp - oa.npw; slot < sp.nx; slot += nxw) {
          const Phase& P = sp.ph[sp.x_ph[slot]];
          const int type = sp.x_type[slot];
          if (type >= 2 && !xa.ham) continue;         // coupling slot, not wanted (warp-uniform)
          C acc[NA];
#pragma unroll
          for (int a = 0; a < NA; ++a) acc[a] = cmk<C>(0.0, 0.0);
          for (int b = lane; b < oa.nbt; b += 32) {
            const int c = b / oa.nbc;
            xd_slot<DL, PARX>(P, type, Mc, xs, ys, blk_pos<DL>(P, b - c * oa.nbc) + c * oa.CS, acc);
          }
#pragma unroll
          for (int a = 0; a < NA; ++a)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              const C v = shfl_xor_c(acc[a], o);
              acc[a].x += v.x;
              acc[a].y += v.y;
            }
          // this lane's level pair
          C mine = cmk<C>(0.0, 0.0);
#pragma unroll
          for (int a = 0; a < DL; ++a)
#pragma unroll
            for (int b = 0; b < DL; ++b)
              if ((!PARX || ((a + b) & 1)) && lane == a * DL + b) mine = acc[xd_i<DL, PARX>(a, b)];
          const C w = cmk<C>(mine.y, -mine.x);             // W = -i C
          oc_contract<DL, R>(xa, Jb, opd, sp.x_gslot[slot], w, lane, Mc, cfs, phs, tq, q, s, A, sq, gFc);
        }
      }
      bool ok = true;
      if (more) {
        cp_wait_all();
        if (!aborted) ok = mb_wait_for(&mbar, parity, oa.wlim);
        parity ^= 1;
      }
      vote(ok, parity ^ 1);
      C* tswap = xs; xs = ks; ks = tswap;
      tswap = ys; ys = yn; yn = tswap;
      buf ^= 1;
    }
  }
  if (aborted) mb_wait_for(&mbar, lost_parity, oa.wlim);   // the copy given up on, if it is still in flight
  for (int e = threadIdx.x; e < oa.ent; e += blockDim.x) pbar_img[(size_t)cta * oa.ent + e] = pb.get(e);
  // add the segment's accumulators to the CTA's global block (GradAcc layout, SG_MAXD strides)
  double* G = acc_cta + (size_t)cta * oa.accd;
  const int MD2 = SG_MAXD * SG_MAXD;
  double* gD = G;
  double* gL = gD + 2ll * oa.K * MD2;
  double* gR = gL + 2ll * oa.ne * MD2;
  double* geB = gR + 2ll * oa.ne * MD2;
  double* geL = geB + (long long)oa.n1 * SG_MAXD;
  double* geR = geL + (long long)oa.ne * SG_MAXD;
  double* gjb = geR + (long long)oa.ne * SG_MAXD;
  for (int i = threadIdx.x; i < oa.K * DD; i += blockDim.x) {
    const int k = i / DD, ab = i - k * DD, a = ab / DL, b = ab - a * DL;
    double* g = gD + 2 * ((size_t)k * MD2 + a * SG_MAXD + b);
    g[0] += (double)A.obD[i].x;
    g[1] += (double)A.obD[i].y;
  }
  for (int i = threadIdx.x; i < oa.ne * DD; i += blockDim.x) {
    const int k = i / DD, ab = i - k * DD, a = ab / DL, b = ab - a * DL;
    double* g = gL + 2 * ((size_t)k * MD2 + a * SG_MAXD + b);
    g[0] += (double)A.obL[i].x;
    g[1] += (double)A.obL[i].y;
    g = gR + 2 * ((size_t)k * MD2 + a * SG_MAXD + b);
    g[0] += (double)A.obR[i].x;
    g[1] += (double)A.obR[i].y;
  }
  for (int i = threadIdx.x; i < oa.n1 * DL; i += blockDim.x) geB[(i / DL) * SG_MAXD + i % DL] += (double)A.ebB[i];
  for (int i = threadIdx.x; i < oa.ne * DL; i += blockDim.x) {
    geL[(i / DL) * SG_MAXD + i % DL] += (double)A.ebL[i];
    geR[(i / DL) * SG_MAXD + i % DL] += (double)A.ebR[i];
  }
  for (int i = threadIdx.x; i < oa.ne; i += blockDim.x) gjb[i] += (double)A.jb[i];
}

// ---------------------------------------------------------------------------
// second-order Suzuki-Trotter (Sec. 2.3, App. A): products of local unitaries
// ---------------------------------------------------------------------------
// Factor kinds: 0 = L (x) R of two modes' 1-body unitaries (row offsets offL, offR),
// 1 = one mode's 1-body unitary (offA), 2 = a coupling's d^2 x d^2 unitary (dense).
constexpr int kMaxQ2F = 40;
struct Q2Factor {
  Phase P;
  int kind;
  int mat;                        // kind 2: index of the d^4 matrix in the edge table
};
struct Q2Args {
  int nf0;                        // 1-body factors (applied first with the initial row,
                                  // and at the end of every step)
  int nfe;                        // coupling factors per step
  int J;                          // Q2 sub-steps per step (Q2 1, Q4 3, Q4j 2)
  int q1;                         // first-order product: each coupling once, full step
  int setoff[3];                  // first matrix of sub-step j's coupling set: 2 ne set(j)
  Q2Factor f[kMaxQ2F];            // [0, nf0): 1-body; [nf0, nf0 + nfe): couplings in order
};

template <int DL, typename C>
__device__ __forceinline__ void q2_apply(const Q2Factor& F, int mat, const OcArgs& oa, const C* __restrict__ M,
                                         const C* __restrict__ edges, const C* __restrict__ ys, C* __restrict__ ks) {
  const Phase& P = F.P;
  for (int b = threadIdx.x; b < oa.nbt; b += blockDim.x) {
    const int c = b / oa.nbc;
    const int pb = blk_pos<DL>(P, b - c * oa.nbc) + c * oa.CS;
    if (F.kind == 2) block_dense<DL>(edges + (size_t)mat * DL * DL * DL * DL, ys, ks, pb, P.psa, P.psb);
    else phase_block<DL, false>(P, M, ys, ks, pb, true);
  }
  __syncthreads();
}

// N Q2 sub-steps for the CTA's columns, lab frame.  rows: (N + 1) x nq x d^2 1-body
// unitaries (row N = the first half of sub-step 0, row n = the last half of sub-step n
// merged with the first of sub-step n + 1); edges: per coupling set (one per distinct
// sub-step length) and coupling the half-step and the full-step (middle) unitary.  Per
// sub-step: couplings 0 .. ne-2 (half), ne-1 (full), ne-2 .. 0 (half), then row n.
template <typename R, int DL>
__global__ void __launch_bounds__(kST, 1)
k_oc_q2(SlabPass sp, OcArgs oa, Q2Args qa, const typename CT<R>::T* __restrict__ rows,
        const typename CT<R>::T* __restrict__ edges, const double2* __restrict__ psi_api,
        double2* __restrict__ psi_out, int N, int rowlen, int nedge) {
  typedef typename CT<R>::T C;
  extern __shared__ __align__(16) unsigned char sm[];
  C* ys = reinterpret_cast<C*>(sm + oa.q_ys);
  C* ks = reinterpret_cast<C*>(sm + oa.q_ks);
  C* const M0 = reinterpret_cast<C*>(sm + oa.q_M);
  C* const M1 = M0 + oa.rowA;
  const int cta = blockIdx.x;
  // the coupling unitaries (constant for the solve) in shared memory when they fit
  const C* G = edges;
  if (nedge > 0) {
    C* Gs = reinterpret_cast<C*>(sm + oa.q_G);
    for (int i = threadIdx.x; i < nedge; i += blockDim.x) Gs[i] = edges[i];
    G = Gs;
  }
  for (int e = threadIdx.x; e < oa.ent; e += blockDim.x) {
    const int c = e / oa.D, t = e - c * oa.D;
    const int col = cta * oa.Sc + c;
    const double2 v = col < oa.S ? psi_api[(size_t)t * oa.S + col] : make_double2(0.0, 0.0);
    ys[oc_pos<DL>(oa, e)] = to_c(v, R(0));
  }
  issue_rows<C>(rows, rowlen, N, M0, threadIdx.x, blockDim.x);       // first half step
  if (N > 0) issue_rows<C>(rows, rowlen, 0, M1, threadIdx.x, blockDim.x);
  cp_wait_all();
  __syncthreads();
  for (int q = 0; q < qa.nf0; ++q) {
    q2_apply<DL>(qa.f[q], 0, oa, M0, G, ys, ks);
    C* t = ys; ys = ks; ks = t;
  }
  int buf = 1;
  for (int n = 0; n < N; ++n) {
    C* const Mc = buf ? M1 : M0;
    const int so = qa.setoff[n % qa.J];
    if (n + 1 < N) issue_rows<C>(rows, rowlen, n + 1, buf ? M0 : M1, threadIdx.x, blockDim.x);
    if (qa.q1) {
      for (int e = 0; e < qa.nfe; ++e) {                             // Q1: each coupling once, full step
        const Q2Factor& F = qa.f[qa.nf0 + e];
        q2_apply<DL>(F, F.mat + so + 1, oa, Mc, G, ys, ks);
        C* t = ys; ys = ks; ks = t;
      }
    } else {
      for (int q = 0; q < 2 * qa.nfe - 1; ++q) {
        const int e = q < qa.nfe ? q : 2 * qa.nfe - 2 - q;           // palindrome over couplings
        const Q2Factor& F = qa.f[qa.nf0 + e];
        q2_apply<DL>(F, F.mat + so + (q == qa.nfe - 1 ? 1 : 0), oa, Mc, G, ys, ks);   // middle: full step
        C* t = ys; ys = ks; ks = t;
      }
    }
    for (int q = 0; q < qa.nf0; ++q) {
      q2_apply<DL>(qa.f[q], 0, oa, Mc, G, ys, ks);
      C* t = ys; ys = ks; ks = t;
    }
    cp_wait_all();
    __syncthreads();
    buf ^= 1;
  }
  for (int e = threadIdx.x; e < oa.ent; e += blockDim.x) {
    const int c = e / oa.D, t = e - c * oa.D;
    const int col = cta * oa.Sc + c;
    if (col < oa.S) {
      const C v = ys[oc_pos<DL>(oa, e)];
      psi_out[(size_t)t * oa.S + col] = make_double2((double)v.x, (double)v.y);
    }
  }
}

// Backward of Q2 for the pulse gradient (Sec. 2.5 on the product of Sec. 2.3).  The
// final states psi and the co-state psibar (lab frame) are pulled back through every
// factor in reverse order, psi <- X^-1 psi and psibar <- X^dag psibar (X^-1 = X^dag for
// the unitary factors of Q2 and Q4; not for the complex steps of Q4j).  A 1-body half
// step is X = prod_i U_i (commuting factors on distinct modes), and for a drive k on
// mode i, dX/df_k = (prod_{j != i} U_j) L_k with L_k the Frechet derivative of the
// local exponential, so with the states before the half step
//   Re <psibar_after, dX/df_k psi_before> = Re <psibar_before, U_i^-1 L_k psi_before>
//                                         = Re sum_ab M_k[a][b] C_i[a][b],
// M_k = U_i^-1 L_k and C_i[a][b] = sum conj(psibar_before[a, ..]) psi_before[b, ..]
// the cross-density over mode i.  Each thread contracts its blocks' cross-densities
// with M_k at once, so a sub-step reduces one scalar per drive over the CTA (warp
// shuffles, then the warps in fixed order) into slot n (the sub-step) of the CTA's gF
// block.  The 1-body factors are applied as Kronecker pairs like the forward.  The
// first-order product Q1 takes the same route with one full-step 1-body factor per
// step and each coupling once.
constexpr int kQ2G = 16;          // drives of a Q2 gradient solve (per-thread partials)
struct Q2AdjArgs {
  int nq, K, ne, n1f;             // modes, drives, couplings, 1-body factors of a half step
  int J;                          // Q2 sub-steps per step
  int q1;                         // first-order product: per step the 1-body factors, then each coupling once
  int setoff[3];                  // first matrix of sub-step j's pull-back coupling set: 4 ne set(j)
  int row;                        // (nq + K) d^2: U_i(n)^dag then M_k(n)
  unsigned driven;                // bit i: a drive acts on mode i
  Phase one[SG_MAXQ / 2 + 1];     // pairs (offL, offR) and an odd last mode (offA)
  Phase mode[SG_MAXQ];            // cross-density block layout of mode i
  Phase edge[32];
  int drv_mode[kQ2G];
};

template <typename R, int DL>
__global__ void __launch_bounds__(kST, 1)
k_oc_q2_adj(SlabPass sp, OcArgs oa, Q2AdjArgs qa, const typename CT<R>::T* __restrict__ rows,
            const typename CT<R>::T* __restrict__ edges, const double2* __restrict__ psi_api,
            const double2* __restrict__ bar_api, int N, double* __restrict__ gF_cta, long long nstK,
            int nedge) {
  typedef typename CT<R>::T C;
  extern __shared__ __align__(16) unsigned char sm[];
  C* xs = reinterpret_cast<C*>(sm + oa.b_x0);         // psi
  C* xb = reinterpret_cast<C*>(sm + oa.b_x1);         // psibar
  C* t1 = reinterpret_cast<C*>(sm + oa.b_x2);
  C* t2 = reinterpret_cast<C*>(sm + oa.b_x3);
  C* const M0 = reinterpret_cast<C*>(sm + oa.b_rows);
  C* const M1 = M0 + oa.b_rowcap;
  double* red = reinterpret_cast<double*>(sm + oa.b_red);   // warps x kQ2G
  const C* G = edges;
  if (nedge > 0) {
    C* Gs = reinterpret_cast<C*>(sm + oa.b_G);
    for (int i = threadIdx.x; i < nedge; i += blockDim.x) Gs[i] = edges[i];
    G = Gs;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, cta = blockIdx.x;
  for (int e = threadIdx.x; e < oa.ent; e += blockDim.x) {
    const int c = e / oa.D, t = e - c * oa.D;
    const int col = cta * oa.Sc + c;
    const int pos = oc_pos<DL>(oa, e);
    xs[pos] = to_c(col < oa.S ? psi_api[(size_t)t * oa.S + col] : make_double2(0.0, 0.0), R(0));
    xb[pos] = to_c(col < oa.S ? bar_api[(size_t)t * oa.S + col] : make_double2(0.0, 0.0), R(0));
  }
  if (N > 0) issue_rows<C>(rows, qa.row, N - 1, M0, threadIdx.x, blockDim.x);
  cp_wait_all();
  __syncthreads();
  double* gFc = gF_cta + (size_t)cta * nstK;
  int buf = 0;
  for (int n = N - 1; n >= 0; --n) {
    const C* U = buf ? M1 : M0;                                        // U^-1 (states)
    const C* Ud = U + qa.nq * DL * DL;                                 // U^dag (co-states)
    const C* Mk = Ud + qa.nq * DL * DL;
    const int so = qa.setoff[n % qa.J];
    if (n > 0) issue_rows<C>(rows, qa.row, n - 1, buf ? M0 : M1, threadIdx.x, blockDim.x);
    R g[kQ2G];
#pragma unroll
    for (int k = 0; k < kQ2G; ++k) g[k] = R(0);
    // Q2: the second half step of the 1-body factors (h = 0), then the couplings and the
    // first half step (h = 1).  Q1: the couplings in reverse order over the full step,
    // then the step's full-step 1-body factors.
    for (int h = qa.q1; h < 2; ++h) {
      if (h == 1) {
        const int nqe = qa.q1 ? qa.ne : 2 * qa.ne - 1;
        for (int q = 0; q < nqe; ++q) {
          const int e = qa.q1 ? qa.ne - 1 - q : (q < qa.ne ? q : 2 * qa.ne - 2 - q);   // Q2: the palindrome
          const bool full = qa.q1 || q == qa.ne - 1;
          const C* Gi = G + (size_t)(so + 4 * e + (full ? 1 : 0)) * DL * DL * DL * DL;
          const C* Gd = Gi + (size_t)2 * DL * DL * DL * DL;
          const Phase& P = qa.edge[e];
          for (int b = threadIdx.x; b < oa.nbt; b += blockDim.x) {
            const int c = b / oa.nbc;
            const int pb = blk_pos<DL>(P, b - c * oa.nbc) + c * oa.CS;
            block_dense<DL>(Gi, xs, t1, pb, P.psa, P.psb);
            block_dense<DL>(Gd, xb, t2, pb, P.psa, P.psb);
          }
          __syncthreads();
          C* tmp = xs; xs = t1; t1 = tmp;
          tmp = xb; xb = t2; t2 = tmp;
        }
      }
      // the 1-body half step of step n (the second half first)
      for (int f = 0; f < qa.n1f; ++f) {
        const Phase& P = qa.one[f];
        for (int b = threadIdx.x; b < oa.nbt; b += blockDim.x) {
          const int c = b / oa.nbc;
          const int pb = blk_pos<DL>(P, b - c * oa.nbc) + c * oa.CS;
          phase_block<DL, false>(P, U, xs, t1, pb, true);
          phase_block<DL, false>(P, Ud, xb, t2, pb, true);
        }
        __syncthreads();
        C* tmp = xs; xs = t1; t1 = tmp;
        tmp = xb; xb = t2; t2 = tmp;
      }
      // cross-densities of the driven modes against the states before the half step
      for (int i = 0; i < qa.nq; ++i) {
        if (!((qa.driven >> i) & 1u)) continue;
        const Phase& P = qa.mode[i];
        for (int b = threadIdx.x; b < oa.nbt; b += blockDim.x) {
          const int c = b / oa.nbc;
          C acc[DL * DL];
#pragma unroll
          for (int a = 0; a < DL * DL; ++a) acc[a] = cmk<C>(0.0, 0.0);
          xd_slot<DL, false>(P, 0, U, xb, xs, blk_pos<DL>(P, b - c * oa.nbc) + c * oa.CS, acc);
#pragma unroll
          for (int k = 0; k < kQ2G; ++k) {
            if (k < qa.K && qa.drv_mode[k] == i) {
              const C* M = Mk + k * DL * DL;
              R v = R(0);
#pragma unroll
              for (int ab = 0; ab < DL * DL; ++ab) v += M[ab].x * acc[ab].x - M[ab].y * acc[ab].y;
              g[k] += v;
            }
          }
        }
      }
    }
    // one scalar per drive over the CTA: warps, then the warps in order
#pragma unroll
    for (int k = 0; k < kQ2G; ++k) {
      if (k < qa.K) {
        R v = g[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp * kQ2G + k] = (double)v;
      }
    }
    cp_wait_all();
    __syncthreads();
    if (threadIdx.x < qa.K) {
      double sacc = 0.0;
      for (int w = 0; w < kST / 32; ++w) sacc += red[w * kQ2G + threadIdx.x];
      gFc[(size_t)n * qa.K + threadIdx.x] += sacc;
    }
    buf ^= 1;
  }
}

// API layout [D][S] -> state image [cta][Sc][D]
__global__ void k_oc_image(OcArgs oa, const double2* __restrict__ api, double2* __restrict__ img) {
  const long long total = (long long)oa.ncta * oa.ent;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long col = e / oa.D;
    const int t = (int)(e - col * oa.D);
    img[e] = col < oa.S ? api[(size_t)t * oa.S + col] : make_double2(0.0, 0.0);
  }
}

// FP64 -> FP32 copy of the per-stage phase and coefficient tables and the operators.
__global__ void k_oc_f32(const double* __restrict__ src, float* __restrict__ dst, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = __double2float_rn(src[i]);
}

// Fixed-order sum over CTAs of the per-CTA gradient blocks.
struct RedArgs {
  long long nstK, accd;
  int ncta, K, n1, ne;
  GradAcc acc;
};
__global__ void k_oc_reduce(RedArgs r, const double* __restrict__ gF_cta, const double* __restrict__ acc_cta) {
  const long long MD2 = SG_MAXD * SG_MAXD;
  const long long total = r.nstK + r.accd;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    if (i < r.nstK) {
      for (int c = 0; c < r.ncta; ++c) s += gF_cta[(size_t)c * r.nstK + i];
      r.acc.gF[i] += s;
      continue;
    }
    long long j = i - r.nstK;
    for (int c = 0; c < r.ncta; ++c) s += acc_cta[(size_t)c * r.accd + j];
    const long long nD = 2 * r.K * MD2, nE = 2 * r.ne * MD2;
    if (j < nD) { reinterpret_cast<double*>(r.acc.obD)[j] += s; continue; }
    j -= nD;
    if (j < nE) { reinterpret_cast<double*>(r.acc.obL)[j] += s; continue; }
    j -= nE;
    if (j < nE) { reinterpret_cast<double*>(r.acc.obR)[j] += s; continue; }
    j -= nE;
    if (j < (long long)r.n1 * SG_MAXD) { r.acc.ebB[j] += s; continue; }
    j -= (long long)r.n1 * SG_MAXD;
    if (j < (long long)r.ne * SG_MAXD) { r.acc.ebL[j] += s; continue; }
    j -= (long long)r.ne * SG_MAXD;
    if (j < (long long)r.ne * SG_MAXD) { r.acc.ebR[j] += s; continue; }
    j -= (long long)r.ne * SG_MAXD;
    if (j < r.ne) r.acc.jb[j] += s;
  }
}

int grid_of(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152ll * 8)); }

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct OnchipPlan {
  SlabPlanHost* h = nullptr;
  OcArgs oa{};
  bool mixed = false, adj_ok = false, fwd_ok = false;
  size_t sm_fwd = 0, sm_adj = 0, limit = 0;
  // everything the plan is built from (the structure of the Kronecker-sum plan,
  // precision, drive count, energy-row length): plans with equal signatures are
  // equal, so their solves can share batched launches
  std::vector<long long> sig;
};

namespace {

size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

// Shared-memory layout for Sc columns per CTA; returns the forward and adjoint bytes.
void layout(OcArgs& a, int DL, size_t cs, size_t& fwd, size_t& adj) {
  const bool pw2 = DL == 2 || DL == 4;
  const size_t rs = cs / 2;                       // real of the stage precision
  a.CS = pw2 ? spad(a.D) : a.D;
  a.CS += a.CS & 1;
  a.CSP = a.Sc * a.CS;
  a.ent = a.Sc * a.D;
  a.nbt = a.Sc * a.nbc;
  a.rowA = a.row + (a.row & 1);
  a.Kp = std::max(2, a.K + (a.K & 1));
  a.sumdA = a.sumd + (a.sumd & 1);
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o = al16(o + bytes); return (int)r; };
  a.f_ys = take(a.CSP * cs);
  a.f_ks = take(a.CSP * cs);
  a.f_ps = take((size_t)a.ent * 16);
  a.f_dl = take((size_t)a.ent * cs);
  a.f_M = take(2 * (size_t)a.rowA * cs);
  fwd = o;
  o = 0;
  a.q_ys = take(a.CSP * cs);
  a.q_ks = take(a.CSP * cs);
  a.q_M = take(2 * (size_t)a.rowA * cs);
  a.q_G = (int)o;                 // coupling unitaries follow (sized per solve)
  o = 0;
  a.b_x0 = take(a.CSP * cs);
  a.b_x1 = take(a.CSP * cs);
  a.b_x2 = take(a.CSP * cs);
  a.b_x3 = take(a.CSP * cs);
  a.b_rowcap = 2 * a.rowA + a.K * DL * DL;                 // rowA >= nq d^2 in the lab frame
  a.b_rowcap += a.b_rowcap & 1;
  a.b_rows = take(2 * (size_t)a.b_rowcap * cs);            // double-buffered step rows
  a.b_red = take((size_t)(kST / 32) * 16 * sizeof(double));
  a.b_G = (int)o;
  o = 0;
  a.a_xs = take(a.CSP * cs);
  a.a_ks = take(a.CSP * cs);
  a.a_ys = take(a.CSP * cs);
  a.a_yn = take(a.CSP * cs);
  a.a_db = take((size_t)a.ent * cs);
  a.a_pb = take((size_t)a.ent * (a.pblo_g ? 8 : 16));
  a.a_M = take(2 * (size_t)a.rowA * cs);
  a.a_cf = take(2 * (size_t)a.Kp * rs);
  a.a_ph = take(2 * (size_t)a.sumdA * cs);
  const int DD = DL * DL;
  a.a_obD = take((size_t)std::max(1, a.K) * DD * cs);
  a.a_obL = take((size_t)std::max(1, a.ne) * DD * cs);
  a.a_obR = take((size_t)std::max(1, a.ne) * DD * cs);
  a.a_ebB = take((size_t)std::max(1, a.n1) * DL * rs);
  a.a_ebL = take((size_t)std::max(1, a.ne) * DL * rs);
  a.a_ebR = take((size_t)std::max(1, a.ne) * DL * rs);
  a.a_jb = take((size_t)std::max(1, a.ne) * rs);
  a.a_gs = take((size_t)std::max(1, a.K) * rs);
  a.a_sq = take((size_t)(kST / 32) * 32 * rs);
  adj = o;
}

}  // namespace

namespace {
std::vector<long long> plan_signature(const KPlan& p, bool mixed, int K, int sumd) {
  std::vector<long long> v = {mixed ? 1 : 0, K, sumd, p.nq, p.S, p.D, p.n1, p.ne, p.row, p.dl, (long long)p.par1,
                              (long long)p.parL, (long long)p.parR};
  for (int i = 0; i < p.nq; ++i) { v.push_back(p.dims[i]); v.push_back(p.st[i]); }
  for (int u = 0; u < p.n1; ++u) { v.push_back(p.s1_mode[u]); v.push_back(p.s1_off[u]); }
  for (int e = 0; e < p.ne; ++e) {
    v.push_back(p.e_a[e]); v.push_back(p.e_b[e]); v.push_back(p.e_offL[e]); v.push_back(p.e_offR[e]);
  }
  return v;
}
}  // namespace

OnchipPlan* onchip_plan_create(const KPlan& p, bool mixed, int K, int sumd, cudaStream_t st) {
  if (p.nq < 2 || p.nq > SG_MAXQ) return nullptr;
  SlabPlanHost* h = slab_plan_create(p, mixed, st, true);
  if (!h) return nullptr;
  const int DL = h->DL;
  bool ok = h->np == 1 && DL >= 2 && DL <= 5 && p.D <= kTmax;
  // single-pass tiles use the API digit order (mode 0 most significant)
  long long s = 1;
  for (int i = p.nq - 1; i >= 0 && ok; --i) {
    ok = p.st[i] == s;
    s *= p.dims[i];
  }
  if (!ok) { slab_plan_destroy(h); return nullptr; }
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t limit = (size_t)std::max(0, optin - 1024);
  OnchipPlan* oc = new OnchipPlan();
  oc->sig = plan_signature(p, mixed, K, sumd);
  oc->h = h;
  oc->mixed = mixed;
  OcArgs& a = oc->oa;
  a.D = (int)p.D;
  a.S = p.S;
  a.nbc = a.D / (DL * DL);
  a.row = p.row;
  a.K = K;
  a.sumd = sumd;
  a.n1 = p.n1;
  a.ne = p.ne;
  const size_t cs = mixed ? sizeof(float2) : sizeof(double2);
  // Columns per CTA: as many as give every thread one block per phase, within shared
  // memory (fewer CTAs per solve amortise the per-stage barriers and contractions).
  int sc0 = std::max(1, std::min(p.S, (kST + a.nbc - 1) / std::max(1, a.nbc)));
  size_t fwd = 0, adj = 0;
  int best_adj = 0, best_fwd = 0;
  // mixed precision: if the adjoint does not fit at one column per CTA, retry with the
  // co-state's low words in global memory
  for (a.pblo_g = 0; a.pblo_g <= (mixed ? 1 : 0) && !best_adj; ++a.pblo_g) {
    for (int sc = sc0; sc >= 1; --sc) {
      a.Sc = sc;
      layout(a, DL, cs, fwd, adj);
      if (!best_fwd && fwd <= limit) best_fwd = sc;
      if (!best_adj && adj <= limit) { best_adj = sc; break; }
    }
    if (best_adj) break;
  }
  if (!best_adj) a.pblo_g = 0;
  int sc = best_adj ? best_adj : best_fwd;
  if (!sc) {
    // neither RK4 kernel fits: one column per CTA may still fit the Q2 kernel (state,
    // scratch and the 1-body rows only; the coupling unitaries go to shared memory only
    // if they fit too)
    a.Sc = 1;
    layout(a, DL, cs, fwd, adj);
    if ((size_t)a.q_G > limit) { onchip_plan_destroy(oc); return nullptr; }
    sc = 1;
  }
  // balance the columns over the CTAs
  a.ncta = (p.S + sc - 1) / sc;
  a.Sc = (p.S + a.ncta - 1) / a.ncta;
  layout(a, DL, cs, fwd, adj);
  oc->adj_ok = adj <= limit;
  oc->fwd_ok = fwd <= limit;
  oc->sm_fwd = fwd;
  oc->sm_adj = adj;
  oc->limit = limit;
  // Adjoint warp split from the complex multiply-adds per stage: a phase block costs
  // 2 d^3 per edge and d^3 per 1-body term, a slot's cross-density d^3 (1-body) or
  // 2 d^3 (edge side); parity-odd operators halve both.  SG_OC_PW overrides (1..7).
  {
    const SlabPass& sp0 = h->pass[0];
    double wp = 0.0, wx = 0.0;
    for (int q = 0; q < sp0.nph; ++q) {
      const Phase& P = sp0.ph[q];
      wp += (P.offL >= 0 ? 2.0 : 0.0) + (P.offA >= 0 ? 1.0 : 0.0) + (P.offB >= 0 ? 1.0 : 0.0);
    }
    for (int x = 0; x < sp0.nx; ++x) wx += sp0.x_type[x] >= 2 ? 2.0 : 1.0;
    const int nw = kST / 32;
    int npw = (int)std::lround(nw * wp / std::max(1e-9, wp + wx));
    npw = std::min(npw, (a.nbt + 31) / 32);                 // no idle phase warps
    npw = std::min(npw, nw - (sp0.nx + 3) / 4);             // at most 4 slots per density warp
    a.npw = std::max(1, std::min(nw - 1, npw));
    if (const char* e = std::getenv("SG_OC_PW")) a.npw = std::max(1, std::min(nw - 1, atoi(e)));
  }
  const long long MD2 = SG_MAXD * SG_MAXD;
  a.accd = 2 * (long long)K * MD2 + 4 * (long long)p.ne * MD2 + (long long)p.n1 * SG_MAXD +
           2 * (long long)p.ne * SG_MAXD + p.ne;
  return oc;
}

void onchip_plan_destroy(OnchipPlan* oc) {
  if (!oc) return;
  slab_plan_destroy(oc->h);
  delete oc;
}

bool onchip_adjoint_ok(const OnchipPlan* oc) { return oc && oc->adj_ok; }
bool onchip_forward_ok(const OnchipPlan* oc) { return oc && oc->fwd_ok; }
bool onchip_colow_global(const OnchipPlan* oc) { return oc->oa.pblo_g != 0; }
bool onchip_mixed(const OnchipPlan* oc) { return oc->mixed; }
long long onchip_state_elems(const OnchipPlan* oc) { return (long long)oc->oa.ncta * oc->oa.ent; }
long long onchip_stage_elems(const OnchipPlan* oc) { return (long long)oc->oa.ncta * oc->oa.CSP; }
int onchip_ctas(const OnchipPlan* oc) { return oc->oa.ncta; }
long long onchip_acc_doubles(const OnchipPlan* oc) { return oc->oa.accd; }

namespace {

// Raise a kernel's dynamic shared-memory limit to the device's opt-in maximum, once
// per kernel (the template parameter is the kernel itself: kernels of one signature
// share a type).  (Setting it per solve to the solve's own size races with concurrent
// solves of other sizes that launch the same kernel: a smaller size set between
// another solve's set and launch fails that launch.)
template <auto kern>
void smem_limit_once() {
  static const bool done = [] {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - 1024);
    return true;
  }();
  (void)done;
}

const OcBatch& no_batch() {
  static const OcBatch b{};
  return b;
}

template <typename R, int DL>
int fwd_t(const OnchipPlan* oc, const void* tab, const double2* psi_api, const double2* img_in, double2* psi_out,
          double2* ck_out, int K, int n0, int n1, double dt, void* segY, cudaStream_t st) {
  typedef typename CT<R>::T C;
  auto kern = k_oc_fwd<R, DL>;
  smem_limit_once<k_oc_fwd<R, DL>>();
  kern<<<oc->oa.ncta, kST, oc->sm_fwd, st>>>(oc->h->pass[0], oc->oa, (const C*)tab, psi_api, img_in, psi_out,
                                             ck_out, std::max(1, K), n0, n1, dt, (C*)segY, no_batch());
  return 1;
}

template <typename R, int DL>
int adj_t(const OnchipPlan* oc, const OnchipTables& tb, const void* segY, double2* pbar_img, int n0, int n1,
          double dt, const XArgs& xa, int nst, double* gF_cta, double* acc_cta, int* err, void* pblo,
          cudaStream_t st) {
  typedef typename CT<R>::T C;
  auto kern = oc->h->allpar ? k_oc_adj<R, DL, true> : k_oc_adj<R, DL, false>;
  smem_limit_once<k_oc_adj<R, DL, true>>();
  smem_limit_once<k_oc_adj<R, DL, false>>();
  OcArgs oa = oc->oa;
  // bounded-wait limit and the test knob that makes one wait run out (tests only)
  oa.wlim = 1 << 22;
  if (const char* e = std::getenv("SG_TEST_WAIT_LIMIT")) oa.wlim = std::max(1, atoi(e));
  const char* sk = std::getenv("SG_TEST_SKIP_BULK");
  oa.skip_first = sk && sk[0] == '1';
  kern<<<oa.ncta, kST, oc->sm_adj, st>>>(oc->h->pass[0], oa, (const C*)tb.tab, (const R*)tb.coef,
                                             (const C*)tb.ph, (const C*)tb.opd, (const C*)segY, pbar_img, n0, n1,
                                             dt, xa, gF_cta, acc_cta, (long long)nst * std::max(1, oc->oa.K), err,
                                             (float2*)pblo, no_batch());
  return 1;
}

// Batched launches: bt.nsys solves of oc's plan shape, CTAs [b ncta, (b + 1) ncta)
// running solve b.
template <typename R, int DL>
int fwd_batch_t(const OnchipPlan* oc, const OcBatch& bt, double dt, cudaStream_t st) {
  smem_limit_once<k_oc_fwd<R, DL>>();
  k_oc_fwd<R, DL><<<bt.nsys * oc->oa.ncta, kST, oc->sm_fwd, st>>>(oc->h->pass[0], oc->oa, nullptr, nullptr, nullptr,
                                                                  nullptr, nullptr, 1, 0, 0, dt, nullptr, bt);
  return 1;
}

template <typename R, int DL>
int adj_batch_t(const OnchipPlan* oc, const OcBatch& bt, double dt, const XArgs& xa, cudaStream_t st) {
  auto kern = oc->h->allpar ? k_oc_adj<R, DL, true> : k_oc_adj<R, DL, false>;
  smem_limit_once<k_oc_adj<R, DL, true>>();
  smem_limit_once<k_oc_adj<R, DL, false>>();
  OcArgs oa = oc->oa;
  oa.wlim = 1 << 22;
  if (const char* e = std::getenv("SG_TEST_WAIT_LIMIT")) oa.wlim = std::max(1, atoi(e));
  oa.skip_first = 0;
  kern<<<bt.nsys * oa.ncta, kST, oc->sm_adj, st>>>(oc->h->pass[0], oa, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                   nullptr, 0, 0, dt, xa, nullptr, nullptr, 0, nullptr, nullptr, bt);
  return 1;
}

}  // namespace

#define OC_DISPATCH(FN, ...)                                                                \
  do {                                                                                      \
    if (oc->mixed) {                                                                        \
      switch (oc->h->DL) {                                                                  \
        case 2: return FN<float, 2>(__VA_ARGS__);                                          \
        case 3: return FN<float, 3>(__VA_ARGS__);                                          \
        case 4: return FN<float, 4>(__VA_ARGS__);                                          \
        default: return FN<float, 5>(__VA_ARGS__);                                         \
      }                                                                                     \
    } else {                                                                                \
      switch (oc->h->DL) {                                                                  \
        case 2: return FN<double, 2>(__VA_ARGS__);                                         \
        case 3: return FN<double, 3>(__VA_ARGS__);                                         \
        case 4: return FN<double, 4>(__VA_ARGS__);                                         \
        default: return FN<double, 5>(__VA_ARGS__);                                        \
      }                                                                                     \
    }                                                                                       \
  } while (0)

// ---------------------------------------------------------------------------
// batcher
// ---------------------------------------------------------------------------
namespace {

struct OcPending {
  int kind;                     // 0 forward, 1 adjoint
  const OnchipPlan* oc;
  OcSys d;
  double dt;
  const XArgs* xa;              // adjoint: the plan's structural arguments
  cudaEvent_t ready, done;
};

thread_local OcBatcher* tl_batcher = nullptr;
thread_local cudaEvent_t tl_ready = nullptr, tl_done = nullptr;

// Two pending launches can share a batched launch: same kernel, plan shape and step.
bool oc_compatible(const OcPending& a, const OcPending& b) {
  if (a.kind != b.kind || a.dt != b.dt) return false;
  const OnchipPlan* x = a.oc;
  const OnchipPlan* y = b.oc;
  if (x == y) return true;
  if (a.kind == 1 && a.xa->ham != b.xa->ham) return false;
  return x->sig == y->sig && x->sm_fwd == y->sm_fwd && x->sm_adj == y->sm_adj;
}

template <typename R, int DL>
int batch_launch_t(const OnchipPlan* oc, int kind, const OcBatch& bt, double dt, const XArgs* xa, cudaStream_t st) {
  return kind == 0 ? fwd_batch_t<R, DL>(oc, bt, dt, st) : adj_batch_t<R, DL>(oc, bt, dt, *xa, st);
}
int batch_launch(const OnchipPlan* oc, int kind, const OcBatch& bt, double dt, const XArgs* xa, cudaStream_t st) {
  OC_DISPATCH(batch_launch_t, oc, kind, bt, dt, xa, st);
}

}  // namespace

struct OcBatcher {
  int device = 0;
  cudaStream_t st = nullptr;
  std::mutex mu;
  std::condition_variable cv;
  int participants = 0;
  std::vector<OcPending*> subs;
  unsigned long long gen = 0;
  long long launches = 0, members = 0;

  // Called with mu held once every participant has handed over a launch: groups
  // them into compatible batches and issues each on st after its members' earlier
  // work, with each member's done event after its batch.
  void launch_round() {
    std::vector<bool> taken(subs.size(), false);
    for (size_t i = 0; i < subs.size(); ++i) {
      if (taken[i]) continue;
      std::vector<OcPending*> grp;
      for (size_t j = i; j < subs.size() && (int)grp.size() < kOcMaxBatch; ++j)
        if (!taken[j] && oc_compatible(*subs[i], *subs[j])) { taken[j] = true; grp.push_back(subs[j]); }
      OcBatch bt{};
      bt.nsys = (int)grp.size();
      for (int b = 0; b < bt.nsys; ++b) {
        cudaStreamWaitEvent(st, grp[b]->ready, 0);
        bt.s[b] = grp[b]->d;
      }
      batch_launch(grp[0]->oc, grp[0]->kind, bt, grp[0]->dt, grp[0]->xa, st);
      for (OcPending* m : grp) cudaEventRecord(m->done, st);
      ++launches;
      members += bt.nsys;
    }
    subs.clear();
    ++gen;
    cv.notify_all();
  }

  int submit(const OcPending& p0, cudaStream_t user) {
    OcPending p = p0;
    p.ready = tl_ready;
    p.done = tl_done;
    cudaEventRecord(p.ready, user);
    std::unique_lock<std::mutex> lk(mu);
    subs.push_back(&p);
    const unsigned long long g = gen;
    if ((int)subs.size() >= participants) launch_round();
    else cv.wait(lk, [&] { return gen != g; });
    lk.unlock();
    cudaStreamWaitEvent(user, p.done, 0);
    return 1;
  }
};

OcBatcher* onchip_batcher_create(int device) {
  OcBatcher* b = new OcBatcher();
  b->device = device;
  cudaSetDevice(device);
  if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return nullptr;
  }
  return b;
}

void onchip_batcher_destroy(OcBatcher* b) {
  if (!b) return;
  cudaStreamSynchronize(b->st);
  cudaStreamDestroy(b->st);
  delete b;
}

void onchip_batcher_join(OcBatcher* b, int n) {
  std::lock_guard<std::mutex> lk(b->mu);
  b->participants += n;
}

void onchip_batcher_bind(OcBatcher* b) {
  cudaEventCreateWithFlags(&tl_ready, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&tl_done, cudaEventDisableTiming);
  tl_batcher = b;
}

void onchip_batcher_release() {
  OcBatcher* b = tl_batcher;
  if (!b) return;
  {
    std::lock_guard<std::mutex> lk(b->mu);
    --b->participants;
    if (!b->subs.empty() && (int)b->subs.size() >= b->participants) b->launch_round();
  }
  cudaEventDestroy(tl_ready);
  cudaEventDestroy(tl_done);
  tl_ready = tl_done = nullptr;
  tl_batcher = nullptr;
}

void onchip_batcher_stats(const OcBatcher* b, long long* launches, long long* members) {
  OcBatcher* m = const_cast<OcBatcher*>(b);
  std::lock_guard<std::mutex> lk(m->mu);
  if (launches) *launches = m->launches;
  if (members) *members = m->members;
}

int onchip_forward(const OnchipPlan* oc, const void* tab, const double2* psi_api, const double2* img_in,
                   double2* psi_out, double2* ck_out, int K, int n0, int n1, double dt, void* segY,
                   cudaStream_t st) {
  if (tl_batcher) {
    OcPending p{};
    p.kind = 0;
    p.oc = oc;
    p.dt = dt;
    p.d.tab = tab;
    p.d.psi_api = psi_api;
    p.d.img_in = img_in;
    p.d.psi_out = psi_out;
    p.d.ck_out = ck_out;
    p.d.segY = segY;
    p.d.K = std::max(1, K);
    p.d.n0 = n0;
    p.d.n1 = n1;
    return tl_batcher->submit(p, st);
  }
  OC_DISPATCH(fwd_t, oc, tab, psi_api, img_in, psi_out, ck_out, K, n0, n1, dt, segY, st);
}

int onchip_adjoint(const OnchipPlan* oc, const OnchipTables& tb, const void* segY, double2* pbar_img, int n0,
                   int n1, double dt, const XArgs& xa, int nst, double* gF_cta, double* acc_cta, int* err,
                   void* colow, cudaStream_t st) {
  if (tl_batcher) {
    OcPending p{};
    p.kind = 1;
    p.oc = oc;
    p.dt = dt;
    p.xa = &xa;
    p.d.tab = tb.tab;
    p.d.coef = tb.coef;
    p.d.ph = tb.ph;
    p.d.opd = tb.opd;
    p.d.segY = const_cast<void*>(segY);
    p.d.pbar_img = pbar_img;
    p.d.gF_cta = gF_cta;
    p.d.acc_cta = acc_cta;
    p.d.err = err;
    p.d.pblo = colow;
    p.d.J = xa.Jdev;
    p.d.nstK = (long long)nst * std::max(1, oc->oa.K);
    p.d.n0 = n0;
    p.d.n1 = n1;
    return tl_batcher->submit(p, st);
  }
  OC_DISPATCH(adj_t, oc, tb, segY, pbar_img, n0, n1, dt, xa, nst, gF_cta, acc_cta, err, colow, st);
}

namespace {

template <typename R, int DL>
int q2_t(const OnchipPlan* oc, const Q2Args& qa, const void* rows, const void* edges, const double2* psi_in,
         double2* psi_out, int N, int rowlen, int nmat, cudaStream_t st) {
  typedef typename CT<R>::T C;
  smem_limit_once<k_oc_q2<R, DL>>();
  // coupling unitaries in shared memory when they fit, else read from global memory
  const int nedge = nmat * DL * DL * DL * DL;
  const size_t gbytes = (size_t)nedge * sizeof(C);
  const bool gsm = oc->oa.q_G + gbytes <= oc->limit;
  const size_t smem = oc->oa.q_G + (gsm ? gbytes : 0);
  k_oc_q2<R, DL><<<oc->oa.ncta, kST, smem, st>>>(oc->h->pass[0], oc->oa, qa, (const C*)rows, (const C*)edges,
                                                 psi_in, psi_out, N, rowlen, gsm ? nedge : 0);
  return 1;
}

}  // namespace

sg_status onchip_q2_forward(const OnchipPlan* oc, const KPlan& p, const void* rows, const void* edges,
                            const double2* psi_in, double2* psi_out, int N, int J, const int* set_of, int nset,
                            cudaStream_t st, int* launches, bool q1) {
  const SlabPass& sp = oc->h->pass[0];
  const int DL = oc->h->DL;
  if (p.nq > 2 * 8 || p.ne > kMaxQ2F - 8 || J < 1 || J > 3) return SG_E_UNSUPPORTED;
  if (p.nq * DL * DL > oc->oa.rowA) return SG_E_UNSUPPORTED;        // 1-body row must fit the row buffer
  Q2Args qa{};
  // 1-body factors: modes in pairs (Kronecker L (x) R), an odd last mode alone
  for (int i = 0; i < p.nq; i += 2) {
    Q2Factor& F = qa.f[qa.nf0++];
    if (i + 1 < p.nq) {
      F.P = make_phase(sp, DL, i, i + 1);
      F.P.offL = i * DL * DL;
      F.P.offR = (i + 1) * DL * DL;
      F.kind = 0;
    } else {
      F.P = make_phase(sp, DL, i, i - 1);
      F.P.offA = i * DL * DL;
      F.kind = 1;
    }
  }
  for (int e = 0; e < p.ne; ++e) {
    Q2Factor& F = qa.f[qa.nf0 + qa.nfe++];
    F.P = make_phase(sp, DL, p.e_a[e], p.e_b[e]);
    F.kind = 2;
    F.mat = 2 * e;                // per set and coupling: half, full
  }
  qa.J = J;
  qa.q1 = q1 ? 1 : 0;
  for (int j = 0; j < J; ++j) qa.setoff[j] = 2 * p.ne * set_of[j];
  const int rowlen = p.nq * DL * DL;
  const int nmat = 2 * p.ne * nset;
  int n = 0;
  if (oc->mixed) {
    switch (DL) {
      case 2: n = q2_t<float, 2>(oc, qa, rows, edges, psi_in, psi_out, N, rowlen, nmat, st); break;
      case 3: n = q2_t<float, 3>(oc, qa, rows, edges, psi_in, psi_out, N, rowlen, nmat, st); break;
      case 4: n = q2_t<float, 4>(oc, qa, rows, edges, psi_in, psi_out, N, rowlen, nmat, st); break;
      default: n = q2_t<float, 5>(oc, qa, rows, edges, psi_in, psi_out, N, rowlen, nmat, st); break;
    }
  } else {
    switch (DL) {
      case 2: n = q2_t<double, 2>(oc, qa, rows, edges, psi_in, psi_out, N, rowlen, nmat, st); break;
      case 3: n = q2_t<double, 3>(oc, qa, rows, edges, psi_in, psi_out, N, rowlen, nmat, st); break;
      case 4: n = q2_t<double, 4>(oc, qa, rows, edges, psi_in, psi_out, N, rowlen, nmat, st); break;
      default: n = q2_t<double, 5>(oc, qa, rows, edges, psi_in, psi_out, N, rowlen, nmat, st); break;
    }
  }
  if (launches) *launches += n;
  return SG_OK;
}

int onchip_dl(const OnchipPlan* oc) { return oc->h->DL; }

namespace {

template <typename R, int DL>
int q2adj_t(const OnchipPlan* oc, const Q2AdjArgs& qa, const void* rows, const void* edges, const double2* psi,
            const double2* bar, int N, int nset, double* gF_cta, long long nstK, cudaStream_t st) {
  typedef typename CT<R>::T C;
  smem_limit_once<k_oc_q2_adj<R, DL>>();
  const int nedge = 4 * qa.ne * nset * DL * DL * DL * DL;
  const bool gsm = oc->oa.b_G + (size_t)nedge * sizeof(C) <= oc->limit;
  const size_t smem = oc->oa.b_G + (gsm ? (size_t)nedge * sizeof(C) : 0);
  k_oc_q2_adj<R, DL><<<oc->oa.ncta, kST, smem, st>>>(oc->h->pass[0], oc->oa, qa, (const C*)rows, (const C*)edges,
                                                           psi, bar, N, gF_cta, nstK, gsm ? nedge : 0);
  return 1;
}

}  // namespace

sg_status onchip_q2_pulse_adjoint(const OnchipPlan* oc, const KPlan& p, const int* drv_mode, int K, const void* rows,
                                  const void* edges, const double2* psi, const double2* bar, int N, int J,
                                  const int* set_of, int nset, long long nstK, double* gF_cta, cudaStream_t st,
                                  int* launches, bool q1) {
  const SlabPass& sp = oc->h->pass[0];
  const int DL = oc->h->DL;
  if ((size_t)oc->oa.b_G > oc->limit || p.nq < 2 || p.ne > 32 || K > kQ2G || K != oc->oa.K || J < 1 || J > 3 ||
      (long long)N * std::max(1, K) > nstK)
    return SG_E_UNSUPPORTED;
  if (p.nq * DL * DL > oc->oa.rowA) return SG_E_UNSUPPORTED;
  Q2AdjArgs qa{};
  qa.nq = p.nq;
  qa.K = K;
  qa.ne = p.ne;
  qa.row = (2 * p.nq + K) * DL * DL;
  for (int i = 0; i < p.nq; i += 2) {
    Phase& P = qa.one[qa.n1f++];
    if (i + 1 < p.nq) {
      P = make_phase(sp, DL, i, i + 1);
      P.offL = i * DL * DL;
      P.offR = (i + 1) * DL * DL;
    } else {
      P = make_phase(sp, DL, i, i - 1);
      P.offA = i * DL * DL;
    }
  }
  for (int i = 0; i < p.nq; ++i) qa.mode[i] = make_phase(sp, DL, i, i == 0 ? 1 : 0);
  for (int e = 0; e < p.ne; ++e) qa.edge[e] = make_phase(sp, DL, p.e_a[e], p.e_b[e]);
  for (int k = 0; k < K; ++k) {
    qa.drv_mode[k] = drv_mode[k];
    qa.driven |= 1u << drv_mode[k];
  }
  qa.J = J;
  qa.q1 = q1 ? 1 : 0;
  for (int j = 0; j < J; ++j) qa.setoff[j] = 4 * p.ne * set_of[j];      // per set and coupling: inverse and adjoint pairs
  int n = 0;
  if (oc->mixed) {
    switch (DL) {
      case 2: n = q2adj_t<float, 2>(oc, qa, rows, edges, psi, bar, N, nset, gF_cta, nstK, st); break;
      case 3: n = q2adj_t<float, 3>(oc, qa, rows, edges, psi, bar, N, nset, gF_cta, nstK, st); break;
      case 4: n = q2adj_t<float, 4>(oc, qa, rows, edges, psi, bar, N, nset, gF_cta, nstK, st); break;
      default: n = q2adj_t<float, 5>(oc, qa, rows, edges, psi, bar, N, nset, gF_cta, nstK, st); break;
    }
  } else {
    switch (DL) {
      case 2: n = q2adj_t<double, 2>(oc, qa, rows, edges, psi, bar, N, nset, gF_cta, nstK, st); break;
      case 3: n = q2adj_t<double, 3>(oc, qa, rows, edges, psi, bar, N, nset, gF_cta, nstK, st); break;
      case 4: n = q2adj_t<double, 4>(oc, qa, rows, edges, psi, bar, N, nset, gF_cta, nstK, st); break;
      default: n = q2adj_t<double, 5>(oc, qa, rows, edges, psi, bar, N, nset, gF_cta, nstK, st); break;
    }
  }
  if (launches) *launches += n;
  return SG_OK;
}

void onchip_to_image(const OnchipPlan* oc, const double2* api, double2* img, cudaStream_t st) {
  k_oc_image<<<grid_of(onchip_state_elems(oc)), 256, 0, st>>>(oc->oa, api, img);
}

void onchip_to_f32(const double* src, float* dst, long long n, cudaStream_t st) {
  k_oc_f32<<<grid_of(n), 256, 0, st>>>(src, dst, n);
}

void onchip_reduce(const OnchipPlan* oc, const double* gF_cta, const double* acc_cta, long long nst, int K,
                   int n1, int ne, GradAcc acc, cudaStream_t st) {
  RedArgs r{};
  r.nstK = nst * std::max(1, K);
  r.accd = acc_cta ? oc->oa.accd : 0;   // no per-CTA accumulator blocks: dF/df only
  r.ncta = oc->oa.ncta;
  r.K = K;
  r.n1 = n1;
  r.ne = ne;
  r.acc = acc;
  k_oc_reduce<<<grid_of(r.nstK + r.accd), 256, 0, st>>>(r, gF_cta, acc_cta);
}
