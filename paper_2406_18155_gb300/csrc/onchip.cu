// On-chip evolution kernels (see onchip.h).
//
// Shared-memory images: column c of a CTA's group starts at c * CS (CS = padded
// column stride, even, so every column and image is 16-byte aligned) and entry t of
// a column sits at spos(t), the bank-conflict-free padding of the tiled kernels.
// The register-blocked phases of the tiled kernels (slab_dev.cuh) apply H; their
// block index runs over all Sc columns.
//
// Adjoint stage (reverse order 3, 2, 1, 0 of one RK4 step), everything in shared
// memory:  ks = H kbar_s (phases) -> epilogue: ybar = i ks, Db, pbar, next kbar (in
// place in ks) -> cross-densities of this stage's term slots between kbar_s and the
// stored stage input y_s, one warp per slot, reduced across the warp and contracted
// by the warp's lanes (one lane per level pair) into shared-memory accumulators.
// The stage input of the next stage arrives by a bulk copy (cp.async.bulk, completion
// on an mbarrier) and the next table rows by cp.async while this stage computes.
#include "sg_internal.h"
#include "kplan.h"
#include "grad.cuh"
#include "slab.h"
#include "slab_dev.cuh"
#include "onchip.h"
#include <algorithm>
#include <cstdint>

namespace {

// ---------------------------------------------------------------------------
// asynchronous copies
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// cp.async of 8 or 16 bytes global -> shared (no registers, completes at cp_wait_all)
__device__ __forceinline__ void cp8(void* s, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp16(void* s, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
template <typename C> __device__ __forceinline__ void cpc(C* s, const C* g);
template <> __device__ __forceinline__ void cpc<float2>(float2* s, const float2* g) { cp8(s, g); }
template <> __device__ __forceinline__ void cpc<double2>(double2* s, const double2* g) { cp16(s, g); }
__device__ __forceinline__ void cpd(double* s, const double* g) { cp8(s, g); }

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
// Bounded wait for the phase `parity` of mb: gives up after about a second,
// records the failure in *err and lets the kernel run to its end without waiting
// again (once *err is set every later wait returns at once).
__device__ __forceinline__ void mb_wait(uint64_t* mb, unsigned parity, int* err) {
  if (*(volatile int*)err) return;
  for (int it = 0; it < (1 << 22); ++it) {
    if (mb_try(mb, parity)) return;
    __nanosleep(64);
  }
  atomicExch(err, 1);
}

// ---------------------------------------------------------------------------
// plan arguments
// ---------------------------------------------------------------------------
struct OcArgs {
  int D, S, Sc, nbc, nbt, CS, CSP, ncta, row, K, sumd, n1, ne;
  int ent;               // Sc * D entries per CTA
  // forward shared-memory byte offsets
  int f_ys, f_ks, f_ps, f_dl, f_M;
  // adjoint shared-memory byte offsets
  int a_xs, a_ks, a_ys, a_yn, a_db, a_pb, a_M, a_T, a_cf, a_ph, a_obD, a_obL, a_obR, a_ebB, a_ebL, a_ebR,
      a_jb, a_gs, a_sq;
  int rowA, Kp;          // row and K rounded up to even counts
  long long accd;        // doubles per CTA accumulator block (global layout)
};

template <int DL>
__device__ __forceinline__ int oc_pos(const OcArgs& oa, int e, int& c, int& t) {
  c = e / oa.D;
  t = e - c * oa.D;
  return c * oa.CS + spos<DL>(t);
}

// All phases of the single pass over the CTA's Sc columns: ks = H ys.  Ends with a barrier.
template <int DL, typename C>
__device__ __forceinline__ void oc_apply(const SlabPass& sp, const OcArgs& oa, const C* __restrict__ M,
                                         const C* __restrict__ ys, C* __restrict__ ks) {
  for (int q = 0; q < sp.nph; ++q) {
    const Phase& P = sp.ph[q];
    for (int b = threadIdx.x; b < oa.nbt; b += blockDim.x) {
      const int c = b / oa.nbc;
      const int pb = blk_pos<DL>(P, b - c * oa.nbc) + c * oa.CS;
      if (P.allpar) phase_block<DL, true>(P, M, ys, ks, pb, q == 0);
      else phase_block<DL, false>(P, M, ys, ks, pb, q == 0);
    }
    __syncthreads();
  }
}

template <typename C>
__device__ __forceinline__ void issue_row(const C* __restrict__ tab, int row, int q, C* dst) {
  const C* src = tab + (size_t)q * row;
  for (int i = threadIdx.x; i < row; i += blockDim.x) cpc<C>(dst + i, src + i);
}

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------
template <typename R, int DL>
__global__ void __launch_bounds__(kST, 1)
k_oc_fwd(SlabPass sp, OcArgs oa, const typename CT<R>::T* __restrict__ tab, const double2* __restrict__ psi_api,
         const double2* __restrict__ img_in, double2* __restrict__ psi_out, double2* __restrict__ ck_out, int K,
         int n0, int n1, double dt, typename CT<R>::T* __restrict__ segY) {
  typedef typename CT<R>::T C;
  extern __shared__ __align__(16) unsigned char sm[];
  C* ys = reinterpret_cast<C*>(sm + oa.f_ys);
  C* ks = reinterpret_cast<C*>(sm + oa.f_ks);
  double2* ps = reinterpret_cast<double2*>(sm + oa.f_ps);
  C* dl = reinterpret_cast<C*>(sm + oa.f_dl);
  C* Mb[2] = {reinterpret_cast<C*>(sm + oa.f_M), reinterpret_cast<C*>(sm + oa.f_M) + oa.rowA};
  const int cta = blockIdx.x;
  const R h = (R)dt;
  for (int e = threadIdx.x; e < oa.ent; e += blockDim.x) {
    int c, t;
    const int pos = oc_pos<DL>(oa, e, c, t);
    const int col = cta * oa.Sc + c;
    double2 v = make_double2(0.0, 0.0);
    if (img_in) v = img_in[(size_t)cta * oa.ent + e];
    else if (col < oa.S) v = psi_api[(size_t)t * oa.S + col];
    ps[e] = v;
    ys[pos] = to_c(v, R(0));
  }
  if (n0 < n1) issue_row<C>(tab, oa.row, 3 * n0, Mb[0]);
  cp_wait_all();
  __syncthreads();
  int buf = 0;
  for (int step = n0; step < n1; ++step) {
    if (ck_out && (step - n0) % K == 0) {
      double2* ck = ck_out + ((size_t)((step - n0) / K) * oa.ncta + cta) * oa.ent;
      for (int e = threadIdx.x; e < oa.ent; e += blockDim.x) ck[e] = ps[e];
    }
#pragma unroll 1
    for (int s = 0; s < 4; ++s) {
      // next stage's table row
      const int nstep = s < 3 ? step : step + 1, ns = s < 3 ? s + 1 : 0;
      if (nstep < n1) issue_row<C>(tab, oa.row, 3 * nstep + (ns == 0 ? 0 : (ns == 3 ? 2 : 1)), Mb[buf ^ 1]);
      if (segY) {
        C* g = segY + ((size_t)(4 * (step - n0) + s) * oa.ncta + cta) * oa.CSP;
        for (int e = threadIdx.x; e < oa.ent; e += blockDim.x) {
          int c, t;
          const int pos = oc_pos<DL>(oa, e, c, t);
          g[pos] = ys[pos];
        }
      }
      oc_apply<DL>(sp, oa, Mb[buf], ys, ks);
      for (int e = threadIdx.x; e < oa.ent; e += blockDim.x) {
        int c, t;
        const int pos = oc_pos<DL>(oa, e, c, t);
        const C a = ks[pos];
        const C kk = cmk<C>(a.y, -a.x);                 // -i H y
        const double2 p = ps[e];
        const C pr = to_c(p, R(0));
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
          const R incx = d.x + h / 6 * kk.x, incy = d.y + h / 6 * kk.y;
          const double2 pn = make_double2(p.x + (double)incx, p.y + (double)incy);
          ps[e] = pn;
          ys[pos] = to_c(pn, R(0));
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
      if (col < oa.S) psi_out[(size_t)t * oa.S + col] = ps[e];
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
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Shared-memory accumulators of one CTA (level-pair stride DL * DL, level stride DL).
struct OcAcc {
  double2 *obD, *obL, *obR;
  double *ebB, *ebL, *ebR, *jb, *gs;
};

// Energy co-gradient of one slot from the lanes' qv(a, b) = -Im(W_ab X_ab) t:
// eb[a] += sum_b qv(a, b) - sum_b qv(b, a).
template <int DL>
__device__ __forceinline__ void eb_rowcol(double qv, int lane, double* sq, double* eb) {
  sq[lane] = qv;
  __syncwarp();
  if (lane < DL) {
    double s = 0.0;
#pragma unroll
    for (int b = 0; b < DL; ++b) s += sq[lane * DL + b] - sq[b * DL + lane];
    eb[lane] += s;
  }
  __syncwarp();
}

// Contraction of one slot's W (lane = level pair a * DL + b, lanes >= DL^2 hold 0)
// into the co-gradients: the same sums as contract_slot, spread over the warp.
//   1-body slot, drive k:  gF[q][k] += Re sum W O_k(t),  obD[k] += f_k conj(W P)
//   edge side:             jb += Re sum W A(t) (side a),  obL/obR += J conj(W P) / conj(W P)
//   interaction frame:     eb[a] += sum_b qv(a, b) - qv(b, a),  qv = -Im(W_ab X_ab(t)) t
//   lab frame, 1-body:     eb[a] += Re W_aa
template <int DL>
__device__ __forceinline__ void oc_contract(const XArgs& xa, int slot, double2 w, int lane, const double2* tabrow,
                                            const double* cf, const double2* phs, double t, int q, int s,
                                            const OcAcc& A, double* sq, double* gFc) {
  const KPlan& p = xa.p;
  const bool inter = xa.frame == SG_FRAME_INTERACTION;
  const bool on = lane < DL * DL;
  const int ia = on ? lane / DL : 0, ib = on ? lane - ia * DL : 0;
  if (slot < p.n1) {
    const int u = slot, i = p.s1_mode[u];
    const double2 P = on ? cmul(phs[xa.eoff[i] + ia], cconj(phs[xa.eoff[i] + ib])) : make_double2(0.0, 0.0);
    for (int x = xa.drv_of_slot_start[u]; x < xa.drv_of_slot_start[u + 1]; ++x) {
      const int k = xa.drv_list[x];
      double g = 0.0;
      if (on) {
        const double2 O = __ldg(xa.opd + xa.opd_off[i] + xa.drv_op[k] * DL * DL + lane);
        const double2 Ot = cmul(O, P);
        g = w.x * Ot.x - w.y * Ot.y;
        const double2 cw = cmul(cconj(w), cconj(P));
        const double fk = cf[k];
        double2& ob = A.obD[k * DL * DL + lane];
        ob.x += fk * cw.x;
        ob.y += fk * cw.y;
      }
      g = warp_sum(g);
      if (lane == 0) {
        // stages 2 and 1 share the slot q = 3n + 1: hold stage 2's share, store once
        if (s == 2) A.gs[k] = g;
        else gFc[(size_t)q * xa.K + k] = s == 1 ? A.gs[k] + g : g;
      }
    }
    double* eb = A.ebB + u * DL;
    if (inter) {
      double qv = 0.0;
      if (on) {
        const double2 v = cmul(w, tabrow[p.s1_off[u] + lane]);
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
  const double sc = side == 0 ? xa.J[qe] : 1.0;
  double jg = 0.0;
  if (on) {
    const double2 P = cmul(phs[xa.eoff[i] + ia], cconj(phs[xa.eoff[i] + ib]));
    const double2 O = __ldg(xa.opd + xa.opd_off[i] + op * DL * DL + lane);
    const double2 At = cmul(O, P);
    jg = w.x * At.x - w.y * At.y;
    const double2 cw = cmul(cconj(w), cconj(P));
    double2& ob = (side == 0 ? A.obL : A.obR)[qe * DL * DL + lane];
    ob.x += sc * cw.x;
    ob.y += sc * cw.y;
  }
  if (inter) {
    double qv = 0.0;
    if (on) {
      const double2 v = cmul(w, tabrow[(side == 0 ? p.e_offL[qe] : p.e_offR[qe]) + lane]);
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
k_oc_adj(SlabPass sp, OcArgs oa, const typename CT<R>::T* __restrict__ tab, const double2* __restrict__ tab64,
         const double* __restrict__ coef, const double2* __restrict__ ph,
         const typename CT<R>::T* __restrict__ segY, double2* __restrict__ pbar_img, int n0, int n1, double dt,
         XArgs xa, double* __restrict__ gF_cta, double* __restrict__ acc_cta, long long nstK,
         int* __restrict__ err) {
  typedef typename CT<R>::T C;
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  C* xs = reinterpret_cast<C*>(sm + oa.a_xs);
  C* ks = reinterpret_cast<C*>(sm + oa.a_ks);
  C* ys = reinterpret_cast<C*>(sm + oa.a_ys);
  C* yn = reinterpret_cast<C*>(sm + oa.a_yn);
  C* db = reinterpret_cast<C*>(sm + oa.a_db);
  double2* pb = reinterpret_cast<double2*>(sm + oa.a_pb);
  C* Mb[2] = {reinterpret_cast<C*>(sm + oa.a_M), reinterpret_cast<C*>(sm + oa.a_M) + oa.rowA};
  double2* Tb[2] = {reinterpret_cast<double2*>(sm + oa.a_T), reinterpret_cast<double2*>(sm + oa.a_T) + oa.row};
  double* cf[2] = {reinterpret_cast<double*>(sm + oa.a_cf), reinterpret_cast<double*>(sm + oa.a_cf) + oa.Kp};
  double2* phb[2] = {reinterpret_cast<double2*>(sm + oa.a_ph), reinterpret_cast<double2*>(sm + oa.a_ph) + oa.sumd};
  OcAcc A;
  A.obD = reinterpret_cast<double2*>(sm + oa.a_obD);
  A.obL = reinterpret_cast<double2*>(sm + oa.a_obL);
  A.obR = reinterpret_cast<double2*>(sm + oa.a_obR);
  A.ebB = reinterpret_cast<double*>(sm + oa.a_ebB);
  A.ebL = reinterpret_cast<double*>(sm + oa.a_ebL);
  A.ebR = reinterpret_cast<double*>(sm + oa.a_ebR);
  A.jb = reinterpret_cast<double*>(sm + oa.a_jb);
  A.gs = reinterpret_cast<double*>(sm + oa.a_gs);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* sq = reinterpret_cast<double*>(sm + oa.a_sq) + warp * 32;
  const int cta = blockIdx.x;
  const R h = (R)dt;
  const int DD = DL * DL;
  for (int i = threadIdx.x; i < oa.K * DD; i += blockDim.x) A.obD[i] = make_double2(0.0, 0.0);
  for (int i = threadIdx.x; i < oa.ne * DD; i += blockDim.x) A.obL[i] = A.obR[i] = make_double2(0.0, 0.0);
  for (int i = threadIdx.x; i < oa.n1 * DL; i += blockDim.x) A.ebB[i] = 0.0;
  for (int i = threadIdx.x; i < oa.ne * DL; i += blockDim.x) A.ebL[i] = A.ebR[i] = 0.0;
  for (int i = threadIdx.x; i < oa.ne; i += blockDim.x) A.jb[i] = 0.0;
  for (int i = threadIdx.x; i < oa.K; i += blockDim.x) A.gs[i] = 0.0;
  if (threadIdx.x == 0) mb_init(&mbar);
  // co-state, and kbar_4 = dt/6 pbar of the segment's last step
  for (int e = threadIdx.x; e < oa.ent; e += blockDim.x) {
    int c, t;
    const int pos = oc_pos<DL>(oa, e, c, t);
    const double2 v = pbar_img[(size_t)cta * oa.ent + e];
    pb[e] = v;
    const C qv = to_c(v, R(0));
    xs[pos] = cmk<C>(h / 6 * qv.x, h / 6 * qv.y);
  }
  __syncthreads();
  const unsigned img_bytes = (unsigned)(oa.CSP * sizeof(C));
  double* gFc = gF_cta + (size_t)cta * nstK;
  // prefetch of stage s of step n into (ydst, buffer b)
  auto issue = [&](int n, int s, C* ydst, int b) {
    if (threadIdx.x == 0)
      bulk_load(ydst, segY + ((size_t)(4 * (n - n0) + s) * oa.ncta + cta) * oa.CSP, img_bytes, &mbar);
    const int q = 3 * n + (s == 0 ? 0 : (s == 3 ? 2 : 1));
    issue_row<C>(tab, oa.row, q, Mb[b]);
    issue_row<double2>(tab64, oa.row, q, Tb[b]);
    for (int i = threadIdx.x; i < oa.K; i += blockDim.x) cpd(cf[b] + i, coef + (size_t)q * oa.K + i);
    for (int i = threadIdx.x; i < oa.sumd; i += blockDim.x) cpc<double2>(phb[b] + i, ph + (size_t)q * oa.sumd + i);
  };
  unsigned parity = 0;
  if (n0 < n1) {
    issue(n1 - 1, 3, ys, 0);
    cp_wait_all();
    mb_wait(&mbar, parity, err);
    parity ^= 1;
  }
  __syncthreads();
  int buf = 0;
  constexpr int NA = xd_n<DL, PARX>();
  for (int step = n1 - 1; step >= n0; --step) {
#pragma unroll 1
    for (int s = 3; s >= 0; --s) {
      const int j = s == 0 ? 0 : (s == 3 ? 2 : 1);
      const int q = 3 * step + j;
      const double tq = (double)(2 * step + j) * dt * 0.5;
      const int pn = s > 0 ? step : step - 1, psn = s > 0 ? s - 1 : 3;
      const bool more = pn >= n0;
      if (more) issue(pn, psn, yn, buf ^ 1);
      oc_apply<DL>(sp, oa, Mb[buf], xs, ks);
      // epilogue: ybar = i H kbar; next kbar written over ks
      for (int e = threadIdx.x; e < oa.ent; e += blockDim.x) {
        int c, t;
        const int pos = oc_pos<DL>(oa, e, c, t);
        const C a = ks[pos];
        const C y = cmk<C>(-a.y, a.x);
        const double2 pv = pb[e];
        const C pr = to_c(pv, R(0));
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
          const double2 pnv = make_double2(pv.x + (double)(d.x + y.x), pv.y + (double)(d.y + y.y));
          pb[e] = pnv;
          const C qq = to_c(pnv, R(0));
          ks[pos] = cmk<C>(h / 6 * qq.x, h / 6 * qq.y);
        }
      }
      // cross-densities of this stage (kbar_s in xs, y_s in ys), one warp per slot
#pragma unroll 1
      for (int sl = 0; sl < kSPW; ++sl) {
        const int slot = warp + sl * (kST / 32);
        if (slot >= sp.nx) continue;                // warp-uniform
        const Phase& P = sp.ph[sp.x_ph[slot]];
        const int type = sp.x_type[slot];
        C acc[NA];
#pragma unroll
        for (int a = 0; a < NA; ++a) acc[a] = cmk<C>(0.0, 0.0);
        for (int b = lane; b < oa.nbt; b += 32) {
          const int c = b / oa.nbc;
          xd_slot<DL, PARX>(P, type, Mb[buf], xs, ys, blk_pos<DL>(P, b - c * oa.nbc) + c * oa.CS, acc);
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
        const double2 w = make_double2((double)mine.y, -(double)mine.x);   // W = -i C
        oc_contract<DL>(xa, sp.x_gslot[slot], w, lane, Tb[buf], cf[buf], phb[buf], tq, q, s, A, sq, gFc);
      }
      if (more) {
        cp_wait_all();
        mb_wait(&mbar, parity, err);
        parity ^= 1;
      }
      __syncthreads();
      C* tswap = xs; xs = ks; ks = tswap;
      tswap = ys; ys = yn; yn = tswap;
      buf ^= 1;
    }
  }
  for (int e = threadIdx.x; e < oa.ent; e += blockDim.x) pbar_img[(size_t)cta * oa.ent + e] = pb[e];
  // add the CTA's accumulators to its global block (GradAcc layout, SG_MAXD strides)
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
    g[0] += A.obD[i].x;
    g[1] += A.obD[i].y;
  }
  for (int i = threadIdx.x; i < oa.ne * DD; i += blockDim.x) {
    const int k = i / DD, ab = i - k * DD, a = ab / DL, b = ab - a * DL;
    double* g = gL + 2 * ((size_t)k * MD2 + a * SG_MAXD + b);
    g[0] += A.obL[i].x;
    g[1] += A.obL[i].y;
    g = gR + 2 * ((size_t)k * MD2 + a * SG_MAXD + b);
    g[0] += A.obR[i].x;
    g[1] += A.obR[i].y;
  }
  for (int i = threadIdx.x; i < oa.n1 * DL; i += blockDim.x) geB[(i / DL) * SG_MAXD + i % DL] += A.ebB[i];
  for (int i = threadIdx.x; i < oa.ne * DL; i += blockDim.x) {
    geL[(i / DL) * SG_MAXD + i % DL] += A.ebL[i];
    geR[(i / DL) * SG_MAXD + i % DL] += A.ebR[i];
  }
  for (int i = threadIdx.x; i < oa.ne; i += blockDim.x) gjb[i] += A.jb[i];
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
  bool mixed = false, adj_ok = false;
  size_t sm_fwd = 0, sm_adj = 0;
};

namespace {

size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

// Shared-memory layout for Sc columns per CTA; returns the forward and adjoint bytes.
void layout(OcArgs& a, int DL, size_t cs, size_t& fwd, size_t& adj) {
  const bool pw2 = DL == 2 || DL == 4;
  a.CS = pw2 ? spad(a.D) : a.D;
  a.CS += a.CS & 1;
  a.CSP = a.Sc * a.CS;
  a.ent = a.Sc * a.D;
  a.nbt = a.Sc * a.nbc;
  a.rowA = a.row + (a.row & 1);
  a.Kp = std::max(2, a.K + (a.K & 1));
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o = al16(o + bytes); return (int)r; };
  a.f_ys = take(a.CSP * cs);
  a.f_ks = take(a.CSP * cs);
  a.f_ps = take((size_t)a.ent * 16);
  a.f_dl = take((size_t)a.ent * cs);
  a.f_M = take(2 * (size_t)a.rowA * cs);
  fwd = o;
  o = 0;
  a.a_xs = take(a.CSP * cs);
  a.a_ks = take(a.CSP * cs);
  a.a_ys = take(a.CSP * cs);
  a.a_yn = take(a.CSP * cs);
  a.a_db = take((size_t)a.ent * cs);
  a.a_pb = take((size_t)a.ent * 16);
  a.a_M = take(2 * (size_t)a.rowA * cs);
  a.a_T = take(2 * (size_t)a.row * 16);
  a.a_cf = take(2 * (size_t)a.Kp * 8);
  a.a_ph = take(2 * (size_t)a.sumd * 16);
  const int DD = DL * DL;
  a.a_obD = take((size_t)std::max(1, a.K) * DD * 16);
  a.a_obL = take((size_t)std::max(1, a.ne) * DD * 16);
  a.a_obR = take((size_t)std::max(1, a.ne) * DD * 16);
  a.a_ebB = take((size_t)std::max(1, a.n1) * DL * 8);
  a.a_ebL = take((size_t)std::max(1, a.ne) * DL * 8);
  a.a_ebR = take((size_t)std::max(1, a.ne) * DL * 8);
  a.a_jb = take((size_t)std::max(1, a.ne) * 8);
  a.a_gs = take((size_t)std::max(1, a.K) * 8);
  a.a_sq = take((size_t)(kST / 32) * 32 * 8);
  adj = o;
}

}  // namespace

OnchipPlan* onchip_plan_create(const KPlan& p, bool mixed, int K, int sumd, cudaStream_t st) {
  if (p.nq < 2 || p.nq > SG_MAXQ) return nullptr;
  SlabPlanHost* h = slab_plan_create(p, mixed, st);
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
  // columns per CTA: enough blocks to give every thread one per phase, within shared memory
  int sc0 = std::max(1, std::min(p.S, std::max(1, kST / std::max(1, a.nbc))));
  size_t fwd = 0, adj = 0;
  int best_adj = 0, best_fwd = 0;
  for (int sc = sc0; sc >= 1; --sc) {
    a.Sc = sc;
    layout(a, DL, cs, fwd, adj);
    if (!best_fwd && fwd <= limit) best_fwd = sc;
    if (!best_adj && adj <= limit) { best_adj = sc; break; }
  }
  const int sc = best_adj ? best_adj : best_fwd;
  if (!sc) { onchip_plan_destroy(oc); return nullptr; }
  // balance the columns over the CTAs
  a.ncta = (p.S + sc - 1) / sc;
  a.Sc = (p.S + a.ncta - 1) / a.ncta;
  layout(a, DL, cs, fwd, adj);
  oc->adj_ok = adj <= limit;
  oc->sm_fwd = fwd;
  oc->sm_adj = adj;
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
long long onchip_state_elems(const OnchipPlan* oc) { return (long long)oc->oa.ncta * oc->oa.ent; }
long long onchip_stage_elems(const OnchipPlan* oc) { return (long long)oc->oa.ncta * oc->oa.CSP; }
int onchip_ctas(const OnchipPlan* oc) { return oc->oa.ncta; }
long long onchip_acc_doubles(const OnchipPlan* oc) { return oc->oa.accd; }

namespace {

template <typename R, int DL>
int fwd_t(const OnchipPlan* oc, const void* tab, const double2* psi_api, const double2* img_in, double2* psi_out,
          double2* ck_out, int K, int n0, int n1, double dt, void* segY, cudaStream_t st) {
  typedef typename CT<R>::T C;
  auto kern = k_oc_fwd<R, DL>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oc->sm_fwd);
  kern<<<oc->oa.ncta, kST, oc->sm_fwd, st>>>(oc->h->pass[0], oc->oa, (const C*)tab, psi_api, img_in, psi_out,
                                             ck_out, std::max(1, K), n0, n1, dt, (C*)segY);
  return 1;
}

template <typename R, int DL>
int adj_t(const OnchipPlan* oc, const void* tab, const double2* tab64, const double* coef, const double2* ph,
          const void* segY, double2* pbar_img, int n0, int n1, double dt, const XArgs& xa, int nst, double* gF_cta,
          double* acc_cta, int* err, cudaStream_t st) {
  typedef typename CT<R>::T C;
  auto kern = oc->h->allpar ? k_oc_adj<R, DL, true> : k_oc_adj<R, DL, false>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oc->sm_adj);
  kern<<<oc->oa.ncta, kST, oc->sm_adj, st>>>(oc->h->pass[0], oc->oa, (const C*)tab, tab64, coef, ph,
                                             (const C*)segY, pbar_img, n0, n1, dt, xa, gF_cta, acc_cta,
                                             (long long)nst * std::max(1, oc->oa.K), err);
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

int onchip_forward(const OnchipPlan* oc, const void* tab, const double2* psi_api, const double2* img_in,
                   double2* psi_out, double2* ck_out, int K, int n0, int n1, double dt, void* segY,
                   cudaStream_t st) {
  OC_DISPATCH(fwd_t, oc, tab, psi_api, img_in, psi_out, ck_out, K, n0, n1, dt, segY, st);
}

int onchip_adjoint(const OnchipPlan* oc, const void* tab, const double2* tab64, const double* coef,
                   const double2* ph, const void* segY, double2* pbar_img, int n0, int n1, double dt,
                   const XArgs& xa, int nst, double* gF_cta, double* acc_cta, int* err, cudaStream_t st) {
  OC_DISPATCH(adj_t, oc, tab, tab64, coef, ph, segY, pbar_img, n0, n1, dt, xa, nst, gF_cta, acc_cta, err, st);
}

void onchip_to_image(const OnchipPlan* oc, const double2* api, double2* img, cudaStream_t st) {
  k_oc_image<<<grid_of(onchip_state_elems(oc)), 256, 0, st>>>(oc->oa, api, img);
}

void onchip_reduce(const OnchipPlan* oc, const double* gF_cta, const double* acc_cta, long long nst, int K,
                   int n1, int ne, GradAcc acc, cudaStream_t st) {
  RedArgs r{};
  r.nstK = nst * std::max(1, K);
  r.accd = oc->oa.accd;
  r.ncta = oc->oa.ncta;
  r.K = K;
  r.n1 = n1;
  r.ne = ne;
  r.acc = acc;
  k_oc_reduce<<<grid_of(r.nstK + r.accd), 256, 0, st>>>(r, gF_cta, acc_cta);
}
