// Gradient accumulators and the per-stage contraction of cross-densities into
// co-gradients (shared by the gather and the tiled evolution kernels).
//
// For a stage with Hamiltonian terms X(t) (B_i, L_e, R_e) and co-state kbar, the
// cross-density of a term slot is C_ab = <kbar, (|a><b| on the slot's mode, the
// other factor of the term applied) y> summed over the slab, and W = -i C gives
// dF = Re sum_ab W_ab dX_ab (Sec. 2.5: the gradient term a_i^T dU_i/dtheta psi_{i-1}).
#pragma once
#include "kplan.h"

struct GradAcc {
  double* gF;          // 3N x K: dF/df_k at each stage slot
  double2* obD;        // K x MAXD^2: co-gradient of drive k's base operator
  double2* obL;        // ne x MAXD^2
  double2* obR;        // ne x MAXD^2
  double* ebB;         // n1 x MAXD
  double* ebL;         // ne x MAXD
  double* ebR;         // ne x MAXD
  double* jb;          // ne
};

struct XArgs {
  KPlan p;
  int K, nW, frame;
  int ham;             // 0: the caller wants no Hamiltonian-parameter gradient, so the
                       // coupling-term slots (slot >= p.n1) are skipped
  double t;            // stage time
  int q;               // stage slot 3n + j
  const double2* tabrow;      // FP64 row of this stage
  const double* coef;         // K values at this stage
  const double2* ph;          // sumd phases at this stage
  const double2* opd;         // flat truncated operators
  int opd_off[SG_MAXQ];
  int eoff[SG_MAXQ];
  const double* E;
  int drv_of_slot_start[SG_MAXQ + 1];
  int drv_list[SG_MAXDRIVE];
  int drv_op[SG_MAXDRIVE];
  int e_opa[SG_MAXEDGE], e_opb[SG_MAXEDGE];
  double J[SG_MAXEDGE];
  const double* Jdev;         // device copy of J (read by batched on-chip launches)
  double2* partial;           // gridDim x nW x DL^2
  unsigned* ticket;
  GradAcc acc;
};


// Contract one slot's W (d x d, leading dimension DL) into the accumulators.
// Called by exactly one thread per slot, in stage order, so the updates are
// race-free and the sums have a fixed order.
__device__ __forceinline__ void contract_slot(const XArgs& a, int slot, const double2* W, int DL) {
  const KPlan& p = a.p;
  const double t = a.t;
  const bool inter = a.frame == SG_FRAME_INTERACTION;
  if (slot < p.n1) {
    const int u = slot, i = p.s1_mode[u], d = p.dims[i];
    const double2* B = a.tabrow + p.s1_off[u];
    for (int x = a.drv_of_slot_start[u]; x < a.drv_of_slot_start[u + 1]; ++x) {
      const int k = a.drv_list[x];
      const double2* O = a.opd + a.opd_off[i] + a.drv_op[k] * d * d;
      const double fk = a.coef[k];
      double g = 0.0;
      for (int ia = 0; ia < d; ++ia)
        for (int ib = 0; ib < d; ++ib) {
          double2 P = cmul(a.ph[a.eoff[i] + ia], cconj(a.ph[a.eoff[i] + ib]));
          double2 w = W[ia * DL + ib];
          double2 Ot = cmul(O[ia * d + ib], P);
          g += w.x * Ot.x - w.y * Ot.y;
          double2 cw = cmul(cconj(w), cconj(P));
          double2* ob = a.acc.obD + (size_t)k * SG_MAXD * SG_MAXD + ia * SG_MAXD + ib;
          ob->x += fk * cw.x;
          ob->y += fk * cw.y;
        }
      a.acc.gF[(size_t)a.q * a.K + k] += g;
    }
    double* eb = a.acc.ebB + u * SG_MAXD;
    for (int ia = 0; ia < d; ++ia)
      for (int ib = 0; ib < d; ++ib) {
        double2 w = W[ia * DL + ib];
        if (inter) {
          double2 v = cmul(w, B[ia * d + ib]);
          double qv = -v.y * t;                            // Re(v * i t)
          eb[ia] += qv;
          eb[ib] -= qv;
        } else if (ia == ib) {
          eb[ia] += w.x;
        }
      }
    return;
  }
  const int side = (slot - p.n1) / p.ne, q = (slot - p.n1) % p.ne;
  const int i = side == 0 ? p.e_a[q] : p.e_b[q];
  const int op = side == 0 ? a.e_opa[q] : a.e_opb[q];
  const int d = p.dims[i];
  const double2* O = a.opd + a.opd_off[i] + op * d * d;
  const double2* X2 = a.tabrow + (side == 0 ? p.e_offL[q] : p.e_offR[q]);
  double2* ob = (side == 0 ? a.acc.obL : a.acc.obR) + (size_t)q * SG_MAXD * SG_MAXD;
  double* eb = (side == 0 ? a.acc.ebL : a.acc.ebR) + q * SG_MAXD;
  const double sc = side == 0 ? a.J[q] : 1.0;
  double jg = 0.0;
  for (int ia = 0; ia < d; ++ia)
    for (int ib = 0; ib < d; ++ib) {
      double2 P = cmul(a.ph[a.eoff[i] + ia], cconj(a.ph[a.eoff[i] + ib]));
      double2 w = W[ia * DL + ib];
      double2 At = cmul(O[ia * d + ib], P);
      jg += w.x * At.x - w.y * At.y;
      double2 cw = cmul(cconj(w), cconj(P));
      ob[ia * SG_MAXD + ib].x += sc * cw.x;
      ob[ia * SG_MAXD + ib].y += sc * cw.y;
      if (inter) {
        double2 v = cmul(w, X2[ia * d + ib]);
        double qv = -v.y * t;
        eb[ia] += qv;
        eb[ib] -= qv;
      }
    }
  if (side == 0) a.acc.jb[q] += jg;
}
