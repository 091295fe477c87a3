// On-chip evolution for systems whose columns fit in one CTA's shared memory.
//
// One CTA owns a group of Sc state columns for the whole run: the state, the RK4
// stage input and increment (forward) or the co-state, kbar and the stage inputs
// (adjoint) stay in shared memory across steps, so a full forward evolution is one
// launch and an adjoint checkpoint segment is two (recompute, then pull back).
// Columns never exchange data during the evolution (Eq. 1's H(t) acts on each
// column separately), so CTAs need no grid synchronisation; the cross-densities of
// the gradient (Sec. 2.5) are contracted per CTA and stage into per-CTA
// accumulators that one reduction sums in a fixed order.
#pragma once
#include "grad.cuh"

struct OnchipPlan;   // opaque

// nullptr unless the plan is a single tile (one pass of the tiled kernels), every
// mode has the same level count (2..5) and at least one column fits in shared memory
// for the Q2 kernel (onchip_forward_ok / onchip_adjoint_ok tell whether the RK4
// kernels fit too).  K drives and sumd = sum of level counts size the adjoint's
// per-stage buffers.
OnchipPlan* onchip_plan_create(const KPlan& p, bool mixed, int K, int sumd, cudaStream_t st);
void onchip_plan_destroy(OnchipPlan* oc);
// The adjoint kernel fits too (gradient solves may use the on-chip path).
bool onchip_adjoint_ok(const OnchipPlan* oc);
// complex128 entries of one state image (CTA-major, Sc columns of D entries per CTA).
long long onchip_state_elems(const OnchipPlan* oc);
// stage-precision entries of one stored stage-input image (all CTAs).
long long onchip_stage_elems(const OnchipPlan* oc);
int onchip_ctas(const OnchipPlan* oc);
// doubles of one CTA's operator/energy/coupling accumulators (GradAcc layout minus gF).
long long onchip_acc_doubles(const OnchipPlan* oc);

// Forward RK4 steps n0 .. n1-1.  The start state is img_in (state image) when
// non-null, else psi_api (D x S, column innermost).  Writes the state before step
// n0 + c K to ck_out + c * state_elems when ck_out is non-null, the final state to
// psi_out (API layout) when non-null, and every stage input of every step to
// segY (stage images, slot 4 (step - n0) + stage) when non-null.  Returns launches.
int onchip_forward(const OnchipPlan* oc, const void* tab, const double2* psi_api, const double2* img_in,
                   double2* psi_out, double2* ck_out, int K, int n0, int n1, double dt, void* segY,
                   cudaStream_t st);
// API layout -> state image (columns past S are zero).
void onchip_to_image(const OnchipPlan* oc, const double2* api, double2* img, cudaStream_t st);
// Per-stage tables the adjoint reads, in the stage precision (complex64 / float in
// mixed precision, complex128 / double otherwise): term rows (3N x row), drive
// coefficients (3N x K), frame phases (3N x sumd) and the flat truncated operators.
struct OnchipTables {
  const void* tab;
  const void* coef;
  const void* ph;
  const void* opd;
};
// Adjoint of steps n1-1 .. n0 from the stage inputs in segY: pbar_img (state image
// of the co-state before the segment's last step) is pulled back in place; the
// cross-densities of every stage are contracted into gF_cta (CTA-major, 3N x K
// each, one store per stage slot) and acc_cta (CTA-major, onchip_acc_doubles
// each, added to).  *err is set when a bounded wait on a bulk copy gives up.
// Returns launches.
// colow: when onchip_colow_global(oc), a device buffer of onchip_state_elems complex64
// entries that holds the low words of the float-float co-state across the segments
// of one backward sweep (contents undefined before the first segment); else null.
int onchip_adjoint(const OnchipPlan* oc, const OnchipTables& tb, const void* segY, double2* pbar_img, int n0,
                   int n1, double dt, const XArgs& xa, int nst, double* gF_cta, double* acc_cta, int* err,
                   void* colow, cudaStream_t st);
bool onchip_colow_global(const OnchipPlan* oc);

#include "batcher.h"
// The RK4 forward kernel fits (a plan may hold only the Q2 layout).
bool onchip_forward_ok(const OnchipPlan* oc);
// Element-wise FP64 -> FP32 copy (tables for the mixed-precision adjoint).
void onchip_to_f32(const double* src, float* dst, long long n, cudaStream_t st);
bool onchip_mixed(const OnchipPlan* oc);
// acc += sum over CTAs (in CTA order) of the per-CTA accumulators.
void onchip_reduce(const OnchipPlan* oc, const double* gF_cta, const double* acc_cta, long long nst, int K,
                   int n1, int ne, GradAcc acc, cudaStream_t st);

// Suzuki-Trotter evolution (Sec. 2.3, App. A) of N Q2 sub-steps, lab frame, from psi_in
// to psi_out (API layout, may alias).  rows: (N + 1) x nq x d^2 1-body unitaries of the
// stage precision (row N = the first half of sub-step 0; row n = the last half of
// sub-step n followed by the first of sub-step n + 1); edges: per set s < nset and
// coupling e the half-step and full-step d^2 x d^2 unitaries at matrix (s ne + e) 2 + {0, 1};
// sub-step n uses set set_of[n % J].  q1: the first-order product instead (per step the
// couplings once each with their full-step unitary, then the next step's full-step
// 1-body row).  SG_E_UNSUPPORTED beyond 16 modes or 32 couplings.
sg_status onchip_q2_forward(const OnchipPlan* oc, const KPlan& p, const void* rows, const void* edges,
                            const double2* psi_in, double2* psi_out, int N, int J, const int* set_of, int nset,
                            cudaStream_t st, int* launches, bool q1 = false);
int onchip_dl(const OnchipPlan* oc);
// Suzuki-Trotter pulse gradient: pulls the final states psi and the co-state bar (API
// layout, lab frame) back through every factor of the N Q2 sub-steps and adds dF/df_k
// at sub-step n to gF_cta (CTA-major blocks of nstK >= N K doubles, slot n K + k;
// zeroed by the caller).  rows: [N][2 nq + K][d^2], per sub-step the inverse 1-body
// half-step factors U_i(n)^-1 (states), their adjoints U_i(n)^dag (co-states), then
// M_k(n) = U_i(n)^-1 L_k(n) with L_k the Frechet derivative of the local exponential
// along drive k's operator; edges: per set and coupling the inverse (half, full) and
// adjoint (half, full) coupling factors.  q1: the first-order product (N steps, rows of
// its full-step factors; the couplings pulled back in reverse order by their full-step
// factors).  SG_E_UNSUPPORTED for one mode, more than 32 couplings or 16 drives, or when
// the layout does not fit in shared memory.
sg_status onchip_q2_pulse_adjoint(const OnchipPlan* oc, const KPlan& p, const int* drv_mode, int K, const void* rows,
                                  const void* edges, const double2* psi, const double2* bar, int N, int J,
                                  const int* set_of, int nset, long long nstK, double* gF_cta, cudaStream_t st,
                                  int* launches, bool q1 = false);
