// Tiled ("slab") RK4 kernels for state slabs that live in HBM.
//
// The Kronecker-sum Hamiltonian is applied one mode group at a time (App. B: local
// operators contracted into the state tensor, never a dense matrix).  A pass loads
// tiles that hold the full extent of a group of modes for one column into shared
// memory and applies every term whose support lies in the group.  Terms are split
// over at most four passes; a stage is one launch per pass.
#pragma once
#include "grad.cuh"

struct SlabPlanHost;   // opaque

// Returns nullptr when the plan is not handled by the slab kernels (non-uniform
// level counts, more than 4 passes, too many terms per pass); the caller then
// uses the gather kernels.
// metadata_only: the plan is only read for its tiles and phases (the on-chip kernels),
// so the tiled kernels' own shared-memory limit does not apply.
SlabPlanHost* slab_plan_create(const KPlan& p, bool mixed, cudaStream_t st, bool metadata_only = false);
void slab_plan_destroy(SlabPlanHost* sp);
int slab_passes(const SlabPlanHost* sp);

// Internal slab layout: column-major [S][D] with a permuted digit order.
void slab_to_internal(const SlabPlanHost* sp, const double2* api, double2* internal, cudaStream_t st);
void slab_from_internal(const SlabPlanHost* sp, const double2* internal, double2* api, cudaStream_t st);

// One forward RK4 step pin -> pout (may alias) on internal buffers.  X holds the
// stage input (R)psi on entry and on exit; Xo, Dacc, kA are scratch slabs of the
// stage precision.  tab: stage rows of the stage precision.  Returns launches.
int slab_fwd_step(const SlabPlanHost* sp, bool mixed, const void* tab, int step, const double2* pin,
                  double2* pout, void*& X, void*& Xo, void* Dacc, void* kA, double dt,
                  cudaStream_t st);
// Forward step that keeps all four stage inputs: Yk[0] holds y1 = (R)psi on entry;
// y2..y4 go to Yk[1..3] and the next step's y1 to Ynext0.  Returns launches.
int slab_fwd_step_keep(const SlabPlanHost* sp, bool mixed, const void* tab, int step, const double2* pin,
                       double2* pout, void* const Yk[4], void* Ynext0, void* Dacc, void* kA, double dt,
                       cudaStream_t st);
// Recompute y2, y3, y4 of one step from y1 = (R)psi_n (STORE mode).  Returns launches.
int slab_fwd_store(const SlabPlanHost* sp, bool mixed, const void* tab, int step, const double2* psi,
                   void* const Y[4], void* kA, double dt, cudaStream_t st);
// One adjoint step: KB holds kbar_4 on entry and kbar_4 of the previous step on
// exit; pbar (complex128) is updated in place; the cross-densities of every
// stage are contracted into the accumulators of xa.  Returns launches.
int slab_adj_step(const SlabPlanHost* sp, bool mixed, const void* tab, int step, void* const Y[4],
                  double2* pbar, void*& KB, void*& KB2, void* Db, void* yA, double dt, XArgs xa,
                  const double2* tab64, const double* coef, const double2* ph, int sumd, int K,
                  cudaStream_t st);
// Size of the per-block partial buffer (double2 elements) slab_adj_step needs.
size_t slab_partial_elems(const SlabPlanHost* sp);

// Real-operator form of the forward stage passes (slab_dev.cuh): usable when every
// term is real in the truncated eigenbasis up to the interaction-frame phases and
// the level count is 2 or 4 (slab_real_shape_ok).  ztab: stage rows of real
// elements (float2 {m, m} pairs in mixed precision, double in FP64) at the complex
// row's offsets, parity-odd rows compressed when slab_allpar; ph: the stage phase
// rows exp(i E t), FP64, sumd per stage slot (3 per step).  Once bound, the
// forward, replay and recompute passes use it (SG_SLAB_REAL=0 at the solve keeps
// the complex rows).
bool slab_real_shape_ok(const SlabPlanHost* sp);
bool slab_allpar(const SlabPlanHost* sp);
// zop: the drive operators' real matrices (K x DL x DL, packed like the rows), with
// the drives of each 1-body slot (drv_list[drv_of_slot_start[u] .. [u + 1]]): the
// adjoint passes of a pulse-only gradient then run in the real-operator form too
// (nullptr keeps the complex-row adjoint).
void slab_bind_real(SlabPlanHost* sp, const void* ztab, const double2* ph, int sumd, const void* zop,
                    const int* drv_of_slot_start, const int* drv_list);

// Suzuki-Trotter products (Sec. 2.3, App. A: the palindromic Q2 sub-steps of Q2, Q4 and
// Q4j) on the tiles of a two-pass plan, for slabs too large for the on-chip kernels.
// One sub-step is two in-place passes over the state (stage precision, internal
// layout): the first group's tiles take the previous sub-step's reversed couplings of
// that group, the merged 1-body factors of its modes and this sub-step's couplings of
// that group; the second group's tiles its other modes' 1-body factors and its part of
// the palindrome (with the middle, full-step coupling).  Needs the couplings of the
// first pass to come before those of the second in term order (the ring's and the
// chain's plans).  slab_q2_ok builds the factor lists (false: unsupported).
bool slab_q2_ok(SlabPlanHost* sp, const KPlan& p, bool mixed);
void slab_q2_free(SlabPlanHost* sp);
int slab_dl(const SlabPlanHost* sp);
// M = N J sub-steps from X (in place).  rows: (M + 1) x nq x DL^2 merged 1-body factors
// (the Q2 tables of the on-chip path), edges: per set and coupling the half- and
// full-step unitaries; sub-step m uses set set_of[m % J].  q1: the first-order product
// (M steps; rows of its full-step factors, each coupling once per step by its full-step
// unitary).  Returns launches.
int slab_q2_run(const SlabPlanHost* sp, bool mixed, const void* rows, const void* edges, void* X, int M, int J,
                const int* set_of, bool q1, cudaStream_t st);
// Pulse gradient of the tiled product (the discrete adjoint of Sec. 2.5): the final
// states X and co-states Lb (internal layout, stage precision) are pulled back through
// every factor in reverse order, X by the inverse factors and Lb by the adjoints, and at
// each 1-body half step every drive k of the pass's modes adds Re <Lb, M_k(s) X> to
// gF[s K + k].  gtab: per sub-step s the gradient tables [2 nq + K][DL^2] (U^-1, U^dag,
// M_k); edges_pb: the pull-back coupling table (per set and coupling the inverse half,
// inverse full, adjoint half and adjoint full factor); gpart: slab_q2_grad_part(sp)
// doubles; ticket: one zeroed counter (left zeroed).  slab_q2_grad_ok: the backward lists
// fit.  Returns launches, or -1 when a drive's mode has no 1-body factor in the plan.
bool slab_q2_grad_ok(const SlabPlanHost* sp);
size_t slab_q2_grad_part(const SlabPlanHost* sp);
int slab_q2_grad_run(const SlabPlanHost* sp, bool mixed, const void* gtab, const void* edges_pb, void* X, void* Lb,
                     int M, int J, const int* set_of, bool q1, int K, const int* drv_mode, double* gF,
                     double* gpart, unsigned* ticket, cudaStream_t st);
