/*
 * sg.h — C ABI of the GB300 superconducting-circuit evolution library (libsupergpu.so).
 *
 * The library computes, on one GPU, the hot path of a differentiable simulator of
 * superconducting processors (arXiv 2406.18155, "SuperGrad"):
 *
 *   define subsystems and couplings  ->  diagonalise and truncate each subsystem
 *   ->  build the drive operators     ->  evolve a batch of state columns with
 *   fixed-step RK4                    ->  gate fidelity and its gradient with
 *   respect to pulse and Hamiltonian parameters.
 *
 * Conventions shared by every call
 * --------------------------------
 *  * Units: energies, amplitudes, frequencies in rad/ns (the paper's 2*pi*GHz,
 *    Sec. 3.1); times in ns.
 *  * Composite index: r = sum_i l_i * prod_{j>i} d_j (mode 0 most significant).
 *    A state slab of D rows and S columns is stored row-major with the column
 *    index innermost: element (r, s) at offset r*S + s, complex128 as (re, im).
 *  * Computational states: each mode in level 0 or 1; label j in [0, 2^Nq) with
 *    mode 0 as the most significant bit.
 *  * Return value: SG_OK (0) or a negative SG_E_* code.  Nothing throws across
 *    the ABI.  sg_last_error() gives a message for the last failed call on the
 *    context.
 *  * All device work is ordered on the context's stream; calls on one context
 *    must come from one host thread at a time.
 *  * Ownership: the library owns contexts, systems and their device tables; the
 *    caller owns every pointer it passes in (host or device).  A call never
 *    retains a caller pointer after it returns.
 */
#ifndef SG_H
#define SG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int sg_status;
typedef struct sg_ctx sg_ctx;
typedef struct sg_system sg_system;
typedef struct sg_server sg_server;

enum {
  SG_OK = 0,
  SG_E_INVALID = -1,      /* bad argument: NaN, out-of-range index, T/dt not integral ... */
  SG_E_NOMEM = -2,        /* device or host allocation failed                            */
  SG_E_STATE = -3,        /* call out of order (e.g. evolve before prepare)               */
  SG_E_CUDA = -4,         /* a CUDA runtime error; the message names it                   */
  SG_E_TIMEOUT = -5,      /* a bounded device wait gave up                                */
  SG_E_PENDING = -6,      /* serving: request not finished yet                            */
  SG_E_NOMEM_RETRY = -7,  /* serving: over the memory budget now, retry later            */
  SG_E_CANCELLED = -8,    /* serving: request was cancelled                               */
  SG_E_NOTFOUND = -9,     /* serving: unknown ticket                                      */
  SG_E_UNSUPPORTED = -10  /* a configuration this build does not handle                    */
};

enum { SG_OP_N = 0, SG_OP_PHI = 1 };                          /* charge n, phase phi         */
/* operators 2, 3, ... of a mode: its local operators (sg_add_local_op), at most 6 */
enum { SG_ENV_GAUSSIAN = 0, SG_ENV_PWC = 1, SG_ENV_COSINE = 2 };
enum { SG_FP64 = 0, SG_MIXED = 1 };                           /* arithmetic of the evolution */
enum { SG_FRAME_INTERACTION = 0, SG_FRAME_LAB = 1 };
enum { SG_FID_AVG = 0, SG_FID_STATE = 1 };

/* ---------------------------------------------------------------------------
 * Contexts
 * ------------------------------------------------------------------------- */

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * (e.g. torch.cuda.current_stream().cuda_stream) or NULL for the legacy default
 * stream.  The stream is borrowed: the caller keeps it alive. */
sg_status sg_ctx_create(sg_ctx** out, int device, void* cuda_stream);
sg_status sg_ctx_destroy(sg_ctx* ctx);
/* Message of the last failed call on `ctx` (or of the last failed sg_ctx_create
 * when ctx is NULL).  Valid until the next call on the same context. */
const char* sg_last_error(const sg_ctx* ctx);
/* Library version string. */
const char* sg_version(void);

/* ---------------------------------------------------------------------------
 * System definition (Sec. 2.1, Eq. 1: 1-body and 2-body local terms)
 * ------------------------------------------------------------------------- */

sg_status sg_system_create(sg_ctx* ctx, sg_system** out);
sg_status sg_system_destroy(sg_system* sys);

/* Transmon, H = 4 E_C (n - n_g)^2 - E_J cos(phi) in the charge basis
 * n in [-ncut, ncut] (2 ncut + 1 states, ncut <= 31), truncated to `levels`
 * eigenstates (2 <= levels <= 8).  Writes the new mode index to *mode_out. */
sg_status sg_add_transmon(sg_system* sys, double ej, double ec, double ng, int ncut,
                          int levels, int* mode_out);

/* Fluxonium, Eq. 8: H = 4 E_C n^2 + E_L phi^2 / 2 - E_J cos(phi - phi_ext) in an
 * n_osc-state oscillator basis (n_osc <= 64), truncated to `levels` eigenstates. */
sg_status sg_add_fluxonium(sg_system* sys, double ej, double ec, double el, double phi_ext,
                           int n_osc, int levels, int* mode_out);

/* 2-body coupling strength * op_a(mode_a) (x) op_b(mode_b) (Eq. 9; the capacitive
 * J_C n n term is op_a = op_b = SG_OP_N).  mode_a != mode_b.  A transmon has only
 * SG_OP_N. */
sg_status sg_add_coupling(sg_system* sys, int mode_a, int op_a, int mode_b, int op_b,
                          double strength, int* term_out);

/* A local operator of one mode for generic Kronecker terms (Eq. 1: every term acts
 * on one or two subsystems): `re_im` is a d x d Hermitian matrix (d = the mode's
 * levels, row-major, interleaved real and imaginary parts, copied) in the mode's
 * truncated eigenbasis (sign gauge of sg_get_spectrum).  It can then be used as the
 * operator of drives and couplings like SG_OP_N; *op_out receives its id (2, 3, ...).
 * Its matrix elements are fixed: the gradient w.r.t. E_J, E_C, E_L sees only its
 * frame phases exp(i (E_a - E_b) t), not a change of the eigenbasis.  Marks the
 * system unprepared.  SG_E_INVALID: bad mode, NULL, non-finite or non-Hermitian
 * (|O - O^dag| > 1e-12 max|O|); SG_E_UNSUPPORTED: more than 6 on one mode. */
sg_status sg_add_local_op(sg_system* sys, int mode, const double* re_im, int* op_out);

/* Mark a mode as a coupler (coupler != 0) or as a qubit (0, the default).  The
 * computational subspace of the fidelity (Eq. 13, Eq. D2) is every qubit mode in
 * level 0 or 1 with every coupler mode in its ground state, Dc = 2^(qubit modes):
 * the schemes of Sec. 4 where qubits interact through a coupler mode (transmon
 * qubits with a transmon coupler; fluxoniums with a transmon coupler, FTF).  A
 * coupler evolves like any other mode.  Targets are Dc x Dc over the qubit modes
 * (mode order, first qubit most significant); a solve needs 1..12 qubit modes.
 * SG_E_INVALID for a bad mode index. */
sg_status sg_set_coupler(sg_system* sys, int mode, int coupler);

/* Drive f(t) * op(mode) with f(t) = E(t) cos(omega_d t + phase) (Eq. C1).
 *   SG_ENV_GAUSSIAN: E = amp exp(-(t - t0)^2 / (2 sigma^2))
 *   SG_ENV_PWC:      E = amps[j] on the j-th of nseg equal segments of [0, length);
 *                    an RK4 step takes the segment of its midpoint; 0 after length.
 *   SG_ENV_COSINE:   E = amp/2 (1 - cos(2 pi t / length)) on [0, length], 0 after (Eq. C2)
 * omega_mode >= 0 ties omega_d to that mode's bare 0-1 frequency E_1 - E_0 (then
 * `omega_d` is ignored and the tie is differentiated through); -1 uses omega_d.
 * `amps` (nseg values) is copied.  length must be a whole number of half steps of
 * every later evolution. */
typedef struct {
  int kind;
  int nseg;
  const double* amps;
  double amp;
  double sigma;
  double t0;
  double length;
  double omega_d;
  int omega_mode;
  double phase;
} sg_pulse;
sg_status sg_add_drive(sg_system* sys, int mode, int op, const sg_pulse* p, int* drive_out);

/* Flat real parameter vector used by sg_get_params / sg_set_params and by the
 * gradient outputs:
 *   pulse part:  for each drive in order: nseg amplitudes (PWC) or 1 amplitude;
 *   ham part:    for each mode (E_J, E_C, E_L) (E_L is unused, 0, for a transmon),
 *                then each coupling's strength.
 * Counts: */
sg_status sg_param_counts(const sg_system* sys, int* n_pulse, int* n_ham);
sg_status sg_get_params(const sg_system* sys, double* pulse, double* ham);
/* Changing a ham parameter marks the system unprepared. */
sg_status sg_set_params(sg_system* sys, const double* pulse, const double* ham);

/* ---------------------------------------------------------------------------
 * Diagonalise and truncate (Sec. 2.1; subsystem eigensolve in FP64 on the GPU)
 * ------------------------------------------------------------------------- */

/* Builds every subsystem matrix, diagonalises it (FP64 Jacobi on the device),
 * fixes each eigenvector's sign (first component with |v_i| >= 1e-3 max|v| is
 * positive), keeps the lowest `levels`, shifts energies so E_0 = 0 and projects
 * n and phi into the truncated eigenbasis.  Idempotent. */
sg_status sg_prepare(sg_system* sys);
/* Host copies of one mode's truncated data: energies[levels], n and phi as
 * levels x levels complex row-major (re, im) (phi is zero for a transmon).  Any
 * output pointer may be NULL. */
sg_status sg_get_spectrum(const sg_system* sys, int mode, double* energies,
                          double* n_re_im, double* phi_re_im);
/* Composite dimension D = prod levels and number of modes. */
sg_status sg_dims(const sg_system* sys, long long* D, int* nmodes);

/* ---------------------------------------------------------------------------
 * Evolution (RK4) and fidelity (Eq. 13, Eq. D2)
 * ------------------------------------------------------------------------- */

typedef struct {
  double T;                     /* duration; T/dt must be an integer (within 1e-9 rel.)   */
  double dt;                    /* RK4 step                                               */
  int precision;                /* SG_FP64 or SG_MIXED (FP32 stages, FP64 state across steps) */
  int frame;                    /* SG_FRAME_INTERACTION (default) or SG_FRAME_LAB          */
  int ncols;                    /* S, number of evolved columns                           */
  const long long* col_index;   /* host, S flat initial basis indices, or NULL: the
                                   columns of psi are the initial states                  */
  int solver;                   /* SG_SOLVER_RK4 (0, default), _Q1, _Q2, _Q4 or _Q4J       */
  int compensation;             /* SG_COMP_NONE (0, default) or SG_COMP_VZ (fidelities)    */
  int basis;                    /* SG_BASIS_PRODUCT (0, default) or SG_BASIS_DRESSED        */
} sg_evolve_opts;

/* Basis of the gate (sg_fidelity, sg_fidelity_grad; App. C).  SG_BASIS_PRODUCT: the
 * computational states are bare product states.  SG_BASIS_DRESSED: they are the
 * eigenstates of the idle Hamiltonian (lab frame, no drives: level energies and
 * couplings) of largest overlap with the bare computational states, each signed so
 * that overlap is positive; the evolved columns start in them and are projected on
 * them (U -> V^dag U V restricted to the computational states).  Needs D <= 1024, a real
 * idle Hamiltonian, non-degenerate dressed computational levels and every evolved
 * column a computational state (each once), else SG_E_INVALID / SG_E_UNSUPPORTED; with
 * sg_fidelity_grad, grad_ham must be NULL (the pulse gradient only). */
enum { SG_BASIS_PRODUCT = 0, SG_BASIS_DRESSED = 1 };

/* Compensation of the gate fidelity (sg_fidelity, sg_fidelity_grad): the paper's gate
 * metric assumes errorless single-qubit gates around the pulses.  SG_COMP_VZ takes
 * M = T^dag Z(a) U Z(b) with a virtual Z gate diag(1, e^{i phase}) on every qubit
 * before and after, the phases maximising |tr M| (coordinate ascent from zero phases,
 * qubit by qubit, each phase set to its exact maximiser, until a sweep does not raise
 * |tr M|, at most 2000 sweeps); F_avg and F_state are those of M.  Needs every
 * computational state evolved exactly once (D_c <= 256), else SG_E_INVALID.  The
 * gradient is that of F at the found phases (F is stationary in them). */
enum { SG_COMP_NONE = 0, SG_COMP_VZ = 1 };

/* Solvers.  SG_SOLVER_Q1: the first-order Suzuki-Trotter product of Sec. 2.3 and App. A,
 * Q1(dt) = prod_k exp(-i H_k dt) over the same local terms in the same order (the first
 * acts first), the time-dependent terms at the step's midpoint.  SG_SOLVER_Q2: the second-order
 * Suzuki-Trotter product of Sec. 2.3 and
 * App. A, Q2(dt) = prod_k exp(-i H_k dt/2) prod_k' exp(-i H_k' dt/2) (k' reversed)
 * over the local terms H_i = diag(E^(i)) + sum_{drives on i} f(t) O (every mode, in mode
 * order) and J A (x) B (the couplings, in order), with the time-dependent terms at the
 * step's midpoint; always in the lab frame (`frame` is ignored).  SG_SOLVER_Q4: the real
 * fourth-order product Q2(p dt) Q2((1-2p) dt) Q2(p dt), p = 1/(2 - 2^(1/3)), each Q2
 * sub-step with its time-dependent terms at its own midpoint.  SG_SOLVER_Q4J: the complex
 * product Q2(p dt) Q2(p* dt), p = (3 - i sqrt 3)/6, the drive coefficients continued to
 * the complex sub-step midpoints; third order (the composition is not palindromic).
 * They run on the on-chip kernels (every mode with the same level count 2..5,
 * D <= 4096) and on the HBM-tiled kernels of a two-pass plan whose first group's
 * couplings come first in term order and whose last coupling lies in the second group;
 * else SG_E_UNSUPPORTED.  sg_fidelity_grad with a Suzuki-Trotter solver
 * computes the pulse-parameter gradient only (grad_ham must be NULL, else
 * SG_E_UNSUPPORTED): the exact discrete adjoint of the product (Sec. 2.5), the states
 * pulled back through each factor's inverse and the co-state through its adjoint (no
 * checkpoints), dU/df by the Frechet derivative of the local exponential; it needs >= 2
 * modes, <= 16 drives, <= 32 couplings and, on-chip, four state images of a CTA's
 * columns in shared memory (mixed precision fits D = 4096, FP64 does not; the tiled
 * kernels hold two tiles of states and two of co-states). */
enum { SG_SOLVER_RK4 = 0, SG_SOLVER_Q1 = 1, SG_SOLVER_Q2 = 2, SG_SOLVER_Q4 = 4, SG_SOLVER_Q4J = 5 };

/* Evolve S columns from t = 0 to T and leave the lab-frame states in psi_dev
 * (device, D*S complex128, column innermost).  If opts->col_index is NULL psi_dev
 * also supplies the initial states. */
sg_status sg_evolve(sg_system* sys, const sg_evolve_opts* opts, void* psi_dev);

/* Same evolution as sg_evolve, for callers that cannot allocate device memory
 * during the call: a program whose GPU memory belongs to another allocator (for
 * example a framework's caching allocator that has reserved the device), or a
 * latency-bound loop that cannot afford cudaMalloc's implicit synchronisation.
 * The paper has no counterpart; this is an interface of this library only.
 * Every per-call buffer lives in one array of 32 MiB compiled into the library,
 * held on every GPU that loads the library until the process exits; the call
 * makes no cudaMalloc or cudaFree (sg_prepare, which allocates the system's own
 * tables, must have run before).  The first call on a device looks up the array's
 * device address; make that first call before any stream capture.  All calls
 * share the one array and it keeps the last call's contents: calls that overlap
 * on the GPU (on different streams or contexts) race.  Uses the generic gather
 * kernels.  It synchronises the context stream before it returns (its small
 * inputs are staged from host buffers that live only for the call).  Returns SG_E_INVALID with the needed size when the evolution needs
 * more than the 32 MiB (stage tables of 3 T/dt rows plus three D x S slabs). */
sg_status sg_evolve_noalloc(sg_system* sys, const sg_evolve_opts* opts, void* psi_dev);

/* Open-system evolution (the paper's LindbladObj, Sec. 2.2; its solver carried over to
 * the vectorised master equation, App. C last paragraph):
 *   d rho/dt = -i [H(t), rho] + sum_c g_c (L_c rho L_c^dag - {L_c^dag L_c, rho} / 2).
 * sg_add_collapse adds a collapse operator L (host, d x d complex row-major (re, im),
 * in the mode's truncated eigenbasis; copied) on one mode at rate g >= 0 (1/ns); in
 * the interaction frame L rotates with the frame like every operator.  At most 16.
 * The evolution runs vec(rho) (row-major, ket index x D + bra index) under
 * -i H_eff on 2 Nq modes (ket modes, then bra modes with negated energies) with
 * the local terms of the generator: ket 1-body H_i(t) - (i/2) sum_c g_c L_c^dag L_c,
 * bra 1-body -H_i(t)^T - (i/2) sum_c g_c (L_c^dag L_c)^T, ket couplings J A (x) B, bra
 * couplings -J A^T (x) B^T, jumps i g_c L_c (x) L_c^*, on the same RK4 kernels (stage
 * times of R2, complex stage rows, FP64 or mixed); at most 8 modes (16 doubled).
 * sg_gate_fidelity_open_grad adds the pulse-parameter gradient of the gate fidelity. */
sg_status sg_add_collapse(sg_system* sys, int mode, const double* L_re_im, double rate, int* id_out);
/* rho(T) (host, D x D complex row-major, lab frame) from rho0 (host, same layout).
 * opts: T, dt, precision, frame; ncols and col_index are ignored. */
sg_status sg_evolve_open(sg_system* sys, const sg_evolve_opts* opts, const double* rho0_re_im,
                         double* rho_out_re_im);
/* Average gate fidelity of the open evolution against the target unitary (host,
 * Dc x Dc complex): the channel on the computational block, S[(a,b),(j,k)] =
 * <c_a| E(|c_j><c_k|) |c_b>, from Dc^2 density-matrix evolutions run as columns of
 * one solve; F_out[1] = F_pro = Re sum conj(T (x) T^*) S / Dc^2 (process fidelity),
 * F_out[0] = F_avg = (Dc^2 F_pro + P) / (Dc (Dc + 1)) with P the population kept in
 * the computational block (Nielsen's relation written for a channel that may leak;
 * for a closed evolution it equals sg_fidelity's F_avg).  1..6 qubit modes. */
sg_status sg_gate_fidelity_open(sg_system* sys, const sg_evolve_opts* opts, const double* target_re_im,
                                double* F_out);
/* sg_gate_fidelity_open with the gradient of one of its fidelities (the paper's
 * back-propagation carried over to the vectorised master equation, App. C last
 * paragraph; Sec. 2.5): kind SG_FID_AVG differentiates F_avg, SG_FID_STATE the process
 * fidelity F_pro.  F_out[2] as sg_gate_fidelity_open; grad_pulse (host, sg_param_counts'
 * pulse count doubles, the order of sg_get_params) receives dF/d(pulse parameters);
 * grad_ham (host, the Hamiltonian count: E_J, E_C, E_L per mode, then J per coupling;
 * NULL: not computed) dF/d(Hamiltonian parameters) through the subsystems'
 * eigen-derivatives (the collapse operators are held fixed in the truncated
 * eigenbasis).  Exact derivative of the discrete map: the Dc^2 columns are pulled back
 * through each RK4 step by the adjoint of the non-Hermitian generator (stage rows of
 * H_eff^dag), from segment checkpoints every ckpt steps (0: round(sqrt(N))).  opts: T,
 * dt, precision, frame (ncols and col_index ignored; RK4 only). */
sg_status sg_gate_fidelity_open_grad(sg_system* sys, const sg_evolve_opts* opts, const double* target_re_im,
                                     int kind, double* F_out, double* grad_pulse, double* grad_ham, int ckpt);

/* Batched dense evolution on the tensor cores: nsys systems of one shape (the same
 * modes and level counts, the same number of drives; parameters, couplings and
 * pulses may differ) evolved together from the basis columns opts->col_index over
 * the same T and dt, leaving the lab-frame states in psi_dev (device, nsys x D x S
 * complex128, system-major, column innermost; caller-owned).  The paper applies H
 * densely where the matrices are small (App. B, the dense versus local cost); here
 * each system's terms, real in the truncated eigenbasis up to the interaction-frame
 * phases, form the constant operand [C; O_1; ...; O_K] of tcgen05 TF32 matrix
 * products with the state z = P^dag y (P the frame phases), each product split into
 * three TF32 products (3xTF32, about FP32 accuracy, accumulated in FP32 in tensor
 * memory); the RK4 stage math is FP32 and the state float-float.  Requires
 * opts->precision == SG_MIXED and the RK4 solver; S = ncols in {4, 8, 16};
 * (1 + drives) x D, with D rounded up to a multiple of 8, at most 128 (for
 * example D = 16 with one drive: 4 systems per CTA; D = 25: 2); D <= 64; every
 * operator of a drive real, every coupling of two real or two imaginary factors
 * (else SG_E_UNSUPPORTED).  All systems must be prepared and share one context.
 * A bounded wait for the tensor-core products that runs out returns SG_E_TIMEOUT.
 * sg_last_stats of the first system gets the device time of the launch (out[0]). */
sg_status sg_evolve_batch(sg_system* const* systems, int nsys, const sg_evolve_opts* opts, void* psi_dev);

/* Evolve the columns named by opts->col_index and reduce them to fidelities.
 * target_re_im: host, Dc x Dc complex (Dc = 2^Nq), row-major (re, im); column j is
 * the target image of computational state j.  Columns whose initial state is not
 * computational are evolved but ignored by the fidelity.
 *   F_avg   = (tr(M M^dag) + |tr M|^2) / (Dc (Dc + 1)),  M = T^dag U_c  (NaN unless
 *             every computational state is evolved exactly once)
 *   F_state = |(1/S_c) sum_s <target_s | psi_s>|^2 over the S_c computational columns
 * F_out[0] = F_avg, F_out[1] = F_state.  Ucomp_out (nullable, host) receives the
 * Dc x S computational rows of the lab-frame columns as complex row-major. */
sg_status sg_fidelity(sg_system* sys, const sg_evolve_opts* opts, const double* target_re_im,
                      double* F_out, double* Ucomp_out);

/* F (of `kind`) and dF/dtheta by the exact discrete adjoint of RK4, with the forward
 * states recomputed per segment from checkpoints every `ckpt_interval` steps (0 =
 * about sqrt(N)).  grad_pulse / grad_ham are host arrays of sg_param_counts sizes.
 * grad_ham may be NULL: the Hamiltonian-parameter gradient is then not computed,
 * which skips the cross-densities of the coupling terms (the pulse gradient needs
 * only those of the driven terms) and gives the same grad_pulse.
 * F_out receives {F_avg, F_state}. */
sg_status sg_fidelity_grad(sg_system* sys, const sg_evolve_opts* opts,
                           const double* target_re_im, int kind, double* F_out,
                           double* grad_pulse, double* grad_ham, int ckpt_interval);

/* Column-sharded F and gradient: the paper distributes the unitary's columns across
 * devices (Sec. 4.2, multi-GPU benchmark).  Each shard (a process, usually one per
 * GPU) calls this with its own columns in opts->col_index; together the shards'
 * columns are the columns of the unsharded sg_fidelity_grad (for SG_FID_AVG every
 * computational state exactly once over all shards).  The columns evolve
 * independently; the fidelity couples them only through sums over columns, so the
 * call exchanges two small vectors through the caller's collective:
 *   1. after the forward evolution, buf = {Re z, Im z, q, S_c} (n = 4) of this
 *      shard, z = sum_s <target_l(s)|psi_s>, q = sum_s ||T^dag psi_s||^2 over its
 *      computational columns, S_c their number;
 *   2. after the adjoint, this shard's gradient {grad_pulse, grad_ham} (n = the
 *      number of pulse parameters, plus 3 Nq + couplings when grad_ham is given).
 * `allreduce(buf, n, user)` must replace buf by its element-wise sum over all
 * shards (every shard calls it the same number of times, in the same order) and
 * return 0; non-zero aborts the call with SG_E_STATE.  F (from the sums) and the
 * gradient (the sum of the shards' gradients, linear in the co-states) then equal
 * the unsharded call's up to summation order, on every shard.  Product basis, no
 * compensation (else SG_E_UNSUPPORTED).  The callback runs on the calling thread
 * between kernel launches, with the context stream idle and the context held: it
 * must not call this library on the same context. */
typedef int (*sg_allreduce_fn)(double* buf, int n, void* user);
sg_status sg_fidelity_grad_sharded(sg_system* sys, const sg_evolve_opts* opts, const double* target_re_im,
                                   int kind, double* F_out, double* grad_pulse, double* grad_ham,
                                   int ckpt_interval, sg_allreduce_fn allreduce, void* user);

/* Timing and memory of the last sg_fidelity / sg_fidelity_grad on this system:
 * out[0] forward ms, out[1] gradient (backward) ms, out[2] peak library device
 * bytes during the call, out[3] checkpoint interval used, out[4] number of kernel
 * launches issued. */
sg_status sg_last_stats(const sg_system* sys, double* out5);

/* Device time per kernel family of the last sg_evolve / sg_fidelity /
 * sg_fidelity_grad on this system.  When the environment variable SG_KTIMING=1 is
 * set at the call, CUDA events on the context stream bracket the launches of every
 * 16th step; out[3k] = bracketed ms, out[3k+1] = bracketed launches, out[3k+2] =
 * all launches of family k, for k = 0 forward stage passes, 1 adjoint stage passes,
 * 2 forward recompute (store) passes.  n is the capacity of out (>= 9). */
sg_status sg_kernel_times(const sg_system* sys, double* out, int n);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of fidelity+gradient solves
 * ------------------------------------------------------------------------- */

typedef struct {
  sg_system* sys;               /* prepared or not; the server prepares it             */
  sg_evolve_opts opts;          /* col_index may be NULL: every computational state    */
  const double* target_re_im;   /* Dc x Dc, copied at submit                            */
  int kind;                     /* SG_FID_AVG or SG_FID_STATE                           */
  int want_grad;                /* 1: also compute the gradient                          */
} sg_request;

typedef struct {
  sg_status status;             /* SG_OK, or the error of the solve                     */
  double F[2];                  /* F_avg, F_state                                        */
  double* grad_pulse;           /* library-owned, valid until sg_server_destroy          */
  double* grad_ham;
  int n_pulse, n_ham;
  double submit_s, start_s, done_s;   /* server clock (seconds since create)            */
  char error[192];              /* the solve's error message when status != SG_OK        */
} sg_result;

typedef struct {
  uint64_t submitted, completed, cancelled, rejected;
  double solves_per_s;          /* completed / busy wall time                           */
  double p50_s, p99_s;          /* latency submit -> done of completed requests          */
  double gpu_busy_frac;
  size_t mem_in_use, mem_budget;
  int active_slots, max_slots;
  long long batches;             /* slot runs that packed several requests (max_batch > 1)  */
  long long batched_requests;    /* requests run in those packs                             */
  long long batched_launches;    /* batched on-chip launches issued                        */
  long long batched_launch_members; /* solves summed over those launches                   */
} sg_stats;

/* A server owns `max_slots` slots, each a worker thread with its own CUDA stream
 * (continuous batching): requests are admitted in arrival order while a slot is
 * free and the device memory they need fits `mem_budget_bytes`; each admitted
 * request runs as one fidelity(+gradient) solve on its slot's stream, so the
 * kernels of all admitted requests overlap on the device, and a request that
 * arrives while others run starts as soon as a slot and memory free up.
 * Results do not depend on what else runs (each solve has its own buffers and
 * fixed-order reductions).  gpu_busy_frac in sg_stats is the fraction of the
 * server's wall time with at least one request running, not a device occupancy. */
sg_status sg_server_create(sg_ctx* ctx, size_t mem_budget_bytes, int max_slots, sg_server** out);
sg_status sg_server_destroy(sg_server* srv);
/* Packing of same-shape requests (max_batch 1..16, default 1: none).  With
 * max_batch > 1 a slot that admits a request also admits up to max_batch - 1 queued
 * requests of the same step shape (modes and level counts, terms, drive kinds,
 * columns, precision, frame and dt; parameter values and T may differ) while memory
 * allows, and runs them together: each on a stream of its own, their on-chip
 * launches (the forward evolution, and per checkpoint segment the recompute and
 * the pull-back) issued as shared batched launches, one CTA range per request
 * (pack members of different T run to the longest one's end in each shared
 * launch).  Each request's arithmetic is that of its solve alone.  Call while no
 * request is queued or running (SG_E_STATE otherwise). */
sg_status sg_server_set_batch(sg_server* srv, int max_batch);
/* Queue a request.  The request's system must stay alive until its result is
 * polled, and the caller makes no other call on it meanwhile (its slot runs it
 * with the slot's context and prepares it if needed).  One system has at most one
 * request queued or running: a second submit of the same system before the first
 * is done (or cancelled) returns SG_E_STATE.  Returns SG_E_NOMEM_RETRY if the
 * request alone exceeds the budget. */
sg_status sg_server_submit(sg_server* srv, const sg_request* req, uint64_t* ticket);
/* SG_OK and *out filled when done; SG_E_PENDING while queued or running. */
sg_status sg_server_poll(sg_server* srv, uint64_t ticket, sg_result* out);
/* Block until the ticket is done (or cancelled); same outputs as poll. */
sg_status sg_server_wait(sg_server* srv, uint64_t ticket, sg_result* out);
sg_status sg_server_cancel(sg_server* srv, uint64_t ticket);
sg_status sg_server_stats(sg_server* srv, sg_stats* out);

#ifdef __cplusplus
}
#endif
#endif /* SG_H */
