// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>
#include <mutex>

#include "../../include/sg.h"

#define SG_MAXQ 16        // modes per system
#define SG_MAXD 8         // truncated levels per mode
#define SG_MAXM 64        // subsystem basis size (charge states or oscillator states)
#define SG_MAXEDGE 48     // 2-body terms per system
#define SG_MAXDRIVE 48    // drives per system
#define SG_MAXOP 8        // operators per mode: n, phi and up to 6 local operators

// ---------------------------------------------------------------------------
// Host-side model of a system
// ---------------------------------------------------------------------------
struct HostMode {
  int kind;        // 0 transmon, 1 fluxonium
  double ej, ec, el, ng, phi_ext;
  int M;           // basis size
  int d;           // kept levels
  int coupler;     // 1: held in its ground state in the computational subspace
  std::vector<double> local;   // local operators, 2 d^2 doubles each (truncated eigenbasis)
};
struct HostCoupling { int a, op_a, b, op_b; double J; };
struct HostDrive {
  int mode, op, kind, nseg;
  std::vector<double> amps;
  double amp, sigma, t0, length, omega_d, phase;
  int omega_mode;
};

// Device layout of one mode's prepared data (all FP64).  Matrices are M x M
// row-major unless noted; complex as double2.
struct ModeDev {
  int kind, M, d, pad;
  double* w;          // M eigenvalues, ascending
  double* V;          // M x M eigenvectors in columns, gauge fixed
  double* dH;         // 3 x M x M: dH/d(ej, ec, el)
  double2* ops;       // 2 x M x M: n, phi (phi zero for transmon)
  double2* dops;      // 2 x 3 x M x M: d(op)/d(param)
  double* E;          // d, ground shifted
  double2* opd;       // 2 x d x d truncated n, phi
};

struct sg_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string last_error;
  std::mutex mu;
};

struct StageTables;  // defined in evolve.cu

// A collapse operator of the open-system evolution: L (d x d complex in the truncated
// eigenbasis, 2 d^2 doubles) on one mode at rate gamma (1/ns).
struct HostCollapse { int mode; std::vector<double> L; double rate; };

struct sg_system {
  sg_ctx* ctx = nullptr;
  std::vector<HostMode> modes;
  std::vector<HostCoupling> couplings;
  std::vector<HostCollapse> collapses;
  std::vector<HostDrive> drives;
  bool prepared = false;
  // device data
  void* mode_block = nullptr;     // one allocation for all modes
  size_t mode_block_bytes = 0;
  std::vector<ModeDev> mdev;      // host copy of the device pointers
  ModeDev* mdev_dev = nullptr;    // device array of ModeDev
  // host copies of the prepared truncated data
  std::vector<std::vector<double>> E_host;       // per mode, d
  std::vector<std::vector<double>> opd_host;     // per mode, 2*d*d complex -> 4*d*d doubles
  std::vector<int> parity_odd;                   // per mode*SG_MAXOP+op: operator is parity-odd
  double last_stats[5] = {0, 0, 0, 0, 0};
  double ktimes[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
};

// error helpers --------------------------------------------------------------
sg_status sg_fail(sg_ctx* ctx, sg_status code, const std::string& msg);
#define SG_CUDA_TRY(ctx, expr)                                                     \
  do {                                                                             \
    cudaError_t _e = (expr);                                                       \
    if (_e != cudaSuccess)                                                         \
      return sg_fail((ctx), SG_E_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)

// prepare.cu
sg_status sg_prepare_impl(sg_system* sys);
// runs the eigen-derivative chain: given per-mode operator co-gradients
// opbar[mode][op][d*d] (complex, device) and energy co-gradients ebar[mode][d]
// (device), writes dL/d(ej, ec, el) per mode into out_dev (3*nq doubles).
sg_status sg_chain_device_params(sg_system* sys, const double2* opbar_dev,
                                 const double* ebar_dev, double* out_dev);

// evolve.cu
sg_status sg_evolve_impl(sg_system* sys, const sg_evolve_opts* o, void* psi_dev);
sg_status sg_evolve_open_impl(sg_system* sys, const sg_evolve_opts* o, const double* rho0, double* rho_out);
sg_status sg_gate_fidelity_open_impl(sg_system* sys, const sg_evolve_opts* o, const double* target, double* F_out);
sg_status sg_gate_fidelity_open_grad_impl(sg_system* sys, const sg_evolve_opts* o, const double* target, int kind,
                                          double* F_out, double* grad_pulse, double* grad_ham, int ckpt);
// lindblad.cu: the doubled (ket/bra) system of the vectorised master equation, its
// conjugate-transposed copy (adjoint rows), and the channel fidelity and its co-state
sg_status lindblad_doubled(const sg_system* sys, double T, sg_system& out);
void lindblad_adjoint_rows(const sg_system& dsys, sg_system& out);
void launch_open_fidelity(const double2* psi, const long long* comp, const double2* Tg, long long D, int Dc,
                          double* F, cudaStream_t st);
void launch_open_costate(const long long* comp, const double2* Tg, long long D, int Dc, int kind, double2* bar,
                         cudaStream_t st);
// the open system's modes (level counts and row strides of its D x D index)
struct OpenModes { int nq; long long D; int dims[SG_MAXQ]; long long st[SG_MAXQ]; };
void launch_open_frame_ebar(const double2* psi, const double2* bar, const long long* comp, const OpenModes& om, int Dc,
                            double T, double* ebar_d, cudaStream_t st);
void launch_open_fold(int nq, const double2* opbar_d, const double* ebar_d, double2* opbar, double* ebar,
                      cudaStream_t st);
sg_status sg_evolve_batch_impl(sg_system* const* systems, int B, const sg_evolve_opts* o, void* psi_dev);
// red (nullable): the column-sharded solve's all-reduce (sg_fidelity_grad_sharded).
sg_status sg_fidelity_impl(sg_system* sys, const sg_evolve_opts* o, const double* target,
                           int kind, double* F_out, double* Ucomp_out, bool grad,
                           double* grad_pulse, double* grad_ham, int ckpt,
                           sg_allreduce_fn red = nullptr, void* red_user = nullptr);

// Dressed computational states (the eigenbasis of the idle Hamiltonian, App. C): the
// D x D idle Hamiltonian is built in global scratch and diagonalised by the parallel
// (round-robin) Jacobi solver, in one block for D <= kMaxDressed and over the whole GPU
// for D <= kMaxDressedLarge (one launch per round, convergence read by the host after
// every sweep); every computational label (Dc <= kMaxDressed) takes the eigenvector of
// largest overlap on its bare state, signed so that this overlap is positive.
constexpr int kMaxDressed = 256;
constexpr int kMaxDressedLarge = 1024;
constexpr int kJacMassBlocks = 152;
struct DressArgs {
  int D, nq, ne, Dc;
  int dims[SG_MAXQ];
  long long st[SG_MAXQ];
  int eoff[SG_MAXQ], opd_off[SG_MAXQ];
  int e_a[SG_MAXEDGE], e_b[SG_MAXEDGE], e_opa[SG_MAXEDGE], e_opb[SG_MAXEDGE];
  double J[SG_MAXEDGE];
  const double* E;              // flat level energies (lab frame, E_k - E_0)
  const double2* opd;           // flat truncated operators
  const long long* comp;        // Dc flat rows of the bare computational states
  double2* Vc;                  // out: D x Dc (row-major)
  double* work;                 // scratch of dressed_work_doubles(D) doubles
  int* err;                     // out: 0, 1 complex idle Hamiltonian, 2 shared dressed
                                // state, 3 degenerate dressed level
};
// Runs the dressed-state solve on stream st: one launch for D <= kMaxDressed (no
// synchronisation), else the launches of the GPU-wide Jacobi with one stream
// synchronisation per sweep.  launches (nullable): incremented by the launch count.
cudaError_t launch_dressed(const DressArgs& a, cudaStream_t st, int* launches);
size_t dressed_work_doubles(int D);
