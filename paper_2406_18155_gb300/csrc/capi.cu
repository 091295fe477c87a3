// C ABI: argument checking, system bookkeeping and dispatch.  See include/sg.h.
#include "sg_internal.h"
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

static thread_local std::string g_create_error;

sg_status sg_fail(sg_ctx* ctx, sg_status code, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  else g_create_error = msg;
  return code;
}

static bool isfin(double x) { return std::isfinite(x); }

extern "C" {

const char* sg_version(void) { return "supergpu 0.1 (sm_103a)"; }

sg_status sg_ctx_create(sg_ctx** out, int device, void* cuda_stream) {
  if (!out) return sg_fail(nullptr, SG_E_INVALID, "out is NULL");
  *out = nullptr;
  // one hardware work queue per concurrent stream (the server's slots); honoured only
  // when this call creates the process's CUDA context, and a value already set is kept
  setenv("CUDA_DEVICE_MAX_CONNECTIONS", "32", 0);
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) return sg_fail(nullptr, SG_E_CUDA, std::string("cudaGetDeviceCount: ") + cudaGetErrorString(e));
  if (device < 0 || device >= n) return sg_fail(nullptr, SG_E_INVALID, "device index out of range");
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return sg_fail(nullptr, SG_E_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  sg_ctx* c = new (std::nothrow) sg_ctx();
  if (!c) return sg_fail(nullptr, SG_E_NOMEM, "out of host memory");
  c->device = device;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  *out = c;
  return SG_OK;
}

sg_status sg_ctx_destroy(sg_ctx* ctx) {
  delete ctx;
  return SG_OK;
}

const char* sg_last_error(const sg_ctx* ctx) {
  return ctx ? ctx->last_error.c_str() : g_create_error.c_str();
}

sg_status sg_system_create(sg_ctx* ctx, sg_system** out) {
  if (!ctx || !out) return sg_fail(ctx, SG_E_INVALID, "null argument");
  sg_system* s = new (std::nothrow) sg_system();
  if (!s) return sg_fail(ctx, SG_E_NOMEM, "out of host memory");
  s->ctx = ctx;
  *out = s;
  return SG_OK;
}

sg_status sg_system_destroy(sg_system* sys) {
  if (!sys) return SG_OK;
  if (sys->mode_block) cudaFree(sys->mode_block);
  if (sys->mdev_dev) cudaFree(sys->mdev_dev);
  delete sys;
  return SG_OK;
}

sg_status sg_add_transmon(sg_system* sys, double ej, double ec, double ng, int ncut, int levels,
                          int* mode_out) {
  if (!sys) return SG_E_INVALID;
  if (!isfin(ej) || !isfin(ec) || !isfin(ng) || ec <= 0.0)
    return sg_fail(sys->ctx, SG_E_INVALID, "transmon parameters must be finite, E_C > 0");
  const int M = 2 * ncut + 1;
  if (ncut < 1 || M > SG_MAXM) return sg_fail(sys->ctx, SG_E_INVALID, "ncut out of range (1..31)");
  if (levels < 2 || levels > SG_MAXD || levels > M)
    return sg_fail(sys->ctx, SG_E_INVALID, "levels out of range (2..8)");
  if ((int)sys->modes.size() >= SG_MAXQ) return sg_fail(sys->ctx, SG_E_UNSUPPORTED, "too many modes");
  HostMode m{};
  m.kind = 0; m.ej = ej; m.ec = ec; m.el = 0.0; m.ng = ng; m.phi_ext = 0.0; m.M = M; m.d = levels;
  sys->modes.push_back(m);
  sys->prepared = false;
  if (mode_out) *mode_out = (int)sys->modes.size() - 1;
  return SG_OK;
}

sg_status sg_add_fluxonium(sg_system* sys, double ej, double ec, double el, double phi_ext, int n_osc,
                           int levels, int* mode_out) {
  if (!sys) return SG_E_INVALID;
  if (!isfin(ej) || !isfin(ec) || !isfin(el) || !isfin(phi_ext) || ec <= 0.0 || el <= 0.0)
    return sg_fail(sys->ctx, SG_E_INVALID, "fluxonium parameters must be finite, E_C, E_L > 0");
  if (n_osc < 2 || n_osc > SG_MAXM) return sg_fail(sys->ctx, SG_E_INVALID, "n_osc out of range (2..64)");
  if (levels < 2 || levels > SG_MAXD || levels > n_osc)
    return sg_fail(sys->ctx, SG_E_INVALID, "levels out of range (2..8)");
  if ((int)sys->modes.size() >= SG_MAXQ) return sg_fail(sys->ctx, SG_E_UNSUPPORTED, "too many modes");
  HostMode m{};
  m.kind = 1; m.ej = ej; m.ec = ec; m.el = el; m.ng = 0.0; m.phi_ext = phi_ext; m.M = n_osc; m.d = levels;
  sys->modes.push_back(m);
  sys->prepared = false;
  if (mode_out) *mode_out = (int)sys->modes.size() - 1;
  return SG_OK;
}

static bool op_ok(const sg_system* sys, int mode, int op) {
  if (mode < 0 || mode >= (int)sys->modes.size()) return false;
  const HostMode& m = sys->modes[mode];
  if (op >= 2) return (size_t)(op - 2) < m.local.size() / (2 * (size_t)m.d * m.d);
  if (op != SG_OP_N && op != SG_OP_PHI) return false;
  if (op == SG_OP_PHI && m.kind == 0) return false;
  return true;
}

sg_status sg_add_local_op(sg_system* sys, int mode, const double* re_im, int* op_out) {
  if (!sys) return SG_E_INVALID;
  if (mode < 0 || mode >= (int)sys->modes.size()) return sg_fail(sys->ctx, SG_E_INVALID, "mode index out of range");
  if (!re_im) return sg_fail(sys->ctx, SG_E_INVALID, "operator is NULL");
  HostMode& m = sys->modes[mode];
  const int d = m.d;
  const int nloc = (int)(m.local.size() / (2 * (size_t)d * d));
  if (nloc >= SG_MAXOP - 2) return sg_fail(sys->ctx, SG_E_UNSUPPORTED, "at most 6 local operators per mode");
  double mx = 0.0, herm = 0.0;
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) {
      const double xr = re_im[2 * (a * d + b)], xi = re_im[2 * (a * d + b) + 1];
      const double yr = re_im[2 * (b * d + a)], yi = re_im[2 * (b * d + a) + 1];
      if (!isfin(xr) || !isfin(xi)) return sg_fail(sys->ctx, SG_E_INVALID, "operator entries must be finite");
      mx = std::max(mx, std::hypot(xr, xi));
      herm = std::max(herm, std::hypot(xr - yr, xi + yi));
    }
  if (herm > 1e-12 * mx) return sg_fail(sys->ctx, SG_E_INVALID, "local operator must be Hermitian");
  m.local.insert(m.local.end(), re_im, re_im + 2 * d * d);
  sys->prepared = false;
  if (op_out) *op_out = 2 + nloc;
  return SG_OK;
}

sg_status sg_add_collapse(sg_system* sys, int mode, const double* L_re_im, double rate, int* id_out) {
  if (!sys) return SG_E_INVALID;
  if (mode < 0 || mode >= (int)sys->modes.size()) return sg_fail(sys->ctx, SG_E_INVALID, "mode index out of range");
  if (!L_re_im) return sg_fail(sys->ctx, SG_E_INVALID, "collapse operator is NULL");
  if (!isfin(rate) || rate < 0.0) return sg_fail(sys->ctx, SG_E_INVALID, "collapse rate must be finite and >= 0");
  const int d = sys->modes[mode].d;
  for (int k = 0; k < 2 * d * d; ++k)
    if (!isfin(L_re_im[k])) return sg_fail(sys->ctx, SG_E_INVALID, "collapse operator entries must be finite");
  if (sys->collapses.size() >= 16) return sg_fail(sys->ctx, SG_E_UNSUPPORTED, "at most 16 collapse operators");
  sys->collapses.push_back(HostCollapse{mode, std::vector<double>(L_re_im, L_re_im + 2 * d * d), rate});
  if (id_out) *id_out = (int)sys->collapses.size() - 1;
  return SG_OK;
}

sg_status sg_evolve_open(sg_system* sys, const sg_evolve_opts* opts, const double* rho0_re_im, double* rho_out_re_im) {
  if (!sys) return SG_E_INVALID;
  std::lock_guard<std::mutex> lk(sys->ctx->mu);
  return sg_evolve_open_impl(sys, opts, rho0_re_im, rho_out_re_im);
}

sg_status sg_gate_fidelity_open(sg_system* sys, const sg_evolve_opts* opts, const double* target_re_im, double* F_out) {
  if (!sys) return SG_E_INVALID;
  std::lock_guard<std::mutex> lk(sys->ctx->mu);
  return sg_gate_fidelity_open_impl(sys, opts, target_re_im, F_out);
}

sg_status sg_gate_fidelity_open_grad(sg_system* sys, const sg_evolve_opts* opts, const double* target_re_im,
                                     int kind, double* F_out, double* grad_pulse, double* grad_ham, int ckpt) {
  if (!sys) return SG_E_INVALID;
  std::lock_guard<std::mutex> lk(sys->ctx->mu);
  return sg_gate_fidelity_open_grad_impl(sys, opts, target_re_im, kind, F_out, grad_pulse, grad_ham, ckpt);
}

sg_status sg_add_coupling(sg_system* sys, int mode_a, int op_a, int mode_b, int op_b, double strength,
                          int* term_out) {
  if (!sys) return SG_E_INVALID;
  if (!op_ok(sys, mode_a, op_a) || !op_ok(sys, mode_b, op_b) || mode_a == mode_b)
    return sg_fail(sys->ctx, SG_E_INVALID, "coupling needs two distinct modes and valid operators");
  if (!isfin(strength)) return sg_fail(sys->ctx, SG_E_INVALID, "coupling strength must be finite");
  if ((int)sys->couplings.size() >= SG_MAXEDGE) return sg_fail(sys->ctx, SG_E_UNSUPPORTED, "too many couplings");
  sys->couplings.push_back(HostCoupling{mode_a, op_a, mode_b, op_b, strength});
  if (term_out) *term_out = (int)sys->couplings.size() - 1;
  return SG_OK;
}

sg_status sg_set_coupler(sg_system* sys, int mode, int coupler) {
  if (!sys) return SG_E_INVALID;
  if (mode < 0 || mode >= (int)sys->modes.size()) return sg_fail(sys->ctx, SG_E_INVALID, "mode index out of range");
  sys->modes[mode].coupler = coupler ? 1 : 0;
  return SG_OK;
}

sg_status sg_add_drive(sg_system* sys, int mode, int op, const sg_pulse* p, int* drive_out) {
  if (!sys) return SG_E_INVALID;
  if (!p) return sg_fail(sys->ctx, SG_E_INVALID, "pulse is NULL");
  if (!op_ok(sys, mode, op)) return sg_fail(sys->ctx, SG_E_INVALID, "bad drive mode or operator");
  if ((int)sys->drives.size() >= SG_MAXDRIVE) return sg_fail(sys->ctx, SG_E_UNSUPPORTED, "too many drives");
  HostDrive d{};
  d.mode = mode; d.op = op; d.kind = p->kind;
  d.amp = p->amp; d.sigma = p->sigma; d.t0 = p->t0; d.length = p->length;
  d.omega_d = p->omega_d; d.omega_mode = p->omega_mode; d.phase = p->phase;
  if (p->kind == SG_ENV_PWC) {
    if (p->nseg < 1 || p->nseg > 1024 || !p->amps)
      return sg_fail(sys->ctx, SG_E_INVALID, "PWC pulse needs 1..1024 amplitudes");
    d.nseg = p->nseg;
    d.amps.assign(p->amps, p->amps + p->nseg);
    for (double a : d.amps) if (!isfin(a)) return sg_fail(sys->ctx, SG_E_INVALID, "non-finite amplitude");
  } else if (p->kind == SG_ENV_GAUSSIAN || p->kind == SG_ENV_COSINE) {
    d.nseg = 1;
    if (!isfin(p->amp)) return sg_fail(sys->ctx, SG_E_INVALID, "non-finite amplitude");
    if (p->kind == SG_ENV_GAUSSIAN && !(p->sigma > 0.0)) return sg_fail(sys->ctx, SG_E_INVALID, "sigma must be > 0");
  } else {
    return sg_fail(sys->ctx, SG_E_INVALID, "unknown envelope kind");
  }
  if (!(p->length > 0.0) || !isfin(p->length)) return sg_fail(sys->ctx, SG_E_INVALID, "length must be > 0");
  if (p->omega_mode >= (int)sys->modes.size() || p->omega_mode < -1)
    return sg_fail(sys->ctx, SG_E_INVALID, "omega_mode out of range");
  if (p->omega_mode < 0 && !isfin(p->omega_d)) return sg_fail(sys->ctx, SG_E_INVALID, "omega_d must be finite");
  if (!isfin(p->phase) || !isfin(p->t0)) return sg_fail(sys->ctx, SG_E_INVALID, "non-finite pulse field");
  sys->drives.push_back(d);
  if (drive_out) *drive_out = (int)sys->drives.size() - 1;
  return SG_OK;
}

sg_status sg_param_counts(const sg_system* sys, int* n_pulse, int* n_ham) {
  if (!sys) return SG_E_INVALID;
  int np = 0;
  for (const HostDrive& d : sys->drives) np += d.kind == SG_ENV_PWC ? d.nseg : 1;
  if (n_pulse) *n_pulse = np;
  if (n_ham) *n_ham = 3 * (int)sys->modes.size() + (int)sys->couplings.size();
  return SG_OK;
}

sg_status sg_get_params(const sg_system* sys, double* pulse, double* ham) {
  if (!sys) return SG_E_INVALID;
  if (pulse) {
    int i = 0;
    for (const HostDrive& d : sys->drives) {
      if (d.kind == SG_ENV_PWC) for (double a : d.amps) pulse[i++] = a;
      else pulse[i++] = d.amp;
    }
  }
  if (ham) {
    int i = 0;
    for (const HostMode& m : sys->modes) { ham[i++] = m.ej; ham[i++] = m.ec; ham[i++] = m.kind == 0 ? 0.0 : m.el; }
    for (const HostCoupling& c : sys->couplings) ham[i++] = c.J;
  }
  return SG_OK;
}

sg_status sg_set_params(sg_system* sys, const double* pulse, const double* ham) {
  if (!sys) return SG_E_INVALID;
  if (pulse) {
    int i = 0;
    for (HostDrive& d : sys->drives) {
      if (d.kind == SG_ENV_PWC) for (double& a : d.amps) { if (!isfin(pulse[i])) return sg_fail(sys->ctx, SG_E_INVALID, "non-finite pulse parameter"); a = pulse[i++]; }
      else { if (!isfin(pulse[i])) return sg_fail(sys->ctx, SG_E_INVALID, "non-finite pulse parameter"); d.amp = pulse[i++]; }
    }
  }
  if (ham) {
    int i = 0;
    for (HostMode& m : sys->modes) {
      double ej = ham[i], ec = ham[i + 1], el = ham[i + 2];
      if (!isfin(ej) || !isfin(ec) || ec <= 0.0 || (m.kind == 1 && !(el > 0.0)))
        return sg_fail(sys->ctx, SG_E_INVALID, "bad device parameter");
      if (ej != m.ej || ec != m.ec || (m.kind == 1 && el != m.el)) sys->prepared = false;
      m.ej = ej; m.ec = ec; if (m.kind == 1) m.el = el;
      i += 3;
    }
    for (HostCoupling& c : sys->couplings) {
      if (!isfin(ham[i])) return sg_fail(sys->ctx, SG_E_INVALID, "bad coupling");
      c.J = ham[i++];
    }
  }
  return SG_OK;
}

sg_status sg_prepare(sg_system* sys) {
  if (!sys) return SG_E_INVALID;
  std::lock_guard<std::mutex> lk(sys->ctx->mu);
  return sg_prepare_impl(sys);
}

sg_status sg_get_spectrum(const sg_system* sys, int mode, double* energies, double* n_re_im,
                          double* phi_re_im) {
  if (!sys) return SG_E_INVALID;
  if (!sys->prepared) return sg_fail(sys->ctx, SG_E_STATE, "system is not prepared");
  if (mode < 0 || mode >= (int)sys->modes.size()) return sg_fail(sys->ctx, SG_E_INVALID, "mode out of range");
  const int d = sys->modes[mode].d;
  if (energies) std::memcpy(energies, sys->E_host[mode].data(), d * sizeof(double));
  if (n_re_im) std::memcpy(n_re_im, sys->opd_host[mode].data(), 2 * d * d * sizeof(double));
  if (phi_re_im) std::memcpy(phi_re_im, sys->opd_host[mode].data() + 2 * d * d, 2 * d * d * sizeof(double));
  return SG_OK;
}

sg_status sg_dims(const sg_system* sys, long long* D, int* nmodes) {
  if (!sys) return SG_E_INVALID;
  long long p = 1;
  for (const HostMode& m : sys->modes) p *= m.d;
  if (D) *D = p;
  if (nmodes) *nmodes = (int)sys->modes.size();
  return SG_OK;
}

sg_status sg_evolve(sg_system* sys, const sg_evolve_opts* opts, void* psi_dev) {
  if (!sys) return SG_E_INVALID;
  std::lock_guard<std::mutex> lk(sys->ctx->mu);
  return sg_evolve_impl(sys, opts, psi_dev);
}

sg_status sg_fidelity(sg_system* sys, const sg_evolve_opts* opts, const double* target_re_im,
                      double* F_out, double* Ucomp_out) {
  if (!sys) return SG_E_INVALID;
  std::lock_guard<std::mutex> lk(sys->ctx->mu);
  return sg_fidelity_impl(sys, opts, target_re_im, SG_FID_AVG, F_out, Ucomp_out, false, nullptr,
                          nullptr, 0);
}

sg_status sg_fidelity_grad(sg_system* sys, const sg_evolve_opts* opts, const double* target_re_im,
                           int kind, double* F_out, double* grad_pulse, double* grad_ham,
                           int ckpt_interval) {
  if (!sys) return SG_E_INVALID;
  if (ckpt_interval < 0) return sg_fail(sys->ctx, SG_E_INVALID, "ckpt_interval must be >= 0");
  std::lock_guard<std::mutex> lk(sys->ctx->mu);
  return sg_fidelity_impl(sys, opts, target_re_im, kind, F_out, nullptr, true, grad_pulse, grad_ham,
                          ckpt_interval);
}

sg_status sg_evolve_batch(sg_system* const* systems, int nsys, const sg_evolve_opts* opts, void* psi_dev) {
  if (!systems || nsys < 1 || !systems[0]) return SG_E_INVALID;
  std::lock_guard<std::mutex> lk(systems[0]->ctx->mu);
  return sg_evolve_batch_impl(systems, nsys, opts, psi_dev);
}

sg_status sg_fidelity_grad_sharded(sg_system* sys, const sg_evolve_opts* opts, const double* target_re_im,
                                   int kind, double* F_out, double* grad_pulse, double* grad_ham,
                                   int ckpt_interval, sg_allreduce_fn allreduce, void* user) {
  if (!sys) return SG_E_INVALID;
  if (!allreduce) return sg_fail(sys->ctx, SG_E_INVALID, "a sharded solve needs the caller's all-reduce");
  if (ckpt_interval < 0) return sg_fail(sys->ctx, SG_E_INVALID, "ckpt_interval must be >= 0");
  std::lock_guard<std::mutex> lk(sys->ctx->mu);
  return sg_fidelity_impl(sys, opts, target_re_im, kind, F_out, nullptr, true, grad_pulse, grad_ham,
                          ckpt_interval, allreduce, user);
}

sg_status sg_last_stats(const sg_system* sys, double* out5) {
  if (!sys || !out5) return SG_E_INVALID;
  for (int i = 0; i < 5; ++i) out5[i] = sys->last_stats[i];
  return SG_OK;
}

sg_status sg_kernel_times(const sg_system* sys, double* out, int n) {
  if (!sys || !out || n < 9) return SG_E_INVALID;
  for (int i = 0; i < 9; ++i) out[i] = sys->ktimes[i];
  return SG_OK;
}

}  // extern "C"
