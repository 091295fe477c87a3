// Open-system evolution: the vectorised Lindblad master equation on the evolution
// kernels (the paper carries its solver and back-propagation over to the
// superoperator of the vectorised equation, App. C last paragraph; LindbladObj of
// Sec. 2.2).
//
// With row-major vec(rho) (index = ket index x D + bra index) the generator is
//     Lv = -i (H (x) I - I (x) H^T) + sum_c g_c (L (x) L^* - (L^dag L) (x) I / 2 - I (x) (L^dag L)^T / 2),
// i.e. -i H_eff on 2 nq modes (nq ket modes, then nq bra modes) with local terms:
//     ket 1-body  H_i(t) - (i/2) sum_c g_c L_c^dag L_c;   bra 1-body  -H_i(t)^T - (i/2) sum_c g_c (L_c^dag L_c)^T
//     ket 2-body  J A (x) B;   bra 2-body  -J A^T (x) B^T;   jump  i g_c L_c (ket) (x) L_c^* (bra).
// In the interaction frame every operator rotates with its mode's phases; a bra mode
// carries the ket energies negated, so (P X P^dag)^T rotates as a bra-mode operator
// and the frame epilogue exp(-i (E_ket - E_bra) T) is exp(-i H_d T) rho exp(i H_d T).
//
// So the library builds, per call, a doubled system of that form from the caller's
// prepared system (operators copied, transposed or conjugated; drives copied onto
// the bra modes with negated amplitudes; the constant non-Hermitian 1-body parts as
// drives of unit envelope) and evolves vec(rho) as columns of it with the ordinary
// RK4 kernels (complex rows: the terms are not real).
#include "sg_internal.h"
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

namespace {

typedef std::complex<double> cd;

// Operator op of mode m of a prepared system, d x d complex.
std::vector<cd> op_of(const sg_system* sys, int m, int op) {
  const int d = sys->modes[m].d;
  std::vector<cd> o((size_t)d * d);
  const std::vector<double>& od = sys->opd_host[m];
  for (int ab = 0; ab < d * d; ++ab) o[ab] = cd(od[2 * ((size_t)op * d * d + ab)], od[2 * ((size_t)op * d * d + ab) + 1]);
  return o;
}
std::vector<cd> transpose(const std::vector<cd>& a, int d, bool conj_too) {
  std::vector<cd> t(a.size());
  for (int x = 0; x < d; ++x)
    for (int y = 0; y < d; ++y) t[(size_t)y * d + x] = conj_too ? std::conj(a[(size_t)x * d + y]) : a[(size_t)x * d + y];
  return t;
}
void append_op(std::vector<double>& od, const std::vector<cd>& o) {
  for (const cd& v : o) { od.push_back(v.real()); od.push_back(v.imag()); }
}

}  // namespace

// The doubled system of sys for an evolution of length T (the unit envelopes of the
// constant terms span [0, T)).  Modes 0..nq-1 ket, nq..2nq-1 bra.
sg_status lindblad_doubled(const sg_system* sys, double T, sg_system& out) {
  sg_ctx* ctx = sys->ctx;
  const int nq = (int)sys->modes.size();
  if (2 * nq > SG_MAXQ) return sg_fail(ctx, SG_E_UNSUPPORTED, "the open evolution doubles the modes: at most 8 modes");
  out = sg_system{};
  out.ctx = sys->ctx;
  out.modes.resize(2 * nq);
  out.opd_host.resize(2 * nq);
  out.E_host.resize(2 * nq);
  out.parity_odd.assign((size_t)2 * nq * SG_MAXOP, 0);
  std::vector<int> nop(nq), anti_op(nq, -1), jump_ket(sys->collapses.size()), jump_bra(sys->collapses.size());
  for (int m = 0; m < nq; ++m) {
    const HostMode& hm = sys->modes[m];
    const int d = hm.d;
    nop[m] = (int)(sys->opd_host[m].size() / (2 * (size_t)d * d));
    out.modes[m] = hm;
    out.modes[m].coupler = 0;
    out.modes[m].local.clear();
    out.modes[nq + m] = out.modes[m];
    out.E_host[m] = sys->E_host[m];
    out.E_host[nq + m] = sys->E_host[m];
    for (double& e : out.E_host[nq + m]) e = -e;
    // operators: the originals (ket) and their transposes (bra), indices unchanged
    for (int op = 0; op < nop[m]; ++op) {
      const std::vector<cd> o = op_of(sys, m, op);
      append_op(out.opd_host[m], o);
      append_op(out.opd_host[nq + m], transpose(o, d, false));
    }
    // -(i/2) sum_c g_c L_c^dag L_c on the ket mode, its transpose on the bra mode
    std::vector<cd> anti((size_t)d * d, cd(0.0, 0.0));
    bool any = false;
    for (const HostCollapse& c : sys->collapses) {
      if (c.mode != m) continue;
      any = true;
      for (int x = 0; x < d; ++x)
        for (int y = 0; y < d; ++y) {
          cd acc(0.0, 0.0);
          for (int z = 0; z < d; ++z)
            acc += std::conj(cd(c.L[2 * (z * d + x)], c.L[2 * (z * d + x) + 1])) * cd(c.L[2 * (z * d + y)], c.L[2 * (z * d + y) + 1]);
          anti[(size_t)x * d + y] += cd(0.0, -0.5 * c.rate) * acc;
        }
    }
    if (any) {
      anti_op[m] = nop[m];
      append_op(out.opd_host[m], anti);
      append_op(out.opd_host[nq + m], transpose(anti, d, false));
    }
  }
  // jump terms: i g L on the ket mode, L^* on the bra mode
  for (size_t k = 0; k < sys->collapses.size(); ++k) {
    const HostCollapse& c = sys->collapses[k];
    const int m = c.mode, d = sys->modes[m].d;
    std::vector<cd> L((size_t)d * d), Lk((size_t)d * d), Lb((size_t)d * d);
    for (int ab = 0; ab < d * d; ++ab) L[ab] = cd(c.L[2 * ab], c.L[2 * ab + 1]);
    for (int ab = 0; ab < d * d; ++ab) { Lk[ab] = cd(0.0, c.rate) * L[ab]; Lb[ab] = std::conj(L[ab]); }
    jump_ket[k] = (int)(out.opd_host[m].size() / (2 * (size_t)d * d));
    append_op(out.opd_host[m], Lk);
    jump_bra[k] = (int)(out.opd_host[nq + m].size() / (2 * (size_t)d * d));
    append_op(out.opd_host[nq + m], Lb);
  }
  for (int m = 0; m < 2 * nq; ++m) {
    const int d = out.modes[m].d;
    if (out.opd_host[m].size() / (2 * (size_t)d * d) > SG_MAXOP)
      return sg_fail(ctx, SG_E_UNSUPPORTED, "too many operators on a mode of the open evolution");
  }
  // drives: the ket copy and the bra copy with negated amplitudes (-H^T); a carrier tied
  // to a mode's 0-1 frequency stays tied to that (ket) mode in both copies
  for (const HostDrive& hd : sys->drives) {
    HostDrive k = hd;
    out.drives.push_back(k);
    HostDrive b = k;
    b.mode = nq + hd.mode;
    b.amp = -hd.amp;
    for (double& a : b.amps) a = -a;
    out.drives.push_back(b);
  }
  // constant non-Hermitian 1-body parts: unit envelope over [0, T), no carrier
  for (int m = 0; m < nq; ++m) {
    if (anti_op[m] < 0) continue;
    HostDrive c{};
    c.kind = SG_ENV_PWC; c.nseg = 1; c.amps = {1.0}; c.amp = 0.0; c.sigma = 1.0; c.t0 = 0.0; c.length = T;
    c.omega_d = 0.0; c.phase = 0.0; c.omega_mode = -1;
    c.mode = m; c.op = anti_op[m];
    out.drives.push_back(c);
    c.mode = nq + m;
    out.drives.push_back(c);
  }
  // couplings: ket-ket J A (x) B, bra-bra -J A^T (x) B^T, jumps i g L (x) L^*
  for (const HostCoupling& c : sys->couplings) {
    out.couplings.push_back(c);
    out.couplings.push_back(HostCoupling{nq + c.a, c.op_a, nq + c.b, c.op_b, -c.J});
  }
  for (size_t k = 0; k < sys->collapses.size(); ++k) {
    const HostCollapse& c = sys->collapses[k];
    out.couplings.push_back(HostCoupling{c.mode, jump_ket[k], nq + c.mode, jump_bra[k], 1.0});
  }
  if ((int)out.couplings.size() > SG_MAXEDGE) return sg_fail(ctx, SG_E_UNSUPPORTED, "too many terms in the open evolution");
  out.prepared = true;
  return SG_OK;
}

// The doubled system with every operator replaced by its conjugate transpose (drives
// and couplings unchanged, their coefficients real): its stage rows are those of
// H_eff^dag, so the adjoint passes, which apply i H to the co-state, apply
// A^dag = i H_eff^dag for the forward generator A = -i H_eff (the discrete adjoint of
// a non-Hermitian generator).
void lindblad_adjoint_rows(const sg_system& dsys, sg_system& out) {
  out = dsys;
  for (size_t m = 0; m < out.modes.size(); ++m) {
    const int d = out.modes[m].d;
    std::vector<double>& od = out.opd_host[m];
    const size_t nop = od.size() / (2 * (size_t)d * d);
    for (size_t op = 0; op < nop; ++op) {
      double* o = od.data() + 2 * op * d * d;
      std::vector<double> t(2 * (size_t)d * d);
      for (int x = 0; x < d; ++x)
        for (int y = 0; y < d; ++y) {
          t[2 * ((size_t)y * d + x)] = o[2 * ((size_t)x * d + y)];
          t[2 * ((size_t)y * d + x) + 1] = -o[2 * ((size_t)x * d + y) + 1];
        }
      std::copy(t.begin(), t.end(), o);
    }
  }
}

namespace {

// Channel on the computational block from the evolved columns |c_j><c_k| (lab frame,
// doubled index ket x D + bra, column innermost), and its average gate fidelity
// against T: S[(a, b), (j, k)] = rho_jk[c_a][c_b]; F_pro = Re sum conj(S_T) S / D_c^2
// with S_T = T (x) T^*; kept = sum_{a, j} Re S[(a, a), (j, j)];
// F_avg = (D_c^2 F_pro + kept) / (D_c (D_c + 1)).  One block, fixed-order sums.
__global__ void k_open_fidelity(const double2* __restrict__ psi, const long long* __restrict__ comp,
                                const double2* __restrict__ Tg, long long D, int Dc, double* F) {
  __shared__ double red[256];
  const int S = Dc * Dc;
  double fp = 0.0, kept = 0.0;
  for (int x = threadIdx.x; x < S * S; x += blockDim.x) {
    const int ab = x / S, jk = x - (x / S) * S;
    const int a = ab / Dc, b = ab - a * Dc, j = jk / Dc, k = jk - j * Dc;
    const double2 s = psi[(comp[a] * D + comp[b]) * S + jk];
    const double2 ta = Tg[a * Dc + j], tb = Tg[b * Dc + k];
    // S_T = T[a][j] conj(T[b][k]); Re(conj(S_T) s)
    const double str = ta.x * tb.x + ta.y * tb.y, sti = ta.y * tb.x - ta.x * tb.y;
    fp += str * s.x + sti * s.y;
    if (a == b && j == k) kept += s.x;
  }
  red[threadIdx.x] = fp;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double Fp = red[0] / ((double)Dc * Dc);
  __syncthreads();
  red[threadIdx.x] = kept;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    F[1] = Fp;
    F[0] = ((double)Dc * Dc * Fp + red[0]) / ((double)Dc * (Dc + 1.0));
  }
}

// Co-state of the open gate fidelity on the evolved columns (lab frame, layout of
// k_open_fidelity; the caller zeroes the rest): F is linear in S, F = Re sum conj(W) S,
// so the co-state (d F / d Re s + i d F / d Im s) of entry (c_a, c_b) of column (j, k)
// is W[(a, b), (j, k)]: S_T / (Dc (Dc + 1)) plus 1 / (Dc (Dc + 1)) where a = b, j = k
// for F_avg (kind SG_FID_AVG), S_T / Dc^2 for F_pro (kind SG_FID_STATE).
__global__ void k_open_costate(const long long* __restrict__ comp, const double2* __restrict__ Tg, long long D,
                               int Dc, int kind, double2* __restrict__ bar) {
  const int S = Dc * Dc;
  const double sc = kind == SG_FID_AVG ? 1.0 / ((double)Dc * (Dc + 1.0)) : 1.0 / ((double)Dc * Dc);
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < S * S; x += gridDim.x * blockDim.x) {
    const int ab = x / S, jk = x - (x / S) * S;
    const int a = ab / Dc, b = ab - a * Dc, j = jk / Dc, k = jk - j * Dc;
    const double2 ta = Tg[a * Dc + j], tb = Tg[b * Dc + k];
    double re = ta.x * tb.x + ta.y * tb.y, im = ta.y * tb.x - ta.x * tb.y;
    if (kind == SG_FID_AVG && a == b && j == k) re += 1.0;
    bar[(comp[a] * D + comp[b]) * S + jk] = make_double2(sc * re, sc * im);
  }
}

}  // namespace

void launch_open_fidelity(const double2* psi, const long long* comp, const double2* Tg, long long D, int Dc,
                          double* F, cudaStream_t st) {
  k_open_fidelity<<<1, 256, 0, st>>>(psi, comp, Tg, D, Dc, F);
}

void launch_open_costate(const long long* comp, const double2* Tg, long long D, int Dc, int kind, double2* bar,
                         cudaStream_t st) {
  const int n = Dc * Dc * Dc * Dc;
  k_open_costate<<<(n + 255) / 256, 256, 0, st>>>(comp, Tg, D, Dc, kind, bar);
}

namespace {

// Energy cotangent of the lab-frame epilogue exp(-i E_tot T) of the doubled columns:
// dF/dE_dm[l] = T sum Re(conj(bar) (-i) psi) over the entries whose doubled mode dm
// (ket modes 0..nq-1, then bra modes) sits in level l; the co-state is non-zero on the
// computational block only (rows comp[a] D + comp[b]).  One block per doubled mode.
__global__ void k_open_frame_ebar(const double2* __restrict__ psi, const double2* __restrict__ bar,
                                  const long long* __restrict__ comp, OpenModes om, int Dc, double T,
                                  double* __restrict__ ebar) {
  __shared__ double red[256][SG_MAXD];
  const int dm = blockIdx.x, m = dm % om.nq;
  const bool bra = dm >= om.nq;
  const int S = Dc * Dc;
  double part[SG_MAXD];
  for (int l = 0; l < SG_MAXD; ++l) part[l] = 0.0;
  for (int x = threadIdx.x; x < S * S; x += blockDim.x) {
    const int ab = x / S, jk = x - (x / S) * S;
    const int a = ab / Dc, b = ab - a * Dc;
    const long long r = comp[a] * om.D + comp[b];
    const int lev = (int)(((bra ? comp[b] : comp[a]) / om.st[m]) % om.dims[m]);
    const double2 bv = bar[r * S + jk], u = psi[r * S + jk];
    part[lev] += T * (bv.x * u.y - bv.y * u.x);
  }
  for (int l = 0; l < SG_MAXD; ++l) red[threadIdx.x][l] = part[l];
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int l = 0; l < SG_MAXD; ++l) red[threadIdx.x][l] += red[threadIdx.x + o][l];
    __syncthreads();
  }
  if (threadIdx.x < SG_MAXD) ebar[dm * SG_MAXD + threadIdx.x] += red[0][threadIdx.x];
}

// Co-gradients of the doubled modes folded onto the open system's modes: a bra mode
// carries the operators transposed and the energies negated, so
//   opbar[m][op] = opbar_d[m][op] + opbar_d[nq + m][op]^T,  ebar[m] = ebar_d[m] - ebar_d[nq + m].
__global__ void k_open_fold(int nq, const double2* __restrict__ opbar_d, const double* __restrict__ ebar_d,
                            double2* __restrict__ opbar, double* __restrict__ ebar) {
  const int MD2 = SG_MAXD * SG_MAXD;
  for (int x = threadIdx.x; x < nq * 2 * MD2; x += blockDim.x) {
    const int mo = x / MD2, ab = x - mo * MD2, a = ab / SG_MAXD, b = ab - a * SG_MAXD;
    const double2 k = opbar_d[x], br = opbar_d[(size_t)nq * 2 * MD2 + mo * MD2 + b * SG_MAXD + a];
    opbar[x] = make_double2(k.x + br.x, k.y + br.y);
  }
  for (int x = threadIdx.x; x < nq * SG_MAXD; x += blockDim.x) ebar[x] = ebar_d[x] - ebar_d[nq * SG_MAXD + x];
}

}  // namespace

void launch_open_frame_ebar(const double2* psi, const double2* bar, const long long* comp, const OpenModes& om, int Dc,
                            double T, double* ebar_d, cudaStream_t st) {
  k_open_frame_ebar<<<2 * om.nq, 256, 0, st>>>(psi, bar, comp, om, Dc, T, ebar_d);
}

void launch_open_fold(int nq, const double2* opbar_d, const double* ebar_d, double2* opbar, double* ebar,
                      cudaStream_t st) {
  k_open_fold<<<1, 256, 0, st>>>(nq, opbar_d, ebar_d, opbar, ebar);
}

sg_status sg_evolve_open_impl(sg_system* sys, const sg_evolve_opts* o, const double* rho0, double* rho_out) {
  sg_ctx* ctx = sys->ctx;
  if (!sys->prepared) return sg_fail(ctx, SG_E_STATE, "system is not prepared (call sg_prepare)");
  if (!o || !rho0 || !rho_out) return sg_fail(ctx, SG_E_INVALID, "open evolution needs opts, rho0 and rho_out");
  sg_system dsys;
  sg_status rc = lindblad_doubled(sys, o->T, dsys);
  if (rc != SG_OK) return rc;
  long long D = 1;
  for (const HostMode& m : sys->modes) D *= m.d;
  const size_t n = (size_t)D * D;
  cudaStream_t st = ctx->stream;
  SG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  double2* v = nullptr;
  SG_CUDA_TRY(ctx, cudaMallocAsync(&v, n * sizeof(double2), st));
  cudaMemcpyAsync(v, rho0, n * sizeof(double2), cudaMemcpyHostToDevice, st);
  sg_evolve_opts od = *o;
  od.ncols = 1;
  od.col_index = nullptr;
  od.compensation = SG_COMP_NONE;
  od.basis = SG_BASIS_PRODUCT;
  rc = sg_evolve_impl(&dsys, &od, v);
  if (rc == SG_OK) {
    cudaMemcpyAsync(rho_out, v, n * sizeof(double2), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = sg_fail(ctx, SG_E_CUDA, "copy of the density matrix failed");
  }
  cudaFreeAsync(v, st);
  for (int k = 0; k < 9; ++k) sys->ktimes[k] = dsys.ktimes[k];
  return rc;
}

sg_status sg_gate_fidelity_open_impl(sg_system* sys, const sg_evolve_opts* o, const double* target, double* F_out) {
  sg_ctx* ctx = sys->ctx;
  if (!sys->prepared) return sg_fail(ctx, SG_E_STATE, "system is not prepared (call sg_prepare)");
  if (!o || !target || !F_out) return sg_fail(ctx, SG_E_INVALID, "open gate fidelity needs opts, target and F_out");
  const int nq = (int)sys->modes.size();
  int nqb = 0;
  for (const HostMode& m : sys->modes) nqb += m.coupler ? 0 : 1;
  if (nqb < 1 || nqb > 6) return sg_fail(ctx, SG_E_UNSUPPORTED, "the open gate fidelity takes 1..6 qubit modes");
  const int Dc = 1 << nqb;
  long long D = 1;
  std::vector<long long> st(nq);
  for (int i = nq - 1; i >= 0; --i) { st[i] = D; D *= sys->modes[i].d; }
  std::vector<long long> comp(Dc), cols((size_t)Dc * Dc);
  for (int j = 0; j < Dc; ++j) {
    long long r = 0;
    for (int i = 0, b = nqb - 1; i < nq; ++i) r += (long long)(sys->modes[i].coupler ? 0 : (j >> b--) & 1) * st[i];
    comp[j] = r;
  }
  for (int j = 0; j < Dc; ++j)
    for (int k = 0; k < Dc; ++k) cols[(size_t)j * Dc + k] = comp[j] * D + comp[k];
  sg_system dsys;
  sg_status rc = lindblad_doubled(sys, o->T, dsys);
  if (rc != SG_OK) return rc;
  cudaStream_t sm = ctx->stream;
  SG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const size_t S = (size_t)Dc * Dc;
  double2 *psi = nullptr, *Tg = nullptr;
  long long* comp_dev = nullptr;
  double* F = nullptr;
  if (cudaMallocAsync(&psi, (size_t)D * D * S * sizeof(double2), sm) != cudaSuccess ||
      cudaMallocAsync(&Tg, (size_t)Dc * Dc * sizeof(double2), sm) != cudaSuccess ||
      cudaMallocAsync(&comp_dev, Dc * sizeof(long long), sm) != cudaSuccess ||
      cudaMallocAsync(&F, 2 * sizeof(double), sm) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeAsync(psi, sm); cudaFreeAsync(Tg, sm); cudaFreeAsync(comp_dev, sm); cudaFreeAsync(F, sm);
    return sg_fail(ctx, SG_E_NOMEM, "device allocation failed");
  }
  cudaMemcpyAsync(Tg, target, (size_t)Dc * Dc * sizeof(double2), cudaMemcpyHostToDevice, sm);
  cudaMemcpyAsync(comp_dev, comp.data(), Dc * sizeof(long long), cudaMemcpyHostToDevice, sm);
  sg_evolve_opts od = *o;
  od.ncols = (int)S;
  od.col_index = cols.data();
  od.compensation = SG_COMP_NONE;
  od.basis = SG_BASIS_PRODUCT;
  rc = sg_evolve_impl(&dsys, &od, psi);
  if (rc == SG_OK) {
    k_open_fidelity<<<1, 256, 0, sm>>>(psi, comp_dev, Tg, D, Dc, F);
    double h[2] = {0.0, 0.0};
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(sm) != cudaSuccess ||
        cudaMemcpy(h, F, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = sg_fail(ctx, SG_E_CUDA, "open gate fidelity reduction failed");
    F_out[0] = h[0];
    F_out[1] = h[1];
  }
  cudaFreeAsync(psi, sm); cudaFreeAsync(Tg, sm); cudaFreeAsync(comp_dev, sm); cudaFreeAsync(F, sm);
  for (int k = 0; k < 9; ++k) sys->ktimes[k] = dsys.ktimes[k];
  return rc;
}
