// Subsystem build, FP64 eigensolve, truncation and projection on the GPU, and the
// eigen-derivative chain that turns operator / energy co-gradients into
// d/d(E_J, E_C, E_L).
//
// Paper: Sec. 2.1 (each qubit is diagonalised first and its low-energy basis kept),
// Eq. 8 (fluxonium), App. D step 1 (operators represented in the single-qubit
// eigenbasis).  One CTA handles one mode; M <= 64 basis states.
#include "sg_internal.h"
#include <cmath>
#include <cstdio>
#include <algorithm>

namespace {

constexpr int kThreads = 256;

// Parallel cyclic Jacobi eigensolver for a symmetric M x M matrix held in shared
// memory (row-major, leading dimension M).  On return A is diagonal (eigenvalues
// on the diagonal, unsorted) and V holds the eigenvectors in columns.  Rotations
// of one round act on disjoint index pairs (round-robin tournament ordering), so
// their row and column updates run in parallel.  Symmetric 2x2 Schur rotations.
__device__ void jacobi_eigen(double* A, double* V, int M, double* cs, int* pairs) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < M * M; i += nt) V[i] = (i / M == i % M) ? 1.0 : 0.0;
  const int Mp = (M + 1) & ~1;           // even number of players; index M is a dummy when M is odd
  const int npair = Mp / 2;
  __shared__ double red[kThreads];
  __syncthreads();
  for (int sweep = 0; sweep < 40; ++sweep) {
    // convergence test on the off-diagonal mass
    double off = 0.0, dia = 0.0;
    for (int i = tid; i < M * M; i += nt) {
      int r = i / M, c = i % M;
      if (r != c) off += A[i] * A[i]; else dia += A[i] * A[i];
    }
    red[tid] = off;
    __syncthreads();
    for (int s = nt / 2; s > 0; s >>= 1) { if (tid < s) red[tid] += red[tid + s]; __syncthreads(); }
    double off_tot = red[0];
    __syncthreads();
    red[tid] = dia;
    __syncthreads();
    for (int s = nt / 2; s > 0; s >>= 1) { if (tid < s) red[tid] += red[tid + s]; __syncthreads(); }
    double dia_tot = red[0];
    __syncthreads();
    if (off_tot <= 1e-32 * dia_tot || off_tot == 0.0) break;
    for (int round = 0; round < Mp - 1; ++round) {
      // pairing of this round (circle method): position 0 holds player 0,
      // position i >= 1 holds 1 + (i - 1 + round) mod (Mp - 1)
      for (int k = tid; k < npair; k += nt) {
        int pa = (k == 0) ? 0 : 1 + ((k - 1 + round) % (Mp - 1));
        int pos_b = Mp - 1 - k;
        int pb = 1 + ((pos_b - 1 + round) % (Mp - 1));
        int p = min(pa, pb), q = max(pa, pb);
        pairs[2 * k] = p;
        pairs[2 * k + 1] = q;
        double c = 1.0, s = 0.0;
        if (q < M) {
          double apq = A[p * M + q];
          if (apq != 0.0) {
            double app = A[p * M + p], aqq = A[q * M + q];
            double tau = (aqq - app) / (2.0 * apq);
            double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        }
        cs[2 * k] = c;
        cs[2 * k + 1] = s;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int i = tid; i < npair * M; i += nt) {
        int k = i / M, col = i % M;
        int p = pairs[2 * k], q = pairs[2 * k + 1];
        if (q >= M) continue;
        double c = cs[2 * k], s = cs[2 * k + 1];
        double ap = A[p * M + col], aq = A[q * M + col];
        A[p * M + col] = c * ap - s * aq;
        A[q * M + col] = s * ap + c * aq;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int i = tid; i < npair * M; i += nt) {
        int k = i / M, row = i % M;
        int p = pairs[2 * k], q = pairs[2 * k + 1];
        if (q >= M) continue;
        double c = cs[2 * k], s = cs[2 * k + 1];
        double ap = A[row * M + p], aq = A[row * M + q];
        A[row * M + p] = c * ap - s * aq;
        A[row * M + q] = s * ap + c * aq;
        double vp = V[row * M + p], vq = V[row * M + q];
        V[row * M + p] = c * vp - s * vq;
        V[row * M + q] = s * vp + c * vq;
      }
      __syncthreads();
      // exact zero of the annihilated pairs keeps the off-diagonal mass honest
      for (int k = tid; k < npair; k += nt) {
        int p = pairs[2 * k], q = pairs[2 * k + 1];
        if (q < M && cs[2 * k + 1] != 0.0) { A[p * M + q] = 0.0; A[q * M + p] = 0.0; }
      }
      __syncthreads();
    }
  }
}

// Sort eigenpairs ascending (stable by index) into (w_out, V_out) and fix the
// sign gauge: the first component with |v_i| >= 1e-3 max|v| is positive.
__device__ void sort_and_gauge(const double* A, const double* V, int M, double* w_out,
                               double* V_out) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int k = tid; k < M; k += nt) {
    double wk = A[k * M + k];
    int rank = 0;
    for (int j = 0; j < M; ++j) {
      double wj = A[j * M + j];
      if (wj < wk || (wj == wk && j < k)) ++rank;
    }
    w_out[rank] = wk;
    double mx = 0.0;
    for (int i = 0; i < M; ++i) mx = fmax(mx, fabs(V[i * M + k]));
    double sgn = 1.0;
    for (int i = 0; i < M; ++i) {
      double v = V[i * M + k];
      if (fabs(v) >= 1e-3 * mx) { sgn = (v < 0.0) ? -1.0 : 1.0; break; }
    }
    for (int i = 0; i < M; ++i) V_out[i * M + rank] = sgn * V[i * M + k];
  }
  __syncthreads();
}

// C = A * diag(g) * A^T for real M x M A (row-major), all in the given buffers.
__device__ void adiag_at(const double* A, const double* g, int M, double* C) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < M * M; i += nt) {
    int r = i / M, c = i % M;
    double acc = 0.0;
    for (int k = 0; k < M; ++k) acc += A[r * M + k] * g[k] * A[c * M + k];
    C[i] = acc;
  }
  __syncthreads();
}

struct BuildArgs {
  int nq;
  int kind[SG_MAXQ], M[SG_MAXQ], d[SG_MAXQ];
  double ej[SG_MAXQ], ec[SG_MAXQ], el[SG_MAXQ], ng[SG_MAXQ], phi_ext[SG_MAXQ];
  ModeDev md[SG_MAXQ];
  double* scratch;   // per mode 4 * SG_MAXM^2 doubles
};

// Builds H, operators and their parameter derivatives for one mode, diagonalises
// H, keeps the lowest d levels.  Transmon: charge basis; fluxonium: oscillator
// basis with the cosine written through the eigenbasis of X = (a + a^dag)/sqrt2.
__global__ void __launch_bounds__(kThreads) k_build_modes(BuildArgs a) {
  extern __shared__ double sm[];
  const int q = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int M = a.M[q], d = a.d[q];
  ModeDev md = a.md[q];
  double* A = sm;                 // M*M
  double* Vs = sm + M * M;        // M*M
  double* cs = Vs + M * M;        // 2*SG_MAXM
  int* pairs = reinterpret_cast<int*>(cs + 2 * SG_MAXM);   // 2*SG_MAXM
  double* scr = a.scratch + (size_t)q * 4 * SG_MAXM * SG_MAXM;
  double* W = scr;                       // X eigenvectors (fluxonium)
  double* cosm = scr + M * M;
  double* sinx = scr + 2 * M * M;
  double* gvec = scr + 3 * M * M;        // M entries
  double* gvec2 = gvec + M;              // M entries
  const double ej = a.ej[q], ec = a.ec[q], el = a.el[q];
  double2* n_full = md.ops;
  double2* phi_full = md.ops + M * M;

  if (a.kind[q] == 0) {
    const int ncut = (M - 1) / 2;
    const double ng = a.ng[q];
    for (int i = tid; i < M * M; i += nt) {
      int r = i / M, c = i % M;
      double nr = (double)(r - ncut) - ng;
      double hop = (abs(r - c) == 1) ? 0.5 : 0.0;       // cos(phi) in the charge basis
      A[i] = (r == c ? 4.0 * ec * nr * nr : 0.0) - ej * hop;
      md.dH[0 * M * M + i] = -hop;
      md.dH[1 * M * M + i] = (r == c) ? 4.0 * nr * nr : 0.0;
      md.dH[2 * M * M + i] = 0.0;
      n_full[i] = make_double2(r == c ? nr : 0.0, 0.0);
      phi_full[i] = make_double2(0.0, 0.0);
      for (int op = 0; op < 2; ++op)
        for (int p = 0; p < 3; ++p) md.dops[(op * 3 + p) * M * M + i] = make_double2(0.0, 0.0);
    }
    __syncthreads();
  } else {
    const double phe = a.phi_ext[q];
    // X = (a + a^dag)/sqrt2, tridiagonal
    for (int i = tid; i < M * M; i += nt) {
      int r = i / M, c = i % M;
      double x = 0.0;
      if (c == r + 1) x = sqrt((double)(r + 1)) * M_SQRT1_2;
      if (r == c + 1) x = sqrt((double)(c + 1)) * M_SQRT1_2;
      A[i] = x;
    }
    __syncthreads();
    jacobi_eigen(A, Vs, M, cs, pairs);
    // nodes x_k = A_kk, eigenvectors W = Vs (order irrelevant for W f(x) W^T)
    for (int i = tid; i < M * M; i += nt) W[i] = Vs[i];
    const double po = pow(8.0 * ec / el, 0.25);
    const double wp = sqrt(8.0 * ec * el);
    for (int k = tid; k < M; k += nt) {
      double x = A[k * M + k];
      double arg = po * x - phe;
      gvec[k] = cos(arg);
      gvec2[k] = sin(arg) * x;
    }
    __syncthreads();
    adiag_at(W, gvec, M, cosm);
    adiag_at(W, gvec2, M, sinx);
    const double dpo[3] = {0.0, po / (4.0 * ec), -po / (4.0 * el)};
    const double dwp[3] = {0.0, wp / (2.0 * ec), wp / (2.0 * el)};
    for (int i = tid; i < M * M; i += nt) {
      int r = i / M, c = i % M;
      double X = 0.0, P = 0.0;     // P = i * Pim ; Pim = (a^dag - a)/sqrt2 entries
      if (c == r + 1) { X = sqrt((double)(r + 1)) * M_SQRT1_2; P = -sqrt((double)(r + 1)) * M_SQRT1_2; }
      if (r == c + 1) { X = sqrt((double)(c + 1)) * M_SQRT1_2; P = sqrt((double)(c + 1)) * M_SQRT1_2; }
      double diag = (r == c) ? (double)r + 0.5 : 0.0;
      A[i] = wp * diag - ej * cosm[i];
      for (int p = 0; p < 3; ++p) {
        double v = dwp[p] * diag + ej * dpo[p] * sinx[i];
        if (p == 0) v -= cosm[i];
        md.dH[p * M * M + i] = v;
      }
      n_full[i] = make_double2(0.0, P / po);          // n = i (a^dag - a) / (sqrt2 phi_osc)
      phi_full[i] = make_double2(po * X, 0.0);
      for (int p = 0; p < 3; ++p) {
        md.dops[(0 * 3 + p) * M * M + i] = make_double2(0.0, -P * dpo[p] / (po * po));
        md.dops[(1 * 3 + p) * M * M + i] = make_double2(dpo[p] * X, 0.0);
      }
    }
    __syncthreads();
  }
  jacobi_eigen(A, Vs, M, cs, pairs);
  sort_and_gauge(A, Vs, M, md.w, md.V);
  // truncated energies and operators
  for (int k = tid; k < d; k += nt) md.E[k] = md.w[k] - md.w[0];
  for (int i = tid; i < 2 * d * d; i += nt) {
    int op = i / (d * d), ab = i % (d * d), ia = ab / d, ib = ab % d;
    const double2* O = md.ops + op * M * M;
    double2 acc = make_double2(0.0, 0.0);
    for (int k = 0; k < M; ++k) {
      double vk = md.V[k * M + ia];
      if (vk == 0.0) continue;
      double2 t = make_double2(0.0, 0.0);
      for (int l = 0; l < M; ++l) {
        double vl = md.V[l * M + ib];
        t.x += O[k * M + l].x * vl;
        t.y += O[k * M + l].y * vl;
      }
      acc.x += vk * t.x;
      acc.y += vk * t.y;
    }
    md.opd[i] = acc;
  }
}

struct ChainArgs {
  int nq;
  ModeDev md[SG_MAXQ];
  const double2* opbar;   // nq x 2 x SG_MAXD^2
  const double* ebar;     // nq x SG_MAXD
  double* out;            // nq x 3
  double* scratch;        // per mode 3 * SG_MAXM * SG_MAXD doubles
};

// Eigen-derivative chain for one mode and one parameter per CTA (grid nq x 3):
//   hv = V^T dH V_d,  dw_a = hv_aa,  dv_a = sum_{c != a} v_c hv_ca / (w_a - w_c),
//   dE_a = dw_a - dw_0,  dO = dv^T O V_d + V_d^T O dv + V_d^T dO V_d,
//   out = Re sum conj(Obar) dO + sum Ebar dE.
__global__ void __launch_bounds__(kThreads) k_chain(ChainArgs a) {
  const int q = blockIdx.x, p = blockIdx.y;
  const int tid = threadIdx.x, nt = blockDim.x;
  const ModeDev md = a.md[q];
  const int M = md.M, d = md.d;
  double* scr = a.scratch + ((size_t)q * 3 + p) * 3 * SG_MAXM * SG_MAXD;
  double* T = scr;                   // M x d : dH V_d
  double* hv = scr + M * d;          // M x d : V^T dH V_d
  double* dv = scr + 2 * M * d;      // M x d
  const double* dH = md.dH + (size_t)p * M * M;
  for (int i = tid; i < M * d; i += nt) {
    int k = i / d, b = i % d;
    double acc = 0.0;
    for (int l = 0; l < M; ++l) acc += dH[k * M + l] * md.V[l * M + b];
    T[i] = acc;
  }
  __syncthreads();
  for (int i = tid; i < M * d; i += nt) {
    int c = i / d, b = i % d;
    double acc = 0.0;
    for (int k = 0; k < M; ++k) acc += md.V[k * M + c] * T[k * d + b];
    hv[i] = acc;
  }
  __syncthreads();
  for (int i = tid; i < M * d; i += nt) {
    int k = i / d, b = i % d;
    double acc = 0.0;
    for (int c = 0; c < M; ++c) {
      if (c == b) continue;
      acc += md.V[k * M + c] * hv[c * d + b] / (md.w[b] - md.w[c]);
    }
    dv[i] = acc;
  }
  __syncthreads();
  __shared__ double red[kThreads];
  double part = 0.0;
  // energies
  for (int b = tid; b < d; b += nt) {
    double dE = hv[b * d + b] - hv[0];
    part += a.ebar[q * SG_MAXD + b] * dE;
  }
  // operators
  for (int i = tid; i < 2 * d * d; i += nt) {
    int op = i / (d * d), ab = i % (d * d), ia = ab / d, ib = ab % d;
    double2 ob = a.opbar[(q * 2 + op) * SG_MAXD * SG_MAXD + ia * SG_MAXD + ib];
    if (ob.x == 0.0 && ob.y == 0.0) continue;
    const double2* O = md.ops + (size_t)op * M * M;
    const double2* dO = md.dops + ((size_t)op * 3 + p) * M * M;
    double2 acc = make_double2(0.0, 0.0);
    for (int k = 0; k < M; ++k) {
      double vka = md.V[k * M + ia], dvka = dv[k * d + ia];
      for (int l = 0; l < M; ++l) {
        double vlb = md.V[l * M + ib], dvlb = dv[l * d + ib];
        double2 o = O[k * M + l], dd = dO[k * M + l];
        double w1 = dvka * vlb + vka * dvlb;
        double w2 = vka * vlb;
        acc.x += w1 * o.x + w2 * dd.x;
        acc.y += w1 * o.y + w2 * dd.y;
      }
    }
    part += ob.x * acc.x + ob.y * acc.y;        // Re(conj(ob) * acc)
  }
  red[tid] = part;
  __syncthreads();
  for (int s = nt / 2; s > 0; s >>= 1) { if (tid < s) red[tid] += red[tid + s]; __syncthreads(); }
  if (tid == 0) a.out[q * 3 + p] = red[0];
}

// Element (r, c) of the idle Hamiltonian H[r][c] = delta_rc sum_i E_i[l_i(r)] + sum_e J_e
// A_e[l_a(r)][l_a(c)] B_e[l_b(r)][l_b(c)] (other digits equal); hi: its imaginary part.
__device__ void dressed_h(const DressArgs& a, int r, int c, double& h, double& hi) {
  h = 0.0;
  hi = 0.0;
  if (r == c)
    for (int q = 0; q < a.nq; ++q) h += a.E[a.eoff[q] + (int)((r / a.st[q]) % a.dims[q])];
  for (int e = 0; e < a.ne; ++e) {
    const int qa = a.e_a[e], qb = a.e_b[e];
    bool same = true;
    for (int q = 0; q < a.nq; ++q)
      if (q != qa && q != qb && (r / a.st[q]) % a.dims[q] != (c / a.st[q]) % a.dims[q]) same = false;
    if (!same) continue;
    const int da = a.dims[qa], db = a.dims[qb];
    const int ra = (int)((r / a.st[qa]) % da), ca = (int)((c / a.st[qa]) % da);
    const int rb = (int)((r / a.st[qb]) % db), cb = (int)((c / a.st[qb]) % db);
    const double2 x = a.opd[a.opd_off[qa] + a.e_opa[e] * da * da + ra * da + ca];
    const double2 y = a.opd[a.opd_off[qb] + a.e_opb[e] * db * db + rb * db + cb];
    h += a.J[e] * (x.x * y.x - x.y * y.y);
    hi += a.J[e] * (x.x * y.y + x.y * y.x);
  }
}

// One block, after the eigensolve (eigenvalues on the diagonal of A, eigenvectors in
// the columns of V): per label j the eigenvector k of largest |V[comp_j][k]| (flag 2 if
// two labels share one, flag 3 if its eigenvalue is within 1e-9 of another), signed so
// that V[comp_j][k] > 0, into Vc; *err from the flags in bad (bit 0: complex H).
__device__ void dressed_pick(const DressArgs& a, const double* A, const double* V, int* kk, int* bad) {
  const int D = a.D, tid = threadIdx.x, nt = blockDim.x;
  for (int j = tid; j < a.Dc; j += nt) {
    const int r = (int)a.comp[j];
    int best = 0;
    double bv = -1.0;
    for (int k = 0; k < D; ++k) {
      const double v = fabs(V[(size_t)r * D + k]);
      if (v > bv) { bv = v; best = k; }
    }
    kk[j] = best;
  }
  __syncthreads();
  double scale = 0.0;
  for (int k = 0; k < D; ++k) scale = fmax(scale, fabs(A[(size_t)k * D + k]));
  for (int j = tid; j < a.Dc; j += nt) {
    for (int m = 0; m < j; ++m)
      if (kk[m] == kk[j]) atomicOr(bad, 2);
    const double lk = A[(size_t)kk[j] * D + kk[j]];
    for (int k = 0; k < D; ++k)
      if (k != kk[j] && fabs(A[(size_t)k * D + k] - lk) <= 1e-9 * fmax(1.0, scale)) atomicOr(bad, 4);
  }
  __syncthreads();
  for (int i = tid; i < D * a.Dc; i += nt) {
    const int r = i / a.Dc, j = i - r * a.Dc;
    const int k = kk[j];
    const double sg = V[(size_t)a.comp[j] * D + k] < 0.0 ? -1.0 : 1.0;
    a.Vc[i] = make_double2(sg * V[(size_t)r * D + k], 0.0);
  }
  __syncthreads();
  if (tid == 0) *a.err = *bad & 1 ? 1 : (*bad & 2 ? 2 : (*bad & 4 ? 3 : 0));
}

// One block (D <= kMaxDressed): the idle Hamiltonian in global scratch, real
// symmetric (flag 1 otherwise), Jacobi eigenpairs in the block, then dressed_pick.
__global__ void __launch_bounds__(kThreads) k_dressed(DressArgs a) {
  const int D = a.D, tid = threadIdx.x, nt = blockDim.x;
  double* A = a.work;                                        // D x D, then V (global: D <= 256)
  double* V = A + (size_t)D * D;
  __shared__ double cs[kMaxDressed];                         // 2 x (D / 2 rounded up) rotations
  __shared__ int pairs[kMaxDressed];
  __shared__ int kk[kMaxDressed];
  __shared__ int bad;
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int i = tid; i < D * D; i += nt) {
    const int r = i / D, c = i - r * D;
    double h, hi;
    dressed_h(a, r, c, h, hi);
    if (fabs(hi) > 1e-12 * (fabs(h) + 1.0)) atomicOr(&bad, 1);
    A[i] = h;
  }
  __syncthreads();
  jacobi_eigen(A, V, D, cs, pairs);
  dressed_pick(a, A, V, kk, &bad);
}

// ---- the same for kMaxDressed < D <= kMaxDressedLarge, over the whole GPU ----------
// The matrix lives in global memory (L2-resident at these sizes) and every round of the
// round-robin Jacobi ordering is one launch: for rows i and index pairs (p', q'),
//   A_new[i][{p', q'}] = (R_k A_old)[i][{p', q'}] J_k'
// with k the pair of i and R_k, J_k' the row and column rotations of pairs k and k'
// (the same 2 x 2 Schur rotations as jacobi_eigen, from A_old's diagonal blocks), and
// V[i][{p', q'}] <- V[i][{p', q'}] J_k'.  Every thread reads only A_old, so the
// rotations of one round need no barrier; A_old and A_new swap per round.

// The pairs of round r (circle method over Mp players; index M is a dummy when M is odd):
// position 0 holds player 0, position pos >= 1 holds 1 + (pos - 1 + r) mod (Mp - 1), and
// positions k and Mp - 1 - k play each other.
__device__ __forceinline__ int jac_player(int pos, int r, int Mp) {
  return pos == 0 ? 0 : 1 + (pos - 1 + r) % (Mp - 1);
}
__device__ __forceinline__ int jac_pos(int i, int r, int Mp) {
  return i == 0 ? 0 : 1 + ((i - 1 - r) % (Mp - 1) + (Mp - 1)) % (Mp - 1);
}
// Rotation (c, s) of the pair (p, q), p < q, from A's diagonal block; (1, 0) for the dummy.
__device__ __forceinline__ void jac_cs(const double* A, int M, int p, int q, double& c, double& s) {
  c = 1.0;
  s = 0.0;
  if (q >= M) return;
  const double apq = A[(size_t)p * M + q];
  if (apq == 0.0) return;
  const double app = A[(size_t)p * M + p], aqq = A[(size_t)q * M + q];
  const double tau = (aqq - app) / (2.0 * apq);
  const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
  c = 1.0 / sqrt(1.0 + t * t);
  s = t * c;
}

__global__ void k_dressed_build(DressArgs a, double* __restrict__ A, double* __restrict__ V) {
  const long long D = a.D, n = D * D;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / D), c = (int)(i - r * D);
    double h, hi;
    dressed_h(a, r, c, h, hi);
    if (fabs(hi) > 1e-12 * (fabs(h) + 1.0)) atomicOr(a.err, 1);
    A[i] = h;
    V[i] = r == c ? 1.0 : 0.0;
  }
}

__global__ void k_jac_round(const double* __restrict__ Ao, double* __restrict__ An, double* __restrict__ V, int M,
                            int Mp, int r) {
  const int npair = Mp / 2;
  const long long n = (long long)M * npair;
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(x / npair), k2 = (int)(x - (long long)i * npair);
    // the pair (p, q) of row i and its rotation
    const int pos = jac_pos(i, r, Mp), k = pos < npair ? pos : Mp - 1 - pos;
    const int a0 = jac_player(k, r, Mp), b0 = jac_player(Mp - 1 - k, r, Mp);
    const int p = min(a0, b0), q = max(a0, b0);
    double c, s;
    jac_cs(Ao, M, p, q, c, s);
    // the column pair (p2, q2) and its rotation
    const int a2 = jac_player(k2, r, Mp), b2 = jac_player(Mp - 1 - k2, r, Mp);
    const int p2 = min(a2, b2), q2 = max(a2, b2);
    double c2, s2;
    jac_cs(Ao, M, p2, q2, c2, s2);
    // row rotation: row p <- c row p - s row q, row q <- s row p + c row q
    const double* rp = Ao + (size_t)p * M;
    const double* rq = q < M ? Ao + (size_t)q * M : rp;
    const bool hq2 = q2 < M;
    const double bp = rp[p2], bq = q < M ? rq[p2] : 0.0;
    const double cp = hq2 ? rp[q2] : 0.0, cq = q < M && hq2 ? rq[q2] : 0.0;
    double u, w;                                           // (R A)[i][p2], (R A)[i][q2]
    if (i == p) { u = c * bp - s * bq; w = c * cp - s * cq; }
    else        { u = s * bp + c * bq; w = s * cp + c * cq; }
    // column rotation: col p2 <- c2 col p2 - s2 col q2, col q2 <- s2 col p2 + c2 col q2
    double np2 = c2 * u - s2 * w, nq2 = s2 * u + c2 * w;
    if (k2 == k && s != 0.0) {                             // the annihilated pair is exactly zero
      if (i == p) nq2 = 0.0;
      else np2 = 0.0;
    }
    double* out = An + (size_t)i * M;
    out[p2] = np2;
    if (hq2) out[q2] = nq2;
    double* v = V + (size_t)i * M;
    if (hq2) {
      const double vp = v[p2], vq = v[q2];
      v[p2] = c2 * vp - s2 * vq;
      v[q2] = s2 * vp + c2 * vq;
    }
  }
}

// Off-diagonal and diagonal squared mass of A: per block partial sums (each thread a
// fixed stride of the entries, then the block in a fixed tree), summed in block order.
__global__ void k_jac_mass(const double* __restrict__ A, int M, double* __restrict__ part) {
  __shared__ double ro[kThreads], rd[kThreads];
  const long long n = (long long)M * M;
  double off = 0.0, dia = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / M), c = (int)(i - (long long)r * M);
    if (r != c) off += A[i] * A[i]; else dia += A[i] * A[i];
  }
  ro[threadIdx.x] = off;
  rd[threadIdx.x] = dia;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) { ro[threadIdx.x] += ro[threadIdx.x + s]; rd[threadIdx.x] += rd[threadIdx.x + s]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { part[2 * blockIdx.x] = ro[0]; part[2 * blockIdx.x + 1] = rd[0]; }
}
__global__ void k_jac_mass_sum(const double* __restrict__ part, int nb, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double o = 0.0, d = 0.0;
    for (int b = 0; b < nb; ++b) { o += part[2 * b]; d += part[2 * b + 1]; }
    out[0] = o;
    out[1] = d;
  }
}

__global__ void __launch_bounds__(kThreads) k_dressed_pick(DressArgs a, const double* __restrict__ A,
                                                           const double* __restrict__ V) {
  __shared__ int kk[kMaxDressed];
  __shared__ int bad;
  if (threadIdx.x == 0) bad = *a.err;                        // bit 0 from the build
  __syncthreads();
  dressed_pick(a, A, V, kk, &bad);
}

}  // namespace

sg_status sg_prepare_impl(sg_system* sys) {
  sg_ctx* ctx = sys->ctx;
  const int nq = (int)sys->modes.size();
  if (nq == 0) return sg_fail(ctx, SG_E_STATE, "system has no modes");
  if (nq > SG_MAXQ) return sg_fail(ctx, SG_E_UNSUPPORTED, "too many modes");
  SG_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  // layout of the per-mode block
  size_t per_mode = 0;
  const size_t MM = (size_t)SG_MAXM * SG_MAXM;
  per_mode += SG_MAXM * sizeof(double);                 // w
  per_mode += MM * sizeof(double);                      // V
  per_mode += 3 * MM * sizeof(double);                  // dH
  per_mode += 2 * MM * sizeof(double2);                 // ops
  per_mode += 6 * MM * sizeof(double2);                 // dops
  per_mode += SG_MAXD * sizeof(double);                 // E
  per_mode += 2 * SG_MAXD * SG_MAXD * sizeof(double2);  // opd
  per_mode = (per_mode + 255) & ~(size_t)255;
  const size_t scratch_bytes = (size_t)nq * 4 * MM * sizeof(double);
  const size_t total = per_mode * nq + scratch_bytes;
  if (sys->mode_block && sys->mode_block_bytes < total) {
    cudaFree(sys->mode_block);
    sys->mode_block = nullptr;
  }
  if (!sys->mode_block) {
    if (cudaMalloc(&sys->mode_block, total) != cudaSuccess)
      return sg_fail(ctx, SG_E_NOMEM, "cudaMalloc of the mode block failed");
    sys->mode_block_bytes = total;
  }
  char* base = static_cast<char*>(sys->mode_block);
  sys->mdev.assign(nq, ModeDev{});
  BuildArgs args{};
  args.nq = nq;
  for (int q = 0; q < nq; ++q) {
    const HostMode& hm = sys->modes[q];
    char* p = base + per_mode * q;
    ModeDev md{};
    md.kind = hm.kind; md.M = hm.M; md.d = hm.d;
    md.w = reinterpret_cast<double*>(p); p += SG_MAXM * sizeof(double);
    md.V = reinterpret_cast<double*>(p); p += MM * sizeof(double);
    md.dH = reinterpret_cast<double*>(p); p += 3 * MM * sizeof(double);
    md.ops = reinterpret_cast<double2*>(p); p += 2 * MM * sizeof(double2);
    md.dops = reinterpret_cast<double2*>(p); p += 6 * MM * sizeof(double2);
    md.E = reinterpret_cast<double*>(p); p += SG_MAXD * sizeof(double);
    md.opd = reinterpret_cast<double2*>(p);
    sys->mdev[q] = md;
    args.kind[q] = hm.kind; args.M[q] = hm.M; args.d[q] = hm.d;
    args.ej[q] = hm.ej; args.ec[q] = hm.ec; args.el[q] = hm.el;
    args.ng[q] = hm.ng; args.phi_ext[q] = hm.phi_ext;
    args.md[q] = md;
  }
  args.scratch = reinterpret_cast<double*>(base + per_mode * nq);
  const size_t smem = (2 * MM + 2 * SG_MAXM) * sizeof(double) + 2 * SG_MAXM * sizeof(int);
  // the limit for the largest basis, once (a per-call size would race with
  // concurrent prepares of other basis sizes on other host threads)
  static const cudaError_t attr = cudaFuncSetAttribute(
      k_build_modes, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)((2 * SG_MAXM * SG_MAXM + 2 * SG_MAXM) * sizeof(double) + 2 * SG_MAXM * sizeof(int)));
  SG_CUDA_TRY(ctx, attr);
  k_build_modes<<<nq, kThreads, smem, ctx->stream>>>(args);
  SG_CUDA_TRY(ctx, cudaGetLastError());
  if (!sys->mdev_dev) SG_CUDA_TRY(ctx, cudaMalloc(&sys->mdev_dev, SG_MAXQ * sizeof(ModeDev)));
  SG_CUDA_TRY(ctx, cudaMemcpyAsync(sys->mdev_dev, sys->mdev.data(), nq * sizeof(ModeDev),
                                   cudaMemcpyHostToDevice, ctx->stream));
  // host copies of the truncated data
  sys->E_host.assign(nq, {});
  sys->opd_host.assign(nq, {});
  sys->parity_odd.assign(SG_MAXOP * nq, 0);
  for (int q = 0; q < nq; ++q) {
    const int d = sys->modes[q].d;
    sys->E_host[q].resize(d);
    sys->opd_host[q].resize(4 * d * d);
    SG_CUDA_TRY(ctx, cudaMemcpyAsync(sys->E_host[q].data(), sys->mdev[q].E, d * sizeof(double),
                                     cudaMemcpyDeviceToHost, ctx->stream));
    SG_CUDA_TRY(ctx, cudaMemcpyAsync(sys->opd_host[q].data(), sys->mdev[q].opd,
                                     2 * d * d * sizeof(double2), cudaMemcpyDeviceToHost,
                                     ctx->stream));
  }
  SG_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  // local operators follow n and phi in each mode's block
  for (int q = 0; q < nq; ++q)
    sys->opd_host[q].insert(sys->opd_host[q].end(), sys->modes[q].local.begin(), sys->modes[q].local.end());
  // parity structure: entries with (a + b) even negligible -> the operator only
  // couples levels of opposite parity (true at n_g = 0 and phi_ext = pi)
  for (int q = 0; q < nq; ++q) {
    const int d = sys->modes[q].d;
    const int nop = (int)(sys->opd_host[q].size() / (2 * (size_t)d * d));
    for (int op = 0; op < nop; ++op) {
      const double* o = sys->opd_host[q].data() + op * 2 * d * d;
      double mx = 0.0, even = 0.0;
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
          double m = std::hypot(o[2 * (a * d + b)], o[2 * (a * d + b) + 1]);
          mx = std::max(mx, m);
          if (((a + b) & 1) == 0) even = std::max(even, m);
        }
      sys->parity_odd[SG_MAXOP * q + op] = (mx > 0.0 && even <= 1e-13 * mx) ? 1 : 0;
    }
  }
  sys->prepared = true;
  return SG_OK;
}

sg_status sg_chain_device_params(sg_system* sys, const double2* opbar_dev, const double* ebar_dev,
                                 double* out_dev) {
  sg_ctx* ctx = sys->ctx;
  const int nq = (int)sys->modes.size();
  ChainArgs a{};
  a.nq = nq;
  for (int q = 0; q < nq; ++q) a.md[q] = sys->mdev[q];
  a.opbar = opbar_dev;
  a.ebar = ebar_dev;
  a.out = out_dev;
  // reuse the build scratch (4*MAXM^2 doubles per mode >= 3*3*MAXM*MAXD)
  const size_t MM = (size_t)SG_MAXM * SG_MAXM;
  size_t per_mode = 0;
  per_mode += SG_MAXM * sizeof(double) + MM * sizeof(double) + 3 * MM * sizeof(double) +
              2 * MM * sizeof(double2) + 6 * MM * sizeof(double2) + SG_MAXD * sizeof(double) +
              2 * SG_MAXD * SG_MAXD * sizeof(double2);
  per_mode = (per_mode + 255) & ~(size_t)255;
  a.scratch = reinterpret_cast<double*>(static_cast<char*>(sys->mode_block) + per_mode * nq);
  k_chain<<<dim3(nq, 3), kThreads, 0, ctx->stream>>>(a);
  SG_CUDA_TRY(ctx, cudaGetLastError());
  return SG_OK;
}

size_t dressed_work_doubles(int D) {
  const size_t D2 = (size_t)D * D;
  return D <= kMaxDressed ? 2 * D2 : 3 * D2 + 2 * (size_t)kJacMassBlocks + 2;
}

cudaError_t launch_dressed(const DressArgs& a, cudaStream_t st, int* launches) {
  if (a.D < 2 || a.D > kMaxDressedLarge || a.Dc > a.D || a.Dc > kMaxDressed) return cudaErrorInvalidValue;
  if (a.D <= kMaxDressed) {
    k_dressed<<<1, kThreads, 0, st>>>(a);
    if (launches) ++*launches;
    return cudaGetLastError();
  }
  const int M = a.D, Mp = (M + 1) & ~1, npair = Mp / 2;
  const size_t D2 = (size_t)M * M;
  double* A = a.work;
  double* B = A + D2;
  double* V = B + D2;
  double* part = V + D2;
  double* mass = part + 2 * kJacMassBlocks;
  cudaError_t e = cudaMemsetAsync(a.err, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  const int gb = (int)std::min<long long>(4096, ((long long)D2 + kThreads - 1) / kThreads);
  k_dressed_build<<<gb, kThreads, 0, st>>>(a, A, V);
  int n = 1;
  const int gr = (int)(((long long)M * npair + kThreads - 1) / kThreads);
  for (int sweep = 0; sweep < 40; ++sweep) {
    k_jac_mass<<<kJacMassBlocks, kThreads, 0, st>>>(A, M, part);
    k_jac_mass_sum<<<1, 32, 0, st>>>(part, kJacMassBlocks, mass);
    n += 2;
    double hm[2] = {0.0, 0.0};
    if ((e = cudaMemcpyAsync(hm, mass, sizeof(hm), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    if (hm[0] <= 1e-32 * hm[1] || hm[0] == 0.0) break;       // the criterion of jacobi_eigen
    for (int r = 0; r < Mp - 1; ++r) {
      k_jac_round<<<gr, kThreads, 0, st>>>(A, B, V, M, Mp, r);
      std::swap(A, B);
    }
    n += Mp - 1;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  k_dressed_pick<<<1, kThreads, 0, st>>>(a, A, V);
  ++n;
  if (launches) *launches += n;
  return cudaGetLastError();
}
