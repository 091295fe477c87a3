// Dense small-dimension RK4 on the tensor cores (tcgen05), batched over systems of
// one shape, with 3xTF32 split-precision products.
//
// For a system whose terms are real in the truncated eigenbasis up to the
// interaction-frame phases (as for the tiled passes' real-operator form), the
// stage derivative is
//     k = -i P (H_r(t) (P^dag y)),   H_r(t) = C + sum_k f_k(t) O_k,   P = diag(exp(i E t)),
// with C (couplings; in the lab frame also diag E) and O_k (drive operators, each
// embedded on its mode) constant real D x D matrices.  So the matrices are the
// constant A operand of one tcgen05.mma per k-step, stacked [C; O_1; ...; O_K] per
// system (R rows) and G = 128 / R systems per CTA (M = 128); the B operand is the
// state z = P^dag y of the CTA's systems as [Re z | Im z] (2S columns each, N = 2 S G
// rows of the K-major B), rewritten every stage.  Each product is split into TF32
// parts, A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi (FP32 accumulation in tensor memory),
// about FP32 accuracy.  Only the diagonal blocks of the 128 x N product (a system's
// rows times its own columns) are read.  The stage math is FP32 and the RK4 state is
// kept as float-float pairs, as in the on-chip kernels.
//
// Shared-memory operands are in the canonical K-major layout without swizzle: 8-row
// groups of K/4 core matrices (8 rows x 16 bytes) stored contiguously, core matrices
// along K 128 bytes apart (leading byte offset), 8-row groups K/4 * 128 bytes apart
// (stride byte offset).
#include "sg_internal.h"
#include "dense.h"
#include <algorithm>
#include <cstdint>

namespace {

__device__ __forceinline__ uint32_t d_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading / stride byte offsets,
// descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t d_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t d_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void d_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
               ::"r"(tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void d_commit(uint64_t* mb) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(d_smem(mb))
               : "memory");
}
__device__ __forceinline__ void d_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void d_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ bool d_mb_try(uint64_t* mb, unsigned parity) {
  unsigned ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(ok) : "r"(d_smem(mb)), "r"(parity) : "memory");
  return ok != 0;
}
// Bounded wait (about a second at the default limit): true once the phase completed.
__device__ __forceinline__ bool d_mb_wait(uint64_t* mb, unsigned parity, int limit) {
  for (int it = 0; it < limit; ++it) {
    if (d_mb_try(mb, parity)) return true;
    __nanosleep(64);
  }
  return false;
}
// TF32 value of x rounded to nearest (the low 13 mantissa bits zero).
__device__ __forceinline__ float d_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
// Tensor-memory load of 32 lanes x NC consecutive 32-bit columns (NC = 8, 16, 32).
template <int NC> __device__ __forceinline__ void d_tld(uint32_t taddr, float (&v)[NC]);
template <> __device__ __forceinline__ void d_tld<8>(uint32_t t, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(t) : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}
template <> __device__ __forceinline__ void d_tld<16>(uint32_t t, float (&v)[16]) {
  uint32_t r[16];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(t) : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
template <> __device__ __forceinline__ void d_tld<32>(uint32_t t, float (&v)[32]) {
  uint32_t r[32];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
               "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                 "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                 "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
               : "r"(t) : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// Float index of element (row r, k) of a K-major no-swizzle operand with Kp columns.
__host__ __device__ __forceinline__ int d_cidx(int r, int k, int Kp) {
  return (r >> 3) * (Kp * 8) + (k >> 2) * 32 + (r & 7) * 4 + (k & 3);
}

// exp(i th) in FP32 after reducing th modulo 2 pi in FP64 (two-term 2 pi).
__device__ __forceinline__ float2 d_cis(double th) {
  const double k = rint(th * 0.15915494309189535);
  const double r = fma(-k, 2.4492935982947064e-16, fma(-k, 6.283185307179586, th));
  float s, c;
  sincosf((float)r, &s, &c);
  return make_float2(c, s);
}
// hi + lo <- hi + lo + x (TwoSum with a fast renormalisation)
__device__ __forceinline__ void d_ff_add(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bb = s - hi;
  const float e = (hi - (s - bb)) + (x - bb);
  const float l = lo + e;
  const float h2 = s + l;
  lo = l - (h2 - s);
  hi = h2;
}

}  // namespace

namespace {

// Shared-memory layout of k_dense_rk4 (bytes from the dynamic base).
struct DenseSmem {
  size_t ahi, alo, bhi, blo, w, ph, fs, mbar, tslot, total;
};
__host__ __device__ inline DenseSmem dense_smem(int Dp, int N, int NC, int G, int D, int K) {
  DenseSmem l{};
  size_t o = 0;
  l.ahi = o; o += (size_t)128 * Dp * 4;
  l.alo = o; o += (size_t)128 * Dp * 4;
  l.bhi = o; o += (size_t)N * Dp * 4;
  l.blo = o; o += (size_t)N * Dp * 4;
  l.w = o; o += (size_t)128 * (NC + 1) * 4;
  o = (o + 15) & ~(size_t)15;
  l.ph = o; o += (size_t)2 * G * D * 8;
  l.fs = o; o += (size_t)2 * G * (K > 0 ? K : 1) * 4;
  o = (o + 15) & ~(size_t)15;
  l.mbar = o; o += 16;
  l.tslot = o; o += 16;
  l.total = o;
  return l;
}

// One CTA (128 threads, 4 warps = the 4 tensor-memory lane quarters) evolves G
// systems for the whole run.  Thread t owns the state entries e = t + 128 j (system
// g, row i, column s) in registers: the stage input y, the increment sum Dacc and
// the float-float state.  Per stage: thread 0 issues the 3 (Dp / 8) MMAs and commits
// them to an mbarrier; the threads meanwhile stage the next phases and drive
// coefficients; after a bounded wait every warp copies its lanes' diagonal block
// from tensor memory to shared memory, and the threads apply the RK4 update and
// write the next B operand.  A wait that runs out sets a.err; the CTA (agreeing by a
// barrier vote) issues no further MMAs, runs to its end and waits (bounded) for the
// MMAs it gave up on before freeing its tensor memory.
template <int EPT, int NC>
__global__ void __launch_bounds__(128, 1) k_dense_rk4(DenseArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int Dp = a.Dp, R = a.R, G = a.G, D = a.D, S = a.S, N = a.N, K = a.K;
  const DenseSmem L = dense_smem(Dp, N, NC, G, D, K);
  float* const Ahi = reinterpret_cast<float*>(sm + L.ahi);
  float* const Alo = reinterpret_cast<float*>(sm + L.alo);
  float* const Bhi = reinterpret_cast<float*>(sm + L.bhi);
  float* const Blo = reinterpret_cast<float*>(sm + L.blo);
  float* const W = reinterpret_cast<float*>(sm + L.w);
  float2* const PH = reinterpret_cast<float2*>(sm + L.ph);     // [2][G D]
  float* const FS = reinterpret_cast<float*>(sm + L.fs);       // [2][G K]
  uint64_t* const mbar = reinterpret_cast<uint64_t*>(sm + L.mbar);
  uint32_t* const tslot = reinterpret_cast<uint32_t*>(sm + L.tslot);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b0 = blockIdx.x * G;
  const uint32_t ncols = N <= 32 ? 32u : (N <= 64 ? 64u : (N <= 128 ? 128u : 256u));
  // constant A operand, split into TF32 parts; rows past the CTA's systems are zero
  for (int x = tid; x < 128 * Dp; x += 128) {
    const int m = x / Dp, k = x - (x / Dp) * Dp, g = m / R, r = m - g * R;
    const double v = (g < G && b0 + g < a.B) ? a.A[((size_t)(b0 + g) * R + r) * Dp + k] : 0.0;
    const float hi = d_tf32((float)v);
    Ahi[d_cidx(m, k, Dp)] = hi;
    Alo[d_cidx(m, k, Dp)] = d_tf32((float)(v - (double)hi));
  }
  for (int x = tid; x < N * Dp; x += 128) { Bhi[x] = 0.f; Blo[x] = 0.f; }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(d_smem(tslot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(d_smem(mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  // state entries of this thread
  float yr[EPT], yi[EPT], dr[EPT], di[EPT], prh[EPT], prl[EPT], pih[EPT], pil[EPT];
  int eg[EPT], ei[EPT], es[EPT];
  bool ok[EPT];
#pragma unroll
  for (int j = 0; j < EPT; ++j) {
    const int e = tid + 128 * j;
    const int g = e / (D * S), rest = e - g * D * S;
    eg[j] = g;
    ei[j] = rest / S;
    es[j] = rest - (rest / S) * S;
    ok[j] = g < G && b0 + g < a.B;
    const float v = ok[j] && a.cols[es[j]] == ei[j] ? 1.f : 0.f;
    yr[j] = v; yi[j] = 0.f; dr[j] = 0.f; di[j] = 0.f;
    prh[j] = v; prl[j] = 0.f; pih[j] = 0.f; pil[j] = 0.f;
  }
  // phases exp(i E t) and drive coefficients of stage slot q into buffer buf
  auto stage_tables = [&](int buf, int q) {
    const double t = (double)(2 * (q / 3) + q % 3) * a.dt * 0.5;
    for (int x = tid; x < G * D; x += 128) {
      const int g = x / D, b = b0 + g;
      PH[buf * G * D + x] = (b < a.B && a.frame == SG_FRAME_INTERACTION) ? d_cis(a.E[(size_t)b * D + x - g * D] * t)
                                                                      : make_float2(1.f, 0.f);
    }
    for (int x = tid; x < G * K; x += 128) {
      const int g = x / K, b = b0 + g;
      FS[buf * G * K + x] = b < a.B ? a.coef[((size_t)b * 3 * a.nsteps + q) * K + x - g * K] : 0.f;
    }
  };
  // B operand of the stage input: z = conj(P) y as [Re z | Im z] rows of each system
  auto write_b = [&](int buf) {
#pragma unroll
    for (int j = 0; j < EPT; ++j) {
      if (!ok[j]) continue;
      const float2 p = PH[buf * G * D + eg[j] * D + ei[j]];
      const float zr = p.x * yr[j] + p.y * yi[j], zi = p.x * yi[j] - p.y * yr[j];
      const int nr = eg[j] * NC + es[j], ni = nr + S;
      const float hr = d_tf32(zr), hi = d_tf32(zi);
      Bhi[d_cidx(nr, ei[j], Dp)] = hr;
      Blo[d_cidx(nr, ei[j], Dp)] = d_tf32(zr - hr);
      Bhi[d_cidx(ni, ei[j], Dp)] = hi;
      Blo[d_cidx(ni, ei[j], Dp)] = d_tf32(zi - hi);
    }
  };
  __syncthreads();
  stage_tables(0, 0);
  __syncthreads();
  write_b(0);
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  d_fence_before();
  __syncthreads();
  d_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = d_idesc(128, N);
  const uint32_t sbo = (uint32_t)Dp * 32;           // 8 rows x Dp floats
  const float h = (float)a.dt;
  unsigned parity = 0, lost = 0;
  bool aborted = false;
  int cur = 0;
  for (int n = 0; n < a.nsteps; ++n) {
#pragma unroll 1
    for (int st = 0; st < 4; ++st) {
      const int qn = st == 3 ? 3 * (n + 1) : 3 * n + (st + 1 == 3 ? 2 : 1);
      if (tid == 0 && !aborted) {
        for (int kk = 0; kk < Dp / 8; ++kk) {
          const uint64_t ah = d_desc(d_smem(Ahi) + kk * 256, 128, sbo), al = d_desc(d_smem(Alo) + kk * 256, 128, sbo);
          const uint64_t bh = d_desc(d_smem(Bhi) + kk * 256, 128, sbo), bl = d_desc(d_smem(Blo) + kk * 256, 128, sbo);
          d_mma(tmem, ah, bh, idesc, kk > 0);
          d_mma(tmem, ah, bl, idesc, 1);
          d_mma(tmem, al, bh, idesc, 1);
        }
        d_commit(mbar);
      }
      if (n + (st == 3) < a.nsteps) stage_tables(cur ^ 1, qn);
      const bool okw = aborted ? true : d_mb_wait(mbar, parity, a.wlim);
      if (!__syncthreads_and(okw ? 1 : 0) && !aborted) {
        aborted = true;
        lost = parity;
        if (tid == 0) atomicExch(a.err, 1);
      }
      parity ^= 1;
      d_fence_after();
      {
        const int m0 = 32 * warp, g = m0 / R;
        if (g < G) {
          float v[NC];
          d_tld<NC>(tmem + ((uint32_t)m0 << 16) + (uint32_t)(g * NC), v);
#pragma unroll
          for (int c = 0; c < NC; ++c) W[(m0 + lane) * (NC + 1) + c] = v[c];
        }
      }
      d_fence_before();
      __syncthreads();
#pragma unroll
      for (int j = 0; j < EPT; ++j) {
        if (!ok[j]) continue;
        const int g = eg[j], i = ei[j], s = es[j];
        const float* wr0 = W + (g * R + i) * (NC + 1);
        float wr = wr0[s], wi = wr0[S + s];
        for (int k = 0; k < K; ++k) {
          const float f = FS[cur * G * K + g * K + k];
          const float* wk = W + (g * R + (1 + k) * Dp + i) * (NC + 1);
          wr = fmaf(f, wk[s], wr);
          wi = fmaf(f, wk[S + s], wi);
        }
        const float2 p = PH[cur * G * D + g * D + i];
        const float hr = p.x * wr - p.y * wi, hv = p.x * wi + p.y * wr;    // H y = P w
        const float kr = hv, ki = -hr;                                     // -i H y
        if (st == 0) {
          dr[j] = h / 6 * kr; di[j] = h / 6 * ki;
          yr[j] = prh[j] + h / 2 * kr; yi[j] = pih[j] + h / 2 * ki;
        } else if (st == 1) {
          dr[j] += h / 3 * kr; di[j] += h / 3 * ki;
          yr[j] = prh[j] + h / 2 * kr; yi[j] = pih[j] + h / 2 * ki;
        } else if (st == 2) {
          dr[j] += h / 3 * kr; di[j] += h / 3 * ki;
          yr[j] = prh[j] + h * kr; yi[j] = pih[j] + h * ki;
        } else {
          d_ff_add(prh[j], prl[j], dr[j] + h / 6 * kr);
          d_ff_add(pih[j], pil[j], di[j] + h / 6 * ki);
          yr[j] = prh[j]; yi[j] = pih[j];
        }
      }
      if (n + (st == 3) < a.nsteps) write_b(cur ^ 1);
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      d_fence_before();
      __syncthreads();
      d_fence_after();
      cur ^= 1;
    }
  }
  // lab-frame states: exp(-i E T) psi_I in FP64
  const double T = (double)a.nsteps * a.dt;
#pragma unroll
  for (int j = 0; j < EPT; ++j) {
    if (!ok[j]) continue;
    const int b = b0 + eg[j];
    const double xr = (double)prh[j] + (double)prl[j], xi = (double)pih[j] + (double)pil[j];
    double c = 1.0, sn = 0.0;
    if (a.frame == SG_FRAME_INTERACTION) sincos(-a.E[(size_t)b * D + ei[j]] * T, &sn, &c);
    a.out[((size_t)b * D + ei[j]) * S + es[j]] = make_double2(c * xr - sn * xi, c * xi + sn * xr);
  }
  if (aborted) d_mb_wait(mbar, lost, a.wlim);        // the MMAs given up on, if still running
  d_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols) : "memory");
}

}  // namespace

bool dense_shape(int D, int S, int K, int* Dp_, int* R_, int* G_, int* N_) {
  const int NC = 2 * S;
  if (D < 1 || K < 0 || !(NC == 8 || NC == 16 || NC == 32)) return false;
  int Dp = ((D + 7) / 8) * 8;
  while (((1 + K) * Dp) % 32 != 0) Dp += 8;
  const int R = (1 + K) * Dp;
  if (R > 128) return false;
  const int G = 128 / R, N = NC * G;
  if (N < 16 || N > 256 || N % 16 != 0) return false;
  const int ept = (G * D * S + 127) / 128;
  if (ept > 16) return false;
  *Dp_ = Dp; *R_ = R; *G_ = G; *N_ = N;
  return true;
}

size_t dense_smem_bytes(const DenseArgs& a) { return dense_smem(a.Dp, a.N, 2 * a.S, a.G, a.D, a.K).total; }

namespace {
template <int EPT, int NC>
cudaError_t dense_go(const DenseArgs& a, cudaStream_t st) {
  const size_t smem = dense_smem_bytes(a);
  static const bool attr = cudaFuncSetAttribute(k_dense_rk4<EPT, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                220 * 1024) == cudaSuccess;
  (void)attr;
  const int grid = (a.B + a.G - 1) / a.G;
  k_dense_rk4<EPT, NC><<<grid, 128, smem, st>>>(a);
  return cudaGetLastError();
}
template <int EPT>
cudaError_t dense_nc(const DenseArgs& a, cudaStream_t st) {
  switch (2 * a.S) {
    case 8: return dense_go<EPT, 8>(a, st);
    case 16: return dense_go<EPT, 16>(a, st);
    default: return dense_go<EPT, 32>(a, st);
  }
}
}  // namespace

cudaError_t dense_launch(const DenseArgs& a, cudaStream_t st) {
  const int ept = (a.G * a.D * a.S + 127) / 128;
  if (ept <= 1) return dense_nc<1>(a, st);
  if (ept <= 2) return dense_nc<2>(a, st);
  if (ept <= 4) return dense_nc<4>(a, st);
  if (ept <= 8) return dense_nc<8>(a, st);
  return dense_nc<16>(a, st);
}
