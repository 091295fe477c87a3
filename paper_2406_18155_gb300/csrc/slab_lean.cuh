// Lean FP32 stage passes for the commonest tiled plan: every mode with 4 levels,
// every operator parity-odd, tiles of 4096 entries (6 tile digits, the groups of the
// 2^20-entry ring and of any 4-level plan with 6-mode groups).  The arithmetic is
// that of the real-operator passes (slab_dev.cuh: P_G H_r P_G^dag y, real rows as
// packed FP32x2 FMAs); what differs is the index work:
//  * a phase over tile digits (ka, kb) runs a block routine compiled for its second
//    digit kb, so a block's accesses are immediate offsets from four row pointers
//    (one per level of ka); the block position and ka's stride come from a per-phase
//    row in shared memory (six routines: one per tile digit; one per digit pair, all
//    fifteen, spilled registers);
//  * tile entry t = tid + 256 j (j = 0..15) sits at global offset lo(tid) + hi(j)
//    (the digit map is linear), so a thread keeps lo and reads hi(j) as one shared
//    broadcast; its phase factor is pl(tid) phi(j) and its shared-memory position
//    spos(tid) + 273 j;
//  * the epilogue's stage and pass kind select a loop compiled for them (no per-entry
//    branches).
#pragma once
#include "slab_dev.cuh"

namespace {
namespace lean {

constexpr int LT = 4096;          // tile entries
constexpr int LJ = LT / kST;      // entries per thread (16)

__host__ __device__ constexpr int lpad(int o) { return o + (o >> 4) + (o >> 8); }
// padded shared-memory stride of tile digit k (tile stride 4^(5 - k))
__host__ __device__ constexpr int lpst(int k) { return lpad(1 << (2 * (5 - k))); }

// The block digits other than (ka, kb) in the bank-conflict-free mapping order of the
// tiled passes (make_phase): the lowest even-exponent digit, the lowest odd-exponent
// one, then the rest by increasing exponent.
__host__ __device__ constexpr int lord(int ka, int kb, int j) {
  int ord[4] = {0, 0, 0, 0};
  int no = 0;
  for (int pass = 0; pass < 3; ++pass)
    for (int k = 5; k >= 0; --k) {
      if (k == ka || k == kb) continue;
      bool used = false;
      for (int i = 0; i < no; ++i) used = used || ord[i] == k;
      if (used) continue;
      const int ex = 5 - k;
      if (pass == 0 && ex % 2 != 0) continue;
      if (pass == 1 && ex % 2 != 1) continue;
      ord[no++] = k;
      if (pass < 2) break;
    }
  return ord[j];
}

// One block of one phase (zphase_block for parity-odd rows, the second digit KB
// compile-time, the first digit's padded stride PA at run time):
//   out[x][z] (+)= sum_a L[x][a] sum_c R[z][c] y[a][c] + sum_a A[x][a] y[a][z] + sum_c B[z][c] y[x][c]
// pb: the block's padded position; oL, oR, oA, oB: row offsets of the terms (-1:
// absent); first: no running sum yet.
template <int KB>
__device__ __forceinline__ void lphase(const float2* __restrict__ M, const float2* __restrict__ ys,
                                       float2* __restrict__ ks, int pb, int PA, int oL, int oR, int oA, int oB,
                                       bool first) {
  constexpr int PB = lpst(KB);
  const float2* yr[4];
  float2* kr[4];
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    yr[x] = ys + pb + x * PA;
    kr[x] = ks + pb + x * PA;
  }
  float2 y[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int z = 0; z < 4; ++z) y[x][z] = yr[x][z * PB];
  const bool hE = oL >= 0, hA = oA >= 0, hB = oB >= 0;
  float2 l[4][2];
  if (hE) {
#pragma unroll
    for (int x = 0; x < 4; ++x) zrow_ld<2>(M + oL + 4 * x, l[x]);
  }
#pragma unroll
  for (int z = 0; z < 4; ++z) {
    float2 o[4];
#pragma unroll
    for (int x = 0; x < 4; ++x) o[x] = first ? make_float2(0.f, 0.f) : kr[x][z * PB];
    if (hE) {
      float2 r[2];
      zrow_ld<2>(M + oR + 4 * z, r);
      float2 u[4];
#pragma unroll
      for (int aa = 0; aa < 4; ++aa) {
        float2 t = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 2; ++k) t = zfma(r[k], y[aa][zcol<true>(z, k)], t);
        u[aa] = t;
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int k = 0; k < 2; ++k) o[x] = zfma(l[x][k], u[zcol<true>(x, k)], o[x]);
    }
    if (hA) {
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        float2 a[2];
        zrow_ld<2>(M + oA + 4 * x, a);
#pragma unroll
        for (int k = 0; k < 2; ++k) o[x] = zfma(a[k], y[zcol<true>(x, k)][z], o[x]);
      }
    }
    if (hB) {
      float2 b[2];
      zrow_ld<2>(M + oB + 4 * z, b);
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int k = 0; k < 2; ++k) o[x] = zfma(b[k], y[x][zcol<true>(z, k)], o[x]);
    }
#pragma unroll
    for (int x = 0; x < 4; ++x) kr[x][z * PB] = o[x];
  }
}

// Drive term of one block (zdrive_block): the sum of Im(conj(k~_a) (O y~)_a) over the
// block, O acting on the digit of padded stride PA, the other block digit KB.
template <int KB>
__device__ __forceinline__ float ldrive(const float2* __restrict__ O, const float2* __restrict__ xs,
                                        const float2* __restrict__ ys, int pb, int PA) {
  constexpr int PB = lpst(KB);
  float2 o[4][2];
#pragma unroll
  for (int a = 0; a < 4; ++a) zrow_ld<2>(O + 4 * a, o[a]);
  float g = 0.f;
#pragma unroll
  for (int z = 0; z < 4; ++z) {
    float2 yv[4], kv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      yv[a] = ys[pb + a * PA + z * PB];
      kv[a] = xs[pb + a * PA + z * PB];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      float2 v = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < 2; ++k) v = zfma(o[a][k], yv[zcol<true>(a, k)], v);
      g = fmaf(kv[a].x, v.y, g);
      g = fmaf(-kv[a].y, v.x, g);
    }
  }
  return g;
}

// Per-phase rows in shared memory (read as broadcasts; a runtime-indexed copy of the
// launch parameters would go to local memory): ka, kb, the term offsets L, R, A, B,
// the padded strides of ka and kb, and those of the other four digits in the
// bank-conflict-free mapping order of the tiled passes (make_phase).
constexpr int kLph = 12;
__device__ __forceinline__ void lphases_to_smem(const SlabPass& sp, int (*lph)[kLph]) {
  if (threadIdx.x < sp.nph) {
    const Phase& P = sp.ph[threadIdx.x];
    int* r = lph[threadIdx.x];
    r[0] = P.ka;
    r[1] = P.kb;
    r[2] = P.offL;
    r[3] = P.offR;
    r[4] = P.offA;
    r[5] = P.offB;
    r[6] = lpst(P.ka);
    r[7] = lpst(P.kb);
    for (int j = 0; j < 4; ++j) r[8 + j] = lpst(lord(P.ka, P.kb, j));
  }
}

// Padded position of thread tid's block in phase row r.
__device__ __forceinline__ int lpb(const int* r, int tid) {
  return (tid & 3) * r[8] + ((tid >> 2) & 3) * r[9] + ((tid >> 4) & 3) * r[10] + ((tid >> 6) & 3) * r[11];
}

// Every phase of the pass: ks = H_r ys.  Each phase ends with a barrier.
__device__ __forceinline__ void lpass(int nph, const int (*lph)[kLph], const float2* __restrict__ M,
                                      const float2* __restrict__ ys, float2* __restrict__ ks, int tid) {
#pragma unroll 1
  for (int q = 0; q < nph; ++q) {
    const int* r = lph[q];
    const int pb = lpb(r, tid), PA = r[6], oL = r[2], oR = r[3], oA = r[4], oB = r[5];
    switch (r[1]) {
#define SG_LCASE(B) case B: lphase<B>(M, ys, ks, pb, PA, oL, oR, oA, oB, q == 0); break;
      SG_LCASE(0) SG_LCASE(1) SG_LCASE(2) SG_LCASE(3) SG_LCASE(4) SG_LCASE(5)
#undef SG_LCASE
      default: break;
    }
    __syncthreads();
  }
}

// A drive on the first (type 0) or second (type 1) digit of phase row r: the block
// contraction of its operator O over thread tid's block of that phase.
__device__ __forceinline__ float ldrive_any(const int* r, int type, const float2* __restrict__ O,
                                            const float2* __restrict__ xs, const float2* __restrict__ ys,
                                            int tid) {
  const int pb = lpb(r, tid);
  const int PA = type == 0 ? r[6] : r[7];
  switch (type == 0 ? r[1] : r[0]) {
#define SG_LDCASE(B) case B: return ldrive<B>(O, xs, ys, pb, PA);
    SG_LDCASE(0) SG_LDCASE(1) SG_LDCASE(2) SG_LDCASE(3) SG_LDCASE(4) SG_LDCASE(5)
#undef SG_LDCASE
    default: return 0.f;
  }
}

// Per-thread constants of a launch: the phase factor pl(tid) of the low tile digits
// (FP64 product of the stage's phases, rounded once), the phase factors phi(j) of the
// two high digits and the global offsets hi(j) in shared memory, lo(tid) from the
// pass's offset table.
__device__ __forceinline__ void lsetup(const SlabPass& sp, const double2* __restrict__ phrow, float2* phi,
                                       int* ohi, float2& pl, int& olo) {
  const int tid = threadIdx.x;
  double pr = 1.0, pi = 0.0;
#pragma unroll
  for (int k = 2; k < 6; ++k) {
    const double2 e = phrow[sp.tphoff[k] + ((tid >> (2 * (5 - k))) & 3)];
    const double nr = pr * e.x - pi * e.y, ni = pr * e.y + pi * e.x;
    pr = nr;
    pi = ni;
  }
  pl = make_float2((float)pr, (float)pi);
  if (tid < LJ) {
    const double2 e0 = phrow[sp.tphoff[0] + (tid >> 2)], e1 = phrow[sp.tphoff[1] + (tid & 3)];
    phi[tid] = make_float2((float)(e0.x * e1.x - e0.y * e1.y), (float)(e0.x * e1.y + e0.y * e1.x));
    ohi[tid] = __ldg(sp.off + tid * kST);
  }
  olo = __ldg(sp.off + tid);
}

// Asynchronous copy of one tile's entries into dense shared memory (raw[t] = X[tile
// entry t]): thread tid copies the entry pairs (2m, 2m + 1), m = tid + 256 j (j < 8), by
// one 16-byte cp.async each.  A pair is contiguous and 16-byte aligned in the slab:
// the lowest tile digit has global stride 1 and every other digit a stride that is a
// multiple of 4 (checked on the host, with the slab's alignment), and the digit map is
// linear in the bits of t, so entry 2m sits at off(2 tid) + off(512 j).
__device__ __forceinline__ void lprefetch(const float2* __restrict__ X, long long base2,
                                          const int* __restrict__ ohi2, float2* raw, int tid) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float2* src = X + base2 + ohi2[j];
    const unsigned dst = (unsigned)__cvta_generic_to_shared(raw + 2 * (tid + kST * j));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void lprefetch_wait() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Whether every tile of the pass is one contiguous run of the slab (tile offset of
// entry t equal to t: by the linear digit map, true when it holds for t < 256 and for
// t = 256 j).  Call from every thread of the block.
__device__ __forceinline__ bool ltile_contig(const SlabPass& sp, int tid) {
  const bool ok = __ldg(sp.off + tid) == tid && (tid >= LJ || __ldg(sp.off + tid * kST) == tid * kST);
  return __syncthreads_and(ok) != 0;
}

// L2 prefetch of one tile of up to three arrays (descriptors in shared memory: base
// address and bytes per entry), so that the loads that follow a while later hit L2
// instead of waiting on DRAM.  A contiguous tile (tb: its first entry) goes by 8 KB
// bulk prefetches, one per thread, when 16-byte aligned; any other tile by one line
// prefetch per entry t = tid + 256 j of thread tid (bl: the thread's base, as in the
// epilogues), which a warp's lanes share by the 16-entry runs of the layout.  The
// arrays are read at run time so that no branch on the pass kind splits the tile loop.
struct LPf {
  const char* p;
  int esz;
};
__device__ __forceinline__ void lprefetch_l2(const LPf* __restrict__ pf, int npf, long long tb, long long bl,
                                             const int* __restrict__ ohi, bool contig, int tid) {
  constexpr int kChunk = 8192;
#pragma unroll 1
  for (int i = 0, c = tid; i < npf; ++i) {
    const char* p = pf[i].p;
    const int esz = pf[i].esz;
    const char* t0 = p + tb * esz;
    if (contig && (reinterpret_cast<unsigned long long>(t0) & 15ull) == 0) {
      const int nc = LT * esz / kChunk;
      if (c >= 0 && c < nc) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(t0 + (long long)c * kChunk), "r"(kChunk));
      c -= nc;
    } else {
#pragma unroll 1
      for (int j = 0; j < LJ; ++j) asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p + (bl + ohi[j]) * esz));
    }
  }
}

}  // namespace lean
}  // namespace
