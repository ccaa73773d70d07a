// Two consecutive TF32 core steps (k, k+1) of Algorithm 2 on the tcgen05
// tensor cores (kind::tf32: FP32 storage, operands with TF32 precision, FP32
// accumulation in TMEM).
//
// As in the BF16 pair kernel (step_tc2.cu), the four positions of a quad
// (bits k and k+1 free) are closed under both steps: a chunk of quads is
// read from HBM once and only y_{k+2} goes back.  kind::tf32 takes both
// operands K-major, while a TMA box of the planar intermediate lands with
// positions contiguous; so both steps run transposed, with the positions
// of the chunk as the M = 128 rows of the MMA:
//   D1^T = Y^T M_k^T        (positions x (2b + i_k))
//   D2^T = T M_{k+1}^T      (positions x (2c + i_{k+1}))
// A chunk is 64 quads: two runs h = 0, 1 of 32 consecutive quads.  For
// k >= 5 a run is 32 consecutive positions (128-byte rows of FP32) in each of
// the four (j_k, j_{k+1}) slices; for k = 3, 4 it is 32 / 2^k such rows of
// 2^k positions, one per value of the bits above k + 1.  With x the
// position in a run:
//   stage S  (two TMA boxes): box h, rows (j_{k+1}, a, j_k) of 32 positions
//            with a 128-byte swizzle (k >= 5), or, for k = 3, 4, rows
//            (hi, j_{k+1}, a, j_k) of 2^k positions, unswizzled
//   X        (TMEM, A of MMA1): lane m = 64 j_{k+1} + 32 h + x, column
//            K = 2a + j_k -- the stage read down its columns by the warp
//            that owns TMEM lanes 32 (2 j_{k+1} + h) .. + 31, stored with
//            tcgen05.st
//   B1       (shared memory, B of MMA1): M_k as rows 2b + i_k, K = 2a + j_k
//   D1^T     (TMEM) lane m, column 2b + i_k
//   T        (shared memory, A of MMA2, D1 rounded to TF32 -- where the
//            unfused sweep rounds the stored y_{k+1}): row
//            n = 64 i_k + 32 h + x, K = j_{k+1} r1p + b, so that each
//            thread stores runs of four consecutive K (16 bytes)
//   B2       (shared memory, B of MMA2): M_{k+1} as rows 2c + i_{k+1},
//            K = j_{k+1} r1p + b
//   D2^T     (TMEM) lane n, column 2c + i_{k+1}
//   y_{k+2}  (HBM) D2^T rounded to TF32, written by the thread of lane n:
//            for each (c, i_{k+1}) the 32 lanes of a warp store 32
//            consecutive positions of one plane (128 bytes)
// Ranks 8 to 32 in and between the steps, r_{k+2} <= 32.  MMA1 is M = 128,
// N = 2 r_{k+1} and K = 2 r_k, MMA2 is M = 128, N = 2 r_{k+2} and
// K = 2 r1p (r1p = r_{k+1} rounded up to 4, so that T's two halves start on
// 16-byte pieces); N is rounded up to 16 and K to 8 (the MMA's multiples),
// the padding rows and columns of the core tiles are zero and the padding
// columns of X are written as zeros.  K = 8 per instruction.
//
// Warp roles (a warp reaches the TMEM lanes 32 (w mod 4) .. + 31), connected
// by mbarriers:
//   warp 0       one lane issues the TMA loads into a ring of S stages
//   warp 1       allocates TMEM; one lane issues MMA1 of every chunk
//   warp 2       one lane issues MMA2 of every chunk (two issuing warps:
//                the MMAs of different chunks never wait behind each
//                other's dependencies, and their issue overlaps)
//   warps 4-7    stage -> X (two X buffers in TMEM)
//   warps 8-11, 12-15   two epilogue groups; group g takes the chunks
//                n = g (mod 2) and owns 128 TMEM columns (D1^T, D2^T) and a
//                T buffer: D1^T -> T, D2^T -> y_{k+2}
// Every wait is bounded (a clock budget, then a shared abort flag: every role
// leaves its loop, the CTA drains its copies, frees its TMEM and records
// QTT_ERR_TIMEOUT in this file's status word, read by qtt_sync_status).
#include <cstdlib>

#include "checked.cuh"
#include "qtt_internal.h"
#include "step_mma.h"
#include "tc_common.cuh"
#include "tf32.cuh"

namespace qtt {

__device__ int g_tcf_status = 0;

namespace {

using namespace tcx;

constexpr int kMaxGroups = 2;
constexpr int kGroupThreads = 128;
constexpr int kProducerWarp = 0;
constexpr int kMma1Warp = 1;
constexpr int kMma2Warp = 2;
constexpr int kXWarp0 = 4;                  // warps 4-7
constexpr int kXThreads = 128;
constexpr int kEpiWarp0 = 8;                // warps 8-15 (8-11 with one group)
constexpr int kThreads = 512;
constexpr int kQ = 64;                      // quads per chunk: two runs of 32
constexpr uint32_t kTmemCols = 512;
constexpr int kNx = 2;                      // X buffers
constexpr int kMaxStages = 8;
constexpr int kMaxRank = 40;                // 2 r <= 80: K and N of both MMAs
constexpr int kBarBytes = 512;
// Two shapes: ranks <= 32 with two epilogue groups (K, N <= 64), ranks <= 40
// with one (K, N <= 80; shared memory holds one T buffer and two stages).
// TMEM columns: X buffers at 0 and KM; group g's D1^T at 2 KM + 2 KM g, its
// D2^T KM further.

// Instruction descriptor of kind::tf32, M = 128: D FP32 (bits 4-5 = 1), A and
// B TF32 (bits 7-9 and 10-12 = 2), both K-major (bits 15, 16 clear), N >> 3
// at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
}

// D (TMEM) = A (TMEM, lanes = M rows, one TF32 per column) x B (shared
// memory descriptor), accumulating when acc != 0.
__device__ __forceinline__ void mma_tf32_ts(uint32_t dtmem, uint32_t atmem, uint64_t db,
                                            uint32_t idesc, int acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(dtmem),
      "r"(atmem), "l"(db), "r"(idesc), "r"(acc));
}
// D (TMEM) = A (shared memory descriptor) x B (shared memory descriptor).
__device__ __forceinline__ void mma_tf32_ss(uint32_t dtmem, uint64_t da, uint64_t db,
                                            uint32_t idesc, int acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}
// 32 lanes x 32 consecutive 32-bit TMEM columns from v[0..31].
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float *v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};\n" ::"r"(
          taddr),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]),
      "f"(v[8]), "f"(v[9]), "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]),
      "f"(v[15]), "f"(v[16]), "f"(v[17]), "f"(v[18]), "f"(v[19]), "f"(v[20]), "f"(v[21]),
      "f"(v[22]), "f"(v[23]), "f"(v[24]), "f"(v[25]), "f"(v[26]), "f"(v[27]), "f"(v[28]),
      "f"(v[29]), "f"(v[30]), "f"(v[31])
      : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float *v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16};\n" ::"r"(taddr),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]),
      "f"(v[8]), "f"(v[9]), "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]),
      "f"(v[15])
      : "memory");
}
// 32 lanes x NC consecutive 32-bit TMEM columns (NC = 64 or 80): loads of
// 32 (and 16) columns in flight, then one wait.
__device__ __forceinline__ void tmem_ld_x32(uint32_t taddr, uint32_t *r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_x16(uint32_t taddr, uint32_t *r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
template <int NC>
__device__ __forceinline__ void tmem_ldn(uint32_t taddr, float (&v)[NC]) {
  uint32_t r[NC];
  tmem_ld_x32(taddr, r);
  tmem_ld_x32(taddr + 32u, r + 32);
  if constexpr (NC == 80) tmem_ld_x16(taddr + 64u, r + 64);
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int e = 0; e < NC; ++e) v[e] = __uint_as_float(r[e]);
}

// Byte offset of element (row r, K index kk) of a K-major 128-byte-swizzled
// TF32 operand with `rows` rows: K in atoms of 32 elements (rows x 128
// bytes each), 16-byte piece (kk % 32) / 4 of row r at piece position
// ((kk % 32) / 4) ^ (r % 8).
__device__ __forceinline__ unsigned kmaj_off(int rows, int r, int kk) {
  return a_offset(rows, r, kk >> 2) + (unsigned)(kk & 3) * 4u;
}

struct Bars {
  unsigned long long full[kMaxStages], empty[kMaxStages];
  unsigned long long xready[kNx], xfree[kNx];
  unsigned long long d1full[kMaxGroups], tready[kMaxGroups], d2full[kMaxGroups], dfree[kMaxGroups];
  uint32_t tmem;
  int abort;
};
static_assert(sizeof(Bars) <= kBarBytes, "mbarrier block");

// Shared-memory plan (byte offsets from a 1024-aligned base): B1 (N1 rows x
// K1) and B2 (N2 rows x K2) K-major, per group a T buffer (128 rows x K2,
// K-major), the stage ring (two boxes of 4 r0 rows of 128 bytes).
struct PlanF {
  unsigned b1, b2, t[kMaxGroups], box, boxs, s0, stage, end;
  int n1, n2, k1, r1p, k2;
};
__host__ __device__ inline unsigned kmaj_bytes(int rows, int Kp) {
  return (unsigned)((Kp + 31) / 32) * (unsigned)rows * 128u;
}
__host__ __device__ inline PlanF make_plan_f(const StepTF2 &s, int S, int G) {
  PlanF p;
  p.k1 = (2 * s.r0 + 7) / 8 * 8;
  p.r1p = (s.r1 + 3) / 4 * 4;
  p.k2 = 2 * p.r1p;
  p.n1 = (2 * s.r1 + 15) / 16 * 16;
  p.n2 = (2 * s.r2 + 15) / 16 * 16;
  p.b1 = up1k(kBarBytes);
  p.b2 = up1k(p.b1 + kmaj_bytes(p.n1, p.k1));
  unsigned o = up1k(p.b2 + kmaj_bytes(p.n2, p.k2));
  for (int g = 0; g < G; ++g) {
    p.t[g] = o;
    o = up1k(o + kmaj_bytes(128, p.k2));
  }
  p.s0 = o;
  p.box = (unsigned)(4 * s.r0) * 128u;
  p.boxs = up1k(p.box);
  p.stage = 2 * p.boxs;
  p.end = p.s0 + (unsigned)S * p.stage;
  return p;
}

template <int G, int KM>
__global__ void __launch_bounds__(kThreads, 1)
    step_tc2f_kernel(const __grid_constant__ CUtensorMap tin, StepTF2 s, int S) {
  constexpr uint32_t kTmemX = 0, kTmemD = 2 * KM;
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char *base = smraw + ((1024u - (su32(smraw) & 1023u)) & 1023u);
  const PlanF P = make_plan_f(s, S, G);
  Bars &B = *reinterpret_cast<Bars *>(base);
  const unsigned base32 = su32(base);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wq = warp & 3;
  const int Kp1 = P.k1, Kp2 = P.k2;  // padded K of the two MMAs

  if (warp == kMma1Warp) {
    asm volatile(
        "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
            su32(&B.tmem)),
        "r"(kTmemCols)
        : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < kMaxStages; ++i) {
      mbar_init(su32(&B.full[i]), 1);
      mbar_init(su32(&B.empty[i]), kXThreads);
    }
    for (int i = 0; i < kNx; ++i) {
      mbar_init(su32(&B.xready[i]), kXThreads);
      mbar_init(su32(&B.xfree[i]), 1);
    }
    for (int i = 0; i < G; ++i) {
      mbar_init(su32(&B.d1full[i]), 1);
      mbar_init(su32(&B.tready[i]), kGroupThreads);
      mbar_init(su32(&B.d2full[i]), 1);
      mbar_init(su32(&B.dfree[i]), kGroupThreads);
    }
    B.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  // B1 = rows 0 .. 2 r1 - 1 of the first core tile, B2 = rows 0 .. N2 - 1 of
  // the second, as K-major operands (16-byte pieces of 4 TF32)
  for (int e = tid; e < P.n1 * (Kp1 / 4); e += kThreads) {
    const int r = e / (Kp1 / 4), kc = e % (Kp1 / 4);
    cpa16(base32 + P.b1 + a_offset(P.n1, r, kc), s.A1 + (size_t)r * Kp1 + 4 * kc, 16);
  }
  for (int e = tid; e < P.n2 * (Kp2 / 4); e += kThreads) {
    const int r = e / (Kp2 / 4), kc = e % (Kp2 / 4);
    cpa16(base32 + P.b2 + a_offset(P.n2, r, kc), s.A2 + (size_t)r * Kp2 + 4 * kc, 16);
  }
  cpa_commit();
  cpa_wait<0>();
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  const uint32_t tmem = B.tmem;
  volatile int *abort = &B.abort;
  const int64_t nq = s.N >> 2;
  const int64_t cpr = nq / kQ;
  const int64_t nchunks = cpr * s.nrhs;
  const int64_t NG = gridDim.x;
  const int lowmask = (1 << s.k) - 1;
  const int mine = nchunks > blockIdx.x ? (int)((nchunks - 1 - blockIdx.x) / NG + 1) : 0;
  const uint64_t tK = smem_desc(0, 16, 1024, 2);  // K-major, 128-byte swizzle, SBO 1024

  if (warp == kProducerWarp) {
    // ------------------------------------------------------------ TMA loads
    // box h of chunk n: quads q0 + 32 h .. + 31 (x = q & lowmask, hi = q >> k)
    if (lane == 0) {
      ChunkWalk cw(blockIdx.x, NG, cpr);
      int n = 0, st = 0;
      unsigned ph = 0;
      for (; n < mine; ++n, cw.next()) {
        if (n >= S && !wait_bar(su32(&B.empty[st]), ph ^ 1u, abort)) break;
        const unsigned fb = su32(&B.full[st]);
        expect_tx(fb, 2 * P.box);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          // the box: quads q .. q + 31 of right-hand side c
          const int64_t q = QTT_CK(cw.w * kQ + 32 * h, (s.N >> 2) - 31, 311);
          const int64_t cc = QTT_CK(cw.c, s.nrhs, 312);
          tma_load5(base32 + P.s0 + (unsigned)st * P.stage + (unsigned)h * P.boxs, &tin,
                    (int)(q & lowmask), 0, (int)(cc * s.r0), 0, (int)(q >> s.k), fb);
        }
        if (++st == S) {
          st = 0;
          ph ^= 1u;
        }
      }
      if (*abort) {
        // loads still in flight land before the CTA's shared memory goes
        volatile int never = 0;
        for (int m = n - S < 0 ? 0 : n - S; m < n; ++m)
          wait_bar(su32(&B.full[m % S]), (unsigned)(m / S) & 1u, &never);
      }
    }
  } else if (warp == kMma1Warp) {
    // ------------------------------------------------------------ MMA1 issue
    // A = X (TMEM columns + 8 ks), B = B1 (K step of 8 TF32 = 32 bytes inside
    // a 128-byte atom; atoms of 32 K are n1 x 128 bytes apart)
    if (lane == 0) {
      const uint32_t id = idesc_tf32(P.n1);
      const int nk = Kp1 / 8;
      for (int n = 0; n < mine; ++n) {
        const int g = n % G, b = n % kNx;
        if (!wait_bar(su32(&B.xready[b]), (unsigned)(n / kNx) & 1u, abort)) break;
        // D1^T of this group was last read by the T write of chunk n - G
        if (n >= G && !wait_bar(su32(&B.tready[g]), (unsigned)(n / G - 1) & 1u, abort)) break;
        tc_fence_after();
        const uint32_t d = tmem + kTmemD + (uint32_t)(g * 2 * KM);
        const uint32_t xa = tmem + kTmemX + (uint32_t)(b * KM);
        for (int ks = 0; ks < nk; ++ks) {
          const unsigned bb =
              base32 + P.b1 + (unsigned)((ks >> 2) * P.n1 * 128 + (ks & 3) * 32);
          mma_tf32_ts(d, xa + 8u * (uint32_t)ks, tK | ((bb >> 4) & 0x3FFFu), id, ks > 0);
        }
        mma_commit(su32(&B.xfree[b]));
        mma_commit(su32(&B.d1full[g]));
      }
    }
  } else if (warp == kMma2Warp) {
    // ------------------------------------------------------------ MMA2 issue
    // A = T (128 rows: atoms 128 x 128 bytes apart), B = B2 (atoms n2 x 128)
    if (lane == 0) {
      const uint32_t id = idesc_tf32(P.n2);
      const int nk = Kp2 / 8;
      for (int m = 0; m < mine; ++m) {
        const int g = m % G;
        if (!wait_bar(su32(&B.tready[g]), (unsigned)(m / G) & 1u, abort)) break;
        // D2^T of this group was last read by the y write of chunk m - G
        if (m >= G && !wait_bar(su32(&B.dfree[g]), (unsigned)(m / G - 1) & 1u, abort)) break;
        tc_fence_after();
        const uint32_t d = tmem + kTmemD + (uint32_t)(g * 2 * KM + KM);
        const unsigned tb = base32 + P.t[g];
        for (int ks = 0; ks < nk; ++ks) {
          const unsigned aa = tb + (unsigned)((ks >> 2) * 128 * 128 + (ks & 3) * 32);
          const unsigned bb =
              base32 + P.b2 + (unsigned)((ks >> 2) * P.n2 * 128 + (ks & 3) * 32);
          mma_tf32_ss(d, tK | ((aa >> 4) & 0x3FFFu), tK | ((bb >> 4) & 0x3FFFu), id, ks > 0);
        }
        mma_commit(su32(&B.d2full[g]));
      }
    }
  } else if (warp >= kXWarp0 && warp < kEpiWarp0) {
    // ------------------------------------------------------------ stage -> X
    // warp q = w - 4 owns TMEM lanes 32 q .. + 31 = positions (j1, h) =
    // (q / 2, q % 2), t = lane: column kr of X is row R = j1 2 r0 + kr of box
    // h at position t (columns 2 r0 .. KM - 1 are written as zeros).  k >= 5: a
    // warp reads whole 128-byte rows, row R at swizzle phase R % 8.
    // k = 3, 4: position t is (hi, x) = (t / 2^k, t % 2^k), at
    // ((hi 4 r0 + R) 2^k + x) floats.
    const int j1 = wq >> 1, h = wq & 1;
    const int kin = 2 * s.r0;
    const bool swz = s.k >= 5;
    const unsigned xc = (unsigned)lane >> 2, xl = (unsigned)(lane & 3) * 4u;
    const unsigned rot = (unsigned)(j1 * kin);
    unsigned pre[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) pre[c] = ((xc ^ (((unsigned)c + rot) & 7u)) << 4) + xl;
    const unsigned rstride = 4u << s.k;  // k = 3, 4: bytes per row
    const unsigned plain =
        ((((unsigned)lane >> s.k) * 4u * (unsigned)s.r0) << s.k) * 4u +
        ((unsigned)lane & ((1u << s.k) - 1u)) * 4u;
    const uint32_t tl = tmem + ((uint32_t)(32 * wq) << 16) + kTmemX;
    int st = 0;
    unsigned ph = 0;
    for (int n = 0; n < mine; ++n) {
      const int b = n % kNx;
      if (!wait_bar(su32(&B.full[st]), ph, abort)) break;
      if (n >= kNx && !wait_bar(su32(&B.xfree[b]), (unsigned)(n / kNx - 1) & 1u, abort)) break;
      const unsigned char *box = base + P.s0 + (unsigned)st * P.stage + (unsigned)h * P.boxs;
      float v[KM];
      if (swz) {
        const unsigned char *rows = box + rot * 128u;
#pragma unroll
        for (int kr = 0; kr < KM; ++kr)
          v[kr] = kr < kin ? *reinterpret_cast<const float *>(rows + kr * 128 + pre[kr & 7]) : 0.f;
      } else {
        const unsigned char *rows = box + plain + rot * rstride;
#pragma unroll
        for (int kr = 0; kr < KM; ++kr)
          v[kr] = kr < kin ? *reinterpret_cast<const float *>(rows + (unsigned)kr * rstride) : 0.f;
      }
      mbar_arrive(su32(&B.empty[st]));  // the stage has been read
      const uint32_t xb = tl + (uint32_t)(b * KM);
      if (Kp1 <= 16) {
        tmem_st16(xb, v);
      } else {
        tmem_st32(xb, v);
        if (Kp1 > 32) tmem_st32(xb + 32u, v + 32);
        if constexpr (KM == 80)
          if (Kp1 > 64) tmem_st16(xb + 64u, v + 64);
      }
      asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
      tc_fence_before();
      mbar_arrive(su32(&B.xready[b]));
      if (++st == S) {
        st = 0;
        ph ^= 1u;
      }
    }
  } else if (warp >= kEpiWarp0 && warp < kEpiWarp0 + 4 * G) {
    // ------------------------------------------------------------ epilogue
    // T write: thread = input position m = 64 j1 + 32 h + x (j1 = q / 2,
    // h = q % 2, x = lane); y_{k+2} write: thread = output position
    // n = 64 i + 32 h + x (i = q / 2).
    const int g = (warp - kEpiWarp0) >> 2;
    const int qhi = wq >> 1, qh = wq & 1;
    const uint32_t d1 = tmem + ((uint32_t)(32 * wq) << 16) + kTmemD + (uint32_t)(g * 2 * KM);
    const uint32_t d2 = d1 + (uint32_t)KM;
    const unsigned x7 = (unsigned)lane & 7u;
    unsigned char *T = base + P.t[g];
    const unsigned tk0 = (unsigned)(qhi * P.r1p);  // this thread's half of T's K
    const int64_t bit1 = (int64_t)1 << (s.k + 1);
    ChunkWalk cw(blockIdx.x + (int64_t)g * NG, (int64_t)G * NG, cpr);
    for (int n = g; n < mine; n += G, cw.next()) {
      const unsigned par = (unsigned)(n / G) & 1u;
      if (epi_any<kGroupThreads>(!wait_bar(su32(&B.d1full[g]), par, abort), g)) break;
      tc_fence_after();
      {
        // D1^T column 2b + i -> T row 64 i + 32 h + x, K = j1 r1p + b: four
        // consecutive b per 16-byte piece, at (K / 32) 16384 + row 128 +
        // ((K / 4 % 8) ^ (row % 8)) 16 (columns b >= r1 of D1^T are zero: the
        // core tile's padding rows).  T was last read by MMA2 of chunk
        // n - G, complete before this group's y write of that chunk began.
        float v[KM];
        tmem_ldn<KM>(d1, v);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          unsigned char *trow = T + (unsigned)(64 * i + 32 * qh + lane) * 128u;
#pragma unroll
          for (int p = 0; p < KM / 8; ++p) {
            if (4 * p < P.r1p) {
              const unsigned kk = tk0 + 4u * (unsigned)p;
              float4 w;
              w.x = tf32_rn(v[8 * p + i]);
              w.y = tf32_rn(v[8 * p + 2 + i]);
              w.z = tf32_rn(v[8 * p + 4 + i]);
              w.w = tf32_rn(v[8 * p + 6 + i]);
              *reinterpret_cast<float4 *>(trow + (kk >> 5) * 16384u +
                                          ((((kk >> 2) & 7u) ^ x7) << 4)) = w;
            }
          }
        }
      }
      fence_async_smem();
      tc_fence_before();
      mbar_arrive(su32(&B.tready[g]));
      if (epi_any<kGroupThreads>(!wait_bar(su32(&B.d2full[g]), par, abort), g)) break;
      tc_fence_after();
      {
        // D2^T column 2c + i1 -> y_{k+2}[rhs][c][position of quad
        // q0 + 32 h + x with bits (k, k+1) = (i, i1)]
        float v[KM];
        tmem_ldn<KM>(d2, v);
        tc_fence_before();
        mbar_arrive(su32(&B.dfree[g]));  // D2^T is in registers
        const int64_t qq = cw.w * kQ + 32 * qh + lane;
        // pos and pos + 2^(k+1) in range, right-hand side c in range
        const int64_t pos = QTT_CK(((qq >> s.k) << (s.k + 2)) | ((int64_t)qhi << s.k) | (qq & lowmask),
                                   s.N - bit1, 313);
        float *y = s.out + QTT_CK(cw.c, s.nrhs, 314) * s.out_rhs_stride + pos;
#pragma unroll
        for (int c = 0; c < KM / 2; ++c) {
          if (c < s.r2) {
            y[0] = tf32_rn(v[2 * c]);
            y[bit1] = tf32_rn(v[2 * c + 1]);
            y += s.N;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kMma1Warp) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
  }
  if (tid == 0 && *abort) atomicCAS(&g_tcf_status, 0, (int)QTT_ERR_TIMEOUT);
}

constexpr size_t kSmemLimit = 227 * 1024;

// 5-D view of the planar FP32 input [P][N] for the pair at bit k: dims
// (x: bits 0..k-1, a: bit k, P, b: bit k+1, hi: bits k+2..), box
// (min(2^k, 32), 2, r0, 2, 32 / min(2^k, 32)) -- smem rows (hi, b, P, a) of
// 32 positions with a 128-byte swizzle (k >= 5), or of 2^k positions
// unswizzled (k = 3, 4).
bool encode_view_f32(CUtensorMap *m, const void *ptr, int k, int64_t N, int64_t planes,
                     int box_p) {
  const cuuint64_t dims[5] = {(cuuint64_t)1 << k, 2, (cuuint64_t)planes, 2,
                              (cuuint64_t)(N >> (k + 2))};
  const cuuint64_t strides[4] = {((cuuint64_t)1 << k) * 4, (cuuint64_t)N * 4,
                                 ((cuuint64_t)1 << (k + 1)) * 4, ((cuuint64_t)1 << (k + 2)) * 4};
  const cuuint32_t bx = k >= 5 ? 32u : (1u << k);
  const cuuint32_t box[5] = {bx, 2, (cuuint32_t)box_p, 2, 32u / bx};
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  const PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return false;
  return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<void *>(ptr), dims, strides, box,
                es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                k >= 5 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int stages_for_f(const StepTF2 &s, int G) {
  const PlanF p0 = make_plan_f(s, 0, G);
  if (p0.end + 2 * p0.stage + 1024 > kSmemLimit) return 0;
  const int S = (int)((kSmemLimit - 1024 - p0.end) / p0.stage);
  return S > kMaxStages ? kMaxStages : S;
}

template <int G, int KM>
cudaError_t launch_tc2f(const CUtensorMap &tin, const StepTF2 &s, cudaStream_t st) {
  const int S = stages_for_f(s, G);
  if (S < 2) return cudaErrorNotSupported;
  const size_t smem = make_plan_f(s, S, G).end + 1024;
  static cudaError_t attr = cudaFuncSetAttribute(
      step_tc2f_kernel<G, KM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit);
  if (attr != cudaSuccess) return attr;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t nchunks = (s.N >> 2) / kQ * s.nrhs;
  const unsigned grid = (unsigned)(nchunks < sms ? nchunks : sms);
  step_tc2f_kernel<G, KM><<<grid, kThreads, smem, st>>>(tin, s, S);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

bool tc2f_steps_eligible(int k, int r0, int r1, int r2, int64_t N) {
  // k >= 3: rows of at least 8 positions (32 bytes); whole chunks of 64
  // quads; ranks 8..40 in and between the steps (K and N of the MMAs at most
  // 80, at least 16 rows of useful work), r2 <= 40
  return k >= 3 && N >= 1024 && ((int64_t)1 << (k + 2)) < N && r0 >= 8 && r0 <= kMaxRank &&
         r1 >= 8 && r1 <= kMaxRank && r2 >= 1 && r2 <= kMaxRank;
}

cudaError_t launch_step_tc2_tf32(const StepTF2 &s, cudaStream_t st) {
  if (!tc2f_steps_eligible(s.k, s.r0, s.r1, s.r2, s.N)) return cudaErrorNotSupported;
  if (s.in_rhs_stride != (int64_t)s.r0 * s.N || s.out_rhs_stride != (int64_t)s.r2 * s.N)
    return cudaErrorNotSupported;
  CUtensorMap tin;
  if (!encode_view_f32(&tin, s.in, s.k, s.N, s.nrhs * s.r0, s.r0)) return cudaErrorNotSupported;
  // ranks <= 32: two epilogue groups; up to 40: one (shared memory)
  if (s.r0 <= 32 && s.r1 <= 32 && s.r2 <= 32) return launch_tc2f<2, 64>(tin, s, st);
  return launch_tc2f<1, 80>(tin, s, st);
}

cudaError_t tcf_status_take(int *status) {
  int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(status, g_tcf_status, sizeof(int));
  if (e == cudaSuccess && *status != 0) e = cudaMemcpyToSymbol(g_tcf_status, &zero, sizeof(int));
  return e;
}

}  // namespace qtt
