// Two consecutive TF32 core steps (k, k+1) of Algorithm 2 on the tcgen05
// tensor cores (kind::tf32: FP32 storage, operands with TF32 precision, FP32
// accumulation in TMEM).
//
// The structure is that of the BF16 pair kernel (step_tc2.cu): the four
// positions of a quad (bits k and k+1 free) are closed under both steps, a
// chunk of quads is read from HBM once and only y_{k+2} goes back.  The
// difference is the operand layout: kind::tf32 takes both operands K-major,
// while a TMA box of the planar intermediate lands MN-major (positions
// contiguous).  So a transposer role sits between the TMA load and the first
// MMA, and the epilogue writes the second MMA's operand K-major directly.
// A chunk is 64 quads: two runs h = 0, 1 of 32 consecutive quads, each 32
// consecutive positions (128-byte rows of FP32) in the four (j_k, j_{k+1})
// slices, so k >= 5.  With x the position in a run:
//   stage S  (two TMA boxes, MN-major, 128-byte swizzle): box h, rows
//            (j_{k+1}, a, j_k) of 32 positions
//   Bk       (transposer): row n = 64 j_{k+1} + 32 h + x, K = 2a + j_k,
//            K-major
//   D1 = M_k Bk      TMEM lanes 2b + i_k, columns 64 j_{k+1} + 32 h + x
//   T        (epilogue, D1 rounded to TF32 -- where the unfused sweep rounds
//            the stored y_{k+1}): row n = 64 i_k + 32 h + x, K = 2b + j_{k+1}
//   D2 = M_{k+1} T   TMEM lanes 2c + i_{k+1}, columns 64 i_k + 32 h + x
//   O        two output tiles (in T's buffer, once MMA2 has read T), tile h
//            rows (i_{k+1}, i_k, c) of 32 positions (rounded to TF32) -- two
//            TMA stores into y_{k+2}
// Both MMAs are M = 128 (rows 2r + i; rows past 2r <= 64 are zero padding of
// the core tiles, so only TMEM lanes 0-63 are ever read), N = 128, K = 8 per
// instruction.  The core tiles M_k and M_{k+1} sit in TMEM (A operands,
// columns = K), so an MMA reads only its B operand from shared memory.
//
// Warp roles (a warp reaches the TMEM lanes 32 (w mod 4) .. + 31), connected
// by mbarriers:
//   warps 0-1, 4-5, 8-9   three epilogue groups of two warps (TMEM lanes
//               0-63); group g takes the chunks n = g (mod 3) and owns 128
//               TMEM columns (D1, then D2 of the same chunk): D1 -> T, D2 ->
//               O -> TMA stores
//   warp 2      one lane issues the TMA loads into a ring of S stages
//   warp 3      allocates TMEM; one lane issues MMA1 of every chunk
//   warp 12     one lane issues MMA2 of every chunk (two issuing warps: the
//               two MMAs of different chunks never wait behind each other's
//               dependencies, and their issue overlaps)
//   warps 6-7, 10-11, 13-15   transpose stage -> Bk (two Bk buffers)
// Every wait is bounded (a clock budget, then a shared abort flag: every role
// leaves its loop, the CTA drains its copies, frees its TMEM and records
// QTT_ERR_TIMEOUT in this file's status word, read by qtt_sync_status).
#include <cstdlib>

#include "qtt_internal.h"
#include "step_mma.h"
#include "tc_common.cuh"

namespace qtt {

__device__ int g_tcf_status = 0;

namespace {

using namespace tcx;

constexpr int kGroups = 3;
constexpr int kGroupThreads = 64;
constexpr int kProducerWarp = 2;
constexpr int kMmaWarp = 3;                 // MMA1
constexpr int kMma2Warp = 12;               // MMA2
constexpr int kXWarps = 7;                  // transposer warps 6, 7, 10, 11, 13-15
constexpr int kXItems = 10;                 // ceil(64 / 7) Bk pieces per lane and chunk
constexpr int kXThreads = 32 * kXWarps;
constexpr int kThreads = 512;
constexpr int kQ = 64;                      // quads per chunk: two runs of 32
constexpr int kCols = 2 * kQ;               // N of both MMAs
constexpr uint32_t kTmemCols = 512;         // D of three groups (384), M_k and M_{k+1} (128)
constexpr uint32_t kTmemA1 = 384, kTmemA2 = 448;
constexpr int kNbk = 2;                     // Bk buffers
constexpr int kMaxStages = 8;
constexpr int kMaxRank = 32;                // 2 r <= 64: K of both MMAs, two K atoms
constexpr int kBarBytes = 512;

// Instruction descriptor of kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32
// (bits 7-9 and 10-12 = 2), both K-major (bits 15, 16 clear), N >> 3 at bit
// 17, M >> 4 at bit 24.
constexpr uint32_t kIdescF = (1u << 4) | (2u << 7) | (2u << 10) | (0u << 15) | (0u << 16) |
                             ((uint32_t)(kCols >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

// D (TMEM) = A (TMEM, lanes = M rows, one TF32 per column) x B (shared
// memory descriptor), accumulating when acc != 0.
__device__ __forceinline__ void mma_tf32_ts(uint32_t dtmem, uint32_t atmem, uint64_t db, int acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(dtmem),
      "r"(atmem), "l"(db), "r"(kIdescF), "r"(acc));
}
// 32 lanes x 32 consecutive 32-bit TMEM columns from v[0..31].
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float (&v)[32]) {
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
// Two loads of 32 columns in flight, then one wait.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float (&v)[64]) {
  uint32_t r[64];
#pragma unroll
  for (int h = 0; h < 2; ++h)
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[32 * h + 0]), "=r"(r[32 * h + 1]), "=r"(r[32 * h + 2]), "=r"(r[32 * h + 3]),
          "=r"(r[32 * h + 4]), "=r"(r[32 * h + 5]), "=r"(r[32 * h + 6]), "=r"(r[32 * h + 7]),
          "=r"(r[32 * h + 8]), "=r"(r[32 * h + 9]), "=r"(r[32 * h + 10]), "=r"(r[32 * h + 11]),
          "=r"(r[32 * h + 12]), "=r"(r[32 * h + 13]), "=r"(r[32 * h + 14]),
          "=r"(r[32 * h + 15]), "=r"(r[32 * h + 16]), "=r"(r[32 * h + 17]),
          "=r"(r[32 * h + 18]), "=r"(r[32 * h + 19]), "=r"(r[32 * h + 20]),
          "=r"(r[32 * h + 21]), "=r"(r[32 * h + 22]), "=r"(r[32 * h + 23]),
          "=r"(r[32 * h + 24]), "=r"(r[32 * h + 25]), "=r"(r[32 * h + 26]),
          "=r"(r[32 * h + 27]), "=r"(r[32 * h + 28]), "=r"(r[32 * h + 29]),
          "=r"(r[32 * h + 30]), "=r"(r[32 * h + 31])
        : "r"(taddr + 32u * (uint32_t)h));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int e = 0; e < 64; ++e) v[e] = __uint_as_float(r[e]);
}

// Round to TF32 (10 explicit mantissa bits), nearest even, as the unfused
// TF32 sweep stores its intermediates: the conversion instruction, its 13
// low bits cleared.
__device__ __forceinline__ float tf32_rne(float x) {
  unsigned r;
  asm("cvt.rn.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r & 0xffffe000u);
}

// Byte offset of element (row r, K index kk) of a K-major 128-byte-swizzled
// TF32 operand with `rows` rows: K in atoms of 32 elements (rows x 128
// bytes each), 16-byte piece (kk % 32) / 4 of row r at piece position
// ((kk % 32) / 4) ^ (r % 8).
__device__ __forceinline__ unsigned kmaj_off(int rows, int r, int kk) {
  return a_offset(rows, r, kk >> 2) + (unsigned)(kk & 3) * 4u;
}
// Byte offset of position x (0..31) of row R in an MN-major tile of
// 128-byte rows (the layout a 128-byte-swizzled TMA box of 32 FP32 values per
// row lands in, and the store box reads).
__device__ __forceinline__ unsigned row_off(int R, int x) {
  return (unsigned)R * 128u + ((unsigned)(((x >> 2) ^ (R & 7)) << 4)) + (unsigned)(x & 3) * 4u;
}

struct Bars {
  unsigned long long full[kMaxStages], empty[kMaxStages];
  unsigned long long bkready[kNbk], bkfree[kNbk];
  unsigned long long d1full[kGroups], tready[kGroups], d2full[kGroups], dfree[kGroups];
  uint32_t tmem;
  int abort;
};
static_assert(sizeof(Bars) <= kBarBytes, "mbarrier block");

// Shared-memory plan (byte offsets from a 1024-aligned base): two Bk buffers
// (128 rows x Kp1, K-major), per group one buffer for T (128 rows x Kp2,
// K-major) and then O (two tiles of 4 r2 rows of 128 bytes, 1024-aligned),
// the stage ring (two boxes of 4 r0 rows of 128 bytes).
struct PlanF {
  unsigned bk[kNbk], to[kGroups], ohalf, box, s0, stage, end;
};
__host__ __device__ inline unsigned kmaj_bytes(int rows, int Kp) {
  return (unsigned)((Kp + 31) / 32) * (unsigned)rows * 128u;
}
__host__ __device__ inline PlanF make_plan_f(const StepTF2 &s, int S) {
  PlanF p;
  const int Kp1 = 2 * s.r0, Kp2 = 2 * s.r1;
  p.bk[0] = up1k(kBarBytes);
  for (int b = 1; b < kNbk; ++b) p.bk[b] = up1k(p.bk[b - 1] + kmaj_bytes(kCols, Kp1));
  p.ohalf = up1k((unsigned)(4 * s.r2) * 128u);
  const unsigned tbytes = kmaj_bytes(kCols, Kp2), obytes = 2 * p.ohalf;
  const unsigned tob = tbytes > obytes ? tbytes : obytes;
  p.to[0] = up1k(p.bk[kNbk - 1] + kmaj_bytes(kCols, Kp1));
  for (int g = 1; g < kGroups; ++g) p.to[g] = up1k(p.to[g - 1] + tob);
  p.s0 = up1k(p.to[kGroups - 1] + tob);
  p.box = (unsigned)(4 * s.r0) * 128u;
  p.stage = up1k(2 * p.box);
  p.end = p.s0 + (unsigned)S * p.stage;
  return p;
}

__global__ void __launch_bounds__(kThreads, 1)
    step_tc2f_kernel(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tout,
                     StepTF2 s, int S) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char *base = smraw + ((1024u - (su32(smraw) & 1023u)) & 1023u);
  const PlanF P = make_plan_f(s, S);
  Bars &B = *reinterpret_cast<Bars *>(base);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wq = warp & 3;
  const int Kp1 = 2 * s.r0, Kp2 = 2 * s.r1;

  if (warp == kMmaWarp) {
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
    for (int i = 0; i < kNbk; ++i) {
      mbar_init(su32(&B.bkready[i]), kXThreads);
      mbar_init(su32(&B.bkfree[i]), 1);
    }
    for (int i = 0; i < kGroups; ++i) {
      mbar_init(su32(&B.d1full[i]), 1);
      mbar_init(su32(&B.tready[i]), kGroupThreads);
      mbar_init(su32(&B.d2full[i]), 1);
      mbar_init(su32(&B.dfree[i]), kGroupThreads);
    }
    B.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = B.tmem;
  // core tiles into TMEM: warps 0-3 write lanes 32 w .. + 31 (row r of M_k
  // and M_{k+1}, K along the columns; rows past 2 r_out are the zeros of the
  // packed copy)
  if (warp < 4) {
    const int r = 32 * warp + lane;
    const uint32_t tl = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float v[32];
      if (32 * h < Kp1) {
        const float4 *src = reinterpret_cast<const float4 *>(s.A1 + (size_t)r * Kp1 + 32 * h);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 t = src[q];
          v[4 * q] = t.x, v[4 * q + 1] = t.y, v[4 * q + 2] = t.z, v[4 * q + 3] = t.w;
        }
        tmem_st32(tl + kTmemA1 + 32u * (uint32_t)h, v);
      }
      if (32 * h < Kp2) {
        const float4 *src = reinterpret_cast<const float4 *>(s.A2 + (size_t)r * Kp2 + 32 * h);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 t = src[q];
          v[4 * q] = t.x, v[4 * q + 1] = t.y, v[4 * q + 2] = t.z, v[4 * q + 3] = t.w;
        }
        tmem_st32(tl + kTmemA2 + 32u * (uint32_t)h, v);
      }
    }
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  const unsigned base32 = su32(base);
  volatile int *abort = &B.abort;
  const int64_t nq = s.N >> 2;
  const int64_t cpr = nq / kQ;
  const int64_t nchunks = cpr * s.nrhs;
  const int64_t NG = gridDim.x;
  const int lowmask = (1 << s.k) - 1;
  const int mine = nchunks > blockIdx.x ? (int)((nchunks - 1 - blockIdx.x) / NG + 1) : 0;

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
          const int64_t q = cw.w * kQ + 32 * h;
          tma_load5(base32 + P.s0 + (unsigned)st * P.stage + (unsigned)h * P.box, &tin,
                    (int)(q & lowmask), 0, (int)(cw.c * s.r0), 0, (int)(q >> s.k), fb);
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
  } else if (warp == kMmaWarp || warp == kMma2Warp) {
    // ------------------------------------------------------------ MMA issue
    // B operands K-major, 128-byte swizzle: a K step of 8 TF32 moves 32 bytes
    // inside a 128-byte atom; atoms of 32 K are 128 x 128 bytes apart.  A
    // operands: TMEM columns kTmemA1/A2 + 8 ks.
    if (lane == 0) {
      const uint64_t tK = smem_desc(0, 16, 1024, 2);
      if (warp == kMmaWarp) {
        const int nk1 = Kp1 / 8;
        for (int n = 0; n < mine; ++n) {
          // D of this group was last read by the O write of chunk n - 3
          const int g = n % kGroups, b = n % kNbk;
          if (!wait_bar(su32(&B.bkready[b]), (unsigned)(n / kNbk) & 1u, abort)) break;
          if (n >= kGroups &&
              !wait_bar(su32(&B.dfree[g]), (unsigned)(n / kGroups - 1) & 1u, abort))
            break;
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(g * kCols);
          const unsigned bkb = base32 + P.bk[b];
          for (int ks = 0; ks < nk1; ++ks) {
            const unsigned bb = bkb + (unsigned)((ks >> 2) * kCols * 128 + (ks & 3) * 32);
            mma_tf32_ts(d, tmem + kTmemA1 + 8u * (uint32_t)ks, tK | ((bb >> 4) & 0x3FFFu),
                        ks > 0);
          }
          mma_commit(su32(&B.bkfree[b]));
          mma_commit(su32(&B.d1full[g]));
        }
      } else {
        const int nk2 = Kp2 / 8;
        for (int m = 0; m < mine; ++m) {
          // D1 of chunk m has been read (T written): D2 overwrites it
          const int gm = m % kGroups;
          if (!wait_bar(su32(&B.tready[gm]), (unsigned)(m / kGroups) & 1u, abort)) break;
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(gm * kCols);
          const unsigned tb = base32 + P.to[gm];
          for (int ks = 0; ks < nk2; ++ks) {
            const unsigned bb = tb + (unsigned)((ks >> 2) * kCols * 128 + (ks & 3) * 32);
            mma_tf32_ts(d, tmem + kTmemA2 + 8u * (uint32_t)ks, tK | ((bb >> 4) & 0x3FFFu),
                        ks > 0);
          }
          mma_commit(su32(&B.d2full[gm]));
        }
      }
    }
  } else if (wq >= 2 || warp >= 13) {
    // ------------------------------------------------------------ transposer
    // box h, row R = j1 (2 r0) + kr (kr = 2a + j0), 32 positions x; Bk row
    // n = 64 j1 + 32 h + x, K index kr.  Lane x of transposer warp xw gathers
    // the four K values of the 16-byte Bk pieces jp = xw, xw + 7, ... (jp =
    // (2 h + j1) npiece + piece): rows R .. R+3 at position x (a warp reads
    // whole 128-byte stage rows), one 16-byte store (eight consecutive Bk
    // rows of a warp land in eight distinct bank groups under the swizzle).
    // R is a multiple of 4, so row R + e has swizzle phase (R & 4) | e.  All
    // loads of a chunk are issued before its stores.
    const int xw = warp < 12 ? ((warp >> 2) - 1) * 2 + (warp & 1) : warp - 9;  // 0..6
    const int lnp = Kp1 == 64 ? 4 : 3;                  // log2(npiece), npiece = Kp1 / 4
    const int njp = 4 << lnp;
    const unsigned xc = (unsigned)lane >> 2;
    unsigned ce[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) ce[e] = (unsigned)e * 128u + ((xc ^ (unsigned)e) << 4);
    const unsigned ldx = (unsigned)(lane & 3) * 4u, stx = (unsigned)lane * 128u;
    const unsigned x7 = (unsigned)lane & 7u;
    int st = 0;
    unsigned ph = 0;
    for (int n = 0; n < mine; ++n) {
      const int b = n % kNbk;
      if (!wait_bar(su32(&B.full[st]), ph, abort)) break;
      if (n >= kNbk && !wait_bar(su32(&B.bkfree[b]), (unsigned)(n / kNbk - 1) & 1u, abort)) break;
      const unsigned char *stg = base + P.s0 + (unsigned)st * P.stage + ldx;
      unsigned char *bk = base + P.bk[b] + stx;
      float4 v[kXItems];
#pragma unroll
      for (int t = 0; t < kXItems; ++t) {
        const int jp = xw + kXWarps * t;
        if (jp < njp) {
          const unsigned hj = (unsigned)jp >> lnp, pc = (unsigned)jp & ((1u << lnp) - 1u);
          const unsigned R = (hj & 1u) * (unsigned)Kp1 + 4u * pc;
          const unsigned char *rb = stg + (hj >> 1) * P.box + R * 128u;
          const unsigned flip = (R & 4u) << 4;
          v[t].x = *reinterpret_cast<const float *>(rb + (ce[0] ^ flip));
          v[t].y = *reinterpret_cast<const float *>(rb + (ce[1] ^ flip));
          v[t].z = *reinterpret_cast<const float *>(rb + (ce[2] ^ flip));
          v[t].w = *reinterpret_cast<const float *>(rb + (ce[3] ^ flip));
        }
      }
#pragma unroll
      for (int t = 0; t < kXItems; ++t) {
        const int jp = xw + kXWarps * t;
        if (jp < njp) {
          // n = 64 j1 + 32 h + x: (pc / 8) 16384 + j1 8192 + h 4096 + x 128 + swizzled piece
          const unsigned hj = (unsigned)jp >> lnp, pc = (unsigned)jp & ((1u << lnp) - 1u);
          *reinterpret_cast<float4 *>(bk + (pc >> 3) * 16384u + (hj & 1u) * 8192u +
                                      (hj >> 1) * 4096u + ((((pc & 7u) ^ x7)) << 4)) = v[t];
        }
      }
      fence_async_smem();  // Bk to the tensor core; the stage back to TMA
      mbar_arrive(su32(&B.bkready[b]));
      mbar_arrive(su32(&B.empty[st]));
      if (++st == S) {
        st = 0;
        ph ^= 1u;
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int g = warp >> 2;
    const int row = 32 * wq + lane;  // TMEM lane = D row (0..63)
    const bool leader = wq == 0 && lane == 0;
    unsigned char *TO = base + P.to[g];
    const uint32_t dg = tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)(g * kCols);
    ChunkWalk cw(blockIdx.x + (int64_t)g * NG, (int64_t)kGroups * NG, cpr);
    for (int n = g; n < mine; n += kGroups, cw.next()) {
      const unsigned par = (unsigned)(n / kGroups) & 1u;
      if (epi_any<kGroupThreads>(!wait_bar(su32(&B.d1full[g]), par, abort), g)) break;
      tc_fence_after();
      if (leader) bulk_wait_read0();  // the group's previous stores have read the buffer
      epi_sync<kGroupThreads>(g);
      // D1 -> T: row 2b + i of D1, column 64 j1 + 32 h + x -> T row
      // n = 64 i + 32 h + x', K = 2b + j1, x' = x ^ 4i (the two lanes of a
      // pair, same K, write rows of different swizzle phase), at
      // (K / 32) 16384 + n 128 + ((K / 4 % 8) ^ (n % 8)) 16 + (K % 4) 4
#pragma unroll
      for (int j1 = 0; j1 < 2; ++j1) {
        float v[64];
        tmem_ld64(dg + 64u * (uint32_t)j1, v);
        if (row < Kp2) {
          const unsigned i = (unsigned)row & 1u;
          const unsigned i9 = i << 9;
          const unsigned kr = ((unsigned)row & ~1u) + (unsigned)j1;
          const unsigned tb = (kr >> 5) * 16384u + i * 8192u + (kr & 3u) * 4u;
          const unsigned k74 = ((((kr >> 2) & 7u) ^ (i << 2))) << 4;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            unsigned char *tp = TO + tb + 4096u * (unsigned)h;
#pragma unroll
            for (int x = 0; x < 32; ++x) {
              const float val = i ? v[32 * h + (x ^ 4)] : v[32 * h + x];
              *reinterpret_cast<float *>(tp + ((((unsigned)x << 7) ^ i9) +
                                               (k74 ^ (((unsigned)x & 7u) << 4)))) =
                  tf32_rne(val);
            }
          }
        }
      }
      fence_async_smem();
      tc_fence_before();
      mbar_arrive(su32(&B.tready[g]));
      if (epi_any<kGroupThreads>(!wait_bar(su32(&B.d2full[g]), par, abort), g)) break;
      tc_fence_after();
      // D2 -> O (MMA2 has read T): row 2c + i1 of D2, column 64 i + 32 h + x
      // -> tile h, row (2 i1 + i) r2 + c
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        float v[64];
        tmem_ld64(dg + 64u * (uint32_t)i, v);
        if (row < 2 * s.r2) {
          const int c = row >> 1, i1 = row & 1;
          const int R = (2 * i1 + i) * s.r2 + c;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            unsigned char *O = TO + (unsigned)h * P.ohalf;
#pragma unroll
            for (int cx = 0; cx < 8; ++cx) {
              float4 w;
              w.x = tf32_rne(v[32 * h + 4 * cx]);
              w.y = tf32_rne(v[32 * h + 4 * cx + 1]);
              w.z = tf32_rne(v[32 * h + 4 * cx + 2]);
              w.w = tf32_rne(v[32 * h + 4 * cx + 3]);
              *reinterpret_cast<float4 *>(O + row_off(R, 4 * cx)) = w;
            }
          }
        }
      }
      tc_fence_before();
      mbar_arrive(su32(&B.dfree[g]));
      fence_async_smem();
      epi_sync<kGroupThreads>(g);
      if (leader) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int64_t q = cw.w * kQ + 32 * h;
          tma_store5(&tout, su32(TO) + (unsigned)h * P.ohalf, (int)(q & lowmask),
                     (int)(cw.c * s.r2), 0, 0, (int)(q >> s.k));
        }
        bulk_commit();
      }
    }
    if (leader) bulk_wait_all();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kMmaWarp) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
  }
  if (tid == 0 && *abort) atomicCAS(&g_tcf_status, 0, (int)QTT_ERR_TIMEOUT);
}

constexpr size_t kSmemLimit = 227 * 1024;

// 5-D views of a planar FP32 buffer [P][N] for the pair at bit k (k >= 5),
// boxes of rows of 32 positions (128 bytes, 128-byte swizzle).
//   input:  dims (x: bits 0..k-1, a: bit k, P, b: bit k+1, hi: bits k+2..),
//           box (32, 2, r0, 2, 1): smem rows (b, P, a)
//   output: dims (x, P, a: bit k, b: bit k+1, hi), box (32, r2, 2, 2, 1):
//           smem rows (b, a, P)
bool encode_view_f32(CUtensorMap *m, const void *ptr, int k, int64_t N, int64_t planes,
                     int box_p, bool planes_second) {
  const cuuint64_t hi = (cuuint64_t)(N >> (k + 2));
  const cuuint64_t sa = ((cuuint64_t)1 << k) * 4, sb = ((cuuint64_t)1 << (k + 1)) * 4,
                   sp = (cuuint64_t)N * 4, sh = ((cuuint64_t)1 << (k + 2)) * 4;
  cuuint64_t dims[5], strides[4];
  cuuint32_t box[5];
  dims[0] = (cuuint64_t)1 << k;
  box[0] = 32;
  if (planes_second) {
    const cuuint64_t d[4] = {(cuuint64_t)planes, 2, 2, hi}, st[4] = {sp, sa, sb, sh};
    const cuuint32_t bx[4] = {(cuuint32_t)box_p, 2, 2, 1};
    for (int i = 0; i < 4; ++i) dims[i + 1] = d[i], strides[i] = st[i], box[i + 1] = bx[i];
  } else {
    const cuuint64_t d[4] = {2, (cuuint64_t)planes, 2, hi}, st[4] = {sa, sp, sb, sh};
    const cuuint32_t bx[4] = {2, (cuuint32_t)box_p, 2, 1};
    for (int i = 0; i < 4; ++i) dims[i + 1] = d[i], strides[i] = st[i], box[i + 1] = bx[i];
  }
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  const PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return false;
  return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<void *>(ptr), dims, strides, box,
                es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int stages_for_f(const StepTF2 &s) {
  const PlanF p0 = make_plan_f(s, 0);
  const unsigned st = up1k(p0.stage);
  if (p0.end + 2 * st + 1024 > kSmemLimit) return 0;
  const int S = (int)((kSmemLimit - 1024 - p0.end) / st);
  return S > kMaxStages ? kMaxStages : S;
}

}  // namespace

bool tc2f_steps_eligible(int k, int r0, int r1, int r2, int64_t N) {
  // k >= 5: runs of 32 positions (128-byte rows) are contiguous; whole chunks
  // of 32 quads; the K of both MMAs (2 r0, 2 r1) whole 128-byte atoms of 32
  // TF32; r2 <= 32 so that D2 fits TMEM lanes 0-63
  return k >= 5 && N >= 512 && ((int64_t)1 << (k + 2)) < N && (r0 == 16 || r0 == 32) &&
         (r1 == 16 || r1 == 32) && r2 >= 1 && r2 <= kMaxRank;
}

cudaError_t launch_step_tc2_tf32(const StepTF2 &s, cudaStream_t st) {
  if (!tc2f_steps_eligible(s.k, s.r0, s.r1, s.r2, s.N)) return cudaErrorNotSupported;
  if (s.in_rhs_stride != (int64_t)s.r0 * s.N || s.out_rhs_stride != (int64_t)s.r2 * s.N)
    return cudaErrorNotSupported;
  const int S = stages_for_f(s);
  if (S < 2) return cudaErrorNotSupported;
  const size_t smem = make_plan_f(s, S).end + 1024;
  CUtensorMap tin, tout;
  if (!encode_view_f32(&tin, s.in, s.k, s.N, s.nrhs * s.r0, s.r0, false) ||
      !encode_view_f32(&tout, s.out, s.k, s.N, s.nrhs * s.r2, s.r2, true))
    return cudaErrorNotSupported;
  static cudaError_t attr = cudaFuncSetAttribute(
      step_tc2f_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit);
  if (attr != cudaSuccess) return attr;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t nchunks = (s.N >> 2) / kQ * s.nrhs;
  const unsigned grid = (unsigned)(nchunks < sms ? nchunks : sms);
  step_tc2f_kernel<<<grid, kThreads, smem, st>>>(tin, tout, s, S);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t tcf_status_take(int *status) {
  int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(status, g_tcf_status, sizeof(int));
  if (e == cudaSuccess && *status != 0) e = cudaMemcpyToSymbol(g_tcf_status, &zero, sizeof(int));
  return e;
}

}  // namespace qtt
