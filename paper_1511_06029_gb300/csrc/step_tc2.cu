// Two consecutive BF16 core steps (k, k+1) of Algorithm 2 on the fifth-
// generation tensor cores: TMA tile loads and stores, tcgen05.mma with
// operands in shared memory and FP32 accumulators in tensor memory (TMEM).
//
// The four positions of a quad (bits k and k+1 free, the others fixed) are
// closed under both steps, so a chunk of 64 quads is read from HBM once and
// only y_{k+2} goes back; the r_{k+1} planes in between stay on chip.
//
// Per chunk (a persistent CTA takes chunks blockIdx.x, + grid, ...):
//   stage S   (B of step k, MN-major, 128-byte swizzle): K rows 2a + j_k,
//             N columns 64 j_{k+1} + quad -- one TMA box of the input planes
//   D1 = M_k S      in TMEM: lanes 2b + i_k, columns 64 j_{k+1} + quad
//   T         (B of step k+1, MN-major, 128-byte swizzle): K rows
//             2b + j_{k+1}, N columns 64 i_k + quad   (D1 rounded to BF16 --
//             the rounding the unfused path applies when it stores y_{k+1})
//   D2 = M_{k+1} T  in TMEM: lanes 2c + i_{k+1}, columns 64 i_k + quad
//   O         output tile, rows (i_k, c, i_{k+1}) of 64 quads (128-byte
//             swizzle) -- one TMA box store into y_{k+2} (k < 6: rows (u / 64,
//             c) of the chunk's 256 consecutive positions u)
// Both MMAs are M = 128 (rows 2b + i; rows past 2 r are padding whose
// results are never read), N = 128, K = 16 per instruction.  M_k and M_{k+1}
// stay in shared memory for the CTA's lifetime (K-major, 128-byte swizzle).
// Every operand is swizzled: the unswizzled core-matrix layouts measured
// about 10 % slower (bank conflicts in the tensor core's operand reads).
//
// TMA boxes.  Within a chunk, runs of X = 2^min(k, 6) quads are X
// consecutive positions in each of the four (j_k, j_{k+1}) slices, and the
// planes of all right-hand sides form one index P = rhs r + a (stride N), so
// one 5-D view (x = position bits 0..k-1, j_k, P, j_{k+1}, position bits
// k+2..) covers the input; its box (X, 2, r_k, 2, 64 / X) lands in shared
// memory exactly as the MMA's MN-major operand, rows of X values with the
// swizzle that spans one row (none, 32, 64 or 128 bytes for X = 8 .. 64).
// The MN order of the stage is then (position bits k+2.., j_{k+1}, x); T and
// the output tile use (bits k+2.., i_k, x).  The output view orders (x,
// i_{k+1}, P, i_k, hi) so that the rows one epilogue warp writes are
// consecutive in the swizzle pattern.  For k < 6 a chunk's positions are 256
// consecutive ones, so the output goes out as 128-byte rows of a 3-D view
// (64 positions, P, position / 64) instead: the TMA engine moves about one
// box row per 4 cycles, and rows of X < 64 values would cap the store.
// r_k % 8 == 0 makes the box's K extent 2 r_k the padded K of the MMA, so no
// plane of a neighbouring right-hand side is read.
//
// Warp roles, connected by mbarriers (a software pipeline over chunks):
//   warp 0      one lane issues the TMA loads into a ring of S stages
//   warp 1      allocates TMEM; one lane issues the MMAs: MMA1 of chunk n
//               (frees its stage on completion) ahead of MMA2 of chunk
//               n - G/2.  This thread sets the pace, so its per-MMA work is
//               one OR of the start address into a descriptor template and
//               chunks and ring slots advance by counters (no divisions)
//   warps 2-17  G epilogue groups of 16 / G warps (G = 4 where the tiles of
//               four leave room for three ring stages, else 2); group g
//               takes the chunks n = g (mod G): D1 -> T[g]; D2 -> O[g] ->
//               TMA store.  While one group waits for its MMA, the others
//               work; MMA2 of chunk n - G/2 follows MMA1 of chunk n.
// TMEM holds G accumulator buffers of 128 columns (chunk n uses n % G; D2
// overwrites D1 of the same chunk once the epilogue has read it).
//
// Every wait is bounded: a clock budget after which the CTA raises a shared
// abort flag, every role leaves its loop, the CTA drains its copies, frees
// its TMEM, records QTT_ERR_TIMEOUT in a device status word (read by
// qtt_sync_status) and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cstdlib>
#include <cuda_bf16.h>

#include "checked.cuh"
#include "qtt_internal.h"
#include "step_mma.h"
#include "tc_common.cuh"

namespace qtt {

__device__ int g_tc_status = 0;

namespace {

using namespace tcx;

constexpr int kProducerWarp = 0;
constexpr int kMmaWarp = 1;
constexpr int kEpiWarp0 = 2;
constexpr int kEpiThreads = 512;           // warps 2-17: G groups of 512 / G threads
constexpr int kMaxGroups = 4;
constexpr int kThreads = 64 + kEpiThreads;
constexpr int kQ = 64;                     // quads per chunk
constexpr int kCols = 2 * kQ;              // N of both MMAs
constexpr int kMaxStages = 8;
constexpr int kMaxKs = 7;                  // K steps of 16: 2 r rounded up to 16, r <= 56
constexpr int kBarBytes = 512;             // mbarriers, TMEM address, abort flag

// Instruction descriptor of kind::f16: D FP32, A and B BF16, A K-major,
// B MN-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (0u << 15) | (1u << 16) |
                            ((uint32_t)(kCols >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t da, uint64_t db, int acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(da), "l"(db), "r"(kIdesc), "r"(acc));
}
__device__ __forceinline__ uint4 pack8(const float *v) {
  uint4 o;
  __nv_bfloat162 h;
  h = __floats2bfloat162_rn(v[0], v[1]);
  o.x = *reinterpret_cast<unsigned *>(&h);
  h = __floats2bfloat162_rn(v[2], v[3]);
  o.y = *reinterpret_cast<unsigned *>(&h);
  h = __floats2bfloat162_rn(v[4], v[5]);
  o.z = *reinterpret_cast<unsigned *>(&h);
  h = __floats2bfloat162_rn(v[6], v[7]);
  o.w = *reinterpret_cast<unsigned *>(&h);
  return o;
}

static_assert((2 * kTc2MaxRank + 15) / 16 <= kMaxKs, "K steps of the largest rank");

struct Bars {
  unsigned long long full[kMaxStages], empty[kMaxStages];
  unsigned long long d1full[kMaxGroups], d2full[kMaxGroups], dfree[kMaxGroups],
      tready[kMaxGroups];
  uint32_t tmem;
  int abort;
};
static_assert(sizeof(Bars) <= kBarBytes, "mbarrier block");

// Self-test of the bounded waits: one thread waits, through wait_bar, for a
// phase of an mbarrier that nothing completes; when the budget runs out it
// records QTT_ERR_TIMEOUT in the status word and returns, as the pair
// kernel's roles do.
__global__ void wait_selftest_kernel(long long budget) {
  __shared__ unsigned long long bar;
  __shared__ int abort;
  if (threadIdx.x != 0) return;
  abort = 0;
  mbar_init(su32(&bar), 1);
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  if (!wait_bar(su32(&bar), 0u, &abort, budget)) atomicCAS(&g_tc_status, 0, (int)QTT_ERR_TIMEOUT);
}

struct Plan {
  unsigned a1, a2, t[kMaxGroups], o[kMaxGroups], s0, stage, obytes, end;
};
// G epilogue groups (a T and an output tile each), S ring stages
__host__ __device__ inline Plan make_plan(const StepMMA2 &s, int S, int G) {
  Plan p;
  const unsigned Kp2 = (unsigned)s.Mp1;
  // every tile 1024-aligned (the 128-byte swizzle repeats every 8 rows)
  p.a1 = up1k(kBarBytes);
  p.a2 = up1k(p.a1 + a_bytes(s.Mp1, s.Kp1));
  // T[0] follows A2: the M = 128 padding rows of M_{k+1} read past A2 into
  // it (finite data; those rows are never used)
  p.t[0] = up1k(p.a2 + a_bytes(s.Mp2, (int)Kp2));
  for (int g = 1; g < G; ++g) p.t[g] = p.t[g - 1] + 2u * Kp2 * 128u;
  p.obytes = (unsigned)(2 * 2 * s.r2 * 128);
  p.o[0] = up1k(p.t[G - 1] + 2u * Kp2 * 128u);
  for (int g = 1; g < G; ++g) p.o[g] = up1k(p.o[g - 1] + p.obytes);
  p.stage = (unsigned)(s.Kp1 * kCols * 2);
  p.s0 = up1k(p.o[G - 1] + p.obytes);
  p.end = p.s0 + (unsigned)S * p.stage;
  return p;
}

// Position runs: X = 2^XLOG quads (XLOG = min(k, 6)) are contiguous, so the
// tile rows are X values (2 X bytes) wide and the swizzle spans one row:
// B = XLOG - 3 bits of 16-byte chunk index (none, 32, 64 or 128 bytes).
template <int XLOG>
struct Rows {
  static constexpr int X = 1 << XLOG;
  static constexpr unsigned bytes = 2u * X;
  static constexpr int B = XLOG - 3;
  // descriptor layout code: none 0, 32-byte 6, 64-byte 4, 128-byte 2
  static constexpr unsigned code = B == 3 ? 2u : B == 2 ? 4u : B == 1 ? 6u : 0u;
  // physical offset of a logical byte offset from a 1024-aligned tile base
  __device__ static unsigned swz(unsigned off) {
    return off ^ (((off >> 7) & ((1u << B) - 1u)) << 4);
  }
  // MN-major operand of Kp rows: descriptor for K rows 16 ks .. 16 ks + 15
  __device__ static uint64_t desc(unsigned tile, int Kp, int ks) {
    if (B == 0)  // core matrices: K groups 128 bytes apart, MN blocks Kp 16
      return smem_desc(tile + ks * 256, 128, (unsigned)Kp * 16, 0);
    return smem_desc(tile + ks * 16 * bytes, (unsigned)Kp * bytes, 8 * bytes, code);
  }
};

// G epilogue groups of 16 / G warps (G = 2 or 4): group g takes the chunks
// n = g (mod G) with TMEM buffer g, T[g] and O[g]; MMA2 of chunk n - G/2
// follows MMA1 of chunk n, so a group has G/2 chunk slots to turn D1 into T
// and as many to read D2 before its buffer is needed again.
template <int XLOG, int G>
__global__ void __launch_bounds__(kThreads, 1)
    step_tc2_kernel(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tout,
                    StepMMA2 s, int S) {
  using Rw = Rows<XLOG>;
  constexpr int kGroupThreads = kEpiThreads / G;
  constexpr int kParts = kGroupThreads / 128;  // warps per TMEM lane quadrant in a group
  constexpr int kColsW = kCols / kParts;       // accumulator columns per warp
  constexpr int kLag = G / 2;
  constexpr uint32_t kTmemCols = 128u * G;
  extern __shared__ __align__(1024) unsigned char smraw[];
  // 1024-aligned base for the swizzled tiles
  unsigned char *base = smraw + ((1024u - (su32(smraw) & 1023u)) & 1023u);
  const Plan P = make_plan(s, S, G);
  Bars &B = *reinterpret_cast<Bars *>(base);
  const int Kp2 = s.Mp1;
  unsigned char *sA1 = base + P.a1, *sA2 = base + P.a2;
  const unsigned base32 = su32(base);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

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
      mbar_init(su32(&B.empty[i]), 1);
    }
    for (int i = 0; i < G; ++i) {
      mbar_init(su32(&B.d1full[i]), 1);
      mbar_init(su32(&B.d2full[i]), 1);
      mbar_init(su32(&B.dfree[i]), kGroupThreads);
      mbar_init(su32(&B.tready[i]), kGroupThreads);
    }
    B.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  // core matrices as swizzled K-major operands (16-byte pieces of 8 columns)
  for (int e = tid; e < s.Mp1 * (s.Kp1 / 8); e += kThreads) {
    const int r = e / (s.Kp1 / 8), kc = e % (s.Kp1 / 8);
    cpa16(su32(sA1 + a_offset(s.Mp1, r, kc)), s.A1 + (size_t)r * s.Kp1 + 8 * kc, 16);
  }
  for (int e = tid; e < s.Mp2 * (Kp2 / 8); e += kThreads) {
    const int r = e / (Kp2 / 8), kc = e % (Kp2 / 8);
    cpa16(su32(sA2 + a_offset(s.Mp2, r, kc)), s.A2 + (size_t)r * Kp2 + 8 * kc, 16);
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

  if (warp == kProducerWarp) {
    // ---------------------------------------------------------------- TMA loads
    if (lane == 0) {
      // chunk t = blockIdx.x + n gridDim.x is (rhs c, chunk w of it); both
      // advance without a division per chunk, as do the ring slot and parity
      ChunkWalk cw(blockIdx.x, NG, cpr);
      int n = 0, st = 0;
      unsigned ph = 0;
      for (;; ++n, cw.next()) {
        if (cw.t >= nchunks) break;
        if (n >= S && !wait_bar(su32(&B.empty[st]), ph ^ 1u, abort)) break;
        // the box: quads q0 .. q0 + kQ - 1 of right-hand side c
        const int64_t q0 = QTT_CK(cw.w * kQ, (s.N >> 2) - kQ + 1, 301);
        const int64_t cc = QTT_CK(cw.c, s.nrhs, 302);
        const unsigned fb = su32(&B.full[st]);
        expect_tx(fb, P.stage);
        tma_load5(base32 + P.s0 + (unsigned)st * P.stage, &tin, (int)(q0 & lowmask), 0,
                  (int)(cc * s.r0), 0, (int)(q0 >> s.k), fb);
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
  } else if (warp == kMmaWarp) {
    // ---------------------------------------------------------------- MMA issue
    if (lane == 0) {
      // Descriptors: every field but the start address (bits 0-13, the
      // shared address >> 4) is fixed per operand, so each MMA ORs the
      // masked start into a template -- the same value smem_desc gives.
      // Per K step of 16: A moves 32 bytes within a 128-byte swizzle atom,
      // Mp rows of 128 bytes per atom of 64; B moves 16 rows of its tile.
      constexpr unsigned kBStep = Rw::B == 0 ? 256u : 16u * Rw::bytes;  // bytes per K step
      const int nk1 = s.Kp1 / 16, nk2 = Kp2 / 16;
      const uint64_t tA = smem_desc(0, 16, 1024, 2);
      const uint64_t tS = Rw::desc(0, s.Kp1, 0), tT = Rw::desc(0, Kp2, 0);
      unsigned aA1[kMaxKs], aA2[kMaxKs];
#pragma unroll
      for (int ks = 0; ks < kMaxKs; ++ks) {
        aA1[ks] = base32 + P.a1 + (unsigned)((ks >> 2) * s.Mp1 * 128 + (ks & 3) * 32);
        aA2[ks] = base32 + P.a2 + (unsigned)((ks >> 2) * s.Mp2 * 128 + (ks & 3) * 32);
      }
      // this CTA's chunks n = 0 .. mine - 1 are blockIdx.x + n gridDim.x
      const int mine = nchunks > blockIdx.x ? (int)((nchunks - 1 - blockIdx.x) / NG + 1) : 0;
      int st = 0;
      unsigned ph = 0;  // ring slot of chunk n and the parity of its fill
      for (int n = 0;; ++n) {
        if (n < mine) {
          const int b = n % G;
          if (!wait_bar(su32(&B.full[st]), ph, abort)) break;
          if (n >= G && !wait_bar(su32(&B.dfree[b]), (unsigned)(n / G - 1) & 1u, abort)) break;
          tc_fence_after();
          const unsigned sb = base32 + P.s0 + (unsigned)st * P.stage;
          const uint32_t d = tmem + (uint32_t)(b * 128);
#pragma unroll
          for (int ks = 0; ks < kMaxKs; ++ks)
            if (ks < nk1)
              mma_bf16(d, tA | ((aA1[ks] >> 4) & 0x3FFFu), tS | (((sb + ks * kBStep) >> 4) & 0x3FFFu),
                       ks > 0);
          mma_commit(su32(&B.empty[st]));
          mma_commit(su32(&B.d1full[b]));
          if (++st == S) {
            st = 0;
            ph ^= 1u;
          }
        }
        const int m = n - kLag;
        if (m >= 0 && m < mine) {
          const int bm = m % G;
          if (!wait_bar(su32(&B.tready[bm]), (unsigned)(m / G) & 1u, abort)) break;
          tc_fence_after();
          const unsigned t32 = base32 + P.t[bm];
          const uint32_t d = tmem + (uint32_t)(bm * 128);
#pragma unroll
          for (int ks = 0; ks < kMaxKs; ++ks)
            if (ks < nk2)
              mma_bf16(d, tA | ((aA2[ks] >> 4) & 0x3FFFu), tT | (((t32 + ks * kBStep) >> 4) & 0x3FFFu),
                       ks > 0);
          mma_commit(su32(&B.d2full[bm]));
        }
        if (m >= mine - 1) break;
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    // group g takes the chunks n = g, g + G, ... (TMEM buffer g, T[g], O[g]),
    // so one group's epilogue overlaps the others' MMAs.  A warp reads the
    // TMEM lanes of its quadrant (warp % 4), columns kColsW part ..
    const int g = (warp - kEpiWarp0) / (kGroupThreads / 32);
    const int qr = warp & 3, part = ((warp - kEpiWarp0) >> 2) % kParts;
    const int row = 32 * qr + lane;  // TMEM lane = D row
    const bool leader = tid == (kEpiWarp0 + (kGroupThreads / 32) * g) * 32;
    unsigned char *sT = base + P.t[g];
    unsigned char *O = base + P.o[g];
    const uint32_t tl = ((uint32_t)(32 * qr) << 16) + (uint32_t)(kColsW * part);
    const int orows = 2 * s.r2;
    ChunkWalk cw(blockIdx.x + (int64_t)g * NG, (int64_t)G * NG, cpr);
    for (int n = g;; n += G, cw.next()) {
      if (cw.t >= nchunks) break;
      const int b = g;
      const uint32_t tb = tmem + tl + (uint32_t)(b * 128);
      if (epi_any<kGroupThreads>(!wait_bar(su32(&B.d1full[b]), (unsigned)(n / G) & 1u, abort), g))
        break;
      tc_fence_after();
      // D1 -> T.  D1 column n = (2 hi + j') X + x (the stage's MN order);
      // T row K2 = 2b + j', its MN order (2 hi + i) X + x
      if (32 * qr < s.Mp1) {
#pragma unroll
        for (int xb = 0; xb < kColsW / 32; ++xb) {
          float v[32];
          tmem_ld32(tb + 32 * xb, v);
          if (row < Kp2) {
            const int i = row & 1, bb = row >> 1;
#pragma unroll
            for (int p = 0; p < 4; ++p) {
              const int n = kColsW * part + 32 * xb + 8 * p;
              const int beta = n >> XLOG, x = n & (Rw::X - 1);
              const int k2 = 2 * bb + (beta & 1), beta2 = (beta & ~1) | i;
              const unsigned off = (unsigned)(beta2 * Kp2 + k2) * Rw::bytes + 2u * x;
              *reinterpret_cast<uint4 *>(sT + Rw::swz(off)) = pack8(v + 8 * p);
            }
          }
        }
      }
      fence_async_smem();
      tc_fence_before();
      mbar_arrive(su32(&B.tready[b]));
      if (epi_any<kGroupThreads>(!wait_bar(su32(&B.d2full[b]), (unsigned)(n / G) & 1u, abort), g))
        break;
      tc_fence_after();
      // D2 -> O[g] -> one TMA store.  D2 column n = (2 hi + i) X + x.  For
      // k < 6 the chunk's 256 positions of a plane are consecutive, u = x +
      // X (i + 2 i_{k+1} + 4 hi): rows (u / 64, c) of 64 values, 128-byte
      // swizzle; else the store box's rows are (2 hi + i, c, i_{k+1}), X
      // values each
      if (leader) bulk_wait_read0();  // the group's previous store has read O
      epi_sync<kGroupThreads>(g);
      if (32 * qr < s.Mp2) {
#pragma unroll
        for (int xb = 0; xb < kColsW / 32; ++xb) {
          float v[32];
          tmem_ld32(tb + 32 * xb, v);
          if (row < orows) {
#pragma unroll
            for (int p = 0; p < 4; ++p) {
              const int n = kColsW * part + 32 * xb + 8 * p;
              const int beta2 = n >> XLOG, x = n & (Rw::X - 1);
              if constexpr (XLOG < 6) {
                const int u = x + Rw::X * ((beta2 & 1) + 2 * (row & 1) + 4 * (beta2 >> 1));
                const unsigned off = (unsigned)((u >> 6) * s.r2 + (row >> 1)) * 128u + 2u * (u & 63);
                *reinterpret_cast<uint4 *>(O + Rows<6>::swz(off)) = pack8(v + 8 * p);
              } else {
                const unsigned off = (unsigned)(beta2 * orows + row) * Rw::bytes + 2u * x;
                *reinterpret_cast<uint4 *>(O + Rw::swz(off)) = pack8(v + 8 * p);
              }
            }
          }
        }
      }
      tc_fence_before();
      mbar_arrive(su32(&B.dfree[b]));
      fence_async_smem();
      epi_sync<kGroupThreads>(g);
      if (leader) {
        const int64_t q0 = QTT_CK(cw.w * kQ, (s.N >> 2) - kQ + 1, 303);
        const int64_t cc = QTT_CK(cw.c, s.nrhs, 304);
        if constexpr (XLOG < 6)
          tma_store3(&tout, su32(O), 0, (int)(cc * s.r2), (int)(q0 >> 4));
        else
          tma_store5(&tout, su32(O), (int)(q0 & lowmask), 0, (int)(cc * s.r2), 0,
                     (int)(q0 >> s.k));
        bulk_commit();
      }
    }
    if (leader) bulk_wait_all();  // output stores complete before the CTA exits
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
  if (tid == 0 && *abort) atomicCAS(&g_tc_status, 0, (int)QTT_ERR_TIMEOUT);
}

constexpr size_t kSmemLimit = 227 * 1024;

// 5-D view of a planar BF16 buffer [P][N] for the pair at bit k: dims (x:
// bits 0..k-1, a: bit `b1`, P, b: bit `b3`, hi: bits k+2..), box (X, 2, box_p,
// 2, 64 / X) with X = 2^min(k, 6), swizzle spanning one X-value row.
// Returns false if the driver rejects it.
// L2 promotion: 256 bytes while a chunk's rows of a plane are contiguous
// (k <= 6); for k > 6 they lie 2^k positions apart and the other half of a
// 256-byte fetch belongs to a chunk another CTA reads later (it measured
// about 30 % extra DRAM reads), so rows are fetched as single 128-byte lines.
bool encode_view(CUtensorMap *m, const void *ptr, int k, int64_t N, int64_t planes, int b1,
                 int b3, int box_p) {
  const int xl = k < 6 ? k : 6;
  const cuuint64_t dims[5] = {(cuuint64_t)1 << k, 2, (cuuint64_t)planes, 2,
                              (cuuint64_t)(N >> (k + 2))};
  const cuuint64_t strides[4] = {((cuuint64_t)1 << b1) * 2, (cuuint64_t)N * 2,
                                 ((cuuint64_t)1 << b3) * 2, ((cuuint64_t)1 << (k + 2)) * 2};
  const cuuint32_t box[5] = {1u << xl, 2, (cuuint32_t)box_p, 2, 64u >> xl};
  const CUtensorMapSwizzle swz = xl == 6   ? CU_TENSOR_MAP_SWIZZLE_128B
                                 : xl == 5 ? CU_TENSOR_MAP_SWIZZLE_64B
                                 : xl == 4 ? CU_TENSOR_MAP_SWIZZLE_32B
                                           : CU_TENSOR_MAP_SWIZZLE_NONE;
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  const PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return false;
  return encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(ptr), dims, strides,
                box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                k > 6 ? CU_TENSOR_MAP_L2_PROMOTION_L2_128B : CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 3-D view of a planar BF16 buffer [P][N] as rows of 64 consecutive
// positions: dims (e < 64, P, position / 64), box (64, box_p, 4) -- one
// chunk's 256 consecutive positions of box_p planes, 128-byte swizzle.
bool encode_flat(CUtensorMap *m, const void *ptr, int64_t N, int64_t planes, int box_p) {
  const cuuint64_t dims[3] = {64, (cuuint64_t)planes, (cuuint64_t)(N >> 6)};
  const cuuint64_t strides[2] = {(cuuint64_t)N * 2, 128};
  const cuuint32_t box[3] = {64, (cuuint32_t)box_p, 4};
  const cuuint32_t es[3] = {1, 1, 1};
  const PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return false;
  return encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(ptr), dims, strides,
                box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

namespace {

template <int XLOG, int G>
cudaError_t launch_x(const CUtensorMap &tin, const CUtensorMap &tout, const StepMMA2 &s, int S,
                     size_t smem, unsigned grid, cudaStream_t st) {
  // one CTA per SM: the shared-memory limit is raised once per instantiation
  static cudaError_t attr = cudaFuncSetAttribute(
      step_tc2_kernel<XLOG, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit);
  if (attr != cudaSuccess) return attr;
  step_tc2_kernel<XLOG, G><<<grid, kThreads, smem, st>>>(tin, tout, s, S);
  count_launches(1);
  return cudaGetLastError();
}

// Ring stages that fit beside the tiles of G groups (0 if fewer than two).
int stages_for(const StepMMA2 &s, int G) {
  const Plan p0 = make_plan(s, 0, G);
  if (p0.end + 2 * p0.stage + 1024 > kSmemLimit) return 0;
  const int S = (int)((kSmemLimit - 1024 - p0.end) / p0.stage);
  return S > kMaxStages ? kMaxStages : S;
}

// QTT_TC2_GROUPS=2 keeps two epilogue groups everywhere (for comparisons).
bool four_groups_allowed() {
  static const bool ok = [] {
    const char *e = getenv("QTT_TC2_GROUPS");
    return !(e && e[0] == '2');
  }();
  return ok;
}

}  // namespace

bool tc2_steps_eligible(int k, int r0, int r1, int r2, int64_t N) {
  // k >= 4: runs of 16 quads are contiguous (the TMA engine moves about one
  // box row per 4 cycles, so 16-byte rows (k = 3) ran at 1.2 TB/s, slower
  // than two single steps; 32-, 64- and 128-byte rows at 2.4, 4.7 and
  // 5.9 TB/s); N >= 256: whole 64-quad chunks; r0 % 8 == 0: the input box is
  // exactly the MMA's padded K; ranks <= 56: two ring stages fit
  return k >= 4 && N >= 256 && (int64_t)1 << (k + 2) < N && r0 % 8 == 0 && r0 >= 8 &&
         r1 >= 8 && r2 >= 8 && r0 <= kTc2MaxRank && r1 <= kTc2MaxRank && r2 <= kTc2MaxRank;
}

cudaError_t launch_step_tc2_bf16(const StepMMA2 &s, cudaStream_t st) {
  // Four epilogue groups (four chunks between their MMAs at once) where
  // their tiles leave room for at least three ring stages -- the small-rank
  // pairs, whose time per chunk is set by the MMA -> epilogue -> MMA chain
  // rather than by bytes; else two.  As many ring stages as fit.
  int G = 4, S = four_groups_allowed() && s.groups_cap != 2 ? stages_for(s, 4) : 0;
  if (S < 3) {
    G = 2;
    S = stages_for(s, 2);
  }
  if (S < 2) return cudaErrorNotSupported;
  const size_t smem = make_plan(s, S, G).end + 1024;
  // the input view needs the buffer to hold exactly nrhs right-hand sides of r_k
  // planes each, back to back (as the apply's scratch does)
  if (s.in_rhs_stride != (int64_t)s.r0 * s.N || s.out_rhs_stride != (int64_t)s.r2 * s.N)
    return cudaErrorNotSupported;
  CUtensorMap tin, tout;
  if (!encode_view(&tin, s.in, s.k, s.N, s.nrhs * s.r0, s.k, s.k + 1, s.r0) ||
      !(s.k < 6 ? encode_flat(&tout, s.out, s.N, s.nrhs * s.r2, s.r2)
                : encode_view(&tout, s.out, s.k, s.N, s.nrhs * s.r2, s.k + 1, s.k, s.r2)))
    return cudaErrorNotSupported;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t nchunks = (s.N >> 2) / kQ * s.nrhs;
  const unsigned grid = (unsigned)(nchunks < sms ? nchunks : sms);
  const int xl = s.k < 6 ? s.k : 6;
  if (G == 4) {
    switch (xl) {
      case 4: return launch_x<4, 4>(tin, tout, s, S, smem, grid, st);
      case 5: return launch_x<5, 4>(tin, tout, s, S, smem, grid, st);
      case 6: return launch_x<6, 4>(tin, tout, s, S, smem, grid, st);
    }
  } else {
    switch (xl) {
      case 4: return launch_x<4, 2>(tin, tout, s, S, smem, grid, st);
      case 5: return launch_x<5, 2>(tin, tout, s, S, smem, grid, st);
      case 6: return launch_x<6, 2>(tin, tout, s, S, smem, grid, st);
    }
  }
  return cudaErrorNotSupported;
}

cudaError_t wait_selftest(double seconds, cudaStream_t st) {
  int dev = 0, khz = 2000000;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
  wait_selftest_kernel<<<1, 32, 0, st>>>((long long)(seconds * 1e3 * khz));
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t tc_status_take(int *status) {
  int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(status, g_tc_status, sizeof(int));
  if (e == cudaSuccess && *status != 0) e = cudaMemcpyToSymbol(g_tc_status, &zero, sizeof(int));
  return e;
}

}  // namespace qtt
