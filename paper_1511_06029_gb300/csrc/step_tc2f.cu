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
// MMA, and the epilogue writes the second MMA's operand K-major directly:
//   stage S  (TMA, MN-major, 128-byte swizzle): rows (j_{k+1}, a, j_k) of 32
//            positions -- 2 r_k rows of K per j_{k+1}
//   Bk       (transposer): row n = 32 j_{k+1} + x, K = 2a + j_k, K-major
//   D1 = M_k Bk      TMEM lanes 2b + i_k, columns 32 j_{k+1} + x
//   T        (epilogue, D1 rounded to TF32 -- where the unfused sweep rounds
//            the stored y_{k+1}): row n = 32 i_k + x, K = 2b + j_{k+1}
//   D2 = M_{k+1} T   TMEM lanes 2c + i_{k+1}, columns 32 i_k + x
//   O        output tile, rows (i_{k+1}, c, i_k) of 32 positions (rounded to
//            TF32) -- one TMA store into y_{k+2}
// Both MMAs are M = 128 (rows 2r + i; rows past 2r are zero padding of the
// core tiles), N = 64, K = 8 per instruction.  A chunk is 32 quads (128
// positions per plane): 32 consecutive positions (128-byte rows of FP32) in
// each of the four (j_k, j_{k+1}) slices, so k >= 5.
//
// Warp roles, connected by mbarriers:
//   warp 0      one lane issues the TMA loads into a ring of S stages
//   warp 1      allocates TMEM; one lane issues the MMAs (MMA1 of chunk n
//               ahead of MMA2 of chunk n - 1)
//   warps 2-5   transpose stage -> Bk (two Bk buffers)
//   warps 6-13  two epilogue groups of four warps; group g takes the chunks
//               n = g (mod 2): D1 -> T[g], D2 -> O[g] -> TMA store
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

constexpr int kGroups = 2;
constexpr int kProducerWarp = 0;
constexpr int kMmaWarp = 1;
constexpr int kXWarp0 = 2;                  // transposer warps 2-5
constexpr int kXThreads = 128;
constexpr int kEpiWarp0 = 6;                // epilogue warps 6-13
constexpr int kGroupThreads = 128;
constexpr int kThreads = 64 + kXThreads + kGroups * kGroupThreads;
constexpr int kQ = 32;                      // quads per chunk
constexpr int kCols = 2 * kQ;               // N of both MMAs
constexpr int kMaxStages = 6;
constexpr int kMaxRank = 32;                // 2 r <= 64: K of both MMAs, two K atoms
constexpr int kBarBytes = 512;

// Instruction descriptor of kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32
// (bits 7-9 and 10-12 = 2), both K-major (bits 15, 16 clear), N >> 3 at bit
// 17, M >> 4 at bit 24.
constexpr uint32_t kIdescF = (1u << 4) | (2u << 7) | (2u << 10) | (0u << 15) | (0u << 16) |
                             ((uint32_t)(kCols >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t da, uint64_t db, int acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(da), "l"(db), "r"(kIdescF), "r"(acc));
}

// Round to TF32 (10 explicit mantissa bits), nearest even, as the unfused
// TF32 sweep stores its intermediates.
__device__ __forceinline__ float tf32_rne(float x) {
  unsigned u = __float_as_uint(x);
  if ((u & 0x7f800000u) != 0x7f800000u) {
    u += 0x0fffu + ((u >> 13) & 1u);
    u &= 0xffffe000u;
  }
  return __uint_as_float(u);
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
  unsigned long long bkready[2], bkfree[2];
  unsigned long long d1full[kGroups], d2full[kGroups], dfree[kGroups], tready[kGroups];
  uint32_t tmem;
  int abort;
};
static_assert(sizeof(Bars) <= kBarBytes, "mbarrier block");

// Shared-memory plan (byte offsets from a 1024-aligned base).  Core tiles:
// 128 rows x Kp TF32, K-major (Kp = 2 r: 32 or 64).
struct PlanF {
  unsigned a1, a2, bk[2], t[kGroups], o[kGroups], s0, stage, end;
};
__host__ __device__ inline unsigned kmaj_bytes(int rows, int Kp) {
  return (unsigned)((Kp + 31) / 32) * (unsigned)rows * 128u;
}
__host__ __device__ inline PlanF make_plan_f(const StepTF2 &s, int S) {
  PlanF p;
  const int Kp1 = 2 * s.r0, Kp2 = 2 * s.r1;
  p.a1 = up1k(kBarBytes);
  p.a2 = up1k(p.a1 + kmaj_bytes(128, Kp1));
  p.bk[0] = up1k(p.a2 + kmaj_bytes(128, Kp2));
  p.bk[1] = up1k(p.bk[0] + kmaj_bytes(kCols, Kp1));
  p.t[0] = up1k(p.bk[1] + kmaj_bytes(kCols, Kp1));
  p.t[1] = up1k(p.t[0] + kmaj_bytes(kCols, Kp2));
  p.o[0] = up1k(p.t[1] + kmaj_bytes(kCols, Kp2));
  const unsigned obytes = (unsigned)(2 * s.r2 * 2) * 128u;
  p.o[1] = up1k(p.o[0] + obytes);
  p.s0 = up1k(p.o[1] + obytes);
  p.stage = (unsigned)(2 * s.r0 * 2) * 128u;
  p.end = p.s0 + (unsigned)S * up1k(p.stage);
  return p;
}

__global__ void __launch_bounds__(kThreads, 1)
    step_tc2f_kernel(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tout,
                     StepTF2 s, int S) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char *base = smraw + ((1024u - (su32(smraw) & 1023u)) & 1023u);
  const PlanF P = make_plan_f(s, S);
  Bars &B = *reinterpret_cast<Bars *>(base);
  const unsigned base32 = su32(base);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int Kp1 = 2 * s.r0, Kp2 = 2 * s.r1;
  const unsigned stage_stride = up1k(P.stage);

  if (warp == kMmaWarp) {
    asm volatile(
        "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
            su32(&B.tmem)),
        "r"((uint32_t)(kCols * kGroups))
        : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < kMaxStages; ++i) {
      mbar_init(su32(&B.full[i]), 1);
      mbar_init(su32(&B.empty[i]), kXThreads);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(su32(&B.bkready[i]), kXThreads);
      mbar_init(su32(&B.bkfree[i]), 1);
    }
    for (int i = 0; i < kGroups; ++i) {
      mbar_init(su32(&B.d1full[i]), 1);
      mbar_init(su32(&B.d2full[i]), 1);
      mbar_init(su32(&B.dfree[i]), kGroupThreads);
      mbar_init(su32(&B.tready[i]), kGroupThreads);
    }
    B.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  // core tiles as K-major operands: 128 rows x Kp, 16-byte pieces of 4 TF32
  for (int e = tid; e < 128 * (Kp1 / 4); e += kThreads) {
    const int r = e / (Kp1 / 4), kc = e % (Kp1 / 4);
    cpa16(base32 + P.a1 + a_offset(128, r, kc), s.A1 + (size_t)r * Kp1 + 4 * kc, 16);
  }
  for (int e = tid; e < 128 * (Kp2 / 4); e += kThreads) {
    const int r = e / (Kp2 / 4), kc = e % (Kp2 / 4);
    cpa16(base32 + P.a2 + a_offset(128, r, kc), s.A2 + (size_t)r * Kp2 + 4 * kc, 16);
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

  if (warp == kProducerWarp) {
    // ------------------------------------------------------------ TMA loads
    if (lane == 0) {
      ChunkWalk cw(blockIdx.x, NG, cpr);
      int n = 0, st = 0;
      unsigned ph = 0;
      for (; n < mine; ++n, cw.next()) {
        if (n >= S && !wait_bar(su32(&B.empty[st]), ph ^ 1u, abort)) break;
        const int64_t q0 = cw.w * kQ;
        const unsigned fb = su32(&B.full[st]);
        expect_tx(fb, P.stage);
        tma_load5(base32 + P.s0 + (unsigned)st * stage_stride, &tin, (int)(q0 & lowmask), 0,
                  (int)(cw.c * s.r0), 0, (int)(q0 >> s.k), fb);
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
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      // K-major, 128-byte swizzle: a K step of 8 TF32 moves 32 bytes inside
      // a 128-byte atom; atoms of 32 K are rows x 128 bytes apart
      const uint64_t tK = smem_desc(0, 16, 1024, 2);
      const int nk1 = Kp1 / 8, nk2 = Kp2 / 8;
      for (int n = 0;; ++n) {
        if (n < mine) {
          const int g = n % kGroups, b = n & 1;
          if (!wait_bar(su32(&B.bkready[b]), (unsigned)(n >> 1) & 1u, abort)) break;
          if (n >= kGroups && !wait_bar(su32(&B.dfree[g]), (unsigned)(n / kGroups - 1) & 1u, abort))
            break;
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(g * kCols);
          const unsigned bkb = base32 + P.bk[b];
          for (int ks = 0; ks < nk1; ++ks) {
            const unsigned aa = base32 + P.a1 + (unsigned)((ks >> 2) * 128 * 128 + (ks & 3) * 32);
            const unsigned bb = bkb + (unsigned)((ks >> 2) * kCols * 128 + (ks & 3) * 32);
            mma_tf32(d, tK | ((aa >> 4) & 0x3FFFu), tK | ((bb >> 4) & 0x3FFFu), ks > 0);
          }
          mma_commit(su32(&B.bkfree[b]));
          mma_commit(su32(&B.d1full[g]));
        }
        const int m = n - 1;  // MMA2 of the previous chunk follows MMA1 of this one
        if (m >= 0 && m < mine) {
          const int gm = m % kGroups;
          if (!wait_bar(su32(&B.tready[gm]), (unsigned)(m / kGroups) & 1u, abort)) break;
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(gm * kCols);
          const unsigned tb = base32 + P.t[gm];
          for (int ks = 0; ks < nk2; ++ks) {
            const unsigned aa = base32 + P.a2 + (unsigned)((ks >> 2) * 128 * 128 + (ks & 3) * 32);
            const unsigned bb = tb + (unsigned)((ks >> 2) * kCols * 128 + (ks & 3) * 32);
            mma_tf32(d, tK | ((aa >> 4) & 0x3FFFu), tK | ((bb >> 4) & 0x3FFFu), ks > 0);
          }
          mma_commit(su32(&B.d2full[gm]));
        }
        if (m >= mine - 1) break;
      }
    }
  } else if (warp < kEpiWarp0) {
    // ------------------------------------------------------------ transposer
    // stage row R = j1 (2 r0) + kr (kr = 2a + j0), 32 positions x; Bk row
    // n = 32 j1 + x, K index kr.  A thread gathers the four K values of one
    // 16-byte Bk piece (rows R .. R+3 at position x: a warp reads whole
    // 128-byte stage rows) and stores the piece (eight consecutive rows of a
    // warp land in eight distinct bank groups under the swizzle).
    const int xt = tid - kXWarp0 * 32;
    const int npiece = Kp1 / 4;           // 16-byte K pieces per Bk row
    const int items = 2 * npiece * 32;    // (j1, piece, x)
    int st = 0;
    unsigned ph = 0;
    for (int n = 0; n < mine; ++n) {
      const int b = n & 1;
      if (!wait_bar(su32(&B.full[st]), ph, abort)) break;
      if (n >= 2 && !wait_bar(su32(&B.bkfree[b]), (unsigned)((n >> 1) - 1) & 1u, abort)) break;
      const unsigned char *stg = base + P.s0 + (unsigned)st * stage_stride;
      unsigned char *bk = base + P.bk[b];
      for (int q = xt; q < items; q += kXThreads) {
        const int x = q & 31, jp = q >> 5;
        const int j1 = jp / npiece, pc = jp - j1 * npiece;
        const int R = j1 * Kp1 + 4 * pc;
        float4 v;
        v.x = *reinterpret_cast<const float *>(stg + row_off(R, x));
        v.y = *reinterpret_cast<const float *>(stg + row_off(R + 1, x));
        v.z = *reinterpret_cast<const float *>(stg + row_off(R + 2, x));
        v.w = *reinterpret_cast<const float *>(stg + row_off(R + 3, x));
        *reinterpret_cast<float4 *>(bk + kmaj_off(kCols, 32 * j1 + x, 4 * pc)) = v;
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
    const int g = (warp - kEpiWarp0) / 4;
    const int qr = warp & 3;
    const int row = 32 * qr + lane;  // TMEM lane = D row
    const bool leader = tid == (kEpiWarp0 + 4 * g) * 32;
    unsigned char *sT = base + P.t[g];
    unsigned char *O = base + P.o[g];
    const uint32_t tl = (uint32_t)(32 * qr) << 16;
    ChunkWalk cw(blockIdx.x + (int64_t)g * NG, (int64_t)kGroups * NG, cpr);
    for (int n = g; n < mine; n += kGroups, cw.next()) {
      const uint32_t tb = tmem + tl + (uint32_t)(g * kCols);
      if (epi_any<kGroupThreads>(!wait_bar(su32(&B.d1full[g]), (unsigned)(n / kGroups) & 1u, abort),
                                 g))
        break;
      tc_fence_after();
      // D1 -> T: row 2b + i of D1, column 32 j1 + x -> T row 32 i + x, K 2b + j1
#pragma unroll
      for (int j1 = 0; j1 < 2; ++j1) {
        float v[32];
        tmem_ld32(tb + 32 * j1, v);
        if (row < Kp2) {
          const int i = row & 1, kr = (row & ~1) + j1;
#pragma unroll
          for (int x = 0; x < 32; ++x)
            *reinterpret_cast<float *>(sT + kmaj_off(kCols, 32 * i + x, kr)) = tf32_rne(v[x]);
        }
      }
      fence_async_smem();
      tc_fence_before();
      mbar_arrive(su32(&B.tready[g]));
      if (epi_any<kGroupThreads>(!wait_bar(su32(&B.d2full[g]), (unsigned)(n / kGroups) & 1u, abort),
                                 g))
        break;
      tc_fence_after();
      if (leader) bulk_wait_read0();  // the group's previous store has read O
      epi_sync<kGroupThreads>(g);
      // D2 -> O: row 2c + i1 of D2, column 32 i + x -> O row (i1 r2 + c) 2 + i
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        float v[32];
        tmem_ld32(tb + 32 * i, v);
        if (row < 2 * s.r2) {
          const int c = row >> 1, i1 = row & 1;
          const int R = (i1 * s.r2 + c) * 2 + i;
#pragma unroll
          for (int cx = 0; cx < 8; ++cx) {
            float4 w;
            w.x = tf32_rne(v[4 * cx]);
            w.y = tf32_rne(v[4 * cx + 1]);
            w.z = tf32_rne(v[4 * cx + 2]);
            w.w = tf32_rne(v[4 * cx + 3]);
            *reinterpret_cast<float4 *>(O + row_off(R, 4 * cx)) = w;
          }
        }
      }
      tc_fence_before();
      mbar_arrive(su32(&B.dfree[g]));
      fence_async_smem();
      epi_sync<kGroupThreads>(g);
      if (leader) {
        const int64_t q0 = cw.w * kQ;
        tma_store5(&tout, su32(O), (int)(q0 & lowmask), 0, (int)(cw.c * s.r2), 0,
                   (int)(q0 >> s.k));
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
                 "r"((uint32_t)(kCols * kGroups))
                 : "memory");
  }
  if (tid == 0 && *abort) atomicCAS(&g_tcf_status, 0, (int)QTT_ERR_TIMEOUT);
}

constexpr size_t kSmemLimit = 227 * 1024;

// 5-D view of a planar FP32 buffer [P][N] for the pair at bit k (k >= 5):
// dims (x: bits 0..k-1, a: bit `b1`, P, b: bit `b3`, hi: bits k+2..), box
// (32, 2, box_p, 2, 1) -- rows of 32 values, 128 bytes, 128-byte swizzle.
bool encode_view_f32(CUtensorMap *m, const void *ptr, int k, int64_t N, int64_t planes, int b1,
                     int b3, int box_p) {
  const cuuint64_t dims[5] = {(cuuint64_t)1 << k, 2, (cuuint64_t)planes, 2,
                              (cuuint64_t)(N >> (k + 2))};
  const cuuint64_t strides[4] = {((cuuint64_t)1 << b1) * 4, (cuuint64_t)N * 4,
                                 ((cuuint64_t)1 << b3) * 4, ((cuuint64_t)1 << (k + 2)) * 4};
  const cuuint32_t box[5] = {32, 2, (cuuint32_t)box_p, 2, 1};
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
  // TF32; every rank <= 32 so that the tiles leave room for two stages
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
  if (!encode_view_f32(&tin, s.in, s.k, s.N, s.nrhs * s.r0, s.k, s.k + 1, s.r0) ||
      !encode_view_f32(&tout, s.out, s.k, s.N, s.nrhs * s.r2, s.k, s.k + 1, s.r2))
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
